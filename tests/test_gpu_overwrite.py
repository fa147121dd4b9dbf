"""Overwriting actions (accumulate = 0) write every dof of y without a memset:
each dof's first cell-node pair in colour order stores its contribution and
the later pairs add theirs.  The result must equal an accumulating action onto
a zero vector value for value (the same sums in the same order), whatever y
held before -- here NaN, so a dof that no pair writes shows up.  The colour
launches of one action also overlap (programmatic dependent launch), so these
cases check that no scatter of a colour runs before the previous colour's."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu


def both(sfx, torch, run, n):
    y_over = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    y_acc = torch.zeros(n, dtype=torch.float64, device="cuda")
    run(y_over, False)
    run(y_acc, True)
    torch.cuda.synchronize()
    return y_over, y_acc


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", [1, 3, 4, 7, 8])
def test_overwrite_equals_accumulate_onto_zero(gpu, fam, prec, form, p):
    sfx, torch, ctx = gpu
    d = (7, 6, 5) if p <= 3 else (5, 4, 3)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, fam, p)
    nrhs = 3 if p == 4 else 1
    xd = torch.from_numpy(inputs.random_vector(sp.ndof, nrhs, seed=1)).cuda()

    def run(y, acc):
        sfx.sfx_assemble_action(ctx, form, sp, xd, y, nrhs=nrhs, accumulate=acc, precision=prec)

    y_over, y_acc = both(sfx, torch, run, sp.ndof * nrhs)
    assert torch.equal(y_over, y_acc)
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("p", [2, 5])
def test_overwrite_collocated_stored_weighted(gpu, p):
    sfx, torch, ctx = gpu
    d = (5, 4, 6)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "Q", p)
    xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
    kd = torch.from_numpy(1.0 + 0.5 * inputs.random_vector(sp.ndof, 1, seed=4)).cuda()
    q = sfx.QData(ctx, sp)
    cases = [
        lambda y, acc: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, y, accumulate=acc, algo="collocated"),
        lambda y, acc: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, y, accumulate=acc, precision="tf32x3",
                                               algo="collocated"),
        lambda y, acc: sfx.sfx_assemble_action_stored(ctx, "helmholtz", sp, q, xd, y, accumulate=acc),
        lambda y, acc: sfx.sfx_assemble_action_stored(ctx, "helmholtz", sp, q, xd, y, accumulate=acc,
                                                      precision="tf32x3"),
        lambda y, acc: sfx.sfx_assemble_weighted_action(ctx, sp, kd, xd, y, accumulate=acc),
    ]
    for run in cases:
        y_over, y_acc = both(sfx, torch, run, sp.ndof)
        assert torch.equal(y_over, y_acc)
    assert ctx.sync_status() == 0


def test_overwrite_general_mesh(gpu):
    """Greedy colouring on a shuffled, rotated box mesh: the first-touch pairs
    follow that colour order."""
    sfx, torch, ctx = gpu
    X, cv = inputs.shuffled_box(4, 5, 3, perturb=0.1, seed=0, shuffle_seed=3)[:2]
    mesh = sfx.Mesh.general(ctx, X, cv)
    for fam, p, prec in (("Q", 3, "fp64"), ("Q", 4, "tf32x3"), ("DQ", 2, "fp64")):
        sp = sfx.Space(mesh, fam, p)
        xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()

        def run(y, acc):
            sfx.sfx_assemble_action(ctx, "laplace", sp, xd, y, accumulate=acc, precision=prec)

        y_over, y_acc = both(sfx, torch, run, sp.ndof)
        assert torch.equal(y_over, y_acc)
    assert ctx.sync_status() == 0


def test_overwrite_inverted_cell(gpu):
    """A skipped (inverted) cell still stores 0 into the dofs it writes first,
    so they hold the other cells' sums, as after a memset."""
    sfx, torch, ctx = gpu
    d = (2, 2, 2)
    X = inputs.box_coords(*d, perturb=0.0)
    X[(1 * 3 + 1) * 3 + 1] = [1.2, 1.2, 1.2]
    mesh = sfx.Mesh.structured(ctx, *d, X)
    for p, prec in ((1, "fp64"), (4, "tf32x3"), (8, "tf32x3")):
        sp = sfx.Space(mesh, "Q", p)
        xd = torch.ones(sp.ndof, dtype=torch.float64, device="cuda")

        def run(y, acc):
            sfx.sfx_assemble_action(ctx, "helmholtz", sp, xd, y, accumulate=acc, precision=prec)

        y_over, y_acc = both(sfx, torch, run, sp.ndof)
        assert torch.equal(y_over, y_acc)
        assert np.isfinite(y_over.cpu().numpy()).all()
        assert ctx.sync_status() & sfx.DEV_INVERTED


@pytest.mark.parametrize("fam,p,prec", [("Q", 8, "tf32x3"), ("Q", 3, "fp64"), ("DQ", 5, "tf32x3")])
def test_action_in_cuda_graph(gpu, fam, p, prec):
    """An action captured in a CUDA graph (its colour launches, programmatic
    dependents of one another, become graph nodes) replays to the same result
    as the eager call, also after the input changes in place."""
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 6, 5, 4, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, fam, p)
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
    y_eager = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "helmholtz", sp, x, y_eager, precision=prec)
    y = torch.full_like(x, float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up on the capture stream
        sfx.sfx_assemble_action(ctx, "helmholtz", sp, x, y, precision=prec, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sfx.sfx_assemble_action(ctx, "helmholtz", sp, x, y, precision=prec, stream=s)
    y.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, y_eager)
    x2 = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=2)).cuda()
    x.copy_(x2)
    g.replay()
    sfx.sfx_assemble_action(ctx, "helmholtz", sp, x2, y_eager, precision=prec)
    torch.cuda.synchronize()
    assert torch.equal(y, y_eager)
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 3), (2, 1, 1), (1, 3, 2)])
@pytest.mark.parametrize("fam,prec,p", [("Q", "fp64", 2), ("Q", "fp64", 8), ("Q", "tf32x3", 8), ("DQ", "fp64", 3),
                                        ("DQ", "tf32x3", 8)])
def test_overwrite_thin_meshes(gpu, dims, fam, prec, p):
    """Meshes whose parity colours are partly empty (the first launched colour
    is not colour 0) still write every dof."""
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, fam, p)
    xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()

    def run(y, acc):
        sfx.sfx_assemble_action(ctx, "helmholtz", sp, xd, y, accumulate=acc, precision=prec)

    y_over, y_acc = both(sfx, torch, run, sp.ndof)
    assert torch.equal(y_over, y_acc)
    assert ctx.sync_status() == 0
