"""GPU parity: the vector mass / Laplace / Helmholtz forms on vector Q_p
(Sec. 3.3) through the C ABI against the oracle, which evaluates them with full
vectors (no component delta assumed).

Bars: FP64 1e-12, TF32x3 2e-5 normwise; element matrices per cell 1e-12.  At
the benchmark's 64^3, Q_8 size the vector action must equal the three scalar
actions bit for bit (same kernels on the component slices)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
HELM = (0.7, -1.3, 0.0, 0.0)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dims_for(p):
    return (4, 3, 3) if p <= 4 else (2, 2, 2)


@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", range(1, 9))
def test_vector_action_parity(gpu, orc, form, p):
    sfx, torch, ctx = gpu
    d = dims_for(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "VQ", p)
    nrhs = 2 if p in (3, 6) else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    prm = HELM if form == "helmholtz" else None
    ref = orc.action("VQ", form, p, d, X, x, params=prm)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    for prec, tol in (("fp64", 1e-12), ("tf32x3", 2e-5)):
        yd = torch.empty_like(xd)
        sfx.sfx_assemble_action(ctx, form, sp, xd, yd, nrhs=nrhs, precision=prec, params=prm)
        assert rel(yd.cpu().numpy(), ref) <= tol, prec
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_vector_cell_matrices_parity(gpu, orc, form, p):
    sfx, torch, ctx = gpu
    d = (3, 2, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=2)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "VQ", p)
    c0, c1 = (0, sp.ncell) if p <= 3 else (4, 7)
    prm = HELM if form == "helmholtz" else None
    A = torch.empty((c1 - c0) * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, form, sp, c0, c1, A, params=prm)
    Ag = A.cpu().numpy().reshape(c1 - c0, sp.nloc, sp.nloc)
    Aref = orc.cell_matrices("VQ", form, p, d, X, c0, c1, params=prm)
    n3 = sp.nloc // 3
    for c in range(c1 - c0):
        assert np.abs(Ag[c] - Aref[c]).max() <= 1e-12 * np.abs(Aref[c]).max()
        for a in range(3):
            for b in range(3):
                if a != b:
                    assert not Ag[c, a * n3:(a + 1) * n3, b * n3:(b + 1) * n3].any()


def test_vector_matrices_chunked_scratch(gpu):
    """Q_8 vector Laplace on more cells than one scratch chunk holds (63 scalar
    blocks of 4.25 MB per 256 MB): the chunk boundary must not show."""
    sfx, torch, ctx = gpu
    d = (5, 4, 4)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "VQ", 8)
    sq = sfx.Space(mesh, "Q", 8)
    n = sp.ncell  # 80 > 63
    A = torch.empty(n * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    S = torch.empty(n * sq.nloc * sq.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, "laplace", sp, 0, n, A)
    sfx.sfx_assemble_cell_matrices(ctx, "laplace", sq, 0, n, S)
    A = A.view(n, 3, sq.nloc, 3, sq.nloc)
    S = S.view(n, sq.nloc, sq.nloc)
    for a in range(3):
        assert torch.equal(A[:, a, :, a, :], S)
    A[:, 0, :, 0, :] = 0
    A[:, 1, :, 1, :] = 0
    A[:, 2, :, 2, :] = 0
    assert not A.any()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_vector_action_64cube_equals_component_actions(gpu, prec):
    sfx, torch, ctx = gpu
    d = (64, 64, 64)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "VQ", 8)
    sq = sfx.Space(mesh, "Q", 8)
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
    y = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "helmholtz", sp, x, y, precision=prec)
    ys = torch.empty(sq.ndof, dtype=torch.float64, device="cuda")
    for a in range(3):
        sl = slice(a * sq.ndof, (a + 1) * sq.ndof)
        sfx.sfx_assemble_action(ctx, "helmholtz", sq, x[sl].contiguous(), ys, precision=prec)
        assert torch.equal(y[sl], ys)
    assert ctx.sync_status() == 0


def test_vector_collocated_action(gpu, orc):
    sfx, torch, ctx = gpu
    d, p = (3, 3, 2), 4
    X = inputs.box_coords(*d, perturb=0.1, seed=3)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "VQ", p)
    x = inputs.random_vector(sp.ndof, 1, seed=4)
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, "laplace", sp, torch.from_numpy(x).cuda(), yd, algo="collocated")
    ref = orc.action("VQ", "laplace", p, d, X, x, qrule="GLL")
    assert rel(yd.cpu().numpy(), ref) <= 1e-12


def test_vector_forms_cell_vectors_unsupported(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    sp = sfx.Space(mesh, "VQ", 1)
    x = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
    cells = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    b = torch.empty(2 * sp.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_cell_vectors(ctx, "mass", sp, x, cells, b)
    assert e.value.code == -2
