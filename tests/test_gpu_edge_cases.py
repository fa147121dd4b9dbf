"""Degenerate and limit cases of the operator action through the C ABI, against
the oracle: one-cell meshes for every family and form (for the shared-dof
families seven of the eight colour passes are empty), thin one-cell-wide meshes, the largest number of
right-hand sides (64), a ragged last CTA for every cells-per-CTA value the
kernels use, and zero input (exactly zero output, no flags)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "tf32x3": 2e-5, "bf16x3": 2e-3}
CASES = [("Q", "mass"), ("Q", "laplace"), ("Q", "helmholtz"), ("DQ", "laplace"), ("NCF", "ncf_mass_divdiv"),
         ("NCE", "nce_curlcurl"), ("VQ", "neohooke"), ("VQ", "svk"), ("VQ", "laplace")]
SPLIT = {("Q", "mass"), ("Q", "laplace"), ("Q", "helmholtz"), ("DQ", "laplace"), ("VQ", "neohooke"),
         ("VQ", "svk"), ("VQ", "laplace")}


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def field(fam, ndof, p, n, seed):
    if fam == "VQ":
        return inputs.displacement(ndof, p, n, seed=seed, amplitude=0.1)
    return inputs.random_vector(ndof, 1, seed=seed)


def check_action(sfx, torch, ctx, orc, d, fam, form, p, precisions):
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, fam, p)
    x = field(fam, sp.ndof, p, max(d), 1)
    ref = orc.action(fam, form, p, d, X, x)
    xd = torch.from_numpy(x).cuda()
    for prec in precisions:
        yd = torch.empty_like(xd)
        sfx.sfx_assemble_action(ctx, form, sp, xd, yd, precision=prec)
        assert rel(yd.cpu().numpy(), ref) <= TOL[prec], (fam, form, p, prec)
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("fam,form", CASES)
@pytest.mark.parametrize("p", [1, 8])
def test_one_cell_mesh(gpu, orc, fam, form, p):
    sfx, torch, ctx = gpu
    precs = ["fp64"] + (["tf32x3", "bf16x3"] if (fam, form) in SPLIT else [])
    check_action(sfx, torch, ctx, orc, (1, 1, 1), fam, form, p, precs)


@pytest.mark.parametrize("d", [(1, 1, 7), (1, 5, 1), (6, 1, 1)])
@pytest.mark.parametrize("fam,form", [("Q", "laplace"), ("NCE", "nce_curlcurl"), ("VQ", "neohooke")])
def test_thin_meshes(gpu, orc, d, fam, form):
    sfx, torch, ctx = gpu
    precs = ["fp64"] + (["tf32x3"] if (fam, form) in SPLIT else [])
    check_action(sfx, torch, ctx, orc, d, fam, form, 3, precs)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
@pytest.mark.parametrize("fam", ["Q", "DQ"])
def test_sixty_four_rhs(gpu, orc, prec, fam):
    sfx, torch, ctx = gpu
    d, p = (3, 2, 2), 4
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, fam, p)
    x = inputs.random_vector(sp.ndof, 64, seed=5)
    ref = orc.action(fam, "helmholtz", p, d, X, x)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, "helmholtz", sp, xd, yd, nrhs=64, precision=prec)
    assert rel(yd.cpu().numpy(), ref) <= TOL[prec]
    with pytest.raises(sfx.SfxError):  # one more than the limit
        x65 = torch.zeros(sp.ndof * 65, dtype=torch.float64, device="cuda")
        sfx.sfx_assemble_action(ctx, "helmholtz", sp, x65, torch.empty_like(x65), nrhs=65)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
@pytest.mark.parametrize("p", range(1, 9))
def test_ragged_last_cta(gpu, orc, prec, p):
    """7 x 3 x 1 = 21 cells: four colour passes hold 8, 6, 4 and 3 cells and four
    are empty, so at every degree a pass ends in a partly filled CTA (or is
    smaller than one)."""
    sfx, torch, ctx = gpu
    check_action(sfx, torch, ctx, orc, (7, 3, 1), "Q", "laplace", p, [prec])


@pytest.mark.parametrize("fam,form", CASES)
def test_zero_input_gives_exact_zero(gpu, fam, form):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 3, 2, 2, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, fam, 3)
    x = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
    precs = ["fp64"] + (["tf32x3", "bf16x3"] if (fam, form) in SPLIT else [])
    for prec in precs:
        y = torch.full_like(x, 7.0)
        sfx.sfx_assemble_action(ctx, form, sp, x, y, precision=prec)
        assert not y.any(), (fam, form, prec)
    assert ctx.sync_status() == 0
