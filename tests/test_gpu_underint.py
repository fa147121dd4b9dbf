"""GPU parity: Q_p with the collocated Gauss-Lobatto rule ("underintegration",
Sec. 4.1; SFX_ALGO_COLLOCATED) through the C ABI against the oracle run with
the same rule.

Bars: FP64 actions and delta-cancelled element matrices <= 1e-12 normwise;
TF32x3 actions <= 2e-5 (the stated split-precision tolerance).  At the
benchmark's size (64^3) the tests check properties that hold at any size."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOL_TF32 = 2e-5


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dims_for(p):
    return (9, 8, 7) if p <= 3 else (6, 5, 4)


@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_collocated_action_parity(gpu, orc, form, p, prec):
    sfx, torch, ctx = gpu
    d = dims_for(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "Q", p)
    nrhs = 2 if p in (3, 6) else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    prm = (0.7, -1.3, 0, 0) if form == "helmholtz" else None
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, nrhs=nrhs, params=prm, precision=prec, algo="collocated")
    yref = orc.action("Q", form, p, d, X, x, params=prm, qrule="GLL")
    assert rel(yd.cpu().numpy(), yref) <= (TOL if prec == "fp64" else TOL_TF32)
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", range(1, 9))
def test_collocated_cell_matrices_parity(gpu, orc, form, p):
    sfx, torch, ctx = gpu
    d = (3, 2, 2) if p <= 4 else (2, 1, 1)
    X = inputs.box_coords(*d, perturb=0.1, seed=2)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "Q", p)
    nc = sp.ncell
    A = torch.empty(nc * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    prm = (0.7, -1.3, 0, 0) if form == "helmholtz" else None
    sfx.sfx_assemble_cell_matrices(ctx, form, sp, 0, nc, A, algo="collocated", params=prm)
    Ag = A.cpu().numpy().reshape(nc, sp.nloc, sp.nloc)
    Aref = orc.cell_matrices("Q", form, p, d, X, params=prm, qrule="GLL")
    for c in range(nc):
        assert np.abs(Ag[c] - Aref[c]).max() <= TOL * np.abs(Aref[c]).max()
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("p", [2, 5, 8])
def test_collocated_matrices_reproduce_action(gpu, p):
    """sum_K P_K^T A^K P_K x with the GPU's delta-cancelled matrices equals the
    GPU's collocated action (two different kernels, same rule)."""
    sfx, torch, ctx = gpu
    d = (5, 4, 3)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "Q", p)
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=3)).cuda()
    y = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "helmholtz", sp, x, y, algo="collocated")
    A = torch.empty(sp.ncell * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, "helmholtz", sp, 0, sp.ncell, A, algo="collocated")
    cmap = torch.from_numpy(sp.cell_map().astype(np.int64)).cuda()
    b = torch.bmm(A.view(sp.ncell, sp.nloc, sp.nloc), x[cmap].unsqueeze(-1)).squeeze(-1)
    ref = torch.zeros_like(x).index_add_(0, cmap.reshape(-1), b.reshape(-1))
    assert ((y - ref).abs().max() / ref.abs().max()).item() <= TOL


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_collocated_full_size_properties(gpu, prec):
    """64^3, p = 8, the launch configuration the benchmark times: the
    collocated rule integrates the volume exactly for p >= 2 (1^T M 1 = 1) and
    the Laplace action annihilates constants."""
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 64, 64, 64, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "Q", 8)
    one = torch.ones(sp.ndof, dtype=torch.float64, device="cuda")
    y = torch.empty_like(one)
    sfx.sfx_assemble_action(ctx, "mass", sp, one, y, precision=prec, algo="collocated")
    assert abs(y.sum().item() - 1.0) <= (1e-11 if prec == "fp64" else 1e-5)
    sfx.sfx_assemble_action(ctx, "laplace", sp, one, y, precision=prec, algo="collocated")
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
    yx = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "laplace", sp, x, yx, precision=prec, algo="collocated")
    scale = yx.abs().max().item()
    assert y.abs().max().item() <= (1e-12 if prec == "fp64" else 1e-5) * scale
    assert ctx.sync_status() == 0


def test_collocated_unsupported(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    for fam, form, prec in [("DQ", "laplace", "fp64"), ("Q", "laplace", "bf16x3"), ("NCF", "ncf_mass_divdiv", "fp64")]:
        sp = sfx.Space(mesh, fam, 2)
        xx = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
        yy = torch.empty_like(xx)
        with pytest.raises(sfx.SfxError) as e:
            sfx.sfx_assemble_action(ctx, form, sp, xx, yy, precision=prec, algo="collocated")
        assert e.value.code == -2
    sp = sfx.Space(mesh, "DQ", 2)
    A = torch.empty(sp.ncell * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_cell_matrices(ctx, "laplace", sp, 0, sp.ncell, A, algo="collocated")
    assert e.value.code == -2
    del x
