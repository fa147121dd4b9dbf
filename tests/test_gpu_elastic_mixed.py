"""Split-precision hyperelastic residuals (vector Q_p, neo-Hookean and SVK;
TF32x3 / BF16x3 contractions on the tensor cores, FP64 geometry, stress and
scatter) against the FP64 oracle.

Tolerance (normwise relative, infinity norm): the gradient H leaves the
tensor cores with the split format's error (TF32x3 ~2^-22, BF16x3 ~2^-16 per
operand) plus FP32 accumulation (~2^-24 per add over n terms per axis);
P(F) in FP64 propagates it linearly, the flux is rounded once to FP32, and
six more split contractions bring it back to the nodes.  Measured errors sit
an order of magnitude below the bounds used here (2e-5 TF32x3, 2e-3 BF16x3),
the same bounds as the scalar split-precision actions."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"tf32x3": 2e-5, "bf16x3": 2e-3}


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", range(1, 9))
def test_elastic_mixed_parity(gpu, orc, prec, form, p):
    sfx, torch, ctx = gpu
    d = (4, 4, 3) if p <= 4 else (3, 3, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), "VQ", p)
    nrhs = 2 if p == 2 else 1
    u = inputs.random_vector(sp.ndof, nrhs, seed=1) * (0.05 / (max(d) * p))
    if form == "svk" and p <= 3:
        u = inputs.random_vector(sp.ndof, nrhs, seed=1, lo=-0.05, hi=0.05)  # the unscaled distribution
    ud = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    yd = torch.empty_like(ud)
    sfx.sfx_assemble_action(ctx, form, sp, ud, yd, nrhs=nrhs, precision=prec)
    assert rel(yd.cpu().numpy(), orc.action("VQ", form, p, d, X, u)) <= TOL[prec]
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_elastic_mixed_params_and_accumulate(gpu, orc, prec):
    """non-default mu, lambda; accumulate adds to y."""
    sfx, torch, ctx = gpu
    d, p = (3, 4, 2), 3
    X = inputs.box_coords(*d, seed=3)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), "VQ", p)
    u = inputs.displacement(sp.ndof, p, 4, seed=2)
    prm = (0, 0, 2.5, 0.7)
    ud = torch.from_numpy(u).cuda()
    y0 = inputs.random_vector(sp.ndof, 1, seed=9) * 1e-3
    yd = torch.from_numpy(y0.copy()).cuda()
    sfx.sfx_assemble_action(ctx, "neohooke", sp, ud, yd, params=prm, accumulate=True, precision=prec)
    ref = orc.action("VQ", "neohooke", p, d, X, u, params=prm)
    assert rel(yd.cpu().numpy() - y0, ref) <= 2 * TOL[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("form", ["neohooke", "svk"])
def test_elastic_mixed_zero_displacement_is_exactly_zero(gpu, prec, form):
    """u = 0 gives H = 0 exactly on the tensor cores, F = I, P = 0: no
    rounding anywhere, so the residual is exactly zero."""
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 5, 4, 3), "VQ", 4)
    yd = torch.full((sp.ndof,), 7.0, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, form, sp, torch.zeros_like(yd), yd, precision=prec)
    assert yd.abs().max().item() == 0.0
    assert ctx.sync_status() == 0


def test_elastic_mixed_detf_flag(gpu):
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 2, 2, 2), "VQ", 2)
    u = inputs.random_vector(sp.ndof, 1, seed=3, lo=-2.0, hi=2.0)
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, "neohooke", sp, torch.from_numpy(u).cuda(), yd, precision="tf32x3")
    assert ctx.sync_status() == sfx.DEV_DETF
    assert torch.isfinite(yd).all()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_elastic_mixed_cell_vectors(gpu, orc, prec):
    sfx, torch, ctx = gpu
    d, p = (4, 3, 3), 5
    X = inputs.box_coords(*d)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), "VQ", p)
    u = inputs.displacement(sp.ndof, p, 4)
    cells = np.array([35, 0, 12, 7, 19], dtype=np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_vectors(ctx, "neohooke", sp, torch.from_numpy(u).cuda(), torch.from_numpy(cells).cuda(),
                                  b, precision=prec)
    ref = orc.cell_vectors("VQ", "neohooke", p, d, X, u, cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL[prec]


@pytest.mark.parametrize("p", [3, 8])
def test_elastic_mixed_full_size_sampled(gpu, orc, p):
    """The precision configuration's 64^3 mesh: sampled cells' b^K against the
    oracle in the per-cell mode, and the full TF32x3 residual against the FP64
    GPU residual (itself at 1e-12 of the oracle in the FP64 tests)."""
    sfx, torch, ctx = gpu
    d = (64, 64, 64)
    mesh = sfx.Mesh.box(ctx, *d)
    sp = sfx.Space(mesh, "VQ", p)
    u = inputs.displacement(sp.ndof, p, d[0])
    ud = torch.from_numpy(u).cuda()
    del u
    rng = np.random.default_rng(11)
    cells = rng.choice(sp.ncell, 8, replace=False).astype(np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_vectors(ctx, "neohooke", sp, ud, torch.from_numpy(cells).cuda(), b, precision="tf32x3")
    ref = orc.cell_vectors("VQ", "neohooke", p, d, inputs.box_coords(*d), ud.cpu().numpy(), cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL["tf32x3"]
    y64 = torch.empty_like(ud)
    ymx = torch.empty_like(ud)
    sfx.sfx_assemble_action(ctx, "neohooke", sp, ud, y64)
    sfx.sfx_assemble_action(ctx, "neohooke", sp, ud, ymx, precision="tf32x3")
    assert ctx.sync_status() == 0
    err = ((ymx - y64).abs().max() / y64.abs().max()).item()
    assert err <= TOL["tf32x3"]
