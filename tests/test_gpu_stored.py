"""Actions with stored geometric factors (sfx_qdata_*) against the FP64 oracle,
and the FP64 stored action against the on-the-fly one (same formulas; the
compiler may fuse multiply-adds differently in the two kernels, so they agree
to roundoff rather than bit for bit)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "tf32x3": 2e-5, "bf16x3": 2e-3}


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_stored_action_parity(gpu, orc, prec, fam, form, p):
    sfx, torch, ctx = gpu
    d = (9, 8, 7) if p <= 3 else (6, 5, 4)
    X = inputs.box_coords(*d)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    q = sfx.QData(ctx, sp, "both")
    nrhs = 2 if p == 2 else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    prm = (0.8, -1.2, 0, 0) if form == "helmholtz" else None
    sfx.sfx_assemble_action_stored(ctx, form, sp, q, xd, yd, nrhs=nrhs, precision=prec, params=prm)
    assert rel(yd.cpu().numpy(), orc.action(fam, form, p, d, X, x, params=prm)) <= TOL[prec]
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("form", ["mass", "laplace"])
def test_stored_fp64_matches_on_the_fly(gpu, fam, form):
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 8, 7, 6), fam, 4)
    q = sfx.QData(ctx, sp, "fp64")
    xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=3)).cuda()
    y1, y2 = torch.empty_like(xd), torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, form, sp, xd, y1)
    sfx.sfx_assemble_action_stored(ctx, form, sp, q, xd, y2)
    assert ((y1 - y2).abs().max() / y1.abs().max()).item() <= 1e-14


def test_stored_argument_errors(gpu):
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 2, 2, 2), "Q", 2)
    q32 = sfx.QData(ctx, sp, "fp32")
    xd = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError):  # FP64 action needs FP64 factors
        sfx.sfx_assemble_action_stored(ctx, "laplace", sp, q32, xd, torch.empty_like(xd))
    sp2 = sfx.Space(sfx.Mesh.box(ctx, 2, 2, 2), "Q", 2)
    with pytest.raises(sfx.SfxError):  # factors of another space
        sfx.sfx_assemble_action_stored(ctx, "laplace", sp2, q32, xd, torch.empty_like(xd), precision="tf32x3")
    with pytest.raises(sfx.SfxError):
        sfx.QData(ctx, sfx.Space(sfx.Mesh.box(ctx, 2, 2, 2), "NCE", 2))
