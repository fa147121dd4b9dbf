"""The warp-specialised split-precision action (producer warps build the FP64
geometry factors of the next batch of cells while consumer warps contract the
current one; hand-off through two mbarriers with bounded waits).

* Against the one-role kernel on the same inputs, with one and two
  right-hand sides: the two kernels round the flux differently (t R (R^T g)
  there, t (R R^T) g here, both with the scaling by t in FP64), so they agree
  within the split's bar (TF32x3 2e-5, BF16x3 2e-3).  One cell per batch on a
  16^3 mesh makes every CTA run several batches, so the barriers go through
  many phases.
* Against the oracle on a mesh with ragged batches (the parity tests of the
  split-precision actions cover the rest).
* The timeout path: with the poll limit at 0 every wait gives up at once; the
  call still returns and the status word carries SFX_DEV_TIMEOUT."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
HELM = (1.0, -1.0, 0.0, 0.0)


def run(sfx, torch, ctx, sp, form, x, nrhs, prec, ws, cb=0):
    p = sp.p
    old = sfx.sfx_tune_get_warp_specialised(p)
    sfx.sfx_tune_set_warp_specialised(p, ws)
    sfx.sfx_tune_set_cells_per_cta("mixed_ws", p, cb)
    try:
        y = torch.empty_like(x)
        sfx.sfx_assemble_action(ctx, form, sp, x, y, nrhs=nrhs, precision=prec,
                                params=HELM if form == "helmholtz" else None)
        torch.cuda.synchronize()
    finally:
        sfx.sfx_tune_set_warp_specialised(p, old)
        sfx.sfx_tune_set_cells_per_cta("mixed_ws", p, 0)
    assert ctx.sync_status() == 0
    return y


@pytest.mark.parametrize("fam,p", [("Q", 3), ("Q", 8), ("DQ", 5)])
@pytest.mark.parametrize("form", ["laplace", "helmholtz"])
@pytest.mark.parametrize("cb", [1, 0])
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_ws_matches_one_role_kernel(gpu, fam, p, form, cb, prec):
    sfx, torch, ctx = gpu
    d = (16, 16, 16)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, fam, p)
    for nrhs in (2, 1):
        x = torch.from_numpy(np.ascontiguousarray(inputs.random_vector(sp.ndof, nrhs, seed=3))).cuda()
        yw = run(sfx, torch, ctx, sp, form, x, nrhs, prec, True, cb)
        y1 = run(sfx, torch, ctx, sp, form, x, nrhs, prec, False)
        err = ((yw - y1).abs().max() / y1.abs().max()).item()
        assert err <= (2e-5 if prec == "tf32x3" else 2e-3), err


@pytest.mark.parametrize("fam,p", [("Q", 4), ("DQ", 7)])
def test_ws_oracle_ragged(gpu, orc, fam, p):
    sfx, torch, ctx = gpu
    d = (7, 5, 3)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    xd = torch.from_numpy(x).cuda()
    for cb in (1, 3, 0):
        y = run(sfx, torch, ctx, sp, "helmholtz", xd, 1, "tf32x3", True, cb).cpu().numpy()
        ref = orc.action(fam, "helmholtz", p, d, X, x, params=HELM)
        assert np.abs(y - ref).max() <= 2e-5 * np.abs(ref).max()


def test_ws_timeout_path(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 8, 8, 8, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "Q", 4)
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
    y = torch.empty_like(x)
    assert sfx.sfx_tune_get_warp_specialised(4)
    sfx.sfx_set_wait_limit(0)
    try:
        sfx.sfx_assemble_action(ctx, "laplace", sp, x, y, precision="tf32x3")
        torch.cuda.synchronize()
        st = ctx.sync_status()
    finally:
        sfx.sfx_set_wait_limit(1 << 21)
    assert st & sfx.DEV_TIMEOUT
    # the context stays usable and the next call is right again
    y2 = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "laplace", sp, x, y2, precision="tf32x3")
    yr = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "laplace", sp, x, yr)
    assert ctx.sync_status() == 0
    assert ((y2 - yr).abs().max() / yr.abs().max()).item() <= 2e-5
