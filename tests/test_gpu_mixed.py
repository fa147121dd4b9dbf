"""GPU parity of the split-precision (TF32x3 / BF16x3 tensor-core) actions
against the FP64 oracle.  Tolerances follow the error model: each of the up to
12 one-dimensional contraction stages carries the FP32 accumulator's rounding
plus the split's representation error (TF32x3 ~2^-22, BF16x3 ~2^-16 per
operand), so the normwise relative error stays below ~1e-5 (TF32x3) and
~1e-3 (BF16x3); the measured values are reported by the benchmark."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"tf32x3": 2e-5, "bf16x3": 2e-3}


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", range(1, 9))
def test_mixed_action_parity(gpu, orc, prec, fam, form, p):
    sfx, torch, ctx = gpu
    d = (9, 8, 7) if p <= 3 else (6, 5, 4)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    nrhs = 2 if p == 3 else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    prm = (1.0, -1.0, 0, 0) if form == "helmholtz" else None
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, nrhs=nrhs, precision=prec, params=prm)
    err = rel(yd.cpu().numpy(), orc.action(fam, form, p, d, X, x, params=prm))
    assert err <= TOL[prec], err
    assert ctx.sync_status() == 0


def test_mixed_cell_vectors(gpu, orc):
    sfx, torch, ctx = gpu
    d, p = (5, 4, 3), 4
    X = inputs.box_coords(*d)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), "Q", p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    cells = np.array([3, 0, 59, 17], dtype=np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_vectors(ctx, "laplace", sp, torch.from_numpy(x).cuda(), torch.from_numpy(cells).cuda(),
                                  b, precision="tf32x3")
    ref = orc.cell_vectors("Q", "laplace", p, d, X, x, cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL["tf32x3"]
