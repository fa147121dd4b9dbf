"""Split-precision linearised hyperelastic operator K(u) du (vector Q_p,
neo-Hookean and SVK; TF32x3 / BF16x3 contractions of both the state u and the
direction du on the tensor cores; FP64 geometry, F, dF, dP, weight scaling
and scatter) against the FP64 oracle -- the operator whose action the
paper's hyperelastic experiments time (Sec. 4.1).

Tolerance (normwise relative, infinity norm): the same error model as the
split-precision residual -- the gradients leave the tensor cores with the
split's error, dP(F; dF) is linear in dF and smooth in F, the flux is
rounded once to FP32 and six more split contractions bring it back -- so
the same bounds: 2e-5 (TF32x3), 2e-3 (BF16x3).  Also: per-cell vectors, and
the element (tangent) matrices stay FP64 only."""
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
def test_linearised_mixed_parity(gpu, orc, prec, form, p):
    sfx, torch, ctx = gpu
    d = (4, 3, 3) if p <= 4 else ((3, 2, 2) if p <= 6 else (2, 1, 2))
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), "VQ", p)
    u = inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)
    nrhs = 2 if p in (2, 5) else 1
    du = inputs.random_vector(sp.ndof, nrhs, seed=2)
    ud = torch.from_numpy(u).cuda()
    dd = torch.from_numpy(np.ascontiguousarray(du)).cuda()
    yd = torch.empty_like(dd)
    sfx.sfx_assemble_linearised_action(ctx, form, sp, ud, dd, yd, nrhs=nrhs, precision=prec)
    assert ctx.sync_status() == 0
    yref = orc.linearised_action(form, p, d, X, u, du)
    assert rel(yd.cpu().numpy(), yref) <= TOL[prec]


def test_linearised_mixed_cell_vectors_and_limits(gpu, orc):
    sfx, torch, ctx = gpu
    d, p = (4, 3, 2), 3
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), "VQ", p)
    u = inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)
    du = inputs.random_vector(sp.ndof, 1, seed=2)
    cells = np.array([5, 0, 23, 11], dtype=np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_vectors(ctx, "svk", sp, torch.from_numpy(u).cuda(), torch.from_numpy(du).cuda(),
                                             torch.from_numpy(cells).cuda(), b, precision="tf32x3")
    ref = orc.linearised_cell_vectors("svk", p, d, X, u, du, cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL["tf32x3"]
    A = torch.empty(sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_linearised_cell_matrices(ctx, "svk", sp, torch.from_numpy(u).cuda(), 0, 1, A,
                                                  precision="tf32x3")
    assert e.value.code == -2
    assert ctx.sync_status() == 0
