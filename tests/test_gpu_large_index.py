"""Maximum sizes: vectors with more than 2^31 entries.  DQ_8 on the 64^3 mesh
with 12 right-hand sides has 191,102,976 x 12 = 2,293,235,712 entries (18.3 GB
per vector), so every dof and map index of the last cells, times nrhs, passes
2^31 and must be formed in 64-bit arithmetic.  DQ dofs belong to one cell, so
y at a cell's dofs is that cell's vector b^K, compared with the oracle.

x[i] = ((i * 2654435761) mod 2^20) / 2^20 - 0.5 for the flat index i (RHS
fastest): exact integer arithmetic, the same on the device and the host."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
NRHS = 12
CELLS = [1000, 250000, 255555, 262143]  # all but the first lie past 2^31 / (729 * 12)


def field(torch, n, device):
    x = torch.empty(n, dtype=torch.float64, device=device)
    step = 1 << 28
    for s in range(0, n, step):
        i = torch.arange(s, min(n, s + step), dtype=torch.int64, device=device)
        x[s:s + len(i)] = ((i * 2654435761) & ((1 << 20) - 1)).double() / (1 << 20) - 0.5
    return x


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("tf32x3", 2e-5)])
def test_dq8_64cube_12rhs_past_2_31(gpu, orc, prec, tol):
    sfx, torch, ctx = gpu
    d, p = (64, 64, 64), 8
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "DQ", p)
    n3 = (p + 1) ** 3
    assert sp.ndof * NRHS > 2 ** 31
    x = field(torch, sp.ndof * NRHS, "cuda")
    y = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "laplace", sp, x, y, nrhs=NRHS, precision=prec)
    assert ctx.sync_status() == 0
    r = NRHS - 1
    dofs = np.concatenate([np.arange(c * n3, (c + 1) * n3) for c in CELLS])
    assert (dofs[-1] * NRHS + r) > 2 ** 31
    idx = torch.from_numpy(dofs * NRHS + r).cuda()
    got = y[idx].cpu().numpy().reshape(len(CELLS), n3)
    # the oracle's input: column r at the sampled cells' dofs (DQ: nothing else enters their b^K)
    xc = np.zeros(sp.ndof)
    i = dofs.astype(np.int64) * NRHS + r
    xc[dofs] = ((i * 2654435761) & ((1 << 20) - 1)).astype(np.float64) / (1 << 20) - 0.5
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    ref = orc.cell_vectors("DQ", "laplace", p, d, X, xc, CELLS)
    for k in range(len(CELLS)):
        assert np.abs(got[k] - ref[k]).max() <= tol * np.abs(ref[k]).max(), (CELLS[k], prec)
    del x, y
    torch.cuda.empty_cache()
