"""GPU parity: the assembled global matrix (sfx_csr_assemble) and its product
with a vector (sfx_csr_spmv) against the oracle.

The reference matrix is sum_K P_K^T A^K P_K of the oracle's element matrices,
summed by scipy.sparse (a library sum of the oracle's values); the reference
product is the oracle's action.  Bar: 1e-12 normwise (FP64)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
scipy_sparse = pytest.importorskip("scipy.sparse")
TOL = 1e-12


def oracle_csr(orc, fam, form, p, dims, X, params=None):
    ndof, nloc = orc.space_size(fam, p, dims)
    A = orc.cell_matrices(fam, form, p, dims, X, params=params)
    cmap = orc.cell_map(fam, p, dims).astype(np.int64)
    rows = np.repeat(cmap, nloc, axis=1).reshape(-1)
    cols = np.tile(cmap, (1, nloc)).reshape(-1)
    M = scipy_sparse.coo_matrix((A.reshape(-1), (rows, cols)), shape=(ndof, ndof)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


@pytest.mark.parametrize("fam,p", [("Q", 1), ("Q", 2), ("Q", 3), ("Q", 4), ("DQ", 2), ("DQ", 5)])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
def test_csr_values_and_spmv(gpu, orc, fam, p, form):
    sfx, torch, ctx = gpu
    d = (4, 3, 3) if p <= 3 else (3, 2, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, fam, p)
    csr = sfx.Csr(sp)
    vals = torch.empty(csr.nnz, dtype=torch.float64, device="cuda")
    prm = (0.7, -1.3, 0, 0) if form == "helmholtz" else None
    sfx.sfx_csr_assemble(ctx, form, csr, vals, params=prm)
    M = oracle_csr(orc, fam, form, p, d, X, params=prm)
    rp, col = csr.pattern()
    np.testing.assert_array_equal(rp, M.indptr)
    np.testing.assert_array_equal(col, M.indices)
    v = vals.cpu().numpy()
    assert np.abs(v - M.data).max() <= TOL * np.abs(M.data).max()
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    sfx.sfx_csr_spmv(ctx, csr, vals, xd, yd)
    yref = orc.action(fam, form, p, d, X, x, params=prm)
    assert np.abs(yd.cpu().numpy() - yref).max() <= TOL * np.abs(yref).max()
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("p", [1, 3, 6])
def test_spmv_equals_matrix_free_action(gpu, p):
    """At a size with several scratch chunks and all colour passes: the
    assembled product equals the matrix-free action (two independent paths),
    and both assembly and product are bitwise reproducible."""
    sfx, torch, ctx = gpu
    d = {1: (40, 40, 40), 3: (20, 20, 20), 6: (10, 10, 10)}[p]
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "Q", p)
    csr = sfx.Csr(sp)
    v1 = torch.empty(csr.nnz, dtype=torch.float64, device="cuda")
    v2 = torch.empty_like(v1)
    sfx.sfx_csr_assemble(ctx, "helmholtz", csr, v1)
    sfx.sfx_csr_assemble(ctx, "helmholtz", csr, v2)
    assert torch.equal(v1, v2)
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=2)).cuda()
    y1, y2, ya = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    sfx.sfx_csr_spmv(ctx, csr, v1, x, y1)
    sfx.sfx_csr_spmv(ctx, csr, v1, x, y2)
    assert torch.equal(y1, y2)
    sfx.sfx_assemble_action(ctx, "helmholtz", sp, x, ya)
    assert ((y1 - ya).abs().max() / ya.abs().max()).item() <= TOL
    assert ctx.sync_status() == 0


def test_csr_errors(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    sp = sfx.Space(mesh, "Q", 2)
    csr = sfx.Csr(sp)
    vals = torch.zeros(csr.nnz, dtype=torch.float64, device="cuda")
    x = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_csr_spmv(ctx, csr, vals, x, x)
    assert e.value.code == -1
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_csr_assemble(ctx, "neohooke", csr, vals)
    assert e.value.code == -1
