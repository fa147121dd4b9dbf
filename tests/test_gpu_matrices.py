"""GPU parity of the local element matrices (Sec. 3.2 argument + sum
factorisation; Sec. 3.5 block splitting for NCF/NCE) and of the naive
(un-factorised) kernels, against the FP64 oracle.  Bar: 1e-12, per cell,
max|A - A_ref| / max|A_ref|."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def cellwise_rel(A, R):
    return max(np.abs(A[c] - R[c]).max() / np.abs(R[c]).max() for c in range(len(R)))


def dims_for(p, fam):
    big = fam in ("NCF", "NCE")
    if p <= 3:
        return (2, 2, 2)
    if p <= 5 and not big:
        return (2, 2, 1)
    return (2, 1, 1) if p <= 6 else (1, 1, 1)


def gpu_matrices(sfx, torch, ctx, sp, form, c0, c1, params=None, algo="sumfact"):
    A = torch.empty((c1 - c0) * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, form, sp, c0, c1, A, params=params, algo=algo)
    return A.cpu().numpy().reshape(c1 - c0, sp.nloc, sp.nloc)


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", range(1, 9))
def test_scalar_matrices(gpu, orc, fam, form, p):
    sfx, torch, ctx = gpu
    d = dims_for(p, fam)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    nc = d[0] * d[1] * d[2]
    prm = (0.9, -1.7, 0, 0) if form == "helmholtz" else None
    A = gpu_matrices(sfx, torch, ctx, sp, form, 0, nc, prm)
    R = orc.cell_matrices(fam, form, p, d, X, params=prm)
    assert cellwise_rel(A, R) <= TOL
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("fam,form", [("NCF", "ncf_mass_divdiv"), ("NCE", "nce_curlcurl")])
@pytest.mark.parametrize("p", range(1, 9))
def test_hdivcurl_matrices(gpu, orc, fam, form, p):
    sfx, torch, ctx = gpu
    d = dims_for(p, fam)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    nc = d[0] * d[1] * d[2]
    prm = (0.6, 1.4, 0, 0)
    A = gpu_matrices(sfx, torch, ctx, sp, form, 0, nc, prm)
    R = orc.cell_matrices(fam, form, p, d, X, params=prm)
    assert cellwise_rel(A, R) <= TOL


@pytest.mark.parametrize("fam,form,p", [("Q", "laplace", 3), ("DQ", "helmholtz", 2), ("NCF", "ncf_mass_divdiv", 2),
                                        ("NCE", "nce_curlcurl", 2)])
def test_matrices_reproduce_action(gpu, fam, form, p):
    """sum_K P_K^T A^K P_K x equals the matrix-free action, both on the GPU,
    over a cell range split into two chunks."""
    sfx, torch, ctx = gpu
    d = (3, 3, 2)
    sp = sfx.Space(sfx.Mesh.box(ctx, *d), fam, p)
    nc = sp.ncell
    A = np.concatenate([gpu_matrices(sfx, torch, ctx, sp, form, 0, 7),
                        gpu_matrices(sfx, torch, ctx, sp, form, 7, nc)])
    m = sp.cell_map()
    x = inputs.random_vector(sp.ndof, 1, seed=2)
    y = np.zeros(sp.ndof)
    for c in range(nc):
        np.add.at(y, m[c], A[c] @ x[m[c]])
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, form, sp, torch.from_numpy(x).cuda(), yd)
    assert np.abs(y - yd.cpu().numpy()).max() <= TOL * np.abs(y).max()


@pytest.mark.parametrize("fam,form,p", [("Q", "laplace", 2), ("Q", "helmholtz", 3), ("DQ", "laplace", 3),
                                        ("NCE", "nce_curlcurl", 2), ("NCF", "ncf_mass_divdiv", 3)])
def test_naive_matrices_agree(gpu, fam, form, p):
    """The O(n^9) naive kernel and the sum-factorised kernel compute the same
    sum in a different order."""
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 2, 2, 1), fam, p)
    A = gpu_matrices(sfx, torch, ctx, sp, form, 0, 4)
    An = gpu_matrices(sfx, torch, ctx, sp, form, 0, 4, algo="naive")
    assert cellwise_rel(A, An) <= TOL


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_naive_action_parity(gpu, orc, fam, form, p):
    sfx, torch, ctx = gpu
    d = (5, 4, 3) if p <= 2 else (3, 3, 2)
    X = inputs.box_coords(*d)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, form, sp, torch.from_numpy(x).cuda(), yd, algo="naive")
    ref = orc.action(fam, form, p, d, X, x)
    assert np.abs(yd.cpu().numpy() - ref).max() <= TOL * np.abs(ref).max()


def test_matrix_argument_errors(gpu):
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 2, 2, 2), "VQ", 2)
    A = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError):  # residual forms have no element matrix
        sfx.sfx_assemble_cell_matrices(ctx, "neohooke", sp, 0, 0, A[:0])
    sp2 = sfx.Space(sfx.Mesh.box(ctx, 2, 2, 2), "Q", 2)
    with pytest.raises(sfx.SfxError):
        sfx.sfx_assemble_cell_matrices(ctx, "laplace", sp2, 3, 9, torch.empty(6 * 27 * 27, dtype=torch.float64,
                                                                               device="cuda"))
