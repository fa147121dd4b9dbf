"""GPU parity: element (tangent) matrices of the hyperelastic residual,
sfx_assemble_linearised_cell_matrices (the Jacobian of the Sec. 4.1 residual,
assembled per cell), through the C ABI against the oracle.

Bar: per cell max|A - A_ref| / max|A_ref| <= 1e-12 (FP64).  Column (b,j) must
equal the GPU per-cell vector of the linearised operator for the unit direction
at that dof to rounding (1e-13: the matrix kernel takes the direction's
gradient from the tabulated derivative and a rank-one dP, the action from
contractions and the full dP), and the assembled matrices must reproduce the
GPU action.  At 48^3 (the hyperelastic mesh of the structured
workload) a range of cells is compared with the oracle."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def case(p):
    """Mesh dims and the cell range compared with the oracle (the oracle's
    matrix costs O(p^9) per cell)."""
    if p <= 3:
        return (3, 2, 2), 0, 12
    if p <= 5:
        return (3, 2, 2), 3, 6
    return (2, 1, 2), 1, 2


def per_cell_rel(A, Aref):
    return max(np.abs(A[c] - Aref[c]).max() / np.abs(Aref[c]).max() for c in range(A.shape[0]))


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", range(1, 9))
def test_tangent_parity(gpu, orc, form, p):
    sfx, torch, ctx = gpu
    d, c0, c1 = case(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "VQ", p)
    u = inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)
    A = torch.empty((c1 - c0) * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_matrices(ctx, form, sp, torch.from_numpy(u).cuda(), c0, c1, A)
    Ag = A.cpu().numpy().reshape(c1 - c0, sp.nloc, sp.nloc)
    Aref = orc.linearised_cell_matrices(form, p, d, X, u, c0, c1)
    assert per_cell_rel(Ag, Aref) <= TOL
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [2, 5])
def test_columns_are_the_cell_vectors_of_unit_directions(gpu, orc, p, form):
    sfx, torch, ctx = gpu
    d = (3, 2, 2)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "VQ", p)
    u = torch.from_numpy(inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)).cuda()
    cell = 7
    A = torch.empty(sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_matrices(ctx, form, sp, u, cell, cell + 1, A)
    A = A.view(sp.nloc, sp.nloc)
    cmap = orc.cell_map("VQ", p, d)
    cells = torch.tensor([cell], dtype=torch.int64, device="cuda")
    b = torch.empty(sp.nloc, dtype=torch.float64, device="cuda")
    scale = A.abs().max().item()
    for j in sorted({0, 1, sp.nloc // 3, sp.nloc // 2, sp.nloc - 1}):
        du = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
        du[int(cmap[cell][j])] = 1.0
        sfx.sfx_assemble_linearised_cell_vectors(ctx, form, sp, u, du, cells, b)
        assert (A[:, j] - b).abs().max().item() <= 1e-13 * scale


@pytest.mark.parametrize("form", ["neohooke", "svk"])
def test_assembled_matrices_give_the_action(gpu, orc, form):
    sfx, torch, ctx = gpu
    d, p = (3, 2, 2), 3
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "VQ", p)
    u = torch.from_numpy(inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)).cuda()
    du = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=2)).cuda()
    A = torch.empty(sp.ncell * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_matrices(ctx, form, sp, u, 0, sp.ncell, A)
    cmap = torch.from_numpy(orc.cell_map("VQ", p, d).astype(np.int64)).cuda()
    A = A.view(sp.ncell, sp.nloc, sp.nloc)
    y = torch.zeros_like(du)
    y.index_add_(0, cmap.reshape(-1), torch.bmm(A, du[cmap].unsqueeze(2)).reshape(-1))
    ref = torch.empty_like(du)
    sfx.sfx_assemble_linearised_action(ctx, form, sp, u, du, ref)
    assert ((y - ref).abs().max() / ref.abs().max()).item() <= TOL


def test_cell_range_matches_full_range(gpu):
    sfx, torch, ctx = gpu
    d, p = (3, 2, 2), 2
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "VQ", p)
    u = torch.from_numpy(inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)).cuda()
    n2 = sp.nloc * sp.nloc
    full = torch.empty(sp.ncell * n2, dtype=torch.float64, device="cuda")
    part = torch.empty(3 * n2, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_matrices(ctx, "svk", sp, u, 0, sp.ncell, full)
    sfx.sfx_assemble_linearised_cell_matrices(ctx, "svk", sp, u, 5, 8, part)
    assert torch.equal(part, full[5 * n2:8 * n2])


def test_tangent_48cube_cell_range(gpu, orc):
    """The 48^3 hyperelastic mesh at p = 3: a range of cells in the middle of
    the mesh against the oracle (same state recipe as the residual workload)."""
    sfx, torch, ctx = gpu
    d, p = (48, 48, 48), 3
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "VQ", p)
    u = inputs.displacement(sp.ndof, p, d[0], seed=1)
    c0, c1 = 55296, 55300
    A = torch.empty((c1 - c0) * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_matrices(ctx, "neohooke", sp, torch.from_numpy(u).cuda(), c0, c1, A)
    Aref = orc.linearised_cell_matrices("neohooke", p, d, X, u, c0, c1)
    assert per_cell_rel(A.cpu().numpy().reshape(c1 - c0, sp.nloc, sp.nloc), Aref) <= TOL
    assert ctx.sync_status() == 0


def test_tangent_errors(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    sp = sfx.Space(mesh, "VQ", 1)
    u = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
    A = torch.empty(sp.ncell * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_linearised_cell_matrices(ctx, "neohooke", sp, u, 0, sp.ncell, A, precision="tf32x3")
    assert e.value.code == -2
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_linearised_cell_matrices(ctx, "laplace", sp, u, 0, sp.ncell, A)
    assert e.value.code == -1
    with pytest.raises(sfx.SfxError) as e:  # range past the mesh
        sfx.sfx_assemble_linearised_cell_matrices(ctx, "svk", sp, u, 1, sp.ncell + 1, A)
    assert e.value.code == -1
    sq = sfx.Space(mesh, "Q", 1)
    uq = torch.zeros(sq.ndof, dtype=torch.float64, device="cuda")
    Aq = torch.empty(sq.ncell * sq.nloc * sq.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_linearised_cell_matrices(ctx, "svk", sq, uq, 0, sq.ncell, Aq)
    assert e.value.code == -1
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    assert sfx.sfx_assemble_linearised_cell_matrices(ctx, "svk", sp, u, 3, 3, empty) is empty
