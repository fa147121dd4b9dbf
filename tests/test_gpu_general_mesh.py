"""GPU parity on general hexahedral meshes (sfx_mesh_create): the library's
actions, residuals and element matrices against the oracle's general-mesh
assembly (its own numbering; the two numberings are related by the unique dof
bijection that maps one cell-node map onto the other, checked to exist).
Meshes: a perturbed box presented with shuffled vertices, shuffled cells and
rotated cells, and an unstructured prism mesh with valence-3 edges.  FP64 bar
1e-12 normwise, TF32x3 2e-5; runs repeat bitwise (colour passes)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
HELM = (1.0, -1.0, 0.0, 0.0)
MESHES = {"shuffled_box": lambda: inputs.shuffled_box(4, 3, 3)[:2],
          "prism": lambda: inputs.prism_mesh(3, 2)[:2]}


def bijection(ma, mb):
    a, b = np.asarray(ma).ravel(), np.asarray(mb).ravel()
    pairs = np.unique(np.stack([a, b], axis=1), axis=0)
    assert len(np.unique(pairs[:, 0])) == len(pairs) and len(np.unique(pairs[:, 1])) == len(pairs)
    f = np.full(int(a.max()) + 1, -1, dtype=np.int64)
    f[pairs[:, 0]] = pairs[:, 1]
    return f


@pytest.mark.parametrize("mesh", sorted(MESHES))
@pytest.mark.parametrize("fam,p", [("Q", 1), ("Q", 2), ("Q", 3), ("Q", 5), ("Q", 8), ("DQ", 3)])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
def test_general_action_parity(gpu, orc, mesh, fam, p, form):
    sfx, torch, ctx = gpu
    xyz, cells = MESHES[mesh]()
    M = sfx.Mesh.general(ctx, xyz, cells)
    sp = sfx.Space(M, fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    prm = HELM if form == "helmholtz" else None
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, params=prm)
    y1 = yd.clone()
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, params=prm)
    assert ctx.sync_status() == 0
    assert torch.equal(y1, yd)
    V = orc.vtk_to_corner_order(cells)
    m, nd = orc.general_map(fam, p, V)
    f = bijection(sp.cell_map(), m)
    xo = np.empty(nd)
    xo[f] = x
    yo, _, _ = orc.general_action(fam, form, p, xyz, cells, xo, params=prm)
    y = yd.cpu().numpy()
    assert np.abs(y - yo[f]).max() <= 1e-12 * np.abs(yo).max()
    yt = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, form, sp, xd, yt, params=prm, precision="tf32x3")
    assert ctx.sync_status() == 0
    assert np.abs(yt.cpu().numpy() - yo[f]).max() <= 2e-5 * np.abs(yo).max()


@pytest.mark.parametrize("mesh", sorted(MESHES))
@pytest.mark.parametrize("form,p", [("neohooke", 2), ("svk", 3)])
def test_general_hyperelastic_residual_parity(gpu, orc, mesh, form, p):
    sfx, torch, ctx = gpu
    xyz, cells = MESHES[mesh]()
    M = sfx.Mesh.general(ctx, xyz, cells)
    sp = sfx.Space(M, "VQ", p)
    x = inputs.random_vector(sp.ndof, 1, seed=4) * (0.05 / (4 * p))
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd)
    assert ctx.sync_status() == 0
    m, nd = orc.general_map("VQ", p, orc.vtk_to_corner_order(cells))
    f = bijection(sp.cell_map(), m)
    xo = np.empty(nd)
    xo[f] = x
    yo, _, _ = orc.general_action("VQ", form, p, xyz, cells, xo)
    assert np.abs(yd.cpu().numpy() - yo[f]).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("mesh", sorted(MESHES))
@pytest.mark.parametrize("fam,form,p", [("Q", "laplace", 2), ("Q", "helmholtz", 4), ("DQ", "mass", 3),
                                        ("VQ", "laplace", 2)])
def test_general_cell_matrices_parity(gpu, orc, mesh, fam, form, p):
    sfx, torch, ctx = gpu
    xyz, cells = MESHES[mesh]()
    M = sfx.Mesh.general(ctx, xyz, cells)
    sp = sfx.Space(M, fam, p)
    prm = HELM if form == "helmholtz" else None
    A = torch.empty(sp.ncell * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, form, sp, 0, sp.ncell, A, params=prm)
    assert ctx.sync_status() == 0
    Ao = orc.general_cell_matrices(fam, form, p, xyz, cells, params=prm)
    Ag = A.cpu().numpy().reshape(Ao.shape)
    for c in range(sp.ncell):
        assert np.abs(Ag[c] - Ao[c]).max() <= 1e-12 * np.abs(Ao[c]).max(), c


def test_general_padaptive_plan(gpu, orc):
    """The p-adaptive DQ batch on the prism mesh against the oracle's per-cell
    vectors (DQ dofs belong to one cell, so the cell-major blocks compare
    directly)."""
    sfx, torch, ctx = gpu
    xyz, cells = MESHES["prism"]()
    M = sfx.Mesh.general(ctx, xyz, cells)
    deg = inputs.padaptive_degrees(len(cells), 6, seed=2)
    plan = sfx.Plan(ctx, M, deg, ["laplace", "mass"], nrhs=2)
    x = inputs.random_vector(plan.ndof, 2, seed=0)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda().reshape(-1)
    ys = [torch.empty_like(xd) for _ in range(2)]
    plan.execute(xd, ys, mode="graph")
    assert ctx.sync_status() == 0
    V = orc.vtk_to_corner_order(cells)
    corners = xyz[V]
    off = plan.cell_offset
    for fi, form in enumerate(["laplace", "mass"]):
        y = ys[fi].cpu().numpy().reshape(-1, 2)
        for p in np.unique(deg):
            cs = np.flatnonzero(deg == p)
            xl = np.stack([x[off[c]:off[c + 1]] for c in cs])
            b = orc.local_vectors("DQ", form, int(p), corners[cs], xl)
            for k, c in enumerate(cs):
                ref = b[k]
                assert np.abs(y[off[c]:off[c + 1]] - ref).max() <= 1e-12 * np.abs(ref).max()
