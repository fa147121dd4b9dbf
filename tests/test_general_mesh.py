"""General hexahedral meshes given by connectivity (sfx_mesh_create), on the
host (host-only context, no GPU), and the colour lists of every space.

Integer results are compared exactly (Sec. 1.1: global assembly sums the cells'
contributions through the cell-node map; several numberings are correct, so
maps are compared as partitions of the (cell, local dof) slots):
* the oracle's own general-mesh numbering (lattice weights of the cell's
  corners) against its structured box numbering on a box presented with
  shuffled vertices, shuffled cells and rotated cells;
* the library's numbering (edges and faces oriented by global vertex ids)
  against the oracle's, on the shuffled box and on an unstructured prism mesh
  with valence-3 edges;
* node coordinates agree from every cell that shares a node;
* the oracle's general-mesh assembly against its box assembly, and its pins on
  the prism (volume, constants in the Laplace kernel, the patch test);
* colour lists: recomputed independently (the parity classes on a box, greedy
  first fit on a general mesh), equal entry for entry, and no two cells of one
  colour share a dof."""
import numpy as np
import pytest

import paper_1711_02473_gb300 as sfx
from paper_1711_02473_gb300 import inputs


@pytest.fixture(scope="module")
def host_ctx():
    return sfx.Context(-1)


def bijection(ma, mb):
    """The dof map f with mb = f(ma) slot by slot, if the two cell-node maps
    define the same partition of the slots; else None."""
    a, b = np.asarray(ma).ravel(), np.asarray(mb).ravel()
    pairs = np.unique(np.stack([a, b], axis=1), axis=0)
    if len(np.unique(pairs[:, 0])) != len(pairs) or len(np.unique(pairs[:, 1])) != len(pairs):
        return None
    f = np.full(int(a.max()) + 1, -1, dtype=np.int64)
    f[pairs[:, 0]] = pairs[:, 1]
    return f


def lattice(p):
    n = p + 1
    return np.array([(i1, i2, i3) for i1 in range(n) for i2 in range(n) for i3 in range(n)])


def box_slots_of_shuffled(p, dims, cell_of, rot):
    """For each (new cell k, local node l') the box (cell, local node) it is."""
    rots = inputs.cube_rotations()
    L = lattice(p)
    n = p + 1
    out_c = np.repeat(np.asarray(cell_of), len(L)).reshape(len(cell_of), len(L))
    out_l = np.empty_like(out_c)
    for k, r in enumerate(rot):
        M = rots[r]
        I = (((2 * L - p) @ M.T) + p) // 2  # i = (M (2 i' - p) + p) / 2
        out_l[k] = (I[:, 0] * n + I[:, 1]) * n + I[:, 2]
    return out_c, out_l


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_oracle_general_map_is_the_box_map(orc, p):
    dims = (3, 2, 4)
    xyz, cells, vnew, cell_of, rot = inputs.shuffled_box(*dims)
    m, nd = orc.general_map("Q", p, orc.vtk_to_corner_order(cells))
    box = orc.cell_map("Q", p, dims)
    oc, ol = box_slots_of_shuffled(p, dims, cell_of, rot)
    assert nd == orc.space_size("Q", p, dims)[0]
    assert bijection(m, box[oc, ol]) is not None


def node_coords(orc, p, xyz, corner_vertices):
    """Physical position of every (cell, local node): the trilinear map at the
    GLL lattice point."""
    g, _ = orc.gauss_lobatto(p + 1)
    L = lattice(p)
    xi = g[L]  # (nloc, 3)
    X = xyz[corner_vertices]  # (ncell, 8, 3)
    out = np.zeros((X.shape[0], len(L), 3))
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = ((xi[:, 0] if a else 1 - xi[:, 0]) * (xi[:, 1] if b else 1 - xi[:, 1])
                     * (xi[:, 2] if c else 1 - xi[:, 2]))
                out += w[None, :, None] * X[:, None, 4 * a + 2 * b + c, :]
    return out


MESHES = {"shuffled_box": lambda: inputs.shuffled_box(3, 2, 4)[:2],
          "prism": lambda: inputs.prism_mesh(2, 2)[:2],
          "prism_fine": lambda: inputs.prism_mesh(3, 3)[:2]}


@pytest.mark.parametrize("mesh", sorted(MESHES))
@pytest.mark.parametrize("fam,p", [("Q", 1), ("Q", 2), ("Q", 3), ("Q", 5), ("VQ", 2), ("DQ", 2)])
def test_library_general_map_matches_oracle(host_ctx, orc, mesh, fam, p):
    xyz, cells = MESHES[mesh]()
    M = sfx.Mesh.general(host_ctx, xyz, cells)
    sp = sfx.Space(M, fam, p)
    V = orc.vtk_to_corner_order(cells)
    m, nd = orc.general_map(fam, p, V)
    assert sp.ndof == nd and sp.nloc == m.shape[1]
    lib_map = sp.cell_map()
    assert lib_map.min() >= 0 and lib_map.max() < sp.ndof
    assert len(np.unique(lib_map)) == sp.ndof or fam != "DQ"
    assert bijection(lib_map, m) is not None
    if fam == "Q":
        # every cell that holds a dof places it at the same point
        X = node_coords(orc, p, xyz, V).reshape(-1, 3)
        ref = np.zeros((sp.ndof, 3))
        ref[lib_map.ravel()] = X
        assert np.abs(ref[lib_map.ravel()] - X).max() <= 1e-14


def test_library_general_map_entity_counts(host_ctx):
    """Q_p dofs = vertices + (p-1) edges + (p-1)^2 faces + (p-1)^3 cells (Euler
    counts of the prism mesh, found from the vertex sets)."""
    xyz, cells, _ = inputs.prism_mesh(2, 2)
    M = sfx.Mesh.general(host_ctx, xyz, cells)
    edges, faces = set(), set()
    C = np.array(cells)
    for c in C:
        b, t = c[:4], c[4:]
        for ring in (b, t):
            for i in range(4):
                edges.add(frozenset((ring[i], ring[(i + 1) % 4])))
        for i in range(4):
            edges.add(frozenset((b[i], t[i])))
            faces.add(frozenset((b[i], b[(i + 1) % 4], t[i], t[(i + 1) % 4])))
        faces.add(frozenset(b))
        faces.add(frozenset(t))
    for p in (1, 2, 3, 4):
        sp = sfx.Space(M, "Q", p)
        assert sp.ndof == len(xyz) + (p - 1) * len(edges) + (p - 1) ** 2 * len(faces) + (p - 1) ** 3 * len(C)


@pytest.mark.parametrize("fam,form,p", [("Q", "mass", 1), ("Q", "laplace", 2), ("Q", "helmholtz", 3),
                                        ("VQ", "neohooke", 2), ("DQ", "laplace", 2)])
def test_oracle_general_action_is_the_box_action(orc, fam, form, p):
    dims = (3, 2, 4)
    X = inputs.box_coords(*dims)
    xyz, cells, vnew, cell_of, rot = inputs.shuffled_box(*dims)
    ndof = orc.space_size(fam, p, dims)[0]
    xb = inputs.random_vector(ndof, 1, seed=1)
    if fam == "VQ":
        xb = xb * 0.01
    yb = orc.action(fam, form, p, dims, X, xb)
    # the same field in the general numbering, through the slot correspondence
    V = orc.vtk_to_corner_order(cells)
    m, nd = orc.general_map(fam, p, V)
    boxmap = orc.cell_map(fam, p, dims)
    if fam == "DQ":
        n3 = (p + 1) ** 3
        oc, ol = box_slots_of_shuffled(p, dims, cell_of, rot)
        bslots = boxmap[oc, ol]
    else:
        nc = 3 if fam == "VQ" else 1
        n3 = (p + 1) ** 3
        oc, ol = box_slots_of_shuffled(p, dims, cell_of, rot)
        bslots = np.concatenate([boxmap[oc, ol + k * n3] for k in range(nc)], axis=1)
    f = bijection(m, bslots)
    assert f is not None
    y, _, _ = orc.general_action(fam, form, p, xyz, cells, xb[f])
    assert np.abs(y - yb[f]).max() <= 1e-12 * np.abs(yb).max()


def test_oracle_prism_pins(orc):
    """Unstructured prism, perturbed: 1^T M 1 = volume (det J is of degree <= 2
    per direction, integrated exactly); the Laplace matrix annihilates
    constants; for u = a . x (in Q_p), u^T A u = |a|^2 volume and the mass
    action against 1 gives the integral of u."""
    xyz, cells, vol = inputs.prism_mesh(2, 2)
    V = orc.vtk_to_corner_order(cells)
    for p in (1, 2, 3):
        m, nd = orc.general_map("Q", p, V)
        one = np.ones(nd)
        ym, _, _ = orc.general_action("Q", "mass", p, xyz, cells, one)
        assert abs(ym.sum() - vol) <= 1e-13
        yl, _, _ = orc.general_action("Q", "laplace", p, xyz, cells, one)
        assert np.abs(yl).max() <= 1e-12
        X = node_coords(orc, p, xyz, V).reshape(-1, 3)
        pos = np.zeros((nd, 3))
        pos[m.ravel()] = X
        a = np.array([0.3, -1.1, 0.7])
        u = pos @ a
        yu, _, _ = orc.general_action("Q", "laplace", p, xyz, cells, u)
        assert abs(u @ yu - (a @ a) * vol) <= 1e-12
        cen = (ym @ pos) / vol  # centroid of the prism: mean of the triangle's corners, z = 1/2
        assert np.abs(cen - np.array([0.5, 0.8 / 3, 0.5])).max() <= 1e-13


# ------------------------------------------------------------------ colours

def parity_colours(dims):
    nx, ny, nz = dims
    c = np.arange(nx * ny * nz)
    i, j, k = c // (ny * nz), (c // nz) % ny, c % nz
    col = 4 * (i & 1) + 2 * (j & 1) + (k & 1)
    off = np.concatenate([[0], np.cumsum(np.bincount(col, minlength=8))])
    return off, np.concatenate([c[col == k] for k in range(8)]).astype(np.int32)


def greedy_colours(cells_vtk):
    ncell = len(cells_vtk)
    by_vertex = {}
    for c, vs in enumerate(cells_vtk):
        for v in vs:
            by_vertex.setdefault(int(v), []).append(c)
    col = [-1] * ncell
    for c, vs in enumerate(cells_vtk):
        used = {col[o] for v in vs for o in by_vertex[int(v)] if o < c}
        k = 0
        while k in used:
            k += 1
        col[c] = k
    col = np.array(col)
    nc = col.max() + 1
    off = np.concatenate([[0], np.cumsum(np.bincount(col, minlength=nc))])
    return off, np.concatenate([np.flatnonzero(col == k) for k in range(nc)]).astype(np.int32)


def no_shared_dof(off, cl, cmap):
    for k in range(len(off) - 1):
        d = cmap[cl[off[k]:off[k + 1]]].ravel()
        if len(np.unique(d)) != len(d):
            return False
    return True


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 3, 2), (4, 1, 1), (2, 2, 2), (3, 4, 5), (5, 2, 3)])
@pytest.mark.parametrize("fam", ["Q", "NCF", "NCE", "VQ", "DQ"])
def test_box_colours_exact(host_ctx, fam, dims):
    M = sfx.Mesh.box(host_ctx, *dims)
    for p in (1, 2, 3):
        sp = sfx.Space(M, fam, p)
        off, cl = sp.colours()
        if fam == "DQ":
            np.testing.assert_array_equal(off, [0, sp.ncell])
            np.testing.assert_array_equal(cl, np.arange(sp.ncell))
        else:
            eo, ec = parity_colours(dims)
            np.testing.assert_array_equal(off, eo)
            np.testing.assert_array_equal(cl, ec)
        assert np.array_equal(np.sort(cl), np.arange(sp.ncell))
        assert no_shared_dof(off, cl, sp.cell_map())


@pytest.mark.parametrize("mesh", sorted(MESHES))
@pytest.mark.parametrize("fam", ["Q", "VQ", "DQ"])
def test_general_colours_exact(host_ctx, mesh, fam):
    xyz, cells = MESHES[mesh]()
    M = sfx.Mesh.general(host_ctx, xyz, cells)
    sp = sfx.Space(M, fam, 2)
    off, cl = sp.colours()
    if fam == "DQ":
        np.testing.assert_array_equal(off, [0, sp.ncell])
        np.testing.assert_array_equal(cl, np.arange(sp.ncell))
    else:
        eo, ec = greedy_colours(cells)
        np.testing.assert_array_equal(off, eo)
        np.testing.assert_array_equal(cl, ec)
    assert no_shared_dof(off, cl, sp.cell_map())


def test_general_mesh_rejects_bad_input(host_ctx):
    xyz, cells, _ = inputs.prism_mesh(1, 1)
    bad = cells.copy()
    bad[0, 3] = len(xyz)  # out of range
    with pytest.raises(sfx.SfxError) as e:
        sfx.Mesh.general(host_ctx, xyz, bad)
    assert e.value.code == -1
    bad = cells.copy()
    bad[1, 5] = bad[1, 0]  # a repeated vertex
    with pytest.raises(sfx.SfxError):
        sfx.Mesh.general(host_ctx, xyz, bad)
    M = sfx.Mesh.general(host_ctx, xyz, cells)
    for fam in ("NCF", "NCE"):
        with pytest.raises(sfx.SfxError) as e:
            sfx.Space(M, fam, 1)
        assert e.value.code == -2
    with pytest.raises(sfx.SfxError) as e:
        sfx.Csr(sfx.Space(M, "Q", 1))
    assert e.value.code == -2


# --------------------------------------------------------------- first touch
def first_touch_reference(off, cl, cmap):
    """The dof's first cell-node pair in colour order, recomputed from the map
    and the colour lists: (cell, l) pairs, one per dof."""
    ncell, nloc = cmap.shape
    bits = np.zeros((ncell, (nloc + 31) // 32), dtype=np.uint32)
    seen = set()
    for k in range(len(off) - 1):
        for c in cl[off[k]:off[k + 1]]:
            for l in range(nloc):
                d = int(cmap[c, l])
                if d not in seen:
                    seen.add(d)
                    bits[c, l >> 5] |= np.uint32(1 << (l & 31))
    return bits


@pytest.mark.parametrize("which", ["box_1x1x1", "box_1x3x2", "box_3x4x2"] + sorted(MESHES))
def test_first_touch_bits_exact(host_ctx, which):
    """Every dof has exactly one first-touch pair, it lies in the earliest
    colour among the cells holding the dof, and the bits match a recomputation
    from the map and the colour lists bit for bit; other families have none."""
    if which.startswith("box_"):
        dims = tuple(int(v) for v in which[4:].split("x"))
        M = sfx.Mesh.box(host_ctx, *dims)
    else:
        xyz, cells = MESHES[which]()
        M = sfx.Mesh.general(host_ctx, xyz, cells)
    for p in (1, 2, 3):
        sp = sfx.Space(M, "Q", p)
        bits = sp.first_touch()
        cmap = sp.cell_map()
        off, cl = sp.colours()
        np.testing.assert_array_equal(bits, first_touch_reference(off, cl, cmap))
        colour = np.empty(sp.ncell, dtype=np.int64)
        for k in range(len(off) - 1):
            colour[cl[off[k]:off[k + 1]]] = k
        l = np.arange(sp.nloc)
        is_first = ((bits[:, l >> 5] >> (l & 31).astype(np.uint32)) & 1).astype(bool)
        counts = np.bincount(cmap[is_first], minlength=sp.ndof)
        assert (counts == 1).all()
        first_col = np.full(sp.ndof, -1)
        first_col[cmap[is_first]] = np.broadcast_to(colour[:, None], cmap.shape)[is_first]
        min_col = np.full(sp.ndof, np.iinfo(np.int64).max)
        np.minimum.at(min_col, cmap.ravel(), np.repeat(colour, sp.nloc))
        np.testing.assert_array_equal(first_col, min_col)
    for fam in ("DQ", "VQ"):
        assert sfx.Space(M, fam, 2).first_touch() is None
