"""Pins for the oracle's dof numbering: exact counts, sharing multiplicities,
and geometric consistency of shared nodes (Sec. 1.1 global assembly; Sec. 3.5
local layout, Eqs. rtcf_split_x/y)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs


def counts(fam, p, d):
    nx, ny, nz = d
    n = p + 1
    if fam == "Q":
        return (p * nx + 1) * (p * ny + 1) * (p * nz + 1), n ** 3
    if fam == "VQ":
        return 3 * (p * nx + 1) * (p * ny + 1) * (p * nz + 1), 3 * n ** 3
    if fam == "DQ":
        return nx * ny * nz * n ** 3, n ** 3
    if fam == "NCF":
        g = ((p * nx + 1) * p * ny * p * nz + p * nx * (p * ny + 1) * p * nz + p * nx * p * ny * (p * nz + 1))
        return g, 3 * p * p * (p + 1)
    if fam == "NCE":
        g = (p * nx * (p * ny + 1) * (p * nz + 1) + (p * nx + 1) * p * ny * (p * nz + 1)
             + (p * nx + 1) * (p * ny + 1) * p * nz)
        return g, 3 * p * (p + 1) ** 2


@pytest.mark.parametrize("fam", ["Q", "DQ", "VQ", "NCF", "NCE"])
@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_counts_and_surjective(orc, fam, p):
    d = (2, 3, 4)
    ndof, nloc = orc.space_size(fam, p, d)
    assert (ndof, nloc) == counts(fam, p, d)
    m = orc.cell_map(fam, p, d)
    assert m.shape == (24, nloc)
    assert m.min() == 0 and m.max() == ndof - 1
    assert len(np.unique(m)) == ndof  # every dof belongs to some cell
    for row in m:
        assert len(np.unique(row)) == nloc  # no dof repeated inside a cell


def test_q_multiplicities(orc):
    """Each dof at an interior vertex is shared by exactly 8 cells, at an
    interior edge by 4, at an interior face by 2, inside a cell by 1."""
    p, d = 3, (3, 3, 3)
    m = orc.cell_map("Q", p, d)
    mult = np.bincount(m.ravel())
    M = p * 3 + 1
    I, J, K = np.unravel_index(np.arange(M ** 3), (M, M, M))
    on = lambda t: (t % p == 0) & (t > 0) & (t < M - 1)  # on an interior grid plane
    inside = lambda t: (t > 0) & (t < M - 1)
    k = on(I).astype(int) + on(J).astype(int) + on(K).astype(int)
    interior = inside(I) & inside(J) & inside(K)
    np.testing.assert_array_equal(mult[interior], (2 ** k)[interior])


@pytest.mark.parametrize("fam,share", [("NCF", 2), ("NCE", 4)])
def test_hdiv_hcurl_sharing(orc, fam, share):
    """NCF dofs live on faces (shared by at most 2 cells), NCE dofs on edges
    (at most 4) or inside; DQ dofs are never shared."""
    m = orc.cell_map(fam, 2, (3, 3, 3))
    mult = np.bincount(m.ravel())
    assert mult.max() == share
    assert orc.cell_map("DQ", 2, (3, 3, 3)).ravel().tolist() == list(range(27 * 27))


@pytest.mark.parametrize("p", [1, 2, 4])
def test_q_node_positions_consistent(orc, p):
    """Shared nodes get the same physical point from every cell: on the
    unperturbed box the node of global index (I,J,K) sits at the GLL point of
    its cell, independently of which cell wrote it."""
    d = (2, 3, 2)
    X = inputs.box_coords(*d, perturb=0.0)
    xyz = orc.q_node_coords(p, d, X)
    gll, _ = orc.gauss_lobatto(p + 1)
    M = [p * n + 1 for n in d]
    I, J, K = np.unravel_index(np.arange(np.prod(M)), M)
    for axis, (t, n) in enumerate(zip((I, J, K), d)):
        cell = np.minimum(t // p, n - 1)
        loc = t - cell * p
        np.testing.assert_allclose(xyz[:, axis], (cell + gll[loc]) / n, atol=1e-15)


def test_cell_dofs_match_map(orc):
    d = (2, 2, 3)
    m = orc.cell_map("NCE", 3, d)
    for c in (0, 5, 11):
        np.testing.assert_array_equal(m[c], orc_cell_dofs(orc, "NCE", 3, d, c))


def orc_cell_dofs(orc, fam, p, d, c):
    import ctypes
    _, nloc = orc.space_size(fam, p, d)
    out = np.zeros(nloc, dtype=np.int64)
    assert orc.lib().orc_cell_dofs(orc.FAMILIES[fam], p, *d, c, out.ctypes.data_as(ctypes.c_void_p)) == 0
    return out
