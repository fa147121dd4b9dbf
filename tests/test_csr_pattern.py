"""The assembled matrix's sparsity pattern (sfx_csr_create, host-only
context, no GPU) equals the pattern that the oracle's cell-node maps define:
row r holds every dof that shares a cell with r, sorted (global assembly,
Sec. 1.1).  Integer work: compared exactly."""
import numpy as np
import pytest

import paper_1711_02473_gb300 as sfx


@pytest.fixture(scope="module")
def host_ctx():
    return sfx.Context(-1)


def pattern_from_map(cmap, ndof):
    rows = [set() for _ in range(ndof)]
    for cell in cmap:
        for r in cell:
            rows[r].update(int(c) for c in cell)
    row_ptr = np.zeros(ndof + 1, dtype=np.int64)
    cols = []
    for r in range(ndof):
        s = sorted(rows[r])
        cols.extend(s)
        row_ptr[r + 1] = row_ptr[r] + len(s)
    return row_ptr, np.array(cols, dtype=np.int32)


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 2, 4)])
def test_pattern_matches_cell_maps(host_ctx, orc, fam, p, dims):
    m = sfx.Mesh.box(host_ctx, *dims)
    s = sfx.Space(m, fam, p)
    csr = sfx.Csr(s)
    rp, col = csr.pattern()
    ndof, _ = orc.space_size(fam, p, dims)
    rp_ref, col_ref = pattern_from_map(orc.cell_map(fam, p, dims), ndof)
    np.testing.assert_array_equal(rp, rp_ref)
    np.testing.assert_array_equal(col, col_ref)


def test_pattern_rejects_other_families(host_ctx):
    m = sfx.Mesh.box(host_ctx, 2, 2, 2)
    with pytest.raises(sfx.SfxError) as e:
        sfx.Csr(sfx.Space(m, "NCF", 2))
    assert e.value.code == -2
