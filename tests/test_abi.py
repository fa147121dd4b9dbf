"""The C-ABI library loads, exports every symbol include/sfx.h declares, and
its host-side logic (1D rules and tables, box coordinates, dof maps,
argument checking) agrees with the oracle and the input generator -- all
without a GPU (host-only context, device = -1)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1711_02473_gb300 as sfx
from paper_1711_02473_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    sfx.build()
    return sfx.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "sfx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sfx_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(sfx.EXPORTS) == syms


def test_status_strings(L):
    for code, text in sfx.STATUS.items():
        assert L.sfx_status_string(code).decode() == text


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 16])
def test_tabulate_matches_oracle(L, orc, n):
    """The library's Newton/barycentric rules and tables against the oracle's
    Golub-Welsch rules and product-formula Lagrange polynomials."""
    x, w, _ = sfx.sfx_tabulate_1d("GL", max(n, 1), "GL", n)
    xo, wo = orc.gauss_legendre(n)
    np.testing.assert_allclose(x, xo, atol=2e-16)
    np.testing.assert_allclose(w, wo, atol=2e-16)
    if n >= 2:
        x, w, _ = sfx.sfx_tabulate_1d("GLL", n, "GLL", n)
        xo, wo = orc.gauss_lobatto(n)
        np.testing.assert_allclose(x, xo, atol=2e-16)
        np.testing.assert_allclose(w, wo, atol=2e-16)
    for nodes in ("GLL", "GL"):
        if nodes == "GLL" and n < 2:
            continue
        xn = (orc.gauss_lobatto if nodes == "GLL" else orc.gauss_legendre)(n)[0]
        for deriv in (0, 1):
            for q in (n, n + 1):
                pts, _, tab = sfx.sfx_tabulate_1d(nodes, n, "GL", q, deriv)
                ref = np.array([[orc.lagrange(xn, i, t, deriv=bool(deriv)) for i in range(n)] for t in pts])
                np.testing.assert_allclose(tab, ref, atol=1e-13 * max(1.0, np.abs(ref).max()))
    # collocated table (nodes = points) is the identity (Sec. 2.5, Eq. colocated)
    _, _, tab = sfx.sfx_tabulate_1d("GL", n, "GL", n, 0)
    np.testing.assert_array_equal(tab, np.eye(n))


def test_tabulate_rejects_bad_arguments(L):
    P = C.c_void_p
    assert L.sfx_tabulate_1d(0, 1, 1, 3, 0, None, None, None) == -1  # GLL needs 2 nodes
    assert L.sfx_tabulate_1d(1, 3, 0, 1, 0, None, None, None) == -1  # GLL rule needs 2 points
    assert L.sfx_tabulate_1d(1, 3, 1, 0, 0, None, None, None) == -1
    assert L.sfx_tabulate_1d(1, 3, 1, 3, 2, None, None, None) == -1
    assert L.sfx_tabulate_1d(7, 3, 1, 3, 0, None, None, None) == -1


@pytest.fixture(scope="module")
def host_ctx(L):
    return sfx.Context(-1)


@pytest.mark.parametrize("dims", [(1, 1, 1), (4, 3, 5), (8, 8, 8)])
def test_box_coords_bit_identical(host_ctx, dims):
    m = sfx.Mesh.box(host_ctx, *dims, perturb=0.1, seed=0)
    np.testing.assert_array_equal(m.coords(), inputs.box_coords(*dims, perturb=0.1, seed=0))
    m2 = sfx.Mesh.box(host_ctx, *dims, perturb=0.05, seed=77)
    np.testing.assert_array_equal(m2.coords(), inputs.box_coords(*dims, perturb=0.05, seed=77))


@pytest.mark.parametrize("fam", ["Q", "DQ", "VQ", "NCF", "NCE"])
@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_cell_maps_bit_identical(host_ctx, orc, fam, p):
    dims = (3, 2, 4)
    m = sfx.Mesh.box(host_ctx, *dims)
    s = sfx.Space(m, fam, p)
    ndof, nloc = orc.space_size(fam, p, dims)
    assert (s.ndof, s.nloc, s.ncell) == (ndof, nloc, 24)
    np.testing.assert_array_equal(s.cell_map(), orc.cell_map(fam, p, dims))


def test_argument_errors(L, host_ctx):
    h = C.c_void_p()
    assert L.sfx_ctx_create(0, None) == -1
    assert L.sfx_ctx_create(-2, C.byref(h)) == -1
    assert L.sfx_mesh_create_box(host_ctx.h, 0, 1, 1, 0.1, 0, C.byref(h)) == -1
    assert L.sfx_mesh_create_box(host_ctx.h, 1, 1, 1, 0.5, 0, C.byref(h)) == -1
    assert L.sfx_mesh_create_box(None, 1, 1, 1, 0.1, 0, C.byref(h)) == -1
    m = sfx.Mesh.box(host_ctx, 2, 2, 2)
    assert L.sfx_space_create(m.h, 9, 2, C.byref(h)) == -1
    assert L.sfx_space_create(m.h, 0, 0, C.byref(h)) == -2
    assert L.sfx_space_create(m.h, 0, 9, C.byref(h)) == -2
    s = sfx.Space(m, "Q", 2)
    # assembly on a host-only context is an argument error, not a crash
    assert L.sfx_assemble_action(host_ctx.h, 1, None, s.h, C.c_void_p(8), C.c_void_p(16), 1, 0, 0, 0, None) == -1
    bits = C.c_uint32()
    assert L.sfx_sync_status(host_ctx.h, None, C.byref(bits)) == -1
    assert L.sfx_assemble_cell_matrices(host_ctx.h, 5, None, s.h, 0, 1, C.c_void_p(8), 0, 0, None) == -1


def test_tuning_table_arguments(L):
    """The launch-shape table (kinds 0..11, degrees 1..8, 0..64 cells) and the
    warp-specialised switch check their arguments as documented and
    round-trip what they store; nothing here touches a device."""
    i = C.c_int()
    saved = {}
    for k in range(12):
        for p in range(1, 9):
            assert L.sfx_tune_get_cells_per_cta(k, p, C.byref(i)) == 0
            saved[k, p] = i.value
    try:
        for k in range(12):
            for p in range(1, 9):
                assert L.sfx_tune_set_cells_per_cta(k, p, (k + p) % 7 + 1) == 0
        for k in range(12):
            for p in range(1, 9):
                assert L.sfx_tune_get_cells_per_cta(k, p, C.byref(i)) == 0 and i.value == (k + p) % 7 + 1
        for args in ((-1, 1, 1), (12, 1, 1), (0, 0, 1), (0, 9, 1), (0, 1, -1), (0, 1, 65)):
            assert L.sfx_tune_set_cells_per_cta(*args) == -1, args
        assert L.sfx_tune_get_cells_per_cta(0, 1, None) == -1
        assert L.sfx_tune_get_cells_per_cta(12, 1, C.byref(i)) == -1
    finally:
        for (k, p), v in saved.items():
            assert L.sfx_tune_set_cells_per_cta(k, p, v) == 0
    e = C.c_int()
    assert L.sfx_tune_get_warp_specialised(4, C.byref(e)) == 0
    ws4 = e.value
    try:
        assert L.sfx_tune_set_warp_specialised(2, 1) == -2   # no warp-specialised kernel below p = 3
        assert L.sfx_tune_set_warp_specialised(2, 0) == 0
        for args in ((0, 1), (9, 0), (4, 2), (4, -1)):
            assert L.sfx_tune_set_warp_specialised(*args) == -1, args
        assert L.sfx_tune_get_warp_specialised(4, None) == -1
        assert L.sfx_tune_get_warp_specialised(0, C.byref(e)) == -1
        assert L.sfx_tune_set_warp_specialised(4, 1 - ws4) == 0
        assert L.sfx_tune_get_warp_specialised(4, C.byref(e)) == 0 and e.value == 1 - ws4
    finally:
        assert L.sfx_tune_set_warp_specialised(4, ws4) == 0
    assert L.sfx_set_wait_limit(0) == 0
    assert L.sfx_set_wait_limit(1 << 21) == 0  # back to the documented default


def test_plan_arguments(L, host_ctx):
    """Plan creation rejects bad form counts, right-hand-side counts,
    precisions, null pointers and a host-only context with SFX_ERR_ARG before
    touching a device; no plan is returned."""
    m = sfx.Mesh.box(host_ctx, 2, 2, 2)
    deg = (C.c_int32 * 8)(*([2] * 8))
    forms = (C.c_int * 2)(1, 0)
    out = C.c_void_p()
    create = L.sfx_plan_create_padaptive_prec
    for nforms, nrhs, prec in ((0, 1, 0), (5, 1, 0), (1, 0, 0), (1, 65, 0), (1, 1, 3), (1, 1, -1)):
        assert create(host_ctx.h, m.h, deg, nforms, forms, None, nrhs, prec, C.byref(out)) == -1
    assert create(host_ctx.h, m.h, deg, 2, forms, None, 4, 0, C.byref(out)) == -1   # host-only context
    assert create(host_ctx.h, None, deg, 2, forms, None, 4, 0, C.byref(out)) == -1
    assert create(host_ctx.h, m.h, None, 2, forms, None, 4, 0, C.byref(out)) == -1
    assert create(host_ctx.h, m.h, deg, 2, forms, None, 4, 0, None) == -1
    assert L.sfx_plan_create_padaptive(host_ctx.h, m.h, deg, 2, forms, None, 4, C.byref(out)) == -1
    assert not out.value


def test_noalloc_arguments(L, host_ctx):
    """The allocation-free p-adaptive action rejects null or aliased
    pointers, bad right-hand-side counts and a host-only context with
    SFX_ERR_ARG before any device call (fake pointers are never dereferenced
    on these paths)."""
    m = sfx.Mesh.box(host_ctx, 2, 2, 2)
    d, off, x, y = C.c_void_p(64), C.c_void_p(128), C.c_void_p(256), C.c_void_p(512)
    call = L.sfx_padaptive_action_noalloc
    assert call(None, m.h, d, off, 1, None, x, y, 1, None) == -1
    assert call(host_ctx.h, None, d, off, 1, None, x, y, 1, None) == -1
    assert call(host_ctx.h, m.h, None, off, 1, None, x, y, 1, None) == -1
    assert call(host_ctx.h, m.h, d, None, 1, None, x, y, 1, None) == -1
    assert call(host_ctx.h, m.h, d, off, 1, None, x, x, 1, None) == -1       # y aliases x
    assert call(host_ctx.h, m.h, d, off, 1, None, x, y, 0, None) == -1
    assert call(host_ctx.h, m.h, d, off, 1, None, x, y, 65, None) == -1
    assert call(host_ctx.h, m.h, d, off, 1, None, x, y, 1, None) == -1       # host-only context


def test_assembly_entry_points_reject_host_only_context(L, host_ctx):
    """Every assembly, matrix, stored-factor and CSR entry point returns
    SFX_ERR_ARG on a host-only context (no device copies exist) instead of
    launching; placeholder pointers are never dereferenced on that path."""
    m = sfx.Mesh.box(host_ctx, 2, 2, 2)
    q = sfx.Space(m, "Q", 2)
    vq = sfx.Space(m, "VQ", 2)
    csr = sfx.Csr(q)
    a, b, c = C.c_void_p(64), C.c_void_p(128), C.c_void_p(256)
    h = host_ctx.h
    out = C.c_void_p()
    calls = [
        lambda: L.sfx_assemble_cell_vectors(h, 1, None, q.h, a, 1, b, 1, c, 0, None),
        lambda: L.sfx_assemble_weighted_action(h, q.h, a, b, c, 1, 0, 0, None),
        lambda: L.sfx_assemble_weighted_cell_matrices(h, q.h, a, 0, 1, b, 0, None),
        lambda: L.sfx_assemble_linearised_action(h, 5, None, vq.h, a, b, c, 1, 0, 0, None),
        lambda: L.sfx_assemble_linearised_cell_vectors(h, 5, None, vq.h, a, b, 1, c, 1, C.c_void_p(512), 0, None),
        lambda: L.sfx_assemble_linearised_cell_matrices(h, 5, None, vq.h, a, 0, 1, b, 0, None),
        lambda: L.sfx_csr_assemble(h, 1, None, csr.h, a, None),
        lambda: L.sfx_csr_spmv(h, csr.h, a, b, c, None),
        lambda: L.sfx_qdata_create(h, q.h, 1, None, C.byref(out)),
        lambda: L.sfx_assemble_action_stored(h, 1, None, q.h, None, a, b, 1, 0, 0, None),
    ]
    for i, call in enumerate(calls):
        assert call() == -1, i
    assert not out.value
