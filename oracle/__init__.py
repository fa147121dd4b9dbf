"""Plain FP64 CPU oracle for sum-factorised hexahedral assembly.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU baseline, its reference arm and its columns of sampled
error against the oracle) may import this package; no GPU result is ever an
input here.  The library never does, and this package never imports the
library.

The C core (``oracle.c``) evaluates every integral by naive quadrature over the
tensor Gauss rule with every basis function evaluated directly (no sum
factorisation); see the header of ``oracle.c`` for the paper sections each
routine follows.  This module only marshals numpy arrays.
"""
import ctypes as C

import numpy as np

from . import build as _build

FAMILIES = {"Q": 0, "DQ": 1, "NCF": 2, "NCE": 3, "VQ": 4}
# quadrature rules: Gauss-Legendre (default) and Gauss-Lobatto-Legendre
QRULES = {"GL": 1, "GLL": 0}
FORMS = {"mass": 0, "laplace": 1, "helmholtz": 2, "ncf_mass_divdiv": 3,
         "nce_curlcurl": 4, "neohooke": 5, "svk": 6}

# default form parameters {alpha, beta, mu, lambda} by form
#   helmholtz: alpha * laplace + beta * mass with beta = -k^2, k = 1
#   ncf: alpha * mass + beta * div-div;  nce: alpha * mass + beta * curl-curl
DEFAULT_PARAMS = {
    "mass": (0.0, 1.0, 0.0, 0.0),
    "laplace": (1.0, 0.0, 0.0, 0.0),
    "helmholtz": (1.0, -1.0, 0.0, 0.0),
    "ncf_mass_divdiv": (1.0, 1.0, 0.0, 0.0),
    "nce_curlcurl": (0.0, 1.0, 0.0, 0.0),
    "neohooke": (0.0, 0.0, 1.0, 10.0),
    "svk": (0.0, 0.0, 1.0, 10.0),
}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i, i64 = C.c_double, C.c_int, C.c_int64
        P = C.c_void_p
        L.orc_gauss_legendre.argtypes = [i, P, P]
        L.orc_gauss_lobatto.argtypes = [i, P, P]
        L.orc_lagrange.argtypes = [P, i, i, d]
        L.orc_lagrange.restype = d
        L.orc_lagrange_deriv.argtypes = [P, i, i, d]
        L.orc_lagrange_deriv.restype = d
        L.orc_space_size.argtypes = [i, i, i, i, i, P, P]
        L.orc_cell_dofs.argtypes = [i, i, i, i, i, i64, P]
        L.orc_cell_map.argtypes = [i, i, i, i, i, P]
        L.orc_cell_vectors.argtypes = [i, i, i, i, P, i, i, i, P, P, i, P, i64, P, i]
        L.orc_action.argtypes = [i, i, i, i, P, i, i, i, P, P, P, i, i]
        L.orc_cell_matrices.argtypes = [i, i, i, i, P, i, i, i, P, i64, i64, P, i]
        L.orc_energy.argtypes = [i, i, i, P, i, i, i, P, P, P]
        L.orc_cell_vectors_rule.argtypes = [i, i, i, i, i, P, i, i, i, P, P, i, P, i64, P, i]
        L.orc_action_rule.argtypes = [i, i, i, i, i, P, i, i, i, P, P, P, i, i]
        L.orc_cell_matrices_rule.argtypes = [i, i, i, i, i, P, i, i, i, P, i64, i64, P, i]
        L.orc_linearised_cell_vectors.argtypes = [i, i, i, P, i, i, i, P, P, P, i, P, i64, P, i]
        L.orc_linearised_action.argtypes = [i, i, i, P, i, i, i, P, P, P, P, i, i]
        L.orc_linearised_cell_matrices.argtypes = [i, i, i, P, i, i, i, P, P, i64, i64, P, i]
        L.orc_weighted_cell_vectors.argtypes = [i, i, i, i, i, i, P, P, P, i, P, i64, P, i]
        L.orc_weighted_action.argtypes = [i, i, i, i, i, i, P, P, P, P, i, i]
        L.orc_weighted_cell_matrices.argtypes = [i, i, i, i, i, i, P, P, i64, i64, P, i]
        L.orc_q_node_coords.argtypes = [i, i, i, i, P, P]
        L.orc_interp_grad_q_to_nce.argtypes = [i, i, i, i, P, P]
        L.orc_interp_curl_nce_to_ncf.argtypes = [i, i, i, i, P, P]
        L.orc_interp_linear_field.argtypes = [i, i, i, i, i, P, P, P, P]
        L.orc_local_vectors.argtypes = [i, i, i, i, P, i64, P, P, i, P, i]
        L.orc_local_matrices.argtypes = [i, i, i, i, P, i64, P, P, i]
        L.orc_set_plant.argtypes = [i]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed (rc=%d)" % (what, rc))


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss_legendre(n, _p(x), _p(w)), "gauss_legendre")
    return x, w


def gauss_lobatto(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss_lobatto(n, _p(x), _p(w)), "gauss_lobatto")
    return x, w


def lagrange(nodes, i, x, deriv=False):
    nodes = _f64(nodes)
    f = lib().orc_lagrange_deriv if deriv else lib().orc_lagrange
    return f(_p(nodes), len(nodes), i, float(x))


def space_size(family, p, dims):
    nd, nl = C.c_int64(), C.c_int()
    _check(lib().orc_space_size(FAMILIES[family], p, *dims, C.byref(nd), C.byref(nl)), "space_size")
    return nd.value, nl.value


def cell_map(family, p, dims):
    ndof, nloc = space_size(family, p, dims)
    m = np.zeros((dims[0] * dims[1] * dims[2], nloc), dtype=np.int32)
    _check(lib().orc_cell_map(FAMILIES[family], p, *dims, _p(m)), "cell_map")
    return m


def _params(form, params):
    return _f64(DEFAULT_PARAMS[form] if params is None else params)


def action(family, form, p, dims, coords, x, nq=None, params=None, nthreads=0, qrule="GL"):
    """y = sum_K P_K^T b^K.  x: (ndof,) or (ndof, nrhs).  qrule "GLL" with the
    default nq = p + 1 is the collocated (underintegrated) rule."""
    ndof, nloc = space_size(family, p, dims)
    x = _f64(x)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    assert x.shape[0] == ndof
    y = np.zeros_like(x)
    pr = _params(form, params)
    coords = _f64(coords)
    _check(lib().orc_action_rule(FAMILIES[family], FORMS[form], p, nq or p + 1, QRULES[qrule], _p(pr), *dims,
                                 _p(coords), _p(x), _p(y), nrhs, nthreads), "action")
    return y


def cell_vectors(family, form, p, dims, coords, x, cells, nq=None, params=None, nthreads=0, qrule="GL"):
    """Per-cell local vectors b^K for the listed cells: (ncells, nloc[, nrhs])."""
    ndof, nloc = space_size(family, p, dims)
    x = _f64(x)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    b = np.zeros((len(cells), nloc, nrhs))
    pr = _params(form, params)
    coords = _f64(coords)
    _check(lib().orc_cell_vectors_rule(FAMILIES[family], FORMS[form], p, nq or p + 1, QRULES[qrule], _p(pr),
                                       *dims, _p(coords), _p(x), nrhs, _p(cells), len(cells), _p(b), nthreads),
           "cell_vectors")
    return b[:, :, 0] if x.ndim == 1 else b


def cell_matrices(family, form, p, dims, coords, cell_begin=0, cell_end=None, nq=None,
                  params=None, nthreads=0, qrule="GL"):
    """A[c, j, i], row = test j, column = trial i."""
    ndof, nloc = space_size(family, p, dims)
    ncell = dims[0] * dims[1] * dims[2]
    cell_end = ncell if cell_end is None else cell_end
    A = np.zeros((cell_end - cell_begin, nloc, nloc))
    pr = _params(form, params)
    coords = _f64(coords)
    _check(lib().orc_cell_matrices_rule(FAMILIES[family], FORMS[form], p, nq or p + 1, QRULES[qrule], _p(pr),
                                        *dims, _p(coords), cell_begin, cell_end, _p(A), nthreads), "cell_matrices")
    return A


def weighted_action(family, p, dims, coords, kappa, x, nq=None, nthreads=0):
    """y = A_kappa x for the weighted Laplace form int kappa grad u . grad v,
    kappa given by its dofs in the same space."""
    ndof, _ = space_size(family, p, dims)
    x, kappa = _f64(x), _f64(kappa)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    assert kappa.shape == (ndof,) and x.shape[0] == ndof
    y = np.zeros_like(x)
    _check(lib().orc_weighted_action(FAMILIES[family], p, nq or p + 1, *dims, _p(_f64(coords)), _p(kappa), _p(x),
                                     _p(y), nrhs, nthreads), "weighted_action")
    return y


def weighted_cell_vectors(family, p, dims, coords, kappa, x, cells, nq=None, nthreads=0):
    ndof, nloc = space_size(family, p, dims)
    x, kappa = _f64(x), _f64(kappa)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    b = np.zeros((len(cells), nloc, nrhs))
    _check(lib().orc_weighted_cell_vectors(FAMILIES[family], p, nq or p + 1, *dims, _p(_f64(coords)), _p(kappa),
                                           _p(x), nrhs, _p(cells), len(cells), _p(b), nthreads),
           "weighted_cell_vectors")
    return b[:, :, 0] if x.ndim == 1 else b


def weighted_cell_matrices(family, p, dims, coords, kappa, cell_begin=0, cell_end=None, nq=None, nthreads=0):
    ndof, nloc = space_size(family, p, dims)
    ncell = dims[0] * dims[1] * dims[2]
    cell_end = ncell if cell_end is None else cell_end
    A = np.zeros((cell_end - cell_begin, nloc, nloc))
    _check(lib().orc_weighted_cell_matrices(FAMILIES[family], p, nq or p + 1, *dims, _p(_f64(coords)),
                                            _p(_f64(kappa)), cell_begin, cell_end, _p(A), nthreads),
           "weighted_cell_matrices")
    return A


def linearised_action(form, p, dims, coords, u, du, nq=None, params=None, nthreads=0):
    """Action of the linearised hyperelastic operator at the state u on the
    direction(s) du: (ndof,) or (ndof, nrhs)."""
    ndof, _ = space_size("VQ", p, dims)
    u, du = _f64(u), _f64(du)
    nrhs = 1 if du.ndim == 1 else du.shape[1]
    assert u.shape == (ndof,) and du.shape[0] == ndof
    y = np.zeros_like(du)
    pr = _params(form, params)
    _check(lib().orc_linearised_action(FORMS[form], p, nq or p + 1, _p(pr), *dims, _p(_f64(coords)), _p(u), _p(du),
                                       _p(y), nrhs, nthreads), "linearised_action")
    return y


def linearised_cell_vectors(form, p, dims, coords, u, du, cells, nq=None, params=None, nthreads=0):
    ndof, nloc = space_size("VQ", p, dims)
    u, du = _f64(u), _f64(du)
    nrhs = 1 if du.ndim == 1 else du.shape[1]
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    b = np.zeros((len(cells), nloc, nrhs))
    pr = _params(form, params)
    _check(lib().orc_linearised_cell_vectors(FORMS[form], p, nq or p + 1, _p(pr), *dims, _p(_f64(coords)), _p(u),
                                             _p(du), nrhs, _p(cells), len(cells), _p(b), nthreads),
           "linearised_cell_vectors")
    return b[:, :, 0] if du.ndim == 1 else b


def linearised_cell_matrices(form, p, dims, coords, u, cell_begin=0, cell_end=None, nq=None, params=None,
                             nthreads=0):
    """Tangent matrices of the hyperelastic residual at the state u (Sec. 4.1),
    (cells, nloc, nloc), row = test, column = trial."""
    ndof, nloc = space_size("VQ", p, dims)
    ncell = dims[0] * dims[1] * dims[2]
    cell_end = ncell if cell_end is None else cell_end
    u = _f64(u)
    assert u.shape == (ndof,)
    A = np.zeros((cell_end - cell_begin, nloc, nloc))
    pr = _params(form, params)
    _check(lib().orc_linearised_cell_matrices(FORMS[form], p, nq or p + 1, _p(pr), *dims, _p(_f64(coords)), _p(u),
                                              cell_begin, cell_end, _p(A), nthreads), "linearised_cell_matrices")
    return A


def energy(form, p, dims, coords, x, nq=None, params=None):
    e = C.c_double()
    pr = _params(form, params)
    coords, x = _f64(coords), _f64(x)
    _check(lib().orc_energy(FORMS[form], p, nq or p + 1, _p(pr), *dims, _p(coords), _p(x),
                            C.byref(e)), "energy")
    return e.value


def q_node_coords(p, dims, coords):
    ndof, _ = space_size("Q", p, dims)
    out = np.zeros((ndof, 3))
    _check(lib().orc_q_node_coords(p, *dims, _p(_f64(coords)), _p(out)), "q_node_coords")
    return out


def interp_grad_q_to_nce(p, dims, xq):
    ndof, _ = space_size("NCE", p, dims)
    out = np.zeros(ndof)
    _check(lib().orc_interp_grad_q_to_nce(p, *dims, _p(_f64(xq)), _p(out)), "interp_grad")
    return out


def interp_curl_nce_to_ncf(p, dims, xnce):
    ndof, _ = space_size("NCF", p, dims)
    out = np.zeros(ndof)
    _check(lib().orc_interp_curl_nce_to_ncf(p, *dims, _p(_f64(xnce)), _p(out)), "interp_curl")
    return out


def interp_linear_field(family, p, dims, coords, A, b):
    """Covariant (NCE) / contravariant (NCF) interpolant of u(x) = A x + b."""
    ndof, _ = space_size(family, p, dims)
    out = np.zeros(ndof)
    _check(lib().orc_interp_linear_field(FAMILIES[family], p, *dims, _p(_f64(coords)),
                                         _p(_f64(A)), _p(_f64(b)), _p(out)), "interp_linear_field")
    return out


class planted:
    """Context manager that switches on one deliberate mistake in the oracle
    (tests only: it shows the pins catch it)."""

    def __init__(self, which):
        self.which = which

    def __enter__(self):
        lib().orc_set_plant(self.which)
        return self

    def __exit__(self, *exc):
        lib().orc_set_plant(0)
        return False


# ---------------------------------------------------------------------------
# Any hexahedral mesh.  The global numbering below is the oracle's own and is
# built differently from the library's: a node of a cell is identified by its
# position relative to the cell's corners, not by the mesh's edges and faces.

# VTK hexahedron: the reference corner of each position in a cell's vertex list
# (bottom face z = 0 counter-clockwise from the origin, then the top face).
VTK_HEX_CORNERS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]


def vtk_to_corner_order(cell_vertices):
    """(ncell, 8) VTK-ordered vertex ids -> (ncell, 8) with reference corner
    (a, b, c) at column 4a + 2b + c (the oracle's corner convention)."""
    cv = np.asarray(cell_vertices)
    out = np.empty_like(cv)
    for pos, (a, b, c) in enumerate(VTK_HEX_CORNERS):
        out[:, 4 * a + 2 * b + c] = cv[:, pos]
    return out


def general_map(family, p, corner_vertices):
    """Cell-node map of Q_p / vector Q_p / DQ_p on any conforming hexahedral
    mesh, and the number of global dofs.

    Q_p: the node with lattice index (i1, i2, i3) of a cell sits at the
    trilinear combination of the cell's corners with weights
    prod_d (i_d if a_d else p - i_d) / p^3 (the GLL nodes are symmetric, so the
    lattice index fixes the node whatever the cell's local axes).  Two cells
    share the node iff they give it the same set of (corner vertex id, integer
    weight) pairs; the dofs are the distinct sets, numbered in sorted order.
    Vector Q_p: three such blocks, component-major.  DQ_p: cell-major."""
    V = np.asarray(corner_vertices, dtype=np.int64)
    ncell, n = V.shape[0], p + 1
    if family == "DQ":
        return np.arange(ncell * n ** 3, dtype=np.int64).reshape(ncell, n ** 3), ncell * n ** 3
    if family not in ("Q", "VQ"):
        raise ValueError("general meshes: Q, VQ or DQ")
    keys = np.full((ncell, n ** 3, 16), -1, dtype=np.int64)
    l = 0
    for i1 in range(n):
        for i2 in range(n):
            for i3 in range(n):
                w = np.array([(i1 if a else p - i1) * (i2 if b else p - i2) * (i3 if c else p - i3)
                              for a in (0, 1) for b in (0, 1) for c in (0, 1)], dtype=np.int64)
                nz = np.flatnonzero(w)
                vid = V[:, nz]
                order = np.argsort(vid, axis=1)
                keys[:, l, :len(nz)] = np.take_along_axis(vid, order, axis=1)
                keys[:, l, 8:8 + len(nz)] = w[nz][order]
                l += 1
    _, inv = np.unique(keys.reshape(-1, 16), axis=0, return_inverse=True)
    m = inv.reshape(ncell, n ** 3).astype(np.int64)
    nd = int(m.max()) + 1
    if family == "VQ":
        return np.concatenate([m + c * nd for c in range(3)], axis=1), 3 * nd
    return m, nd


def _corners(xyz, corner_vertices):
    return np.ascontiguousarray(np.asarray(xyz, dtype=np.float64)[np.asarray(corner_vertices)])


def local_vectors(family, form, p, corners, xl, nq=None, params=None, nthreads=0):
    """b^K (ncells, nloc, nrhs) from the cells' corner coordinates (ncells, 8, 3)
    and local coefficients xl (ncells, nloc, nrhs)."""
    corners = _f64(corners)
    xl = _f64(xl)
    nrhs = xl.shape[2]
    b = np.zeros_like(xl)
    pr = _params(form, params)
    _check(lib().orc_local_vectors(FAMILIES[family], FORMS[form], p, nq or p + 1, _p(pr), corners.shape[0],
                                   _p(corners), _p(xl), nrhs, _p(b), nthreads), "local_vectors")
    return b


def general_action(family, form, p, xyz, cell_vertices_vtk, x, nq=None, params=None, nthreads=0):
    """y = sum_K P_K^T b^K on any hexahedral mesh, in the oracle's own
    numbering (general_map).  Returns (y, map, ndof)."""
    V = vtk_to_corner_order(cell_vertices_vtk)
    m, nd = general_map(family, p, V)
    x = _f64(x)
    x2 = x.reshape(nd, -1)
    xl = np.ascontiguousarray(x2[m])
    b = local_vectors(family, form, p, _corners(xyz, V), xl, nq=nq, params=params, nthreads=nthreads)
    y = np.zeros_like(x2)
    for c in range(m.shape[0]):  # cells in order
        y[m[c]] += b[c]
    return y.reshape(x.shape), m, nd


def general_cell_matrices(family, form, p, xyz, cell_vertices_vtk, nq=None, params=None, nthreads=0):
    """A[c, j, i] (row = test) of every cell of a mesh given by connectivity."""
    V = vtk_to_corner_order(cell_vertices_vtk)
    corners = _corners(xyz, V)
    ncell = corners.shape[0]
    nloc = general_map(family, p, V[:1])[0].shape[1]
    A = np.zeros((ncell, nloc, nloc))
    pr = _params(form, params)
    _check(lib().orc_local_matrices(FAMILIES[family], FORMS[form], p, nq or p + 1, _p(pr), ncell, _p(corners),
                                    _p(A), nthreads), "local_matrices")
    return A
