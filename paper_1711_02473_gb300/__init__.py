"""Python binding of the sfx C ABI (include/sfx.h): argument marshalling only.

Every computation runs in the CUDA library ``_build/libsfx.so``; this module
passes pointers and sizes.  Device arrays are torch CUDA tensors (float64,
int64), used for memory and streams only.  If the library has not been built
the first call raises ``RuntimeError``; there is no CPU fallback.

Function names mirror the C entry points: ``sfx_assemble_action`` etc.; the
small classes ``Context``, ``Mesh`` and ``Space`` own the C objects.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfx.so")

FAMILY = {"Q": 0, "DQ": 1, "NCF": 2, "NCE": 3, "VQ": 4}
FORM = {"mass": 0, "laplace": 1, "helmholtz": 2, "ncf_mass_divdiv": 3, "nce_curlcurl": 4,
        "neohooke": 5, "svk": 6}
NODES = {"GLL": 0, "GL": 1}
PRECISION = {"fp64": 0, "tf32x3": 1, "bf16x3": 2}
ALGO = {"sumfact": 0, "naive": 1, "collocated": 2}
DEV_INVERTED, DEV_DETF, DEV_BADCELL, DEV_TIMEOUT = 1, 2, 4, 8
STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported combination", -3: "CUDA runtime error",
          -4: "allocation failed", -5: "size exceeds 32-bit indexing"}

# every symbol include/sfx.h declares
EXPORTS = ["sfx_ctx_create", "sfx_ctx_destroy", "sfx_sync_status", "sfx_status_string",
           "sfx_mesh_create_box", "sfx_mesh_create_structured", "sfx_mesh_create", "sfx_mesh_info",
           "sfx_mesh_destroy", "sfx_space_create", "sfx_space_info", "sfx_space_colours", "sfx_space_first_touch",
           "sfx_space_destroy",
           "sfx_tabulate_1d",
           "sfx_assemble_action", "sfx_assemble_cell_vectors", "sfx_assemble_cell_matrices",
           "sfx_plan_create_padaptive", "sfx_plan_create_padaptive_prec", "sfx_plan_info", "sfx_plan_execute",
           "sfx_plan_destroy",
           "sfx_padaptive_action_noalloc", "sfx_qdata_create", "sfx_qdata_destroy",
           "sfx_assemble_action_stored", "sfx_tune_set_cells_per_cta", "sfx_tune_get_cells_per_cta",
           "sfx_tune_set_warp_specialised", "sfx_tune_get_warp_specialised", "sfx_set_wait_limit",
           "sfx_probe_launch",
           "sfx_assemble_linearised_action", "sfx_assemble_linearised_cell_vectors",
           "sfx_assemble_linearised_cell_matrices",
           "sfx_csr_create", "sfx_csr_info", "sfx_csr_assemble", "sfx_csr_spmv", "sfx_csr_destroy",
           "sfx_assemble_weighted_action", "sfx_assemble_weighted_cell_matrices"]
TUNE_KERNEL = {"fp64": 0, "mixed": 1, "mixed_stored": 2, "elastic_mixed": 3, "mixed_ws": 4, "batched": 5,
               "hdivcurl": 6, "elastic": 7, "linearised": 8, "linearised_mixed": 9, "hdivcurl_mixed": 10,
               "batched_mixed": 11}
QDATA = {"fp64": 1, "fp32": 2, "both": 3}
EXEC = {"graph": 0, "per_launch": 1}


class SfxError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, STATUS.get(code, "unknown"), code))
        self.code = code


class _Params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("mu", C.c_double), ("lam", C.c_double)]


_lib = None


def build(force=False):
    """Compile the CUDA library for sm_103a (nvcc) into _build/."""
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsfx.so is not built (%s); run paper_1711_02473_gb300.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P, i, i64, u64, d = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
        L.sfx_ctx_create.argtypes = [i, C.POINTER(P)]
        L.sfx_ctx_destroy.argtypes = [P]
        L.sfx_ctx_destroy.restype = None
        L.sfx_sync_status.argtypes = [P, P, C.POINTER(C.c_uint32)]
        L.sfx_status_string.argtypes = [i]
        L.sfx_status_string.restype = C.c_char_p
        L.sfx_mesh_create_box.argtypes = [P, i, i, i, d, u64, C.POINTER(P)]
        L.sfx_mesh_create_structured.argtypes = [P, i, i, i, P, C.POINTER(P)]
        L.sfx_mesh_create.argtypes = [P, i64, P, i64, P, C.POINTER(P)]
        L.sfx_mesh_info.argtypes = [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(P)]
        L.sfx_space_colours.argtypes = [P, C.POINTER(i), C.POINTER(P), C.POINTER(P)]
        L.sfx_space_first_touch.argtypes = [P, C.POINTER(i), C.POINTER(P)]
        L.sfx_mesh_destroy.argtypes = [P]
        L.sfx_mesh_destroy.restype = None
        L.sfx_space_create.argtypes = [P, i, i, C.POINTER(P)]
        L.sfx_space_info.argtypes = [P, C.POINTER(i64), C.POINTER(i), C.POINTER(i64), C.POINTER(P)]
        L.sfx_space_destroy.argtypes = [P]
        L.sfx_space_destroy.restype = None
        L.sfx_tabulate_1d.argtypes = [i, i, i, i, i, P, P, P]
        L.sfx_assemble_action.argtypes = [P, i, C.POINTER(_Params), P, P, P, i, i, i, i, P]
        L.sfx_assemble_linearised_action.argtypes = [P, i, C.POINTER(_Params), P, P, P, P, i, i, i, P]
        L.sfx_csr_create.argtypes = [P, C.POINTER(P)]
        L.sfx_assemble_weighted_action.argtypes = [P, P, P, P, P, i, i, i, P]
        L.sfx_assemble_weighted_cell_matrices.argtypes = [P, P, P, i64, i64, P, i, P]
        L.sfx_csr_info.argtypes = [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(P), C.POINTER(P)]
        L.sfx_csr_assemble.argtypes = [P, i, C.POINTER(_Params), P, P, P]
        L.sfx_csr_spmv.argtypes = [P, P, P, P, P, P]
        L.sfx_csr_destroy.argtypes = [P]
        L.sfx_csr_destroy.restype = None
        L.sfx_assemble_linearised_cell_vectors.argtypes = [P, i, C.POINTER(_Params), P, P, P, i, P, i64, P, i, P]
        L.sfx_assemble_linearised_cell_matrices.argtypes = [P, i, C.POINTER(_Params), P, P, i64, i64, P, i, P]
        L.sfx_assemble_cell_vectors.argtypes = [P, i, C.POINTER(_Params), P, P, i, P, i64, P, i, P]
        L.sfx_assemble_cell_matrices.argtypes = [P, i, C.POINTER(_Params), P, i64, i64, P, i, i, P]
        L.sfx_plan_create_padaptive.argtypes = [P, P, P, i, P, P, i, C.POINTER(P)]
        L.sfx_plan_create_padaptive_prec.argtypes = [P, P, P, i, P, P, i, i, C.POINTER(P)]
        L.sfx_plan_info.argtypes = [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(P)]
        L.sfx_plan_execute.argtypes = [P, P, P, i, P]
        L.sfx_plan_destroy.argtypes = [P]
        L.sfx_plan_destroy.restype = None
        L.sfx_qdata_create.argtypes = [P, P, i, P, C.POINTER(P)]
        L.sfx_qdata_destroy.argtypes = [P]
        L.sfx_qdata_destroy.restype = None
        L.sfx_assemble_action_stored.argtypes = [P, i, C.POINTER(_Params), P, P, P, P, i, i, i, P]
        L.sfx_tune_set_cells_per_cta.argtypes = [i, i, i]
        L.sfx_tune_get_cells_per_cta.argtypes = [i, i, C.POINTER(i)]
        L.sfx_tune_set_warp_specialised.argtypes = [i, i]
        L.sfx_tune_get_warp_specialised.argtypes = [i, C.POINTER(i)]
        L.sfx_set_wait_limit.argtypes = [C.c_uint32]
        L.sfx_probe_launch.argtypes = [i, i, i, i, P, P, C.POINTER(d)]
        L.sfx_padaptive_action_noalloc.argtypes = [P, P, P, P, i, C.POINTER(_Params), P, P, i, P]
        for name in EXPORTS:
            f = getattr(L, name)
            if f.restype is C.c_int:
                f.restype = C.c_int32
        _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        raise SfxError(rc, what)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, dtype_name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError("expected %s, got %s" % (dtype_name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _params(params):
    if params is None:
        return None
    a = tuple(params) + (0.0,) * (4 - len(params))
    return C.byref(_Params(*a))


class Context:
    def __init__(self, device=0):
        self.h = C.c_void_p()
        _check(lib().sfx_ctx_create(device, C.byref(self.h)), "sfx_ctx_create")

    def sync_status(self, stream=None):
        bits = C.c_uint32()
        _check(lib().sfx_sync_status(self.h, _stream(stream), C.byref(bits)), "sfx_sync_status")
        return bits.value

    def close(self):
        if self.h:
            lib().sfx_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx, h, dims):
        self.ctx, self.h, self.dims = ctx, h, (tuple(dims) if dims is not None else None)
        nv, nc, p = C.c_int64(), C.c_int64(), C.c_void_p()
        _check(lib().sfx_mesh_info(self.h, C.byref(nv), C.byref(nc), C.byref(p)), "sfx_mesh_info")
        self.nvert, self.ncell = nv.value, nc.value

    @classmethod
    def box(cls, ctx, nx, ny, nz, perturb=0.1, seed=0):
        h = C.c_void_p()
        _check(lib().sfx_mesh_create_box(ctx.h, nx, ny, nz, perturb, seed, C.byref(h)), "sfx_mesh_create_box")
        return cls(ctx, h, (nx, ny, nz))

    @classmethod
    def structured(cls, ctx, nx, ny, nz, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        if xyz.shape != ((nx + 1) * (ny + 1) * (nz + 1), 3):
            raise ValueError("xyz must be (nvert, 3)")
        h = C.c_void_p()
        _check(lib().sfx_mesh_create_structured(ctx.h, nx, ny, nz, xyz.ctypes.data_as(C.c_void_p), C.byref(h)),
               "sfx_mesh_create_structured")
        return cls(ctx, h, (nx, ny, nz))

    @classmethod
    def general(cls, ctx, xyz, cell_vertices):
        """Any hexahedral connectivity: xyz (nvert, 3), cell_vertices (ncell,
        8) in VTK hexahedron order."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        cv = np.ascontiguousarray(cell_vertices, dtype=np.int32)
        if xyz.ndim != 2 or xyz.shape[1] != 3 or cv.ndim != 2 or cv.shape[1] != 8:
            raise ValueError("xyz must be (nvert, 3) and cell_vertices (ncell, 8)")
        h = C.c_void_p()
        _check(lib().sfx_mesh_create(ctx.h, xyz.shape[0], xyz.ctypes.data_as(C.c_void_p), cv.shape[0],
                                     cv.ctypes.data_as(C.c_void_p), C.byref(h)), "sfx_mesh_create")
        return cls(ctx, h, None)

    def coords(self):
        nv, nc, p = C.c_int64(), C.c_int64(), C.c_void_p()
        _check(lib().sfx_mesh_info(self.h, C.byref(nv), C.byref(nc), C.byref(p)), "sfx_mesh_info")
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(C.c_double)), shape=(nv.value, 3)).copy()

    def close(self):
        if self.h:
            lib().sfx_mesh_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Space:
    def __init__(self, mesh, family, degree):
        self.mesh, self.family, self.p = mesh, family, degree
        self.h = C.c_void_p()
        _check(lib().sfx_space_create(mesh.h, FAMILY[family], degree, C.byref(self.h)), "sfx_space_create")
        nd, nl, nc, mp = C.c_int64(), C.c_int(), C.c_int64(), C.c_void_p()
        _check(lib().sfx_space_info(self.h, C.byref(nd), C.byref(nl), C.byref(nc), C.byref(mp)), "sfx_space_info")
        self.ndof, self.nloc, self.ncell = nd.value, nl.value, nc.value
        self._map = mp

    def cell_map(self):
        return np.ctypeslib.as_array(C.cast(self._map, C.POINTER(C.c_int32)), shape=(self.ncell, self.nloc)).copy()

    def colours(self):
        """(colour_off int64 (ncolour+1,), cells int32 (ncell,)): host copies."""
        nc, off, cl = C.c_int(), C.c_void_p(), C.c_void_p()
        _check(lib().sfx_space_colours(self.h, C.byref(nc), C.byref(off), C.byref(cl)), "sfx_space_colours")
        o = np.ctypeslib.as_array(C.cast(off, C.POINTER(C.c_int64)), shape=(nc.value + 1,)).copy()
        c = np.ctypeslib.as_array(C.cast(cl, C.POINTER(C.c_int32)), shape=(self.ncell,)).copy()
        return o, c

    def first_touch(self):
        """Host copy of the first-touch bits, uint32 (ncell, words), or None
        for families other than scalar Q_p."""
        w, bits = C.c_int(), C.c_void_p()
        _check(lib().sfx_space_first_touch(self.h, C.byref(w), C.byref(bits)), "sfx_space_first_touch")
        if w.value == 0:
            return None
        return np.ctypeslib.as_array(C.cast(bits, C.POINTER(C.c_uint32)), shape=(self.ncell, w.value)).copy()

    def close(self):
        if self.h:
            lib().sfx_space_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Csr:
    """Global sparse matrix pattern (CSR) of a Q_p / DQ_p space; values are
    caller-owned device arrays of nnz doubles (sfx_csr_assemble fills them)."""

    def __init__(self, space):
        self.space = space
        self.h = C.c_void_p()
        _check(lib().sfx_csr_create(space.h, C.byref(self.h)), "sfx_csr_create")
        nr, nz, rp, cl = C.c_int64(), C.c_int64(), C.c_void_p(), C.c_void_p()
        _check(lib().sfx_csr_info(self.h, C.byref(nr), C.byref(nz), C.byref(rp), C.byref(cl)), "sfx_csr_info")
        self.nrows, self.nnz = nr.value, nz.value
        self._rp, self._col = rp, cl

    def pattern(self):
        """Host copies (row_ptr int64, col int32)."""
        rp = np.ctypeslib.as_array(C.cast(self._rp, C.POINTER(C.c_int64)), shape=(self.nrows + 1,)).copy()
        col = np.ctypeslib.as_array(C.cast(self._col, C.POINTER(C.c_int32)), shape=(self.nnz,)).copy()
        return rp, col

    def close(self):
        if self.h:
            lib().sfx_csr_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfx_csr_assemble(ctx, form, csr, values, params=None, stream=None):
    if values.numel() != csr.nnz:
        raise ValueError("values must hold nnz doubles")
    _check(lib().sfx_csr_assemble(ctx.h, FORM[form], _params(params), csr.h, _dptr(values, "float64"),
                                  _stream(stream)), "sfx_csr_assemble")
    return values


def sfx_csr_spmv(ctx, csr, values, x, y, stream=None):
    if values.numel() != csr.nnz or x.numel() != csr.nrows or y.numel() != csr.nrows:
        raise ValueError("values: nnz doubles; x, y: nrows doubles")
    _check(lib().sfx_csr_spmv(ctx.h, csr.h, _dptr(values, "float64"), _dptr(x, "float64"), _dptr(y, "float64"),
                              _stream(stream)), "sfx_csr_spmv")
    return y


def sfx_tabulate_1d(nodes, ndof1d, qrule, nq, deriv=0):
    pts, wts, tab = np.zeros(nq), np.zeros(nq), np.zeros((nq, ndof1d))
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib().sfx_tabulate_1d(NODES[nodes], ndof1d, NODES[qrule], nq, deriv, P(pts), P(wts), P(tab)),
           "sfx_tabulate_1d")
    return pts, wts, tab


def sfx_assemble_action(ctx, form, space, x, y, nrhs=None, accumulate=False, precision="fp64",
                        algo="sumfact", params=None, stream=None):
    nrhs = nrhs if nrhs is not None else (1 if x.dim() == 1 else x.shape[1])
    if x.numel() != space.ndof * nrhs or y.numel() != space.ndof * nrhs:
        raise ValueError("x and y must hold ndof * nrhs doubles")
    _check(lib().sfx_assemble_action(ctx.h, FORM[form], _params(params), space.h, _dptr(x, "float64"),
                                     _dptr(y, "float64"), nrhs, int(bool(accumulate)), PRECISION[precision],
                                     ALGO[algo], _stream(stream)), "sfx_assemble_action")
    return y


def sfx_assemble_weighted_action(ctx, space, kappa, x, y, nrhs=None, accumulate=False, precision="fp64",
                                 stream=None):
    nrhs = nrhs if nrhs is not None else (1 if x.dim() == 1 else x.shape[1])
    if kappa.numel() != space.ndof or x.numel() != space.ndof * nrhs or y.numel() != space.ndof * nrhs:
        raise ValueError("kappa must hold ndof doubles; x and y ndof * nrhs")
    _check(lib().sfx_assemble_weighted_action(ctx.h, space.h, _dptr(kappa, "float64"), _dptr(x, "float64"),
                                              _dptr(y, "float64"), nrhs, int(bool(accumulate)),
                                              PRECISION[precision], _stream(stream)), "sfx_assemble_weighted_action")
    return y


def sfx_assemble_weighted_cell_matrices(ctx, space, kappa, cell_begin, cell_end, A, precision="fp64", stream=None):
    if A.numel() != (cell_end - cell_begin) * space.nloc * space.nloc or kappa.numel() != space.ndof:
        raise ValueError("A must hold ncells * nloc * nloc doubles, kappa ndof")
    _check(lib().sfx_assemble_weighted_cell_matrices(ctx.h, space.h, _dptr(kappa, "float64"), cell_begin, cell_end,
                                                     _dptr(A, "float64"), PRECISION[precision], _stream(stream)),
           "sfx_assemble_weighted_cell_matrices")
    return A


def sfx_assemble_linearised_action(ctx, form, space, u, du, y, nrhs=None, accumulate=False, precision="fp64",
                                   params=None, stream=None):
    nrhs = nrhs if nrhs is not None else (1 if du.dim() == 1 else du.shape[1])
    if u.numel() != space.ndof or du.numel() != space.ndof * nrhs or y.numel() != space.ndof * nrhs:
        raise ValueError("u must hold ndof doubles; du and y ndof * nrhs")
    _check(lib().sfx_assemble_linearised_action(ctx.h, FORM[form], _params(params), space.h, _dptr(u, "float64"),
                                                _dptr(du, "float64"), _dptr(y, "float64"), nrhs,
                                                int(bool(accumulate)), PRECISION[precision], _stream(stream)),
           "sfx_assemble_linearised_action")
    return y


def sfx_assemble_linearised_cell_vectors(ctx, form, space, u, du, cells, b, nrhs=None, precision="fp64",
                                         params=None, stream=None):
    nrhs = nrhs if nrhs is not None else (1 if du.dim() == 1 else du.shape[1])
    if b.numel() != cells.numel() * space.nloc * nrhs:
        raise ValueError("b must hold ncells * nloc * nrhs doubles")
    _check(lib().sfx_assemble_linearised_cell_vectors(ctx.h, FORM[form], _params(params), space.h,
                                                      _dptr(u, "float64"), _dptr(du, "float64"), nrhs,
                                                      _dptr(cells, "int64"), cells.numel(), _dptr(b, "float64"),
                                                      PRECISION[precision], _stream(stream)),
           "sfx_assemble_linearised_cell_vectors")
    return b


def sfx_assemble_linearised_cell_matrices(ctx, form, space, u, cell_begin, cell_end, A, precision="fp64",
                                          params=None, stream=None):
    if A.numel() != (cell_end - cell_begin) * space.nloc * space.nloc:
        raise ValueError("A must hold (cell_end - cell_begin) * nloc * nloc doubles")
    _check(lib().sfx_assemble_linearised_cell_matrices(ctx.h, FORM[form], _params(params), space.h,
                                                       _dptr(u, "float64"), cell_begin, cell_end,
                                                       _dptr(A, "float64"), PRECISION[precision], _stream(stream)),
           "sfx_assemble_linearised_cell_matrices")
    return A


def sfx_assemble_cell_vectors(ctx, form, space, x, cells, b, nrhs=None, precision="fp64", params=None,
                              stream=None):
    nrhs = nrhs if nrhs is not None else (1 if x.dim() == 1 else x.shape[1])
    if b.numel() != cells.numel() * space.nloc * nrhs:
        raise ValueError("b must hold ncells * nloc * nrhs doubles")
    _check(lib().sfx_assemble_cell_vectors(ctx.h, FORM[form], _params(params), space.h, _dptr(x, "float64"), nrhs,
                                           _dptr(cells, "int64"), cells.numel(), _dptr(b, "float64"),
                                           PRECISION[precision], _stream(stream)), "sfx_assemble_cell_vectors")
    return b


def sfx_assemble_cell_matrices(ctx, form, space, cell_begin, cell_end, A, precision="fp64", algo="sumfact",
                               params=None, stream=None):
    if A.numel() != (cell_end - cell_begin) * space.nloc * space.nloc:
        raise ValueError("A must hold ncells * nloc * nloc doubles")
    _check(lib().sfx_assemble_cell_matrices(ctx.h, FORM[form], _params(params), space.h, cell_begin, cell_end,
                                            _dptr(A, "float64"), PRECISION[precision], ALGO[algo],
                                            _stream(stream)), "sfx_assemble_cell_matrices")
    return A


def sfx_tune_set_cells_per_cta(kernel, degree, cells):
    _check(lib().sfx_tune_set_cells_per_cta(TUNE_KERNEL[kernel], degree, cells), "sfx_tune_set_cells_per_cta")


def sfx_tune_get_cells_per_cta(kernel, degree):
    v = C.c_int()
    _check(lib().sfx_tune_get_cells_per_cta(TUNE_KERNEL[kernel], degree, C.byref(v)), "sfx_tune_get_cells_per_cta")
    return v.value


def sfx_tune_set_warp_specialised(degree, enable):
    _check(lib().sfx_tune_set_warp_specialised(degree, int(bool(enable))), "sfx_tune_set_warp_specialised")


def sfx_tune_get_warp_specialised(degree):
    v = C.c_int()
    _check(lib().sfx_tune_get_warp_specialised(degree, C.byref(v)), "sfx_tune_get_warp_specialised")
    return bool(v.value)


def sfx_set_wait_limit(polls):
    _check(lib().sfx_set_wait_limit(int(polls)), "sfx_set_wait_limit")


PROBE = {"dfma": 0, "ffma": 1, "mma_tf32": 2, "mma_bf16": 3, "dmma": 4}


def sfx_probe_launch(kind, blocks, threads, iters, sink, stream=None):
    """One probe launch (see include/sfx.h); returns the operations it does."""
    if sink.numel() < blocks * threads:
        raise ValueError("sink must hold blocks * threads doubles")
    ops = C.c_double()
    _check(lib().sfx_probe_launch(PROBE[kind], blocks, threads, iters, _dptr(sink, "float64"), _stream(stream),
                                  C.byref(ops)), "sfx_probe_launch")
    return ops.value


class QData:
    """Stored geometric factors of a Q_p / DQ_p space (sfx_qdata_*)."""

    def __init__(self, ctx, space, formats="both", stream=None):
        self.space = space
        self.h = C.c_void_p()
        _check(lib().sfx_qdata_create(ctx.h, space.h, QDATA[formats], _stream(stream), C.byref(self.h)),
               "sfx_qdata_create")

    def close(self):
        if self.h:
            lib().sfx_qdata_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfx_assemble_action_stored(ctx, form, space, qdata, x, y, nrhs=None, accumulate=False, precision="fp64",
                               params=None, stream=None):
    nrhs = nrhs if nrhs is not None else (1 if x.dim() == 1 else x.shape[1])
    if x.numel() != space.ndof * nrhs or y.numel() != space.ndof * nrhs:
        raise ValueError("x and y must hold ndof * nrhs doubles")
    _check(lib().sfx_assemble_action_stored(ctx.h, FORM[form], _params(params), space.h, qdata.h,
                                            _dptr(x, "float64"), _dptr(y, "float64"), nrhs, int(bool(accumulate)),
                                            PRECISION[precision], _stream(stream)), "sfx_assemble_action_stored")
    return y


def sfx_padaptive_action_noalloc(ctx, mesh, degree, cell_offset, form, x, y, nrhs=1, params=None, stream=None):
    """p-adaptive DQ action that allocates nothing (see include/sfx.h): for
    callers that cannot allocate device memory at the point of the call.
    degree: int32 CUDA tensor (ncell); cell_offset: int64 CUDA tensor (ncell+1).
    The lengths are checked here; reading ndof = cell_offset[-1] waits for the
    stream."""
    ncell = mesh.ncell
    if degree.numel() != ncell or cell_offset.numel() != ncell + 1:
        raise ValueError("degree must hold ncell int32, cell_offset ncell + 1 int64")
    ndof = int(cell_offset[-1].item())
    if x.numel() != ndof * nrhs or y.numel() != ndof * nrhs:
        raise ValueError("x and y must hold cell_offset[-1] * nrhs doubles")
    _check(lib().sfx_padaptive_action_noalloc(ctx.h, mesh.h, _dptr(degree, "int32"), _dptr(cell_offset, "int64"),
                                              FORM[form], _params(params), _dptr(x, "float64"),
                                              _dptr(y, "float64"), nrhs, _stream(stream)),
           "sfx_padaptive_action_noalloc")
    return y


class Plan:
    """Batched actions on a p-adaptive DQ mesh (sfx_plan_*): one persistent,
    graph-captured launch for all forms and right-hand sides; precision "fp64"
    or a split precision ("tf32x3", "bf16x3") for the tile body."""

    def __init__(self, ctx, mesh, degree, forms, nrhs=1, params=None, precision="fp64"):
        degree = np.ascontiguousarray(degree, dtype=np.int32)
        self.ctx, self.mesh, self.forms, self.nrhs = ctx, mesh, list(forms), nrhs
        self.precision = precision
        fa = (C.c_int * len(forms))(*[FORM[f] for f in forms])
        pa = None
        if params is not None:
            arr = (_Params * len(forms))(*[_Params(*(tuple(p) + (0.0,) * (4 - len(p)))) for p in params])
            pa = C.cast(arr, C.c_void_p)
        self.h = C.c_void_p()
        _check(lib().sfx_plan_create_padaptive_prec(ctx.h, mesh.h, degree.ctypes.data_as(C.c_void_p), len(forms),
                                                    C.cast(fa, C.c_void_p), pa, nrhs, PRECISION[precision],
                                                    C.byref(self.h)),
               "sfx_plan_create_padaptive_prec")
        nd, nt, off = C.c_int64(), C.c_int64(), C.c_void_p()
        _check(lib().sfx_plan_info(self.h, C.byref(nd), C.byref(nt), C.byref(off)), "sfx_plan_info")
        self.ndof, self.ntiles = nd.value, nt.value
        self.cell_offset = np.ctypeslib.as_array(C.cast(off, C.POINTER(C.c_int64)), shape=(len(degree) + 1,)).copy()

    def execute(self, x, ys, mode="graph", stream=None):
        if len(ys) != len(self.forms):
            raise ValueError("one output per form")
        for t in [x] + list(ys):
            if t.numel() != self.ndof * self.nrhs:
                raise ValueError("vectors must hold ndof * nrhs doubles")
        yp = (C.c_void_p * len(ys))(*[_dptr(y, "float64").value for y in ys])
        _check(lib().sfx_plan_execute(self.h, _dptr(x, "float64"), C.cast(yp, C.c_void_p), EXEC[mode],
                                      _stream(stream)), "sfx_plan_execute")
        return ys

    def close(self):
        if self.h:
            lib().sfx_plan_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
