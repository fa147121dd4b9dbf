"""Seeded synthetic inputs: perturbed box meshes, input vectors, degree maps.

This module holds none of the assembly arithmetic.  It is the one module both
the CUDA path's tests/benchmark and the oracle-side tests draw inputs from.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based stream:
draw k (k = 0, 1, ...) of stream ``seed`` is mix(seed + (k + 1) * GAMMA) with
GAMMA = 0x9E3779B97F4A7C15 and the finaliser below, and the uniform variate is
(z >> 11) * 2^-53 in [0, 1).  The library's ``sfx_mesh_create_box`` implements
the same definition in C++, so both produce bit-identical vertex coordinates.

Conventions:
  * vertices of an nx*ny*nz box on [0,1]^3 are numbered (I, J, K) with K
    fastest: v = (I*(ny+1) + J)*(nz+1) + K;
  * each interior vertex is moved by perturb*h_d*(2u-1) along each axis d
    (three draws per interior vertex, x then y then z, interior vertices in
    vertex order); boundary vertices stay put, so the domain is exactly [0,1]^3;
  * input vectors take one draw per entry in (dof, rhs) order, rhs fastest,
    mapped to uniform[-1, 1).
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    z = splitmix64(seed, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def box_coords(nx: int, ny: int, nz: int, perturb: float = 0.1, seed: int = 0) -> np.ndarray:
    """Vertex coordinates ((nx+1)(ny+1)(nz+1), 3) of the perturbed unit box."""
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    xyz = np.stack([I / nx, J / ny, K / nz], axis=-1).reshape(-1, 3).astype(np.float64)
    if perturb != 0.0:
        interior = ((I > 0) & (I < nx) & (J > 0) & (J < ny) & (K > 0) & (K < nz)).reshape(-1)
        m = int(interior.sum())
        u = uniform01(seed, 3 * m).reshape(m, 3)
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        xyz[interior] += perturb * h * (2.0 * u - 1.0)
    return xyz


def random_vector(ndof: int, nrhs: int = 1, seed: int = 1, lo: float = -1.0, hi: float = 1.0):
    """uniform[lo, hi) entries, (ndof,) for nrhs == 1 else (ndof, nrhs), rhs fastest.
    Generated in chunks so that large vectors need no full-size temporaries."""
    n = ndof * nrhs
    v = np.empty(n, dtype=np.float64)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        v[s:s + c] = lo + (hi - lo) * uniform01(seed, c, start=s)
    return v if nrhs == 1 else v.reshape(ndof, nrhs)


def displacement(ndof: int, p: int, n_cells_axis: int, seed: int = 1, amplitude: float = 0.05):
    """Nodal displacement for the hyperelastic residual: amplitude*(h/p)*U[-1,1)
    per entry (h = 1/n_cells_axis), which keeps |grad u| small so det F > 0."""
    return random_vector(ndof, 1, seed) * (amplitude / (n_cells_axis * p))


def padaptive_degrees(ncell: int, pmax: int = 8, seed: int = 2) -> np.ndarray:
    """Per-cell degree p in 1..pmax, i.i.d. with P(p) proportional to 1/p,
    drawn by inverse CDF from the stream ``seed`` (int32 array)."""
    w = 1.0 / np.arange(1, pmax + 1)
    cdf = np.cumsum(w) / w.sum()
    u = uniform01(seed, ncell)
    return (np.searchsorted(cdf, u, side="right") + 1).clip(1, pmax).astype(np.int32)
