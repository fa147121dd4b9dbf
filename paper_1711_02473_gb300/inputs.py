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


# --------------------------------------------------------------------------
# General hexahedral meshes (given by connectivity), for the general-mesh path.
# Cells are listed in VTK hexahedron order: the corners (0,0,0) (1,0,0) (1,1,0)
# (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1) of the reference cell.

VTK_CORNERS = ((0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1))


def cube_rotations():
    """The 24 proper rotations of the cube [0,1]^3 as 3x3 signed permutation
    matrices M (det M = +1), acting on corners by x -> (M (2x - 1) + 1) / 2."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3), dtype=np.int64)
            for i in range(3):
                M[i, perm[i]] = signs[i]
            if round(np.linalg.det(M)) == 1:
                out.append(M)
    return out


def shuffled_box(nx, ny, nz, perturb=0.1, seed=0, shuffle_seed=9):
    """The perturbed box of box_coords, presented as a general mesh: vertex ids
    permuted, cells in a shuffled order, and each cell's vertex list rotated by
    one of the 24 proper rotations of the reference cube (so that neighbouring
    cells see shared edges and faces in different local orientations).
    Returns (xyz, cells_vtk, vnew, cell_of, rot): vnew[v] = new id of box vertex
    v; new cell k is box cell cell_of[k], whose local corner x sits at box
    corner (M (2x - 1) + 1) / 2 with M = cube_rotations()[rot[k]]."""
    X = box_coords(nx, ny, nz, perturb, seed)
    nv, ncell = X.shape[0], nx * ny * nz
    vnew = np.argsort(np.argsort(uniform01(shuffle_seed, nv)))
    cell_of = np.argsort(uniform01(shuffle_seed + 1, ncell))
    rots = cube_rotations()
    rot = np.minimum((uniform01(shuffle_seed + 2, ncell) * len(rots)).astype(np.int64), len(rots) - 1)
    xyz = np.empty_like(X)
    xyz[vnew] = X
    cells = np.empty((ncell, 8), dtype=np.int32)
    for k in range(ncell):
        c = int(cell_of[k])
        i, j, l = c // (ny * nz), (c // nz) % ny, c % nz
        M = rots[rot[k]]
        for pos, x in enumerate(VTK_CORNERS):
            a, b, cc = ((M @ (2 * np.array(x) - 1)) + 1) // 2
            v = ((i + a) * (ny + 1) + (j + b)) * (nz + 1) + (l + cc)
            cells[k, pos] = vnew[v]
    return xyz, cells, vnew, cell_of, rot


def prism_mesh(m=2, nz=2, perturb=0.1, seed=3):
    """An unstructured hexahedral mesh of the triangular prism T x [0,1],
    T = triangle (0,0), (1,0), (0.5,0.8): T is cut into three quadrilaterals
    through its centroid and edge midpoints, each split into m x m bilinear
    sub-quadrilaterals, and the result is extruded in nz layers.  The edges
    through the centroid are shared by three cells per layer (a valence no
    logically Cartesian mesh has).  Vertices strictly inside the prism move by
    perturb * h * (2u - 1) per axis (h = 1/(2m) in the plane, 1/nz along z).
    Returns (xyz, cells_vtk, volume) with volume = area(T) exactly."""
    A, B, Cc = np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.5, 0.8])
    O = (A + B + Cc) / 3.0
    mab, mbc, mca = (A + B) / 2, (B + Cc) / 2, (Cc + A) / 2
    quads = [(A, mab, O, mca), (B, mbc, O, mab), (Cc, mca, O, mbc)]
    pts, key, quads2d = [], {}, []

    def pid(pt):
        k = (round(pt[0], 12), round(pt[1], 12))
        if k not in key:
            key[k] = len(pts)
            pts.append(pt)
        return key[k]

    for q in quads:
        q = [np.asarray(v) for v in q]
        area2 = sum(q[i][0] * q[(i + 1) % 4][1] - q[(i + 1) % 4][0] * q[i][1] for i in range(4))
        if area2 < 0:
            q = q[::-1]
        g = {}
        for s in range(m + 1):
            for t in range(m + 1):
                u, w = s / m, t / m
                g[s, t] = pid((1 - u) * (1 - w) * q[0] + u * (1 - w) * q[1] + u * w * q[2] + (1 - u) * w * q[3])
        for s in range(m):
            for t in range(m):
                quads2d.append((g[s, t], g[s + 1, t], g[s + 1, t + 1], g[s, t + 1]))
    P = np.array(pts)
    n2 = len(P)

    def on_boundary(pt):
        for a, b in ((A, B), (B, Cc), (Cc, A)):
            d = b - a
            cr = d[0] * (pt[1] - a[1]) - d[1] * (pt[0] - a[0])
            if abs(cr) < 1e-12:
                return True
        return False

    xyz = np.zeros((n2 * (nz + 1), 3))
    for k in range(nz + 1):
        xyz[k * n2:(k + 1) * n2, :2] = P
        xyz[k * n2:(k + 1) * n2, 2] = k / nz
    interior = np.array([(0 < k < nz) and not on_boundary(P[i]) for k in range(nz + 1) for i in range(n2)])
    if perturb != 0.0:
        u = uniform01(seed, 3 * int(interior.sum())).reshape(-1, 3)
        h = np.array([0.5 / m, 0.5 / m, 1.0 / nz])
        xyz[interior] += perturb * h * (2.0 * u - 1.0)
    cells = []
    for k in range(nz):
        for (a, b, c, d) in quads2d:
            cells.append([a + k * n2, b + k * n2, c + k * n2, d + k * n2,
                          a + (k + 1) * n2, b + (k + 1) * n2, c + (k + 1) * n2, d + (k + 1) * n2])
    area = 0.5 * abs((B - A)[0] * (Cc - A)[1] - (B - A)[1] * (Cc - A)[0])
    return xyz, np.array(cells, dtype=np.int32), area
