"""Pins for the oracle's scalar forms (mass, Laplace, Helmholtz) on Q_p and DQ_p.

Sec. 1.1 (Eqs. laplace_form, laplace_quadrature, laplace_prefiat) defines the
integrals; these tests pin the oracle to facts fixed by the mathematics:
exact rational integrals on single cells (sympy), volume and moment identities,
the patch test, constants in the Laplace kernel, symmetry and rank.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

sympy = pytest.importorskip("sympy")

DIMS = (3, 2, 3)


def mesh(dims=DIMS, seed=0):
    return inputs.box_coords(*dims, perturb=0.1, seed=seed)


# ---------------------------------------------------------------- exact cells
def _lagrange_sym(nodes, i, t):
    v = sympy.Integer(1)
    for k, xk in enumerate(nodes):
        if k != i:
            v *= (t - xk) / (nodes[i] - xk)
    return sympy.expand(v)


def _integrate01(expr, syms):
    poly = expr if isinstance(expr, sympy.Poly) else sympy.Poly(sympy.expand(expr), *syms)
    tot = sympy.Integer(0)
    for mon, c in poly.terms():
        den = 1
        for e in mon:
            den *= e + 1
        tot += c / den
    return tot


def _basis(p, syms):
    nodes = {1: [0, 1], 2: [0, sympy.Rational(1, 2), 1]}[p]
    n = p + 1
    ph = [[_lagrange_sym(nodes, i, s) for i in range(n)] for s in syms]
    out = []
    for i1 in range(n):
        for i2 in range(n):
            for i3 in range(n):
                out.append(sympy.Poly(ph[0][i1] * ph[1][i2] * ph[2][i3], *syms))
    return out


def _single_cell(verts):
    """coords of a 1x1x1 'box' whose 8 vertices are given in (a,b,c) order."""
    return np.array([[float(v) for v in x] for x in verts])


AFFINE_A = [[Fraction(6, 5), Fraction(1, 5), Fraction(-1, 10)],
            [Fraction(1, 10), Fraction(9, 10), Fraction(1, 5)],
            [Fraction(-1, 5), Fraction(1, 10), Fraction(11, 10)]]
X0 = [Fraction(1, 3), Fraction(-1, 4), Fraction(1, 7)]


def _affine_verts():
    vs = []
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                vs.append([X0[i] + AFFINE_A[i][0] * a + AFFINE_A[i][1] * b + AFFINE_A[i][2] * c for i in range(3)])
    return vs


@pytest.mark.parametrize("p", [1, 2])
def test_affine_cell_exact(orc, p):
    """On a parallelepiped J = A is constant: mass and Laplace integrands are
    polynomials of degree 2p per direction, so the (p+1)-point rule is exact
    and must equal the rational integrals computed symbolically."""
    syms = sympy.symbols("x y z")
    psi = _basis(p, syms)
    A = sympy.Matrix(3, 3, lambda i, j: sympy.Rational(AFFINE_A[i][j].numerator, AFFINE_A[i][j].denominator))
    detA, Ginv = A.det(), A.inv()
    K = Ginv * Ginv.T  # G G^T with G = A^{-1}
    grads = [[f.diff(s) for s in syms] for f in psi]
    n = len(psi)
    M = np.zeros((n, n))
    L = np.zeros((n, n))
    for i in range(n):
        # K grad psi_i, as polynomials
        kg = [sum((grads[i][b] * K[a, b] for b in range(3)), sympy.Poly(0, *syms)) for a in range(3)]
        for j in range(i, n):
            M[j, i] = M[i, j] = float(detA * _integrate01(psi[i] * psi[j], syms))
            g = sum((grads[j][a] * kg[a] for a in range(3)), sympy.Poly(0, *syms))
            L[j, i] = L[i, j] = float(detA * _integrate01(g, syms))
    X = _single_cell(_affine_verts())
    Mo = orc.cell_matrices("Q", "mass", p, (1, 1, 1), X)[0]
    Lo = orc.cell_matrices("Q", "laplace", p, (1, 1, 1), X)[0]
    np.testing.assert_allclose(Mo, M, rtol=0, atol=1e-14 * np.abs(M).max())
    np.testing.assert_allclose(Lo, L, rtol=0, atol=1e-13 * np.abs(L).max())


TRILINEAR = [[0, 0, 0], [Fraction(1, 10), Fraction(-1, 10), 1], [0, 1, Fraction(1, 5)], [Fraction(-1, 5), 1, 1],
             [1, 0, 0], [Fraction(6, 5), Fraction(1, 10), Fraction(9, 10)], [Fraction(9, 10), Fraction(4, 5), 0],
             [Fraction(11, 10), Fraction(11, 10), Fraction(6, 5)]]


@pytest.mark.parametrize("p", [1, 2])
def test_trilinear_cell_mass_exact(orc, p):
    """Non-affine cell: det J has degree 2 per direction, so with p+2 Gauss
    points the mass integrand is integrated exactly."""
    syms = sympy.symbols("x y z")
    psi = _basis(p, syms)
    xmap = [sympy.Integer(0)] * 3
    for v, (a, b, c) in enumerate([(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]):
        N = (syms[0] if a else 1 - syms[0]) * (syms[1] if b else 1 - syms[1]) * (syms[2] if c else 1 - syms[2])
        for i in range(3):
            xmap[i] += sympy.Rational(Fraction(TRILINEAR[v][i]).numerator, Fraction(TRILINEAR[v][i]).denominator) * N
    J = sympy.Matrix(3, 3, lambda i, j: sympy.diff(xmap[i], syms[j]))
    S = sympy.Poly(sympy.expand(J.det()), *syms)
    n = len(psi)
    M = np.zeros((n, n))
    for j in range(n):
        for i in range(j, n):
            M[j, i] = M[i, j] = float(_integrate01(psi[i] * psi[j] * S, syms))
    X = _single_cell(TRILINEAR)
    Mo = orc.cell_matrices("Q", "mass", p, (1, 1, 1), X, nq=p + 2)[0]
    np.testing.assert_allclose(Mo, M, rtol=0, atol=1e-14 * np.abs(M).max())
    # and the cell volume is the integral of det J
    assert abs(Mo.sum() - float(_integrate01(S, syms))) < 1e-14


# ------------------------------------------------------------ mesh identities
@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_moments(orc, fam, p):
    """1^T M 1 = |Omega| = 1 (S has degree 2 per direction: exact for q >= 2);
    for Q_p also 1^T M I(x) = 1/2 and, for p >= 2, 1^T M I(x^2) = 1/3."""
    X = mesh()
    ndof, _ = orc.space_size(fam, p, DIMS)
    assert abs(orc.action(fam, "mass", p, DIMS, X, np.ones(ndof)).sum() - 1.0) < 1e-13
    if fam == "Q":
        xq = orc.q_node_coords(p, DIMS, X)
        for k in range(3):
            assert abs(orc.action(fam, "mass", p, DIMS, X, xq[:, k]).sum() - 0.5) < 1e-13
            if p >= 2:
                assert abs(orc.action(fam, "mass", p, DIMS, X, xq[:, k] ** 2).sum() - 1 / 3) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_laplace_patch_test(orc, p):
    """u = a.x lies in Q_p; grad u = a exactly at every point, and the cell
    integrals of a.grad v are exact, so (A u)_j = 0 at every interior dof
    (divergence theorem) and u^T A u = |a|^2 |Omega|.  A G/G^T mix-up, a
    dropped S or a wrong weight breaks this on a perturbed mesh."""
    X = mesh()
    a = np.array([0.3, -0.7, 1.1])
    xq = orc.q_node_coords(p, DIMS, X)
    u = xq @ a
    Au = orc.action("Q", "laplace", p, DIMS, X, u)
    M = [p * d + 1 for d in DIMS]
    I, J, K = np.unravel_index(np.arange(len(u)), M)
    interior = (I > 0) & (I < M[0] - 1) & (J > 0) & (J < M[1] - 1) & (K > 0) & (K < M[2] - 1)
    assert np.abs(Au[interior]).max() < 1e-13
    assert np.abs(Au[~interior]).max() > 1e-3  # boundary fluxes are not zero
    assert abs(u @ Au - a @ a) < 1e-13
    if p >= 2:
        u2 = xq[:, 0] ** 2  # grad = (2x, 0, 0): u^T A u = int 4 x^2 = 4/3
        assert abs(u2 @ orc.action("Q", "laplace", p, DIMS, X, u2) - 4 / 3) < 1e-13


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_cell_matrices_structure(orc, fam, p):
    X = mesh()
    M = orc.cell_matrices(fam, "mass", p, DIMS, X)
    L = orc.cell_matrices(fam, "laplace", p, DIMS, X)
    n = (p + 1) ** 3
    one = np.ones(n)
    assert np.abs(L - L.transpose(0, 2, 1)).max() <= 1e-15 * np.abs(L).max()
    assert np.abs(M - M.transpose(0, 2, 1)).max() <= 1e-15 * np.abs(M).max()
    assert np.abs(L @ one).max() < 1e-13  # constants in the kernel
    assert abs(M.sum() - 1.0) < 1e-13  # cell volumes add up to |Omega|
    for c in range(0, len(L), 5):
        ev = np.linalg.eigvalsh(L[c])
        assert ev[0] > -1e-13 and np.sum(ev > 1e-10 * ev[-1]) == n - 1  # rank n^3 - 1
        assert np.linalg.eigvalsh(M[c])[0] > 0


@pytest.mark.parametrize("fam", ["Q", "DQ"])
def test_action_equals_sum_of_cell_matrices(orc, fam):
    """The operator action equals sum_K P_K^T A^K P_K x (Sec. 1.1)."""
    p = 2
    X = mesh()
    ndof, nloc = orc.space_size(fam, p, DIMS)
    m = orc.cell_map(fam, p, DIMS)
    x = inputs.random_vector(ndof, 1, seed=5)
    for form in ("mass", "laplace", "helmholtz"):
        A = orc.cell_matrices(fam, form, p, DIMS, X)
        y = np.zeros(ndof)
        for c in range(len(m)):
            np.add.at(y, m[c], A[c] @ x[m[c]])
        y2 = orc.action(fam, form, p, DIMS, X, x)
        assert np.abs(y - y2).max() < 1e-13 * np.abs(y2).max()


def test_helmholtz_is_combination(orc):
    p, X = 2, mesh()
    ndof, _ = orc.space_size("Q", p, DIMS)
    x = inputs.random_vector(ndof, 2, seed=3)
    L = orc.action("Q", "laplace", p, DIMS, X, x)
    M = orc.action("Q", "mass", p, DIMS, X, x)
    H = orc.action("Q", "helmholtz", p, DIMS, X, x, params=(2.0, -3.0, 0, 0))
    assert np.abs(H - (2 * L - 3 * M)).max() < 1e-13 * np.abs(H).max()


def test_multiple_rhs_are_independent(orc):
    p, X = 2, mesh()
    ndof, _ = orc.space_size("Q", p, DIMS)
    x = inputs.random_vector(ndof, 3, seed=4)
    Y = orc.action("Q", "laplace", p, DIMS, X, x)
    for r in range(3):
        np.testing.assert_array_equal(Y[:, r], orc.action("Q", "laplace", p, DIMS, X, x[:, r].copy()))


@pytest.mark.parametrize("p", [5, 6, 7, 8])
def test_high_degree_identities(orc, p):
    """The degrees the benchmark runs, on the perturbed mesh.  Physical x is
    trilinear in the reference coordinates and S = det J has degree 2 per
    direction, so with (p+1) Gauss points (exact to degree 2p+1) these hold to
    rounding:
      1^T M I(x_k^p) = 1/(p+1)         (integrand degree p+2),
      (A u)_j = 0 at interior dofs and u^T A u = |a|^2 for u = a.x (patch test),
      u^T A u = p^2/(2p-1) for u = x_k^p (integrand degree 2p: a rule one
      point short, exact only to 2p-1, misses it),
    and Helmholtz = alpha Laplace + beta mass; on DQ_p 1^T M 1 = 1 and the
    Laplace action annihilates constants."""
    X = mesh()
    xq = orc.q_node_coords(p, DIMS, X)
    for k in range(3):
        assert abs(orc.action("Q", "mass", p, DIMS, X, xq[:, k] ** p).sum() - 1 / (p + 1)) < 1e-13
    a = np.array([0.3, -0.7, 1.1])
    u = xq @ a
    Au = orc.action("Q", "laplace", p, DIMS, X, u)
    M = [p * d + 1 for d in DIMS]
    I, J, K = np.unravel_index(np.arange(len(u)), M)
    interior = (I > 0) & (I < M[0] - 1) & (J > 0) & (J < M[1] - 1) & (K > 0) & (K < M[2] - 1)
    assert np.abs(Au[interior]).max() < 1e-12
    assert abs(u @ Au - a @ a) < 1e-12
    k = p % 3
    up = xq[:, k] ** p
    assert abs(up @ orc.action("Q", "laplace", p, DIMS, X, up) - p * p / (2 * p - 1)) < 1e-12
    x = inputs.random_vector(len(u), 1, seed=p)
    H = orc.action("Q", "helmholtz", p, DIMS, X, x, params=(2.0, -3.0, 0, 0))
    L = orc.action("Q", "laplace", p, DIMS, X, x)
    Mx = orc.action("Q", "mass", p, DIMS, X, x)
    assert np.abs(H - (2 * L - 3 * Mx)).max() < 1e-13 * np.abs(H).max()
    nd, _ = orc.space_size("DQ", p, DIMS)
    one = np.ones(nd)
    assert abs(orc.action("DQ", "mass", p, DIMS, X, one).sum() - 1.0) < 1e-13
    assert np.abs(orc.action("DQ", "laplace", p, DIMS, X, one)).max() < 1e-12


@pytest.mark.parametrize("p,dims", [(5, (3, 2, 3)), (8, (2, 1, 1))])
def test_cell_matrices_high_degree(orc, p, dims):
    """Element matrices at the high degrees the GPU matrix kernels are
    compared at: symmetric, constants in the Laplace kernel, cell volumes
    summing to 1, Laplace rank n^3 - 1; assembled, they reproduce the action
    and the exact energies 1^T M 1 = 1 and u^T A u = p^2/(2p-1) for u = x^p
    (integrands of degree <= 2p, exact with p+1 Gauss points)."""
    X = inputs.box_coords(*dims, perturb=0.1, seed=0)
    L = orc.cell_matrices("Q", "laplace", p, dims, X)
    M = orc.cell_matrices("Q", "mass", p, dims, X)
    n = (p + 1) ** 3
    assert np.abs(L - L.transpose(0, 2, 1)).max() <= 1e-15 * np.abs(L).max()
    assert np.abs(M - M.transpose(0, 2, 1)).max() <= 1e-15 * np.abs(M).max()
    assert np.abs(L @ np.ones(n)).max() < 1e-12
    assert abs(M.sum() - 1.0) < 1e-13
    ev = np.linalg.eigvalsh(L[0])
    assert ev[0] > -1e-13 and np.sum(ev > 1e-10 * ev[-1]) == n - 1
    ndof, _ = orc.space_size("Q", p, dims)
    m = orc.cell_map("Q", p, dims)

    def assemble(A, v):
        y = np.zeros(ndof)
        for c in range(len(m)):
            np.add.at(y, m[c], A[c] @ v[m[c]])
        return y

    x = inputs.random_vector(ndof, 1, seed=5)
    for form, A in (("laplace", L), ("mass", M)):
        y2 = orc.action("Q", form, p, dims, X, x)
        assert np.abs(assemble(A, x) - y2).max() < 1e-13 * np.abs(y2).max()
    u = orc.q_node_coords(p, dims, X)[:, 2] ** p
    assert abs(u @ assemble(L, u) - p * p / (2 * p - 1)) < 1e-12
    assert abs(np.ones(ndof) @ assemble(M, np.ones(ndof)) - 1.0) < 1e-13
