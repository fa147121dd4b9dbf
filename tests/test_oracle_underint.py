"""Pins for the oracle's collocated Gauss-Lobatto rule on Q_p ("underintegration").

With the (p+1)-point Gauss-Lobatto rule the quadrature points are the Q_p nodes
(Sec. 2.5, Eq. colocated): the basis tabulates to the identity and the
derivative tabulation takes the delta structure of the substitution in Sec. 4.1.
The rule is not exact for these forms (Sec. 4.1 says as much); the tests pin
what it still fixes:
  * mass: diagonal, entries w_i1 w_i2 w_i3 |J|(x_i); on an axis-aligned cube
    h^3 (w x w x w) with the closed-form GLL weights;
  * Laplace on an axis-aligned cube of side h:
    h (K x W x W + W x K x W + W x W x K), K the exact 1D stiffness matrix of
    the GLL Lagrange basis (sympy) and W = diag(w) -- the rule integrates the
    1D stiffness exactly (degree 2p-2 <= 2p-1);
  * perturbed cells, p >= 2: every integrand below is a polynomial of degree
    <= p+1 <= 2p-1 per direction, integrated exactly -- volume, constants in the
    kernel, the patch test and the energy |a|^2 of u = a.x; symmetry throughout.
"""
import functools

import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

sympy = pytest.importorskip("sympy")

GLL_NODES = {
    1: ["0", "1"],
    2: ["0", "1/2", "1"],
    3: ["0", "1/2 - sqrt(5)/10", "1/2 + sqrt(5)/10", "1"],
    4: ["0", "1/2 - sqrt(21)/14", "1/2", "1/2 + sqrt(21)/14", "1"],
}
GLL_WEIGHTS = {
    1: ["1/2", "1/2"],
    2: ["1/6", "2/3", "1/6"],
    3: ["1/12", "5/12", "5/12", "1/12"],
    4: ["1/20", "49/180", "16/45", "49/180", "1/20"],
}


def _w(p):
    return np.array([float(sympy.sympify(v)) for v in GLL_WEIGHTS[p]])


@functools.lru_cache(maxsize=None)
def _stiffness_1d(p):
    """K_ij = int_0^1 l_i'(t) l_j'(t) dt for the Lagrange basis on the
    closed-form GLL nodes, by exact polynomial arithmetic (numpy's power-basis
    products, derivative and antiderivative; only the node values are rounded)."""
    from numpy.polynomial import Polynomial as Poly
    nodes = [float(sympy.sympify(v)) for v in GLL_NODES[p]]
    dl = []
    for i in range(p + 1):
        others = [x for k, x in enumerate(nodes) if k != i]
        num = Poly.fromroots(others)
        dl.append((num / num(nodes[i])).deriv())
    K = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            prim = (dl[i] * dl[j]).integ()
            K[i, j] = prim(1.0) - prim(0.0)
    return K


def test_oracle_gll_rule_closed_forms(orc):
    for p in GLL_NODES:
        x, w = orc.gauss_lobatto(p + 1)
        assert np.allclose(x, [float(sympy.sympify(v)) for v in GLL_NODES[p]], atol=1e-15)
        assert np.allclose(w, _w(p), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_collocated_mass_is_diagonal(orc, p):
    # axis-aligned cube of side h = 1/2: entries h^3 w_i1 w_i2 w_i3
    dims = (2, 2, 2)
    A = orc.cell_matrices("Q", "mass", p, dims, inputs.box_coords(*dims, perturb=0.0), qrule="GLL")
    w = _w(p)
    d = np.einsum("a,b,c->abc", w, w, w).reshape(-1) * 0.125
    for c in range(A.shape[0]):
        assert np.array_equal(A[c], np.diag(np.diag(A[c])))
        assert np.allclose(np.diag(A[c]), d, rtol=1e-14, atol=0)
    # perturbed: still exactly diagonal, positive
    dims = (3, 2, 3)
    A = orc.cell_matrices("Q", "mass", p, dims, inputs.box_coords(*dims, perturb=0.1, seed=3), qrule="GLL")
    for c in range(A.shape[0]):
        assert np.array_equal(A[c], np.diag(np.diag(A[c])))
        assert (np.diag(A[c]) > 0).all()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 2])
def test_collocated_laplace_cube_kronecker(orc, p, n):
    dims = (n, n, n)
    h = 1.0 / n
    A = orc.cell_matrices("Q", "laplace", p, dims, inputs.box_coords(*dims, perturb=0.0), qrule="GLL")
    K = _stiffness_1d(p)
    W = np.diag(_w(p))
    ref = h * (np.kron(np.kron(K, W), W) + np.kron(np.kron(W, K), W) + np.kron(np.kron(W, W), K))
    # 1e-12: the power-basis polynomial products of the reference lose a few
    # digits at p = 4 (the oracle itself agrees to ~1e-15 at p <= 3)
    for c in range(A.shape[0]):
        assert np.abs(A[c] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8])
def test_collocated_perturbed_invariants(orc, p):
    dims = (3, 2, 3)
    X = inputs.box_coords(*dims, perturb=0.1, seed=0)
    M = orc.cell_matrices("Q", "mass", p, dims, X, qrule="GLL")
    assert abs(M.sum() - 1.0) < 1e-13                       # volume of [0,1]^3
    A = orc.cell_matrices("Q", "laplace", p, dims, X, qrule="GLL")
    scale = np.abs(A).max()
    for c in range(A.shape[0]):
        assert np.abs(A[c] - A[c].T).max() <= 1e-14 * scale   # symmetric
        assert np.abs(A[c].sum(axis=1)).max() <= 1e-13 * scale  # constants in the kernel
    # patch test: u = a . x is in Q_p; (A u)_j = int a . grad psi_j = 0 at interior dofs
    a = np.array([0.3, -1.1, 0.7])
    xn = orc.q_node_coords(p, dims, X)
    u = xn @ a
    y = orc.action("Q", "laplace", p, dims, X, u, qrule="GLL")
    tol = 1e-13
    interior = np.all((xn > tol) & (xn < 1 - tol), axis=1)
    assert interior.sum() > 0
    assert np.abs(y[interior]).max() <= 1e-12 * np.abs(y).max()
    assert abs(u @ y - a @ a) <= 1e-12                       # energy of a linear field


@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
def test_collocated_action_is_sum_of_cell_matrices(orc, form):
    p, dims = 3, (2, 3, 2)
    X = inputs.box_coords(*dims, perturb=0.1, seed=4)
    ndof, nloc = orc.space_size("Q", p, dims)
    x = inputs.random_vector(ndof, 1, seed=5)
    y = orc.action("Q", form, p, dims, X, x, qrule="GLL")
    A = orc.cell_matrices("Q", form, p, dims, X, qrule="GLL")
    cmap = orc.cell_map("Q", p, dims)
    ref = np.zeros(ndof)
    for c in range(A.shape[0]):
        np.add.at(ref, cmap[c], A[c] @ x[cmap[c]])
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_collocated_differs_from_gauss(orc):
    """The collocated rule under-integrates the mass form: on the unit cube its
    matrix is the lumped diagonal, not the consistent Gauss-rule matrix."""
    p, dims = 2, (1, 1, 1)
    X = inputs.box_coords(*dims, perturb=0.0)
    Ml = orc.cell_matrices("Q", "mass", p, dims, X, qrule="GLL")[0]
    Mc = orc.cell_matrices("Q", "mass", p, dims, X)[0]
    assert abs(Ml.sum() - Mc.sum()) < 1e-14   # both integrate 1 exactly
    assert np.abs(Mc - np.diag(np.diag(Mc))).max() > 1e-3
