"""The pins catch plausible mistakes: each test switches on one deliberate
error inside the oracle (on the CPU) and checks that a pin from the other
oracle test files now fails, then that it passes again once switched off."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

D = (3, 2, 3)


def patch_ok(orc):
    p, X = 2, inputs.box_coords(*D, perturb=0.1, seed=0)
    a = np.array([0.3, -0.7, 1.1])
    u = orc.q_node_coords(p, D, X) @ a
    Au = orc.action("Q", "laplace", p, D, X, u)
    M = [p * d + 1 for d in D]
    I, J, K = np.unravel_index(np.arange(len(u)), M)
    inner = (I > 0) & (I < M[0] - 1) & (J > 0) & (J < M[1] - 1) & (K > 0) & (K < M[2] - 1)
    return np.abs(Au[inner]).max() < 1e-13 and abs(u @ Au - a @ a) < 1e-13


def moments_ok(orc):
    p, X = 2, inputs.box_coords(*D, perturb=0.1, seed=0)
    ndof, _ = orc.space_size("Q", p, D)
    xq = orc.q_node_coords(p, D, X)
    return (abs(orc.action("Q", "mass", p, D, X, np.ones(ndof)).sum() - 1) < 1e-13
            and abs(orc.action("Q", "mass", p, D, X, xq[:, 0]).sum() - 0.5) < 1e-13)


def sequence_ok(orc):
    p, d = 2, (2, 2, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=3)
    nq, _ = orc.space_size("Q", p, d)
    g = orc.interp_grad_q_to_nce(p, d, inputs.random_vector(nq, 1, seed=11))
    y = orc.action("NCE", "nce_curlcurl", p, d, X, g, params=(0, 1, 0, 0))
    return np.abs(y).max() < 1e-10


def curl_energy_ok(orc):
    """NCE_2 covariant interpolant of u = A x: u^T K u = |curl u|^2."""
    p, d = 2, (2, 2, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=6)
    A = np.array([[0.3, -0.5, 0.2], [0.4, 0.1, -0.6], [-0.2, 0.7, 0.5]])
    u = orc.interp_linear_field("NCE", p, d, X, A, np.zeros(3))
    W = A - A.T
    c = np.array([W[2, 1], W[0, 2], W[1, 0]])
    return abs(u @ orc.action("NCE", "nce_curlcurl", p, d, X, u, params=(0, 1, 0, 0)) - c @ c) < 1e-12


def rotation_ok(orc):
    p, d = 2, (2, 1, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=4)
    th = 0.6
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    v = orc.q_node_coords(p, d, X) @ (R - np.eye(3)).T
    u = np.concatenate([v[:, 0], v[:, 1], v[:, 2]])
    return np.abs(orc.action("VQ", "neohooke", p, d, X, u)).max() < 1e-12


def lagrange_ok(orc):
    nodes, _ = orc.gauss_lobatto(4)
    t = 0.37
    return all(abs(sum(nodes[i] ** k * orc.lagrange(nodes, i, t, deriv=True) for i in range(4))
                   - k * t ** (k - 1)) < 1e-12 for k in range(1, 4))


def piola_scale_ok(orc):
    p, h = 1, 0.5
    X = inputs.box_coords(2, 2, 2, perturb=0.0)
    A = orc.cell_matrices("NCF", "ncf_mass_divdiv", p, (2, 2, 2), X, params=(1, 0, 0, 0))[0]
    A1 = orc.cell_matrices("NCF", "ncf_mass_divdiv", p, (1, 1, 1), inputs.box_coords(1, 1, 1, perturb=0.0),
                           params=(1, 0, 0, 0))[0]
    return np.abs(A - A1 / h).max() < 1e-13


def linearisation_ok(orc):
    """The neo-Hookean linearisation matches central differences of the
    residual at a state with volume change (ln J != 0)."""
    p, d = 1, (2, 1, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=4)
    ndof, _ = orc.space_size("VQ", p, d)
    u = orc.q_node_coords(p, d, X) @ np.diag([0.08, 0.05, -0.03])
    u = np.concatenate([u[:, 0], u[:, 1], u[:, 2]]) + 0.01 * inputs.random_vector(ndof, 1, seed=9)
    du = inputs.random_vector(ndof, 1, seed=13)
    k = orc.linearised_action("neohooke", p, d, X, u, du)
    e = 1e-5
    fd = (orc.action("VQ", "neohooke", p, d, X, u + e * du) - orc.action("VQ", "neohooke", p, d, X, u - e * du)) / (2 * e)
    return np.abs(k - fd).max() <= 1e-7 * np.abs(k).max()


def tangent_ok(orc):
    p, d = 1, (2, 1, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=4)
    ndof, nloc = orc.space_size("VQ", p, d)
    u = 0.03 * inputs.random_vector(ndof, 1, seed=9)
    cell = 1
    A = orc.linearised_cell_matrices("svk", p, d, X, u, cell, cell + 1)[0]
    cmap = orc.cell_map("VQ", p, d)
    e = 1e-5
    fd = np.zeros((nloc, nloc))
    for j in range(nloc):
        v = np.zeros(ndof)
        v[cmap[cell][j]] = e
        fd[:, j] = (orc.cell_vectors("VQ", "svk", p, d, X, u + v, [cell])[0]
                    - orc.cell_vectors("VQ", "svk", p, d, X, u - v, [cell])[0]) / (2 * e)
    return np.abs(A - fd).max() <= 1e-7 * np.abs(A).max()


def vector_delta_ok(orc):
    p, d = 1, (2, 1, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=4)
    A = orc.cell_matrices("VQ", "mass", p, d, X)
    As = orc.cell_matrices("Q", "mass", p, d, X)
    n3 = A.shape[1] // 3
    for a in range(3):
        for b in range(3):
            blk = A[:, a * n3:(a + 1) * n3, b * n3:(b + 1) * n3]
            if (a != b and blk.any()) or (a == b and np.abs(blk - As).max() > 1e-14 * np.abs(As).max()):
                return False
    return True


def weighted_energy_ok(orc):
    p, d = 2, (3, 2, 3)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    xn = orc.q_node_coords(p, d, X)
    a, b, c = np.array([0.4, -0.9, 1.3]), 1.7, np.array([0.3, -0.5, 0.8])
    u = xn @ a
    y = orc.weighted_action("Q", p, d, X, b + xn @ c, u)
    return abs(u @ y - (a @ a) * (b + c @ np.array([0.5, 0.5, 0.5]))) <= 1e-12


def svk_linearisation_ok(orc):
    p, d = 1, (2, 1, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=4)
    ndof, _ = orc.space_size("VQ", p, d)
    u = 0.05 * inputs.random_vector(ndof, 1, seed=9)
    du = inputs.random_vector(ndof, 1, seed=13)
    k = orc.linearised_action("svk", p, d, X, u, du)
    e = 1e-5
    fd = (orc.action("VQ", "svk", p, d, X, u + e * du) - orc.action("VQ", "svk", p, d, X, u - e * du)) / (2 * e)
    return np.abs(k - fd).max() <= 1e-7 * np.abs(k).max()


def gauss_rule_ok(orc):
    x2, w2 = orc.gauss_legendre(2)
    x3, w3 = orc.gauss_legendre(3)
    r = np.sqrt(3.0) / 6.0
    return (np.abs(np.sort(x2) - [0.5 - r, 0.5 + r]).max() < 1e-15
            and np.abs(np.sort(w3) - [5 / 18, 5 / 18, 4 / 9]).max() < 1e-15)


def q_map_ok(orc):
    p, d = 2, (3, 2, 3)
    ndof, _ = orc.space_size("Q", p, d)
    m = orc.cell_map("Q", p, d)  # integer map only: no value is written through it
    return int(m.max()) < ndof and len(np.unique(m)) == ndof


def high_degree_energy_ok(orc):
    """Q_6 Laplace energy of u = x^6 on the perturbed mesh: 36/11 (exact with
    7 Gauss points).  A mistake confined to 7 or more nodes is seen only by
    the pins at those sizes (this one, the p = 6..8 scalar-form identities and
    the 1D Lagrange-basis pins at n = 8, 9), not by the p <= 4 assembly pins
    or the n = 4 check above."""
    p, X = 6, inputs.box_coords(*D, perturb=0.1, seed=0)
    u = orc.q_node_coords(p, D, X)[:, 0] ** p
    return abs(u @ orc.action("Q", "laplace", p, D, X, u) - p * p / (2 * p - 1)) < 1e-12


PLANTS = {
    1: ("G used where G^T belongs", patch_ok),
    2: ("|J| dropped from the scalar forms", moments_ok),
    3: ("sign error in one curl component", curl_energy_ok),
    4: ("wrong quadrature-weight index", moments_ok),
    5: ("F^{-1} used for F^{-T}", rotation_ok),
    6: ("a term dropped from the Lagrange derivative", lagrange_ok),
    7: ("1/|J| dropped from the contravariant Piola map", piola_scale_ok),
    8: ("lambda ln J dropped from the neo-Hookean linearisation", linearisation_ok),
    9: ("trial direction transposed in the tangent matrix", tangent_ok),
    10: ("test component used for the trial in the vector mass matrix", vector_delta_ok),
    11: ("coefficient kappa interpolated with the neighbouring basis function", weighted_energy_ok),
    12: ("geometric term dF S dropped from the SVK linearisation", svk_linearisation_ok),
    13: ("wrong off-diagonal of the Gauss-Legendre Jacobi matrix", gauss_rule_ok),
    14: ("continuous factor advanced by p+1 nodes per cell (no shared dofs)", q_map_ok),
    15: ("Lagrange derivative loop bound fixed at 6 nodes (wrong for p >= 6 only)", high_degree_energy_ok),
}


@pytest.mark.parametrize("which", sorted(PLANTS))
def test_planted_mistake_is_caught(orc, which):
    name, check = PLANTS[which]
    assert check(orc), "pin fails on the correct oracle: " + name
    with orc.planted(which):
        caught = not check(orc)
    assert caught, "planted mistake not caught: " + name
    assert check(orc)
