"""Pins for the oracle's linearised hyperelastic operator K(u) du (the Jacobian
of the residual of Sec. 4.1, whose action the paper benchmarks).

Pins, each independent of the linearisation code:
  * K(u) du equals the central difference of the (separately pinned) residual,
    (r(u + e du) - r(u - e du)) / 2e, to O(e^2);
  * K(u) is symmetric: it is the Hessian of the discrete stored energy;
  * at u = 0 both laws reduce to linear elasticity: for du = A x,
    du . K(0) du = 2 mu |sym A|^2 + lambda (tr A)^2 exactly (unit volume), and
    infinitesimal rotations du = W x (W skew) lie in the kernel;
  * the action is linear in du (several directions at once).
"""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

D = (2, 1, 2)


def mesh(seed=4):
    return inputs.box_coords(*D, perturb=0.1, seed=seed)


def nodal_field(orc, p, X, fn, dims=D):
    xq = orc.q_node_coords(p, dims, X)
    v = fn(xq)
    return np.concatenate([v[:, 0], v[:, 1], v[:, 2]])


def state(orc, p, X, seed=9, scale=0.03):
    """A random state whose displacement gradient stays small: nodal values
    of 0.03 at p <= 2, scaled by 2/p above (nodes p times closer together), so
    det F > 0 at every point."""
    ndof, _ = orc.space_size("VQ", p, D)
    return scale * min(1.0, 2.0 / p) * inputs.random_vector(ndof, 1, seed=seed)


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [1, 2, 5])
def test_linearisation_matches_central_difference(orc, form, p):
    X = mesh()
    ndof, _ = orc.space_size("VQ", p, D)
    u = state(orc, p, X)
    # the truncation error is O(eps^2 |grad du|^3): keep |grad du| as at p = 2
    du = min(1.0, 2.0 / p) * inputs.random_vector(ndof, 1, seed=13)
    k = orc.linearised_action(form, p, D, X, u, du)
    eps = 1e-5
    fd = (orc.action("VQ", form, p, D, X, u + eps * du) - orc.action("VQ", form, p, D, X, u - eps * du)) / (2 * eps)
    assert np.abs(k - fd).max() <= 1e-7 * np.abs(k).max()


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [2, 5])
def test_linearisation_is_symmetric(orc, form, p):
    X = mesh()
    ndof, _ = orc.space_size("VQ", p, D)
    u = state(orc, p, X)
    d1 = inputs.random_vector(ndof, 1, seed=21)
    d2 = inputs.random_vector(ndof, 1, seed=22)
    a = d2 @ orc.linearised_action(form, p, D, X, u, d1)
    b = d1 @ orc.linearised_action(form, p, D, X, u, d2)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_small_strain_limit_is_linear_elasticity(orc, form, p):
    X = mesh(seed=6)
    ndof, _ = orc.space_size("VQ", p, D)
    mu, lam = 1.0, 10.0
    A = np.array([[0.3, -0.5, 0.2], [0.4, 0.1, -0.6], [-0.2, 0.7, 0.5]])
    du = nodal_field(orc, p, X, lambda x: x @ A.T)
    k = orc.linearised_action(form, p, D, X, np.zeros(ndof), du)
    sym = 0.5 * (A + A.T)
    assert abs(du @ k - (2 * mu * np.sum(sym * sym) + lam * np.trace(A) ** 2)) <= 1e-12 * 10
    W = 0.5 * (A - A.T)
    rot = nodal_field(orc, p, X, lambda x: x @ W.T)
    assert np.abs(orc.linearised_action(form, p, D, X, np.zeros(ndof), rot)).max() <= 1e-13


def test_linearisation_is_linear_in_direction(orc):
    p = 2
    X = mesh()
    ndof, _ = orc.space_size("VQ", p, D)
    u = state(orc, p, X)
    d = np.stack([inputs.random_vector(ndof, 1, seed=s) for s in (31, 32)], axis=1)
    k2 = orc.linearised_action("neohooke", p, D, X, u, d)
    for r in range(2):
        k1 = orc.linearised_action("neohooke", p, D, X, u, np.ascontiguousarray(d[:, r]))
        assert np.abs(k2[:, r] - k1).max() <= 1e-14 * np.abs(k1).max()
    kc = orc.linearised_action("neohooke", p, D, X, u, 2.0 * d[:, 0] - 3.0 * d[:, 1])
    assert np.abs(kc - (2.0 * k2[:, 0] - 3.0 * k2[:, 1])).max() <= 1e-13 * np.abs(kc).max()
