"""Pins for the oracle's vector-Q_p hyperelastic residuals (Sec. 4.1: F = I +
grad u, Saint Venant-Kirchhoff S = lambda tr(E) I + 2 mu E, P = F S; the
neo-Hookean residual is the same skeleton with P = mu (F - F^{-T}) +
lambda ln(J) F^{-T}).

Pins: r(0) = 0, translations and rigid rotations give r = 0 (frame
indifference), r is the gradient of the stored energy (central differences),
both models agree with each other in the small-strain limit, and the energy of
a homogeneous deformation is the strain-energy density times the volume.
"""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

D = (2, 1, 2)


def mesh(seed=4):
    return inputs.box_coords(*D, perturb=0.1, seed=seed)


def nodal_field(orc, p, X, fn):
    """Vector Q_p dofs (component-major) interpolating fn(x) -> (3,) at GLL nodes."""
    xq = orc.q_node_coords(p, D, X)
    v = fn(xq)  # (nnode, 3)
    return np.concatenate([v[:, 0], v[:, 1], v[:, 2]])


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_zero_translation_rotation(orc, form, p):
    X = mesh()
    ndof, _ = orc.space_size("VQ", p, D)
    assert np.abs(orc.action("VQ", form, p, D, X, np.zeros(ndof))).max() == 0.0
    t = nodal_field(orc, p, X, lambda x: np.tile([0.02, -0.03, 0.01], (len(x), 1)))
    assert np.abs(orc.action("VQ", form, p, D, X, t)).max() < 1e-14
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    ax = np.array([1.0, 2.0, -1.0]) / np.sqrt(6)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = R @ (np.eye(3) + np.sin(0.4) * K + (1 - np.cos(0.4)) * K @ K)
    u = nodal_field(orc, p, X, lambda x: x @ (R - np.eye(3)).T)
    r = orc.action("VQ", form, p, D, X, u)
    # a generic displacement of the same size gives O(1) residuals
    g = nodal_field(orc, p, X, lambda x: 0.3 * np.sin(3 * x))
    assert np.abs(r).max() < 1e-12 * np.abs(orc.action("VQ", form, p, D, X, g)).max()


@pytest.mark.parametrize("form", ["neohooke", "svk"])
def test_residual_is_energy_gradient(orc, form):
    p = 2
    X = mesh()
    ndof, _ = orc.space_size("VQ", p, D)
    u = 0.02 * inputs.random_vector(ndof, 1, seed=9)
    r = orc.action("VQ", form, p, D, X, u)
    eps = 1e-6
    rng = np.random.default_rng(1)
    for j in rng.choice(ndof, 12, replace=False):
        e = np.zeros(ndof)
        e[j] = eps
        fd = (orc.energy(form, p, D, X, u + e) - orc.energy(form, p, D, X, u - e)) / (2 * eps)
        assert abs(fd - r[j]) < 1e-7 * np.abs(r).max(), (j, fd, r[j])


def test_models_agree_at_small_strain(orc):
    """Both stress laws linearise to the same linear elasticity (mu, lambda),
    so r(eps u)/eps from either converges to the same vector at rate O(eps)."""
    p = 2
    X = mesh()
    ndof, _ = orc.space_size("VQ", p, D)
    u = inputs.random_vector(ndof, 1, seed=21)
    diffs = []
    for eps in (1e-3, 1e-4):
        a = orc.action("VQ", "neohooke", p, D, X, eps * u) / eps
        b = orc.action("VQ", "svk", p, D, X, eps * u) / eps
        diffs.append(np.abs(a - b).max() / np.abs(a).max())
    assert diffs[0] < 1e-1 and diffs[1] < 1e-2
    assert 5 < diffs[0] / diffs[1] < 20  # linear convergence


@pytest.mark.parametrize("form", ["neohooke", "svk"])
def test_homogeneous_energy(orc, form):
    """u = (F0 - I) x gives grad u = F0 - I everywhere, so W = |Omega| W(F0)
    exactly (integrand constant)."""
    p = 1
    X = mesh()
    F0 = np.array([[1.05, 0.02, -0.01], [0.03, 0.97, 0.02], [0.0, -0.02, 1.01]])
    u = nodal_field(orc, p, X, lambda x: x @ (F0 - np.eye(3)).T)
    mu, lam = 1.0, 10.0
    if form == "neohooke":
        J = np.linalg.det(F0)
        W = 0.5 * mu * (np.trace(F0.T @ F0) - 3) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2
    else:
        E = 0.5 * (F0.T @ F0 - np.eye(3))
        W = 0.5 * lam * np.trace(E) ** 2 + mu * np.trace(E @ E)
    assert abs(orc.energy(form, p, D, X, u) - W) < 1e-14


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [2, 5, 8])
def test_homogeneous_patch_test(orc, form, p):
    """u = (F0 - I) x lies in vector Q_p and gives a constant F, hence a
    constant P; the cell integrals of P : grad psi_j are integrated exactly
    (adj J^T grad^ psi_j is a polynomial of degree p + 2 per direction), so by
    the divergence theorem every interior row of the residual vanishes while
    the boundary rows carry the traction P n."""
    X = mesh()
    F0 = np.array([[1.05, 0.02, -0.01], [0.03, 0.97, 0.02], [0.0, -0.02, 1.01]])
    u = nodal_field(orc, p, X, lambda x: x @ (F0 - np.eye(3)).T)
    r = orc.action("VQ", form, p, D, X, u)
    M = [p * d + 1 for d in D]
    I, J, K = np.unravel_index(np.arange(M[0] * M[1] * M[2]), M)
    interior = (I > 0) & (I < M[0] - 1) & (J > 0) & (J < M[1] - 1) & (K > 0) & (K < M[2] - 1)
    rows = np.concatenate([interior] * 3)
    assert interior.any()
    assert np.abs(r[rows]).max() < 1e-12 * np.abs(r).max()
    assert np.abs(r[~rows]).max() > 1e-3
