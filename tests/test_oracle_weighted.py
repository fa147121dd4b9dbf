"""Pins for the oracle's weighted Laplace form a(u, v) = int kappa grad u .
grad v (Sec. 1.1, Eq. weighted_laplace), kappa given by its dofs in the space.

Pins fixed by the mathematics (the (p+1)-point Gauss rule integrates each
integrand below exactly for p >= 1 on the trilinear cells):
  * for u = a.x (so grad u = a) and kappa = b + c.x, the energy
    u . A_kappa u = |a|^2 int kappa = |a|^2 (b + c . (1/2, 1/2, 1/2)) on [0,1]^3;
  * the divergence theorem at interior dofs: (A_kappa u)_j = -(c . a) int psi_j,
    with int psi_j = (M 1)_j from the (separately pinned) mass action;
  * constants in the kernel, symmetric element matrices, and kappa = const
    scaling the Laplace form; action = sum of the element matrices.
"""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

D = (3, 2, 3)


def setup(orc, fam, p, seed=0):
    X = inputs.box_coords(*D, perturb=0.1, seed=seed)
    ndof, _ = orc.space_size(fam, p, D)
    return X, ndof


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_energy_and_divergence_theorem(orc, p):
    X, ndof = setup(orc, "Q", p)
    xn = orc.q_node_coords(p, D, X)
    a = np.array([0.4, -0.9, 1.3])
    b, c = 1.7, np.array([0.3, -0.5, 0.8])
    kappa = b + xn @ c
    u = xn @ a
    y = orc.weighted_action("Q", p, D, X, kappa, u)
    assert abs(u @ y - (a @ a) * (b + c @ np.array([0.5, 0.5, 0.5]))) <= 1e-12
    m1 = orc.action("Q", "mass", p, D, X, np.ones(ndof))
    interior = np.all((xn > 1e-12) & (xn < 1 - 1e-12), axis=1)
    assert interior.sum() > 0
    assert np.abs(y[interior] + (c @ a) * m1[interior]).max() <= 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("p", [1, 2, 4, 8])
def test_constant_kappa_scales_laplace(orc, fam, p):
    X, ndof = setup(orc, fam, p, seed=2)
    x = inputs.random_vector(ndof, 1, seed=3)
    y = orc.weighted_action(fam, p, D, X, np.full(ndof, 2.5), x)
    ref = 2.5 * orc.action(fam, "laplace", p, D, X, x)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("fam", ["Q", "DQ"])
def test_matrices_symmetric_constants_and_action(orc, fam):
    p = 2
    X, ndof = setup(orc, fam, p, seed=4)
    kappa = 1.0 + 0.5 * inputs.random_vector(ndof, 1, seed=5)
    A = orc.weighted_cell_matrices(fam, p, D, X, kappa)
    scale = np.abs(A).max()
    for c in range(A.shape[0]):
        assert np.abs(A[c] - A[c].T).max() <= 1e-14 * scale
        assert np.abs(A[c].sum(axis=1)).max() <= 1e-13 * scale
    x = inputs.random_vector(ndof, 1, seed=6)
    cmap = orc.cell_map(fam, p, D)
    ref = np.zeros(ndof)
    for c in range(A.shape[0]):
        np.add.at(ref, cmap[c], A[c] @ x[cmap[c]])
    y = orc.weighted_action(fam, p, D, X, kappa, x)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
