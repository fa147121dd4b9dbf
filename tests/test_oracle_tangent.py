"""Pins for the oracle's tangent (element) matrices of the hyperelastic
residual, A^K(u) = d b^K / d u_K (Sec. 4.1: the linearised operator, here
assembled per cell; row = test, column = trial).

Pins, each independent of the matrix routine:
  * every column equals the central difference of the (separately pinned)
    residual cell vector under a perturbation of that local dof, to O(e^2);
  * A^K is symmetric: it is the Hessian of the cell's stored energy;
  * constant trial fields (translations) give dF = 0, so A^K t = 0;
  * sum_K P_K^T A^K P_K du equals the (separately pinned) linearised action;
  * at u = 0 both laws reduce to linear elasticity, so the neo-Hookean and
    SVK matrices coincide there.
"""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

D = (2, 1, 2)


def setup(orc, p, seed=4, scale=0.03):
    X = inputs.box_coords(*D, perturb=0.1, seed=seed)
    ndof, nloc = orc.space_size("VQ", p, D)
    u = scale * inputs.random_vector(ndof, 1, seed=9)
    return X, ndof, nloc, u


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [1, 2])
def test_columns_match_central_difference_of_residual(orc, form, p):
    X, ndof, nloc, u = setup(orc, p)
    cell = 2
    A = orc.linearised_cell_matrices(form, p, D, X, u, cell, cell + 1)[0]
    cmap = orc.cell_map("VQ", p, D)
    eps = 1e-5
    fd = np.zeros((nloc, nloc))
    for j in range(nloc):
        e = np.zeros(ndof)
        e[cmap[cell][j]] = eps
        bp = orc.cell_vectors("VQ", form, p, D, X, u + e, [cell])[0]
        bm = orc.cell_vectors("VQ", form, p, D, X, u - e, [cell])[0]
        fd[:, j] = (bp - bm) / (2 * eps)
    assert np.abs(A - fd).max() <= 1e-7 * np.abs(A).max()


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetric_and_translations_in_kernel(orc, form, p):
    X, ndof, nloc, u = setup(orc, p)
    A = orc.linearised_cell_matrices(form, p, D, X, u)
    n3 = nloc // 3
    scale = np.abs(A).max()
    for c in range(A.shape[0]):
        assert np.abs(A[c] - A[c].T).max() <= 1e-13 * scale
        for b in range(3):  # component-major local numbering: block b holds component b
            t = np.zeros(nloc)
            t[b * n3:(b + 1) * n3] = 1.0
            assert np.abs(A[c] @ t).max() <= 1e-13 * scale


@pytest.mark.parametrize("form", ["neohooke", "svk"])
def test_assembled_matrices_give_the_action(orc, form):
    p = 2
    X, ndof, nloc, u = setup(orc, p, seed=5)
    A = orc.linearised_cell_matrices(form, p, D, X, u)
    cmap = orc.cell_map("VQ", p, D)
    du = inputs.random_vector(ndof, 1, seed=17)
    y = np.zeros(ndof)
    for c in range(A.shape[0]):
        np.add.at(y, cmap[c], A[c] @ du[cmap[c]])
    ref = orc.linearised_action(form, p, D, X, u, du)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_both_laws_are_linear_elasticity_at_zero(orc):
    p = 2
    X, ndof, nloc, _ = setup(orc, p, seed=6)
    z = np.zeros(ndof)
    An = orc.linearised_cell_matrices("neohooke", p, D, X, z)
    As = orc.linearised_cell_matrices("svk", p, D, X, z)
    assert np.abs(An - As).max() <= 1e-13 * np.abs(As).max()


def test_cell_range(orc):
    p = 1
    X, ndof, nloc, u = setup(orc, p)
    full = orc.linearised_cell_matrices("svk", p, D, X, u)
    part = orc.linearised_cell_matrices("svk", p, D, X, u, 1, 3)
    assert np.array_equal(part, full[1:3])
