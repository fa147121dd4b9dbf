"""Pins for the oracle's vector forms on vector Q_p (Sec. 3.3: the vector
mass form and, alike, int grad u : grad v and their Helmholtz combination),
which the oracle writes with full vectors, so the component delta is an outcome
to check, not an assumption.

  * the element matrix has the delta pattern: blocks (a, b) with a != b are
    exactly zero, and the diagonal blocks equal the (separately pinned) scalar
    Q_p matrices;
  * closed forms on the perturbed unit cube: for a constant field u = c,
    u . M u = |c|^2; for u = A x, u . K u = |A|_F^2 and (K u)_j = 0 at interior
    dofs (patch test, per component);
  * the action equals the assembled element matrices and, per component, the
    scalar action; Helmholtz = alpha K + beta M.
"""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

D = (2, 3, 2)


def setup(orc, p, seed=0):
    X = inputs.box_coords(*D, perturb=0.1, seed=seed)
    ndof, nloc = orc.space_size("VQ", p, D)
    nq, _ = orc.space_size("Q", p, D)
    return X, ndof, nloc, nq


@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", [1, 2])
def test_delta_pattern_and_scalar_blocks(orc, form, p):
    X, ndof, nloc, nq = setup(orc, p)
    prm = (0.7, -1.3, 0.0, 0.0) if form == "helmholtz" else None
    A = orc.cell_matrices("VQ", form, p, D, X, params=prm)
    As = orc.cell_matrices("Q", form, p, D, X, params=prm)
    n3 = nloc // 3
    for c in range(A.shape[0]):
        for a in range(3):
            for b in range(3):
                blk = A[c, a * n3:(a + 1) * n3, b * n3:(b + 1) * n3]
                if a != b:
                    assert not blk.any()
                else:
                    assert np.abs(blk - As[c]).max() <= 1e-14 * np.abs(As[c]).max()


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_closed_forms(orc, p):
    X, ndof, nloc, nq = setup(orc, p, seed=1)
    xn = orc.q_node_coords(p, D, X)
    c = np.array([0.3, -1.1, 0.8])
    u = np.concatenate([np.full(nq, c[0]), np.full(nq, c[1]), np.full(nq, c[2])])
    assert abs(u @ orc.action("VQ", "mass", p, D, X, u) - c @ c) <= 1e-13
    A = np.array([[0.4, -0.2, 0.9], [1.1, 0.3, -0.5], [-0.7, 0.6, 0.2]])
    v = xn @ A.T  # v[:, a] = (A x)_a
    u = np.concatenate([v[:, 0], v[:, 1], v[:, 2]])
    Ku = orc.action("VQ", "laplace", p, D, X, u)
    assert abs(u @ Ku - np.sum(A * A)) <= 1e-12
    M = [p * d + 1 for d in D]
    I, J, K = np.unravel_index(np.arange(nq), M)
    inner = (I > 0) & (I < M[0] - 1) & (J > 0) & (J < M[1] - 1) & (K > 0) & (K < M[2] - 1)
    assert inner.any()
    for a in range(3):
        assert np.abs(Ku[a * nq:(a + 1) * nq][inner]).max() <= 1e-12


@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
def test_action_matrices_components_and_helmholtz(orc, form):
    p = 2
    X, ndof, nloc, nq = setup(orc, p, seed=2)
    x = inputs.random_vector(ndof, 2, seed=3)
    prm = (0.7, -1.3, 0.0, 0.0) if form == "helmholtz" else None
    y = orc.action("VQ", form, p, D, X, x, params=prm)
    A = orc.cell_matrices("VQ", form, p, D, X, params=prm)
    cmap = orc.cell_map("VQ", p, D)
    ref = np.zeros_like(x)
    for c in range(A.shape[0]):
        np.add.at(ref, cmap[c], A[c] @ x[cmap[c]])
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    for a in range(3):
        ys = orc.action("Q", form, p, D, X, x[a * nq:(a + 1) * nq], params=prm)
        assert np.abs(y[a * nq:(a + 1) * nq] - ys).max() <= 1e-14 * np.abs(ys).max()
    if form == "helmholtz":
        yk = orc.action("VQ", "laplace", p, D, X, x)
        ym = orc.action("VQ", "mass", p, D, X, x)
        assert np.abs(y - (0.7 * yk - 1.3 * ym)).max() <= 1e-13 * np.abs(y).max()
