"""Pins for the oracle's H(div) NCF_p and H(curl) NCE_p forms.

The elements are built as in Sec. 2.6-2.7 (Eq. rtcf_impl: enriched sums of
HDiv/HCurl-wrapped tensor products of P_p on GLL nodes and dP_{p-1} on Gauss
nodes) with the split-Concatenate local layout of Sec. 3.5 (Eqs. rtcf_split_x/y);
the curl-curl form is Eq. curl_curl_form.  Pins: on the unit cube the matrices
are Kronecker products of 1D integrals computed here with numpy; the Piola
maps scale with the cell size as the mathematics fixes; ranks; and the exact
sequence grad Q_p -> NCE_p -> curl -> NCF_p -> div (curl grad = 0, div curl = 0)
holds on perturbed meshes.
"""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs


def nodes_1d(kind, n):
    """GLL nodes from numpy's Legendre class (roots of P'_{n-1}), Gauss nodes
    from numpy's leggauss, both mapped to [0,1]."""
    if kind == "GL":
        t = np.polynomial.legendre.leggauss(n)[0]
    else:
        t = np.concatenate([[-1.0], np.sort(np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots().real), [1.0]])
    return 0.5 * (t + 1.0)


def lag_polys(xn):
    out = []
    for i in range(len(xn)):
        others = np.delete(xn, i)
        c = np.polynomial.polynomial.polyfromroots(others) / np.prod(xn[i] - others)
        out.append(np.polynomial.Polynomial(c))
    return out


def int01(f, g):
    t, w = np.polynomial.legendre.leggauss(24)
    x = 0.5 * (t + 1.0)
    return 0.5 * np.sum(w * f(x) * g(x))


def gram(fs, gs):
    return np.array([[int01(f, g) for f in fs] for g in gs])  # row = test g, col = trial f


def factors(fam, p, c):
    """Per-axis 1D bases of block c."""
    out = []
    for d in range(3):
        cont = (d == c) if fam == "NCF" else (d != c)
        out.append(lag_polys(nodes_1d("GLL", p + 1) if cont else nodes_1d("GL", p)))
    return out


def kron3(mats):
    return np.kron(np.kron(mats[0], mats[1]), mats[2])


def unit_cube_matrix(fam, p, part):
    """Reference-cell matrix on [0,1]^3 (J = I): part 'mass', 'div' or 'curl'."""
    blocks = [factors(fam, p, c) for c in range(3)]
    sizes = [int(np.prod([len(b[d]) for d in range(3)])) for b in blocks]
    off = np.concatenate([[0], np.cumsum(sizes)])
    A = np.zeros((off[-1], off[-1]))
    # curl of f e_c: list of (component, derivative axis, sign)
    curl_terms = {0: [(1, 2, 1.0), (2, 1, -1.0)], 1: [(0, 2, -1.0), (2, 0, 1.0)], 2: [(0, 1, 1.0), (1, 0, -1.0)]}
    for ci in range(3):       # trial block
        for cj in range(3):   # test block
            M = np.zeros((sizes[cj], sizes[ci]))
            if part == "mass" and ci == cj:
                M = kron3([gram(blocks[ci][d], blocks[cj][d]) for d in range(3)])
            elif part == "div":
                mats = []
                for d in range(3):
                    fi = [f.deriv() if d == ci else f for f in blocks[ci][d]]
                    gj = [g.deriv() if d == cj else g for g in blocks[cj][d]]
                    mats.append(gram(fi, gj))
                M = kron3(mats)
            elif part == "curl":
                for (ki, ai, si) in curl_terms[ci]:
                    for (kj, aj, sj) in curl_terms[cj]:
                        if ki != kj:
                            continue
                        mats = []
                        for d in range(3):
                            fi = [f.deriv() if d == ai else f for f in blocks[ci][d]]
                            gj = [g.deriv() if d == aj else g for g in blocks[cj][d]]
                            mats.append(gram(fi, gj))
                        M = M + si * sj * kron3(mats)
            A[off[cj]:off[cj + 1], off[ci]:off[ci + 1]] = M
    return A


CUBE = inputs.box_coords(1, 1, 1, perturb=0.0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_ncf_unit_cube_kronecker(orc, p):
    Am = orc.cell_matrices("NCF", "ncf_mass_divdiv", p, (1, 1, 1), CUBE, params=(1, 0, 0, 0))[0]
    Ad = orc.cell_matrices("NCF", "ncf_mass_divdiv", p, (1, 1, 1), CUBE, params=(0, 1, 0, 0))[0]
    np.testing.assert_allclose(Am, unit_cube_matrix("NCF", p, "mass"), atol=1e-14)
    np.testing.assert_allclose(Ad, unit_cube_matrix("NCF", p, "div"), atol=1e-13 * np.abs(Ad).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_nce_unit_cube_kronecker(orc, p):
    Am = orc.cell_matrices("NCE", "nce_curlcurl", p, (1, 1, 1), CUBE, params=(1, 0, 0, 0))[0]
    Ac = orc.cell_matrices("NCE", "nce_curlcurl", p, (1, 1, 1), CUBE, params=(0, 1, 0, 0))[0]
    np.testing.assert_allclose(Am, unit_cube_matrix("NCE", p, "mass"), atol=1e-14)
    np.testing.assert_allclose(Ac, unit_cube_matrix("NCE", p, "curl"), atol=1e-13 * np.abs(Ac).max())


def test_piola_scalings(orc):
    """Cube of side h: contravariant mass ~ 1/h, div-div ~ 1/h^3; covariant
    mass ~ h, curl-curl ~ 1/h (each relative to the unit cube)."""
    p, h = 2, 0.5
    X = inputs.box_coords(2, 2, 2, perturb=0.0)
    for fam, form, prm, scale in [("NCF", "ncf_mass_divdiv", (1, 0, 0, 0), 1 / h),
                                  ("NCF", "ncf_mass_divdiv", (0, 1, 0, 0), 1 / h ** 3),
                                  ("NCE", "nce_curlcurl", (1, 0, 0, 0), h),
                                  ("NCE", "nce_curlcurl", (0, 1, 0, 0), 1 / h)]:
        A = orc.cell_matrices(fam, form, p, (2, 2, 2), X, params=prm)
        A1 = orc.cell_matrices(fam, form, p, (1, 1, 1), CUBE, params=prm)[0]
        for c in range(8):
            np.testing.assert_allclose(A[c], scale * A1, atol=1e-13 * scale * np.abs(A1).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_ranks_on_perturbed_cells(orc, p):
    d = (2, 2, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=7)
    Ad = orc.cell_matrices("NCF", "ncf_mass_divdiv", p, d, X, params=(0, 1, 0, 0))
    Ac = orc.cell_matrices("NCE", "nce_curlcurl", p, d, X, params=(0, 1, 0, 0))
    Am = orc.cell_matrices("NCF", "ncf_mass_divdiv", p, d, X, params=(1, 0, 0, 0))
    for c in range(8):
        ev = np.linalg.eigvalsh(0.5 * (Ad[c] + Ad[c].T))
        assert ev[0] > -1e-12 * ev[-1] and np.sum(ev > 1e-10 * ev[-1]) == p ** 3
        ev = np.linalg.eigvalsh(0.5 * (Ac[c] + Ac[c].T))
        assert np.sum(ev > 1e-10 * ev[-1]) == 3 * p * (p + 1) ** 2 - ((p + 1) ** 3 - 1)
        assert np.linalg.eigvalsh(0.5 * (Am[c] + Am[c].T))[0] > 0


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_exact_sequence(orc, p):
    """curl-curl annihilates gradients of Q_p fields and div-div annihilates
    curls of NCE_p fields, on a perturbed mesh (the Piola maps commute with
    grad/curl/div), while random fields are not annihilated."""
    d = (2, 3, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=3)
    nq, _ = orc.space_size("Q", p, d)
    ne, _ = orc.space_size("NCE", p, d)
    phi = inputs.random_vector(nq, 1, seed=11)
    g = orc.interp_grad_q_to_nce(p, d, phi)
    ycc = orc.action("NCE", "nce_curlcurl", p, d, X, g, params=(0, 1, 0, 0))
    rnd = inputs.random_vector(ne, 1, seed=12)
    yrnd = orc.action("NCE", "nce_curlcurl", p, d, X, rnd, params=(0, 1, 0, 0))
    assert np.abs(ycc).max() < 1e-12 * np.abs(g).max() * np.abs(yrnd).max() / np.abs(rnd).max() * 10
    assert np.abs(yrnd).max() > 1e-3
    cu = orc.interp_curl_nce_to_ncf(p, d, rnd)
    ydd = orc.action("NCF", "ncf_mass_divdiv", p, d, X, cu, params=(0, 1, 0, 0))
    nf, _ = orc.space_size("NCF", p, d)
    rf = inputs.random_vector(nf, 1, seed=13)
    yrf = orc.action("NCF", "ncf_mass_divdiv", p, d, X, rf, params=(0, 1, 0, 0))
    assert np.abs(ydd).max() < 1e-11 * np.abs(cu).max() * np.abs(yrf).max() / np.abs(rf).max()
    assert np.abs(yrf).max() > 1e-3


@pytest.mark.parametrize("fam,form", [("NCF", "ncf_mass_divdiv"), ("NCE", "nce_curlcurl")])
def test_action_equals_cell_matrices(orc, fam, form):
    p, d = 2, (2, 2, 3)
    X = inputs.box_coords(*d, perturb=0.1, seed=1)
    ndof, _ = orc.space_size(fam, p, d)
    m = orc.cell_map(fam, p, d)
    prm = (0.7, 1.3, 0, 0)
    A = orc.cell_matrices(fam, form, p, d, X, params=prm)
    x = inputs.random_vector(ndof, 1, seed=2)
    y = np.zeros(ndof)
    for c in range(len(m)):
        np.add.at(y, m[c], A[c] @ x[m[c]])
    y2 = orc.action(fam, form, p, d, X, x, params=prm)
    assert np.abs(y - y2).max() < 1e-13 * np.abs(y2).max()


A_LIN = np.array([[0.3, -0.5, 0.2], [0.4, 0.1, -0.6], [-0.2, 0.7, 0.5]])
B_LIN = np.array([0.1, -0.2, 0.3])


def _cube_l2(A, b):
    """int over [0,1]^3 of |A x + b|^2 (x uniform: mean 1/2, variance 1/12)."""
    m = A @ np.full(3, 0.5) + b
    return m @ m + np.sum(A * A) / 12.0


@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_nce_linear_field_on_perturbed_mesh(orc, p):
    """The covariant interpolant of a linear field is exact for p >= 2 even on
    trilinear cells, so curl u = (A - A^T) axial vector exactly and
    u^T K u = |curl u|^2 |Omega|, u^T M u = int |u|^2 (Omega = [0,1]^3)."""
    d = (2, 2, 3)
    X = inputs.box_coords(*d, perturb=0.1, seed=6)
    u = orc.interp_linear_field("NCE", p, d, X, A_LIN, B_LIN)
    K = orc.action("NCE", "nce_curlcurl", p, d, X, u, params=(0, 1, 0, 0))
    M = orc.action("NCE", "nce_curlcurl", p, d, X, u, params=(1, 0, 0, 0))
    W = A_LIN - A_LIN.T
    curl = np.array([W[2, 1], W[0, 2], W[1, 0]])
    assert abs(u @ K - curl @ curl) < 1e-12
    assert abs(u @ M - _cube_l2(A_LIN, B_LIN)) < 1e-12


@pytest.mark.parametrize("p", [3, 5, 8])
def test_ncf_linear_field_on_perturbed_mesh(orc, p):
    """The contravariant interpolant of a linear field is exact for p >= 3 on
    trilinear cells: div u = tr A, u^T D u = (tr A)^2, u^T M u = int |u|^2."""
    d = (2, 2, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=8)
    u = orc.interp_linear_field("NCF", p, d, X, A_LIN, B_LIN)
    Dd = orc.action("NCF", "ncf_mass_divdiv", p, d, X, u, params=(0, 1, 0, 0))
    M = orc.action("NCF", "ncf_mass_divdiv", p, d, X, u, params=(1, 0, 0, 0))
    assert abs(u @ Dd - np.trace(A_LIN) ** 2) < 1e-12
    assert abs(u @ M - _cube_l2(A_LIN, B_LIN)) < 1e-12
