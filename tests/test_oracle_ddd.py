"""Pins of the oracle's 3PCF monopole by triple connection coefficients (Eq. 3PCF-ddd-monopole,
Eq. con-coeff, Eq. DDD-vector-product) against facts that do not come from the oracle's
stencil itself:

* the one-dimensional overlap table: hand-integrated values for the linear spline, the
  autocorrelation identity sum_b gamma(a, b) = M_2p(a), total mass 1, its symmetries;
* the whole estimator against a closed form for planted Fourier modes (Poisson summation of
  the spline fields, no stencil, no FFT of a grid);
* the stencil contraction against an independent exact quadrature of the triple product of
  the spline fields, evaluated point by point from the basis functions;
* p = 1 (box basis, Gamma the identity) against the cell sum zeta_0.
"""
import numpy as np
import pytest

from oracle import hermes_oracle as O


def test_overlap_table_of_the_linear_spline_by_hand():
    # hat(u) = 1 - |u|: int hat^3 = 2 int_0^1 (1-t)^3 = 1/2; one neighbour: int_0^1 t (1-t)^2 = 1/12;
    # the two opposite neighbours meet only at u = 0
    g = O.triple_overlap_1d(2)
    want = np.array([[1 / 12, 1 / 12, 0.0], [1 / 12, 0.5, 1 / 12], [0.0, 1 / 12, 1 / 12]])
    np.testing.assert_allclose(g, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_overlap_table_identities(p):
    g = O.triple_overlap_1d(p)
    a = np.arange(-(p - 1), p)
    # partition of unity: sum_b M_p(u - b) = 1, so the row sums are the autocorrelation M_p * M_p = M_2p
    np.testing.assert_allclose(g.sum(axis=1), O.bspline(2 * p, a.astype(float)), rtol=0, atol=1e-14)
    assert abs(g.sum() - 1.0) < 1e-13
    np.testing.assert_allclose(g, g.T, atol=1e-15)
    np.testing.assert_allclose(g, g[::-1, ::-1], atol=1e-15)        # M_p is even
    # gamma(a, b) vanishes when two of the three supports do not overlap
    assert np.all(g[np.abs(a[:, None] - a[None, :]) >= p] == 0.0)
    G = O.connection_coefficients(p)
    assert G.shape == ((2 * p - 1) ** 3,) * 2 and abs(G.sum() - 1.0) < 1e-12


def _planted(N, modes, amps):
    l = np.indices((N, N, N)).reshape(3, -1).T
    d = np.zeros(N ** 3)
    for n, a in zip(modes, amps):
        d += a * np.cos(2 * np.pi * (l @ np.asarray(n)) / N)
    return d.reshape(N, N, N)


@pytest.mark.parametrize("p,tol", [(2, 1e-7), (3, 1e-10), (4, 1e-10), (5, 1e-10), (6, 1e-10)])
def test_monopole_matches_the_poisson_closed_form_for_planted_modes(p, tol):
    # three modes that close a triangle (n_a + n_b + n_c = 0) and one that does not
    N, L = 16, 200.0
    modes = [(1, 2, 0), (2, -1, 1), (-3, -1, -1), (0, 3, 2)]
    amps = [0.3, 0.2, 0.25, 0.15]
    delta = _planted(N, modes, amps)
    edges = [10.0, 30.0, 60.0, 90.0]
    got = O.ddd_monopole(delta, N, L, p, edges)
    ref = O.planted_ddd(N, L, p, edges, modes, amps)
    assert np.abs(ref).max() > 1e-4
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max())
    np.testing.assert_allclose(got, got.T, atol=1e-15)


def _spline_at(coef, p, u):
    """sum_l coef_l prod_d M_p(u_d - l_d) at points u [n, 3], term by term (periodic)."""
    N = coef.shape[0]
    out = np.zeros(u.shape[0])
    base = np.floor(u - p / 2.0).astype(np.int64) + 1          # first l with |u - l| < p/2
    for ox in range(p):
        for oy in range(p):
            for oz in range(p):
                l = base + np.array([ox, oy, oz])
                w = (O.bspline(p, u[:, 0] - l[:, 0]) * O.bspline(p, u[:, 1] - l[:, 1])
                     * O.bspline(p, u[:, 2] - l[:, 2]))
                out += w * coef[l[:, 0] % N, l[:, 1] % N, l[:, 2] % N]
    return out


@pytest.mark.parametrize("p", [2, 3, 4])
def test_stencil_equals_the_exact_triple_product_integral(p):
    # (1/N^3) int F_delta F_1 F_2 du over the box, with the spline fields evaluated from their
    # coefficients at Gauss points of every knot cell (the integrand is a polynomial of degree
    # 3(p-1) per axis there; 2p points per axis are exact)
    rng = np.random.default_rng(5 + p)
    N = 6
    d, f1, f2 = (rng.standard_normal((N, N, N)) for _ in range(3))
    x, wt = np.polynomial.legendre.leggauss(2 * p)
    t, wt = 0.5 * (x + 1.0), 0.5 * wt
    o = 0.0 if p % 2 == 0 else -0.5                               # knots: integers or half-integers
    cells = np.indices((N, N, N)).reshape(3, -1).T.astype(float) + o
    tg = np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1).reshape(-1, 3)
    wg = np.einsum("i,j,k->ijk", wt, wt, wt).ravel()
    tot = 0.0
    for g in range(tg.shape[0]):
        u = cells + tg[g]
        tot += wg[g] * np.sum(_spline_at(d, p, u) * _spline_at(f1, p, u) * _spline_at(f2, p, u))
    got = O.ddd_from_fields(d, [f1, f2], p)[0, 1]
    assert abs(got - tot / N ** 3) < 1e-12 * max(1.0, abs(tot / N ** 3))


def test_box_basis_reduces_to_the_cell_sum_zeta0():
    # p = 1: gamma = [[1]], so the two-fold coefficients are f_b1 f_b2 and DDD = zeta_0
    rng = np.random.default_rng(3)
    N, L = 16, 100.0
    pos = rng.uniform(0, L, size=(3000, 3))
    eps, sw, _ = O.assign(pos, None, N, L, 1)
    delta = O.delta_from_eps(eps, sw)
    edges = [5.0, 15.0, 30.0]
    ddd = O.ddd_monopole(delta, N, L, 1, edges)
    z, imag = O.zeta_multipoles(delta, N, L, 1, edges, 0)
    np.testing.assert_allclose(ddd, z[0], rtol=1e-10, atol=1e-14)


def test_constant_coefficients_give_the_total_mass():
    # partition of unity: F = 1 everywhere when every coefficient is 1, so DDD = 1
    for p in (2, 3, 4):
        one = np.ones((5, 5, 5))
        assert abs(O.ddd_from_fields(one, [one], p)[0, 0] - 1.0) < 1e-12
