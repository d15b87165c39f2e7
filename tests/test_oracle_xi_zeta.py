"""Pins of the oracle's xi, xi_l and zeta_l pipelines.

Checks against: the exact planted-mode closed forms, brute-force pair sums with
the effective kernel (one pair and one node pair at a time), a direct O(N^6)
real-space convolution, the self-pair term evaluated particle by particle, the
Poisson expectation xi ~ 0, the conjugation identity of harmonic fields and an
exact three-mode closed form for zeta_l.
"""
import numpy as np
import pytest

from oracle import hermes_oracle as O
from synthetic import catalogues as C


def _mode(N, n0):
    l = np.arange(N)
    return np.cos(2 * np.pi * (n0[0] * l[:, None, None] + n0[1] * l[None, :, None]
                               + n0[2] * l[None, None, :]) / N)


@pytest.mark.parametrize("ell", [0, 2, 4])
def test_planted_single_mode(ell):
    # delta = cos(2 pi n0.l/N)  =>  (1/N^3) sum delta delta~ = K(n0)/2 exactly
    N, L, p = 16, 80.0, 4
    n0 = (2, 1, 3)
    d = _mode(N, n0)
    dh = O.forward(d)
    K = O.window_xi(N, L, p, 10.0, 16.0, ell)
    ref = 0.5 * K[n0]
    assert O.xi_parseval(dh, K) == pytest.approx(ref, rel=1e-12, abs=1e-15)
    assert O.xi_cell_contraction(d, dh, K) == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_direct_convolution_matches_fft_filter():
    N, L, p = 8, 40.0, 4
    rng = np.random.default_rng(4)
    f = rng.standard_normal((N, N, N))
    K = O.window_xi(N, L, p, 5.0, 9.0, 0)
    kap = O.kappa_from_K(K).real
    direct = O.direct_convolution(f, kap)
    via_fft = np.fft.ifftn(np.fft.fftn(f) * K).real
    np.testing.assert_allclose(direct, via_fft, atol=1e-12)


@pytest.mark.parametrize("p,n,ell", [(2, 40, 0), (4, 10, 0), (2, 30, 2)])
def test_brute_force_pairs(p, n, ell):
    # sum_l eps_l eps~_l = sum_ij w_i w_j K_eff(x_i, x_j): the grid route minus the
    # self-pair term must equal the pair sum over i != j
    N, L = 8, 40.0
    rng = np.random.default_rng(5 + p + ell)
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, size=n)
    r_edges = [4.0, 9.0, 15.0]
    res = O.xi_multipoles(pos, w, N, L, p, r_edges, ells=(ell,))
    for b in range(2):
        K = O.window_xi(N, L, p, r_edges[b], r_edges[b + 1], ell)
        bf = O.xi_brute_force(pos, w, N, L, p, K)
        assert res["xi"][0, b] == pytest.approx(bf, rel=1e-9, abs=1e-11)


def test_shot_noise_particle_by_particle():
    N, L, p = 8, 40.0, 4
    rng = np.random.default_rng(9)
    pos = rng.uniform(0, L, size=(6, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, size=6)
    K = O.window_xi(N, L, p, 3.0, 8.0, 0)
    S = O.self_pair_table(pos, w, N, L, p)
    sn = O.shot_noise(S, K, N, w.sum())
    first, m = O.node_weights(pos, N, L, p)
    kap = O.kappa_from_K(K).real
    direct = sum(w[i] ** 2 * O.keff_pair_direct(kap, first[i], m[i], first[i], m[i], N)
                 for i in range(6))
    eps_bar = w.sum() / N ** 3
    assert sn == pytest.approx(direct / (N ** 3 * eps_bar ** 2), rel=1e-12)


def test_cell_route_equals_parseval_route():
    N, L, p = 16, 100.0, 4
    pos = C.mixed_poisson_sp(3000, L, seed=11)
    edges = [5.0, 15.0, 25.0, 35.0]
    a = O.xi_multipoles(pos, None, N, L, p, edges, ells=(0, 2), route="parseval")
    b = O.xi_multipoles(pos, None, N, L, p, edges, ells=(0, 2), route="cell")
    c = O.xi_multipoles(pos, None, N, L, p, edges, ells=(0, 2), route="half")
    np.testing.assert_allclose(a["xi"], b["xi"], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(a["xi"], c["xi"], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(a["sn"], c["sn"], rtol=1e-10, atol=1e-13)


def test_poisson_catalogue_is_uncorrelated():
    N, L, p = 32, 250.0, 4
    n = 20000
    pos = C.poisson_uniform(n, L, seed=21)
    edges = np.arange(20.0, 101.0, 20.0)
    res = O.xi_multipoles(pos, None, N, L, p, edges, ells=(0, 2, 4))
    nbar = n / L ** 3
    for b in range(len(edges) - 1):
        V = 4 * np.pi / 3 * (edges[b + 1] ** 3 - edges[b] ** 3)
        sigma = np.sqrt(2.0 / (n * nbar * V))
        for a, ell in enumerate((0, 2, 4)):
            assert abs(res["xi"][a, b]) < 5 * sigma * (2 * ell + 1) ** 0.5


def test_harmonic_field_conjugation_identity():
    # real delta: a_{l,-m} = (-1)^m conj(a_{l,m})
    N, L, p = 8, 50.0, 4
    rng = np.random.default_rng(12)
    d = rng.standard_normal((N, N, N))
    dh = O.forward(d)
    for ell, m in [(1, 1), (2, 2), (3, 1)]:
        ap = np.fft.ifftn(dh * O.window_zeta(N, L, p, 6.0, 12.0, ell, m))
        am = np.fft.ifftn(dh * O.window_zeta(N, L, p, 6.0, 12.0, ell, -m))
        np.testing.assert_allclose(am, (-1) ** m * np.conj(ap), atol=1e-12)


def test_zeta_three_mode_closed_form():
    # delta = sum_{n in S} cos(2 pi n.l/N) with n_a + n_b + n_c = 0.  Then
    # a_{b lm} = sum_{n in +-S} (1/2) K_{b lm}(n) e^{2 pi i n.l/N} and
    # zeta_l(b1,b2) = 1/(4 pi) * (1/8) * sum_m sum_{n,n',n'' in +-S, n'' + n' = n} conj(K1(n)) K2(n')
    N, L, p = 8, 40.0, 4
    S = [(1, 0, 2), (2, 1, -1), (-3, -1, -1)]
    d = sum(_mode(N, s) for s in S)
    pm = S + [tuple(-x for x in s) for s in S]
    edges = [5.0, 10.0, 16.0]
    l_max = 3
    got, imag = O.zeta_multipoles(d, N, L, p, edges, l_max)
    assert imag < 1e-10
    for ell in range(l_max + 1):
        for b1 in range(2):
            for b2 in range(2):
                tot = 0.0
                for m in range(-ell, ell + 1):
                    K1 = O.window_zeta(N, L, p, edges[b1], edges[b1 + 1], ell, m)
                    K2 = O.window_zeta(N, L, p, edges[b2], edges[b2 + 1], ell, m)
                    for n in pm:
                        for n1 in pm:
                            for n2 in pm:
                                if tuple(a + b for a, b in zip(n1, n2)) == n:
                                    tot += (np.conj(K1[tuple(x % N for x in n)])
                                            * K2[tuple(x % N for x in n1)])
                ref = (tot / 8.0 / (4 * np.pi)).real
                assert got[ell, b1, b2] == pytest.approx(ref, rel=1e-10, abs=1e-13)


def test_zeta_symmetric_and_real():
    N, L, p = 8, 50.0, 4
    pos = C.mixed_poisson_sp(800, L, seed=13)
    eps, sw, _ = O.assign(pos, None, N, L, p)
    d = O.delta_from_eps(eps, sw)
    z, imag = O.zeta_multipoles(d, N, L, p, [4.0, 9.0, 14.0, 20.0], 2)
    assert imag < 1e-10 * max(1.0, np.abs(z).max())
    for ell in range(3):
        np.testing.assert_allclose(z[ell], z[ell].T, rtol=1e-10, atol=1e-14)


def test_windows_at_listed_modes_equal_the_full_grid():
    # the mode-list forms (used where a grid is too large to tabulate) give the
    # full-grid windows entry by entry, Nyquist zeros and n = 0 included
    import itertools
    N, L, p = 16, 80.0, 4
    f = O.signed_freqs(N)
    modes = np.array(list(itertools.product(f, f, f)))
    idx = tuple((modes % N).T)
    for ell in (0, 2, 4):
        K = O.window_xi(N, L, p, 10.0, 16.0, ell)
        np.testing.assert_allclose(O.window_xi_at(N, L, p, 10.0, 16.0, ell, modes), K[idx], rtol=1e-12, atol=1e-15)
    for ell, m in ((0, 0), (1, -1), (3, 2), (6, -5)):
        K = O.window_zeta(N, L, p, 6.0, 13.0, ell, m)
        np.testing.assert_allclose(O.window_zeta_at(N, L, p, 6.0, 13.0, ell, m, modes), K[idx],
                                   rtol=1e-12, atol=1e-15)


def test_planted_xi_sum_of_modes_matches_cell_contraction():
    # several planted modes: the cross terms vanish and each mode adds K(n_j)/2
    N, L, p = 16, 80.0, 4
    modes = [(1, 2, 3), (5, -2, 1), (-7, 3, 6), (2, 0, 0)]
    d = sum(_mode(N, s) for s in modes)
    dh = O.forward(d)
    edges = [3.0, 8.0, 14.0, 25.0]
    ref = O.planted_xi(N, L, p, edges, (0, 2, 4), modes)
    for a, ell in enumerate((0, 2, 4)):
        for b in range(3):
            K = O.window_xi(N, L, p, edges[b], edges[b + 1], ell)
            assert O.xi_cell_contraction(d, dh, K) == pytest.approx(ref[a, b], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("N,L,S,edges,l_max", [
    (8, 40.0, [(1, 0, 2), (2, 1, -1), (-3, -1, -1)], [5.0, 10.0, 16.0], 3),
    (16, 80.0, [(1, 2, -3), (3, -1, 2), (-4, -1, 1)], [4.0, 9.0, 15.0, 22.0], 4),
])
def test_planted_zeta_triples_match_explicit_harmonic_fields(N, L, S, edges, l_max):
    # the finite triple sum against the oracle's explicit inverse transforms of every m
    p = 4
    d = sum(_mode(N, s) for s in S)
    got, imag = O.zeta_multipoles(d, N, L, p, edges, l_max)
    assert imag < 1e-10
    np.testing.assert_allclose(O.planted_zeta(N, L, p, edges, l_max, S), got, rtol=1e-10, atol=1e-14)
