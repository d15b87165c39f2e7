"""Pins of the oracle's explicit-random (Landy-Szalay) estimator, Sec. 3.3 and
Eq. (xi-deltaDD-over-RR): brute-force DD - 2 DR + RR over RR pair sums with the
spline-smeared kernel, and the closed form for a lattice of randoms (a uniform
field by the partition of unity)."""
import numpy as np
import pytest

from oracle import hermes_oracle as O
from synthetic import catalogues as S


def _pair_sum(kap, fa, ma, wa, fb, mb, wb, N, same):
    tot = 0.0
    for i in range(len(wa)):
        for j in range(len(wb)):
            if same and i == j:
                continue
            tot += wa[i] * wb[j] * O.keff_pair_direct(kap, fa[i], ma[i], fb[j], mb[j], N)
    return tot


def test_landy_szalay_equals_brute_force_pair_counts():
    N, L, p = 16, 40.0, 3
    pd = S.mixed_poisson_sp(40, L, seed=3)
    wd = S.lognormal_masses(pd.shape[0], seed=4).astype(np.float64)  # pair products in float64
    pr = S.poisson_uniform(60, L, seed=5)
    wr = np.linspace(0.5, 1.5, pr.shape[0])
    edges = [2.0, 6.0, 12.0]
    got = O.xi_randoms(pd, wd, pr, wr, N, L, p, edges, ells=(0,))
    fd, md = O.node_weights(pd, N, L, p)
    fr, mr = O.node_weights(pr, N, L, p)
    alpha = wd.sum() / wr.sum()
    for b in range(2):
        kap = O.kappa_from_K(O.window_xi(N, L, p, edges[b], edges[b + 1], 0)).real
        dd = _pair_sum(kap, fd, md, wd, fd, md, wd, N, True)
        dr = _pair_sum(kap, fd, md, wd, fr, mr, wr, N, False)
        rr = _pair_sum(kap, fr, mr, wr, fr, mr, wr, N, True)
        ref = (dd - 2 * alpha * dr + alpha * alpha * rr) / (alpha * alpha * rr)
        assert got[0, b] == pytest.approx(ref, rel=1e-9, abs=1e-12)


def test_lattice_randoms_reduce_to_the_analytic_estimator():
    # randoms on every grid node: eps_R = 1 everywhere (partition of unity), so the
    # difference field is delta itself, RR_b = 1 - alpha^2 SN_R(K_0,b) and the numerator
    # is the analytic one less the randoms' own self pairs, alpha^2 SN_R(K_l,b)
    N, L, p = 16, 64.0, 4
    pd = S.lognormal_catalogue(3000, L, seed=8, n_grid=16)
    g = (np.arange(N) * (L / N)).astype(np.float32)
    pr = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    edges = np.linspace(4.0, 28.0, 5)
    got = O.xi_randoms(pd, None, pr, None, N, L, p, edges, ells=(0, 2))
    ana = O.xi_multipoles(pd, None, N, L, p, edges, ells=(0, 2))["xi"]
    s_r = O.self_pair_table(pr, None, N, L, p)
    alpha = pd.shape[0] / pr.shape[0]
    for b in range(len(edges) - 1):
        K0 = O.window_xi(N, L, p, edges[b], edges[b + 1], 0)
        rr = 1.0 - O.shot_noise(alpha * alpha * s_r, K0, N, float(pd.shape[0]))
        for a, ell in enumerate((0, 2)):
            Kl = O.window_xi(N, L, p, edges[b], edges[b + 1], ell)
            sn_r = O.shot_noise(alpha * alpha * s_r, Kl, N, float(pd.shape[0]))
            assert got[a, b] * rr == pytest.approx(ana[a, b] - sn_r, rel=1e-10, abs=1e-13)
