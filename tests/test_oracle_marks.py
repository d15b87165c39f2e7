"""Pins of the oracle's smoothed density at the particles and the density marks
(Sec. 3.3, the power-law and inverse-density marks): brute-force sums with the
spline-smeared kernel, a constant field, the mean of the gather, and the mark
formulas' fixed points."""
import numpy as np
import pytest
import scipy.special as sps

from oracle import hermes_oracle as O
from synthetic import catalogues as S


def test_density_at_equals_the_kernel_sum_over_neighbours():
    N, L, p = 16, 40.0, 3
    pos = S.mixed_poisson_sp(60, L, seed=31)
    w = S.lognormal_masses(pos.shape[0], seed=32).astype(np.float64)
    ev = pos[:6]
    for kind, R in (("sphere", 6.0), ("gauss", 3.0)):
        got = O.density_at(ev, pos, w, N, L, p, kind, R)
        kap = O.kappa_from_K(O.smoothing_window(N, L, p, kind, R)).real
        f, m = O.node_weights(pos, N, L, p)
        fe, me = O.node_weights(ev, N, L, p)
        ebar = w.sum() / N ** 3
        for i in range(len(ev)):
            ref = sum(w[j] * O.keff_pair_direct(kap, fe[i], me[i], f[j], m[j], N) for j in range(len(w))) / ebar
            assert got[i] == pytest.approx(ref, rel=1e-10, abs=1e-12)


def test_density_of_a_lattice_is_uniform_and_the_window_is_table_a1():
    N, L, p = 16, 32.0, 4
    g = (np.arange(N) * (L / N))
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ev = S.poisson_uniform(20, L, seed=4)
    np.testing.assert_allclose(O.density_at(ev, lat, None, N, L, p, "sphere", 5.0), 1.0, atol=1e-12)
    # row (b): the sphere transform at k = 2 pi / L along x, and the Gaussian row (c)
    k = 2 * np.pi / L
    ph = O.phi_hat_1d(N, p)[1]
    x = k * 5.0
    assert O.smoothing_window(N, L, p, "sphere", 5.0)[1, 0, 0] == pytest.approx(
        3 * (np.sin(x) - x * np.cos(x)) / x ** 3 * ph, rel=1e-12)
    assert O.smoothing_window(N, L, p, "gauss", 5.0)[0, 1, 0] == pytest.approx(np.exp(-0.5 * x * x) * ph, rel=1e-12)


def test_mark_formulas():
    rho = np.array([0.0, 0.5, 1.0, 3.0])
    np.testing.assert_allclose(O.density_marks(rho, "power", 0.0, 0.1), 1.0)         # alpha = 0: unmarked
    np.testing.assert_allclose(O.density_marks(rho, "power", 1.0, 0.1), rho + 0.1)
    np.testing.assert_allclose(O.density_marks(np.array([1.0]), "inverse", 2.0, 1.0), 1.0)  # mean density -> 1
    np.testing.assert_allclose(O.density_marks(rho, "inverse", 1.0, 1.0), 2.0 / (1.0 + rho))
    np.testing.assert_allclose(O.density_marks(rho, "power", 1.0, 0.0, self_count=0.7), np.maximum(rho - 0.7, 0))
