"""Pins of the oracle's axisymmetric (anisotropic 2PCF) windows, Sec. 3.4.4 and
Table A1 rows (f)-(i), against facts fixed independently of its quadrature:
closed forms printed in the paper, thin-bin limits, additivity of volume
averages, and brute-force pair sums with the spline-smeared kernel."""
import numpy as np
import pytest
import scipy.special as sps

from oracle import hermes_oracle as O
from synthetic import catalogues as S

K = np.concatenate([[0.0], np.geomspace(1e-3, 3.0, 40)])


def test_disk_is_the_table_a1_closed_form():
    # row (f)/(h): transverse filled disk 2 J_1(kR) / (kR)
    for R in (1.0, 7.5, 30.0):
        x = K * R
        ref = np.where(x > 0, 2.0 * sps.j1(x) / np.where(x > 0, x, 1.0), 1.0)
        np.testing.assert_allclose(O.annulus_avg_j0(K, 0.0, R), ref, rtol=1e-12, atol=1e-14)


def test_annulus_is_a_difference_of_bessel_integrals():
    # int_0^r rho J_0(k rho) d rho = r J_1(k r) / k, so the annulus average is fixed
    a, b = 4.0, 9.0
    k = K[1:]
    ref = (b * sps.j1(k * b) - a * sps.j1(k * a)) / k / (0.5 * (b * b - a * a))
    np.testing.assert_allclose(O.annulus_avg_j0(k, a, b), ref, rtol=1e-11, atol=1e-14)


def test_thin_ring_and_gaussian_ring_limits():
    R = 12.0
    for eps in (1e-2, 1e-3):
        got = O.annulus_avg_j0(K, R - eps, R + eps)
        assert np.max(np.abs(got - sps.j0(K * R))) < 5 * (K.max() * eps) ** 2
    sig = 5.0
    np.testing.assert_allclose(O.annulus_avg_j0(K, R, R, sig), sps.j0(K * R) * np.exp(-0.5 * (K * sig) ** 2),
                               rtol=1e-14, atol=1e-16)


def test_slab_pair_matches_the_finite_bin_product_form():
    # Sec. 3.4.4: sin(k D/2)/(k D/2) cos(k r_par) for the bin r_par +- D/2
    k = K[1:]
    for (a, b) in ((0.0, 10.0), (6.0, 8.0), (20.0, 35.0)):
        mid, d = 0.5 * (a + b), b - a
        ref = np.sin(0.5 * k * d) / (0.5 * k * d) * np.cos(k * mid)
        np.testing.assert_allclose(O.slab_avg_cos(k, a, b), ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(O.slab_avg_cos(K, 15.0, 15.0), np.cos(15.0 * K), rtol=0, atol=1e-15)  # row (i)


def test_volume_averages_are_additive():
    a, b, c = 2.0, 5.0, 11.0
    lhs = (b * b - a * a) * O.annulus_avg_j0(K, a, b) + (c * c - b * b) * O.annulus_avg_j0(K, b, c)
    np.testing.assert_allclose(lhs, (c * c - a * a) * O.annulus_avg_j0(K, a, c), rtol=1e-12, atol=1e-12)
    lhs = (b - a) * O.slab_avg_cos(K, a, b) + (c - b) * O.slab_avg_cos(K, b, c)
    np.testing.assert_allclose(lhs, (c - a) * O.slab_avg_cos(K, a, c), rtol=1e-12, atol=1e-12)


def test_window_is_unit_at_k0_zero_on_nyquist_and_half_matches_full():
    N, L, p = 16, 64.0, 4
    Kf = O.window_cyl(N, L, p, 3.0, 9.0, 2.0, 6.0)
    assert Kf[0, 0, 0] == pytest.approx(1.0, abs=1e-15)
    assert np.all(Kf[N // 2, :, :] == 0) and np.all(Kf[:, :, N // 2] == 0)
    Kh = O.window_cyl(N, L, p, 3.0, 9.0, 2.0, 6.0, half=True)
    np.testing.assert_allclose(Kh[:, :, : N // 2], Kf[:, :, : N // 2], rtol=0, atol=1e-15)
    # even in every component: the kernel is real and symmetric
    idx = (-np.arange(N)) % N
    np.testing.assert_allclose(Kf, Kf[idx][:, idx][:, :, idx], rtol=0, atol=1e-15)


def test_xi_cylinders_equals_brute_force_pair_sums():
    # the estimator is exactly the pair sum with the smeared kernel (reading 1)
    N, L, p = 16, 48.0, 3
    pos = S.mixed_poisson_sp(70, L, seed=12)
    w = S.lognormal_masses(pos.shape[0], seed=13)
    rperp, rpar = [2.0, 6.0, 11.0], [0.0, 4.0, 9.0]
    got = O.xi_cylinders(pos, w, N, L, p, rperp, rpar)
    for j, i in ((0, 1), (1, 0)):
        Kc = O.window_cyl(N, L, p, rperp[i], rperp[i + 1], rpar[j], rpar[j + 1])
        ref = O.xi_brute_force(pos, w, N, L, p, Kc)
        assert got[j, i] == pytest.approx(ref, rel=1e-9, abs=1e-12)
