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


def _modes(N, L):
    f = O.signed_freqs(N)
    nx, ny, nz = np.meshgrid(f, f, f, indexing="ij")
    kf = 2.0 * np.pi / L
    nyq = (np.abs(nx) == N // 2) | (np.abs(ny) == N // 2) | (np.abs(nz) == N // 2)
    return kf * np.sqrt(nx ** 2 + ny ** 2), kf * nz, nyq


def test_thin_ring_is_table_a1_row_i():
    # J_0(k_perp R) cos(k_par H) Phi^, written out here from the printed closed form
    N, L, p = 16, 64.0, 4
    kp, kz, nyq = _modes(N, L)
    ph = O.phi_hat_1d(N, p)
    phi3 = ph[:, None, None] * ph[None, :, None] * ph[None, None, :]
    for R, H in ((7.0, 3.0), (0.0, 10.0), (12.5, 0.0)):
        ref = np.where(nyq, 0.0, sps.j0(kp * R) * np.cos(kz * H) * phi3)
        np.testing.assert_allclose(O.window_ring(N, L, p, R, H), ref, rtol=1e-13, atol=1e-15)


def test_finite_ring_is_the_printed_finite_bin_form():
    # Sec. 3.4.4: sin(k_par D/2)/(k_par D/2) cos(k_par r_par) <J_0(k_perp r_perp)>_{Delta r_perp},
    # <J_0> = 1/(r_perp Delta) int rho J_0 d rho = [rho J_1(k rho) / k] / (r_perp Delta)
    N, L, p = 16, 64.0, 4
    kp, kz, nyq = _modes(N, L)
    ph = O.phi_hat_1d(N, p)
    phi3 = ph[:, None, None] * ph[None, :, None] * ph[None, None, :]
    R, dR, H, dH = 9.0, 3.0, 6.0, 2.0
    a, b = R - dR / 2, R + dR / 2
    with np.errstate(invalid="ignore", divide="ignore"):
        j0avg = np.where(kp > 0, (b * sps.j1(kp * b) - a * sps.j1(kp * a)) / kp / (R * dR), 1.0)
        los = np.where(kz != 0, np.sin(0.5 * kz * dH) / (0.5 * kz * dH), 1.0) * np.cos(kz * H)
    ref = np.where(nyq, 0.0, j0avg * los * phi3)
    np.testing.assert_allclose(O.window_ring(N, L, p, R, H, dR, dH), ref, rtol=1e-11, atol=1e-14)


def test_ring_bins_clipped_at_zero_are_the_disk_and_filled_slab():
    # a ring whose bins reach below zero covers [0, R + dR/2] and |z| in [0, H + dH/2]
    N, L, p = 16, 64.0, 4
    got = O.window_ring(N, L, p, 1.0, 0.5, 4.0, 3.0)
    np.testing.assert_allclose(got, O.window_cyl(N, L, p, 0.0, 3.0, 0.0, 2.0), rtol=0, atol=1e-15)


def test_xi_rings_equal_brute_force_pair_sums():
    N, L, p = 16, 48.0, 3
    pos = S.mixed_poisson_sp(60, L, seed=14)
    w = S.lognormal_masses(pos.shape[0], seed=15)
    R, H, dR, dH = [4.0, 7.0], [2.0, 5.0], [0.0, 2.0], [0.0, 3.0]
    got = O.xi_rings(pos, w, N, L, p, R, H, dR, dH)
    for i in range(2):
        Kr = O.window_ring(N, L, p, R[i], H[i], dR[i], dH[i])
        assert got[i] == pytest.approx(O.xi_brute_force(pos, w, N, L, p, Kr), rel=1e-9, abs=1e-12)
