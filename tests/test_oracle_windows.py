"""Pins of the oracle's Fourier conventions and window kernels.

Checks against: a direct O(N^6) DFT, Parseval, single-mode spikes, Table A1
rows (a)/(b), Eq. (Wshell_k), the thin-shell limit, a Si-function closed form of
the l=2 bin average, the spherical-harmonic addition theorem and low-order
explicit harmonics, and the continuum rotational average of two plane waves
(Eq. 2-fold-translation) done by quadrature over SO(3).
"""
import numpy as np
import pytest
import scipy.special as sps

from oracle import hermes_oracle as O


@pytest.mark.parametrize("N", [4, 8])
def test_forward_fft_matches_direct_dft(N):
    rng = np.random.default_rng(N)
    d = rng.standard_normal((N, N, N))
    got = O.forward(d)
    l = np.arange(N)
    ref = np.zeros((N, N, N), dtype=complex)
    for a in range(N):
        for b in range(N):
            for c in range(N):
                ph = np.exp(-2j * np.pi * (a * l[:, None, None] + b * l[None, :, None]
                                           + c * l[None, None, :]) / N)
                ref[a, b, c] = np.sum(d * ph)
    ref[0, 0, 0] = 0.0
    np.testing.assert_allclose(got, ref, atol=1e-12)


def test_parseval_and_single_mode():
    N = 16
    rng = np.random.default_rng(1)
    d = rng.standard_normal((N, N, N))
    d -= d.mean()
    dh = O.forward(d)
    assert np.sum(d * d) == pytest.approx(np.sum(np.abs(dh) ** 2) / N ** 3, rel=1e-12)
    l = np.arange(N)
    n0 = (1, 3, 2)
    d1 = np.cos(2 * np.pi * (n0[0] * l[:, None, None] + n0[1] * l[None, :, None]
                             + n0[2] * l[None, None, :]) / N)
    dh1 = O.forward(d1)
    assert dh1[n0] == pytest.approx(N ** 3 / 2)
    assert dh1[(-n0[0]) % N, (-n0[1]) % N, (-n0[2]) % N] == pytest.approx(N ** 3 / 2)
    mask = np.ones_like(dh1, dtype=bool)
    mask[n0] = False
    mask[(-n0[0]) % N, (-n0[1]) % N, (-n0[2]) % N] = False
    assert np.max(np.abs(dh1[mask])) < 1e-9


def test_shell_l0_table_a1_and_limits():
    k = np.linspace(1e-4, 3.0, 400)
    # a thin shell approaches sin(kR)/(kR), Table A1 row (a)
    R = 20.0
    w = O.shell_window_l0(k, R - 1e-3, R + 1e-3)
    np.testing.assert_allclose(w, np.sin(k * R) / (k * R), atol=1e-6)
    # a shell with r_lo = 0 is the top-hat sphere, Table A1 row (b)
    x = k * 7.0
    np.testing.assert_allclose(O.shell_window_l0(k, 0.0, 7.0),
                               3 * (np.sin(x) - x * np.cos(x)) / x ** 3, rtol=1e-9, atol=1e-12)
    # W^(0) = 1 for a normalised window
    assert O.shell_window_l0(np.array([0.0]), 5.0, 10.0)[0] == pytest.approx(1.0, abs=1e-15)


def test_bin_average_l0_quadrature_equals_closed_form():
    k = np.linspace(0.0, 2.8, 300)
    for lo, hi in [(5.0, 10.0), (2.0, 7.0), (0.0, 3.0), (100.0, 105.0)]:
        np.testing.assert_allclose(O.shell_avg_jl(0, k, lo, hi), O.shell_window_l0(k, lo, hi),
                                   rtol=1e-11, atol=1e-13)


def test_bin_average_l2_against_si_closed_form():
    # int_0^x t^2 j_2(t) dt = 3 Si(x) - 4 sin x + x cos x
    def F(x):
        si, _ = sps.sici(x)
        return 3 * si - 4 * np.sin(x) + x * np.cos(x)

    k = np.linspace(0.05, 2.8, 200)
    for lo, hi in [(5.0, 10.0), (20.0, 25.0), (2.0, 202.0)]:
        ref = 3 * (F(k * hi) - F(k * lo)) / (k ** 3 * (hi ** 3 - lo ** 3))
        np.testing.assert_allclose(O.shell_avg_jl(2, k, lo, hi), ref, rtol=1e-8, atol=1e-12)


def test_window_xi_conventions():
    N, L, p = 16, 100.0, 4
    K0 = O.window_xi(N, L, p, 10.0, 15.0, 0)
    assert K0[0, 0, 0] == pytest.approx(1.0, abs=1e-15)           # W^(0) Phi^(0) = 1
    h = N // 2
    assert np.all(K0[h, :, :] == 0) and np.all(K0[:, h, :] == 0) and np.all(K0[:, :, h] == 0)
    # real and even: K(-n) = K(n)
    idx = (-np.arange(N)) % N
    np.testing.assert_array_equal(K0, K0[idx][:, idx][:, :, idx])
    K2 = O.window_xi(N, L, p, 10.0, 15.0, 2)
    assert K2[0, 0, 0] == 0.0
    # l = 2 kernel along the line of sight: 5 * (-1) * <j_2> * L_2(1) * Phi^
    n = (0, 0, 3)
    k = 2 * np.pi * 3 / L
    ph = O.phi_hat_1d(N, p)
    expect = -5.0 * O.shell_avg_jl(2, np.array([k]), 10.0, 15.0)[0] * ph[3]
    assert K2[n] == pytest.approx(expect, rel=1e-12)
    # half-spectrum layout agrees with the full one
    Kh = O.window_xi(N, L, p, 10.0, 15.0, 2, half=True)
    np.testing.assert_array_equal(Kh[:, :, : h], K2[:, :, : h])


def test_phi_hat_is_ft_of_basis_autocorrelation():
    # Phi(d) = sum over lattice of M_2p; its DFT on a fine periodic lattice equals
    # sinc^{2p} summed over aliases; at low n the alias sum is dominated by the
    # unaliased term, which is what the oracle uses
    p, N = 4, 64
    d = np.arange(-p, p + 1)
    phi = O.bspline(2 * p, d.astype(float))        # M_p * M_p = M_2p sampled at lags
    n = np.arange(4)
    dft = np.array([np.sum(phi * np.cos(2 * np.pi * nn * d / N)) for nn in n])
    alias = np.zeros(len(n))
    for a in range(-50, 51):
        x = np.pi * (n / N + a)
        s = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1, x))
        alias += s ** (2 * p)
    np.testing.assert_allclose(dft, alias, rtol=1e-9)
    ph = O.phi_hat_1d(N, p)
    np.testing.assert_allclose(ph[n], alias, rtol=1e-6)


def test_spherical_harmonics_conventions():
    rng = np.random.default_rng(2)
    th = np.arccos(rng.uniform(-1, 1, 50))
    ph = rng.uniform(0, 2 * np.pi, 50)
    for ell in range(0, 7):
        s = sum(np.abs(sps.sph_harm_y(ell, m, th, ph)) ** 2 for m in range(-ell, ell + 1))
        np.testing.assert_allclose(s, (2 * ell + 1) / (4 * np.pi), rtol=1e-12)
    np.testing.assert_allclose(sps.sph_harm_y(1, 0, th, ph), np.sqrt(3 / (4 * np.pi)) * np.cos(th))
    np.testing.assert_allclose(sps.sph_harm_y(1, 1, th, ph),
                               -np.sqrt(3 / (8 * np.pi)) * np.sin(th) * np.exp(1j * ph))


def test_window_zeta_conjugation_identity():
    # K_{l,-m}(n) = (-1)^m conj(K_{l,m}(-n))
    N, L, p = 8, 60.0, 4
    idx = (-np.arange(N)) % N
    for ell, m in [(1, 1), (2, 1), (2, 2), (3, 2), (4, 3)]:
        Kp = O.window_zeta(N, L, p, 8.0, 14.0, ell, m)
        Km = O.window_zeta(N, L, p, 8.0, 14.0, ell, -m)
        ref = (-1) ** m * np.conj(Kp[idx][:, idx][:, :, idx])
        np.testing.assert_allclose(Km, ref, atol=1e-13)


def _rot_average_quadrature(k1, r1vec, k2, r2vec, n=48):
    """<exp(i k1.R r1) exp(i k2.R r2)> over SO(3) by a product Gauss rule in Euler angles."""
    xa = np.linspace(0, 2 * np.pi, n, endpoint=False)
    xb, wb = np.polynomial.legendre.leggauss(n)            # cos(beta)
    tot = 0.0
    for al in xa:
        for cb, wgt in zip(xb, wb):
            sb = np.sqrt(1 - cb * cb)
            ga = xa
            ca, sa = np.cos(al), np.sin(al)
            cg, sg = np.cos(ga), np.sin(ga)
            # R = Rz(al) Ry(beta) Rz(ga), applied to both vectors
            def rot(v):
                x1 = cg * v[0] - sg * v[1]
                y1 = sg * v[0] + cg * v[1]
                z1 = v[2] * np.ones_like(ga)
                x2 = cb * x1 + sb * z1
                z2 = -sb * x1 + cb * z1
                return ca * x2 - sa * y1, sa * x2 + ca * y1, z2
            a = rot(r1vec)
            b = rot(r2vec)
            ph = (k1[0] * a[0] + k1[1] * a[1] + k1[2] * a[2]
                  + k2[0] * b[0] + k2[1] * b[1] + k2[2] * b[2])
            tot += wgt * np.sum(np.exp(1j * ph))
    return tot / (2.0 * n * n)


def test_two_fold_rotational_average_sign_and_normalisation():
    # Eq. (2-fold-translation) with conj on the first field's kernel at -k1:
    # <e^{ik1.r1} e^{ik2.r2}>_rot = sum_l L_l(r1^.r2^) (1/4pi) sum_m conj(W1(-k1)) W2(k2)
    k1 = np.array([0.3, -0.2, 0.25])
    k2 = np.array([-0.1, 0.35, 0.15])
    r1, r2, th = 4.0, 6.0, 1.1
    r1v = np.array([0.0, 0.0, r1])
    r2v = r2 * np.array([np.sin(th), 0.0, np.cos(th)])
    lhs = _rot_average_quadrature(k1, r1v, k2, r2v)

    def W(kv, r, ell, m):
        kk = np.linalg.norm(kv)
        t = np.arccos(kv[2] / kk)
        f = np.mod(np.arctan2(kv[1], kv[0]), 2 * np.pi)
        return 4 * np.pi * (1j ** ell) * sps.spherical_jn(ell, kk * r) * sps.sph_harm_y(ell, m, t, f)

    rhs = 0.0
    for ell in range(0, 25):
        s = sum(np.conj(W(-k1, r1, ell, m)) * W(k2, r2, ell, m) for m in range(-ell, ell + 1))
        rhs += sps.eval_legendre(ell, np.cos(th)) * s / (4 * np.pi)
    assert abs(lhs - rhs) < 1e-9
    # and the reading "conjugate the kernel at +k1" is off by (-1)^l for odd l
    wrong = 0.0
    for ell in range(0, 25):
        s = sum(np.conj(W(k1, r1, ell, m)) * W(k2, r2, ell, m) for m in range(-ell, ell + 1))
        wrong += sps.eval_legendre(ell, np.cos(th)) * s / (4 * np.pi)
    assert abs(lhs - wrong) > 1e-3


def test_mode_count_golden():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mode_counts.json")))
    for c in g["cases"]:
        assert len(O.lm_modes(c["l_max"])) == c["n_m"]


def test_window_xi_is_the_legendre_projected_translation_average():
    # K_l(n)/Phi^(n) = <(2l+1)/2 int dmu_r L_l(mu_r) <e^{ik.r}>_phi_r>_{r in bin}, by quadrature
    N, L, p = 16, 100.0, 4
    lo, hi = 10.0, 16.0
    n = (2, -1, 3)
    kv = 2 * np.pi * np.array(n) / L
    ph = O.phi_hat_1d(N, p)
    phin = ph[n[0] % N] * ph[n[1] % N] * ph[n[2] % N]
    xr, wr = np.polynomial.legendre.leggauss(24)
    rr = 0.5 * (hi - lo) * xr + 0.5 * (hi + lo)
    wrr = 0.5 * (hi - lo) * wr * rr ** 2 / ((hi ** 3 - lo ** 3) / 3)
    xm, wm = np.polynomial.legendre.leggauss(64)
    phis = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    for ell in (0, 2, 4):
        K = O.window_xi(N, L, p, lo, hi, ell)[tuple(x % N for x in n)]
        tot = 0.0
        for r, wgt in zip(rr, wrr):
            s = np.sqrt(1 - xm ** 2)
            dirs = np.stack([s[:, None] * np.cos(phis), s[:, None] * np.sin(phis),
                             xm[:, None] * np.ones_like(phis)], axis=-1)
            e = np.exp(1j * r * (dirs @ kv)).mean(axis=1)          # phi average
            tot += wgt * (2 * ell + 1) / 2 * np.sum(wm * sps.eval_legendre(ell, xm) * e)
        assert K / phin == pytest.approx(tot.real, rel=1e-9, abs=1e-12)
        assert abs(tot.imag) < 1e-12


def test_window_zeta_reproduces_rotational_average_on_the_grid():
    # sum_l L_l(cos th) (1/4pi) sum_m conj(K1_lm(-n1)) K2_lm(n2)
    #   = Phi^(n1) Phi^(n2) < <e^{ik1.r1} e^{ik2.r2}>_rot >_{r1 in b1, r2 in b2}
    N, L, p = 16, 200.0, 4
    n1, n2 = (1, -1, 1), (0, 1, 2)
    b1, b2 = (6.0, 9.0), (10.0, 14.0)
    th = 0.9
    ph = O.phi_hat_1d(N, p)
    k1 = 2 * np.pi * np.array(n1) / L
    k2 = 2 * np.pi * np.array(n2) / L
    rhs = 0.0
    for ell in range(0, 12):
        s = 0.0
        for m in range(-ell, ell + 1):
            K1 = O.window_zeta(N, L, p, b1[0], b1[1], ell, m)
            K2 = O.window_zeta(N, L, p, b2[0], b2[1], ell, m)
            s += np.conj(K1[tuple((-x) % N for x in n1)]) * K2[tuple(x % N for x in n2)]
        rhs += sps.eval_legendre(ell, np.cos(th)) * s / (4 * np.pi)
    xr, wr = np.polynomial.legendre.leggauss(6)

    def nodes(lo, hi):
        r = 0.5 * (hi - lo) * xr + 0.5 * (hi + lo)
        return r, 0.5 * (hi - lo) * wr * r ** 2 / ((hi ** 3 - lo ** 3) / 3)

    lhs = 0.0
    for r1, w1 in zip(*nodes(*b1)):
        for r2, w2 in zip(*nodes(*b2)):
            lhs += w1 * w2 * _rot_average_quadrature(
                k1, np.array([0, 0, r1]), k2, r2 * np.array([np.sin(th), 0, np.cos(th)]), n=24)
    phi12 = (ph[n1[0] % N] * ph[n1[1] % N] * ph[n1[2] % N]
             * ph[n2[0] % N] * ph[n2[1] % N] * ph[n2[2] % N])
    assert abs(rhs - phi12 * lhs) < 1e-9
