"""FP64 CPU oracle of the field-window estimator -- TEST INFRASTRUCTURE ONLY.

This module is the parity reference for the CUDA path.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product path never calls it.  It shares no code with the CUDA library:
its inputs come from ``synthetic/`` and everything else is computed here, in
float64, by the plainest route that follows the paper:

  step                          paper passage
  ----------------------------  ---------------------------------------------------
  node / fraction rule          Eq. (phi_projection) with a centred order-p B-spline
  B-spline scatter  eps_l       Eq. (phi_projection): eps_l = sum_i w_i phi_l(x_i)
  density contrast  delta       delta = n / nbar - 1 (Sec. 2, notation)
  forward FFT                   non-unitary convention f^(k) = int f e^{-ik.x} (Sec. 2)
  basis autocorrelation  Phi^   Sec. 3.5 window construction, K_W = W^ Phi^
  shell window (l = 0)          Eq. (Wshell_k) difference of two top-hats
  multipole shell  (xi_l)       Sec. 3.4.3: (2l+1) i^l j_l(kr) L_l(mu_k); finite bin
                                = radial average of j_l
  harmonic shell   (zeta_l)     Eq. (multipole-window): 4 pi i^l j_l(kr) Y_lm(k^)
  xi via Parseval               Eq. (pair-counting-kspace)
  xi via cell contraction       Eq. (pair-counting), Eq. (2rdEs)
  Landy-Szalay with uniform R   Eq. (xi-deltaDD-over-RR)
  zeta_l                        Eq. (2-fold-translation), Eq. (particle_nfold)
  density-dependent marks       Sec. 3.3: smoothed density read at the particles (the
                                adjoint of the scatter), Eq. (power-law-mark),
                                Eq. (inverse-density-mark)
  explicit randoms (LS)         Sec. 3.3 estimator: Delta = D - R, xi = Delta DD / RR,
                                Eq. (xi-deltaDD-over-RR) with a random field
  anisotropic xi(r_perp, r_par) Sec. 3.4.4 ring window with finite bins; Table A1 rows
                                (f)-(i): separable transverse x line-of-sight windows
  3PCF monopole DDD             Eq. (3PCF-ddd-monopole) two-fold coefficients through the
                                triple connection coefficients of Eq. (con-coeff), then
                                Eq. (DDD-vector-product)

Readings of silent or ambiguous points (all restated in the design notes):
  * basis: centred cardinal B-spline M_p on unit cell spacing, partition of unity;
  * node rule: u = fl32(x * fl32(N/L)); for odd p, v = fl32(u + 0.5) else v = u;
    i = floor(v); t = v - i; first node i - (p/2 - 1) (even p) or i - (p-1)/2 (odd p);
  * Phi^(n) = prod_d sinc^{2p}(pi n_d / N), unaliased; K = 0 on every Nyquist plane;
  * delta^(0) := 0;
  * finite-bin j_l = r^2-weighted (volume) average over [r_lo, r_hi);
  * the exact self-pair term SN is subtracted from xi and xi_l;
  * zeta_l are Legendre coefficients, computed with conj(a) on the first field,
    returned raw (self terms included), normalised by 1/(4 pi N^3).

Every function here is pinned by ``tests/test_oracle_*.py`` against facts the
paper or mathematics fixes (closed forms, identities, brute force).  No function
is "parity unpinned".
"""
from __future__ import annotations

from math import comb, factorial

import numpy as np
import scipy.special as sps

__all__ = [
    "scale_f32", "node_rule", "bspline", "node_weights", "assign", "delta_from_eps",
    "signed_freqs", "phi_hat_1d", "shell_avg_jl", "shell_window_l0", "window_xi",
    "window_zeta", "xi_parseval", "xi_cell_contraction", "self_pair_table",
    "kappa_from_K", "shot_noise", "xi_multipoles", "zeta_multipoles", "lm_modes",
    "keff_pair_direct", "xi_brute_force", "direct_convolution", "annulus_avg_j0", "slab_avg_cos",
    "window_cyl", "xi_cylinders", "xi_randoms", "smoothing_window", "density_at", "density_marks",
    "window_xi_at", "window_zeta_at", "planted_xi", "planted_zeta", "window_ring", "xi_rings",
    "triple_overlap_1d", "connection_coefficients", "ddd_from_fields", "ddd_monopole", "planted_ddd",
]


# --------------------------------------------------------------------------
# (a1) index bookkeeping
# --------------------------------------------------------------------------
def scale_f32(N: int, L: float) -> np.float32:
    """Grid units per length unit, N/L computed in float64 and rounded to float32."""
    return np.float32(float(N) / float(L))


def node_rule(pos: np.ndarray, N: int, L: float, p: int):
    """Return (first_node[n,3] int64 in [0,N), dist[n,3,p] float64).

    dist[i, d, o] = u_{i,d} - (first + o) is the signed offset of point i from
    its o-th supporting node along axis d, in grid units.  The rule follows the
    compact support of phi_{jl} in Eq. (phi_projection): exactly the p nodes
    with |u - l| < p/2 carry weight.
    """
    s = scale_f32(N, L)
    u = np.asarray(pos, dtype=np.float32) * s            # IEEE float32 multiply
    if p % 2 == 1:
        v = u + np.float32(0.5)                          # float32 add
    else:
        v = u
    fl = np.floor(v)
    i0 = fl.astype(np.int64)
    t = (v - fl).astype(np.float64)                      # exact in float32
    if p % 2 == 0:
        first = i0 - (p // 2 - 1)
        base = t + (p // 2 - 1)
    else:
        first = i0 - (p - 1) // 2
        base = t - 0.5 + (p - 1) // 2
    o = np.arange(p, dtype=np.float64)
    dist = base[..., None] - o                           # [n,3,p]
    return np.mod(first, N), dist


def bspline(p: int, x: np.ndarray) -> np.ndarray:
    """Centred cardinal B-spline M_p(x) of order p (degree p-1), float64.

    Written as the truncated-power sum
        M_p(x) = 1/(p-1)! * sum_{k=0}^{p} (-1)^k C(p,k) (x + p/2 - k)_+^{p-1},
    the textbook closed form of p-fold convolution of the unit box, evaluated
    at -|x| (M_p is even).
    """
    x = np.asarray(x, dtype=np.float64)
    if p == 1:
        return np.where((x >= -0.5) & (x < 0.5), 1.0, 0.0)
    # M_p is even; evaluating at -|x| makes only the k = 0 term survive near the
    # support edge, which avoids cancellation between large terms there
    xa = -np.abs(x)
    acc = np.zeros_like(x)
    for k in range(p + 1):
        y = xa + p / 2.0 - k
        acc += (-1) ** k * comb(p, k) * np.where(y > 0, y, 0.0) ** (p - 1)
    out = acc / factorial(p - 1)
    # outside the support the sum cancels to rounding noise; make it exact
    return np.where(np.abs(x) < p / 2.0, out, 0.0)


def node_weights(pos, N, L, p):
    """(first_node[n,3], m[n,3,p]) with m = M_p(dist): phi_{jl}(x_i) per axis."""
    first, dist = node_rule(pos, N, L, p)
    return first, bspline(p, dist)


# --------------------------------------------------------------------------
# (a2) scatter, Eq. (phi_projection)
# --------------------------------------------------------------------------
def assign(pos, w, N: int, L: float, p: int, chunk: int = 400_000):
    """eps_l = sum_i w_i prod_d M_p(u_{i,d} - l_d) on the periodic N^3 grid.

    Returns (eps[N,N,N] float64, sum_w, sum_w2).  w=None means unit weights.
    """
    pos = np.asarray(pos)
    n = pos.shape[0]
    w = np.ones(n, dtype=np.float64) if w is None else np.asarray(w, dtype=np.float64)
    eps = np.zeros(N ** 3, dtype=np.float64)
    for s0 in range(0, n, chunk):
        first, m = node_weights(pos[s0:s0 + chunk], N, L, p)
        ww = w[s0:s0 + chunk]
        o = np.arange(p)
        ix = (first[:, 0, None] + o) % N                 # [c,p]
        iy = (first[:, 1, None] + o) % N
        iz = (first[:, 2, None] + o) % N
        flat = (ix[:, :, None, None] * N + iy[:, None, :, None]) * N + iz[:, None, None, :]
        val = (ww[:, None, None, None] * m[:, 0, :, None, None]
               * m[:, 1, None, :, None] * m[:, 2, None, None, :])
        eps += np.bincount(flat.ravel(), weights=val.ravel(), minlength=N ** 3)
    return eps.reshape(N, N, N), float(w.sum()), float((w * w).sum())


def delta_from_eps(eps, sum_w):
    """delta = eps / eps_bar - 1 with eps_bar = sum_w / N^3 (uniform random field)."""
    N3 = eps.size
    return eps / (sum_w / N3) - 1.0


# --------------------------------------------------------------------------
# Fourier-space windows
# --------------------------------------------------------------------------
def signed_freqs(N: int) -> np.ndarray:
    """Integer frequencies n in FFT order: 0, 1, ..., N/2-1, -N/2, ..., -1."""
    return np.rint(np.fft.fftfreq(N, d=1.0 / N)).astype(np.int64)


def phi_hat_1d(N: int, p: int) -> np.ndarray:
    """sinc^{2p}(pi n / N) in FFT order: FT of the autocorrelation M_p * M_p = M_2p."""
    n = signed_freqs(N).astype(np.float64)
    x = np.pi * n / N
    s = np.ones_like(x)
    nz = x != 0
    s[nz] = np.sin(x[nz]) / x[nz]
    return s ** (2 * p)


def _gl_nodes(m):
    x, wt = np.polynomial.legendre.leggauss(m)
    return x, wt


def shell_avg_jl(ell: int, k: np.ndarray, r_lo: float, r_hi: float, panels: int | None = None):
    """r^2-weighted average of j_l(k r) over r in [r_lo, r_hi] (float64).

    Composite 16-point Gauss-Legendre in r; the number of panels keeps the
    phase advance k*dr per panel below ~1.5 rad so the rule is exact to
    float64 rounding.  j_l from scipy (library routine).
    """
    k = np.asarray(k, dtype=np.float64)
    if panels is None:
        kmax = float(np.max(k)) if k.size else 0.0
        panels = max(1, int(np.ceil(kmax * (r_hi - r_lo) / 1.5)))
    x, wt = _gl_nodes(16)
    edges = np.linspace(r_lo, r_hi, panels + 1)
    num = np.zeros_like(k)
    for a, b in zip(edges[:-1], edges[1:]):
        r = 0.5 * (b - a) * x + 0.5 * (a + b)
        rw = 0.5 * (b - a) * wt * r * r
        num += (sps.spherical_jn(ell, k[..., None] * r) * rw).sum(axis=-1)
    den = (r_hi ** 3 - r_lo ** 3) / 3.0
    return num / den


def _sphere_hat(x):
    """3 (sin x - x cos x) / x^3 (Table A1 row b), with its Taylor series at small x."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    sm = np.abs(x) < 1e-2
    xs = x[sm]
    out[sm] = 1.0 - xs ** 2 / 10.0 + xs ** 4 / 280.0 - xs ** 6 / 15120.0
    xl = x[~sm]
    out[~sm] = 3.0 * (np.sin(xl) - xl * np.cos(xl)) / xl ** 3
    return out


def shell_window_l0(k, r_lo, r_hi):
    """Eq. (Wshell_k): volume-normalised difference of two spherical top-hats."""
    vp, vm = r_hi ** 3, r_lo ** 3
    return (vp * _sphere_hat(k * r_hi) - vm * _sphere_hat(k * r_lo)) / (vp - vm)


def _mode_grid(N, L, half=False):
    """Signed integer modes (n_x, n_y, n_z), |n|^2, |k| and the Nyquist mask.

    half=True keeps n_z in [0, N/2] only (the layout of a real-to-complex FFT).
    """
    n = signed_freqs(N)
    nzs = np.arange(N // 2 + 1, dtype=np.int64) if half else n
    nx, ny, nz = np.meshgrid(n, n, nzs, indexing="ij")
    nyq = (np.abs(nx) == N // 2) | (np.abs(ny) == N // 2) | (np.abs(nz) == N // 2)
    q = nx * nx + ny * ny + nz * nz
    k = (2.0 * np.pi / L) * np.sqrt(q.astype(np.float64))
    return nx, ny, nz, q, k, nyq


def _radial_table(ell, q, L, r_lo, r_hi):
    """<j_l>_bin(k) at every mode, k = 2 pi |n| / L.

    l = 0 uses the closed form of Eq. (Wshell_k) mode by mode; l > 0 evaluates
    the quadrature once per distinct |n|^2 and scatters it back.
    """
    if ell == 0:
        return shell_window_l0((2.0 * np.pi / L) * np.sqrt(q.astype(np.float64)), r_lo, r_hi)
    uq, inv = np.unique(q.ravel(), return_inverse=True)
    ku = (2.0 * np.pi / L) * np.sqrt(uq.astype(np.float64))
    vals = shell_avg_jl(ell, ku, r_lo, r_hi)
    return vals[inv].reshape(q.shape)


def window_xi(N: int, L: float, p: int, r_lo: float, r_hi: float, ell: int,
              half: bool = False) -> np.ndarray:
    """K_{b,l}(n) = (2l+1) i^l <j_l>_b(k) L_l(k_z/k) Phi^(n) for even l (real), Nyquist = 0.

    l = 0 is the finite shell of Eq. (Wshell_k); the line of sight is the z axis.
    half=True returns only n_z in [0, N/2] (rfft layout).
    """
    if ell % 2:
        raise ValueError("odd l gives an identically zero auto-multipole")
    nx, ny, nz, q, k, nyq = _mode_grid(N, L, half)
    rad = _radial_table(ell, q, L, r_lo, r_hi)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(q > 0, nz / np.sqrt(q.astype(np.float64)), 0.0)
    leg = sps.eval_legendre(ell, mu)
    ph = phi_hat_1d(N, p)
    phz = ph[: N // 2 + 1] if half else ph
    phz = phz.copy()
    if half:
        phz[N // 2] = ph[N // 2]                       # n_z = +N/2 equals -N/2 in magnitude
    phi3 = ph[:, None, None] * ph[None, :, None] * phz[None, None, :]
    K = (2 * ell + 1) * np.real(1j ** ell) * rad * leg * phi3
    K[nyq] = 0.0
    return K


def annulus_avg_j0(k, a: float, b: float, sigma: float = 0.0):
    """Area-weighted average of J_0(k rho) over the annulus a <= rho < b (the finite-bin
    transverse ring factor of Sec. 3.4.4), times exp(-k^2 sigma^2 / 2) (Gaussian ring).

    a = b is the thin ring J_0(k a); a = 0 the filled disk.  Composite 16-point
    Gauss-Legendre in rho with the phase advance per panel below 1.5 rad; J_0 from
    scipy (library routine).
    """
    k = np.asarray(k, dtype=np.float64)
    g = np.exp(-0.5 * (k * sigma) ** 2)
    if b - a <= 0.0:
        return sps.j0(k * a) * g
    kmax = float(np.max(k)) if k.size else 0.0
    panels = max(1, int(np.ceil(kmax * (b - a) / 1.5)))
    x, wt = _gl_nodes(16)
    edges = np.linspace(a, b, panels + 1)
    num = np.zeros_like(k)
    for lo, hi in zip(edges[:-1], edges[1:]):
        r = 0.5 * (hi - lo) * x + 0.5 * (lo + hi)
        num += (sps.j0(k[..., None] * r) * (0.5 * (hi - lo) * wt * r)).sum(axis=-1)
    return num / (0.5 * (b * b - a * a)) * g


def slab_avg_cos(k, a: float, b: float):
    """Average of cos(k z) over the pair of slabs a <= |z| < b (the line-of-sight factor
    of the finite-bin ring window, Sec. 3.4.4); a = b is the double delta cos(k a),
    a = 0 the filled slab.  16-point Gauss-Legendre panels as annulus_avg_j0."""
    k = np.asarray(k, dtype=np.float64)
    if b - a <= 0.0:
        return np.cos(k * a)
    kmax = float(np.max(np.abs(k))) if k.size else 0.0
    panels = max(1, int(np.ceil(kmax * (b - a) / 1.5)))
    x, wt = _gl_nodes(16)
    edges = np.linspace(a, b, panels + 1)
    num = np.zeros_like(k)
    for lo, hi in zip(edges[:-1], edges[1:]):
        z = 0.5 * (hi - lo) * x + 0.5 * (lo + hi)
        num += (np.cos(k[..., None] * z) * (0.5 * (hi - lo) * wt)).sum(axis=-1)
    return num / (b - a)


def window_cyl(N: int, L: float, p: int, rp_lo: float, rp_hi: float, rz_lo: float, rz_hi: float,
               sigma_perp: float = 0.0, half: bool = False) -> np.ndarray:
    """K(n) = <J_0>_annulus(k_perp) <cos>_slabs(k_par) Phi^(n), Nyquist = 0; line of sight z.

    The separable axisymmetric window of Sec. 3.4.4 / Table A1 (f)-(i) with finite
    transverse and line-of-sight bins, evaluated once per distinct n_x^2 + n_y^2 and |n_z|.
    """
    nx, ny, nz, q, k, nyq = _mode_grid(N, L, half)
    qp = nx * nx + ny * ny
    uq, inv = np.unique(qp.ravel(), return_inverse=True)
    tperp = annulus_avg_j0((2.0 * np.pi / L) * np.sqrt(uq.astype(np.float64)), rp_lo, rp_hi, sigma_perp)
    uz, invz = np.unique(np.abs(nz).ravel(), return_inverse=True)
    tpar = slab_avg_cos((2.0 * np.pi / L) * uz.astype(np.float64), rz_lo, rz_hi)
    ph = phi_hat_1d(N, p)
    phz = ph[: N // 2 + 1].copy() if half else ph
    if half:
        phz[N // 2] = ph[N // 2]
    phi3 = ph[:, None, None] * ph[None, :, None] * phz[None, None, :]
    K = tperp[inv].reshape(q.shape) * tpar[invz].reshape(q.shape) * phi3
    K[nyq] = 0.0
    return K


def xi_cylinders(pos, w, N, L, p, rperp_edges, rpar_edges, sigma_perp=0.0):
    """xi(r_perp, r_par) for every (line-of-sight bin j, transverse bin i): Parseval on the
    full spectrum minus the exact self-pair term.  Returns [n_par][n_perp]."""
    eps, sw, _ = assign(pos, w, N, L, p)
    delta = delta_from_eps(eps, sw)
    dh = forward(delta)
    S = self_pair_table(pos, w, N, L, p)
    npar, nperp = len(rpar_edges) - 1, len(rperp_edges) - 1
    out = np.zeros((npar, nperp))
    for j in range(npar):
        for i in range(nperp):
            K = window_cyl(N, L, p, rperp_edges[i], rperp_edges[i + 1], rpar_edges[j], rpar_edges[j + 1],
                           sigma_perp)
            out[j, i] = xi_parseval(dh, K) - shot_noise(S, K, N, sw)
    return out


def window_ring(N: int, L: float, p: int, R: float, H: float, dR: float = 0.0, dH: float = 0.0,
                sigma_perp: float = 0.0, half: bool = False) -> np.ndarray:
    """Ring window at (r_perp, r_par) = (R, H), Sec. 3.4.4 and Table A1 row (i).

    Thin (dR = dH = 0): J_0(k_perp R) cos(k_par H) Phi^.  Finite widths: the
    axisymmetric window of the transverse bin R +- dR/2 and the line-of-sight bin
    H +- dH/2, each clipped at 0 (the separations pairs can have), which is the
    printed form sin(k dH/2)/(k dH/2) cos(k H) <J_0>_dR whenever the bins stay above 0.
    """
    return window_cyl(N, L, p, max(0.0, R - 0.5 * dR), R + 0.5 * dR, max(0.0, H - 0.5 * dH), H + 0.5 * dH,
                      sigma_perp, half)


def xi_rings(pos, w, N, L, p, R, H, dR=None, dH=None, sigma_perp=0.0):
    """xi for every ring window (R_i, H_i, dR_i, dH_i): Parseval on the full spectrum minus the
    exact self-pair term.  Widths None mean thin rings.  Returns [n]."""
    eps, sw, _ = assign(pos, w, N, L, p)
    delta = delta_from_eps(eps, sw)
    dh = forward(delta)
    S = self_pair_table(pos, w, N, L, p)
    n = len(R)
    dR = np.zeros(n) if dR is None else np.broadcast_to(np.asarray(dR, dtype=np.float64), (n,))
    dH = np.zeros(n) if dH is None else np.broadcast_to(np.asarray(dH, dtype=np.float64), (n,))
    out = np.zeros(n)
    for i in range(n):
        K = window_ring(N, L, p, R[i], H[i], dR[i], dH[i], sigma_perp)
        out[i] = xi_parseval(dh, K) - shot_noise(S, K, N, sw)
    return out


def window_zeta(N: int, L: float, p: int, r_lo: float, r_hi: float, ell: int, m: int) -> np.ndarray:
    """K_{b,lm}(n) = 4 pi i^l <j_l>_b(k) Y_lm(k^) Phi^(n), Eq. (multipole-window); complex.

    Y_lm orthonormal with the Condon-Shortley phase (scipy.special.sph_harm_y);
    Nyquist planes are zero.  At n = 0 the direction is taken as +z (the
    value multiplies delta^(0) = 0 and never matters).
    """
    nx, ny, nz, q, k, nyq = _mode_grid(N, L)
    rad = _radial_table(ell, q, L, r_lo, r_hi)
    r = np.sqrt(q.astype(np.float64))
    with np.errstate(invalid="ignore", divide="ignore"):
        ct = np.where(q > 0, nz / r, 1.0)
    theta = np.arccos(np.clip(ct, -1.0, 1.0))
    phi = np.mod(np.arctan2(ny.astype(np.float64), nx.astype(np.float64)), 2 * np.pi)
    Y = sps.sph_harm_y(ell, m, theta, phi)
    ph = phi_hat_1d(N, p)
    phi3 = ph[:, None, None] * ph[None, :, None] * ph[None, None, :]
    K = 4.0 * np.pi * (1j ** ell) * rad * Y * phi3
    K[nyq] = 0.0
    return K


def _modes_at(N: int, L: float, p: int, modes):
    """Signed integer modes n [m,3], |n|^2, |k|, Phi^(n) and the Nyquist mask of a mode list."""
    n = np.asarray(modes, dtype=np.int64).reshape(-1, 3)
    q = np.sum(n * n, axis=1)
    k = (2.0 * np.pi / L) * np.sqrt(q.astype(np.float64))
    ph = phi_hat_1d(N, p)
    phi3 = ph[n[:, 0] % N] * ph[n[:, 1] % N] * ph[n[:, 2] % N]
    nyq = np.any(np.abs(n) == N // 2, axis=1)
    return n, q, k, phi3, nyq


def window_xi_at(N: int, L: float, p: int, r_lo: float, r_hi: float, ell: int, modes) -> np.ndarray:
    """window_xi evaluated only at the listed signed modes (for grids too large to tabulate).

    Same definition: (2l+1) i^l <j_l>_b(k) L_l(n_z/|n|) Phi^(n), zero on Nyquist planes;
    <j_l>_b by Eq. (Wshell_k) for l = 0 and by the Gauss-Legendre average otherwise.
    """
    if ell % 2:
        raise ValueError("odd l gives an identically zero auto-multipole")
    n, q, k, phi3, nyq = _modes_at(N, L, p, modes)
    rad = shell_window_l0(k, r_lo, r_hi) if ell == 0 else shell_avg_jl(ell, k, r_lo, r_hi)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(q > 0, n[:, 2] / np.sqrt(q.astype(np.float64)), 0.0)
    K = (2 * ell + 1) * np.real(1j ** ell) * rad * sps.eval_legendre(ell, mu) * phi3
    return np.where(nyq, 0.0, K)


def window_zeta_at(N: int, L: float, p: int, r_lo: float, r_hi: float, ell: int, m: int, modes) -> np.ndarray:
    """window_zeta evaluated only at the listed signed modes: 4 pi i^l <j_l>_b Y_lm(k^) Phi^."""
    n, q, k, phi3, nyq = _modes_at(N, L, p, modes)
    rad = shell_window_l0(k, r_lo, r_hi) if ell == 0 else shell_avg_jl(ell, k, r_lo, r_hi)
    r = np.sqrt(q.astype(np.float64))
    with np.errstate(invalid="ignore", divide="ignore"):
        ct = np.where(q > 0, n[:, 2] / r, 1.0)
    theta = np.arccos(np.clip(ct, -1.0, 1.0))
    phi = np.mod(np.arctan2(n[:, 1].astype(np.float64), n[:, 0].astype(np.float64)), 2 * np.pi)
    K = 4.0 * np.pi * (1j ** ell) * rad * sps.sph_harm_y(ell, m, theta, phi) * phi3
    return np.where(nyq, 0.0, K)


def planted_xi(N: int, L: float, p: int, r_edges, ells, modes) -> np.ndarray:
    """xi_l of the planted field delta_l = sum_j cos(2 pi n_j.l / N) with no catalogue.

    delta^ is N^3/2 at +-n_j and zero elsewhere, so Eq. (pair-counting-kspace) gives
    (1/N^3) sum_l delta delta~ = sum_j K(n_j) / 2 exactly (distinct n_j, none the
    negative of another, none zero).  Returns [n_ells, n_bins].
    """
    nb = len(r_edges) - 1
    out = np.zeros((len(ells), nb))
    for a, ell in enumerate(ells):
        for b in range(nb):
            out[a, b] = 0.5 * float(np.sum(window_xi_at(N, L, p, r_edges[b], r_edges[b + 1], ell, modes)))
    return out


def planted_zeta(N: int, L: float, p: int, r_edges, l_max: int, modes) -> np.ndarray:
    """zeta_l of delta_l = sum_{s in S} cos(2 pi s.l / N) as a finite sum over mode triples.

    a_{b lm}(l) = (1/2) sum_{n in +-S} K_{b lm}(n) e^{2 pi i n.l/N}, and the cell sum of
    Eq. (2-fold-translation) keeps the triples with n' + n'' = n:
      zeta_l(b1, b2) = 1/(4 pi) (1/8) sum_m sum_{n, n', n'' in +-S, n' + n'' = n} conj(K_b1(n)) K_b2(n'),
    all m in [-l, l] written out (no conjugation shortcut).  Returns [l_max+1, nb, nb].
    """
    S = [tuple(int(x) for x in s) for s in modes]
    pm = S + [tuple(-x for x in s) for s in S]
    members = {tuple(x % N for x in n) for n in pm}
    if len(members) != len(pm):
        raise ValueError("planted modes must be distinct and none the negative of another (mod N)")
    # index pairs (n, n') of +-S whose difference n'' = n - n' is also in +-S (modes are
    # periodic in N: the cell sum of e^{2 pi i (n' + n'' - n).l/N} is N^3 when n' + n'' = n mod N)
    trip = [(a, c) for a, n in enumerate(pm) for c, n1 in enumerate(pm)
            if tuple((x - y) % N for x, y in zip(n, n1)) in members]
    nb = len(r_edges) - 1
    out = np.zeros((l_max + 1, nb, nb))
    for ell in range(l_max + 1):
        for m in range(-ell, ell + 1):
            Kb = [window_zeta_at(N, L, p, r_edges[b], r_edges[b + 1], ell, m, pm) for b in range(nb)]
            for b1 in range(nb):
                for b2 in range(nb):
                    tot = 0.0
                    for (a, c) in trip:
                        tot += np.conj(Kb[b1][a]) * Kb[b2][c]
                    out[ell, b1, b2] += (tot / 8.0 / (4.0 * np.pi)).real
    return out


# --------------------------------------------------------------------------
# contractions
# --------------------------------------------------------------------------
def forward(delta):
    """delta^ = sum_l delta_l e^{-2 pi i n.l/N} (numpy FFT), with delta^(0) := 0."""
    dh = np.fft.fftn(delta)
    dh[0, 0, 0] = 0.0
    return dh


def forward_half(delta):
    """delta^ on the rfft half spectrum (n_z in [0, N/2]), with delta^(0) := 0."""
    dh = np.fft.rfftn(delta)
    dh[0, 0, 0] = 0.0
    return dh


def xi_parseval(delta_hat, K):
    """Eq. (pair-counting-kspace): (1/N^3) sum_l delta delta~ = (1/N^6) sum_n |delta^_n|^2 K(n)."""
    N3 = delta_hat.size
    return float(np.sum(np.abs(delta_hat) ** 2 * K).real) / (N3 * N3)


def xi_parseval_half(delta_hat_half, K_half, N):
    """Eq. (pair-counting-kspace) on the rfft half spectrum (n_z in [0, N/2]).

    The full sum counts each n_z in (0, N/2) twice (its mirror -n is the
    complex conjugate with the same |.|^2 and K), and n_z = 0, N/2 once.
    """
    wz = np.full(N // 2 + 1, 2.0)
    wz[0] = 1.0
    wz[N // 2] = 1.0
    s = np.sum(np.abs(delta_hat_half) ** 2 * K_half * wz[None, None, :])
    return float(s) / float(N) ** 6


def xi_cell_contraction(delta, delta_hat, K):
    """Eq. (pair-counting)/(2rdEs): (1/N^3) sum_l delta_l delta~_l with delta~ = iFFT(delta^ K)."""
    filt = np.fft.ifftn(delta_hat * K)
    return float(np.sum(delta * filt.real)) / delta.size


def self_pair_table(pos, w, N, L, p):
    """S[a,b,c] = sum_i w_i^2 prod_d s(a_d; x_i), s(d; x) = sum_l phi_l(x) phi_{l+d}(x), 0 <= a_d < p."""
    pos = np.asarray(pos)
    n = pos.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    _, m = node_weights(pos, N, L, p)                   # [n,3,p]
    s = np.zeros((n, 3, p))
    for d in range(p):
        s[:, :, d] = np.sum(m[:, :, : p - d] * m[:, :, d:], axis=-1)
    S = np.einsum("i,ia,ib,ic->abc", w * w, s[:, 0, :], s[:, 1, :], s[:, 2, :])
    return S


def kappa_from_K(K):
    """kappa(d) = (1/N^3) sum_n K(n) e^{+2 pi i n.d/N}: the window on the lattice of lags."""
    return np.fft.ifftn(K)


def shot_noise(S, K, N, sum_w):
    """SN = (1/(N^3 eps_bar^2)) sum_i w_i^2 K_eff(x_i, x_i), K_eff(x,x) = sum_d kappa(d) s(d).

    The lag sum runs over d in [-(p-1), p-1]^3 using the even table S(|d|).
    """
    p = S.shape[0]
    kap = kappa_from_K(K).real
    tot = 0.0
    for dx in range(-(p - 1), p):
        for dy in range(-(p - 1), p):
            for dz in range(-(p - 1), p):
                tot += S[abs(dx), abs(dy), abs(dz)] * kap[dx % N, dy % N, dz % N]
    eps_bar = sum_w / N ** 3
    return tot / (N ** 3 * eps_bar * eps_bar)


def shot_noise_half(S, K_half, N, sum_w):
    """shot_noise() with kappa from the half spectrum of the real, even kernel (irfftn)."""
    p = S.shape[0]
    kap = np.fft.irfftn(K_half, s=(N, N, N), axes=(0, 1, 2))
    tot = 0.0
    for dx in range(-(p - 1), p):
        for dy in range(-(p - 1), p):
            for dz in range(-(p - 1), p):
                tot += S[abs(dx), abs(dy), abs(dz)] * kap[dx % N, dy % N, dz % N]
    eps_bar = sum_w / N ** 3
    return tot / (N ** 3 * eps_bar * eps_bar)


def xi_multipoles(pos, w, N, L, p, r_edges, ells=(0,), route="parseval"):
    """xi_l(r_b) for every bin b and even l: Landy-Szalay Delta DD / RR with uniform R.

    route: "parseval" (full spectrum), "half" (rfft half spectrum, same sums),
    or "cell" (inverse transform and cell-by-cell contraction).

    Returns dict(xi=[n_ell, n_bins], sn=[n_ell, n_bins], raw=[n_ell, n_bins]).
    raw is (1/N^3) sum delta delta~ before the self-pair subtraction.
    """
    eps, sw, _ = assign(pos, w, N, L, p)
    delta = delta_from_eps(eps, sw)
    del eps
    dh = forward_half(delta) if route == "half" else forward(delta)
    S = self_pair_table(pos, w, N, L, p)
    nb = len(r_edges) - 1
    raw = np.zeros((len(ells), nb))
    sn = np.zeros((len(ells), nb))
    for a, ell in enumerate(ells):
        for b in range(nb):
            if route == "half":
                K = window_xi(N, L, p, r_edges[b], r_edges[b + 1], ell, half=True)
                raw[a, b] = xi_parseval_half(dh, K, N)
                sn[a, b] = shot_noise_half(S, K, N, sw)
                continue
            K = window_xi(N, L, p, r_edges[b], r_edges[b + 1], ell)
            if route == "parseval":
                raw[a, b] = xi_parseval(dh, K)
            else:
                raw[a, b] = xi_cell_contraction(delta, dh, K)
            sn[a, b] = shot_noise(S, K, N, sw)
    return dict(xi=raw - sn, sn=sn, raw=raw, delta=delta, delta_hat=dh)


def xi_randoms(pos, w, pos_r, w_r, N, L, p, r_edges, ells=(0,), cyl=None):
    """Landy-Szalay with an explicit random catalogue, in the field language of Sec. 3.3:
    Delta = D - alpha R (alpha = sum w_D / sum w_R), both in units of the mean data
    density, xi[W] = Delta DD[W] / RR[W] (Eq. xi-deltaDD-over-RR) with the self pairs of
    D and R removed from the products (SN terms with the tables S_D + alpha^2 S_R and
    alpha^2 S_R).  Multipoles divide by RR of the l = 0 window of the same bin.
    cyl = (perp_edges, par_edges) measures xi(r_perp, r_par) instead ([n_par][n_perp]).
    Parseval on the full spectrum; the random field keeps its k = 0 mode."""
    eps_d, swd, _ = assign(pos, w, N, L, p)
    eps_r, swr, _ = assign(pos_r, w_r, N, L, p)
    alpha = swd / swr
    ebar = swd / N ** 3
    hd = forward((eps_d - alpha * eps_r) / ebar)    # its mean is 0 by the choice of alpha
    hr = np.fft.fftn(alpha * eps_r / ebar)           # the k = 0 mode carries most of RR
    s_d = self_pair_table(pos, w, N, L, p)
    s_r = self_pair_table(pos_r, w_r, N, L, p)

    def ratio(K, K0):
        num = xi_parseval(hd, K) - shot_noise(s_d + alpha * alpha * s_r, K, N, swd)
        rr = xi_parseval(hr, K0) - shot_noise(alpha * alpha * s_r, K0, N, swd)
        return num / rr

    if cyl is not None:
        pe, ze = cyl
        out = np.zeros((len(ze) - 1, len(pe) - 1))
        for j in range(len(ze) - 1):
            for i in range(len(pe) - 1):
                K = window_cyl(N, L, p, pe[i], pe[i + 1], ze[j], ze[j + 1])
                out[j, i] = ratio(K, K)
        return out
    nb = len(r_edges) - 1
    out = np.zeros((len(ells), nb))
    for b in range(nb):
        K0 = window_xi(N, L, p, r_edges[b], r_edges[b + 1], 0)
        for a, ell in enumerate(ells):
            K = K0 if ell == 0 else window_xi(N, L, p, r_edges[b], r_edges[b + 1], ell)
            out[a, b] = ratio(K, K0)
    return out


def smoothing_window(N: int, L: float, p: int, kind: str, R: float) -> np.ndarray:
    """K(n) = W^(k) Phi^(n) on the full grid, Nyquist = 0: Table A1 row (b) sphere
    3 (sin x - x cos x) / x^3 or row (c) Gaussian exp(-x^2 / 2), x = k R."""
    nx, ny, nz, q, k, nyq = _mode_grid(N, L)
    if kind == "sphere":
        W = _sphere_hat(k * R)
    elif kind == "gauss":
        W = np.exp(-0.5 * (k * R) ** 2)
    else:
        raise ValueError(kind)
    ph = phi_hat_1d(N, p)
    K = W * ph[:, None, None] * ph[None, :, None] * ph[None, None, :]
    K[nyq] = 0.0
    return K


def density_at(pos_eval, pos, w, N, L, p, kind, R):
    """1 + delta_W(x) at every evaluation point: the field filtered with K (its coefficients
    delta~ = iFT(delta^ K)) read back through the same basis, sum_l phi_l(x) delta~_l, plus 1
    (the mean, K(0) = 1).  Equals sum_j w_j K_eff(x, x_j) / eps_bar."""
    eps, sw, _ = assign(pos, w, N, L, p)
    dt = np.fft.ifftn(forward(delta_from_eps(eps, sw)) * smoothing_window(N, L, p, kind, R)).real
    first, m = node_weights(np.asarray(pos_eval), N, L, p)
    o = np.arange(p)
    ix = (first[:, 0, None] + o) % N
    iy = (first[:, 1, None] + o) % N
    iz = (first[:, 2, None] + o) % N
    vals = dt[ix[:, :, None, None], iy[:, None, :, None], iz[:, None, None, :]]
    wts = m[:, 0, :, None, None] * m[:, 1, None, :, None] * m[:, 2, None, None, :]
    return 1.0 + np.sum(vals * wts, axis=(1, 2, 3))


def density_marks(rho, kind: str, a: float, b: float, self_count: float = 0.0):
    """Marks from densities rho in units of the mean (density_at).  The self count (one
    object per window volume, in units of the mean) is removed and the result clipped at
    0 first.  "power": Eq. (power-law-mark) (rho + b)^a, b the regulariser epsilon;
    "inverse": Eq. (inverse-density-mark) ((b + 1) / (b + rho))^a, b = rho_* / rho_bar."""
    r = np.maximum(np.asarray(rho, dtype=np.float64) - self_count, 0.0)
    if kind == "power":
        return (r + b) ** a
    if kind == "inverse":
        return ((b + 1.0) / (b + r)) ** a
    raise ValueError(kind)


def lm_modes(l_max: int):
    """(l, m) with m >= 0 in l-major order; count (l_max+1)(l_max+2)/2 (Sec. 4.5)."""
    return [(l, m) for l in range(l_max + 1) for m in range(l + 1)]


def zeta_multipoles(delta, N, L, p, r_edges, l_max):
    """zeta_l(b1, b2) = 1/(4 pi N^3) sum_x delta(x) sum_{m=-l}^{l} conj(a_{b1 lm}(x)) a_{b2 lm}(x).

    a_{b lm} = iFFT[delta^ K_{b lm}] (Eq. iFFT-multipoleSFC) is built for every
    m in [-l, l] -- no conjugation shortcut.  Returns [l_max+1, nb, nb] float64
    and the largest |imaginary part| seen (should be rounding noise).
    """
    dh = forward(delta)
    nb = len(r_edges) - 1
    out = np.zeros((l_max + 1, nb, nb))
    imag_max = 0.0
    for ell in range(l_max + 1):
        acc = np.zeros((nb, nb), dtype=np.complex128)
        for m in range(-ell, ell + 1):
            fields = []
            for b in range(nb):
                K = window_zeta(N, L, p, r_edges[b], r_edges[b + 1], ell, m)
                fields.append(np.fft.ifftn(dh * K))
            for b1 in range(nb):
                c1 = np.conj(fields[b1]) * delta
                for b2 in range(nb):
                    acc[b1, b2] += np.sum(c1 * fields[b2])
        acc /= 4.0 * np.pi * N ** 3
        out[ell] = acc.real
        imag_max = max(imag_max, float(np.max(np.abs(acc.imag))))
    return out, imag_max


# --------------------------------------------------------------------------
# 3PCF monopole by triple connection coefficients: Eq. (3pcfddd), Eq. (2-fold-density),
# Eq. (3PCF-ddd-monopole), Eq. (con-coeff), Eq. (DDD-vector-product)
# --------------------------------------------------------------------------
def triple_overlap_1d(p: int) -> np.ndarray:
    """gamma[a + p - 1, b + p - 1] = int M_p(u) M_p(u - a) M_p(u - b) du for |a|, |b| <= p - 1.

    The one-dimensional factor of the triple connection coefficients of Eq. (con-coeff) for
    the centred order-p B-spline (unit integral, grid units).  The three splines share one
    knot lattice (integers for even p, half-integers for odd p), so between two knots the
    integrand is a polynomial of degree 3(p - 1); a 2p-point Gauss-Legendre rule (exact to
    degree 4p - 1) on each of the p knot intervals of the support of M_p(u) integrates it
    exactly up to float64 rounding.
    """
    x, wt = np.polynomial.legendre.leggauss(2 * p)
    t, wt = 0.5 * (x + 1.0), 0.5 * wt
    u = (-0.5 * p + np.arange(p)[:, None] + t[None, :]).ravel()   # the knot intervals of M_p(u)
    w = np.tile(wt, p)
    r = np.arange(-(p - 1), p)
    m0 = bspline(p, u)
    sh = bspline(p, u[None, :] - r[:, None])
    return np.einsum("k,k,ak,bk->ab", w, m0, sh, sh)


def connection_coefficients(p: int) -> np.ndarray:
    """Gamma_{a,b} of Eq. (con-coeff) over the lags a, b in [-(p-1), p-1]^3, as a matrix
    [(2p-1)^3, (2p-1)^3] in the lag order of _lag_stack: the basis is a product of one-
    dimensional splines, so Gamma_{a,b} = prod_d gamma(a_d, b_d).  Normalised to the unit-
    integral basis in grid units (sum_{a,b} Gamma_{a,b} = 1), the paper's 1/N_j being
    the 1/N^3 of ddd_from_fields."""
    g = triple_overlap_1d(p)
    n = 2 * p - 1
    return np.einsum("ad,be,cf->abcdef", g, g, g).reshape(n ** 3, n ** 3)


def _lag_stack(f, p):
    """Rows f(l + a) (periodic) for every lag a = (ax, ay, az) in [-(p-1), p-1]^3, az fastest."""
    r = range(-(p - 1), p)
    return np.stack([np.roll(f, shift=(-ax, -ay, -az), axis=(0, 1, 2)).ravel()
                     for ax in r for ay in r for az in r])


def ddd_from_fields(delta, fields, p: int) -> np.ndarray:
    """(1/N^3) sum_l delta_l eps~_l(b1, b2) for coefficient fields f_b (Eq. DDD-vector-product),
    with the two-fold coefficients of Eq. (3PCF-ddd-monopole)
        eps~_l(b1, b2) = sum_a sum_b Gamma_{a,b} f_b1(l + a) f_b2(l + b),
    the double sum over the lag cube taken as a matrix product.  Returns [nb, nb]."""
    N = delta.shape[0]
    G = connection_coefficients(p)
    stacks = [_lag_stack(np.asarray(f, dtype=np.float64), p) for f in fields]
    d = np.asarray(delta, dtype=np.float64).ravel()
    nb = len(fields)
    out = np.zeros((nb, nb))
    for b2 in range(nb):
        gb = G @ stacks[b2]                      # sum_b Gamma_{a,b} f_b2(l + b), every lag a
        for b1 in range(nb):
            two_fold = np.einsum("an,an->n", stacks[b1], gb)
            out[b1, b2] = float(d @ two_fold) / N ** 3
    return out


def ddd_monopole(delta, N: int, L: float, p: int, r_edges) -> np.ndarray:
    """3PCF monopole DDD(b1, b2) of delta by the triple connection coefficients: the shell-
    filtered coefficients f_b = iFFT[delta^ K_b] with K_b the l = 0 shell window of
    window_xi (<j_0>_b Phi^), then ddd_from_fields.  Replacing Gamma by the identity stencil
    (a = b = 0) gives the cell sum (1/N^3) sum_l delta f_b1 f_b2, i.e. zeta_0 of
    zeta_multipoles.  Returns [nb, nb] float64."""
    dh = forward(delta)
    nb = len(r_edges) - 1
    fields = [np.fft.ifftn(dh * window_xi(N, L, p, r_edges[b], r_edges[b + 1], 0)).real for b in range(nb)]
    return ddd_from_fields(delta, fields, p)


def planted_ddd(N: int, L: float, p: int, r_edges, modes, amps, mmax: int = 40) -> np.ndarray:
    """ddd_monopole of delta_l = sum_q amps_q cos(2 pi n_q.l / N) by Poisson summation.

    With complex amplitudes c_s (amps_q / 2 at +-n_q), a coefficient field sum_s c_s e^{i k_s.l}
    is the spline field sum_s c_s sum_{m in Z^3} M^(k_s + 2 pi m) e^{i (k_s + 2 pi m).u}, where
    M^(w) = prod_d sinc^p(w_d / 2) is the transform of the unit-integral centred B-spline.  The
    box integral of a product of three such fields keeps the alias triples whose wavevectors
    sum to zero, so
        DDD(b1, b2) = sum_{s0, s1, s2} c_s0 c_s1 c_s2 K_b1(n_s1) K_b2(n_s2) prod_d A_d,
        A_d = sum_{m0, m1} s(k0 + 2 pi m0) s(k1 + 2 pi m1) s(k2 + 2 pi (M - m0 - m1)),
    with s(w) = sinc^p(w / 2), k_i = 2 pi n_i / N along axis d and M = -(n0 + n1 + n2) / N,
    which must be an integer (otherwise the triple contributes nothing).  The alias sums
    are truncated at |m| <= mmax; their terms decay like |m|^(-2p).  Returns [nb, nb].
    """
    modes = [tuple(int(x) for x in n) for n in modes]
    pm = modes + [tuple(-x for x in n) for n in modes]
    c = np.concatenate([np.asarray(amps, dtype=np.float64) / 2.0] * 2)
    nb = len(r_edges) - 1
    K = np.array([window_xi_at(N, L, p, r_edges[b], r_edges[b + 1], 0, pm) for b in range(nb)])
    m = np.arange(-mmax, mmax + 1)

    def s(w):
        return np.sinc(w / (2.0 * np.pi)) ** p

    def alias(n0, n1, n2):
        tot = n0 + n1 + n2
        if tot % N:
            return 0.0
        M = -tot // N
        k0, k1, k2 = (2.0 * np.pi * n / N for n in (n0, n1, n2))
        a0 = s(k0 + 2.0 * np.pi * m)[:, None]
        a1 = s(k1 + 2.0 * np.pi * m)[None, :]
        a2 = s(k2 + 2.0 * np.pi * (M - m[:, None] - m[None, :]))
        return float(np.sum(a0 * a1 * a2))

    out = np.zeros((nb, nb))
    ns = len(pm)
    for i0 in range(ns):
        for i1 in range(ns):
            for i2 in range(ns):
                A = 1.0
                for d in range(3):
                    A *= alias(pm[i0][d], pm[i1][d], pm[i2][d])
                    if A == 0.0:
                        break
                if A != 0.0:
                    out += c[i0] * c[i1] * c[i2] * A * np.outer(K[:, i1], K[:, i2])
    return out


# --------------------------------------------------------------------------
# brute-force cross-checks of the oracle itself (tiny inputs only)
# --------------------------------------------------------------------------
def keff_pair_direct(kap_real, first_i, m_i, first_j, m_j, N):
    """K_eff(x_i, x_j) = sum_{l in supp i} sum_{m in supp j} phi_l(x_i) phi_m(x_j) kappa(l - m).

    All p^3 x p^3 node pairs are summed one by one.
    """
    p = m_i.shape[-1]
    tot = 0.0
    for a in range(p):
        for b in range(p):
            for c in range(p):
                wi = m_i[0, a] * m_i[1, b] * m_i[2, c]
                li = ((first_i[0] + a) % N, (first_i[1] + b) % N, (first_i[2] + c) % N)
                for a2 in range(p):
                    for b2 in range(p):
                        for c2 in range(p):
                            wj = m_j[0, a2] * m_j[1, b2] * m_j[2, c2]
                            d = ((li[0] - first_j[0] - a2) % N, (li[1] - first_j[1] - b2) % N,
                                 (li[2] - first_j[2] - c2) % N)
                            tot += wi * wj * kap_real[d]
    return tot


def xi_brute_force(pos, w, N, L, p, K):
    """xi = (1/(N^3 eps_bar^2)) sum_{i != j} w_i w_j K_eff(x_i, x_j) - K(0): pairs one by one."""
    pos = np.asarray(pos)
    n = pos.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    first, m = node_weights(pos, N, L, p)
    kap = kappa_from_K(K).real
    tot = 0.0
    for i in range(n):
        for j in range(n):
            if i != j:
                tot += w[i] * w[j] * keff_pair_direct(kap, first[i], m[i], first[j], m[j], N)
    eps_bar = w.sum() / N ** 3
    return tot / (N ** 3 * eps_bar ** 2) - float(K[0, 0, 0].real)


def direct_convolution(field, kap):
    """eps~_l = sum_m kappa(l - m) field_m over all N^3 lags (O(N^6); tiny grids only)."""
    N = field.shape[0]
    out = np.zeros(field.shape, dtype=np.result_type(field, kap))
    for dx in range(N):
        for dy in range(N):
            for dz in range(N):
                c = kap[dx, dy, dz]
                if c != 0:
                    out += c * np.roll(field, shift=(dx, dy, dz), axis=(0, 1, 2))
    return out
