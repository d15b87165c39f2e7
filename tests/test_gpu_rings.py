"""GPU parity of the ring windows (Sec. 3.4.4, Table A1 row (i)): xi at a list of
(r_perp, r_par) points such as the (s, mu) samples of xi(s, mu), thin and with
finite widths, by inverse transforms and by Parseval, against the FP64 oracle at the
estimator's bar (1e-4 relative or 1e-6 absolute)."""
import numpy as np
import pytest

from oracle import hermes_oracle as O
from synthetic import catalogues as S

pytestmark = pytest.mark.gpu
REL, ABS = 1e-4, 1e-6


def _hermes():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_23494_b300 import hermes as H
    return H


def _close(got, ref, rel=REL, ab=ABS):
    got, ref = np.asarray(got), np.asarray(ref)
    err = np.abs(got - ref)
    bad = err > np.maximum(rel * np.abs(ref), ab)
    assert not bad.any(), (f"{bad.sum()} of {bad.size} outside tolerance; worst abs err {err.max():.3e}; "
                           f"got {got[bad][:5]} ref {ref[bad][:5]}")


def _s_mu(s, mu):
    R = (np.asarray(s)[:, None] * np.sqrt(1.0 - np.asarray(mu)[None, :] ** 2)).ravel()
    H = (np.asarray(s)[:, None] * np.asarray(mu)[None, :]).ravel()
    return R, H


@pytest.mark.parametrize("N,p,L,finite,sigma", [(64, 4, 240.0, False, 0.0), (64, 4, 240.0, True, 0.0),
                                                (32, 3, 100.0, True, 3.0)])
def test_s_mu_rings_match_oracle_both_routes(N, p, L, finite, sigma):
    # 5 separations x 7 orientations (mu = 0 and 1 included) = 35 rings: batches of 16 leave
    # a ragged tail of 3; the finite form gives every ring dR = ds and dH = s dmu
    H_ = _hermes()
    pos = S.lognormal_catalogue(25000, L, seed=N + 31, n_grid=N)
    mass = S.lognormal_masses(pos.shape[0], seed=N + 32)
    s = np.linspace(L / 30, L / 6, 5)
    mu = np.linspace(0.0, 1.0, 7)
    R, Hz = _s_mu(s, mu)
    ds, dmu = (L / 60, 1.0 / 7) if finite else (0.0, 0.0)
    dR = np.full(R.shape, ds) if finite else None
    dH = np.repeat(s * dmu, len(mu)) if finite else None
    with H_.Context(L, N, p) as ctx:
        ctx.window_s_mu(s, mu, ds=ds, dmu=dmu, sigma_perp=sigma)
        ctx.assign(pos, mass)
        got = ctx.xi_rings()
        gk = ctx.xi_rings(kspace=True)
    ref = O.xi_rings(pos, mass, N, L, p, R, Hz, dR, dH, sigma_perp=sigma)
    assert got.shape == (35,)
    _close(got, ref)
    _close(gk, ref)


def test_ring_planted_mode_errors_and_state():
    # delta = cos(2 pi n0.x / N) gives xi_w = K_w(n0) / 2 exactly
    H_ = _hermes()
    L, N, p = 90.0, 32, 4
    n0 = (2, -3, 4)
    x = np.arange(N)
    ph = 2 * np.pi * (n0[0] * x[:, None, None] + n0[1] * x[None, :, None] + n0[2] * x[None, None, :]) / N
    R, Hz = [3.0, 7.5, 11.0, 0.0], [0.0, 4.0, 9.5, 6.0]
    with H_.Context(L, N, p) as ctx:
        with pytest.raises(H_.HermesError) as ei:
            ctx.window_rings([1.0, -2.0], [0.0, 1.0])
        assert ei.value.code == H_.ERR_RANGE
        with pytest.raises(H_.HermesError) as ei:
            ctx.window_rings([44.0], [1.0], dR=3.0)          # reaches beyond L/2
        assert ei.value.code == H_.ERR_RANGE
        ctx.window_rings(R, Hz)
        with pytest.raises(H_.HermesError) as ei:
            ctx.xi_rings()                                   # no field yet
        assert ei.value.code == H_.ERR_STATE
        ctx.set_delta(np.cos(ph).astype(np.float32))
        got = ctx.xi_rings()
        gk = ctx.xi_rings(kspace=True)
        ctx.window_cylinders([0.0, 5.0], [0.0, 5.0])         # cylinders replace the rings
        with pytest.raises(H_.HermesError) as ei:
            ctx.xi_rings()
        assert ei.value.code == H_.ERR_STATE
    for w in range(4):
        K = O.window_ring(N, L, p, R[w], Hz[w])
        ref = 0.5 * K[n0[0] % N, n0[1] % N, n0[2] % N]
        assert abs(got[w] - ref) <= max(2e-5 * abs(ref), 1e-7), (w, got[w], ref)
        assert abs(gk[w] - ref) <= max(2e-5 * abs(ref), 1e-7), (w, gk[w], ref)


def test_rings_with_explicit_randoms_match_oracle_via_cylinder_bins():
    # a finite ring is the cylinder bin [R -+ dR/2] x [H -+ dH/2]: with explicit randoms the
    # ring route must give the cylinder route's Landy-Szalay values
    H_ = _hermes()
    L, N, p = 100.0, 32, 4
    pd = S.lognormal_catalogue(8000, L, seed=71, n_grid=N)
    pr = S.poisson_uniform(24000, L, seed=72)
    rperp, rpar = np.array([2.0, 6.0, 10.0]), np.array([1.0, 5.0, 9.0])
    Rc, Hc = 0.5 * (rperp[:-1] + rperp[1:]), 0.5 * (rpar[:-1] + rpar[1:])
    R = np.repeat(Rc[None, :], 2, 0).ravel()               # [par][perp] order
    Hz = np.repeat(Hc[:, None], 2, 1).ravel()
    with H_.Context(L, N, p) as ctx:
        ctx.assign_randoms(pr)
        ctx.assign(pd)
        ctx.window_cylinders(rperp, rpar)
        cyl = ctx.xi_cylinders().ravel()
        ctx.window_rings(R, Hz, dR=4.0, dH=4.0)
        ring = ctx.xi_rings()
        ringk = ctx.xi_rings(kspace=True)
    _close(ring, cyl)
    _close(ringk, cyl)
    ref = O.xi_randoms(pd, None, pr, None, N, L, p, None, cyl=(rperp, rpar)).ravel()
    _close(ring, ref)
