"""The 3PCF monopole by triple connection coefficients (hermes_ddd_monopole) on the GPU:
against the FP64 oracle's stencil (Eq. 3PCF-ddd-monopole with Eq. con-coeff) on catalogues
at small grids, against the Poisson-summation closed form for planted modes at 256^3 and
512^3, against zeta_0 for the box basis (where Gamma is the identity), and its errors.
Tolerance: 1e-4 relative or 1e-6 absolute, element by element."""
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


@pytest.mark.parametrize("N,p,L,nb", [(16, 2, 120.0, 4), (16, 3, 120.0, 10), (16, 4, 120.0, 16), (32, 4, 200.0, 5),
                                      (32, 1, 200.0, 3), (16, 4, 120.0, 17), (16, 3, 120.0, 27)])
def test_monopole_matches_the_oracle_stencil(N, p, L, nb):
    # nb > 8 runs the off-diagonal bin tile; 10 and 5 leave ragged tiles; more than 16 bins run
    # every pair of 8-bin blocks (17: a one-bin block; 27: four blocks, the last of three bins)
    H = _hermes()
    pos = S.lognormal_catalogue(6000 if N == 16 else 20000, L, seed=N + p, n_grid=16)
    w = S.lognormal_masses(pos.shape[0], seed=7 * p)
    edges = np.linspace(0.08 * L, 0.45 * L, nb + 1)
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos, w)
        ctx.window_shells(edges, l_max=0)
        got = ctx.ddd_monopole()
    eps, sw, _ = O.assign(pos, w, N, L, p)
    delta = O.delta_from_eps(eps, sw)
    ref = O.ddd_monopole(delta, N, L, p, edges)
    assert got.shape == (nb, nb)
    np.testing.assert_array_equal(got, got.T)
    _close(got, ref)


def test_box_basis_monopole_equals_zeta0_on_the_gpu():
    # p = 1: the triple overlap is the identity stencil, so the monopole is the cell sum zeta_0
    H = _hermes()
    N, L, p = 64, 300.0, 1
    pos = S.lognormal_catalogue(40000, L, seed=5, n_grid=32)
    edges = np.linspace(10.0, 120.0, 9)
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos)
        ctx.window_shells(edges, l_max=0)
        ddd = ctx.ddd_monopole()
        z0 = ctx.zeta_multipoles()[0]
    _close(ddd, z0)


def _planted(N, modes, amps):
    l = np.arange(N, dtype=np.float64)
    d = np.zeros((N, N, N), dtype=np.float64)
    for n, a in zip(modes, amps):
        ph = (2 * np.pi / N) * (n[0] * l[:, None, None] + n[1] * l[None, :, None] + n[2] * l[None, None, :])
        d += a * np.cos(ph)
    return d.astype(np.float32)


@pytest.mark.parametrize("N,p,L,nb", [(256, 3, 600.0, 16), (512, 4, 1000.0, 12)])
def test_monopole_matches_the_planted_closed_form_at_full_size(N, p, L, nb):
    # a closed triangle of modes (n_a + n_b + n_c = 0) and a mode outside any triangle:
    # the launch shapes of the measured grids, exact value by Poisson summation
    H = _hermes()
    modes = [(3, 1, 2), (-1, 4, -2), (-2, -5, 0), (0, 2, 6)]
    amps = [0.3, 0.25, 0.2, 0.15]
    edges = np.linspace(0.03 * L, 0.2 * L, nb + 1)
    with H.Context(L, N, p) as ctx:
        ctx.set_delta(_planted(N, modes, amps))
        ctx.window_shells(edges, l_max=0)
        got = ctx.ddd_monopole()
    ref = O.planted_ddd(N, L, p, edges, modes, amps)
    assert np.abs(ref).max() > 1e-4
    _close(got, ref)


def test_monopole_errors():
    H = _hermes()
    N, L = 16, 100.0
    with H.Context(L, N, 4) as ctx:
        with pytest.raises(H.HermesError) as ei:
            ctx.window_shells(np.linspace(5.0, 40.0, 5), l_max=0)
            ctx.ddd_monopole()
        assert ei.value.code == H.ERR_STATE                       # no field yet
        ctx.assign(S.poisson_uniform(2000, L, seed=1))
        ctx.assign_randoms(S.poisson_uniform(4000, L, seed=2))
        with pytest.raises(H.HermesError) as ei:
            ctx.ddd_monopole()
        assert ei.value.code == H.ERR_STATE                       # explicit randoms set
    with H.Context(L, N, 5) as ctx:
        ctx.window_shells(np.linspace(5.0, 40.0, 5), l_max=0)
        ctx.assign(S.poisson_uniform(2000, L, seed=3))
        with pytest.raises(H.HermesError) as ei:
            ctx.ddd_monopole()
        assert ei.value.code == H.ERR_ARG                         # order above the built kernels
