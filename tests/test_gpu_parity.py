"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (the estimator's stated bar): indices and bin bookkeeping exact;
xi, xi_l and zeta_l within 1e-4 relative or 1e-6 absolute of the oracle.
Intermediate fields (delta, delta^) are compared at the float32 level.
"""
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


@pytest.mark.parametrize("form", ["tiled", "atomic"])
@pytest.mark.parametrize("p", range(1, 9))
def test_scatter_and_delta_match_oracle(p, form, monkeypatch):
    # both scatter forms (the library picks by catalogue density; forced here)
    monkeypatch.setenv("HERMES_SCATTER", form)
    H = _hermes()
    N, L = 32, 100.0
    pos = S.mixed_poisson_sp(5000, L, seed=30 + p)
    w = S.lognormal_masses(5000, seed=3)
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos, w)
        d = ctx.get_delta().astype(np.float64)
        sums, tab = ctx.get_sums()
    eps, sw, sw2 = O.assign(pos, w, N, L, p)
    dref = O.delta_from_eps(eps, sw)
    assert np.max(np.abs(d - dref) / (1.0 + np.abs(dref))) < 2e-5
    assert sums[0] == pytest.approx(sw, rel=1e-12)
    assert sums[1] == pytest.approx(sw2, rel=1e-12)
    np.testing.assert_allclose(tab, O.self_pair_table(pos, w, N, L, p), rtol=2e-5)


@pytest.mark.parametrize("p", range(1, 9))
def test_node_bookkeeping_is_bit_exact(p):
    # first supporting node of every point and axis: identical integers on both sides,
    # including coordinates on knots, at 0, at the largest float32 below L and u = N
    H = _hermes()
    N, L = 64, 1000.0
    rng = np.random.default_rng(40 + p)
    pos = rng.uniform(0, L, size=(20000, 3)).astype(np.float32)
    edge = np.array([0.0, np.nextafter(np.float32(L), np.float32(0)), L / N * 7, L / N * 7.5,
                     np.float32(L / 2)], dtype=np.float32)
    pos[:5] = edge[:, None]
    with H.Context(L, N, p) as ctx:
        first, wts = ctx.nodes(pos)
        wfirst, _ = ctx.nodes((pos + np.float32(3 * L)).astype(np.float32), wrap=True)
    ref_first, ref_w = O.node_weights(pos, N, L, p)
    np.testing.assert_array_equal(first, ref_first)
    np.testing.assert_allclose(wts, ref_w, atol=2e-7)
    assert np.all(wfirst >= 0)


@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_forward_spectrum_matches_oracle(N):
    H = _hermes()
    L = 200.0
    pos = S.mixed_poisson_sp(8000, L, seed=N)
    with H.Context(L, N, 4) as ctx:
        ctx.assign(pos)
        spec = ctx.get_spectrum().astype(np.complex128)
        d = ctx.get_delta().astype(np.float64)
    ref = np.fft.rfftn(d)[:, :, : N // 2]
    ref[0, 0, 0] = 0
    rel = np.linalg.norm(spec - ref) / np.linalg.norm(ref)
    assert rel < 2e-6, rel
    assert np.max(np.abs(spec - ref)) < 1e-5 * np.max(np.abs(ref))


def test_planted_single_mode_exact_closed_form():
    # delta = cos(2 pi n0.l/N) gives xi_b = K_b(n0)/2 and xi_l the same with K_{b,l}
    H = _hermes()
    N, L, p = 32, 160.0, 4
    n0 = (3, -2, 5)
    l = np.arange(N)
    d = np.cos(2 * np.pi * (n0[0] * l[:, None, None] + n0[1] * l[None, :, None] + n0[2] * l[None, None, :]) / N)
    edges = [8.0, 14.0, 20.0, 30.0]
    with H.Context(L, N, p) as ctx:
        ctx.set_delta(d)
        ctx.window_shells(edges, l_max=4)
        got = ctx.xi_multipoles([0, 2, 4])
    for a, ell in enumerate((0, 2, 4)):
        for b in range(3):
            K = O.window_xi(N, L, p, edges[b], edges[b + 1], ell)
            ref = 0.5 * K[n0[0] % N, n0[1] % N, n0[2] % N]
            assert abs(got[a, b] - ref) <= max(2e-5 * abs(ref), 1e-7), (ell, b, got[a, b], ref)


def test_xi_config_two_point_plain():
    # 20,000 points: half uniform Poisson, half Soneira-Peebles; L = 250, 64^3, p = 4,
    # 20 linear shells in [5, 105); unit weights
    H = _hermes()
    L, N, p = 250.0, 64, 4
    pos = S.mixed_poisson_sp(20000, L, seed=2024)
    edges = np.linspace(5.0, 105.0, 21)
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos)
        ctx.window_shells(edges, l_max=0)
        got = ctx.xi()
    ref = O.xi_multipoles(pos, None, N, L, p, edges, ells=(0,))["xi"][0]
    _close(got, ref)


def test_xi_multipoles_and_marked_ragged_batches():
    # 3 multipoles x 13 bins = 39 windows: batches of 16 leave a ragged tail of 7
    H = _hermes()
    L, N, p = 300.0, 64, 4
    pos = S.lognormal_catalogue(30000, L, seed=77, n_grid=64)
    mass = S.lognormal_masses(pos.shape[0], seed=78)
    edges = np.linspace(4.0, 82.0, 14)
    ells = (0, 2, 4)
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=4)
        ctx.assign(pos)
        got = ctx.xi_multipoles(ells)
        ctx.assign(pos, mass)
        got_m = ctx.xi_multipoles(ells)
    ref = O.xi_multipoles(pos, None, N, L, p, edges, ells=ells)["xi"]
    ref_m = O.xi_multipoles(pos, mass, N, L, p, edges, ells=ells)["xi"]
    _close(got, ref)
    _close(got_m, ref_m)


def test_xi_multipoles_to_order_20_match_oracle():
    # Legendre windows up to l = 20: the host tables switch between the power series and
    # the closed-form recurrences of the Bessel moments at x = l + 4
    H = _hermes()
    N, L, p = 32, 120.0, 4
    pos = S.mixed_poisson_sp(8000, L, seed=205)
    edges = np.linspace(3.0, 45.0, 7)
    ells = (0, 8, 14, 20)
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos)
        ctx.window_shells(edges, l_max=20)
        got = ctx.xi_multipoles(ells)
        gk = ctx.xi_multipoles_kspace(ells)
    ref = O.xi_multipoles(pos, None, N, L, p, edges, ells=ells)["xi"]
    _close(got, ref)
    _close(gk, ref)


def test_xi_other_orders_and_sizes():
    H = _hermes()
    for (N, p, L) in [(16, 2, 50.0), (32, 3, 120.0), (128, 6, 400.0)]:
        pos = S.mixed_poisson_sp(6000, L, seed=N + p)
        edges = np.linspace(L / 40, L / 4, 6)
        with H.Context(L, N, p) as ctx:
            ctx.assign(pos)
            ctx.window_shells(edges, l_max=2)
            got = ctx.xi_multipoles([0, 2])
        ref = O.xi_multipoles(pos, None, N, L, p, edges, ells=(0, 2))["xi"]
        _close(got, ref)


def test_single_point_and_wrap_and_device_pointers():
    import torch
    H = _hermes()
    L, N, p = 100.0, 32, 4
    edges = [2.0, 6.0, 12.0]
    one = np.array([[10.0, 20.0, 30.0]], dtype=np.float32)
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=0)
        ctx.assign(one)
        g1 = ctx.xi()
        r = O.xi_multipoles(one, None, N, L, p, edges)
        # one point: xi = -1 exactly, computed as raw - SN with SN ~ N^3 kappa ~ 600; the
        # float32 fields leave an absolute error ~2e-7 SN (the error model of sparse catalogues)
        assert np.all(np.abs(g1 - r["xi"][0]) <= np.maximum(1e-6, 4e-7 * r["sn"][0]))
        # wrapped coordinates give the same field as the wrapped catalogue
        pos = S.poisson_uniform(3000, L, seed=9)
        shifted = (pos + np.float32(L)).astype(np.float32)
        with pytest.raises(H.HermesError) as ei:
            ctx.assign(shifted)
        assert ei.value.code == H.ERR_RANGE
        with pytest.raises(H.HermesError) as ei:
            ctx.xi()
        assert ei.value.code == H.ERR_STATE
        ctx.assign(pos)
        base = ctx.xi()
        ctx.assign(shifted, wrap=True)
        wrapped = ctx.xi()
        ref = O.xi_multipoles(shifted, None, N, L, p, edges)["xi"][0]
        _close(wrapped, ref)
        _close(base, O.xi_multipoles(pos, None, N, L, p, edges)["xi"][0])
        # torch device tensors through HERMES_DEVICE_PTR, on a torch stream
        tpos = torch.from_numpy(pos).cuda()
        tw = torch.ones(pos.shape[0], dtype=torch.float32, device="cuda")
        s = torch.cuda.Stream()
        ctx.set_stream(s)
        ctx.assign(tpos, tw)
        dev = ctx.xi()
        ctx.set_stream(None)
        np.testing.assert_allclose(dev, base, rtol=1e-6, atol=1e-9)


def test_argument_errors():
    H = _hermes()
    with H.Context(100.0, 32, 4) as ctx:
        with pytest.raises(H.HermesError) as ei:
            ctx.xi()
        assert ei.value.code == H.ERR_STATE
        with pytest.raises(H.HermesError) as ei:
            ctx.window_shells([1.0, 60.0], 0)          # beyond L/2
        assert ei.value.code == H.ERR_RANGE
        with pytest.raises(H.HermesError) as ei:
            ctx.assign(np.zeros((0, 3), np.float32))   # empty catalogue
        assert ei.value.code == H.ERR_ARG
        ctx.window_shells(np.linspace(1, 40, 18), 2)
        ctx.assign(S.poisson_uniform(100, 100.0, 1))
        with pytest.raises(H.HermesError) as ei:
            ctx.xi_multipoles([1])
        assert ei.value.code == H.ERR_ARG
        with pytest.raises(H.HermesError) as ei:
            ctx.window_shells(np.linspace(1, 40, 18), 25)  # l_max beyond 24
        assert ei.value.code == H.ERR_ARG
        bad = S.poisson_uniform(10, 100.0, 2)
        bad[3, 1] = np.nan
        with pytest.raises(H.HermesError) as ei:
            ctx.assign(bad)
        assert ei.value.code == H.ERR_RANGE


@pytest.mark.parametrize("N,nb,l_max", [(16, 3, 3), (32, 4, 4), (32, 16, 2), (32, 20, 2), (32, 3, 14)])
def test_zeta_multipoles_match_oracle(N, nb, l_max):
    # 20 bins: blocks of 8, 8 and 4 run as the six pairs of blocks; l_max 14: the paper's
    # DDD_l runs reach l_max 14 and 20
    H = _hermes()
    L, p = 4.0 * N, 4
    pos = S.mixed_poisson_sp(3000, L, seed=N + nb)
    edges = np.linspace(L / 32, L / 3, nb + 1)
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos)
        ctx.window_shells(edges, l_max=l_max)
        got = ctx.zeta_multipoles()
        d = ctx.get_delta().astype(np.float64)
    eps, sw, _ = O.assign(pos, None, N, L, p)
    ref, imag = O.zeta_multipoles(O.delta_from_eps(eps, sw), N, L, p, edges, l_max)
    _close(got, ref)
    for ell in range(l_max + 1):
        np.testing.assert_array_equal(got[ell], got[ell].T)


@pytest.mark.parametrize("N,L,n", [(64, 300.0, 30000), (256, 1000.0, 200000), (512, 1000.0, 300000)])
def test_fused_yz_pass_matches_three_pass_path(N, L, n, monkeypatch):
    # the cluster kernel (inverse y + c2r z + contraction in one pass) against the
    # separate y and z passes, and both against the oracle where it is affordable
    H = _hermes()
    pos = S.lognormal_catalogue(n, L, seed=N, n_grid=64)
    edges = np.linspace(L / 100, L / 10, 6)
    res = {}
    for flag in ("1", "0"):  # opt-in cluster kernel vs the default three-pass path
        monkeypatch.setenv("HERMES_YZ_FUSED", flag)
        with H.Context(L, N, 4) as ctx:
            ctx.window_shells(edges, l_max=2)
            ctx.assign(pos)
            res[flag] = ctx.xi_multipoles([0, 2])
    np.testing.assert_allclose(res["1"], res["0"], rtol=2e-5, atol=1e-7)
    if N <= 64:
        _close(res["1"], O.xi_multipoles(pos, None, N, L, 4, edges, ells=(0, 2))["xi"])


def test_zeta_two_warp_lines_at_512_match_block_synchronised_gram(monkeypatch):
    # at 512^3 each 512-point z line of the SIMT Gram pass spans two warps that wait on
    # a named barrier of their own; the opt-in tensor-core pass transforms the same lines
    # with block-wide barriers, so the two agree only if the per-line barriers are right
    H = _hermes()
    N, p, L, l_max = 512, 4, 500.0, 2
    pos = S.lognormal_catalogue(100000, L, seed=512, n_grid=64)
    edges = np.linspace(10.0, 90.0, 9)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("HERMES_ZETA_TC", flag)
        with H.Context(L, N, p) as ctx:
            ctx.assign(pos)
            ctx.window_shells(edges, l_max=l_max)
            res[flag] = ctx.zeta_multipoles()
    assert np.all(np.isfinite(res["0"]))
    # the two Grams round differently (split TF32 in TMEM vs float32 partials flushed
    # to float64 every 8 lines) and at 512^3 they differ by up to ~1.3e-4 relative; a
    # barrier fault would corrupt whole lines, an error of the order of the values
    _close(res["1"], res["0"], rel=1e-3, ab=1e-7)
    for ell in range(l_max + 1):
        np.testing.assert_array_equal(res["0"][ell], res["0"][ell].T)


@pytest.mark.parametrize("N,nb", [(32, 16), (64, 7), (128, 16), (256, 5)])
def test_zeta_tensor_core_gram_matches_simt_and_oracle(N, nb, monkeypatch):
    # the tcgen05 split-TF32 Gram (opt-in, unpacked fields) against the float32 SIMT Gram
    # (default: m = 0 bins packed in pairs; at 256^3 an odd bin count leaves idle lines),
    # and both against the oracle at 32^3
    H = _hermes()
    L, p, l_max = 3.0 * N, 4, 3
    pos = S.mixed_poisson_sp(8000, L, seed=N + 3 * nb)
    edges = np.linspace(L / 40, L / 3, nb + 1)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("HERMES_ZETA_TC", flag)
        with H.Context(L, N, p) as ctx:
            ctx.assign(pos)
            ctx.window_shells(edges, l_max=l_max)
            res[flag] = ctx.zeta_multipoles()
    _close(res["1"], res["0"], rel=1e-4, ab=1e-7)
    if N == 32:
        eps, sw, _ = O.assign(pos, None, N, L, p)
        ref, _ = O.zeta_multipoles(O.delta_from_eps(eps, sw), N, L, p, edges, l_max)
        _close(res["1"], ref)
        _close(res["0"], ref)


@pytest.mark.parametrize("N,p,L,ells", [(64, 4, 300.0, (0, 2, 4)), (16, 2, 50.0, (0,)), (128, 6, 400.0, (2, 0))])
def test_kspace_route_matches_oracle_and_real_space_path(N, p, L, ells):
    # Eq. pair-counting-kspace: the Parseval sum over the half spectrum gives the
    # same xi_l as the inverse-FFT cell contraction (and the oracle's full-spectrum sum)
    H = _hermes()
    pos = S.lognormal_catalogue(30000, L, seed=N + 5, n_grid=N)
    mass = S.lognormal_masses(pos.shape[0], seed=N + 6)
    edges = np.linspace(L / 60, L / 4, 12)
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=max(ells))
        ctx.assign(pos, mass)
        got = ctx.xi_multipoles_kspace(ells)
        real = ctx.xi_multipoles(ells)
    ref = O.xi_multipoles(pos, mass, N, L, p, edges, ells=ells)["xi"]
    assert got.shape == (len(ells), len(edges) - 1)
    _close(got, ref)
    _close(got, real)


def test_inverse_passes_at_1024_match_kspace_route():
    # 1024^3 has its own launch shapes: 1024-thread strided tiles (one per SM), the
    # plain inverse y pass instead of the persistent one, and 512-point z lines that
    # span two warps (one named barrier per line).  The real-space xi_l must equal the
    # Parseval route, which reads only delta^ and the radial tables (that route is
    # pinned to the oracle at small grids above).
    # Every variant of the inverse y pass (radix 8, 32 and 16 values per thread) and of the
    # contraction pass (radix 8, 16 values per thread) at 1024^3.
    H = _hermes()
    N, p, L = 1024, 4, 2000.0
    pos = S.lognormal_catalogue(200000, L, seed=1024, n_grid=64)
    mass = S.lognormal_masses(pos.shape[0], seed=1025)
    edges = np.linspace(L / 200, L / 20, 7)
    reals = []
    try:
        with H.Context(L, N, p) as ctx:
            ctx.window_shells(edges, l_max=2)
            ctx.assign(pos, mass)
            ks = ctx.xi_multipoles_kspace((0, 2))
            for pass_ in (H.PASS_INV_Y, H.PASS_CONTRACT):
                for v in range(len(H.fft_variants(N, pass_)["variants"])):
                    H.fft_set_variant(N, v, pass_)
                    reals.append(ctx.xi_multipoles((0, 2)))
                H.fft_set_variant(N, 0, pass_)
    finally:
        H.fft_set_variant(N, -1, H.PASS_INV_Y)
        H.fft_set_variant(N, -1, H.PASS_CONTRACT)
    assert len(reals) >= 2
    for real in reals:
        assert np.all(np.isfinite(real)) and real.shape == (2, 6)
        _close(real, ks)


def test_kspace_route_planted_mode_and_errors():
    # delta = cos(2 pi n0.x / N): |delta^|^2 = (N^3/2)^2 at +-n0, so
    # xi_{b,l} = K_{b,l}(n0) / 2 with no self-pair term (the field has no catalogue)
    H = _hermes()
    L, N, p = 100.0, 32, 3
    n0 = (3, -2, 5)
    x = np.arange(N)
    ph = 2 * np.pi * (n0[0] * x[:, None, None] + n0[1] * x[None, :, None] + n0[2] * x[None, None, :]) / N
    delta = np.cos(ph).astype(np.float32)
    edges = np.array([3.0, 9.0, 15.0, 25.0])
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=4)
        ctx.set_delta(delta)
        got = ctx.xi_multipoles_kspace([0, 2, 4])
        for bad in ([1], [6], [], list(range(0, 18, 2))):
            with pytest.raises(H.HermesError) as ei:
                ctx.xi_multipoles_kspace(bad)
            assert ei.value.code == H.ERR_ARG
    for a, ell in enumerate((0, 2, 4)):
        for b in range(3):
            K = O.window_xi(N, L, p, edges[b], edges[b + 1], ell)
            ref = 0.5 * K[n0[0] % N, n0[1] % N, n0[2] % N]
            assert abs(got[a, b] - ref) <= max(2e-5 * abs(ref), 1e-7), (ell, b, got[a, b], ref)


def test_cached_window_tables_serve_smaller_orders():
    # a table built for l_max = 4 is reused (its leading blocks) by later
    # contexts asking l_max = 0 or 2 with the same L, N and shells
    # (the same field is set directly in every context, so only the tables can differ;
    # two scatters of one catalogue differ by float-atomic order)
    H = _hermes()
    L, N, p = 180.0, 32, 4
    edges = np.linspace(3.0, 60.0, 10)
    pos = S.mixed_poisson_sp(6000, L, seed=91)
    eps, sw, _ = O.assign(pos, None, N, L, p)
    delta = O.delta_from_eps(eps, sw).astype(np.float32)
    with H.Context(L, N, p) as c4:
        c4.window_shells(edges, l_max=4)
        c4.assign(pos)
        x4 = c4.xi_multipoles([0, 2, 4])
        c4.set_delta(delta)
        d4 = c4.xi_multipoles([0, 2, 4])
    for lm, ells in ((0, [0]), (2, [0, 2])):
        with H.Context(L, N, p) as c:
            c.window_shells(edges, l_max=lm)
            c.set_delta(delta)
            got = c.xi_multipoles(ells)
        np.testing.assert_allclose(got, d4[:len(ells)], rtol=1e-9, atol=1e-12)
    ref = O.xi_multipoles(pos, None, N, L, p, edges, ells=(0, 2, 4))["xi"]
    _close(x4, ref)


@pytest.mark.parametrize("N,p,L,sigma", [(64, 4, 240.0, 0.0), (32, 3, 100.0, 4.0), (16, 2, 60.0, 0.0)])
def test_cylinder_windows_match_oracle_both_routes(N, p, L, sigma):
    # xi(r_perp, r_par): 7 transverse annuli (the first a disk) x 5 line-of-sight slab pairs
    # (the first a filled slab); S = 4 window batches leave a ragged tail of 3
    H = _hermes()
    pos = S.lognormal_catalogue(25000, L, seed=N + 11, n_grid=N)
    mass = S.lognormal_masses(pos.shape[0], seed=N + 12)
    rperp = np.concatenate([[0.0], np.linspace(L / 40, L / 5, 7)])
    rpar = np.linspace(0.0, L / 6, 6)
    with H.Context(L, N, p) as ctx:
        ctx.window_cylinders(rperp, rpar, sigma_perp=sigma)
        ctx.assign(pos, mass)
        got = ctx.xi_cylinders()
        gk = ctx.xi_cylinders(kspace=True)
    ref = O.xi_cylinders(pos, mass, N, L, p, rperp, rpar, sigma_perp=sigma)
    assert got.shape == (5, 7)
    _close(got, ref)
    _close(gk, ref)


def test_cylinder_planted_mode_and_errors():
    # delta = cos(2 pi n0.x / N) gives xi_{j,i} = K_{j,i}(n0) / 2 exactly
    H = _hermes()
    L, N, p = 90.0, 32, 4
    n0 = (2, -3, 4)
    x = np.arange(N)
    ph = 2 * np.pi * (n0[0] * x[:, None, None] + n0[1] * x[None, :, None] + n0[2] * x[None, None, :]) / N
    rperp, rpar = [1.0, 6.0, 15.0], [0.0, 5.0, 12.0]
    with H.Context(L, N, p) as ctx:
        with pytest.raises(H.HermesError) as ei:
            ctx.window_cylinders([3.0, 2.0], rpar)
        assert ei.value.code == H.ERR_RANGE
        with pytest.raises(H.HermesError) as ei:
            ctx.window_cylinders(rperp, [0.0, L])
        assert ei.value.code == H.ERR_RANGE
        ctx.window_cylinders(rperp, rpar)
        with pytest.raises(H.HermesError) as ei:
            ctx.xi_cylinders()
        assert ei.value.code == H.ERR_STATE
        ctx.set_delta(np.cos(ph).astype(np.float32))
        got = ctx.xi_cylinders()
        gk = ctx.xi_cylinders(kspace=True)
    for j in range(2):
        for i in range(2):
            K = O.window_cyl(N, L, p, rperp[i], rperp[i + 1], rpar[j], rpar[j + 1])
            ref = 0.5 * K[n0[0] % N, n0[1] % N, n0[2] % N]
            assert abs(got[j, i] - ref) <= max(2e-5 * abs(ref), 1e-7), (j, i, got[j, i], ref)
            assert abs(gk[j, i] - ref) <= max(2e-5 * abs(ref), 1e-7), (j, i, gk[j, i], ref)


@pytest.mark.parametrize("N,p,L", [(32, 4, 100.0), (64, 3, 200.0)])
def test_explicit_randoms_landy_szalay_matches_oracle(N, p, L):
    # data: clustered catalogue with masses; randoms: 3x as many weighted uniform points;
    # xi_l over RR_0 by inverse transforms and by Parseval, xi(r_perp, r_par) over RR
    H = _hermes()
    pd = S.lognormal_catalogue(8000, L, seed=N + 21, n_grid=N)
    wd = S.lognormal_masses(pd.shape[0], seed=N + 22)
    pr = S.poisson_uniform(24000, L, seed=N + 23)
    wr = (0.5 + np.random.default_rng(N).random(pr.shape[0])).astype(np.float32)
    edges = np.linspace(L / 25, L / 4, 8)
    rperp, rpar = np.linspace(0.0, L / 5, 5), np.linspace(0.0, L / 6, 4)
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=2)
        ctx.window_cylinders(rperp, rpar)
        ctx.assign_randoms(pr, wr)
        with pytest.raises(H.HermesError) as ei:  # the data field must be rebuilt
            ctx.xi_multipoles([0])
        assert ei.value.code == H.ERR_STATE
        ctx.assign(pd, wd)
        got = ctx.xi_multipoles([0, 2])
        gk = ctx.xi_multipoles_kspace([0, 2])
        gc = ctx.xi_cylinders()
        gck = ctx.xi_cylinders(kspace=True)
        with pytest.raises(H.HermesError) as ei:
            ctx.zeta_multipoles()
        assert ei.value.code == H.ERR_STATE
        ctx.clear_randoms()
        ctx.assign(pd, wd)
        plain = ctx.xi_multipoles([0, 2])
    ref = O.xi_randoms(pd, wd, pr, wr, N, L, p, edges, ells=(0, 2))
    refc = O.xi_randoms(pd, wd, pr, wr, N, L, p, None, cyl=(rperp, rpar))
    _close(got, ref)
    _close(gk, ref)
    _close(gc, refc)
    _close(gck, refc)
    _close(plain, O.xi_multipoles(pd, wd, N, L, p, edges, ells=(0, 2))["xi"])


def test_density_marks_match_oracle_and_feed_the_marked_xi():
    import torch
    H = _hermes()
    L, N, p = 120.0, 64, 4
    pos = S.lognormal_catalogue(20000, L, seed=61, n_grid=64)
    n = pos.shape[0]
    edges = np.linspace(3.0, 40.0, 8)
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos)
        rho = ctx.density_marks(pos, "sphere", 8.0, "density")
        mpl = ctx.density_marks(pos, "sphere", 8.0, "power", a=0.5, b=0.1, remove_self=True)
        minv = ctx.density_marks(pos, "gauss", 5.0, "inverse", a=1.0, b=1.0)
        dev = ctx.density_marks(torch.from_numpy(pos).cuda(), "sphere", 8.0, "power", a=0.5, b=0.1,
                                remove_self=True)
        with pytest.raises(H.HermesError) as ei:
            ctx.density_marks(pos, "sphere", 0.7 * L, "density")
        assert ei.value.code == H.ERR_RANGE
        ctx.window_shells(edges, l_max=2)
        ctx.assign(pos, mpl)
        xi_m = ctx.xi_multipoles([0, 2])
    ref_rho = O.density_at(pos, pos, None, N, L, p, "sphere", 8.0)
    ref_g = O.density_at(pos, pos, None, N, L, p, "gauss", 5.0)
    self_count = L ** 3 / (4.0 * np.pi * 8.0 ** 3 / 3.0 * n)
    tol = 2e-5 * max(1.0, np.abs(ref_rho).max())
    np.testing.assert_allclose(rho, ref_rho, rtol=0, atol=tol)
    np.testing.assert_allclose(mpl, O.density_marks(ref_rho, "power", 0.5, 0.1, self_count), rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(minv, O.density_marks(ref_g, "inverse", 1.0, 1.0), rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(dev.cpu().numpy(), mpl, rtol=0, atol=1e-6)
    # the marks are the weights of the marked field: same xi_l as the oracle given those marks
    _close(xi_m, O.xi_multipoles(pos, mpl.astype(np.float64), N, L, p, edges, ells=(0, 2))["xi"])
