"""Batched measurements through the C ABI (hermes_xi_multipoles_batch).

Each catalogue of a batch is an independent measurement: its xi_l must equal
what the single-catalogue path gives for it, and the oracle's value, within the
estimator's tolerance (1e-4 relative or 1e-6 absolute).  Plans (windows and
catalogues per launch), the CUDA graph's reuse across calls and the argument
checks are covered too.
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
    return torch, H


def _close(got, ref, rel=REL, ab=ABS):
    got, ref = np.asarray(got), np.asarray(ref)
    err = np.abs(got - ref)
    bad = err > np.maximum(rel * np.abs(ref), ab)
    assert not bad.any(), (f"{bad.sum()} of {bad.size} outside tolerance; worst abs err {err.max():.3e}; "
                           f"got {got[bad][:5]} ref {ref[bad][:5]}")


def _batch(L, N, sizes, seed, weights=True):
    cats, ws = [], []
    for k, n in enumerate(sizes):
        pos = S.lognormal_catalogue(int(n), L, seed=seed + k, n_grid=N) if k % 2 == 0 else \
            S.mixed_poisson_sp(int(n), L, seed=seed + k)
        cats.append(pos)
        ws.append(S.lognormal_masses(pos.shape[0], seed=seed + 100 + k))
    offs = np.concatenate([[0], np.cumsum([c.shape[0] for c in cats])]).astype(np.int64)
    pos = np.concatenate(cats).astype(np.float32)
    w = np.concatenate(ws).astype(np.float32) if weights else None
    return pos, w, offs


def _single(H, L, N, p, edges, l_max, pos, w, offs, ells):
    out = []
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=l_max)
        for k in range(len(offs) - 1):
            a, b = offs[k], offs[k + 1]
            ctx.assign(pos[a:b], None if w is None else w[a:b])
            out.append(ctx.xi_multipoles(ells))
    return np.array(out)


def test_batch_matches_single_path_and_oracle():
    # 5 uneven catalogues, 7 bins x 2 orders: S = 4 leaves a ragged tail of 3 bins,
    # C = 2 a ragged tail of one catalogue
    torch, H = _hermes()
    L, N, p = 200.0, 64, 4
    edges = np.linspace(4.0, 60.0, 8)
    ells = (0, 2)
    pos, w, offs = _batch(L, N, [3000, 20000, 700, 12000, 5000], seed=11)
    with H.Context(L, N, p) as ctx:
        ctx.set_stream(torch.cuda.Stream())
        ctx.window_shells(edges, l_max=2)
        ctx.batch_set_plan(4, 2)
        got = ctx.xi_multipoles_batch(pos, w, offs, ells)
        info = ctx.batch_info()
    assert got.shape == (5, 2, 7)
    assert (info["S"], info["C"]) == (4, 2) and info["graph_kernels"] > 0
    ref = _single(H, L, N, p, edges, 2, pos, w, offs, ells)
    _close(got, ref)
    for k in (0, 2):
        a, b = offs[k], offs[k + 1]
        o = O.xi_multipoles(pos[a:b], w[a:b], N, L, p, edges, ells=ells)["xi"]
        _close(got[k], o)


@pytest.mark.parametrize("plan", [(4, 1), (8, 3), (16, 6), (32, 2)])
def test_batch_plans_agree(plan):
    torch, H = _hermes()
    L, N, p = 150.0, 32, 3
    edges = np.linspace(3.0, 50.0, 11)
    ells = (0, 2, 4)
    pos, w, offs = _batch(L, N, [400, 2500, 900, 1600, 300, 5000], seed=23, weights=False)
    ref = _single(H, L, N, p, edges, 4, pos, None, offs, ells)
    with H.Context(L, N, p) as ctx:
        ctx.set_stream(torch.cuda.Stream())
        ctx.window_shells(edges, l_max=4)
        ctx.batch_set_plan(*plan)
        got = ctx.xi_multipoles_batch(pos, None, offs, ells)
    _close(got, ref)


def test_batch_graph_is_replayed_with_new_offsets_and_data():
    torch, H = _hermes()
    L, N, p = 100.0, 32, 4
    edges = np.linspace(3.0, 40.0, 6)
    ells = (0,)
    pos, w, offs = _batch(L, N, [1000, 3000, 2000], seed=5)
    # same total and shape, different split and data: the cached graph serves both
    n = int(offs[-1])
    pos2 = S.poisson_uniform(n, L, seed=7).astype(np.float32)
    w2 = S.lognormal_masses(n, seed=8).astype(np.float32)
    offs2 = np.array([0, n // 2, n // 2 + n // 6, n], dtype=np.int64)
    with H.Context(L, N, p) as ctx:
        ctx.set_stream(torch.cuda.Stream())
        ctx.window_shells(edges, l_max=0)
        ctx.batch_set_plan(4, 3)
        a = ctx.xi_multipoles_batch(pos, w, offs, ells)
        i1 = ctx.batch_info()
        b = ctx.xi_multipoles_batch(pos2, w2, offs2, ells)
        i2 = ctx.batch_info()
        a2 = ctx.xi_multipoles_batch(torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda(), offs, ells)
        i3 = ctx.batch_info()
    assert i2["graph_replays"] == i1["graph_replays"] + 1
    assert i3["graph_replays"] == i2["graph_replays"] + 1
    _close(a, _single(H, L, N, p, edges, 0, pos, w, offs, ells))
    _close(b, _single(H, L, N, p, edges, 0, pos2, w2, offs2, ells))
    _close(a2, a)


def test_batch_autotuner_picks_a_timed_plan():
    torch, H = _hermes()
    L, N, p = 120.0, 32, 4
    edges = np.linspace(3.0, 50.0, 13)
    pos, w, offs = _batch(L, N, [800, 1500, 600, 2000, 1000], seed=31)
    with H.Context(L, N, p) as ctx:
        ctx.set_stream(torch.cuda.Stream())
        ctx.window_shells(edges, l_max=2)
        got = ctx.xi_multipoles_batch(pos, w, offs, (0, 2))
        info = ctx.batch_info()
    tried = {(int(s), int(c)) for s, c, _ in info["tuning"]}
    assert (info["S"], info["C"]) in tried and len(tried) >= 3
    best = min(info["tuning"], key=lambda t: t[2])
    assert (int(best[0]), int(best[1])) == (info["S"], info["C"])
    _close(got, _single(H, L, N, p, edges, 2, pos, w, offs, (0, 2)))


def test_batch_eager_launches_match_the_graph():
    torch, H = _hermes()
    L, N, p = 100.0, 16, 2
    edges = np.linspace(2.0, 30.0, 5)
    pos, w, offs = _batch(L, N, [500, 900], seed=41)
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=0)
        ctx.batch_set_plan(4, 2)
        n0 = ctx.launch_count()
        eager = ctx.xi_multipoles_batch(pos, w, offs, (0,), graph=False)
        n_eager = ctx.launch_count() - n0
        assert ctx.batch_info()["graph_replays"] == 0
        graphed = ctx.xi_multipoles_batch(pos, w, offs, (0,))
        info = ctx.batch_info()
        assert info["graph_replays"] == 1 and info["graph_kernels"] == n_eager
    _close(eager, _single(H, L, N, p, edges, 0, pos, w, offs, (0,)))
    _close(graphed, eager)


def test_batch_argument_and_range_errors():
    torch, H = _hermes()
    L, N, p = 100.0, 16, 4
    pos, w, offs = _batch(L, N, [300, 400], seed=3)
    with H.Context(L, N, p) as ctx:
        with pytest.raises(H.HermesError) as ei:  # no bins yet
            ctx.xi_multipoles_batch(pos, w, offs, (0,))
        assert ei.value.code == H.ERR_STATE
        ctx.window_shells([2.0, 10.0, 20.0], l_max=2)
        for bad_offs in ([0, 300, 300, 700], [1, 300, 700]):
            n = bad_offs[-1]
            with pytest.raises(H.HermesError) as ei:
                ctx.xi_multipoles_batch(pos[:n], w[:n], np.array(bad_offs), (0,))
            assert ei.value.code == H.ERR_ARG
        with pytest.raises(H.HermesError) as ei:
            ctx.xi_multipoles_batch(pos, w, offs, (1,))
        assert ei.value.code == H.ERR_ARG
        with pytest.raises(H.HermesError) as ei:
            ctx.batch_set_plan(6, 2)
        assert ei.value.code == H.ERR_ARG
        bad = pos.copy()
        bad[350, 1] = 2 * L  # in the second catalogue
        with pytest.raises(H.HermesError) as ei:
            ctx.xi_multipoles_batch(bad, w, offs, (0,))
        assert ei.value.code == H.ERR_RANGE
        wz = w.copy()
        wz[300:] = 0.0  # second catalogue weighs nothing
        with pytest.raises(H.HermesError) as ei:
            ctx.xi_multipoles_batch(pos, wz, offs, (0,))
        assert ei.value.code == H.ERR_RANGE and "catalogue 1" in str(ei.value)
        got = ctx.xi_multipoles_batch(pos, w, offs, (0, 2))  # the context still works
        assert np.all(np.isfinite(got))


def test_batch_many_small_catalogues_grow_the_result_buffers():
    # 40 catalogues x 2 orders x 20 bins: results and sums outgrow the context's
    # initial pinned read-back buffer; the batch state must survive the growth
    torch, H = _hermes()
    L, N, p = 80.0, 16, 4
    edges = np.linspace(2.0, 38.0, 21)
    sizes = S.batched_catalogue_sizes(40, 50, 600, seed=9)
    cats = [S.poisson_uniform(int(n), L, seed=200 + k) for k, n in enumerate(sizes)]
    offs = np.concatenate([[0], np.cumsum([c.shape[0] for c in cats])]).astype(np.int64)
    pos = np.concatenate(cats).astype(np.float32)
    with H.Context(L, N, p) as ctx:
        ctx.set_stream(torch.cuda.Stream())
        ctx.window_shells(edges, l_max=2)
        ctx.batch_set_plan(8, 16)
        a = ctx.xi_multipoles_batch(pos, None, offs, (0, 2))
        b = ctx.xi_multipoles_batch(pos, None, offs, (0, 2))
        assert ctx.batch_info()["graph_replays"] == 2
    assert a.shape == (40, 2, 20)
    ref = _single(H, L, N, p, edges, 2, pos, None, offs, (0, 2))
    _close(a, ref)
    _close(b, ref)
