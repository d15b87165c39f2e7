"""The request server (hermes_server_*): continuous batching on one GPU.

Every result must be the same alone (its own context, nothing else running)
and in a mix of concurrent requests of other grid sizes, statistics and
catalogues, within the estimator's tolerance (1e-4 relative or 1e-6 absolute);
admission must keep the reserved device memory within the budget; resident
fields must be reused across statistics.
"""
import numpy as np
import pytest

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


GRIDS = {"a": (200.0, 64, 4), "b": (100.0, 32, 3), "c": (160.0, 128, 4)}


def _catalogues():
    cats = {}
    for fid, (g, n, seed) in enumerate([("a", 20000, 1), ("a", 8000, 2), ("b", 5000, 3), ("c", 30000, 4)]):
        L = GRIDS[g][0]
        pos = S.lognormal_catalogue(n, L, seed=seed, n_grid=32) if seed % 2 else S.mixed_poisson_sp(n, L, seed=seed)
        cats[fid] = (g, pos.astype(np.float32), S.lognormal_masses(pos.shape[0], seed=seed + 50).astype(np.float32))
    return cats


def _requests(H, cats):
    """A mix of statistics over the catalogues (several per field, so fields get reused)."""
    reqs = []
    for fid, (g, pos, w) in cats.items():
        L = GRIDS[g][0]
        reqs.append(dict(fid=fid, stat=H.STAT_XI, edges=np.linspace(L / 50, L / 4, 11)))
        reqs.append(dict(fid=fid, stat=H.STAT_XI_MULTIPOLES, edges=np.linspace(L / 40, L / 5, 9), ells=(0, 2, 4)))
        if g != "c":
            reqs.append(dict(fid=fid, stat=H.STAT_ZETA, edges=np.linspace(L / 30, L / 5, 7), l_max=2))
    return reqs


def _alone(H, cats, q):
    g, pos, w = cats[q["fid"]]
    L, N, p = GRIDS[g]
    with H.Context(L, N, p) as ctx:
        ctx.assign(pos, w)
        if q["stat"] == H.STAT_XI:
            ctx.window_shells(q["edges"], l_max=0)
            return ctx.xi()
        if q["stat"] == H.STAT_XI_MULTIPOLES:
            ctx.window_shells(q["edges"], l_max=max(q["ells"]))
            return ctx.xi_multipoles(q["ells"])
        ctx.window_shells(q["edges"], l_max=q["l_max"])
        return ctx.zeta_multipoles()


def _submit(srv, H, cats, q, with_pos=True):
    g, pos, w = cats[q["fid"]]
    L, N, p = GRIDS[g]
    return srv.submit(L, N, p, q["stat"], q["edges"], pos=pos if with_pos else None, w=w if with_pos else None,
                      ells=q.get("ells"), l_max=q.get("l_max", 0), field_id=q["fid"])


def test_results_are_the_same_alone_and_in_the_mix():
    torch, H = _hermes()
    cats = _catalogues()
    reqs = _requests(H, cats)
    alone = [_alone(H, cats, q) for q in reqs]
    with H.Server(0, hbm_budget=16 << 30, n_streams=4) as srv:
        order = np.random.default_rng(3).permutation(len(reqs))
        tickets = {int(i): _submit(srv, H, cats, reqs[i]) for i in order}
        got = {i: srv.wait(t) for i, t in tickets.items()}
        st = srv.stats()
    for i, (out, res) in got.items():
        assert res["status"] == H.OK, res["msg"]
        _close(out, alone[i])
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["in_flight"] == 0
    assert st["peak_in_flight"] >= 2, st           # requests overlapped on the device
    assert st["reused_fields"] >= 1, st            # fields served several statistics
    assert st["peak_bytes_reserved"] <= 16 << 30


def test_admission_keeps_within_a_tight_budget():
    torch, H = _hermes()
    cats = _catalogues()
    reqs = _requests(H, cats)
    alone = [_alone(H, cats, q) for q in reqs]
    biggest = 0
    for q in reqs:
        g, pos, _ = cats[q["fid"]]
        lm = {H.STAT_XI: 0, H.STAT_XI_MULTIPOLES: 4, H.STAT_ZETA: q.get("l_max", 0)}[q["stat"]]
        biggest = max(biggest, H.estimate_bytes(GRIDS[g][1], q["stat"], len(q["edges"]) - 1, lm, pos.shape[0]))
    budget = int(biggest * 1.2)
    with H.Server(0, hbm_budget=budget, n_streams=4) as srv:
        tickets = [_submit(srv, H, cats, q) for q in reqs]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    for (out, res), ref in zip(got, alone):
        assert res["status"] == H.OK, res["msg"]
        _close(out, ref)
    assert st["peak_bytes_reserved"] <= budget, (st, budget)
    assert st["evicted"] >= 1, st


def test_resident_field_serves_a_later_statistic_without_positions():
    torch, H = _hermes()
    cats = _catalogues()
    q1 = dict(fid=0, stat=H.STAT_XI, edges=np.linspace(4.0, 50.0, 11))
    q2 = dict(fid=0, stat=H.STAT_XI_MULTIPOLES, edges=np.linspace(5.0, 40.0, 9), ells=(0, 2))
    with H.Server(0, hbm_budget=8 << 30, n_streams=2) as srv:
        a, ra = srv.wait(_submit(srv, H, cats, q1))
        b, rb = srv.wait(_submit(srv, H, cats, q2, with_pos=False))
        c, rc = srv.wait(srv.submit(200.0, 64, 4, H.STAT_XI, q1["edges"], field_id=99))  # nothing resident
    assert ra["status"] == H.OK and not ra["reused_field"]
    assert rb["status"] == H.OK and rb["reused_field"], rb
    _close(a, _alone(H, cats, q1))
    _close(b, _alone(H, cats, q2))
    assert rc["status"] == H.ERR_ARG and "field_id" in rc["msg"]


def test_server_errors_and_oversized_requests():
    torch, H = _hermes()
    cats = _catalogues()
    g, pos, w = cats[2]
    L, N, p = GRIDS[g]
    with H.Server(0, hbm_budget=1 << 20, n_streams=1) as srv:  # 1 MiB: nothing fits
        out, res = srv.wait(srv.submit(L, N, p, H.STAT_XI, [2.0, 10.0, 20.0], pos=pos))
        assert res["status"] == H.ERR_NOMEM
        with pytest.raises(H.HermesError):
            srv.submit(L, N, p, 7, [2.0, 10.0], pos=pos)
        with pytest.raises(H.HermesError):
            srv.submit(L, N, p, H.STAT_XI, [2.0], pos=pos)
        with pytest.raises(H.HermesError):
            srv.wait(12345)
    with H.Server(0, hbm_budget=4 << 30, n_streams=2) as srv:
        bad = pos.copy()
        bad[10, 0] = 3 * L
        out, res = srv.wait(srv.submit(L, N, p, H.STAT_XI, [2.0, 10.0, 20.0], pos=bad, field_id=5))
        assert res["status"] == H.ERR_RANGE
        out, res = srv.wait(srv.submit(L, N, p, H.STAT_XI, [2.0, 10.0, 20.0], field_id=5))  # not resident
        assert res["status"] == H.ERR_ARG
        out, res = srv.wait(srv.submit(L, N, p, H.STAT_XI, [2.0, 10.0, 20.0], pos=pos, w=w, field_id=5))
        assert res["status"] == H.OK


def test_contexts_on_concurrent_host_threads_with_different_window_batches():
    # Two host threads drive their own 256^3 contexts at once: one measures 40 shells
    # (window batches of 16, 16 and 8), the other 5 shells (one batch of 5), and the
    # zeta_l pass runs beside them with its own bin count.  The batches stage radial
    # tables of different sizes in shared memory; every launch must still run and
    # every result equal the same call made alone.
    import threading
    torch, H = _hermes()
    L, N, p = 400.0, 256, 4
    pos = S.lognormal_catalogue(60000, L, seed=33, n_grid=64)
    jobs = {"wide": (np.linspace(4.0, 84.0, 41), "xi"), "narrow": (np.linspace(6.0, 31.0, 6), "xi"),
            "zeta": (np.linspace(8.0, 40.0, 7), "zeta")}

    def run(edges, kind, reps, out, key):
        try:
            with H.Context(L, N, p) as ctx:
                ctx.window_shells(edges, l_max=2)
                ctx.assign(pos)
                res = []
                for _ in range(reps):
                    res.append(ctx.xi_multipoles([0, 2]) if kind == "xi" else ctx.zeta_multipoles())
                out[key] = res
        except Exception as e:  # reported by the main thread
            out[key] = e

    alone = {}
    for key, (edges, kind) in jobs.items():
        run(edges, kind, 1, alone, key)
        assert not isinstance(alone[key], Exception), alone[key]
    mixed = {}
    threads = [threading.Thread(target=run, args=(edges, kind, 6, mixed, key)) for key, (edges, kind) in jobs.items()]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for key in jobs:
        assert not isinstance(mixed[key], Exception), (key, mixed[key])
        for r in mixed[key]:
            _close(r, alone[key][0])


def test_release_buffers_keeps_the_field_and_frees_the_transients():
    torch, H = _hermes()
    L, N, p = 200.0, 64, 4
    pos = S.lognormal_catalogue(20000, L, seed=44, n_grid=64)
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(np.linspace(4.0, 60.0, 9), l_max=2)
        ctx.assign(pos)
        xi = ctx.xi_multipoles([0, 2])
        z = ctx.zeta_multipoles()
        full = H.lib().hermes_device_bytes(ctx._h)
        ctx.release_buffers()
        small = H.lib().hermes_device_bytes(ctx._h)
        assert small < full - 8 * N ** 3 * 8      # at least the 8 harmonic fields are gone
        np.testing.assert_allclose(ctx.xi_multipoles([0, 2]), xi, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(ctx.zeta_multipoles(), z, rtol=1e-9, atol=1e-12)
