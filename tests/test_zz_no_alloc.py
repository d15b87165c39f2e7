"""hermes_assign_noalloc: the scatter entry point for callers that cannot allocate
GPU memory while they run -- hosts whose device memory belongs to an allocator of
their own (a framework's caching pool, a fixed budget), where a cudaMalloc behind
their back may fail and a cudaFree stalls every stream, and serving loops that must
not wait on the allocator.  Its reduction scratch is a fixed static device array
instead of context buffers that grow on demand.

Through the C ABI, two calls in a row must reproduce what hermes_assign gives for
the same inputs (resident field, sums, self-pair table and the xi_l measured from
it), and sizes beyond the fixed scratch and host pointers must be rejected.
Kept in a file that pytest collects last, so that a stop at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from synthetic import catalogues as S

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-6


def _env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_23494_b300 import hermes as H
    return torch, H


def _state(ctx, ells):
    s, tab = ctx.get_sums()
    return ctx.get_delta().astype(np.float64), ctx.get_spectrum(), s, tab, ctx.xi_multipoles(ells)


def test_noalloc_matches_assign_on_two_calls_in_a_row():
    torch, H = _env()
    L, N, p = 200.0, 64, 4
    edges = np.linspace(4.0, 60.0, 9)
    ells = (0, 2)
    cat_a = (S.mixed_poisson_sp(20000, L, seed=101), None)
    pos_b = S.lognormal_catalogue(30000, L, seed=102, n_grid=64)
    cat_b = (pos_b, S.lognormal_masses(pos_b.shape[0], seed=103))
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=2)
        dev = []
        for pos, w in (cat_a, cat_b):
            dev.append((torch.from_numpy(pos).cuda(), None if w is None else torch.from_numpy(w).cuda()))
        refs = []
        for tpos, tw in dev:
            ctx.assign(tpos, tw)
            refs.append(_state(ctx, ells))
        for (tpos, tw), ref in zip(dev, refs):  # two no-alloc calls back to back
            ctx.assign_noalloc(tpos, tw)
            got = _state(ctx, ells)
            d, spec, sums, tab, xi = got
            rd, rspec, rsums, rtab, rxi = ref
            assert np.max(np.abs(d - rd) / (1.0 + np.abs(rd))) < 1e-5
            assert np.linalg.norm(spec - rspec) <= 1e-5 * np.linalg.norm(rspec)
            np.testing.assert_allclose(sums, rsums, rtol=1e-12)
            np.testing.assert_allclose(tab, rtab, rtol=1e-5)
            err = np.abs(xi - rxi)
            assert np.all(err <= np.maximum(REL * np.abs(rxi), ABS)), (xi, rxi)


def test_noalloc_rejects_orders_beyond_its_scratch():
    torch, H = _env()
    pos = torch.from_numpy(S.poisson_uniform(1000, 100.0, seed=5)).cuda()
    with H.Context(100.0, 32, 7) as ctx:
        with pytest.raises(H.HermesError) as ei:
            ctx.assign_noalloc(pos)
        assert ei.value.code == H.ERR_ARG
        assert "p <= 6" in str(ei.value)
        ctx.assign(pos)  # the allocating entry point still serves this order


def test_noalloc_rejects_host_pointers():
    torch, H = _env()
    pos = S.poisson_uniform(1000, 100.0, seed=6)
    with H.Context(100.0, 32, 4) as ctx:
        rc = H.lib().hermes_assign_noalloc(ctx._h, pos.ctypes.data_as(ctypes.c_void_p), None, 1000, 0)
        assert rc == H.ERR_ARG
