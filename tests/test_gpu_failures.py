"""Failure detection on the GPU without faulting it.

  * Bounded device waits: a kernel waits, with the same bounded mbarrier wait that
    guards the bulk-copy pipelines, on a barrier phase that nothing completes (no
    copy is issued).  The wait must give up, the call must report
    HERMES_ERR_TIMEOUT, and the context must keep working.
  * Allocation failures: a host-side hook makes the library's next device
    allocations report out of memory.  The failing call must return
    HERMES_ERR_NOMEM without leaking or losing what it held, and a retry must
    succeed with the same result.
"""
import time

import numpy as np
import pytest

from synthetic import catalogues as S

pytestmark = pytest.mark.gpu


def _hermes():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_23494_b300 import hermes as H
    return H


def test_bounded_wait_gives_up_and_the_context_survives():
    H = _hermes()
    L, N, p = 100.0, 32, 4
    pos = S.mixed_poisson_sp(4000, L, seed=17)
    edges = np.linspace(3.0, 30.0, 6)
    with H.Context(L, N, p) as ctx:
        ctx.window_shells(edges, l_max=2)
        ctx.assign(pos)
        before = ctx.xi_multipoles([0, 2])
        t0 = time.time()
        rc = H.lib().hermes_debug_bounded_wait(ctx._h)
        dt = time.time() - t0
        assert rc == H.ERR_TIMEOUT
        assert b"gave up" in H.lib().hermes_last_error(ctx._h)
        assert 0.5 < dt < 30.0, dt
        after = ctx.xi_multipoles([0, 2])       # same context, same stream, still usable
        np.testing.assert_array_equal(after, before)
        ctx.assign(pos)   # a new scatter: float atomics may add in another order
        again = ctx.xi_multipoles([0, 2])
        assert np.all(np.abs(again - before) <= np.maximum(1e-4 * np.abs(before), 1e-6))


def test_allocation_failure_reports_nomem_keeps_state_and_recovers():
    H = _hermes()
    lib = H.lib()
    L, N, p = 120.0, 64, 4
    pos = S.lognormal_catalogue(20000, L, seed=23, n_grid=64)
    edges = np.linspace(4.0, 40.0, 10)
    try:
        # creation: the first device allocation fails, the context is not created
        lib.hermes_debug_fail_allocs(1)
        with pytest.raises(H.HermesError) as ei:
            H.Context(L, N, p)
        assert ei.value.code == H.ERR_NOMEM
        assert lib.hermes_debug_fail_allocs(0) == 0   # the failure was consumed
        with H.Context(L, N, p) as ref_ctx:
            ref_ctx.window_shells(edges, l_max=2)
            ref_ctx.assign(pos)
            ref = ref_ctx.xi_multipoles([0, 2])
        with H.Context(L, N, p) as ctx:
            ctx.window_shells(edges, l_max=2)
            ctx.assign(pos)
            held = lib.hermes_device_bytes(ctx._h)
            # the first measurement grows the window work buffer: make that fail
            lib.hermes_debug_fail_allocs(1)
            with pytest.raises(H.HermesError) as ei:
                ctx.xi_multipoles([0, 2])
            assert ei.value.code == H.ERR_NOMEM
            assert lib.hermes_device_bytes(ctx._h) == held
            got = ctx.xi_multipoles([0, 2])          # the resident field survived
            np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9)
            # a failing staging allocation in assign (host inputs) leaves no field behind
            ctx2 = H.Context(L, N, p)
            try:
                ctx2.window_shells(edges, l_max=0)
                lib.hermes_debug_fail_allocs(1)
                with pytest.raises(H.HermesError) as ei:
                    ctx2.assign(pos)
                assert ei.value.code == H.ERR_NOMEM
                with pytest.raises(H.HermesError) as ei:
                    ctx2.xi()
                assert ei.value.code == H.ERR_STATE
                ctx2.assign(pos)
                np.testing.assert_allclose(ctx2.xi(), ref[0], rtol=1e-6, atol=1e-9)
            finally:
                ctx2.close()
    finally:
        lib.hermes_debug_fail_allocs(0)
