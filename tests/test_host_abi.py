"""CPU checks of the C ABI: the library loads, exports every declared entry point,
validates arguments before touching a GPU, and its float64 host window tables
agree with the oracle's independent quadrature."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import hermes_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hermes.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hermes_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2607_23494_b300 import hermes as H
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(H.lib(), n), n


def test_create_rejects_bad_arguments_without_a_gpu():
    from paper_2607_23494_b300 import hermes as H
    lib = H.lib()
    h = ctypes.c_void_p()
    assert lib.hermes_create(100.0, 48, 4, 5, ctypes.byref(h)) == H.ERR_ARG   # not a power of two
    assert lib.hermes_create(100.0, 64, 4, 5, ctypes.byref(h)) == H.ERR_ARG   # N != 2^j
    assert lib.hermes_create(-1.0, 64, 4, 6, ctypes.byref(h)) == H.ERR_ARG
    assert lib.hermes_create(100.0, 64, 9, 6, ctypes.byref(h)) == H.ERR_ARG   # p > 8
    assert lib.hermes_create(100.0, 16, 9, 4, ctypes.byref(h)) == H.ERR_ARG
    assert lib.hermes_create(100.0, 64, 4, 6, None) == H.ERR_ARG
    assert lib.hermes_destroy(None) == H.OK
    assert lib.hermes_shell_table_len(48) == -1


def test_no_gpu_means_an_error_status_not_a_crash():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2607_23494_b300 import hermes as H
    h = ctypes.c_void_p()
    assert H.lib().hermes_create(100.0, 64, 4, 6, ctypes.byref(h)) == H.ERR_CUDA
    assert not h.value


@pytest.mark.parametrize("N,L", [(64, 250.0), (32, 1000.0)])
def test_host_shell_tables_match_oracle_quadrature(N, L):
    from paper_2607_23494_b300 import shell_table_host
    # orders up to 24 (the paper's 3PCF runs reach l_max 20): the series and the closed-form
    # recurrences must each be used only where they are accurate
    edges = [0.0, 2.0, 5.0, 7.5, 30.0, 100.0, L / 2]
    l_max = 24
    tab = shell_table_host(L, N, edges, l_max)
    Q = tab.shape[-1]
    assert Q == 3 * (N // 2 - 1) ** 2 + 1
    q = np.arange(Q)
    k = 2 * np.pi * np.sqrt(q) / L
    for b in range(len(edges) - 1):
        lo, hi = edges[b], edges[b + 1]
        ref0 = O.shell_window_l0(k, lo, hi)
        np.testing.assert_allclose(tab[b, 0], ref0, rtol=1e-10, atol=1e-13)
        for ell in range(1, l_max + 1):
            ref = O.shell_avg_jl(ell, k, lo, hi)
            np.testing.assert_allclose(tab[b, ell], ref, rtol=1e-8, atol=1e-11 + 1e-9 * np.abs(ref).max(),
                                       err_msg=f"bin {b} l {ell}")


def test_host_tables_reject_bad_edges():
    from paper_2607_23494_b300 import hermes as H
    with pytest.raises(H.HermesError):
        H.shell_table_host(100.0, 32, [5.0, 5.0, 10.0], 0)
    with pytest.raises(H.HermesError):
        H.shell_table_host(100.0, 32, [-1.0, 5.0], 0)


def test_server_and_accounting_entry_points_without_a_gpu():
    import torch
    from paper_2607_23494_b300 import hermes as H
    lib = H.lib()
    h = ctypes.c_void_p()
    assert lib.hermes_server_create(0, 1 << 30, 0, ctypes.byref(h)) == H.ERR_ARG     # no worker
    assert lib.hermes_server_create(0, 0, 2, ctypes.byref(h)) == H.ERR_ARG           # no budget
    assert lib.hermes_server_create(0, 1 << 30, 2, None) == H.ERR_ARG
    assert lib.hermes_server_destroy(None) == H.OK
    assert lib.hermes_device_bytes(None) == -1
    if not torch.cuda.is_available():
        assert lib.hermes_server_create(0, 1 << 30, 2, ctypes.byref(h)) == H.ERR_CUDA
        assert not h.value


def test_footprint_estimate_follows_the_allocation_rules():
    from paper_2607_23494_b300.hermes import STAT_XI, STAT_XI_MULTIPOLES, STAT_ZETA, estimate_bytes
    assert estimate_bytes(48, STAT_XI, 10, 0, 1000) == -1
    assert estimate_bytes(64, 3, 10, 0, 1000) == -1
    assert estimate_bytes(64, STAT_XI, 0, 0, 1000) == -1
    for N in (64, 256, 1024):
        n3 = N ** 3
        xi = estimate_bytes(N, STAT_XI, 40, 0, 10 ** 6, host_inputs=False)
        # grid (4 B) + half spectrum (4 B) + at least four windows of work (4 B each) per cell
        assert 24 * n3 <= xi < 24 * n3 + 72 * n3 + (1 << 26)
        # zeta keeps n_bins full complex fields (8 B per cell each)
        z = estimate_bytes(N, STAT_ZETA, 12, 4, 10 ** 6, host_inputs=False)
        assert z >= 8 * n3 + 12 * 8 * n3
        # host inputs are staged: 16 B per point
        assert estimate_bytes(N, STAT_XI, 40, 0, 10 ** 6, host_inputs=True) - xi == 16 * 10 ** 6
        # more orders only enlarge the tables
        assert estimate_bytes(N, STAT_XI_MULTIPOLES, 40, 4, 10 ** 6, host_inputs=False) > xi
    assert estimate_bytes(512, STAT_XI, 40, 0, 0) > estimate_bytes(256, STAT_XI, 40, 0, 0)


def test_allocation_failure_hook_counts_without_a_gpu():
    from paper_2607_23494_b300 import hermes as H
    lib = H.lib()
    assert lib.hermes_debug_fail_allocs(3) == 0
    assert lib.hermes_debug_fail_allocs(-5) == 3     # negative disarms
    assert lib.hermes_debug_fail_allocs(0) == 0


def test_fft_variant_table_and_arguments_without_a_gpu():
    # the inverse y pass has a radix-8 variant everywhere and 16 / 32 values per
    # thread (radix-16 / radix-32 stages) from 128^3 up; fixing one is recorded,
    # -1 returns to autotuning, anything else is an argument error
    from paper_2607_23494_b300 import hermes as H
    for N, n_min in ((16, 1), (64, 1), (128, 2), (256, 3), (512, 3), (1024, 2)):
        info = H.fft_variants(N)
        assert len(info["variants"]) >= n_min
        kind, E, W, _ = info["variants"][0]
        assert (kind, E) == (0, 8)
        for kind, E, W, minb in info["variants"]:
            assert kind in (0, 1, 2) and E in (8, 16, 32) and W >= 1 and N % E == 0
    # the window pass: one window at a time everywhere; two windows in flight, or the k_y and
    # N - k_y lines together, at 256^3 and 512^3, and at 512^3 (8-column tiles) the same in the
    # paired order (kind 4, and kind 5 by tiled bulk stores; the zeta_l x pass has kind 4);
    # the contraction pass: radix 8 everywhere, 16 values per thread at 256^3 and 512^3 (kind 2:
    # its split twiddles in a shared table);
    # the zeta_l y pass: radix 8 everywhere, 16 or 32 values per thread at 256^3 and 512^3
    # (and 16-column tiles at 256^3 and 512^3)
    for pass_, N, kinds in ((1, 64, [0]), (1, 256, [0, 1, 2, 3]), (1, 512, [0, 1, 2, 3, 4, 5]), (2, 64, [0]),
                            (2, 256, [0, 1, 1, 1, 2]), (2, 512, [0, 1, 1, 1, 2]), (2, 1024, [0]), (3, 64, [0]),
                            (3, 256, [0, 1, 1, 1, 1]), (3, 512, [0, 1, 1, 1, 1]), (4, 512, [0, 2, 3, 4]),
                            (5, 512, [0, 2, 3, 4]), (5, 256, [0, 2, 3]), (4, 1024, [0])):
        info = H.fft_variants(N, pass_)
        assert [v[0] for v in info["variants"]] == kinds
    n512 = len(H.fft_variants(512)["variants"])
    H.fft_set_variant(512, 1)
    assert H.fft_variants(512)["forced"] == 1
    H.fft_set_variant(512, -1)
    info = H.fft_variants(512)
    assert info["forced"] == -1 and info["chosen"] == -1 and all(m == -1.0 for m in info["ms"])
    for bad in ((48, 0, 0), (512, n512, 0), (512, -2, 0), (512, 0, 6), (512, 6, 1), (256, 4, 1), (512, 5, 2), (512, 5, 3),
                (512, 4, 4), (256, 3, 5)):
        with pytest.raises(H.HermesError) as ei:
            H.fft_set_variant(bad[0], bad[1], pass_=bad[2])
        assert ei.value.code == H.ERR_ARG
    with pytest.raises(H.HermesError):
        H.fft_variants(2048)
