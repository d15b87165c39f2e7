"""Python binding of libhermes.so (ctypes; argument marshalling only).

Every step of the estimator runs in the CUDA library; this module converts
numpy arrays / torch tensors to pointers and status codes to exceptions.  If the
shared library is missing the import fails loudly -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhermes.so")

OK = 0
ERR_ARG = -1
ERR_RANGE = -2
ERR_NOMEM = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_STATE = -6
DEVICE_PTR = 1
WRAP = 2
EAGER = 4
SMOOTH_SPHERE, SMOOTH_GAUSS = 0, 1
MARK_DENSITY, MARK_POWER, MARK_INVERSE = 0, 1, 2

_NAMES = {ERR_ARG: "HERMES_ERR_ARG", ERR_RANGE: "HERMES_ERR_RANGE", ERR_NOMEM: "HERMES_ERR_NOMEM",
          ERR_CUDA: "HERMES_ERR_CUDA", ERR_TIMEOUT: "HERMES_ERR_TIMEOUT", ERR_STATE: "HERMES_ERR_STATE"}


class HermesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


STAT_XI, STAT_XI_MULTIPOLES, STAT_ZETA = 0, 1, 2


class Request(C.Structure):
    """hermes_request (include/hermes.h)."""
    _fields_ = [("L", C.c_double), ("N", C.c_int), ("p", C.c_int), ("stat", C.c_int),
                ("r_edges", C.POINTER(C.c_double)), ("n_edges", C.c_int),
                ("ells", C.POINTER(C.c_int)), ("n_ells", C.c_int), ("l_max", C.c_int),
                ("pos", C.c_void_p), ("w", C.c_void_p), ("n", C.c_int64), ("flags", C.c_uint),
                ("field_id", C.c_int64), ("out", C.POINTER(C.c_double))]


class Result(C.Structure):
    """hermes_result (include/hermes.h)."""
    _fields_ = [("status", C.c_int), ("reused_field", C.c_int), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double), ("device_bytes", C.c_int64), ("msg", C.c_char * 256)]


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhermes.so not built at {LIB_PATH}; run `python paper_2607_23494_b300/build.py`")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dp, fp, u32 = C.c_void_p, C.c_int, C.c_int64, C.POINTER(C.c_double), C.c_void_p, C.c_uint
    sig = {
        "hermes_create": (i32, [C.c_double, i32, i32, i32, C.POINTER(vp)]),
        "hermes_destroy": (i32, [vp]),
        "hermes_set_stream": (i32, [vp, vp]),
        "hermes_release_buffers": (i32, [vp]),
        "hermes_assign": (i32, [vp, fp, fp, i64, u32]),
        "hermes_assign_noalloc": (i32, [vp, fp, fp, i64, u32]),
        "hermes_assign_randoms": (i32, [vp, fp, fp, i64, u32]),
        "hermes_clear_randoms": (i32, [vp]),
        "hermes_density_marks": (i32, [vp, i32, C.c_double, i32, C.c_double, C.c_double, i32, fp, i64, u32, fp]),
        "hermes_window_shells": (i32, [vp, dp, i32, i32]),
        "hermes_xi": (i32, [vp, dp]),
        "hermes_xi_multipoles": (i32, [vp, C.POINTER(i32), i32, dp]),
        "hermes_xi_multipoles_kspace": (i32, [vp, C.POINTER(i32), i32, dp]),
        "hermes_xi_multipoles_batch": (i32, [vp, vp, vp, C.POINTER(C.c_int64), i32, C.POINTER(i32), i32, C.c_uint,
                                             dp]),
        "hermes_batch_set_plan": (i32, [vp, i32, i32]),
        "hermes_batch_info": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64), dp, i32, C.POINTER(i32)]),
        "hermes_zeta_multipoles": (i32, [vp, dp]),
        "hermes_ddd_monopole": (i32, [vp, dp]),
        "hermes_window_cylinders": (i32, [vp, dp, i32, dp, i32, C.c_double]),
        "hermes_xi_cylinders": (i32, [vp, dp]),
        "hermes_xi_cylinders_kspace": (i32, [vp, dp]),
        "hermes_window_rings": (i32, [vp, dp, dp, dp, dp, i32, C.c_double]),
        "hermes_xi_rings": (i32, [vp, dp]),
        "hermes_xi_rings_kspace": (i32, [vp, dp]),
        "hermes_last_error": (C.c_char_p, [vp]),
        "hermes_debug_get_delta": (i32, [vp, fp]),
        "hermes_debug_get_spectrum": (i32, [vp, fp]),
        "hermes_debug_set_delta": (i32, [vp, fp]),
        "hermes_debug_get_sums": (i32, [vp, dp, dp]),
        "hermes_debug_nodes": (i32, [vp, fp, i64, u32, fp, fp]),
        "hermes_debug_bounded_wait": (i32, [vp]),
        "hermes_debug_fail_allocs": (i32, [i32]),
        "hermes_shell_table_host": (i32, [C.c_double, i32, dp, i32, i32, dp]),
        "hermes_shell_table_len": (i64, [i32]),
        "hermes_trace_enable": (i32, [vp, i32]),
        "hermes_trace_read": (i32, [vp, dp, C.POINTER(i64), i32]),
        "hermes_kernel_name": (C.c_char_p, [i32]),
        "hermes_launch_count": (i64, [vp]),
        "hermes_device_bytes": (i64, [vp]),
        "hermes_estimate_bytes": (i64, [i32, i32, i32, i32, i64, i32]),
        "hermes_fft_set_variant": (i32, [i32, i32, i32]),
        "hermes_fft_variants": (i32, [i32, i32, C.POINTER(i32), dp, i32, C.POINTER(i32), C.POINTER(i32)]),
        "hermes_server_create": (i32, [i32, i64, i32, C.POINTER(vp)]),
        "hermes_server_submit": (i32, [vp, C.POINTER(Request), C.POINTER(i64)]),
        "hermes_server_wait": (i32, [vp, i64, C.POINTER(Result)]),
        "hermes_server_stats": (i32, [vp, C.POINTER(i64), i32]),
        "hermes_server_destroy": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib() -> C.CDLL:
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def shell_table_host(L: float, N: int, r_edges: Sequence[float], l_max: int) -> np.ndarray:
    """Host-built float64 table <j_l>_b(k_q), shape [n_bins, l_max+1, Q]."""
    e = np.ascontiguousarray(r_edges, dtype=np.float64)
    Q = int(_lib.hermes_shell_table_len(N))
    if Q < 0:
        raise HermesError(ERR_ARG, f"bad N={N}")
    out = np.empty((len(e) - 1, l_max + 1, Q), dtype=np.float64)
    rc = _lib.hermes_shell_table_host(float(L), int(N), _dptr(e), len(e), int(l_max), _dptr(out))
    if rc != OK:
        raise HermesError(rc, "hermes_shell_table_host")
    return out


class Context:
    """One resident field on one GPU: hermes_create ... hermes_destroy."""

    def __init__(self, L: float, N: int, p: int = 4):
        j = int(N).bit_length() - 1
        h = C.c_void_p()
        rc = _lib.hermes_create(float(L), int(N), int(p), j, C.byref(h))
        if rc != OK:
            raise HermesError(rc, f"hermes_create(L={L}, N={N}, p={p})")
        self._h = h
        self.L, self.N, self.p = float(L), int(N), int(p)
        self.n_bins = 0
        self.l_max = -1

    def close(self):
        if getattr(self, "_h", None):
            _lib.hermes_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc: int, what: str):
        if rc != OK:
            msg = _lib.hermes_last_error(self._h)
            raise HermesError(rc, f"{what}: {msg.decode() if msg else ''}")

    def release_buffers(self) -> None:
        """hermes_release_buffers: free the transient device buffers; the field stays."""
        self._check(_lib.hermes_release_buffers(self._h), "hermes_release_buffers")

    def set_stream(self, stream) -> None:
        """stream: a torch.cuda.Stream, an integer handle, or None for the context's own stream."""
        handle = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._check(_lib.hermes_set_stream(self._h, handle), "hermes_set_stream")

    def assign(self, pos, w=None, wrap: bool = False) -> None:
        """pos: (n,3) float32 numpy array or CUDA tensor; w: (n,) float32 or None."""
        flags = WRAP if wrap else 0
        if hasattr(pos, "data_ptr"):  # torch tensor
            import torch
            assert pos.dtype == torch.float32 and pos.is_contiguous() and pos.dim() == 2 and pos.shape[1] == 3
            n = pos.shape[0]
            wp = None
            if w is not None:
                assert w.dtype == torch.float32 and w.is_contiguous() and w.shape[0] == n
                wp = w.data_ptr() if w.is_cuda else w.data_ptr()
            if pos.is_cuda:
                flags |= DEVICE_PTR
                if w is not None and not w.is_cuda:
                    raise ValueError("pos and w must live on the same kind of memory")
            rc = _lib.hermes_assign(self._h, pos.data_ptr(), wp, n, flags)
        else:
            pos = np.ascontiguousarray(pos, dtype=np.float32)
            if pos.ndim != 2 or pos.shape[1] != 3:
                raise ValueError("pos must have shape (n, 3)")
            n = pos.shape[0]
            wp = None
            if w is not None:
                w = np.ascontiguousarray(w, dtype=np.float32)
                if w.shape != (n,):
                    raise ValueError("w must have shape (n,)")
                wp = w.ctypes.data
            rc = _lib.hermes_assign(self._h, pos.ctypes.data if n else None, wp, n, flags)
        self._check(rc, "hermes_assign")

    def _points(self, pos, w):
        """(pos pointer, w pointer, n, device flag, keep-alive) for numpy arrays or torch tensors."""
        if hasattr(pos, "data_ptr"):
            import torch
            assert pos.dtype == torch.float32 and pos.is_contiguous() and pos.dim() == 2 and pos.shape[1] == 3
            if w is not None:
                assert w.dtype == torch.float32 and w.is_contiguous() and w.is_cuda == pos.is_cuda
            return pos.data_ptr(), (None if w is None else w.data_ptr()), pos.shape[0], \
                (DEVICE_PTR if pos.is_cuda else 0), (pos, w)
        pos = np.ascontiguousarray(pos, dtype=np.float32)
        if pos.ndim != 2 or pos.shape[1] != 3:
            raise ValueError("pos must have shape (n, 3)")
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float32)
            if w.shape != (pos.shape[0],):
                raise ValueError("w must have shape (n,)")
        return pos.ctypes.data if pos.shape[0] else None, (None if w is None else w.ctypes.data), pos.shape[0], 0, \
            (pos, w)

    def assign_randoms(self, pos, w=None, wrap: bool = False) -> None:
        """hermes_assign_randoms: an explicit random catalogue for the Landy-Szalay estimator;
        call assign() with the data afterwards."""
        pp, wp, n, flags, _keep = self._points(pos, w)
        self._check(_lib.hermes_assign_randoms(self._h, pp, wp, n, flags | (WRAP if wrap else 0)),
                    "hermes_assign_randoms")

    def density_marks(self, pos, window: str = "sphere", R: float = 8.0, kind: str = "density", a: float = 1.0,
                      b: float = 0.0, remove_self: bool = False, wrap: bool = False):
        """hermes_density_marks: smoothed density (kind "density") or the "power" / "inverse" mark at
        every position; numpy in, numpy out (CUDA tensor in, CUDA tensor out)."""
        win = {"sphere": SMOOTH_SPHERE, "gauss": SMOOTH_GAUSS}[window]
        kd = {"density": MARK_DENSITY, "power": MARK_POWER, "inverse": MARK_INVERSE}[kind]
        pp, _, n, flags, keep = self._points(pos, None)
        if flags & DEVICE_PTR:
            import torch
            out = torch.empty(n, dtype=torch.float32, device=pos.device)
            op = out.data_ptr()
        else:
            out = np.empty(n, dtype=np.float32)
            op = out.ctypes.data
        self._check(_lib.hermes_density_marks(self._h, win, float(R), kd, float(a), float(b), int(remove_self), pp, n,
                                              flags | (WRAP if wrap else 0), op), "hermes_density_marks")
        return out

    def clear_randoms(self) -> None:
        self._check(_lib.hermes_clear_randoms(self._h), "hermes_clear_randoms")

    def assign_noalloc(self, pos, w=None, wrap: bool = False) -> None:
        """hermes_assign_noalloc: pos / w are CUDA tensors; no device memory is allocated."""
        n = pos.shape[0]
        rc = _lib.hermes_assign_noalloc(self._h, pos.data_ptr(), None if w is None else w.data_ptr(), n,
                                        WRAP if wrap else 0)
        self._check(rc, "hermes_assign_noalloc")

    def window_shells(self, r_edges: Sequence[float], l_max: int = 0) -> None:
        e = np.ascontiguousarray(r_edges, dtype=np.float64)
        self._check(_lib.hermes_window_shells(self._h, _dptr(e), len(e), int(l_max)), "hermes_window_shells")
        self.n_bins = len(e) - 1
        self.l_max = int(l_max)

    def xi(self) -> np.ndarray:
        out = np.empty(self.n_bins, dtype=np.float64)
        self._check(_lib.hermes_xi(self._h, _dptr(out)), "hermes_xi")
        return out

    def xi_multipoles(self, ells: Sequence[int]) -> np.ndarray:
        ea = np.ascontiguousarray(ells, dtype=np.int32)
        out = np.empty((len(ea), self.n_bins), dtype=np.float64)
        self._check(_lib.hermes_xi_multipoles(self._h, ea.ctypes.data_as(C.POINTER(C.c_int)), len(ea), _dptr(out)),
                    "hermes_xi_multipoles")
        return out

    def xi_multipoles_kspace(self, ells: Sequence[int]) -> np.ndarray:
        ea = np.ascontiguousarray(ells, dtype=np.int32)
        out = np.empty((len(ea), self.n_bins), dtype=np.float64)
        self._check(_lib.hermes_xi_multipoles_kspace(self._h, ea.ctypes.data_as(C.POINTER(C.c_int)), len(ea),
                                                     _dptr(out)), "hermes_xi_multipoles_kspace")
        return out

    def xi_multipoles_batch(self, pos, w, offsets, ells: Sequence[int], wrap: bool = False,
                            graph: bool = True) -> np.ndarray:
        """xi_l of every catalogue: catalogue k is rows offsets[k]:offsets[k+1] of pos (n,3) and w (n,) or None.
        pos / w: float32 numpy arrays or torch tensors (CUDA tensors are read in place).
        Returns [n_cat, len(ells), n_bins]."""
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        n_cat = len(offs) - 1
        ea = np.ascontiguousarray(ells, dtype=np.int32)
        flags = (WRAP if wrap else 0) | (0 if graph else EAGER)
        keep = []
        if hasattr(pos, "data_ptr"):
            import torch
            assert pos.dtype == torch.float32 and pos.is_contiguous() and pos.dim() == 2 and pos.shape[1] == 3
            if w is not None:
                assert w.dtype == torch.float32 and w.is_contiguous() and w.is_cuda == pos.is_cuda
            if pos.is_cuda:
                flags |= DEVICE_PTR
            pp, wp = pos.data_ptr(), (None if w is None else w.data_ptr())
        else:
            pos = np.ascontiguousarray(pos, dtype=np.float32)
            if pos.ndim != 2 or pos.shape[1] != 3:
                raise ValueError("pos must have shape (n, 3)")
            keep.append(pos)
            pp = pos.ctypes.data
            wp = None
            if w is not None:
                w = np.ascontiguousarray(w, dtype=np.float32)
                keep.append(w)
                wp = w.ctypes.data
        if n_cat >= 1 and offs[-1] != pos.shape[0]:
            raise ValueError(f"offsets[-1] = {offs[-1]} but pos has {pos.shape[0]} rows")
        out = np.empty((max(n_cat, 0), len(ea), self.n_bins), dtype=np.float64)
        rc = _lib.hermes_xi_multipoles_batch(self._h, pp, wp, offs.ctypes.data_as(C.POINTER(C.c_int64)), n_cat,
                                             ea.ctypes.data_as(C.POINTER(C.c_int)), len(ea), flags, _dptr(out))
        self._check(rc, "hermes_xi_multipoles_batch")
        return out

    def batch_set_plan(self, S: int = 0, C_: int = 0) -> None:
        self._check(_lib.hermes_batch_set_plan(self._h, int(S), int(C_)), "hermes_batch_set_plan")

    def batch_info(self) -> dict:
        S, Cc, n_t = C.c_int(), C.c_int(), C.c_int()
        gk, gr = C.c_int64(), C.c_int64()
        tune = np.zeros(3 * 64, dtype=np.float64)
        self._check(_lib.hermes_batch_info(self._h, C.byref(S), C.byref(Cc), C.byref(gk), C.byref(gr), _dptr(tune),
                                           64, C.byref(n_t)), "hermes_batch_info")
        n = min(n_t.value, 64)
        return {"S": S.value, "C": Cc.value, "graph_kernels": gk.value, "graph_replays": gr.value,
                "tuning": [tuple(tune[3 * i:3 * i + 3]) for i in range(n)]}

    def window_cylinders(self, perp_edges: Sequence[float], par_edges: Sequence[float],
                         sigma_perp: float = 0.0) -> None:
        pe = np.ascontiguousarray(perp_edges, dtype=np.float64)
        ze = np.ascontiguousarray(par_edges, dtype=np.float64)
        self._check(_lib.hermes_window_cylinders(self._h, _dptr(pe), len(pe), _dptr(ze), len(ze), float(sigma_perp)),
                    "hermes_window_cylinders")
        self.n_perp, self.n_par = len(pe) - 1, len(ze) - 1

    def xi_cylinders(self, kspace: bool = False) -> np.ndarray:
        """xi(r_perp, r_par) as [n_par, n_perp]; kspace=True uses the Parseval route."""
        out = np.empty((self.n_par, self.n_perp), dtype=np.float64)
        f = _lib.hermes_xi_cylinders_kspace if kspace else _lib.hermes_xi_cylinders
        self._check(f(self._h, _dptr(out)), "hermes_xi_cylinders" + ("_kspace" if kspace else ""))
        return out

    def window_rings(self, R: Sequence[float], H: Sequence[float], dR=None, dH=None,
                     sigma_perp: float = 0.0) -> None:
        """Ring windows at the (R, H) = (r_perp, r_par) points (hermes_window_rings); dR, dH
        are per-ring widths (scalars broadcast; None = thin)."""
        r = np.ascontiguousarray(R, dtype=np.float64).ravel()
        h = np.ascontiguousarray(H, dtype=np.float64).ravel()
        if r.shape != h.shape:
            raise HermesError(ERR_ARG, "R and H need the same length")

        def widths(d):
            if d is None:
                return None
            return np.ascontiguousarray(np.broadcast_to(np.asarray(d, dtype=np.float64), r.shape))

        wr, wh = widths(dR), widths(dH)
        self._check(_lib.hermes_window_rings(self._h, _dptr(r), _dptr(h), None if wr is None else _dptr(wr),
                                             None if wh is None else _dptr(wh), len(r), float(sigma_perp)),
                    "hermes_window_rings")
        self.n_rings = len(r)

    def window_s_mu(self, s: Sequence[float], mu: Sequence[float], ds: float = 0.0, dmu: float = 0.0,
                    sigma_perp: float = 0.0) -> None:
        """Ring windows on the s x mu sample grid of xi(s, mu) (ordered [s][mu]):
        r_perp = s sqrt(1 - mu^2), r_par = s mu; thin when ds = dmu = 0, otherwise each ring
        gets widths dR = ds and dH = s dmu."""
        sv = np.asarray(s, dtype=np.float64)
        mv = np.asarray(mu, dtype=np.float64)
        R = (sv[:, None] * np.sqrt(np.clip(1.0 - mv[None, :] ** 2, 0.0, None))).ravel()
        H = (sv[:, None] * mv[None, :]).ravel()
        thin = ds == 0.0 and dmu == 0.0
        dH = None if thin else np.repeat(sv * dmu, len(mv))
        self.window_rings(R, H, dR=None if thin else ds, dH=dH, sigma_perp=sigma_perp)
        self.s_mu_shape = (len(sv), len(mv))

    def xi_rings(self, kspace: bool = False) -> np.ndarray:
        """xi for every ring window (n,); kspace=True uses the Parseval route."""
        out = np.empty(self.n_rings, dtype=np.float64)
        f = _lib.hermes_xi_rings_kspace if kspace else _lib.hermes_xi_rings
        self._check(f(self._h, _dptr(out)), "hermes_xi_rings" + ("_kspace" if kspace else ""))
        return out

    def zeta_multipoles(self) -> np.ndarray:
        out = np.empty((self.l_max + 1, self.n_bins, self.n_bins), dtype=np.float64)
        self._check(_lib.hermes_zeta_multipoles(self._h, _dptr(out)), "hermes_zeta_multipoles")
        return out

    def ddd_monopole(self) -> np.ndarray:
        """hermes_ddd_monopole: the 3PCF monopole DDD(b1, b2) by triple connection
        coefficients, [n_bins, n_bins] (at most 16 bins)."""
        out = np.empty((self.n_bins, self.n_bins), dtype=np.float64)
        self._check(_lib.hermes_ddd_monopole(self._h, _dptr(out)), "hermes_ddd_monopole")
        return out

    # tracing
    def trace(self, on: bool = True) -> None:
        self._check(_lib.hermes_trace_enable(self._h, 1 if on else 0), "hermes_trace_enable")

    def trace_read(self) -> dict:
        """{kernel name: (device ms, launches)} since the last enable/read."""
        ms = np.zeros(32, dtype=np.float64)
        cnt = np.zeros(32, dtype=np.int64)
        k = _lib.hermes_trace_read(self._h, _dptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64)), 32)
        if k < 0:
            self._check(k, "hermes_trace_read")
        return {_lib.hermes_kernel_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(k) if cnt[i] > 0}

    def launch_count(self) -> int:
        return int(_lib.hermes_launch_count(self._h))

    # inspection hooks
    def get_delta(self) -> np.ndarray:
        out = np.empty((self.N,) * 3, dtype=np.float32)
        self._check(_lib.hermes_debug_get_delta(self._h, out.ctypes.data), "hermes_debug_get_delta")
        return out

    def get_spectrum(self) -> np.ndarray:
        out = np.empty((self.N, self.N, self.N // 2), dtype=np.complex64)
        self._check(_lib.hermes_debug_get_spectrum(self._h, out.ctypes.data), "hermes_debug_get_spectrum")
        return out

    def set_delta(self, delta: np.ndarray) -> None:
        d = np.ascontiguousarray(delta, dtype=np.float32)
        assert d.shape == (self.N,) * 3
        self._check(_lib.hermes_debug_set_delta(self._h, d.ctypes.data), "hermes_debug_set_delta")

    def nodes(self, pos, wrap: bool = False):
        """Device node rule: (first[n,3] int32, weights[n,3,p] float32)."""
        pos = np.ascontiguousarray(pos, dtype=np.float32)
        n = pos.shape[0]
        first = np.empty((n, 3), dtype=np.int32)
        wts = np.empty((n, 3, self.p), dtype=np.float32)
        self._check(_lib.hermes_debug_nodes(self._h, pos.ctypes.data, n, WRAP if wrap else 0,
                                            first.ctypes.data, wts.ctypes.data), "hermes_debug_nodes")
        return first, wts

    def get_sums(self):
        s = np.empty(2, dtype=np.float64)
        t = np.empty(self.p ** 3, dtype=np.float64)
        self._check(_lib.hermes_debug_get_sums(self._h, _dptr(s), _dptr(t)), "hermes_debug_get_sums")
        return s, t.reshape(self.p, self.p, self.p)


def estimate_bytes(N: int, stat: int, n_bins: int, l_max: int, n_points: int, host_inputs: bool = True) -> int:
    """hermes_estimate_bytes: device footprint of one request of this kind (-1 on a bad argument)."""
    return int(_lib.hermes_estimate_bytes(int(N), int(stat), int(n_bins), int(l_max), int(n_points),
                                          1 if host_inputs else 0))


PASS_INV_Y, PASS_WINDOW, PASS_CONTRACT, PASS_ZETA_Y, PASS_ZETA_X, PASS_ZETA_X_M0 = 0, 1, 2, 3, 4, 5


def fft_variants(N: int, pass_: int = PASS_INV_Y) -> dict:
    """hermes_fft_variants: the variants of an FFT pass for grid size N, as
    {"variants": [(kind, E, W, minb), ...], "ms": [...], "chosen": i, "forced": j}."""
    desc = np.zeros(4 * 8, dtype=np.int32)
    ms = np.zeros(8, dtype=np.float64)
    chosen, forced = C.c_int(-1), C.c_int(-1)
    n = _lib.hermes_fft_variants(int(N), int(pass_), desc.ctypes.data_as(C.POINTER(C.c_int)), _dptr(ms), 8,
                                 C.byref(chosen), C.byref(forced))
    if n < 0:
        raise HermesError(n, "hermes_fft_variants")
    return {"variants": [tuple(int(x) for x in desc[4 * i:4 * i + 4]) for i in range(n)],
            "ms": [float(x) for x in ms[:n]], "chosen": chosen.value, "forced": forced.value}


def fft_set_variant(N: int, variant: int, pass_: int = PASS_INV_Y) -> None:
    """hermes_fft_set_variant: fix a variant for grid size N (-1: autotune again)."""
    rc = _lib.hermes_fft_set_variant(int(N), int(pass_), int(variant))
    if rc != OK:
        raise HermesError(rc, "hermes_fft_set_variant")


class Server:
    """hermes_server_*: continuous-batching request server on one GPU.

    submit() returns a ticket; the arrays it was given (positions, weights) are
    kept referenced until wait() returns the (result array, hermes_result) pair."""

    def __init__(self, device: int = 0, hbm_budget: int = 64 << 30, n_streams: int = 4):
        h = C.c_void_p()
        rc = _lib.hermes_server_create(int(device), int(hbm_budget), int(n_streams), C.byref(h))
        if rc != OK:
            raise HermesError(rc, f"hermes_server_create(device={device}, budget={hbm_budget}, "
                                  f"streams={n_streams})")
        self._h = h
        self._live = {}

    def submit(self, L: float, N: int, p: int, stat: int, r_edges, pos=None, w=None, ells=None, l_max: int = 0,
               field_id: int = -1, wrap: bool = False) -> int:
        edges = np.ascontiguousarray(r_edges, dtype=np.float64)
        nb = len(edges) - 1
        keep = [edges]
        flags = WRAP if wrap else 0
        n = 0
        pp = wp = None
        if pos is not None:
            if hasattr(pos, "data_ptr"):
                if pos.is_cuda:
                    flags |= DEVICE_PTR
                pp, n = pos.data_ptr(), pos.shape[0]
                wp = None if w is None else w.data_ptr()
                keep += [pos, w]
            else:
                pos = np.ascontiguousarray(pos, dtype=np.float32)
                pp, n = pos.ctypes.data, pos.shape[0]
                keep.append(pos)
                if w is not None:
                    w = np.ascontiguousarray(w, dtype=np.float32)
                    wp = w.ctypes.data
                    keep.append(w)
        ea = None
        if stat == STAT_XI:
            shape = (nb,)
        elif stat == STAT_XI_MULTIPOLES:
            ea = np.ascontiguousarray(ells, dtype=np.int32)
            keep.append(ea)
            shape = (len(ea), nb)
        else:
            shape = (l_max + 1, nb, nb)
        out = np.zeros(shape, dtype=np.float64)
        req = Request(L=float(L), N=int(N), p=int(p), stat=int(stat), r_edges=_dptr(edges), n_edges=len(edges),
                      ells=None if ea is None else ea.ctypes.data_as(C.POINTER(C.c_int)),
                      n_ells=0 if ea is None else len(ea), l_max=int(l_max), pos=pp, w=wp, n=int(n),
                      flags=flags, field_id=int(field_id), out=_dptr(out))
        t = C.c_int64()
        rc = _lib.hermes_server_submit(self._h, C.byref(req), C.byref(t))
        if rc != OK:
            raise HermesError(rc, "hermes_server_submit")
        self._live[t.value] = (out, keep)
        return t.value

    def wait(self, ticket: int):
        res = Result()
        rc = _lib.hermes_server_wait(self._h, int(ticket), C.byref(res))
        if rc != OK:
            raise HermesError(rc, f"hermes_server_wait({ticket})")
        out, _ = self._live.pop(ticket)
        return out, {"status": res.status, "reused_field": bool(res.reused_field), "queue_ms": res.queue_ms,
                     "latency_ms": res.latency_ms, "device_bytes": res.device_bytes,
                     "msg": res.msg.decode(errors="replace")}

    def stats(self) -> dict:
        v = (C.c_int64 * 9)()
        _lib.hermes_server_stats(self._h, v, 9)
        keys = ["completed", "in_flight", "queued", "bytes_reserved", "peak_bytes_reserved", "peak_in_flight",
                "reused_fields", "resident_contexts", "evicted"]
        return dict(zip(keys, list(v)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.hermes_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
