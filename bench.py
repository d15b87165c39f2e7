#!/usr/bin/env python
"""Benchmark of the field-window estimator on B300.

One step = one full 2PCF measurement of a 512^3 field through the C ABI:
  1e7 points Poisson-sampled from a lognormal field (P(k) ~ k^-1.5 exp(-(k/0.5)^2),
  sigma_ln = 1) in a periodic box L = 1000 Mpc/h, cubic B-spline (p = 4);
  40 linear shells in [2, 202) Mpc/h; multipoles l = 0, 2, 4 along z;
  done once with unit weights and once with log-normal masses (marked field):
  2 scatters + 2 forward 3-D FFTs + 240 windows (window multiply, inverse 3-D FFT,
  cell contraction, self-pair subtraction).
metric = grid cells x windows per second = 512^3 * 240 / step time.

Also reported: the 3PCF multipoles zeta_l (2e6 points, L = 500, 512^3, 16 shells in
[10, 170), l_max = 6) as an extra measurement, the dominant kernel's achieved HBM
bandwidth from live CUDA events, clocks sampled during the timed region, an
end-to-end number through host buffers, and the FP64 oracle timed on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hermes|reference] [--no-zeta]
Under torchrun every rank runs its own replica (independent catalogue); the
value is the aggregate over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-cell x window evals/s at 512^3"
UNIT = "cell-window/s"

# workload (the isotropic + anisotropic 2PCF configuration, with its marked variant)
L2, N2, P2, NPTS2 = 1000.0, 512, 4, 10_000_000
EDGES2 = np.linspace(2.0, 202.0, 41)
ELLS2 = (0, 2, 4)
# batched configuration
L4, N4, NCAT4 = 500.0, 256, 64
EDGES4 = np.linspace(5.0, 155.0, 31)
# serving configuration
L5, NPOOL5 = 1000.0, 6
# 3PCF multipoles configuration
L3, N3, NPTS3 = 500.0, 512, 2_000_000
EDGES3 = np.linspace(10.0, 170.0, 17)
LMAX3 = 6


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def rank_seeds(rank: int) -> dict:
    """Seeds of each replica's independent catalogues (one set per rank)."""
    return {"xi": 1234 + 17 * rank, "batch": 777 + 17 * rank, "serve": 4242 + 17 * rank, "zeta": 4321 + 17 * rank}


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time: all_reduce(MAX) over the process group (nccl on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(cells: float, windows_per_step: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job throughput of `world` replicas: every rank's cell-windows over the slowest rank's time."""
    return world * cells * windows_per_step * steps / (ms_max / 1e3)


def gen_catalogue(seed: int):
    from synthetic import catalogues as S
    pos = S.lognormal_catalogue(NPTS2, L2, seed=seed, n_grid=512)
    mass = S.lognormal_masses(pos.shape[0], seed=seed + 1)
    return pos, mass


def gen_catalogue3(seed: int):
    from synthetic import catalogues as S
    return S.lognormal_catalogue(NPTS3, L3, seed=seed, n_grid=512)


# Stored FP64 oracle values (written by tests/golden/make_fullsize_golden.py) for the
# per-statistic error report; each file carries a digest of the catalogue it was made from.
GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_golden(name: str):
    try:
        with open(os.path.join(GOLDEN, name)) as f:
            return json.load(f)
    except OSError:
        return None


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def err_stats(got, ref) -> dict:
    """Largest absolute and relative error and the largest error in units of the
    tolerance (1e-4 relative or 1e-6 absolute; <= 1 passes)."""
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    err = np.abs(got - ref)
    big = np.abs(ref) > 1e-6
    return {"n": int(ref.size), "max_abs_err": float(err.max()),
            "max_rel_err": float((err[big] / np.abs(ref[big])).max()) if big.any() else None,
            "max_in_tolerance_units": round(float((err / np.maximum(1e-4 * np.abs(ref), 1e-6)).max()), 4)}


def error_vs_oracle(res, pos, mass, zeta128) -> dict:
    """Error of every statistic against the FP64 oracle at the configuration sizes:
    xi of the 20,000-point 64^3 catalogue in full; xi_l (l = 0, 2, 4) of the timed
    1e7-point 512^3 step, unit and marked fields, on 6 of the 40 shells; zeta_l of the
    2e6-point catalogue regridded on 128^3 (l_max = 6, 16 shells) in full."""
    from paper_2607_23494_b300 import Context
    from synthetic import catalogues as S
    out = {"tolerance": "1e-4 relative or 1e-6 absolute (max_in_tolerance_units <= 1 passes); max_rel_err over "
                        "entries with |oracle| > 1e-6",
           "oracle": "stored FP64 oracle values, tests/golden/make_fullsize_golden.py"}
    g = load_golden("xi_mixed_2e4_64.json")
    if g:
        c = g["config"]
        p1 = S.mixed_poisson_sp(c["n"], c["L"], seed=c["seed"])
        if sha256(p1) == g["pos_sha256"]:
            with Context(c["L"], c["N"], c["p"]) as ctx:
                ctx.assign(p1)
                ctx.window_shells(c["edges"], l_max=0)
                out["xi_20k_64"] = err_stats(ctx.xi(), g["xi"])
    g = load_golden("xi_lognormal_1e7_512_sample.json")
    if g and sha256(pos) == g["pos_sha256"] and sha256(mass) == g["mass_sha256"]:
        bins = g["config"]["bins"]
        for name, r in (("unit", res[0]), ("marked", res[1])):
            for a, ell in enumerate(g["config"]["ells"]):
                out[f"{name}_xi_l{ell}_1e7_512_bins_{'_'.join(map(str, bins))}"] = \
                    err_stats(np.asarray(r)[a][bins], g["xi"][name][a])
    if zeta128 is not None:
        out["zeta_l_2e6_128"] = err_stats(zeta128[0], zeta128[1])
    return out


# DRAM bytes measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) for the inverse
# passes at 512^3 on a 5-window launch of the current kernels: bytes per launch (read once
# per launch) and per window.
NCU_TRAFFIC_512 = {
    "inv_x_window/k0e8w8": {"per_launch": 0.560689e9, "per_window": 2.634067e9 / 5},
    "inv_x_window/k1e8w8": {"per_launch": 0.561371e9, "per_window": 2.634040e9 / 5},
    "inv_x_window/k2e8w8": {"per_launch": 0.576038e9, "per_window": 2.796381e9 / 5},
    "inv_x_window/k3e8w8": {"per_launch": 0.571600e9, "per_window": 2.632482e9 / 5},
    "inv_x_window/k4e8w8": {"per_launch": 0.583437e9, "per_window": 2.626260e9 / 5},
    "inv_y/k0e8w8": {"per_launch": 0.0, "per_window": (2.684387e9 + 2.630191e9) / 5},
    "inv_y/k1e32w8": {"per_launch": 0.0, "per_window": (2.684618e9 + 2.630152e9) / 5},
    "inv_y/k1e32w16": {"per_launch": 0.0, "per_window": (2.684860e9 + 2.624219e9) / 5},
    "inv_y/k1e32w16p": {"per_launch": 0.0, "per_window": (2.684456e9 + 2.624291e9) / 5},
    "inv_z_c2r_contract/k0e8w1": {"per_launch": 0.0, "per_window": (3.221783e9 + 0.005084e9) / 5},
    "inv_z_c2r_contract/k1e16w1": {"per_launch": 0.0, "per_window": (3.221317e9 + 0.013573e9) / 5},
}
TUNED_PASSES = {"inv_y": 0, "inv_x_window": 1, "inv_z_c2r_contract": 2}  # trace name -> hermes_fft_variants pass


def variant_tag(H, N: int, pass_: int) -> str:
    """The variant of a tuned pass in use for grid N as kind / values per thread / tile width
    (a trailing p: the inverse y pass reading the paired order of the window pass)."""
    def tag(p_):
        info = H.fft_variants(N, p_)
        v = info["forced"] if info["forced"] >= 0 else max(info["chosen"], 0)
        return info["variants"][v]
    kind, E, W, _ = tag(pass_)
    paired = pass_ == 0 and N == 512 and (kind, E, W) == (1, 32, 16) and tag(1)[0] == 4
    return f"k{kind}e{E}w{W}" + ("p" if paired else "")


def ncu_traffic(H, name: str, windows_per_launch: float) -> float | None:
    """DRAM bytes per launch from an ncu capture of the same kernel (None when the
    variant in use was not captured)."""
    key = f"{name}/{variant_tag(H, N2, TUNED_PASSES[name])}" if name in TUNED_PASSES else name
    t = NCU_TRAFFIC_512.get(key)
    return None if t is None else t["per_launch"] + t["per_window"] * windows_per_launch


def alg_bytes(name: str, launches: int, n_windows: int, n_batches: int, n_pts_bytes: float) -> float | None:
    """Algorithmic HBM bytes of one kernel class over the timed region (N = 512)."""
    n3 = float(N2) ** 3
    if name == "inv_y":
        return 8.0 * n3 * n_windows
    if name == "inv_x_window":
        return 4.0 * n3 * (n_windows + n_batches)
    if name == "inv_z_c2r_contract":
        return 4.0 * n3 * (n_windows + n_batches)
    if name == "fwd_z_r2c":
        return 12.0 * n3 * launches
    if name in ("fwd_y", "fwd_x"):
        return 8.0 * n3 * launches
    if name == "scatter":
        return n_pts_bytes + 4.0 * n3 * launches
    return None


def run_hermes(args, rank, world, local_rank):
    import torch
    from paper_2607_23494_b300 import Context

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(local_rank)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    pos, mass = gen_catalogue(rank_seeds(rank)["xi"])
    n = pos.shape[0]
    pos_d = torch.from_numpy(pos).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(L2, N2, P2)
    ctx.set_stream(stream)
    ctx.window_shells(EDGES2, l_max=4)
    nb = len(EDGES2) - 1
    windows_per_step = 2 * len(ELLS2) * nb
    batches_per_step = 2 * len(ELLS2) * -(-nb // 16)

    def step(p_, m_):
        ctx.assign(p_)
        a = ctx.xi_multipoles(ELLS2)
        ctx.assign(p_, m_)
        b = ctx.xi_multipoles(ELLS2)
        return a, b

    for _ in range(args.warmup):
        step(pos_d, mass_d)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_id)
    time.sleep(0.3)
    ctx.trace(True)
    launches0 = ctx.launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        res = step(pos_d, mass_d)
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    dev_ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    trace = ctx.trace_read()
    ctx.trace(False)
    clk = clocks.stop()
    ms_max = max_over_ranks(dev_ms, world, dev)
    ms_per_step = ms_max / args.steps
    cells = float(N2) ** 3
    value = replica_value(cells, windows_per_step, args.steps, ms_max, world)

    # end to end through host buffers (pinned), host->device copies inside the timed region
    pos_h = torch.from_numpy(pos).pin_memory().numpy()
    mass_h = torch.from_numpy(mass).pin_memory().numpy()
    step(pos_h, mass_h)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(pos_h, mass_h)
    e1.record(stream)
    stream.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    e2e_value = replica_value(cells, windows_per_step, args.steps, e2e_ms, world)
    h2d = 12 * n + (12 * n + 4 * n)
    d2h = 2 * 20 + 2 * 16 * (len(ELLS2) * nb)

    # roofline of the dominant kernel (live events on the launching stream)
    pk, pk_src = peaks()
    total_k_ms = sum(v[0] for v in trace.values()) or 1.0
    kern = {}
    for name, (kms, cnt) in sorted(trace.items(), key=lambda kv: -kv[1][0]):
        b = alg_bytes(name, cnt, windows_per_step * args.steps, batches_per_step * args.steps,
                      (12 * n + 16 * n) * args.steps)
        kern[name] = {"ms": round(kms, 3), "launches": cnt, "share": round(kms / total_k_ms, 4),
                      "alg_GBps": round(b / (kms / 1e3) / 1e9, 1) if b else None}
    dom = max(trace.items(), key=lambda kv: kv[1][0])[0]
    dom_b = alg_bytes(dom, trace[dom][1], windows_per_step * args.steps, batches_per_step * args.steps,
                      (12 * n + 16 * n) * args.steps)
    achieved = dom_b / (trace[dom][0] / 1e3) / 1e9 if dom_b else None
    from paper_2607_23494_b300 import hermes as Hm
    traffic = ncu_traffic(Hm, dom, windows_per_step / batches_per_step)  # per launch, scaled from ncu
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1) if achieved else None,
            "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / pk["hbm_gbs"], 4) if achieved else None,
            "traffic": round(traffic) if traffic else None,
            "alg_bytes_per_launch": round(dom_b / trace[dom][1]) if dom_b else None,
            "traffic_source": "ncu dram bytes of a 5-window launch at 512^3 scaled to this launch's windows",
            "peak_source": f"{pk_src} hbm_gbs (MEASURED_PEAKS.json)" if pk_src == "measured"
            else "fallback 6.4 TB/s"}

    # the k-space (Parseval) route on the resident marked field: same xi_l, no inverse FFTs
    ks = cyl = smu = None
    if not args.minimal:
        ks = run_kspace(ctx, stream, res[1])
        cyl = run_cylinders(ctx, stream)
        smu = run_s_mu(ctx, stream, pos_d, mass_d)
    plain = None
    if not args.no_plain:
        ctx.close()
        ctx = None
        plain = run_plain_fp32(pos_d, mass_d, res)
        plain["speedup"] = round(value / world / plain["value"], 2)

    batch = None
    if not args.no_batch:
        batch = run_batch(args, dev, stream, rank)

    serve = None
    if not args.no_serve and args.serve_requests > 0:
        serve = run_serve(args, dev, rank)

    zeta = None
    if not args.no_zeta:
        zeta = run_zeta(args, dev, stream, rank)

    if ctx is not None:
        ctx.close()
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "2PCF xi + xi_l (l=0,2,4) of a 1e7-point lognormal catalogue, unit weights and "
                                   "log-normal mass marks, 512^3 grid, L=1000 Mpc/h, p=4, 40 shells [2,202)",
                       "grid": N2, "L": L2, "p": P2, "n_points": n, "n_bins": nb, "ells": list(ELLS2),
                       "windows_per_step": windows_per_step, "parallelism": f"replicas x{world}",
                       "l2": "no flush needed: every pass streams >=512 MB (grid 512 MB, spectra 8 GB) > 126 MB L2"},
            "clocks": clk,
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "ms_per_step": round(e2e_ms / args.steps, 3),
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roof,
            "kernels": kern,
            "fft_variants": {f"{name}_{N2}": {**Hm.fft_variants(N2, p), "in_use": variant_tag(Hm, N2, p)}
                             for name, p in TUNED_PASSES.items()},
            "xi_sample": {"l0_first3": [float(x) for x in res[0][0][:3]]},
        }
        for key, val in (("kspace", ks), ("cylinders", cyl), ("s_mu", smu)):
            if val is not None:
                out[key] = val
        if plain:
            out["vs_plain_fp32"] = plain
        if batch:
            out["batch"] = batch
        if serve:
            out["serve"] = serve
        z128 = zeta.pop("_z128", None) if zeta else None
        if zeta:
            out["zeta"] = zeta
        if not args.minimal:
            out["error_vs_oracle"] = error_vs_oracle(res, pos, mass, z128)
    return out, pos


def run_cylinders(ctx, stream):
    """xi(r_perp, r_par) of the resident marked 512^3 field: 20 transverse annuli x 20
    line-of-sight slab pairs in [0, 100) Mpc/h (400 windows), by inverse transforms
    and by the Parseval route."""
    import torch
    ctx.window_cylinders(np.linspace(0.0, 100.0, 21), np.linspace(0.0, 100.0, 21))
    out = {}
    for route, ks in (("inverse_fft", False), ("kspace", True)):
        ctx.xi_cylinders(kspace=ks)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        got = ctx.xi_cylinders(kspace=ks)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        out[route] = {"ms": round(ms, 2), "cell_window_evals_per_s": round(float(N2) ** 3 * 400 / (ms / 1e3), 1)}
        out[route + "_xi"] = got
    a, b = out.pop("inverse_fft_xi"), out.pop("kspace_xi")
    out["diff_between_routes_in_tolerances"] = round(float(np.max(np.abs(a - b) / np.maximum(1e-4 * np.abs(b), 1e-6))), 4)
    out["workload"] = "xi(r_perp, r_par), marked 1e7-point field, 512^3, 20 x 20 bins in [0, 100) Mpc/h"
    return out


def run_s_mu(ctx, stream, pos_d, mass_d):
    """xi(s, mu) on ring windows at the paper's sampling of its DD(s, mu) benchmark: 46
    separations x 51 orientations = 2346 thin rings (r_perp = s sqrt(1 - mu^2), r_par = s mu),
    s = 2.5 .. 227.5 Mpc/h, mu = 0 .. 1; on the resident marked 512^3 field (both routes) and
    on the same catalogue gridded at 256^3 (the paper's J = 8)."""
    import torch
    from paper_2607_23494_b300 import Context
    s = np.arange(2.5, 230.0, 5.0)
    mu = np.linspace(0.0, 1.0, 51)
    out = {"workload": f"xi(s, mu) on {len(s)} x {len(mu)} thin ring windows, s in [2.5, 227.5] Mpc/h, mu in [0, 1], "
                       "marked 1e7-point field, L=1000"}

    def timed(c, ks):
        c.xi_rings(kspace=ks)  # warm-up
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        got = c.xi_rings(kspace=ks)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1), got

    nwin = len(s) * len(mu)
    ctx.window_s_mu(s, mu)
    res = {}
    for route, ks in (("inverse_fft", False), ("kspace", True)):
        ms, got = timed(ctx, ks)
        res[route] = got
        out[f"512_{route}"] = {"ms": round(ms, 2), "ms_per_sample": round(ms / nwin, 4),
                               "cell_window_evals_per_s": round(float(N2) ** 3 * nwin / (ms / 1e3), 1)}
    out["512_diff_between_routes_in_tolerances"] = round(float(np.max(
        np.abs(res["inverse_fft"] - res["kspace"]) / np.maximum(1e-4 * np.abs(res["kspace"]), 1e-6))), 4)
    with Context(L2, 256, P2) as c256:
        c256.set_stream(stream)
        c256.assign(pos_d, mass_d)
        c256.window_s_mu(s, mu)
        for route, ks in (("inverse_fft", False), ("kspace", True)):
            ms, _ = timed(c256, ks)
            out[f"256_{route}"] = {"ms": round(ms, 2), "ms_per_sample": round(ms / nwin, 4)}
    out["paper_context"] = "paper: 2346 ring samples at J = 8 (256^3) in 120 s on 8 MPI x 8 threads, 51.0 ms/sample"
    return out


def run_kspace(ctx, stream, real):
    import torch
    reps = 5
    got = ctx.xi_multipoles_kspace(ELLS2)
    torch.cuda.synchronize()
    ctx.trace(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        got = ctx.xi_multipoles_kspace(ELLS2)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / reps
    tr = ctx.trace_read()
    ctx.trace(False)
    nb = len(EDGES2) - 1
    n3 = float(N2) ** 3
    hist_ms = tr.get("kspace_hist", (0.0, 0))[0] / reps
    # algorithmic bytes of the histogram pass: one read of the half spectrum (8 B per stored mode)
    spec_b = 8.0 * N2 * N2 * (N2 // 2)
    # agreement with the inverse-FFT route, in units of the parity tolerance (1e-4 rel or 1e-6 abs)
    tol_units = float(np.max(np.abs(got - real) / np.maximum(1e-4 * np.abs(real), 1e-6)))
    return {"workload": "xi_l (l=0,2,4), marked 1e7-point field, 512^3, 40 shells, Parseval route",
            "ms_per_call": round(ms, 3), "cell_window_evals_per_s": round(n3 * len(ELLS2) * nb / (ms / 1e3), 1),
            "hist_ms": round(hist_ms, 3),
            "hist_GBps": round(spec_b / (hist_ms / 1e3) / 1e9, 1) if hist_ms else None,
            "diff_vs_real_space_in_tolerances": round(tol_units, 4),
            "kernels": {k: {"ms": round(v[0] / reps, 3), "launches": v[1] // reps} for k, v in tr.items()}}


class PlainPipeline:
    """The plain one-request-at-a-time FP32 pipeline on the same GPU, for the ratio
    the metric asks for: torch ops and cuFFT only (index_add_ B-spline scatter,
    rfftn, then per window: build K on the device, multiply, irfftn, cell dot
    product, self-pair term).  Comparison arm only; cubic B-spline (p = 4)."""

    def __init__(self, N, L, edges, ells, dev):
        import torch
        from paper_2607_23494_b300.hermes import shell_table_host
        self.N, self.L, self.p, self.dev, self.torch = N, L, 4, dev, torch
        p, H = self.p, N // 2
        self.T = torch.from_numpy(shell_table_host(L, N, edges, max(ells)).astype(np.float32)).to(dev)
        fxy = torch.fft.fftfreq(N, d=1.0 / N, device=dev).round().to(torch.int64)
        fz = torch.arange(H + 1, device=dev, dtype=torch.int64)
        q = (fxy[:, None, None] ** 2 + fxy[None, :, None] ** 2 + fz[None, None, :] ** 2)
        ph1 = torch.sinc(fxy.double() / N) ** (2 * p)
        ph1z = torch.sinc(fz.double() / N) ** (2 * p)
        keep = ((fxy.abs() != H)[:, None, None] & (fxy.abs() != H)[None, :, None] & (fz != H)[None, None, :])
        self.phi = (ph1[:, None, None] * ph1[None, :, None] * ph1z[None, None, :]).float() * keep
        self.q = torch.where(keep, q, torch.zeros((), device=dev, dtype=q.dtype))  # tables stop below Nyquist
        mu = torch.where(q > 0, fz[None, None, :].float() / q.float().clamp(min=1).sqrt(), torch.zeros((), device=dev))
        self.leg = {0: torch.ones_like(mu), 2: 0.5 * (3 * mu ** 2 - 1), 4: (35 * mu ** 4 - 30 * mu ** 2 + 3) / 8}
        self.wz = torch.full((H + 1,), 2.0, device=dev)
        self.wz[0] = 1.0
        self.wz[H] = 1.0
        self.cxy = torch.stack([torch.ones(N, device=dev, dtype=torch.float64)] +
                               [2 * torch.cos(2 * np.pi * fxy.double() * a / N) for a in range(1, p)], 1)
        self.cz = torch.stack([torch.ones(H + 1, device=dev, dtype=torch.float64)] +
                              [2 * torch.cos(2 * np.pi * fz.double() * a / N) for a in range(1, p)], 1)

    @staticmethod
    def _mp(x):  # centred cubic B-spline
        import torch
        ax = x.abs()
        return torch.where(ax < 1, 2.0 / 3 - ax ** 2 + 0.5 * ax ** 3,
                           torch.where(ax < 2, (2 - ax) ** 3 / 6, torch.zeros_like(ax)))

    def catalogue(self, pos, w):
        torch, N, L, p, dev = self.torch, self.N, self.L, self.p, self.dev
        grid = torch.zeros(N ** 3, device=dev, dtype=torch.float32)
        S = torch.zeros(p, p, p, device=dev, dtype=torch.float64)
        sw = torch.zeros((), device=dev, dtype=torch.float64)
        for c0 in range(0, pos.shape[0], 2_000_000):
            x = pos[c0:c0 + 2_000_000]
            ww = torch.ones(x.shape[0], device=dev) if w is None else w[c0:c0 + 2_000_000]
            u = x * np.float32(N / L)
            i = torch.floor(u)
            t = u - i
            j = torch.arange(p, device=dev, dtype=torch.float32)
            wts = self._mp(t[:, :, None] + 1 - j)                          # [n, 3, 4]
            nodes = (i.long()[:, :, None] - 1 + j.long()) % N             # [n, 3, 4]
            flat = (nodes[:, 0, :, None, None] * N + nodes[:, 1, None, :, None]) * N + nodes[:, 2, None, None, :]
            val = ww[:, None, None, None] * wts[:, 0, :, None, None] * wts[:, 1, None, :, None] * wts[:, 2, None, None, :]
            grid.index_add_(0, flat.reshape(-1), val.reshape(-1))
            sw += ww.double().sum()
            sd = torch.stack([(wts[..., :p - d] * wts[..., d:]).sum(-1) for d in range(p)], -1).double()
            S += torch.einsum("n,na,nb,nc->abc", ww.double() ** 2, sd[:, 0], sd[:, 1], sd[:, 2])
        ebar = sw / N ** 3
        delta = grid.view(N, N, N) / ebar.float() - 1
        dh = torch.fft.rfftn(delta)
        dh[0, 0, 0] = 0
        shat = torch.einsum("abc,xa,yb,zc->xyz", S, self.cxy, self.cxy, self.cz).float()
        snw = shat * self.wz / float(N) ** 6 / ebar.float() ** 2  # K carries Phi^ already
        return delta, dh, snw

    def window(self, field, b, ell):
        torch, N = self.torch, self.N
        delta, dh, snw = field
        c = (2 * ell + 1) * (-1) ** (ell // 2)
        K = c * self.T[b, ell][self.q] * self.phi * self.leg[ell]
        dt = torch.fft.irfftn(dh * K, s=(N, N, N))
        return (delta * dt).sum(dtype=torch.float64) / N ** 3 - (K * snw).sum(dtype=torch.float64)


def run_plain_fp32(pos_d, mass_d, real_res, n_win=6):
    """Plain pipeline on the 512^3 workload: the per-catalogue part is timed on both
    fields, the per-window part on n_win windows of each field (every window costs
    the same); the step estimate is 2 * catalogue + 240 * window."""
    import torch
    nb = len(EDGES2) - 1
    pp = PlainPipeline(N2, L2, EDGES2, ELLS2, pos_d.device)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    pp.catalogue(pos_d, None)  # warm-up (cuFFT plans, allocator)
    torch.cuda.synchronize()
    e[0].record()
    fields = [pp.catalogue(pos_d, None), pp.catalogue(pos_d, mass_d)]
    e[1].record()
    picks = [(b, ELLS2[k % len(ELLS2)]) for k, b in enumerate(np.linspace(0, nb - 1, n_win).astype(int))]
    pp.window(fields[0], 0, 0)
    e[2].record()
    got = [[float(pp.window(fields[f], b, ell)) for (b, ell) in picks] for f in range(2)]
    e[3].record()
    torch.cuda.synchronize()
    cat_ms = e[0].elapsed_time(e[1]) / 2
    win_ms = e[2].elapsed_time(e[3]) / (2 * n_win)
    step_ms = 2 * cat_ms + 2 * len(ELLS2) * nb * win_ms
    worst = 0.0
    for f in range(2):
        for (b, ell), g in zip(picks, got[f]):
            r = float(real_res[f][ELLS2.index(ell)][b])
            worst = max(worst, abs(g - r) / max(1e-4 * abs(r), 1e-6))
    del fields, pp
    torch.cuda.empty_cache()
    return {"value": round(N2 ** 3 * 2 * len(ELLS2) * nb / (step_ms / 1e3), 1), "unit": UNIT,
            "ms_per_step": round(step_ms, 2), "ms_per_catalogue": round(cat_ms, 3), "ms_per_window": round(win_ms, 3),
            "windows_timed": 2 * n_win, "what": "torch index_add_ scatter + cuFFT rfftn/irfftn, one window at a time",
            "diff_vs_hermes_in_tolerances": round(worst, 3)}


def gen_batch(seed: int):
    """64 lognormal catalogues, sizes log-uniform in [1e5, 5e6], one seed each."""
    from synthetic import catalogues as S
    sizes = S.batched_catalogue_sizes(NCAT4, 1e5, 5e6, seed=seed)
    cats = [S.lognormal_catalogue(int(n), L4, seed=seed + 1 + k, n_grid=128) for k, n in enumerate(sizes)]
    offs = np.concatenate([[0], np.cumsum([c.shape[0] for c in cats])]).astype(np.int64)
    return np.concatenate(cats).astype(np.float32), offs


def run_batch(args, dev, stream, rank):
    """The batched configuration: 64 uneven catalogues, 256^3, 30 shells, l = 0.
    Three arms on the same catalogues: the batched call (graph replay, autotuned
    plan), the same library one catalogue at a time, and the plain FP32 pipeline."""
    import torch
    from paper_2607_23494_b300 import Context, fft_variants
    pos, offs = gen_batch(rank_seeds(rank)["batch"])
    pos_d = torch.from_numpy(pos).to(dev)
    ncat, nb = len(offs) - 1, len(EDGES4) - 1
    cw = float(N4) ** 3 * nb * ncat  # cell-window evaluations per batch
    ctx = Context(L4, N4, 4)
    ctx.set_stream(stream)
    ctx.window_shells(EDGES4, l_max=0)
    t0 = time.time()
    ref = ctx.xi_multipoles_batch(pos_d, None, offs, (0,))  # tunes, captures the graph
    first_s = time.time() - t0
    reps = max(2, min(args.steps, 5))
    ctx.xi_multipoles_batch(pos_d, None, offs, (0,))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    e0.record(stream)
    for _ in range(reps):
        got = ctx.xi_multipoles_batch(pos_d, None, offs, (0,))
    e1.record(stream)
    stream.synchronize()
    b_ms = e0.elapsed_time(e1) / reps
    launches = (ctx.launch_count() - l0) // reps
    info = ctx.batch_info()
    # one catalogue at a time through hermes_assign + hermes_xi_multipoles
    seq = np.empty_like(got)
    e0.record(stream)
    for k in range(ncat):
        ctx.assign(pos_d[offs[k]:offs[k + 1]])
        seq[k] = ctx.xi_multipoles((0,))
    e1.record(stream)
    stream.synchronize()
    s_ms = e0.elapsed_time(e1)
    ctx.close()
    diff = float(np.max(np.abs(got - seq) / np.maximum(1e-4 * np.abs(seq), 1e-6)))
    # plain FP32 pipeline, every catalogue and window
    pp = PlainPipeline(N4, L4, EDGES4, (0,), dev)
    pp.catalogue(pos_d[:offs[1]], None)
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record()
    plain_vals = []
    for k in range(ncat):
        f = pp.catalogue(pos_d[offs[k]:offs[k + 1]], None)
        plain_vals.append([pp.window(f, b, 0) for b in range(nb)])
        del f
    plain_vals = np.array([[float(v) for v in row] for row in plain_vals])
    e3.record()
    torch.cuda.synchronize()
    p_ms = e2.elapsed_time(e3)
    pdiff = float(np.max(np.abs(plain_vals - got[:, 0, :]) / np.maximum(1e-4 * np.abs(got[:, 0, :]), 1e-6)))
    del pp
    torch.cuda.empty_cache()
    return {"workload": f"{ncat} lognormal catalogues, {int(offs[-1])} points (log-uniform sizes in [1e5, 5e6]), "
                        f"L={L4:g}, {N4}^3, p=4, {nb} shells [5,155), l=0",
            "batched": {"value": round(cw / (b_ms / 1e3), 1), "unit": UNIT, "ms_per_batch": round(b_ms, 2),
                        "plan": {"S": info["S"], "C": info["C"]}, "graph_kernels": info["graph_kernels"],
                        "gpu_launches_per_batch": launches, "first_call_s_incl_tuning": round(first_s, 2),
                        "tuning": [[int(a), int(b), round(c, 4)] for a, b, c in info["tuning"]]},
            "one_at_a_time": {"value": round(cw / (s_ms / 1e3), 1), "ms_per_batch": round(s_ms, 2),
                              "diff_vs_batched_in_tolerances": round(diff, 4)},
            "fft_variants_256": {"inv_y": fft_variants(N4, 0), "inv_x_window": fft_variants(N4, 1),
                                 "inv_z_c2r_contract": fft_variants(N4, 2)},
            "plain_fp32": {"value": round(cw / (p_ms / 1e3), 1), "ms_per_batch": round(p_ms, 2),
                           "diff_vs_batched_in_tolerances": round(pdiff, 4)},
            "speedup_vs_plain": round(p_ms / b_ms, 2), "speedup_vs_one_at_a_time": round(s_ms / b_ms, 2)}


def gen_serve_pool(seed: int):
    """Catalogues the serving trace draws from, L = 1000: six with sizes log-uniform in
    [1e5, 2e7] and one of 1e8 points (the top of the workload's size range)."""
    from synthetic import catalogues as S
    sizes = list(S.batched_catalogue_sizes(NPOOL5, 1e5, 2e7, seed=seed)) + [100_000_000]
    return [S.lognormal_catalogue(int(n), L5, seed=seed + 1 + k, n_grid=128) for k, n in enumerate(sizes)]


STAT_NAMES = ("xi", "xi_l", "zeta_l")


def serve_trace(n_req: int, rate: float, n_pool: int, seed: int, grids=(128, 256, 512, 1024),
                grid_p=(0.4, 0.3, 0.2, 0.1)):
    """Poisson arrivals (rate 0: all at once); grid 128/256/512/1024^3 with probability
    .4/.3/.2/.1; statistic xi (40 shells), xi_l (l <= 4, 40 shells) or zeta_l (l_max 4,
    12 shells) uniformly; catalogue uniform over the pool.  Even requests pass device
    inputs with the catalogue's field id (a resident field may serve them); odd requests
    pass pinned host inputs and no field id, so their host-to-device copy, scatter and
    forward transform are inside their latency."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req)) if rate > 0 else np.zeros(n_req)
    grids = rng.choice(list(grids), size=n_req, p=list(grid_p))
    stats = rng.integers(0, 3, size=n_req)
    cats = rng.integers(0, n_pool, size=n_req)
    return [(float(t[i]), int(grids[i]), int(stats[i]), int(cats[i]), i % 2 == 1) for i in range(n_req)]


SERVE_EDGES_XI = np.linspace(2.0, 202.0, 41)
SERVE_EDGES_Z = np.linspace(10.0, 130.0, 13)


def run_serve_trace(H, pool_d, pool_h, trace, n_streams, budget):
    t_wall0 = time.time()
    with H.Server(0, hbm_budget=budget, n_streams=n_streams) as srv:
        tickets = []
        t0 = time.time()
        for (ta, N, stat, k, host) in trace:
            dt = ta - (time.time() - t0)
            if dt > 0:
                time.sleep(dt)
            pos, fid = (pool_h[k], -1) if host else (pool_d[k], k)
            if stat == H.STAT_XI:
                tk = srv.submit(L5, N, 4, stat, SERVE_EDGES_XI, pos=pos, field_id=fid)
            elif stat == H.STAT_XI_MULTIPOLES:
                tk = srv.submit(L5, N, 4, stat, SERVE_EDGES_XI, pos=pos, ells=(0, 2, 4), field_id=fid)
            else:
                tk = srv.submit(L5, N, 4, stat, SERVE_EDGES_Z, pos=pos, l_max=4, field_id=fid)
            tickets.append(tk)
        res = [srv.wait(tk) for tk in tickets]
        wall = time.time() - t0
        st = srv.stats()
    lat = np.array([r[1]["latency_ms"] for r in res])
    service = lat - np.array([r[1]["queue_ms"] for r in res])
    ok = sum(1 for r in res if r[1]["status"] == H.OK)
    classes = {}
    for (ta, N, stat, k, host), l in zip(trace, lat):
        classes.setdefault(f"{N}^3 {STAT_NAMES[stat]}", []).append(l)
    per_class = {c: {"n": len(v), "p50_ms": round(float(np.percentile(v, 50)), 1),
                     "p99_ms": round(float(np.percentile(v, 99)), 1)} for c, v in sorted(classes.items())}
    failures = [{"request": i, "class": f"{trace[i][1]}^3 {STAT_NAMES[trace[i][2]]}", "n_points": len(pool_d[trace[i][3]]),
                 "host_input": trace[i][4], "status": r[1]["status"], "msg": r[1]["msg"]}
                for i, r in enumerate(res) if r[1]["status"] != H.OK]
    return {"p50_ms": round(float(np.percentile(lat, 50)), 1), "p99_ms": round(float(np.percentile(lat, 99)), 1),
            "mean_ms": round(float(lat.mean()), 1), "requests_per_s": round(len(trace) / wall, 3),
            "ok": ok, "peak_in_flight": st["peak_in_flight"], "reused_fields": st["reused_fields"],
            "evicted": st["evicted"], "peak_reserved_GB": round(st["peak_bytes_reserved"] / 2 ** 30, 1),
            "wall_s": round(wall, 1), "setup_s": round(t0 - t_wall0, 2), "per_class": per_class,
            "failures": failures}, \
        [r[0] for r in res], service


def run_serve_plain(pool_d, pool_h, trace, dev, n_max: int):
    """The plain FP32 pipeline, one request at a time, on the first n_max xi / xi_l
    requests of a trace with grids up to 512^3 (zeta_l has no plain form here); host-input
    requests copy their catalogue inside the timing, and no field is ever reused."""
    import torch
    picks = [i for i, (_, N, stat, _, _) in enumerate(trace) if stat < 2 and N <= 512][:n_max]
    pipes = {}
    lat = []
    for i in picks:
        _, N, stat, k, host = trace[i]
        if N not in pipes:
            pipes[N] = PlainPipeline(N, L5, SERVE_EDGES_XI, (0, 2, 4), dev)
        pp = pipes[N]
        ells = (0,) if stat == 0 else (0, 2, 4)
        torch.cuda.synchronize()
        t = time.perf_counter()
        f = pp.catalogue(torch.from_numpy(pool_h[k]).to(dev) if host else pool_d[k], None)
        vals = [float(pp.window(f, b, ell)) for ell in ells for b in range(len(SERVE_EDGES_XI) - 1)]
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t) * 1e3)
        del f, vals
    del pipes
    torch.cuda.empty_cache()
    return picks, np.array(lat)


def run_serve(args, dev, rank):
    """Serving: mixed requests (grids 128-1024^3, catalogues 1e5-1e8 points, xi / xi_l /
    zeta_l, half of them from pinned host memory) through the request server with 4
    concurrent workers and with 1 (the same library one request at a time):
      - open loop: Poisson arrivals at 0.75 x the measured one-at-a-time capacity
        (latency under load);
      - saturated: every request submitted at once (throughput);
      - the plain FP32 pipeline one request at a time on the saturated trace's xi / xi_l
        requests up to 512^3, against the same requests in the two server arms.
    p50 / p99 latency overall and per (grid, statistic) class."""
    import torch
    from paper_2607_23494_b300 import hermes as H
    pool = gen_serve_pool(rank_seeds(rank)["serve"])
    pool_d = [torch.from_numpy(c).to(dev) for c in pool]
    pool_h = [torch.from_numpy(c).pin_memory().numpy() for c in pool]
    budget = 200 << 30
    n_open, n_sat = args.serve_requests, max(args.serve_requests, args.serve_saturated)
    # capacity of the one-at-a-time server on a calibration trace (back to back)
    cal = serve_trace(12, 0.0, len(pool), seed=99)
    run_serve_trace(H, pool_d, pool_h, cal[:3], 1, budget)  # warm-up (tables, allocator)
    c1, _, _ = run_serve_trace(H, pool_d, pool_h, cal, 1, budget)
    capacity = c1["requests_per_s"]
    rate = 0.75 * capacity
    trace = serve_trace(n_open, rate, len(pool), seed=7)
    cont, out_c, _ = run_serve_trace(H, pool_d, pool_h, trace, 4, budget)
    one, out_1, _ = run_serve_trace(H, pool_d, pool_h, trace, 1, budget)
    sat = serve_trace(n_sat, 0.0, len(pool), seed=8)
    sat4, out_s4, _ = run_serve_trace(H, pool_d, pool_h, sat, 4, budget)
    sat1, out_s1, svc1 = run_serve_trace(H, pool_d, pool_h, sat, 1, budget)
    small = serve_trace(2 * n_sat, 0.0, len(pool) - 1, seed=9, grids=(128, 256), grid_p=(0.6, 0.4))
    sm4, out_m4, _ = run_serve_trace(H, pool_d, pool_h, small, 4, budget)
    sm1, out_m1, _ = run_serve_trace(H, pool_d, pool_h, small, 1, budget)
    worst = 0.0
    for a, b in list(zip(out_c, out_1)) + list(zip(out_s4, out_s1)) + list(zip(out_m4, out_m1)):
        if np.all(a == 0) or np.all(b == 0):  # a failed request (listed under failures)
            continue
        worst = max(worst, float(np.max(np.abs(a - b) / np.maximum(1e-4 * np.abs(b), 1e-6))))
    picks, plat = run_serve_plain(pool_d, pool_h, sat, dev, 12)
    sizes = [len(c) for c in pool]
    return {"workload": f"mixed requests, grids 128/256/512/1024^3 (p .4/.3/.2/.1), L={L5:g}, p=4; xi 40 shells / "
                        f"xi_l l<=4 / zeta_l l_max 4 12 shells; {len(pool)} lognormal catalogues of "
                        f"{min(sizes)}..{max(sizes)} points; even requests device inputs with field reuse, odd "
                        f"requests pinned host inputs (copy, scatter and transform inside the latency)",
            "open_loop": {"requests": n_open, "rate_per_s": round(rate, 3),
                          "what": f"Poisson arrivals at 0.75 x the measured one-at-a-time capacity {capacity:.2f}/s",
                          "continuous_4_streams": cont, "one_at_a_time": one},
            "saturated": {"requests": n_sat, "what": "all requests submitted at once",
                          "continuous_4_streams": sat4, "one_at_a_time": sat1,
                          "throughput_gain": round(sat4["requests_per_s"] / sat1["requests_per_s"], 3)},
            "saturated_small": {"requests": len(small),
                                "what": "all submitted at once; grids 128^3 / 256^3 (p .6 / .4), catalogues up to "
                                        "2e7 points",
                                "continuous_4_streams": sm4, "one_at_a_time": sm1,
                                "throughput_gain": round(sm4["requests_per_s"] / sm1["requests_per_s"], 3)},
            "plain_fp32_one_at_a_time": {
                "requests": len(picks), "what": "torch index_add_ scatter + cuFFT per window, xi / xi_l requests "
                                                "<= 512^3 of the saturated trace, device inputs, back to back",
                "mean_ms": round(float(plat.mean()), 1) if len(plat) else None,
                "sum_ms": round(float(plat.sum()), 1),
                "hermes_same_requests_service_sum_ms": round(float(svc1[picks].sum()), 1),
                "note": "service time = latency - queueing, from the one-at-a-time saturated arm"},
            "results_mix_vs_alone_in_tolerances": round(worst, 4),
            "reduced": f"{n_open} + {n_sat} requests instead of the workload's 1000, to keep the run to minutes"}


def run_zeta(args, dev, stream, rank):
    import torch
    from paper_2607_23494_b300 import Context
    from paper_2607_23494_b300 import hermes as Hz
    pos = gen_catalogue3(rank_seeds(rank)["zeta"])
    pos_d = torch.from_numpy(pos).to(dev)
    ctx = Context(L3, N3, 4)
    ctx.set_stream(stream)
    ctx.window_shells(EDGES3, l_max=LMAX3)

    def step():
        ctx.assign(pos_d)
        return ctx.zeta_multipoles()

    step()
    torch.cuda.synchronize()
    ctx.trace(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    zsteps = max(1, min(2, args.steps))
    e0.record(stream)
    for _ in range(zsteps):
        z = step()
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / zsteps
    tr = ctx.trace_read()
    # the 3PCF monopole by triple connection coefficients (hermes_ddd_monopole) on the same field
    # and shells, against the cell-sum zeta_0 of the step (they differ by the basis smoothing)
    ctx.window_shells(EDGES3, l_max=0)
    ctx.ddd_monopole()  # buffers
    torch.cuda.synchronize()
    ctx.trace(True)
    e0.record(stream)
    dm = ctx.ddd_monopole()
    e1.record(stream)
    stream.synchronize()
    trd = ctx.trace_read()
    ddd_cc = {"workload": "DDD(b1, b2) monopole by triple connection coefficients, the zeta_l field, 512^3, p=4, "
                          "16 shells [10,170): 125 Gauss samples per cell",
              "ms": round(e0.elapsed_time(e1), 2),
              "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in trd.items()},
              "diag_ratio_to_zeta0": [round(float(dm[b, b] / z[0, b, b]), 4) for b in range(dm.shape[0])]}
    ctx.close()
    # the paper's DDD_l(20, 40) runs (its performance table: one (r12, r13) pair at l_max 7, 14
    # and 20, J = 9 i.e. 512^3): two 2 Mpc/h shells at 20 and 40 Mpc/h on the same field
    ddd = {}
    c2 = Context(L3, N3, 4)
    c2.set_stream(stream)
    c2.assign(pos_d)
    for lm_ in (7, 14, 20):
        c2.window_shells([19.0, 21.0, 39.0, 41.0], l_max=lm_)
        c2.zeta_multipoles()  # tables and buffers
        torch.cuda.synchronize()
        e0.record(stream)
        zz = c2.zeta_multipoles()
        e1.record(stream)
        stream.synchronize()
        nm = (lm_ + 1) * (lm_ + 2) // 2
        ddd[f"l_max_{lm_}"] = {"ms": round(e0.elapsed_time(e1), 2), "m_modes": nm,
                               "ms_per_m": round(e0.elapsed_time(e1) / nm, 3), "zeta0_12": float(zz[0, 0, 2])}
    c2.close()
    ddd["paper_context"] = ("paper, J = 9 (512^3): l_max 7 in 219 s (6.07 s/m), l_max 14 in 822 s (6.85 s/m) on "
                            "12 MPI x 8 threads + an RTX 4090; shells here [19, 21) and [39, 41) Mpc/h (the paper's "
                            "r12 = 20, r13 = 40; its bin widths are not given)")
    # the same catalogue regridded on 128^3 against the stored FP64 oracle zeta_l
    z128 = None
    g = load_golden("zeta_lognormal_2e6_128_lmax6.json")
    if g and sha256(pos) == g["pos_sha256"]:
        c = g["config"]
        with Context(c["L"], c["N"], c["p"]) as c128:
            c128.set_stream(stream)
            c128.window_shells(c["edges"], l_max=c["l_max"])
            c128.assign(pos_d)
            z128 = (c128.zeta_multipoles(), np.array(g["zeta"]))
    nb = len(EDGES3) - 1
    nlm = (LMAX3 + 1) * (LMAX3 + 2) // 2
    nfields = nb * nlm
    # complex transforms actually run: the m = 0 fields are real, two bins per transform
    ntrans = nb * (nlm - (LMAX3 + 1)) + (LMAX3 + 1) * ((nb + 1) // 2)
    n3 = float(N3) ** 3
    tot = sum(v[0] for v in tr.values()) or 1.0
    # algorithmic bytes per pass over the step: Z1 reads delta^ (4 B / cell) once per (l, m) and
    # writes every transform (8 B / cell); Z2 reads and writes them (16 B); Z3 reads them (8 B)
    # and delta (4 B) once per (l, m)
    zb = {"zeta_x": (4.0 * nlm + 8.0 * ntrans) * n3, "zeta_y": 16.0 * ntrans * n3,
          "zeta_z_gram": (8.0 * ntrans + 4.0 * nlm) * n3}
    kern = {}
    for k, v in sorted(tr.items(), key=lambda kv: -kv[1][0]):
        kern[k] = {"ms": round(v[0] / zsteps, 3), "launches": v[1] // zsteps, "share": round(v[0] / tot, 4)}
        if k in zb and v[0] > 0:
            kern[k]["alg_GBps"] = round(zb[k] / (v[0] / zsteps / 1e3) / 1e9, 1)
    return {"workload": "zeta_l, 2e6-point lognormal catalogue, L=500, 512^3, 16 shells [10,170), l_max=6",
            "ms_per_step": round(ms, 2), "complex_fields": nfields, "complex_transforms": ntrans,
            "cell_field_evals_per_s": round(n3 * nfields / (ms / 1e3), 1),
            "kernels": kern, "zeta0_diag_first2": [float(z[0, 0, 0]), float(z[0, 1, 1])],
            "ddd_l_20_40": ddd, "ddd_monopole_cc": ddd_cc, "_z128": z128,
            "fft_variants": {name: {**Hz.fft_variants(N3, p_), "in_use": variant_tag(Hz, N3, p_)}
                             for name, p_ in (("zeta_y", 3), ("zeta_x", 4), ("zeta_x_m0", 5))}}


def oracle_sample(pos, b: int = 0):
    """FP64 oracle on a bounded sample: 512^3 grid, 500k points, one l=0 window (half-spectrum route)."""
    from oracle import hermes_oracle as O
    sub = pos[:500_000]
    t = time.perf_counter()
    O.xi_multipoles(sub, None, N2, L2, P2, [EDGES2[b], EDGES2[b + 1]], ells=(0,), route="half")
    dt = time.perf_counter() - t
    return float(N2) ** 3 / dt, dt


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample_all_cores(pos):
    """The same bounded sample run as one process per usable core (spawned, so no CUDA state is
    inherited), each on its own shell; each process holds ~8 GB, so the count is also bounded by
    the available host memory.  Throughput = processes x 512^3 / wall time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    k = max(1, min(cores, int(avail // (10 << 30)), 32))
    sub = np.ascontiguousarray(pos[:500_000])
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(k) as pool:
        pool.starmap(oracle_sample, [(sub, i % 40) for i in range(k)])
    wall = time.perf_counter() - t
    return k * float(N2) ** 3 / wall, wall, k, cores


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, one window per step on a resident field."""
    from oracle import hermes_oracle as O
    pos, _ = gen_catalogue(1234)
    sub = pos[:1_000_000]
    t0 = time.perf_counter()
    eps, sw, _ = O.assign(sub, None, N2, L2, P2)
    delta = O.delta_from_eps(eps, sw)
    del eps
    dh = O.forward_half(delta)
    S = O.self_pair_table(sub, None, N2, L2, P2)
    setup = time.perf_counter() - t0

    def one(b):
        K = O.window_xi(N2, L2, P2, EDGES2[b], EDGES2[b + 1], 0, half=True)
        return O.xi_parseval_half(dh, K, N2) - O.shot_noise_half(S, K, N2, sw)

    for i in range(args.warmup):
        one(i % 40)
    t = time.perf_counter()
    for i in range(args.steps):
        one(i % 40)
    dt = (time.perf_counter() - t) / args.steps
    value = float(N2) ** 3 / dt
    sample = (f"one l=0 shell window per step (window kernel, Parseval sum, self-pair term) on a resident "
              f"512^3 field of the first 1e6 of the 1e7 points; field setup {setup:.1f} s outside the steps; "
              f"numpy single thread")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "2PCF xi + xi_l (l=0,2,4) of a 1e7-point lognormal catalogue, unit weights and "
                                   "log-normal mass marks, 512^3 grid, L=1000 Mpc/h, p=4, 40 shells [2,202)",
                       "grid": N2, "L": L2, "p": P2},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """Small case for ncu captures: 512^3 field of 300k Poisson points, 5 l=0 windows (one batch).
    --y-variant / --x-variant fix the tuned passes' variants, so no tuning trials run."""
    import torch
    from paper_2607_23494_b300 import Context, fft_set_variant
    from synthetic import catalogues as S
    fft_set_variant(N2, args.y_variant, 0)
    fft_set_variant(N2, args.x_variant, 1)
    fft_set_variant(N2, args.z_variant, 2)
    pos = torch.from_numpy(S.poisson_uniform(300_000, L2, seed=7)).cuda()
    ctx = Context(L2, N2, P2)
    ctx.window_shells(np.linspace(2.0, 52.0, 6), l_max=0)
    ctx.assign(pos)
    for _ in range(2):
        x = ctx.xi()
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"profile_case": "xi 512^3, 5 windows", "xi": [float(v) for v in x]}))


def run_profile_zeta(args):
    """Small zeta case for ncu captures: 256^3 field, 200k points, 16 shells, l_max = 1.
    --zy-variant / --zx-variant fix the zeta y / x pass variants (no tuning trials)."""
    import torch
    from paper_2607_23494_b300 import Context, fft_set_variant
    from synthetic import catalogues as S
    if args.zy_variant >= 0:
        fft_set_variant(256, args.zy_variant, 3)
    if args.zx_variant >= 0:
        fft_set_variant(256, args.zx_variant, 4)
        fft_set_variant(256, args.zx_variant, 5)
    pos = torch.from_numpy(S.poisson_uniform(200_000, L3, seed=8)).cuda()
    ctx = Context(L3, 256, 4)
    ctx.window_shells(np.linspace(10.0, 170.0, 17), l_max=1)
    ctx.assign(pos)
    z = ctx.zeta_multipoles()
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"profile_case": "zeta 256^3, 16 shells, l_max 1", "zeta00": float(z[0, 0, 0])}))


def run_profile_ddd(args):
    """Small case for ncu captures of the connection-coefficient monopole: 256^3 field of 200k
    Poisson points, p = 4, 16 shells (about 3 GB on the device), two calls."""
    import torch
    from paper_2607_23494_b300 import Context
    from synthetic import catalogues as S
    pos = torch.from_numpy(S.poisson_uniform(200_000, L3, seed=9)).cuda()
    ctx = Context(L3, 256, 4)
    ctx.window_shells(np.linspace(10.0, 170.0, 17), l_max=0)
    ctx.assign(pos)
    for _ in range(2):
        d = ctx.ddd_monopole()
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"profile_case": "ddd monopole 256^3, 16 shells, p 4", "ddd00": float(d[0, 0])}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hermes", choices=["hermes", "reference"])
    ap.add_argument("--no-zeta", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain torch/cuFFT comparison arm")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-catalogue measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=60, help="requests in the open-loop serving trace")
    ap.add_argument("--serve-saturated", type=int, default=80,
                    help="requests in the saturated mixed serving trace (twice as many in the small-grid one)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true", help="skip the all-cores oracle timing")
    ap.add_argument("--minimal", action="store_true",
                    help="the timed step and its end-to-end form only (implies --no-plain --no-batch --no-serve "
                         "--no-zeta --no-cpu-baseline); for launch-list captures")
    ap.add_argument("--profile-case", action="store_true", help="small workload for ncu captures")
    ap.add_argument("--profile-zeta", action="store_true", help="small zeta workload for ncu captures")
    ap.add_argument("--profile-ddd", action="store_true", help="small monopole workload for ncu captures")
    ap.add_argument("--y-variant", type=int, default=0, help="inverse y-pass variant of --profile-case")
    ap.add_argument("--x-variant", type=int, default=0, help="window-pass variant of --profile-case")
    ap.add_argument("--z-variant", type=int, default=0, help="contraction-pass variant of --profile-case")
    ap.add_argument("--zy-variant", type=int, default=-1, help="zeta y-pass variant of --profile-zeta")
    ap.add_argument("--zx-variant", type=int, default=-1, help="zeta x-pass variant of --profile-zeta")
    ap.add_argument("--fft-variants", default="",
                    help="Y,X,Z: fix the 512^3 inverse y, window and contraction pass variants instead of tuning "
                         "(ncu distorts the tuner's trial timings, so launch lists run with the plain run's choice)")
    args = ap.parse_args()
    if args.minimal:
        args.no_plain = args.no_batch = args.no_serve = args.no_zeta = args.no_cpu_baseline = True
    if args.fft_variants:
        from paper_2607_23494_b300 import fft_set_variant
        for pass_, v in zip((0, 1, 2), (int(x) for x in args.fft_variants.split(","))):
            fft_set_variant(N2, v, pass_)
    if args.profile_case:
        run_profile_case(args)
        return 0
    if args.profile_zeta:
        run_profile_zeta(args)
        return 0
    if args.profile_ddd:
        run_profile_ddd(args)
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)))
        return 0
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out, pos = run_hermes(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            v, dt = oracle_sample(pos)
            out["cpu_baseline"] = {"value": round(v, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "cpu_model": cpu_model(),
                                   "sample": f"512^3 grid, first 500k of the 1e7 points, one l=0 shell window "
                                             f"(scatter, FFT, window, Parseval sum, self-pair term): {dt:.1f} s, "
                                             f"numpy single thread; per-catalogue work not amortised"}
            if not args.no_cpu_all_cores:
                va, wall, k, cores = oracle_sample_all_cores(pos)
                out["cpu_baseline"]["all_cores"] = {
                    "value": round(va, 1), "unit": UNIT, "processes": k, "cores_available": cores,
                    "sample": f"the same sample in {k} spawned processes (one shell each), {wall:.1f} s wall"}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
