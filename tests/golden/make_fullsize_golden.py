"""Writes the stored FP64 oracle values that the full-size parity tests and the
benchmark's error report compare against.  It calls only ``oracle/`` (and
``synthetic/`` for the seeded inputs); nothing here comes from the CUDA path.

  python tests/golden/make_fullsize_golden.py [xi64] [xi512] [zeta128]

xi64    -- the 20,000-point catalogue (half uniform Poisson, half Soneira-Peebles, seed
           2024) in L = 250 Mpc/h on the 64^3 grid with the cubic B-spline: xi on the 20
           shells [5, 105), unit weights, in full.  Seconds.
xi512   -- the 1e7-point lognormal catalogue (L = 1000 Mpc/h, seed 1234, log-normal
           masses seed 1235) on the 512^3 grid with the cubic B-spline: xi_l for
           l = 0, 2, 4 on a sample of the 40 shells [2, 202), unit weights and mass
           marks, by Parseval on the rfft half spectrum (Eq. pair-counting-kspace)
           minus the exact self-pair term.  About 10 minutes on one core.
zeta128 -- the 2e6-point lognormal catalogue (L = 500 Mpc/h, seed 4321) regridded on
           128^3: zeta_l for l <= 6 on the 16 shells [10, 170), every m in [-l, l]
           built as an explicit inverse transform (Eq. 2-fold-translation).  About
           15 minutes on one core.

Each file records a SHA-256 of the catalogue bytes, so a test can tell that it
regenerated exactly the same inputs.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import hermes_oracle as O  # noqa: E402
from synthetic import catalogues as S  # noqa: E402

XI64_FILE = os.path.join(HERE, "xi_mixed_2e4_64.json")
XI_FILE = os.path.join(HERE, "xi_lognormal_1e7_512_sample.json")
ZETA_FILE = os.path.join(HERE, "zeta_lognormal_2e6_128_lmax6.json")

XI64 = dict(n=20_000, L=250.0, seed=2024, N=64, p=4, edges=np.linspace(5.0, 105.0, 21).tolist())
XI = dict(n_mean=10_000_000, L=1000.0, seed=1234, mass_seed=1235, n_grid=512, N=512, p=4,
          edges=np.linspace(2.0, 202.0, 41).tolist(), ells=[0, 2, 4], bins=[0, 1, 5, 14, 27, 39])
ZETA = dict(n_mean=2_000_000, L=500.0, seed=4321, n_grid=512, N=128, p=4,
            edges=np.linspace(10.0, 170.0, 17).tolist(), l_max=6)


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def make_xi64():
    c = XI64
    pos = S.mixed_poisson_sp(c["n"], c["L"], seed=c["seed"])
    res = O.xi_multipoles(pos, None, c["N"], c["L"], c["p"], c["edges"], ells=(0,))
    out = {"what": "FP64 oracle xi (Parseval on the full spectrum minus the exact self-pair term) of the "
                   "20,000-point Poisson + Soneira-Peebles catalogue, 64^3, p = 4, 20 shells [5, 105)",
           "generated_by": "tests/golden/make_fullsize_golden.py xi64",
           "config": c, "n_points": int(pos.shape[0]), "pos_sha256": digest(pos), "xi": res["xi"][0].tolist()}
    with open(XI64_FILE, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {XI64_FILE}", flush=True)


def make_xi512():
    c = XI
    t0 = time.time()
    pos = S.lognormal_catalogue(c["n_mean"], c["L"], seed=c["seed"], n_grid=c["n_grid"])
    mass = S.lognormal_masses(pos.shape[0], seed=c["mass_seed"])
    N, L, p, edges = c["N"], c["L"], c["p"], c["edges"]
    print(f"catalogue {pos.shape[0]} points in {time.time() - t0:.1f} s", flush=True)
    fields = {}
    for name, w in (("unit", None), ("marked", mass)):
        t = time.time()
        eps, sw, _ = O.assign(pos, w, N, L, p)
        delta = O.delta_from_eps(eps, sw)
        del eps
        dh = O.forward_half(delta)
        del delta
        fields[name] = (dh, O.self_pair_table(pos, w, N, L, p), sw)
        print(f"field {name}: {time.time() - t:.1f} s", flush=True)
    xi = {name: [[None] * len(c["bins"]) for _ in c["ells"]] for name in fields}
    for a, ell in enumerate(c["ells"]):
        for j, b in enumerate(c["bins"]):
            t = time.time()
            K = O.window_xi(N, L, p, edges[b], edges[b + 1], ell, half=True)
            for name, (dh, Sp, sw) in fields.items():
                xi[name][a][j] = O.xi_parseval_half(dh, K, N) - O.shot_noise_half(Sp, K, N, sw)
            del K
            print(f"l={ell} bin {b}: {time.time() - t:.1f} s", flush=True)
    out = {"what": "FP64 oracle xi_l (Parseval on the half spectrum minus the exact self-pair term) of the "
                   "1e7-point lognormal catalogue, unit weights and log-normal mass marks, 512^3, p = 4",
           "generated_by": "tests/golden/make_fullsize_golden.py xi512",
           "config": c, "n_points": int(pos.shape[0]), "pos_sha256": digest(pos), "mass_sha256": digest(mass),
           "xi": xi}
    with open(XI_FILE, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {XI_FILE} in {time.time() - t0:.1f} s", flush=True)


def make_zeta128():
    c = ZETA
    t0 = time.time()
    pos = S.lognormal_catalogue(c["n_mean"], c["L"], seed=c["seed"], n_grid=c["n_grid"])
    N, L, p = c["N"], c["L"], c["p"]
    eps, sw, _ = O.assign(pos, None, N, L, p)
    delta = O.delta_from_eps(eps, sw)
    del eps
    zeta, imag = O.zeta_multipoles(delta, N, L, p, c["edges"], c["l_max"])
    out = {"what": "FP64 oracle zeta_l (explicit inverse transforms of every m in [-l, l], cell sums) of the "
                   "2e6-point lognormal catalogue regridded on 128^3, p = 4, 16 shells [10, 170), l_max = 6",
           "generated_by": "tests/golden/make_fullsize_golden.py zeta128",
           "config": c, "n_points": int(pos.shape[0]), "pos_sha256": digest(pos), "imag_max": imag,
           "zeta": zeta.tolist()}
    with open(ZETA_FILE, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {ZETA_FILE} in {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["xi64", "xi512", "zeta128"]
    if "xi64" in which:
        make_xi64()
    if "xi512" in which:
        make_xi512()
    if "zeta128" in which:
        make_zeta128()
