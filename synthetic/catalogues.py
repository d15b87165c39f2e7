"""Seeded synthetic point catalogues shaped like the halo catalogues of the paper.

The paper measures on Quijote and Kun halo catalogues (Sec. 2 data description,
Sec. 4.5 benchmarks), which are not available here.  These generators stand in
for them.  This module holds no arithmetic of the estimator itself: it only
draws positions, weights and marks, which both the CUDA path and the oracle
then take as plain inputs.

Every generator is deterministic in its ``seed`` and returns positions as
float32 arrays of shape (n, 3) inside [0, L) and weights as float32 arrays.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "poisson_uniform",
    "soneira_peebles",
    "mixed_poisson_sp",
    "gaussian_field",
    "lognormal_catalogue",
    "lognormal_masses",
    "batched_catalogue_sizes",
    "clamp_into_box",
]


def clamp_into_box(pos: np.ndarray, L: float) -> np.ndarray:
    """Wrap float64 positions periodically into [0, L) and cast to float32.

    A float64 value just below L can round up to exactly L in float32; such
    values are replaced by the largest float32 below L so every position is
    strictly inside the box.
    """
    p = np.mod(np.asarray(pos, dtype=np.float64), L)
    p32 = p.astype(np.float32)
    top = np.nextafter(np.float32(L), np.float32(0))
    p32 = np.where(p32 >= np.float32(L), top, p32)
    p32 = np.where(p32 < 0, np.float32(0), p32)
    return np.ascontiguousarray(p32, dtype=np.float32)


def poisson_uniform(n: int, L: float, seed: int) -> np.ndarray:
    """n points uniform in the periodic box (a homogeneous Poisson sample)."""
    rng = np.random.default_rng(seed)
    return clamp_into_box(rng.random((n, 3)) * L, L)


def soneira_peebles(n: int, L: float, seed: int, eta: int = 2, lam: float = 1.9,
                    levels: int = 10, radius: float = 25.0) -> np.ndarray:
    """Soneira-Peebles hierarchical clusters, truncated to n points.

    Each cluster starts at a uniform centre.  At every level each current point
    spawns ``eta`` children placed uniformly inside a sphere of radius
    ``radius / lam**level`` around it; after ``levels`` levels a cluster holds
    eta**levels points.  Clusters are drawn until n points exist, then the
    set is truncated and wrapped periodically.
    """
    rng = np.random.default_rng(seed)
    per_cluster = eta ** levels
    n_clusters = max(1, -(-n // per_cluster))
    out = []
    for _ in range(n_clusters):
        pts = rng.random((1, 3)) * L
        r = radius
        for _lvl in range(levels):
            # uniform points in a ball: direction from a normal draw, radius ~ u^(1/3)
            m = pts.shape[0] * eta
            d = rng.normal(size=(m, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            rr = r * rng.random(m) ** (1.0 / 3.0)
            pts = np.repeat(pts, eta, axis=0) + d * rr[:, None]
            r = r / lam
        out.append(pts)
    allp = np.concatenate(out, axis=0)[:n]
    return clamp_into_box(allp, L)


def mixed_poisson_sp(n: int, L: float, seed: int) -> np.ndarray:
    """Half uniform Poisson, half Soneira-Peebles clustered points (shuffled)."""
    n_u = n // 2
    a = poisson_uniform(n_u, L, seed)
    b = soneira_peebles(n - n_u, L, seed + 1)
    pos = np.concatenate([a, b], axis=0)
    rng = np.random.default_rng(seed + 2)
    return np.ascontiguousarray(pos[rng.permutation(n)])


def gaussian_field(n_grid: int, L: float, seed: int, slope: float = -1.5,
                   k_cut: float = 0.5, sigma: float = 1.0) -> np.ndarray:
    """A periodic Gaussian random field with P(k) ~ k^slope exp(-(k/k_cut)^2).

    White noise is filtered by sqrt(P) in Fourier space and the result is
    rescaled so that its sample variance equals sigma^2.  Returns float64
    (n_grid, n_grid, n_grid).
    """
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n_grid, n_grid, n_grid))
    try:
        import scipy.fft as sfft
        wk = sfft.rfftn(white, workers=-1)
    except Exception:  # pragma: no cover - scipy is present in this image
        wk = np.fft.rfftn(white)
    del white
    kf = 2.0 * np.pi / L
    kx = np.fft.fftfreq(n_grid, d=1.0 / n_grid) * kf
    kz = np.fft.rfftfreq(n_grid, d=1.0 / n_grid) * kf
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    k = np.sqrt(k2)
    with np.errstate(divide="ignore"):
        amp = np.where(k > 0, k ** (slope / 2.0) * np.exp(-0.5 * (k / k_cut) ** 2), 0.0)
    wk *= amp
    del amp, k, k2
    try:
        g = sfft.irfftn(wk, s=(n_grid,) * 3, workers=-1)
    except Exception:  # pragma: no cover
        g = np.fft.irfftn(wk, s=(n_grid,) * 3)
    g -= g.mean()
    g *= sigma / g.std()
    return g


def lognormal_catalogue(n_mean: int, L: float, seed: int, n_grid: int = 128,
                        sigma_ln: float = 1.0, slope: float = -1.5,
                        k_cut: float = 0.5) -> np.ndarray:
    """Points Poisson-sampled from a lognormal density field.

    G is a Gaussian field with var(G) = sigma_ln^2; the lognormal contrast is
    delta = exp(G - sigma_ln^2/2) - 1.  Each generation cell receives a
    Poisson count with mean n_mean * (1 + delta) / n_grid^3 (renormalised so
    that the expected total is n_mean); points are uniform inside their cell.
    """
    g = gaussian_field(n_grid, L, seed, slope=slope, k_cut=k_cut, sigma=sigma_ln)
    rho = np.exp(g - 0.5 * sigma_ln ** 2)
    del g
    rho *= n_mean / rho.sum()
    rng = np.random.default_rng(seed + 7919)
    counts = rng.poisson(rho.ravel())
    del rho
    n = int(counts.sum())
    cells = np.repeat(np.arange(counts.size, dtype=np.int64), counts)
    del counts
    h = L / n_grid
    ix = cells // (n_grid * n_grid)
    iy = (cells // n_grid) % n_grid
    iz = cells % n_grid
    del cells
    pos = np.empty((n, 3), dtype=np.float64)
    u = rng.random((n, 3))
    pos[:, 0] = (ix + u[:, 0]) * h
    pos[:, 1] = (iy + u[:, 1]) * h
    pos[:, 2] = (iz + u[:, 2]) * h
    del u, ix, iy, iz
    perm = rng.permutation(n)
    return clamp_into_box(pos[perm], L)


def lognormal_masses(n: int, seed: int, mu: float = 12.0, sigma_dex: float = 0.5) -> np.ndarray:
    """Halo-like masses with log10 M ~ Normal(mu, sigma_dex), divided by their mean.

    Dividing by the mean (in float64, before the float32 cast) keeps the
    weights near unity; an overall rescaling of a mark cancels in the marked
    correlation function anyway.
    """
    rng = np.random.default_rng(seed)
    m = 10.0 ** rng.normal(mu, sigma_dex, size=n)
    m /= m.mean()
    return m.astype(np.float32)


def batched_catalogue_sizes(n_cat: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Catalogue sizes drawn log-uniformly in [lo, hi] (int64)."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_cat)).astype(np.int64)
