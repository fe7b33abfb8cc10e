"""Seeded synthetic inputs shaped like the paper's workloads (§5: synthetic
uniform / correlated / anticorrelated data; HOU and RES stand-ins).

This module holds no skyline arithmetic: it only draws points.  Both the CUDA
path's tests and benchmark and the oracle's tests take their inputs from here.
All generators use numpy's PCG64 stream from ``seed`` and return C-contiguous
FP32 arrays of shape [N, d].

Recipes (the paper leaves its generators unspecified, §5):

* ``anticorrelated``: per point a plane offset s ~ N(0.5, 0.05) clipped to
  [0, 1]; coordinates uniform on the simplex {y >= 0, sum y = d*s} (normalised
  exponentials); points leaving [0, 1]^d are rejected and redrawn.
* ``independent``: U[0, 1]^d, optionally quantised to multiples of 1/256.
* ``correlated``: t ~ U(0, 1), x_j = clip(t + N(0, 0.05), 0, 1), optionally
  quantised to multiples of 1/256.
* ``skewed``: log-normal attributes (mu = 0, sigma = 1) from an equicorrelated
  Gaussian copula (correlation max(-0.313, -0.95/(d-1)), the most negative
  feasible value near the Spearman -0.3 target); 5 % of the cells set to their
  column maximum; 10 % of the rows replaced by copies of other rows.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def quantise(x: np.ndarray, levels: int = 256) -> np.ndarray:
    """Round to the nearest multiple of 1/levels (ties to even); exact in FP32."""
    return (np.rint(x * levels) / levels).astype(np.float32)


def anticorrelated(n: int, d: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    out = np.empty((n, d), dtype=np.float32)
    got = 0
    while got < n:
        need = n - got
        batch = max(1024, int(need * 4.0) + 64)
        s = np.clip(rng.normal(0.5, 0.05, size=batch), 0.0, 1.0)
        e = rng.exponential(1.0, size=(batch, d))
        tot = e.sum(axis=1, keepdims=True)
        tot[tot == 0] = 1.0
        y = e / tot * (d * s)[:, None]
        ok = np.all(y <= 1.0, axis=1)
        y = y[ok][:need]
        out[got:got + y.shape[0]] = y.astype(np.float32)
        got += y.shape[0]
    return out


def anticorrelated_blocks(n: int, d: int, seed: int, block: int = 10_000_000) -> np.ndarray:
    """``anticorrelated`` drawn in independent blocks of ``block`` points
    (block i from seed + i), so that very large inputs need memory for one
    block's draws only; for n <= block it equals anticorrelated(n, d, seed)."""
    out = np.empty((n, d), dtype=np.float32)
    for i, lo in enumerate(range(0, n, block)):
        hi = min(n, lo + block)
        out[lo:hi] = anticorrelated(hi - lo, d, seed + i)
    return out


def independent(n: int, d: int, seed: int, quantised: bool = True) -> np.ndarray:
    rng = _rng(seed)
    x = rng.random(size=(n, d))
    return quantise(x) if quantised else x.astype(np.float32)


def correlated(n: int, d: int, seed: int, quantised: bool = True, sigma: float = 0.05) -> np.ndarray:
    rng = _rng(seed)
    t = rng.random(size=(n, 1))
    x = np.clip(t + rng.normal(0.0, sigma, size=(n, d)), 0.0, 1.0)
    return quantise(x) if quantised else x.astype(np.float32)


def skewed_correlation(d: int) -> float:
    """Equicorrelation used by ``skewed``: the Gaussian value for Spearman -0.3
    (2 sin(pi * rho / 6) = -0.313), limited to what keeps the matrix positive
    definite for d attributes."""
    target = 2.0 * np.sin(np.pi * -0.3 / 6.0)
    if d <= 1:
        return 0.0
    return float(max(target, -0.95 / (d - 1)))


def skewed(n: int, d: int, seed: int, dup_frac: float = 0.10, max_frac: float = 0.05) -> np.ndarray:
    rng = _rng(seed)
    r = skewed_correlation(d)
    cov = np.full((d, d), r)
    np.fill_diagonal(cov, 1.0)
    L = np.linalg.cholesky(cov)
    z = rng.standard_normal(size=(n, d)) @ L.T
    x = np.exp(z).astype(np.float32)
    if n:
        colmax = x.max(axis=0)
        cells = rng.random(size=(n, d)) < max_frac
        x = np.where(cells, colmax[None, :], x).astype(np.float32)
        ndup = int(round(dup_frac * n))
        if ndup and n > ndup:
            perm = rng.permutation(n)
            dst, keep = perm[:ndup], perm[ndup:]
            src = keep[rng.integers(0, keep.shape[0], size=ndup)]
            x[dst] = x[src]
    return np.ascontiguousarray(x, dtype=np.float32)


GENERATORS = {
    "anticorrelated": anticorrelated,
    "independent": independent,
    "correlated": correlated,
    "skewed": skewed,
}


def make(kind: str, n: int, d: int, seed: int) -> np.ndarray:
    return GENERATORS[kind](n, d, seed)


def serving_trace(num_queries: int, seed: int, n_lo: float = 1e3, n_hi: float = 1e6,
                  d_lo: int = 3, d_hi: int = 8):
    """Query shapes of the serving workload: per query (kind, N, d, seed) with
    N log-uniform in [n_lo, n_hi] and d uniform in {d_lo..d_hi}; kind is
    anticorrelated or independent with probability 1/2 each."""
    rng = _rng(seed)
    out = []
    for q in range(num_queries):
        n = int(10 ** rng.uniform(np.log10(n_lo), np.log10(n_hi)))
        d = int(rng.integers(d_lo, d_hi + 1))
        kind = "anticorrelated" if rng.random() < 0.5 else "independent"
        out.append((kind, n, d, seed * 100003 + q))
    return out


def poisson_arrivals(num: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=num))
