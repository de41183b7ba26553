"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers (numpy's PCG64, seeded); it holds none
of the sort's arithmetic, and it is the one piece of Python shared by the CUDA
path's tests and the CPU oracle.  All keys are uint64; payloads are uint32
original indices.

The paper evaluates 64-bit integers from a seeded Mersenne twister in five
families (uniform, normal, power-law skewed, nearly sorted, high duplicate,
section "Experimental Results"); it states no parameters.  The families and
their parameters below are the stand-ins, one per named workload.
"""
from __future__ import annotations

import numpy as np

U64_MAX_F = 18446744073709549568.0  # largest double below 2^64


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _raw_u64(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.bit_generator.random_raw(n).astype(np.uint64, copy=False)


def _f64_to_u64(x: np.ndarray) -> np.ndarray:
    x = np.floor(x)
    np.clip(x, 0.0, U64_MAX_F, out=x)
    return x.astype(np.uint64)


def index_payload(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.uint32)


def uniform(n: int, seed: int) -> np.ndarray:
    """Uniform over [0, 2^64)."""
    return _raw_u64(_rng(seed), n)


def normal(n: int, seed: int, mean: float = 2.0 ** 62, sd: float = 2.0 ** 58) -> np.ndarray:
    """floor(N(mean, sd)) clipped to the uint64 range."""
    return _f64_to_u64(_rng(seed).normal(mean, sd, n))


def zipf(n: int, seed: int, s: float = 1.1, distinct: int = 10_000) -> np.ndarray:
    """Duplicate heavy: Zipf(s) ranks over `distinct` values; the value of each
    rank is a uniform uint64 drawn in rank order."""
    rng = _rng(seed)
    values = _raw_u64(rng, distinct)
    p = np.arange(1, distinct + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    ranks = np.searchsorted(cdf, rng.random(n), side="right")
    np.minimum(ranks, distinct - 1, out=ranks)
    return values[ranks]


def nearly_sorted(n: int, seed: int, swap_frac: float = 0.05) -> np.ndarray:
    """Ascending uniform keys, then floor(swap_frac * n) swaps of random,
    pairwise disjoint position pairs."""
    rng = _rng(seed)
    keys = np.sort(_raw_u64(rng, n))
    m = min(int(swap_frac * n), n // 2)
    if m:
        idx = rng.choice(n, size=2 * m, replace=False)
        a, b = idx[:m], idx[m:]
        keys[a], keys[b] = keys[b].copy(), keys[a].copy()
    return keys


def descending(n: int, seed: int = 0) -> np.ndarray:
    """Strictly descending: key_i = (n - i) * floor((2^64 - 1) / n)."""
    if n == 0:
        return np.zeros(0, dtype=np.uint64)
    step = np.uint64((2 ** 64 - 1) // n)
    return (np.arange(n, 0, -1, dtype=np.uint64) * step).astype(np.uint64)


def lognormal(n: int, seed: int, mu: float = 30.0, sigma: float = 2.0) -> np.ndarray:
    """floor(exp(N(mu, sigma))) clipped to 2^64 - 1."""
    x = _rng(seed).normal(mu, sigma, n)
    np.exp(x, out=x)
    return _f64_to_u64(x)


def gaussian_mixture(n: int, seed: int, comps: int = 8, lo: float = 2.0 ** 60,
                     hi: float = 2.0 ** 63, sd: float = 2.0 ** 55) -> np.ndarray:
    """Equal-weight mixture of `comps` normals, means evenly spaced over
    [lo, hi], common sd; floor and clip."""
    rng = _rng(seed)
    means = np.linspace(lo, hi, comps)
    c = rng.integers(0, comps, n)
    x = rng.normal(0.0, sd, n)
    x += means[c]
    return _f64_to_u64(x)


def dense_interval_u64(n: int, seed: int, p: float = 0.9, base: int = 2 ** 40,
                       width: int = 2 ** 20) -> np.ndarray:
    """Adversarial skew: with probability p uniform in [base, base+width),
    otherwise uniform over [0, 2^64)."""
    rng = _rng(seed)
    wide = _raw_u64(rng, n)
    dense = np.uint64(base) + (_raw_u64(rng, n) % np.uint64(width))
    pick = rng.random(n) < p
    return np.where(pick, dense, wide)


def dense_interval_i64(n: int, seed: int, p: float = 0.9, half: int = 2 ** 19) -> np.ndarray:
    """The same law recentred on 0 for int64: dense in [-half, half), else
    uniform int64.  Returns int64."""
    rng = _rng(seed)
    wide = _raw_u64(rng, n).view(np.int64)
    dense = (_raw_u64(rng, n) % np.uint64(2 * half)).astype(np.int64) - half
    pick = rng.random(n) < p
    return np.where(pick, dense, wide)


def normal_f64_specials(n: int, seed: int, p_inf: float = 0.005, p_zero: float = 0.01) -> np.ndarray:
    """float64 N(0,1) with p_inf each of +inf and -inf and p_zero zeros split
    evenly between -0.0 and +0.0.  Returns float64."""
    rng = _rng(seed)
    x = rng.standard_normal(n)
    u = rng.random(n)
    x[u < p_inf] = np.inf
    x[(u >= p_inf) & (u < 2 * p_inf)] = -np.inf
    z = (u >= 2 * p_inf) & (u < 2 * p_inf + p_zero)
    zsign = rng.random(n) < 0.5
    x[z & zsign] = -0.0
    x[z & ~zsign] = 0.0
    return x


FAMILIES = {
    "uniform": uniform,
    "normal": normal,
    "zipf": zipf,
    "nearly_sorted": nearly_sorted,
    "descending": descending,
}


def segment_sizes(nseg: int, seed: int, lo: int = 32, hi: int = 2 ** 20) -> np.ndarray:
    """Log-uniform sizes floor(exp(U(ln lo, ln hi)))."""
    rng = _rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), nseg))).astype(np.int64)


def segmented(nseg: int, seed: int, lo: int = 32, hi: int = 2 ** 20):
    """Batch of `nseg` arrays with log-uniform sizes, each drawn from one of
    the five families chosen uniformly.  Returns (keys, vals, offsets, names):
    vals are within-segment indices, offsets has nseg + 1 uint64 entries."""
    sizes = segment_sizes(nseg, seed, lo, hi)
    rng = _rng(seed + 1)
    names = list(FAMILIES)
    fam = rng.integers(0, len(names), nseg)
    off = np.zeros(nseg + 1, dtype=np.uint64)
    off[1:] = np.cumsum(sizes).astype(np.uint64)
    total = int(off[-1])
    keys = np.empty(total, dtype=np.uint64)
    vals = np.empty(total, dtype=np.uint32)
    for i in range(nseg):
        a, b = int(off[i]), int(off[i + 1])
        keys[a:b] = FAMILIES[names[fam[i]]](b - a, seed * 1_000_003 + i)
        vals[a:b] = np.arange(b - a, dtype=np.uint32)
    return keys, vals, off, [names[f] for f in fam]


def _fill_segments(args):
    """Worker of segmented_parallel: draws segments [i0, i1) into the shared
    key and payload buffers (same per-segment seeds as segmented)."""
    from multiprocessing import shared_memory

    shm_name, total, off, fam, seed, i0, i1 = args
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        keys = np.ndarray((total,), dtype=np.uint64, buffer=shm.buf)
        vals = np.ndarray((total,), dtype=np.uint32, buffer=shm.buf, offset=8 * total)
        names = list(FAMILIES)
        for i in range(i0, i1):
            a, b = int(off[i]), int(off[i + 1])
            keys[a:b] = FAMILIES[names[fam[i]]](b - a, seed * 1_000_003 + i)
            vals[a:b] = np.arange(b - a, dtype=np.uint32)
        del keys, vals
    finally:
        shm.close()
    return i1 - i0


def segmented_parallel(nseg: int, seed: int, lo: int = 32, hi: int = 2 ** 20, workers: int = 0):
    """segmented(nseg, seed, lo, hi), bit for bit, drawn by a pool of worker
    processes (started with spawn) into shared memory; for batches of
    billions of pairs.  Falls back to segmented() if shared memory cannot be
    had."""
    import multiprocessing as mp
    import os
    from multiprocessing import shared_memory

    sizes = segment_sizes(nseg, seed, lo, hi)
    rng = _rng(seed + 1)
    names = list(FAMILIES)
    fam = rng.integers(0, len(names), nseg)
    off = np.zeros(nseg + 1, dtype=np.uint64)
    off[1:] = np.cumsum(sizes).astype(np.uint64)
    total = int(off[-1])
    workers = workers or min(32, os.cpu_count() or 1)
    try:
        shm = shared_memory.SharedMemory(create=True, size=max(12 * total, 1))
    except OSError:
        return segmented(nseg, seed, lo, hi)
    try:
        # share the work out by pairs, not by segments (sizes span 2^15)
        bounds = [0]
        target = total / (4 * workers)
        acc = 0
        for i in range(nseg):
            acc += int(sizes[i])
            if acc >= target:
                bounds.append(i + 1)
                acc = 0
        if bounds[-1] != nseg:
            bounds.append(nseg)
        jobs = [(shm.name, total, off, fam, seed, bounds[j], bounds[j + 1]) for j in range(len(bounds) - 1)]
        with mp.get_context("spawn").Pool(workers) as pool:
            done = sum(pool.map(_fill_segments, jobs))
        assert done == nseg
        keys = np.ndarray((total,), dtype=np.uint64, buffer=shm.buf).copy()
        vals = np.ndarray((total,), dtype=np.uint32, buffer=shm.buf, offset=8 * total).copy()
    finally:
        shm.close()
        shm.unlink()
    return keys, vals, off, [names[f] for f in fam]
