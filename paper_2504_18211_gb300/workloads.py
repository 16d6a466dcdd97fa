"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Pure input generation: numpy PCG64 streams, no allocator arithmetic.  Seeds
default to 0x0A110C00 + workload index.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x0A110C00


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def small_sizes(threads: int = 40 * 256, size: int = 16) -> np.ndarray:
    """Plain-method small run: every thread asks for the same size."""
    return np.full(threads, size, dtype=np.uint32)


def sweep_sizes(threads: int = 1 << 20, seed: int = SEED_BASE + 1, kmin: int = 4,
                kmax: int = 13) -> np.ndarray:
    """Size sweep: each thread asks for 2**k bytes, k uniform in [kmin, kmax]."""
    k = rng(seed).integers(kmin, kmax + 1, size=threads)
    return (np.uint32(1) << k.astype(np.uint32)).astype(np.uint32)


def uniform_sizes(threads: int, lo: int = 4, hi: int = 8192, seed: int = SEED_BASE + 3) -> np.ndarray:
    """Sizes uniform over the integers [lo, hi]."""
    return rng(seed).integers(lo, hi + 1, size=threads).astype(np.uint32)


def single_size(threads: int, size: int) -> np.ndarray:
    return np.full(threads, size, dtype=np.uint32)


def batching_workload(n_batches: int = 256, lo: float = 10.0, hi: float = 20.0, smin: int = 4, smax: int = 8192,
                      seed: int = SEED_BASE + 3):
    """Request batches: threads per batch round(2^u), u uniform in [lo, hi];
    sizes uniform over the integers [smin, smax].  Returns (sizes, offs)
    with batch b = sizes[offs[b]:offs[b+1]]."""
    r = rng(seed)
    threads = np.round(2.0 ** r.uniform(lo, hi, n_batches)).astype(np.int64)
    sizes = r.integers(smin, smax + 1, size=int(threads.sum())).astype(np.uint32)
    offs = np.concatenate([[0], np.cumsum(threads)]).astype(np.uint64)
    return sizes, offs


def serving_workload(steps: int = 2000, rate: float = 2000.0, dt: float = 0.01, median_bytes: int = 4 << 20,
                     sigma: float = 1.0, block_bytes: int = 16384, max_blocks: int = 4096,
                     seed: int = SEED_BASE + 4):
    """Sessions arriving as a Poisson process (rate per second) on a virtual
    clock of `steps` steps of dt seconds; each session's total size is
    lognormal (median, sigma), in blocks of block_bytes, at most max_blocks.
    Returns (arrive_step, blocks), sessions in arrival order."""
    r = rng(seed)
    horizon = steps * dt
    n = int(r.poisson(rate * horizon))
    t = np.sort(r.uniform(0.0, horizon, n))
    arrive = np.minimum(np.floor(t / dt), steps - 1).astype(np.uint32)
    size = r.lognormal(np.log(median_bytes), sigma, n)
    blocks = np.clip(np.ceil(size / block_bytes), 1, max_blocks).astype(np.uint32)
    return arrive, blocks


def graph_workload(n_vertices: int = 1 << 20, n_edges: int = 1 << 24, alpha: float = 2.1,
                   seed: int = SEED_BASE + 2):
    """Directed edges whose endpoints follow a power law over a seeded
    permutation of the vertices.  alpha is read as the degree-distribution
    exponent, so the rank-frequency exponent is s = 1 / (alpha - 1).
    Returns (src, dst) uint32 arrays."""
    r = rng(seed)
    s = 1.0 / (alpha - 1.0)
    w = np.arange(1, n_vertices + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    perm = r.permutation(n_vertices).astype(np.uint32)
    src = perm[np.minimum(np.searchsorted(cdf, r.random(n_edges), side="right"), n_vertices - 1)]
    dst = perm[np.minimum(np.searchsorted(cdf, r.random(n_edges), side="right"), n_vertices - 1)]
    return src.astype(np.uint32), dst.astype(np.uint32)


def mixed_sizes(threads: int, seed: int, chunk_bytes: int = 8192) -> np.ndarray:
    """Requests of every kind a kernel may make: powers of two 16 B .. one
    chunk (most), any byte count up to one chunk (30 %: sizes that are not a
    multiple of 4 included), runs of chunks up to 64 KiB (2 %), 0 bytes (2 %)
    and above 1 MiB (2 %, answered with null)."""
    r = rng(seed)
    kmax = int(chunk_bytes).bit_length() - 1
    s = (np.int64(1) << r.integers(4, kmax + 1, size=threads)).astype(np.int64)
    pick = r.random(threads)
    odd = pick < 0.30
    s[odd] = r.integers(1, chunk_bytes + 1, size=int(odd.sum()))
    run = (pick >= 0.30) & (pick < 0.32)
    s[run] = r.integers(chunk_bytes + 1, 65536 + 1, size=int(run.sum()))
    s[(pick >= 0.32) & (pick < 0.34)] = 0
    s[(pick >= 0.34) & (pick < 0.36)] = 2 << 20
    return s.astype(np.uint32)
