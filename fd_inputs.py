"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds none of the FD method's arithmetic: it only draws blocks of
vectors and random sparse symmetric matrices (NumPy's PCG64, seeded), which
both the CUDA library and the CPU oracle then receive as the same inputs.
"""
import numpy as np


def random_block(D, m, seed, dtype=np.float64):
    """D x m row-major block with standard normal entries."""
    return np.random.default_rng(seed).standard_normal((D, m)).astype(dtype)


def random_symmetric_csr(D, mean_offdiag, seed, max_row=None, scale=1.0):
    """Random symmetric CSR with ragged rows (int64 rowptr, int32 col, f64 val).

    The diagonal is always present; off-diagonal pairs (i, j), i != j, are drawn
    uniformly, so row lengths follow a Poisson-like spread.  ``max_row`` caps a
    few rows at a long length to make the ragged tail explicit.
    """
    rng = np.random.default_rng(seed)
    npairs = int(D * mean_offdiag / 2)
    i = rng.integers(0, D, npairs)
    j = rng.integers(0, D, npairs)
    keep = i != j
    i, j = i[keep], j[keep]
    if max_row:
        hubs = rng.choice(D, size=max(1, D // 1000), replace=False)
        hi = np.repeat(hubs, max_row)
        hj = rng.integers(0, D, len(hi))
        k2 = hi != hj
        i, j = np.concatenate([i, hi[k2]]), np.concatenate([j, hj[k2]])
    v = rng.uniform(-scale, scale, len(i))
    rows = np.concatenate([i, j, np.arange(D)])
    cols = np.concatenate([j, i, np.arange(D)])
    vals = np.concatenate([v, v, rng.uniform(-scale, scale, D)])
    key = rows * D + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uniq, first = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, first)
    rows, cols = uniq // D, uniq % D
    counts = np.bincount(rows, minlength=D)
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, cols.astype(np.int32), summed.astype(np.float64)


def _splitmix_uniform(seed, stream, i):
    """u = (mix64(key + (i+1) gamma) >> 11) 2^-53, key = mix64(seed ^ mix64(stream)):
    the SplitMix64 counter stream (Steele, Lea, Flood 2014) used for problem sizes."""
    M = 2 ** 64

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) % M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) % M
        return z ^ (z >> 31)
    key = mix(seed ^ mix(stream))
    return (mix((key + (i + 1) * 0x9E3779B97F4A7C15) % M) >> 11) * 2.0 ** -53


def anderson_instance(s):
    """Size L in 16..48 and disorder W in [2, 16] of batched instance s (streams 5, 6)."""
    return 16 + int(33.0 * _splitmix_uniform(s, 5, 0)), 2.0 + 14.0 * _splitmix_uniform(s, 6, 0)
