"""Seeded synthetic inputs for the hierarchical collective path.

This module holds no collective arithmetic: it only draws the per-rank
buffers and the request mixes that both the CUDA path and the CPU oracle are
fed with. Every generator is a pure function of its arguments and seed
(NumPy PCG64), so the two sides see bit-identical inputs.

Workload shapes follow the paper's evaluation: buffers of p*d elements per
rank (Sec. 6.2, throughput d*p/t), values drawn per rank.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "uniform_ranks",
    "int_ranks",
    "scaled_normal_ranks",
    "random_leaf_set",
    "batch_mix",
    "poisson_requests",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_ranks(P: int, n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """P rows of n float32 values drawn from U[lo, hi)."""
    g = rng(seed)
    return g.uniform(lo, hi, size=(P, n)).astype(np.float32)


def int_ranks(P: int, n: int, seed: int = 0, lo: int = -(2**31), hi: int = 2**31 - 1) -> np.ndarray:
    """P rows of n int32 values, full range by default (sums wrap)."""
    g = rng(seed)
    return g.integers(lo, hi, size=(P, n), dtype=np.int64, endpoint=True).astype(np.int32)


def scaled_normal_ranks(P: int, n: int, seed: int = 0, decades: float = 3.0) -> np.ndarray:
    """Rank r holds N(0,1) * 10**u_r with u_r ~ U(-decades, decades) (float32)."""
    g = rng(seed)
    u = g.uniform(-decades, decades, size=(P, 1))
    x = g.standard_normal(size=(P, n)) * (10.0 ** u)
    return x.astype(np.float32)


def random_leaf_set(P: int, seed: int, min_size: int = 1) -> list[int]:
    """A random non-empty subset of ranks (sorted)."""
    g = rng(seed)
    k = int(g.integers(min_size, P, endpoint=True))
    return sorted(int(v) for v in g.choice(P, size=k, replace=False))


_TWO_LEVEL = {8: [(2, 4), (4, 2)], 16: [(4, 4)], 32: [(4, 8), (8, 4)], 64: [(4, 16), (8, 8)]}


def batch_mix(n: int = 256, seed: int = 0, min_bytes: int = 4096, max_bytes: int = 16 << 20,
              ranks=(8, 16, 32), kinds=("allgather", "reducescatter", "allreduce"),
              dtypes=("f32", "bf16")) -> list[dict]:
    """A list of n collective descriptions: kind, P, two-level hierarchy,
    per-rank bytes (log-uniform, rounded to a multiple of 16*P bytes so that
    every per-rank chunk starts on a 16-byte boundary), dtype."""
    g = rng(seed)
    out = []
    for _ in range(n):
        P = int(g.choice(ranks))
        hs = _TWO_LEVEL[P]
        h = hs[int(g.integers(0, len(hs)))]
        b = float(np.exp(g.uniform(np.log(min_bytes), np.log(max_bytes))))
        quantum = 16 * P
        nbytes = max(quantum, int(b) // quantum * quantum)
        out.append({
            "kind": str(kinds[int(g.integers(0, len(kinds)))]),
            "P": P,
            "hierarchy": list(h),
            "bytes_per_rank": nbytes,
            "dtype": str(dtypes[int(g.integers(0, len(dtypes)))]),
        })
    return out


def poisson_requests(rate_hz: float, duration_s: float, seed: int = 0,
                     kinds=("broadcast", "scatter", "gather", "allgather", "reducescatter",
                            "allreduce", "alltoall"),
                     ranks=(8, 16, 64), min_bytes: int = 1024, max_bytes: int = 256 << 20,
                     dtypes=("f32", "bf16", "i32"), shapes: int = 0) -> list[dict]:
    """Arrival times (Poisson process) and descriptions of served requests.
    With ``shapes`` > 0, that many request shapes are drawn first (from the
    same distributions) and every arrival takes one of them uniformly, so
    that shapes recur as they do in a service that runs a fixed model."""
    g = rng(seed)
    hier = {8: [2, 4], 16: [4, 4], 64: [4, 4, 4]}

    def draw():
        P = int(g.choice(ranks))
        b = float(np.exp(g.uniform(np.log(min_bytes), np.log(max_bytes))))
        quantum = 16 * P
        nbytes = max(quantum, int(b) // quantum * quantum)
        return {"kind": str(kinds[int(g.integers(0, len(kinds)))]), "P": P, "hierarchy": list(hier[P]),
                "bytes_per_rank": nbytes, "dtype": str(dtypes[int(g.integers(0, len(dtypes)))])}

    pool = [draw() for _ in range(shapes)]
    t = 0.0
    out = []
    while True:
        t += float(g.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        d = dict(pool[int(g.integers(0, shapes))]) if shapes else draw()
        d["t"] = t
        out.append(d)
    return out
