"""Seeded test programs shared by the CPU and GPU parity tests."""
from __future__ import annotations

import numpy as np

from oracle.model import Program
from synth import random_leaf_set


def random_program(P: int, seed: int, dtype: str = "f32", chunks: int = 3, max_n: int = 40) -> Program:
    """Two epochs over disjoint chunks: epoch 0 mixes multicasts and
    reductions with random roots and sparse leaf sets; epoch 1 forwards, in
    place, what a root holds in its receive chunk."""
    g = np.random.Generator(np.random.PCG64(seed))
    prog = Program(P, dtype)
    n = int(g.integers(1, max_n))
    send = [prog.buffer(("send", r), n * chunks) for r in range(P)]
    recv = [prog.buffer(("recv", r), n * chunks) for r in range(P)]
    for c in range(chunks):
        leaves = random_leaf_set(P, seed * 31 + c)
        root = int(g.integers(0, P))
        if g.integers(0, 2):
            prog.multicast(root, leaves, n, send[root].shift(c * n),
                           {j: recv[j].shift(c * n) for j in leaves})
        else:
            prog.reduction(leaves, root, n, {i: send[i].shift(c * n) for i in leaves},
                           recv[root].shift(c * n))
    prog.fence()
    for c in range(chunks):
        root = int(g.integers(0, P))
        leaves = [j for j in random_leaf_set(P, seed * 97 + c) if j != root]
        if not leaves:
            continue
        prog.multicast(root, leaves, n, recv[root].shift(c * n),
                       {j: recv[j].shift(c * n) for j in leaves})
    return prog


def fill(prog: Program, seed: int, zero_frac: float = 0.0) -> dict:
    """Random contents for every buffer of ``prog`` (NumPy): uniform[-1, 1]
    values (encoded for BF16 / FP8 payloads), full-range int32; with
    ``zero_frac`` a random fraction of the elements (f32, i32, bf16) is then
    set to +0, so that logical-or and max / min see zeros and ties."""
    from oracle.lowprec import encode
    mem = prog.allocate()
    g = np.random.Generator(np.random.PCG64(seed))
    for k, v in mem.items():
        if prog.dtype == "f32":
            v[...] = g.uniform(-1, 1, size=v.shape).astype(np.float32)
        elif prog.dtype == "i32":
            v[...] = g.integers(-2**31, 2**31 - 1, size=v.shape, endpoint=True, dtype=np.int64)
        elif prog.dtype == "bf16":
            v[...] = encode(g.uniform(-1, 1, size=v.shape).astype(np.float32), "bf16")
        else:   # fp8 blocks of 128 values
            v[...] = encode(g.uniform(-1, 1, size=v.shape[0] * 128).astype(np.float32), "fp8")
    if zero_frac > 0 and prog.dtype != "fp8":
        z = np.random.Generator(np.random.PCG64(seed + 7919))
        for v in mem.values():
            v[z.random(v.shape) < zero_frac] = 0
    return mem
