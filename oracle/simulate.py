"""Execute a factorized plan on NumPy buffers (the schedule simulator).

Operations run one at a time, either in emission order or -- to exercise the
claim that fences are dependencies rather than barriers (Sec. 3.3) -- in a
seeded random order that respects only the plan's dependency edges.
"""
from __future__ import annotations

import numpy as np

from .factorize import Plan
from .lowprec import from_acc, to_acc
from .model import DTYPES
from .semantics import combine


def _view(mem, ref, n):
    return mem[ref.key][ref.off:ref.off + n]


def execute_op(op, mem: dict, dtype: str | None = None) -> None:
    """Run one operation.  A reduce folds its inputs in order; reduced-precision
    payloads are decoded to binary32, folded, and encoded once (lowprec)."""
    if op.kind == "copy":
        src = _view(mem, op.srcs[0][1], op.n).copy()
        for _, d in op.dsts:
            _view(mem, d, op.n)[...] = src
        return
    if dtype in ("bf16", "fp8"):
        acc = to_acc(_view(mem, op.srcs[0][1], op.n), dtype).copy()
        for _, s in op.srcs[1:]:
            acc = combine(acc, to_acc(_view(mem, s, op.n), dtype), op.op).astype(np.float32)
        _view(mem, op.dsts[0][1], op.n)[...] = from_acc(acc, dtype)
        return
    acc = _view(mem, op.srcs[0][1], op.n).copy()
    for _, s in op.srcs[1:]:
        acc = combine(acc, _view(mem, s, op.n), op.op)
    _view(mem, op.dsts[0][1], op.n)[...] = acc


def topo_order(plan: Plan, seed: int | None):
    """A random order of the steps that respects every dependency (any such
    order is a valid execution, Sec. 3.3); emission order for seed None."""
    n = len(plan.ops)
    if seed is None:
        return list(range(n))
    rng = np.random.Generator(np.random.PCG64(seed))
    indeg = [len(op.deps) for op in plan.ops]
    succ = [[] for _ in range(n)]
    for i, op in enumerate(plan.ops):
        for j in op.deps:
            succ[j].append(i)
    ready = [i for i in range(n) if indeg[i] == 0]
    order = []
    while ready:
        k = int(rng.integers(0, len(ready)))
        ready[k], ready[-1] = ready[-1], ready[k]
        i = ready.pop()
        order.append(i)
        for j in succ[i]:
            indeg[j] -= 1
            if indeg[j] == 0:
                ready.append(j)
    if len(order) != n:
        raise AssertionError("dependency cycle in plan")
    return order


def simulate(plan: Plan, mem: dict, order_seed: int | None = None) -> dict:
    """Run every op of ``plan`` on ``mem`` (modified in place; relay buffers
    are added under their scratch keys)."""
    dt = DTYPES[plan.dtype]
    for k, n in plan.scratch.items():
        mem[k] = np.zeros(n, dtype=dt)
    for i in topo_order(plan, order_seed):
        execute_op(plan.ops[i], mem, plan.dtype)
    return mem
