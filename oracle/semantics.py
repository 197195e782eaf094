"""Plain semantics of primitives and collectives (paper Sec. 3.1-3.3, Table 2).

Readings (the paper is silent on these; each is stated once here):

* Sum order.  A reduction's result is the *hierarchical nested fold*: a rank
  contributes its own values; a level-l group contributes the left fold, in
  the payload's arithmetic (FP32 round-to-nearest-even, no fused
  multiply-add; int32 wraps; BF16 and FP8 decoded to FP32, folded, and the
  group's result encoded once), of the contributions of its non-empty
  subgroups in ascending index order.  It depends only on the hierarchy and
  the leaf set -- not on the root, striping, pipeline depth or
  representatives -- so a factorized schedule must reproduce it exactly.
* Races.  Two primitives of one epoch that write overlapping ranges, or where
  one writes what another reads, race (Sec. 3.2: the result is undefined).
  ``find_race`` reports them; the library rejects such programs.
* A multicast whose root is also a leaf delivers to the root's own
  destination (nothing to do when source and destination coincide, the
  "dashed edges" of Fig. 4).
* Ring order (Sec. 4.4).  With ``ring(n)`` the n nodes (the groups of P/n
  ranks) form a chain that starts at the root's node and visits the nodes in
  ascending order, cyclically; nodes without leaves are skipped.  Partial
  results travel the chain backwards, so the reduction is a right fold over
  the chain: the last node contributes its nested fold; every earlier node
  folds its own subgroups' contributions and then the partial received from
  its successor (one reduce step, encoded once).  The result depends on the
  root's node; it equals the tree's for order-free arithmetic (int32).
"""
from __future__ import annotations

import numpy as np

from .hierarchy import check, group_sizes, ring_level
from .lowprec import from_acc, to_acc
from .model import Multicast, Program, Reduction


# ---------------------------------------------------------------------------
# the fixed-order sum
# ---------------------------------------------------------------------------

def combine(a: np.ndarray, b: np.ndarray, op: str = "sum") -> np.ndarray:
    """One step of a reduction's fold (Sec. 3.1: sum, max, logical or, ...).
    sum: the arrays' own arithmetic; max / min: IEEE maxNum / minNum for
    floats (a NaN operand yields the other), plain for int32; lor (int32): 1
    where either operand is nonzero, else 0."""
    if op == "sum":
        return a + b
    if op == "max":
        return np.fmax(a, b) if a.dtype.kind == "f" else np.maximum(a, b)
    if op == "min":
        return np.fmin(a, b) if a.dtype.kind == "f" else np.minimum(a, b)
    if op == "lor":
        return ((a != 0) | (b != 0)).astype(a.dtype)
    raise ValueError(op)


def nested_fold(values: dict, hierarchy, dtype: str | None = None, op: str = "sum", ring: int = 1,
                root: int = 0) -> np.ndarray:
    """Hierarchical nested fold of ``values`` (rank -> array) over ``hierarchy``.

    S(rank r) = values[r]; S(group) = the left fold over the S(subgroup) of
    the subgroups that hold at least one contributing rank, in ascending
    order.  For f32 / i32 (and ``dtype`` None) the fold adds in the arrays'
    own dtype (IEEE RNE for float32, wrapping for int32).  For the reduced
    precision payloads ("bf16", "fp8") the subgroup values are decoded to
    binary32, folded with binary32 adds and the group's result encoded once
    (lowprec); a group with a single contributing subgroup passes its value
    through unchanged (Sec. 3.1: with one leaf the operation is omitted).
    ``op`` selects the combining operation (``combine``).  With ``ring`` > 1
    the levels above the ring's nodes are folded along the chain that starts
    at ``root``'s node (ring order, above) instead.
    """
    if not values:
        raise ValueError("empty leaf set")
    h = list(hierarchy)
    G = group_sizes(h)
    ranks = sorted(values)
    low = dtype in ("bf16", "fp8")

    def S(level: int, base: int, members: list):
        if level == len(h):
            return values[base]
        sub = G[level + 1]
        parts = []
        for q in range(h[level]):
            lo = base + q * sub
            inside = [r for r in members if lo <= r < lo + sub]
            if inside:
                parts.append(S(level + 1, lo, inside))
        if len(parts) == 1:
            return parts[0].copy()
        return fold(parts)

    def fold(parts):
        if not low:
            acc = parts[0].copy()
            for p in parts[1:]:
                acc = combine(acc, p, op)
            return acc
        acc = to_acc(parts[0], dtype).copy()
        for p in parts[1:]:
            acc = combine(acc, to_acc(p, dtype), op).astype(np.float32)
        return from_acc(acc, dtype)

    if ring == 1:
        return S(0, 0, ranks)
    lr = ring_level(h, ring)
    N = G[lr]
    a0 = root // N
    chain = []
    for i in range(ring):
        a = (a0 + i) % ring
        inside = [r for r in ranks if a * N <= r < (a + 1) * N]
        if inside:
            chain.append((a, inside))

    def node_parts(a, members):
        """Contributions the node folds: its non-empty subgroups (the node's
        own value when a node is a single rank)."""
        if lr == len(h):
            return [values[a]]
        sub = G[lr + 1]
        out = []
        for q in range(h[lr]):
            lo = a * N + q * sub
            inside = [r for r in members if lo <= r < lo + sub]
            if inside:
                out.append(S(lr + 1, lo, inside))
        return out

    acc = None
    for a, members in reversed(chain):
        if acc is None:
            acc = S(lr, a * N, members)
        else:
            acc = fold(node_parts(a, members) + [acc])
    return acc


def fsum64(values: list) -> np.ndarray:
    """Elementwise FP64 sum (the error reference of the reduced-precision payloads)."""
    acc = np.zeros_like(np.asarray(values[0], dtype=np.float64))
    for v in values:
        acc = acc + np.asarray(v, dtype=np.float64)
    return acc


# ---------------------------------------------------------------------------
# primitives and programs
# ---------------------------------------------------------------------------

def _view(mem: dict, ref, n: int) -> np.ndarray:
    return mem[ref.key][ref.off:ref.off + n]


def apply_multicast(p: Multicast, mem: dict) -> None:
    """M(i, j, d): every leaf's destination receives the root's d elements (Sec. 3.1)."""
    src = _view(mem, p.src, p.count).copy()
    for j in p.leaves:
        _view(mem, p.dsts[j], p.count)[...] = src


def apply_reduction(p: Reduction, mem: dict, hierarchy, dtype: str | None = None, ring: int = 1) -> None:
    """R(i, j, d, op): the root's destination receives the fixed-order fold of
    the leaves' d elements (Sec. 3.1)."""
    if p.count == 0:
        return
    vals = {i: _view(mem, p.srcs[i], p.count).copy() for i in p.leaves}
    _view(mem, p.dst, p.count)[...] = nested_fold(vals, hierarchy, dtype, p.op, ring, p.root)


def run_program(prog: Program, mem: dict, hierarchy, ring: int = 1) -> dict:
    """Execute the program's epochs in order; inside an epoch the (race-free)
    primitives are applied in registration order, which Sec. 3.2 makes
    irrelevant.  ``ring`` selects the ring order of the sums (Sec. 4.4)."""
    check(hierarchy, prog.P)
    ring_level(hierarchy, ring)
    for epoch in prog.epochs:
        for p in epoch:
            if isinstance(p, Multicast):
                apply_multicast(p, mem)
            else:
                apply_reduction(p, mem, hierarchy, prog.dtype, ring)
    return mem


# ---------------------------------------------------------------------------
# races (Sec. 3.2)
# ---------------------------------------------------------------------------

def accesses(p) -> tuple[list, list]:
    """(reads, writes) of a primitive as (key, lo, hi) element ranges (Sec. 3.2)."""
    if isinstance(p, Multicast):
        reads = [(p.src.key, p.src.off, p.src.off + p.count)]
        writes = []
        for j in p.leaves:
            d = p.dsts[j]
            if j == p.root and d == p.src:
                continue                      # in-place root: nothing written
            writes.append((d.key, d.off, d.off + p.count))
        return (reads if p.count else []), (writes if p.count else [])
    reads = [(p.srcs[i].key, p.srcs[i].off, p.srcs[i].off + p.count) for i in p.leaves]
    writes = [(p.dst.key, p.dst.off, p.dst.off + p.count)]
    return (reads if p.count else []), (writes if p.count else [])


def _overlap(a, b) -> bool:
    return a[0] == b[0] and a[1] < b[2] and b[1] < a[2]


def find_race(prog: Program):
    """First pair of primitives of one epoch that race, or None.  A primitive
    whose own writes overlap each other (two leaves sharing a destination) or
    overlap its own source is reported as racing with itself."""
    for e, epoch in enumerate(prog.epochs):
        acc = [accesses(p) for p in epoch]
        for a in range(len(epoch)):
            ra, wa = acc[a]
            for x in range(len(wa)):
                for y in range(x + 1, len(wa)):
                    if _overlap(wa[x], wa[y]):
                        return (e, a, a)
                for r in ra:
                    if _overlap(wa[x], r):
                        return (e, a, a)
            for b in range(a + 1, len(epoch)):
                rb, wb = acc[b]
                if any(_overlap(w, v) for w in wa for v in wb + rb) or \
                        any(_overlap(w, v) for w in wb for v in ra):
                    return (e, a, b)
    return None


# ---------------------------------------------------------------------------
# direct definitions of the collectives (Table 2, Sec. 3.2), without primitives
# x[r] is rank r's send buffer, the result y[r] its receive buffer.
# ---------------------------------------------------------------------------

def _chunks(v: np.ndarray, P: int):
    d = v.shape[0] // P
    return [v[k * d:(k + 1) * d] for k in range(P)]


def def_broadcast(x, root):
    """Table 2, Broadcast: y_r = x_root for every r."""
    return [x[root].copy() for _ in range(len(x))]


def def_reduce(x, root, hierarchy, dtype=None):
    """Table 2, Reduce: only the root's result is defined; other ranks' y are
    untouched (None)."""
    y = [None] * len(x)
    y[root] = nested_fold({r: x[r] for r in range(len(x))}, hierarchy, dtype)
    return y


def def_allgather(x):
    """Table 2, All-gather: chunk i of y_r = x_i."""
    return [np.concatenate(x) for _ in range(len(x))]


def def_reducescatter(x, hierarchy, dtype=None):
    """Table 2, Reduce-scatter: y_j = sum over r of chunk j of x_r (the
    nested fold)."""
    P = len(x)
    return [nested_fold({r: _chunks(x[r], P)[j] for r in range(P)}, hierarchy, dtype) for j in range(P)]


def def_allreduce(x, hierarchy, dtype=None):
    """Table 2, All-reduce: y_r = sum over r' of x_r' (the nested fold)."""
    s = nested_fold({r: x[r] for r in range(len(x))}, hierarchy, dtype)
    return [s.copy() for _ in range(len(x))]


def def_scatter(x, root):
    """Table 2, Scatter: y_j = chunk j of x_root."""
    return [c.copy() for c in _chunks(x[root], len(x))]


def def_gather(x, root):
    """Table 2, Gather: chunk i of y_root = x_i."""
    y = [None] * len(x)
    y[root] = np.concatenate(x)
    return y


def def_alltoall(x):
    """Table 2, All-to-all: chunk i of y_j = chunk j of x_i."""
    P = len(x)
    ch = [_chunks(x[i], P) for i in range(P)]
    return [np.concatenate([ch[i][j] for i in range(P)]) for j in range(P)]
