"""The optimizer of paper Sec. 4: striping, tree factorization, pipelining.

Each primitive is factorized, in the paper's order (Sec. 4.4: striping, then
the ring, then the tree), into point-to-point operations within one level of
the hierarchy:

* a *copy* moves n elements from one rank to one or more ranks -- one
  multicast hop of a tree node (the holder forwards to the representatives
  of its sibling subgroups), a striping transfer, or a local self-copy;
* a *reduce* folds the partial sums of f subgroups, in ascending subgroup
  order, into one output (the fixed-order sum of ``semantics``).

Readings (the paper is silent or ambiguous; each is stated once):

1. Representative.  When a holder at level l forwards into a sibling
   subgroup q, the receiving rank is the rank of q at the holder's offset
   within its own subgroup (this yields the hops g0->g6, g0->g3, g6->g9 of
   the {2,2,3} example in Sec. 4.3) if that rank is a leaf, else the lowest
   leaf of q.  Subgroups without leaves are pruned (Sec. 4.2).  A reduction
   mirrors this: a subgroup's partial sum is formed at its representative
   and read from there by the parent's representative.
2. Stripe ranks (Sec. 4.3).  The s branches are rooted at the ranks
   o, o+1, ..., o+s-1 (mod G) of the root's smallest enclosing group of size
   G >= s, where o is the root's offset in it; branch 0 is the root.  A
   multicast first copies piece b from the root to stripe rank k_b (into its
   destination when k_b is a leaf, else into a relay buffer) and then
   multicasts it from k_b; a reduction reduces piece b at k_b and then copies
   it to the root ("sum_j R(0, j, d/s)" of Sec. 4.3 is read as single-leaf
   reductions, i.e. copies).  A primitive none of whose leaves lies outside
   the stripe group has no inter-group traffic to spread and is not striped.
3. Pieces.  A primitive of ``count`` elements is cut into s*m pieces (s
   branches of m pipeline channels, Sec. 4.5) at the boundaries
   min(count, roundup(ceil(count*k/(s*m)), q)), k = 0..s*m, where q is the
   16-byte quantum of the payload (4 elements of f32/i32, 8 of bf16, 128 of
   fp8).  Branch b owns pieces b*m .. b*m+m-1; empty pieces are skipped.
4. Self-delivery.  A multicast root that is also a leaf needs nothing when
   its source and destination coincide (the dashed edges of Fig. 4).
   Otherwise the branch rooted at the root itself copies the piece locally,
   and every other branch b delivers its piece to the root like to any other
   leaf (Sec. 4.3: each striping GPU multicasts its piece to all GPUs but
   itself).  The reduction mirror is the same: the root's own contribution
   to piece b is folded at k_b and the result copied back.
5. Fences (Sec. 3.3) are data dependencies, not barriers: an operation of a
   later epoch follows exactly the earlier-epoch operations whose user-buffer
   ranges it reads after they write, writes after they read, or writes after
   they write.
6. Ring (Sec. 4.4).  ``ring(n)`` chains the n nodes -- the groups of P/n
   ranks, which must be the groups of one hierarchy level
   (``hierarchy.ring_level``) -- starting at the node of the branch's stripe
   rank and going up cyclically; nodes without leaves are skipped.  The rank
   entering a node is chosen like a representative (reading 1) from the
   previous node's entry rank.  A multicast hops node to node and each entry
   rank multicasts inside its node with the tree; a reduction mirrors it:
   the last node's tree fold travels backwards, and every other entry rank
   folds its node's subgroup partials followed by the incoming partial in
   one reduce (the ring order of ``semantics``).  With n > 1 the stripe may
   not exceed the node size, so that all branches start in the root's node.

Byte accounting.  ``level_bytes[l]``: for every copy destination, and every
reduce input, that sits on another rank, n elements cross the level of the
two ranks (``hierarchy.level_of``).  ``hbm_bytes``: a copy reads n and writes
n per destination; an f-input reduce reads f*n and writes n.
"""
from __future__ import annotations

import bisect
from dataclasses import dataclass, field
from math import ceil

from .hierarchy import check, group_sizes, level_of, ring_level
from .model import DTYPES, QUANTUM, Multicast, Program, Ref


@dataclass
class Op:
    """One point-to-point step of a factorized primitive (Sec. 4): a copy of
    n units to every destination, or an in-order fold of the sources into one
    destination."""
    kind: str                 # "copy" | "reduce"
    srcs: list                # [(rank, Ref)]
    dsts: list                # [(rank, Ref)]
    n: int
    level: int | None         # hierarchy level crossed; None for a local copy
    deps: list = field(default_factory=list)
    prim: int = -1
    epoch: int = 0
    branch: int = 0
    channel: int = 0
    op: str = "sum"           # combining operation of a reduce


@dataclass
class Plan:
    """A factorized program (Sec. 4): its steps in emission order, each after
    its dependencies, and its relay buffers."""
    P: int
    hierarchy: list
    stripe: int
    pipeline: int
    dtype: str
    ops: list
    scratch: dict             # key -> length
    esize: int
    ring: int = 1

    # ---- accounting -------------------------------------------------------
    def level_bytes(self) -> list:
        """Bytes that cross each hierarchy level (Sec. 4.1; Table 3's per-node
        volumes are the top-level entry)."""
        out = [0] * len(self.hierarchy)
        for op in self.ops:
            if op.kind == "copy":
                a = op.srcs[0][0]
                pairs = [(a, b) for b, _ in op.dsts]
            else:
                t = op.dsts[0][0]
                pairs = [(a, t) for a, _ in op.srcs]
            for a, b in pairs:
                lv = level_of(a, b, self.hierarchy)
                if lv is not None:
                    out[lv] += op.n * self.esize
        return out

    def hbm_bytes(self) -> tuple:
        """Schedule bytes (read, written): a copy reads n and writes n per
        destination; an f-input fold reads f*n and writes n."""
        rd = wr = 0
        for op in self.ops:
            if op.kind == "copy":
                rd += op.n
                wr += op.n * len(op.dsts)
            else:
                rd += op.n * len(op.srcs)
                wr += op.n
        return rd * self.esize, wr * self.esize

    def depths(self) -> list:
        """Dependency depth of every step, i.e. its stage (Sec. 4.5)."""
        d = [0] * len(self.ops)
        for i, op in enumerate(self.ops):        # ops are emitted after their deps
            d[i] = 1 + max((d[j] for j in op.deps), default=-1)
        return d

    def stages(self) -> int:
        """Length of the longest dependency chain (number of pipeline stages
        of the unpipelined schedule, Sec. 4.5)."""
        return 1 + max(self.depths(), default=-1) if self.ops else 0

    def slots(self) -> int:
        """Slots of the overlapped pipeline (Sec. 4.5, Fig. 7): channel c of a
        piece starts at slot c and an op runs one slot after its latest
        dependency, so S dependent stages over m channels fill S + m - 1
        slots (reading: the figure staggers the channels by one stage)."""
        s = [0] * len(self.ops)
        for i, op in enumerate(self.ops):        # ops are emitted after their deps
            s[i] = max(op.channel, 1 + max((s[j] for j in op.deps), default=-1))
        return 1 + max(s, default=-1) if self.ops else 0


def piece_bounds(count: int, parts: int, quantum: int) -> list:
    """Reading 3: boundaries of ``parts`` pieces."""
    out = []
    for k in range(parts + 1):
        b = ceil(count * k / parts)
        b = -(-b // quantum) * quantum
        out.append(min(count, b))
    return out


class Factorizer:
    """The factorization of Sec. 4 in the paper's order: striping (Sec. 4.3),
    ring (Sec. 4.4) and tree (Sec. 4.2) per primitive, pipeline channels
    (Sec. 4.5), fence dependencies (Sec. 3.3)."""
    def __init__(self, prog: Program, hierarchy, stripe: int = 1, pipeline: int = 1, ring: int = 1):
        self.prog = prog
        self.h = check(hierarchy, prog.P)
        self.L = len(self.h)
        self.G = group_sizes(self.h)
        if stripe < 1 or stripe > prog.P or pipeline < 1:
            raise ValueError("stripe must be in [1, P] and pipeline >= 1")
        self.ring = int(ring)
        self.lr = ring_level(self.h, self.ring)      # level of the ring's nodes
        if self.ring > 1 and stripe > self.G[self.lr]:
            raise ValueError("with a ring, the stripe may not exceed the node size")
        self.s = stripe
        self.m = pipeline
        self.ops: list = []
        self.scratch: dict = {}
        self._cur = None            # (prim, epoch, branch, channel)
        self._op = "sum"

    # ---- helpers -------------------------------------------------------------
    def _emit(self, kind, srcs, dsts, n, level, deps) -> int:
        prim, epoch, b, c = self._cur
        self.ops.append(Op(kind, srcs, dsts, n, level, sorted(set(d for d in deps if d is not None)),
                           prim, epoch, b, c, self._op))
        return len(self.ops) - 1

    def _new_scratch(self, n: int) -> Ref:
        key = ("scratch", len(self.scratch))
        self.scratch[key] = n
        return Ref(key, 0)

    def _lvl(self, a, b):
        return level_of(a, b, self.h)

    def stripe_ranks(self, root: int, leaves) -> list:
        """Reading 2."""
        if self.s == 1:
            return [root]
        l = max(l for l in range(self.L + 1) if self.G[l] >= self.s)
        g = self.G[l]
        base, o = root - root % g, root % g
        if all(base <= r < base + g for r in leaves):
            return [root]
        return [base + (o + b) % g for b in range(self.s)]

    def _rep(self, qbase, sub, holder, qleaves):
        """Reading 1."""
        cand = qbase + holder % sub
        return cand if cand in qleaves else min(qleaves)

    # ---- multicast tree (Sec. 4.2) --------------------------------------------
    def _mcast_tree(self, l, base, holder, src: Ref, src_op, leaves, dst_of, n):
        if l == self.L or not leaves:
            return
        sub = self.G[l + 1]
        own = None
        hops = []
        for q in range(self.h[l]):
            qb = base + q * sub
            ql = [r for r in leaves if qb <= r < qb + sub]
            if qb <= holder < qb + sub:
                own = (qb, ql)
            elif ql:
                hops.append((qb, self._rep(qb, sub, holder, ql), ql))
        op = None
        if hops:
            op = self._emit("copy", [(holder, src)], [(rep, dst_of(rep)) for _, rep, _ in hops],
                            n, l, [src_op])
        if own is not None:
            self._mcast_tree(l + 1, own[0], holder, src, src_op, own[1], dst_of, n)
        for qb, rep, ql in hops:
            self._mcast_tree(l + 1, qb, rep, dst_of(rep), op, [r for r in ql if r != rep], dst_of, n)

    # ---- reduction tree (Sec. 4.2, mirrored) ------------------------------------
    def _red_tree(self, l, base, target, leaves, src_of, out, n):
        """Forms the fold of ``leaves`` (all inside this level-l group) at rank
        ``target``; returns (Ref, producing op or None).  ``out`` is the
        required location of the result, or None for "anywhere at target"."""
        if l == self.L:
            ref = src_of(target)                 # the group is the leaf ``target`` itself
            if out is None or out == ref:
                return ref, None
            return out, self._emit("copy", [(target, ref)], [(target, out)], n, None, [])
        sub = self.G[l + 1]
        parts = []
        for q in range(self.h[l]):
            qb = base + q * sub
            ql = [r for r in leaves if qb <= r < qb + sub]
            if not ql:
                continue
            rep = target if qb <= target < qb + sub else self._rep(qb, sub, target, ql)
            parts.append((qb, rep, ql))
        if len(parts) == 1 and parts[0][1] == target:
            return self._red_tree(l + 1, parts[0][0], target, parts[0][2], src_of, out, n)
        inputs = [(rep,) + self._red_tree(l + 1, qb, rep, ql, src_of, None, n) for qb, rep, ql in parts]
        if out is None:
            out = self._new_scratch(n)
        kind = "reduce" if len(inputs) > 1 else "copy"
        op = self._emit(kind, [(rep, ref) for rep, ref, _ in inputs], [(target, out)], n, l,
                        [o for _, _, o in inputs])
        return out, op

    # ---- ring across nodes (Sec. 4.4), tree inside them ----------------------------
    def _node_leaves(self, a, leaves):
        N = self.G[self.lr]
        return [r for r in leaves if a * N <= r < (a + 1) * N]

    def _mcast_ring(self, holder, src: Ref, src_op, leaves, dst_of, n):
        if self.ring == 1:
            self._mcast_tree(0, 0, holder, src, src_op, leaves, dst_of, n)
            return
        N = self.G[self.lr]
        a0 = holder // N
        self._mcast_tree(self.lr, a0 * N, holder, src, src_op, self._node_leaves(a0, leaves), dst_of, n)
        for i in range(1, self.ring):
            a = (a0 + i) % self.ring
            nl = self._node_leaves(a, leaves)
            if not nl:
                continue
            e = self._rep(a * N, N, holder, nl)
            hop = self._emit("copy", [(holder, src)], [(e, dst_of(e))], n, self._lvl(holder, e), [src_op])
            self._mcast_tree(self.lr, a * N, e, dst_of(e), hop, [r for r in nl if r != e], dst_of, n)
            holder, src, src_op = e, dst_of(e), hop

    def _red_ring(self, target, leaves, src_of, out, n):
        """The ring-order fold of ``leaves`` at ``target`` (semantics, ring
        order); returns (Ref, producing op or None) like ``_red_tree``."""
        if self.ring == 1:
            return self._red_tree(0, 0, target, leaves, src_of, out, n)
        N = self.G[self.lr]
        a0 = target // N
        chain = []
        prev = target
        for i in range(self.ring):
            a = (a0 + i) % self.ring
            nl = self._node_leaves(a, leaves)
            if not nl:
                continue
            e = target if a == a0 else self._rep(a * N, N, prev, nl)
            chain.append((a, nl, e))
            prev = e
        inc = None
        for idx in range(len(chain) - 1, -1, -1):
            a, nl, e = chain[idx]
            o = out if (idx == 0 and e == target) else None
            if inc is None:
                ref, op = self._red_tree(self.lr, a * N, e, nl, src_of, o, n)
            else:
                ref, op = self._red_node(a, e, nl, src_of, o, n, inc)
            inc = (e, ref, op)
        e, ref, op = inc
        if e == target:
            return ref, op
        dst = out if out is not None else self._new_scratch(n)
        return dst, self._emit("copy", [(e, ref)], [(target, dst)], n, self._lvl(e, target), [op])

    def _red_node(self, a, target, nl, src_of, out, n, inc):
        """One ring node that is not the chain's last: fold the node's
        subgroup partials, then the partial ``inc`` = (rank, Ref, op) received
        from the next node, into one reduce at ``target``."""
        if self.lr == self.L:
            inputs = [(target, src_of(target), None)]
        else:
            sub = self.G[self.lr + 1]
            inputs = []
            for q in range(self.h[self.lr]):
                qb = a * self.G[self.lr] + q * sub
                ql = [r for r in nl if qb <= r < qb + sub]
                if not ql:
                    continue
                rep = target if qb <= target < qb + sub else self._rep(qb, sub, target, ql)
                inputs.append((rep,) + self._red_tree(self.lr + 1, qb, rep, ql, src_of, None, n))
        inputs.append(inc)
        if out is None:
            out = self._new_scratch(n)
        level = min(lv for lv in (self._lvl(r, target) for r, _, _ in inputs) if lv is not None)
        op = self._emit("reduce", [(r, ref) for r, ref, _ in inputs], [(target, out)], n, level,
                        [o for _, _, o in inputs])
        return out, op

    # ---- one primitive -----------------------------------------------------------
    def _multicast(self, p: Multicast):
        if p.count == 0:
            return
        ks = self.stripe_ranks(p.root, p.leaves)
        nb = len(ks)
        bounds = piece_bounds(p.count, nb * self.m, QUANTUM[self.prog.dtype])
        self_copy = p.root in p.leaves and p.dsts[p.root] != p.src
        leaves = [j for j in p.leaves if j != p.root]
        if self_copy:
            leaves_k = leaves + [p.root]           # the root as a leaf of the other branches
        else:
            leaves_k = leaves
        for b in range(nb):
            for c in range(self.m):
                lo, hi = bounds[b * self.m + c], bounds[b * self.m + c + 1]
                if hi <= lo:
                    continue
                n = hi - lo
                self._cur = (self._cur[0], self._cur[1], b, c)
                src = p.src.shift(lo)
                k = ks[b]
                holder_src, holder_op = src, None
                if k == p.root:
                    if self_copy:
                        self._emit("copy", [(p.root, src)], [(p.root, p.dsts[p.root].shift(lo))],
                                   n, None, [])
                    branch = leaves
                else:
                    dst = p.dsts[k].shift(lo) if k in p.dsts else self._new_scratch(n)
                    holder_op = self._emit("copy", [(p.root, src)], [(k, dst)], n, self._lvl(p.root, k), [])
                    holder_src = dst
                    branch = sorted(j for j in leaves_k if j != k)
                self._mcast_ring(k, holder_src, holder_op, branch, lambda r, lo=lo: p.dsts[r].shift(lo), n)

    def _reduction(self, p):
        if p.count == 0:
            return
        ks = self.stripe_ranks(p.root, p.leaves)
        nb = len(ks)
        bounds = piece_bounds(p.count, nb * self.m, QUANTUM[self.prog.dtype])
        for b in range(nb):
            for c in range(self.m):
                lo, hi = bounds[b * self.m + c], bounds[b * self.m + c + 1]
                if hi <= lo:
                    continue
                n = hi - lo
                self._cur = (self._cur[0], self._cur[1], b, c)
                final = p.dst.shift(lo)
                k = ks[b]
                src_of = (lambda r, lo=lo: p.srcs[r].shift(lo))
                if k == p.root:
                    self._red_ring(k, list(p.leaves), src_of, final, n)
                else:
                    ref, op = self._red_ring(k, list(p.leaves), src_of, None, n)
                    self._emit("copy", [(k, ref)], [(p.root, final)], n, self._lvl(k, p.root),
                               [op])

    # ---- whole program -----------------------------------------------------------
    def run(self) -> Plan:
        """Emit the steps of every primitive in program order, then the fence
        dependencies between epochs (Sec. 3.3, reading 5 above)."""
        pid = 0
        for e, epoch in enumerate(self.prog.epochs):
            first = len(self.ops)
            for p in epoch:
                self._cur = (pid, e, 0, 0)
                if isinstance(p, Multicast):
                    self._op = "sum"
                    self._multicast(p)
                else:
                    self._op = p.op
                    self._reduction(p)
                pid += 1
            if e > 0:
                self._fence_deps(first)
        return Plan(self.prog.P, self.h, self.s, self.m, self.prog.dtype, self.ops,
                    dict(self.scratch), DTYPES[self.prog.dtype].itemsize, self.ring)

    def _fence_deps(self, first: int):
        """Reading 5: dependencies of the ops emitted from ``first`` on (one
        epoch) on the ops of earlier epochs, by overlap of user-buffer ranges."""
        index: dict = {}                        # key -> sorted [(lo, hi, op, is_write)]
        maxlen: dict = {}
        for i in range(first):
            for key, lo, hi, w in _op_accesses(self.ops[i]):
                index.setdefault(key, []).append((lo, hi, i, w))
                maxlen[key] = max(maxlen.get(key, 0), hi - lo)
        for v in index.values():
            v.sort()
        for i in range(first, len(self.ops)):
            extra = set()
            for key, lo, hi, w in _op_accesses(self.ops[i]):
                lst = index.get(key)
                if not lst:
                    continue
                k = bisect.bisect_left(lst, (lo - maxlen[key], -1, -1, False))
                while k < len(lst) and lst[k][0] < hi:
                    a_lo, a_hi, j, aw = lst[k]
                    if a_hi > lo and a_lo < hi and (w or aw):
                        extra.add(j)
                    k += 1
            if extra:
                self.ops[i].deps = sorted(set(self.ops[i].deps) | extra)


def _op_accesses(op: Op):
    """(key, lo, hi, is_write) user-buffer ranges of an op (relay buffers are
    private to their primitive and never cross a fence)."""
    out = []
    for _, r in op.srcs:
        if r.key[0] != "scratch":
            out.append((r.key, r.off, r.off + op.n, False))
    for _, r in op.dsts:
        if r.key[0] != "scratch":
            out.append((r.key, r.off, r.off + op.n, True))
    return out


def factorize(prog: Program, hierarchy, stripe: int = 1, pipeline: int = 1, ring: int = 1) -> Plan:
    """Factorize ``prog`` over ``hierarchy`` with stripe s, pipeline depth m
    and ring(n) (Sec. 4; readings 1-6 above)."""
    return Factorizer(prog, hierarchy, stripe, pipeline, ring).run()
