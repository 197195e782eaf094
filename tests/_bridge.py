"""Test-side glue between an oracle ``Program`` (used as a description of a
collective) and the C-ABI library: register the same primitives on a library
communicator at given buffer addresses, and -- on machines without a GPU --
interpret the library's exported step table on NumPy buffers.

The interpreter here is test code: it executes the *library's* plan (its
steps, relay offsets and order) so that the host factorizer can be checked
against the oracle without a GPU.  It shares nothing with the oracle's own
factorizer or simulator.
"""
from __future__ import annotations

import numpy as np

from oracle.lowprec import from_acc, to_acc
from oracle.semantics import combine
from oracle.model import DTYPES, Multicast
from paper_2408_05962_gb300 import hiccl as H

# the oracle counts FP8 programs in 128-value blocks, the C ABI in values
COUNT_SCALE = {"f32": 1, "i32": 1, "bf16": 1, "fp8": 128}


class FakeAddresses:
    """Disjoint 256-byte aligned fake device addresses for every buffer key."""

    def __init__(self, prog, base=0x7f0000000000, gap=4096):
        self.esize = DTYPES[prog.dtype].itemsize
        self.base = {}
        a = base
        for key, n in prog.buffers.items():
            self.base[key] = a
            a += (n * self.esize + gap + 255) // 256 * 256
        self.end = a

    def addr(self, ref) -> int:
        return self.base[ref.key] + ref.off * self.esize

    def resolve(self, addr: int):
        """(buffer key, byte offset) of a fake address."""
        best = None
        for key, b in self.base.items():
            if b <= addr and (best is None or b > best[1]):
                best = (key, b)
        if best is None:
            raise KeyError(hex(addr))
        return best[0], addr - best[1]


def register(prog, addr_of, dtype=None) -> H.Comm:
    """A library communicator holding ``prog``'s primitives at ``addr_of(ref)``."""
    comm = H.Comm(prog.P, dtype or prog.dtype)
    P = prog.P
    k = COUNT_SCALE[prog.dtype]
    for e, epoch in enumerate(prog.epochs):
        if e:
            comm.add_fence()
        for p in epoch:
            send = [0] * P
            recv = [0] * P
            if isinstance(p, Multicast):
                send[p.root] = addr_of(p.src)
                for j in p.leaves:
                    recv[j] = addr_of(p.dsts[j])
                comm.add_multicast(send, recv, p.count * k, p.root, p.leaves)
            else:
                for i in p.leaves:
                    send[i] = addr_of(p.srcs[i])
                recv[p.root] = addr_of(p.dst)
                comm.add_reduction(send, recv, p.count * k, p.leaves, p.root, p.op)
    return comm


def interpret(comm: H.Comm, fake: FakeAddresses, mem: dict, dtype: str) -> dict:
    """Run the library's step table, in table order, on the NumPy buffers
    ``mem`` (keyed like the program's buffers); a reduce step combines with
    the operator the table gives it."""
    info = comm.plan_info()
    dt = DTYPES[dtype]
    byte_views = {k: v.view(np.uint8) for k, v in mem.items()}
    scratch = np.zeros(info["scratch_bytes"] + 16, dtype=np.uint8)

    def view(rank_addr_scr, n):
        _, a, scr = rank_addr_scr
        if scr:
            return scratch[a:a + n]
        key, off = fake.resolve(a)
        return byte_views[key][off:off + n]

    for i in range(info["steps"]):
        st = comm.step(i)
        assert all(q < i for q in st["preds"]), "table order must be topological"
        n = st["nbytes"]
        op = st["op"]
        if st["kind"] == "copy":
            src = view(st["srcs"][0], n).copy()
            for d in st["dsts"]:
                view(d, n)[...] = src
        elif dtype in ("bf16", "fp8"):
            acc = to_acc(view(st["srcs"][0], n).copy().view(dt), dtype).copy()
            for s in st["srcs"][1:]:
                acc = combine(acc, to_acc(view(s, n).copy().view(dt), dtype), op).astype(np.float32)
            view(st["dsts"][0], n)[...] = from_acc(acc, dtype).view(np.uint8)
        else:
            acc = view(st["srcs"][0], n).copy().view(dt)
            for s in st["srcs"][1:]:
                acc = combine(acc, view(s, n).copy().view(dt), op)
            view(st["dsts"][0], n)[...] = acc.view(np.uint8)
    return mem


def interpret_image(comm: H.Comm, fake: FakeAddresses, mem: dict, dtype: str, seed=None) -> dict:
    """Run the library's *table image* -- the work-item records the executor
    reads (``hiccl_debug_image``) -- on the NumPy buffers ``mem``, the way the
    kernel walks it: each item's segments through its runs (segment j lies in
    the run with the largest prefix sum <= j, at byte run.off + (j - prefix) *
    seg of that run's first entry's step), each segment copied or folded with
    the operator and payload its meta word gives.  Operand pointers come from
    the record when inline, else from the step table (the global pointer
    array holds the same values).

    Items run in ticket order, or with ``seed`` in a random order that only
    the image's own dependency data constrain, as concurrent CTAs could run
    them: an item is ready when every entry's step has as many released
    predecessors as its dependency count; a step is complete when as many
    items as its completion target have finished it, and then releases the
    successors its record lists (or, for an item whose lists stay global,
    the step table's)."""
    import struct
    from oracle.model import DTYPES as _DT
    info = comm.plan_info()
    seg = 4032 if dtype == "fp8" else 4096
    dt = _DT[dtype]
    byte_views = {k: v.view(np.uint8) for k, v in mem.items()}
    scratch = np.zeros(info["scratch_bytes"] + 16, dtype=np.uint8)
    lo_user = min(fake.base.values())
    recs, items = comm.image()
    steps = {}

    def view(addr, n):
        if addr < lo_user:                      # relay arena offset (relay base 0)
            return scratch[addr:addr + n]
        key, off = fake.resolve(addr)
        return byte_views[key][off:off + n]

    decoded = []
    for rec, nent, nrun, nptr, nsucc, *_ in items.tolist():
        o = rec * 16
        ent = [struct.unpack_from("<4I", recs, o + 16 * k) for k in range(nent)]
        o += nent * 16
        rpre = list(struct.unpack_from(f"<{nrun + 1}I", recs, o))
        o += ((nrun + 1) * 4 + 15) & ~15
        runs = [struct.unpack_from("<IIQQ", recs, o + 24 * k) for k in range(nrun)]
        o += (nrun * 24 + 15) & ~15
        ptr = list(struct.unpack_from(f"<{nptr}Q", recs, o))
        o += (nptr * 8 + 15) & ~15
        ncmp = 2 * nent + 1 + (0 if nsucc == 0xFFFFFFFF else nsucc)
        cmp = list(struct.unpack_from(f"<{ncmp}I", recs, o))
        decoded.append((ent, rpre, runs, ptr, cmp, nsucc))

    order = list(range(len(decoded)))
    if seed is not None:
        rng = np.random.Generator(np.random.PCG64(seed))
        N = info["steps"]
        succ_table = None
        dep = np.zeros(N, dtype=np.int64)
        done = np.zeros(N, dtype=np.int64)
        indeg = np.zeros(N, dtype=np.int64)
        step_items = [[] for _ in range(N)]
        wait = []                                   # entries of an item whose step is not yet released
        for i, d in enumerate(decoded):
            for e in d[0]:
                indeg[e[0]] = e[3]
                step_items[e[0]].append(i)
            wait.append(sum(1 for e in d[0] if e[3] > 0))
        ready = [i for i in range(len(decoded)) if wait[i] == 0]
        order = []
        while ready:
            r = int(rng.integers(0, len(ready)))
            ready[r], ready[-1] = ready[-1], ready[r]
            i = ready.pop()
            order.append(i)
            ent, _, _, _, cmp, nsucc = decoded[i]
            nent = len(ent)
            for k, e in enumerate(ent):
                done[e[0]] += 1
                if done[e[0]] != cmp[k]:
                    continue
                if nsucc != 0xFFFFFFFF:
                    soff = cmp[nent:2 * nent + 1]
                    lst = cmp[2 * nent + 1:][soff[k]:soff[k + 1]]
                else:
                    if succ_table is None:
                        succ_table = [[] for _ in range(N)]
                        for t in range(N):
                            for q in comm.step(t)["preds"]:
                                succ_table[q].append(t)
                    lst = succ_table[e[0]]
                for t in lst:
                    dep[t] += 1
                    if dep[t] == indeg[t]:
                        for it2 in step_items[t]:
                            wait[it2] -= 1
                            if wait[it2] == 0:
                                ready.append(it2)
        assert len(order) == len(decoded), "some items never became ready: the image's dependencies cannot all be met"

    for idx in order:
        ent, rpre, runs, ptr, _, _ = decoded[idx]
        nrun = len(runs)
        for j in range(rpre[nrun]):
            k = max(r for r in range(nrun) if rpre[r] <= j)
            entry, _, off, nbytes = runs[k]
            step, meta, poff, _ = ent[entry]
            ns, nd = (meta >> 10) & 2047, (meta >> 21) & 2047
            if poff & 0x80000000:
                if step not in steps:
                    st = comm.step(step)
                    steps[step] = [a for (_, a, _) in st["srcs"]] + [a for (_, a, _) in st["dsts"]]
                ops = steps[step]
            else:
                ops = ptr[poff:poff + ns + nd]
            s = j - rpre[k]
            lo = off + s * seg
            n = min(seg, nbytes - s * seg)
            srcs = [view(a + lo, n) for a in ops[:ns]]
            dsts = [view(a + lo, n) for a in ops[ns:]]
            if meta & 3 == 0:
                data = srcs[0].copy()
                for d in dsts:
                    d[...] = data
                continue
            op = H.OP_NAMES[(meta >> 7) & 7]
            if dtype in ("bf16", "fp8"):
                acc = to_acc(srcs[0].copy().view(dt), dtype).copy()
                for x in srcs[1:]:
                    acc = combine(acc, to_acc(x.copy().view(dt), dtype), op).astype(np.float32)
                dsts[0][...] = from_acc(acc, dtype).view(np.uint8)
            else:
                acc = srcs[0].copy().view(dt)
                for x in srcs[1:]:
                    acc = combine(acc, x.copy().view(dt), op)
                dsts[0][...] = acc.view(np.uint8)
    return mem
