"""The collectives of Table 2 composed from primitives (paper Sec. 3.2-3.3).

Every builder returns a ``Program`` over P ranks with per-rank buffers
``("send", r)`` and ``("recv", r)`` (and ``("work", r)`` where a multi-step
form needs an intermediate).  ``d`` is the chunk length in elements: the
largest per-rank buffer holds d*P elements (Sec. 3.2, "largest buffer size is
chosen as dp").

Single-step forms follow Table 2 (Single); the multi-step forms follow Table 2
(Multiple), read right to left with a fence between the two collectives
(Sec. 3.3); ``allreduce`` is the program of Listing 2 (Reduce-scatter, fence,
in-place All-gather whose leaves are all ranks but the root).
"""
from __future__ import annotations

from .model import Program, Ref


def _bufs(prog: Program, P: int, send_len: int, recv_len: int):
    send = [prog.buffer(("send", r), send_len) for r in range(P)]
    recv = [prog.buffer(("recv", r), recv_len) for r in range(P)]
    return send, recv


def _all(P):
    return list(range(P))


# ---- single-step (Table 2, Single) --------------------------------------------

def broadcast(P, d, root=0, dtype="f32"):
    """M(i, U, dp) (Table 2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    prog.multicast(root, _all(P), d * P, send[root], {r: recv[r] for r in range(P)})
    return prog


def reduce(P, d, root=0, dtype="f32", op="sum"):
    """R(U, j, dp, op) (Table 2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    prog.reduction(_all(P), root, d * P, {r: send[r] for r in range(P)}, recv[root], op)
    return prog


def allgather(P, d, dtype="f32"):
    """sum_i M(i, U, d) (Table 2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d, d * P)
    for i in range(P):
        prog.multicast(i, _all(P), d, send[i], {r: recv[r].shift(i * d) for r in range(P)})
    return prog


def reducescatter(P, d, dtype="f32", op="sum"):
    """sum_j R(U, j, d, op) (Table 2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d)
    for j in range(P):
        prog.reduction(_all(P), j, d, {r: send[r].shift(j * d) for r in range(P)}, recv[j], op)
    return prog


def allreduce_single(P, d, dtype="f32", op="sum"):
    """sum_j R(U, j, dp, op) -- moves d*p^2 data (Sec. 3.2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    for j in range(P):
        prog.reduction(_all(P), j, d * P, {r: send[r] for r in range(P)}, recv[j], op)
    return prog


def scatter(P, d, root=0, dtype="f32"):
    """sum_j R(i, j, d): single-leaf reductions, i.e. point-to-point (Table 2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d)
    for j in range(P):
        prog.reduction([root], j, d, {root: send[root].shift(j * d)}, recv[j])
    return prog


def gather(P, d, root=0, dtype="f32"):
    """sum_i M(i, j, d) (Table 2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d, d * P)
    for i in range(P):
        prog.multicast(i, [root], d, send[i], {root: recv[root].shift(i * d)})
    return prog


def alltoall(P, d, dtype="f32"):
    """sum_i sum_j M(i, j, d) (Table 2)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    for i in range(P):
        for j in range(P):
            prog.multicast(i, [j], d, send[i].shift(j * d), {j: recv[j].shift(i * d)})
    return prog


# ---- Listing 2 ------------------------------------------------------------------

def allreduce(P, d, dtype="f32", op="sum"):
    """Reduce-scatter, fence, in-place All-gather (Listing 2, Fig. 4)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    for j in range(P):
        prog.reduction(_all(P), j, d, {r: send[r].shift(j * d) for r in range(P)},
                       recv[j].shift(j * d), op)
    prog.fence()
    for i in range(P):
        others = [r for r in range(P) if r != i]
        prog.multicast(i, others, d, recv[i].shift(i * d), {r: recv[r].shift(i * d) for r in others})
    return prog


# ---- multi-step (Table 2, Multiple); "a . b" runs b, a fence, then a -------------

def broadcast_ag_scatter(P, d, root=0, dtype="f32"):
    """Broadcast = All-gather . Scatter."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    for j in range(P):
        prog.reduction([root], j, d, {root: send[root].shift(j * d)}, recv[j].shift(j * d))
    prog.fence()
    for i in range(P):
        others = [r for r in range(P) if r != i]
        prog.multicast(i, others, d, recv[i].shift(i * d), {r: recv[r].shift(i * d) for r in others})
    return prog


def reduce_gather_rs(P, d, root=0, dtype="f32"):
    """Reduce = Gather . Reduce-scatter (chunk j is reduced at rank j, then gathered)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    for j in range(P):
        prog.reduction(_all(P), j, d, {r: send[r].shift(j * d) for r in range(P)},
                       recv[j].shift(j * d))
    prog.fence()
    for j in range(P):
        if j == root:
            continue
        prog.multicast(j, [root], d, recv[j].shift(j * d), {root: recv[root].shift(j * d)})
    return prog


def allgather_bcast_gather(P, d, root=0, dtype="f32"):
    """All-gather = Broadcast . Gather."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d, d * P)
    for i in range(P):
        prog.multicast(i, [root], d, send[i], {root: recv[root].shift(i * d)})
    prog.fence()
    others = [r for r in range(P) if r != root]
    prog.multicast(root, others, d * P, recv[root], {r: recv[r] for r in others})
    return prog


def reducescatter_scatter_reduce(P, d, root=0, dtype="f32"):
    """Reduce-scatter = Scatter . Reduce (the full sum lands in the root's work buffer)."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d)
    work = prog.buffer(("work", root), d * P)
    prog.reduction(_all(P), root, d * P, {r: send[r] for r in range(P)}, work)
    prog.fence()
    for j in range(P):
        prog.reduction([root], j, d, {root: work.shift(j * d)}, recv[j])
    return prog


def allreduce_bcast_reduce(P, d, root=0, dtype="f32"):
    """All-reduce = Broadcast . Reduce."""
    prog = Program(P, dtype)
    send, recv = _bufs(prog, P, d * P, d * P)
    prog.reduction(_all(P), root, d * P, {r: send[r] for r in range(P)}, recv[root])
    prog.fence()
    others = [r for r in range(P) if r != root]
    prog.multicast(root, others, d * P, recv[root], {r: recv[r] for r in others})
    return prog


SEVEN = ("broadcast", "scatter", "gather", "allgather", "reducescatter", "allreduce", "alltoall")

BUILDERS = {
    "broadcast": broadcast, "reduce": reduce, "allgather": allgather,
    "reducescatter": reducescatter, "allreduce_single": allreduce_single,
    "scatter": scatter, "gather": gather, "alltoall": alltoall, "allreduce": allreduce,
    "broadcast_ag_scatter": broadcast_ag_scatter, "reduce_gather_rs": reduce_gather_rs,
    "allgather_bcast_gather": allgather_bcast_gather,
    "reducescatter_scatter_reduce": reducescatter_scatter_reduce,
    "allreduce_bcast_reduce": allreduce_bcast_reduce,
}
