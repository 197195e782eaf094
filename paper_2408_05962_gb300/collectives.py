"""Standard collectives composed through the C ABI (paper Table 2, Listing 2).

Each ``compose_*`` registers primitives on a ``Comm`` for per-rank buffers
given as device addresses (``send[r]``, ``recv[r]``); ``d`` is the chunk
length in elements, so the largest per-rank buffer holds ``d * P`` elements
(Sec. 3.2).  Single-step forms follow Table 2 (Single); ``allreduce`` is the
Reduce-scatter / fence / in-place All-gather program of Listing 2; the
``*_via_*`` forms follow Table 2 (Multiple).  ``Buffers`` allocates the
per-rank buffers as rows of one device tensor.

Buffer lengths each collective expects (elements per rank):

===================  ==========  ==========
collective           send        recv
===================  ==========  ==========
broadcast, reduce    d*P         d*P
allgather, gather    d           d*P
reducescatter        d*P         d
scatter              d*P         d
allreduce(_single)   d*P         d*P
alltoall             d*P         d*P
===================  ==========  ==========
"""
from __future__ import annotations

from .hiccl import FP8_BLOCK_BYTES, Comm, nbytes

SEND_RECV = {
    "broadcast": (1, 1), "reduce": (1, 1), "allgather": (0, 1), "gather": (0, 1),
    "reducescatter": (1, 0), "scatter": (1, 0), "allreduce": (1, 1), "allreduce_single": (1, 1),
    "alltoall": (1, 1), "broadcast_via_ag_scatter": (1, 1), "reduce_via_gather_rs": (1, 1),
    "allgather_via_bcast_gather": (0, 1), "allreduce_via_bcast_reduce": (1, 1),
}


def buffer_lengths(kind: str, P: int, d: int) -> tuple:
    s, r = SEND_RECV[kind]
    return (d * P if s else d), (d * P if r else d)


class Buffers:
    """P send rows and P recv rows in two device tensors (row r = rank r).
    For FP8 payloads pass ``torch.uint8``: rows then hold the 144-byte blocks
    of ``ls`` / ``lr`` values."""

    def __init__(self, kind: str, P: int, d: int, torch_dtype, device="cuda", pad_elems: int = 0):
        import torch
        self.kind, self.P, self.d = kind, P, d
        ls, lr = buffer_lengths(kind, P, d)
        self.ls, self.lr = ls, lr
        if torch_dtype == torch.uint8:           # FP8 blocks
            self.send = torch.empty((P, ls // 128 * FP8_BLOCK_BYTES + pad_elems), dtype=torch_dtype, device=device)
            self.recv = torch.empty((P, lr // 128 * FP8_BLOCK_BYTES + pad_elems), dtype=torch_dtype, device=device)
        else:
            self.send = torch.empty((P, ls + pad_elems), dtype=torch_dtype, device=device)
            self.recv = torch.empty((P, lr + pad_elems), dtype=torch_dtype, device=device)

    def send_ptrs(self):
        return [int(self.send[r].data_ptr()) for r in range(self.P)]

    def recv_ptrs(self):
        return [int(self.recv[r].data_ptr()) for r in range(self.P)]


def _off(ptrs, k_elems, dtype):
    b = nbytes(dtype, k_elems)
    return [p + b if p else 0 for p in ptrs]


def _one(P, r, addr):
    v = [0] * P
    v[r] = addr
    return v


def compose(comm: Comm, kind: str, d: int, send, recv, root: int = 0) -> None:
    """Register collective ``kind`` over chunk length ``d`` on ``comm``."""
    P, e = comm.P, comm.dtype
    ranks = list(range(P))

    def at(base, k_elems):                        # address of element k of a buffer
        return base + nbytes(e, k_elems)

    if kind == "broadcast":                       # M(i, U, dp)
        comm.add_multicast(send, recv, d * P, root, ranks)
    elif kind == "reduce":                        # R(U, j, dp)
        comm.add_reduction(send, recv, d * P, ranks, root)
    elif kind == "allgather":                     # sum_i M(i, U, d)
        for i in ranks:
            comm.add_multicast(send, _off(recv, i * d, e), d, i, ranks)
    elif kind == "reducescatter":                 # sum_j R(U, j, d)
        for j in ranks:
            comm.add_reduction(_off(send, j * d, e), recv, d, ranks, j)
    elif kind == "allreduce_single":              # sum_j R(U, j, dp)
        for j in ranks:
            comm.add_reduction(send, recv, d * P, ranks, j)
    elif kind == "scatter":                       # sum_j R(i, j, d)
        for j in ranks:
            comm.add_reduction(_one(P, root, at(send[root], j * d)), recv, d, [root], j)
    elif kind == "gather":                        # sum_i M(i, j, d)
        for i in ranks:
            comm.add_multicast(send, _one(P, root, at(recv[root], i * d)), d, i, [root])
    elif kind == "alltoall":                      # sum_i sum_j M(i, j, d)
        for i in ranks:
            for j in ranks:
                comm.add_multicast(_one(P, i, at(send[i], j * d)), _one(P, j, at(recv[j], i * d)),
                                   d, i, [j])
    elif kind == "allreduce":                     # Listing 2
        for j in ranks:
            comm.add_reduction(_off(send, j * d, e), _one(P, j, at(recv[j], j * d)), d, ranks, j)
        comm.add_fence()
        for i in ranks:
            others = [r for r in ranks if r != i]
            comm.add_multicast(_off(recv, i * d, e), _off(recv, i * d, e), d, i, others)
    elif kind == "broadcast_via_ag_scatter":      # All-gather . Scatter
        for j in ranks:
            comm.add_reduction(_one(P, root, at(send[root], j * d)), _one(P, j, at(recv[j], j * d)),
                               d, [root], j)
        comm.add_fence()
        for i in ranks:
            others = [r for r in ranks if r != i]
            comm.add_multicast(_off(recv, i * d, e), _off(recv, i * d, e), d, i, others)
    elif kind == "reduce_via_gather_rs":          # Gather . Reduce-scatter
        for j in ranks:
            comm.add_reduction(_off(send, j * d, e), _one(P, j, at(recv[j], j * d)), d, ranks, j)
        comm.add_fence()
        for j in ranks:
            if j != root:
                comm.add_multicast(_one(P, j, at(recv[j], j * d)), _one(P, root, at(recv[root], j * d)),
                                   d, j, [root])
    elif kind == "allgather_via_bcast_gather":    # Broadcast . Gather
        for i in ranks:
            comm.add_multicast(send, _one(P, root, at(recv[root], i * d)), d, i, [root])
        comm.add_fence()
        others = [r for r in ranks if r != root]
        comm.add_multicast(recv, recv, d * P, root, others)
    elif kind == "allreduce_via_bcast_reduce":    # Broadcast . Reduce
        comm.add_reduction(send, recv, d * P, ranks, root)
        comm.add_fence()
        others = [r for r in ranks if r != root]
        comm.add_multicast(recv, recv, d * P, root, others)
    else:
        raise ValueError(f"unknown collective {kind}")
