"""Serving with continuous batching: requests of mixed kinds, sizes and
payloads arrive while others run, are admitted under a device-memory budget,
planned on host threads and launched in groups on two overlapping slots.
Each served result equals the oracle's result for the request alone, bit for
bit; batching and overlap actually happen; a tight budget admits requests in
order without deadlock."""
import time

import numpy as np
import pytest

from oracle import lowprec as LP
from oracle import programs as PR
from oracle import semantics as S
from synth import rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


KINDS = ["broadcast", "scatter", "gather", "allgather", "reducescatter", "allreduce", "alltoall"]
HIER = {8: [2, 4], 16: [4, 4]}
NPDT = {"f32": np.float32, "i32": np.int32, "bf16": np.uint16}


def _requests(n, seed):
    from paper_2408_05962_gb300.serving import Request
    g = rng(seed)
    out = []
    for i in range(n):
        P = int(g.choice([8, 16]))
        dt = str(g.choice(["f32", "i32", "bf16"]))
        d = int(g.integers(1, 300)) * 8
        es = 2 if dt == "bf16" else 4
        out.append(Request(kind=KINDS[i % len(KINDS)], P=P, hierarchy=HIER[P], bytes_per_rank=d * P * es,
                           dtype=dt, root=int(g.integers(0, P))))
    return out


def _expected(req, seed):
    prog = PR.BUILDERS[req.kind](req.P, req.d, dtype=req.dtype,
                                 **({"root": req.root} if req.kind in ("broadcast", "scatter", "gather") else {}))
    mem = prog.allocate()
    g = rng(seed)
    for r in range(req.P):
        v = mem[("send", r)]
        if req.dtype == "i32":
            v[...] = g.integers(-2**31, 2**31 - 1, size=v.shape, endpoint=True, dtype=np.int64)
        elif req.dtype == "bf16":
            v[...] = LP.f32_to_bf16(g.uniform(-1, 1, size=v.shape).astype(np.float32))
        else:
            v[...] = g.uniform(-1, 1, size=v.shape).astype(np.float32)
    sends = {r: mem[("send", r)].copy() for r in range(req.P)}
    S.run_program(prog, mem, req.hierarchy)
    return sends, {r: mem[("recv", r)].copy() for r in range(req.P)}


def _serve(reqs, budget, slots=2, max_batch=6, burst=6, gap_s=0.001):
    import torch
    from paper_2408_05962_gb300.serving import Server
    es = {"f32": 4, "i32": 4, "bf16": 2}
    # inputs and the oracle's answers, computed before serving
    data = []
    for k, req in enumerate(reqs):
        req.d = req.bytes_per_rank // es[req.dtype] // req.P
        data.append(_expected(req, 1000 + k))
    index = {id(req): k for k, req in enumerate(reqs)}
    results = {}

    def on_admit(req):
        sends, recvs = data[index[id(req)]]
        for r in range(req.P):
            off = req.send_ptrs[r] - srv.arena.base
            b = sends[r].view(np.uint8)
            srv.arena.buf[off:off + b.size].copy_(torch.from_numpy(b.copy()))
            off = req.recv_ptrs[r] - srv.arena.base
            srv.arena.buf[off:off + recvs[r].nbytes].zero_()
        torch.cuda.synchronize()

    def on_done(req):
        recvs = data[index[id(req)]][1]
        out = {}
        for r in range(req.P):
            off = req.recv_ptrs[r] - srv.arena.base
            out[r] = srv.arena.buf[off:off + recvs[r].nbytes].cpu().numpy()
        results[index[id(req)]] = out

    srv = Server(budget, slots=slots, max_batch=max_batch, planners=4, on_admit=on_admit, on_done=on_done)
    for k in range(0, len(reqs), burst):      # bursts of arrivals interleaved with progress
        for req in reqs[k:k + burst]:
            srv.submit(req)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < gap_s:
            srv.poll()
    srv.drain()
    srv.close()
    expected = {k: data[k][1] for k in range(len(reqs))}
    return srv, expected, results, index


def test_served_results_equal_alone():
    reqs = _requests(42, seed=5)
    srv, expected, results, index = _serve(reqs, budget=256 << 20)
    assert len(srv.done) == len(reqs) and not any(r.error for r in srv.done)
    for k, req in enumerate(reqs):
        for r in range(req.P):
            assert np.array_equal(results[k][r], expected[k][r].view(np.uint8)), (req.kind, req.dtype, req.P, r)
    assert srv.launches < len(reqs)               # requests were batched together


def test_concurrent_slots_results_equal_alone():
    """Each request launched alone, up to 8 at a time on separate streams."""
    reqs = _requests(28, seed=9)
    srv, expected, results, index = _serve(reqs, budget=256 << 20, slots=8, max_batch=1)
    assert len(srv.done) == len(reqs) and not any(r.error for r in srv.done)
    for k, req in enumerate(reqs):
        for r in range(req.P):
            assert np.array_equal(results[k][r], expected[k][r].view(np.uint8)), (req.kind, req.dtype, req.P, r)


def test_tight_budget_admits_in_order():
    reqs = _requests(10, seed=6)
    big = max(r.P * 2 * r.bytes_per_rank for r in reqs)
    srv, expected, results, index = _serve(reqs, budget=((big + 255) // 256) * 256 + 4096, slots=2, max_batch=4)
    assert len(srv.done) == len(reqs)
    admits = [r.t_admit for r in sorted(srv.done, key=lambda r: r.id)]
    assert admits == sorted(admits)               # FIFO admission
    for k, req in enumerate(reqs):
        for r in range(req.P):
            assert np.array_equal(results[k][r], expected[k][r].view(np.uint8))
