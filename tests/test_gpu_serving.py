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


def _serve(reqs, budget, slots=2, max_batch=6, burst=6, gap_s=0.001, **server_kw):
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

    srv = Server(budget, slots=slots, max_batch=max_batch, planners=4, on_admit=on_admit, on_done=on_done,
                 **server_kw)
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
    srv, expected, results, index = _serve(reqs, budget=((big + 255) // 256) * 256 + 4096, slots=2, max_batch=4,
                                           bypass_frac=0)
    assert len(srv.done) == len(reqs)
    admits = [r.t_admit for r in sorted(srv.done, key=lambda r: r.id)]
    assert admits == sorted(admits)               # FIFO admission
    for k, req in enumerate(reqs):
        for r in range(req.P):
            assert np.array_equal(results[k][r], expected[k][r].view(np.uint8))


def test_tight_budget_small_requests_pass_the_waiting_head():
    """The same tight budget, launched one request per slot, with small
    requests allowed to pass a head that waits for memory: every result is
    still the one it has alone."""
    reqs = _requests(16, seed=6)
    big = max(r.P * 2 * r.bytes_per_rank for r in reqs)
    budget = 2 * ((big + 255) // 256) * 256 + (1 << 20)     # room for the largest request's tables too
    srv, expected, results, index = _serve(reqs, budget=budget, slots=4, max_batch=1, bypass_frac=1 / 8,
                                           bypass_cap_frac=1 / 4)
    assert len(srv.done) == len(reqs) and not any(r.error for r in srv.done) and srv.bypass_held == 0
    for k, req in enumerate(reqs):
        for r in range(req.P):
            assert np.array_equal(results[k][r], expected[k][r].view(np.uint8)), (req.kind, req.dtype, req.P, r)


def test_memoized_plans_equal_fresh(monkeypatch):
    """Six shapes, each requested four times with new inputs: every shape is
    factorized once (later requests reuse the resident table and buffers),
    and every result equals the oracle's for the request alone."""
    from paper_2408_05962_gb300 import hiccl as H
    planned = []
    orig = H.Comm.plan

    def counting_plan(self, *a, **k):
        planned.append(1)
        return orig(self, *a, **k)

    monkeypatch.setattr(H.Comm, "plan", counting_plan)
    shapes = _requests(6, seed=21)
    reqs = []
    for rep in range(4):
        for s in shapes:
            from paper_2408_05962_gb300.serving import Request
            reqs.append(Request(kind=s.kind, P=s.P, hierarchy=s.hierarchy, bytes_per_rank=s.bytes_per_rank,
                                dtype=s.dtype, root=s.root))
    srv, expected, results, index = _serve(reqs, budget=256 << 20, slots=1, max_batch=1, burst=1, gap_s=0.002)
    assert len(srv.done) == len(reqs) and not any(r.error for r in srv.done)
    assert len(planned) == len(shapes) and srv.plan_cache_hits == len(reqs) - len(shapes)
    assert sum(r.cached for r in srv.done) == len(reqs) - len(shapes)
    for k, req in enumerate(reqs):
        for r in range(req.P):
            assert np.array_equal(results[k][r], expected[k][r].view(np.uint8)), (k, req.kind, req.dtype, r)


def test_slots_overlap_on_the_device():
    """Two requests launched on two slots run at the same time: the executor
    trace (global timestamps of every work item) of one launch overlaps the
    other's.  Large work items keep each launch on a part of the GPU."""
    from paper_2408_05962_gb300 import hiccl as H
    from paper_2408_05962_gb300.serving import Request, Server
    spans = {}

    def on_done(req):
        t = np.array(req.comm.trace(), dtype=np.uint64).reshape(-1, 6)
        spans[req.id] = (int(t[:, 0].min()), int(t[:, 3].max()))

    srv = Server(8 << 30, slots=2, max_batch=1, planners=2, on_done=on_done, cache_entries=0,
                 comm_options={H.OPT_TRACE: 1, H.OPT_ITEM_BYTES: 8 << 20})
    for _ in range(2):
        srv.submit(Request(kind="allgather", P=8, hierarchy=[2, 4], bytes_per_rank=256 << 20, dtype="f32"))
    srv.drain()
    srv.close()
    assert len(spans) == 2 and not any(r.error for r in srv.done)
    (a0, a1), (b0, b1) = spans.values()
    assert max(a0, b0) < min(a1, b1), spans       # the two intervals intersect


def _expected_at(kind, P, d, root, xs_at, r, k, h, dtype):
    """Expected value of receive element k of rank r, from the inputs:
    xs_at(i, m) is element m of rank i's send buffer (Table 2)."""
    if kind == "broadcast":
        return xs_at(root, k)
    if kind == "scatter":
        return xs_at(root, r * d + k)
    if kind == "gather":
        return xs_at(k // d, k % d)
    if kind == "allgather":
        return xs_at(k // d, k % d)
    if kind == "alltoall":
        return xs_at(k // d, r * d + k % d)
    m = r * d + k if kind == "reducescatter" else k
    fold_dt = None if dtype == "f32" else dtype
    return S.nested_fold({i: np.asarray([xs_at(i, m)]) for i in range(P)}, h, fold_dt)[0]


@pytest.mark.parametrize("shapes", [0, 6])
def test_served_full_size_sampled(shapes):
    """Config 5 at full size: requests drawn from the serving distribution
    (the seven collectives, P in {8, 16, 64}, 1 KiB .. 256 MiB per rank,
    fp32 / bf16 / int32; with ``shapes``, drawn from that many recurring
    shapes so memoized plans serve the repeats) under a 64 GB budget on eight
    launch slots.  Every result is checked on sampled elements, each computed
    by the oracle from the inputs read back from the device."""
    import torch
    from paper_2408_05962_gb300.serving import Request, Server
    from synth import poisson_requests
    descs = poisson_requests(2000.0, 0.02, seed=5, shapes=shapes)[:24]
    TD = {"f32": torch.float32, "bf16": torch.bfloat16, "i32": torch.int32}
    NV = {"f32": np.float32, "bf16": np.uint16, "i32": np.int32}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    checked = []

    def rows(req, ptrs, n):
        es = 2 if req.dtype == "bf16" else 4
        off = [p - srv.arena.base for p in ptrs]
        return [srv.arena.buf[o:o + n * es].view(TD[req.dtype]) for o in off]

    def on_admit(req):
        from paper_2408_05962_gb300.collectives import buffer_lengths
        ls, lr = buffer_lengths(req.kind, req.P, req.d)
        for t in rows(req, req.send_ptrs, ls):
            if req.dtype == "i32":
                t.copy_(torch.randint(-2**31, 2**31 - 1, t.shape, generator=gen, device="cuda", dtype=torch.int32))
            else:
                t.copy_(torch.empty(t.shape, device="cuda").uniform_(-1, 1, generator=gen))
        for t in rows(req, req.recv_ptrs, lr):
            t.view(torch.uint8).fill_(0x5A)
        torch.cuda.synchronize()

    def on_done(req):
        from paper_2408_05962_gb300.collectives import buffer_lengths
        ls, lr = buffer_lengths(req.kind, req.P, req.d)
        g = np.random.Generator(np.random.PCG64(req.id))
        send = rows(req, req.send_ptrs, ls)
        recv = rows(req, req.recv_ptrs, lr)
        targets = [req.root] if req.kind == "gather" else list(range(req.P))
        cache = {}

        def xs_at(i, m):
            if (i, m) not in cache:
                cache[(i, m)] = send[i][m:m + 1].cpu().view(
                    torch.int16 if req.dtype == "bf16" else TD[req.dtype]).numpy().view(NV[req.dtype])[0]
            return cache[(i, m)]
        for r in targets:
            for k in sorted(set(g.integers(0, lr, 6).tolist()) | {0, lr - 1}):
                got = recv[r][k:k + 1].cpu().view(torch.int16 if req.dtype == "bf16" else TD[req.dtype]).numpy()
                got = got.view(NV[req.dtype])[0]
                exp = _expected_at(req.kind, req.P, req.d, req.root, xs_at, r, k, req.hierarchy, req.dtype)
                a = np.asarray([got], dtype=NV[req.dtype]).view(np.uint8)
                b = np.asarray([exp], dtype=NV[req.dtype]).view(np.uint8)
                assert np.array_equal(a, b), (req.kind, req.P, req.bytes_per_rank, req.dtype, r, k)
        checked.append(req.id)

    srv = Server(64 << 30, slots=8, max_batch=1, planners=4, on_admit=on_admit, on_done=on_done)
    for wave in (descs[:12], descs[12:]):      # the second wave finds the first wave's plans idle
        for dsc in wave:
            srv.submit(Request(kind=dsc["kind"], P=dsc["P"], hierarchy=dsc["hierarchy"],
                               bytes_per_rank=dsc["bytes_per_rank"], dtype=dsc["dtype"]))
        srv.drain()
    srv.close()
    assert not any(r.error for r in srv.done), [r.error for r in srv.done if r.error]
    assert len(checked) == len(descs)
    assert max(d["bytes_per_rank"] for d in descs) > (16 << 20)      # the large end of the range is served
    if shapes:
        assert srv.plan_cache_hits > 0
