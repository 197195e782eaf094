"""Memoized plans of the serving loop (Sec. 5.2: a schedule is optimized
once and reused), on the host: the LRU cache of idle plans, and a server on
the CPU (which admits, plans and memoizes but launches nothing) showing that
a request whose shape was served before is admitted straight to the launch
queue with its predecessor's communicator and buffers -- no factorization,
no upload -- while the budget counts buffers and device tables together and
evicts idle plans when it needs their memory."""
import concurrent.futures
import time

import pytest

from paper_2408_05962_gb300 import hiccl as H
from paper_2408_05962_gb300.serving import PlanCache, Request, Server


def test_plan_cache_lru():
    c = PlanCache(max_entries=3)
    assert c.take("a") is None
    assert c.put("a", 1) == [] and c.put("b", 2) == [] and c.put("a", 3) == []
    assert len(c) == 3
    assert c.take("a") == 1                            # oldest entry of the shape
    assert c.put("c", 4) == [] and c.put("d", 5) == [2]   # the cap pushes out the oldest overall
    assert c.evict_lru() == 3 and c.evict_lru() == 4 and c.evict_lru() == 5 and c.evict_lru() is None
    assert len(c) == 0 and c.by_shape == {}


class _Pool:
    """Runs host planning at once; records uploads without running them
    (no GPU here)."""

    def __init__(self):
        self.calls = []

    def submit(self, fn, *args):
        self.calls.append(fn.__name__)
        fut = concurrent.futures.Future()
        if fn.__name__ == "_plan":
            fn(*args)
        fut.set_result(None)
        return fut

    def shutdown(self):
        pass


def _step(srv):
    """One round of the server's host logic, then 'complete' everything ready."""
    with srv.lock:
        srv._admit()
    srv.planning = srv._collect(srv.planning, srv.to_upload.append)
    srv._reserve_uploads()
    srv.uploading = srv._collect(srv.uploading, srv.ready.append)
    out = list(srv.ready)
    srv.ready.clear()
    for r in out:
        srv._finish(r, time.perf_counter())
    return out


def test_cache_hit_performs_no_factorization(monkeypatch):
    planned = []
    orig = H.Comm.plan

    def counting_plan(self, *a, **k):
        planned.append(self)
        return orig(self, *a, **k)

    monkeypatch.setattr(H.Comm, "plan", counting_plan)
    srv = Server(64 << 20, slots=2, device="cpu")
    srv.pool = _Pool()
    a = Request(kind="allreduce", P=8, hierarchy=[2, 4], bytes_per_rank=8 * 1024 * 4, dtype="f32")
    srv.submit(a)
    assert _step(srv) == [a] and not a.cached
    assert len(planned) == 1 and srv.pool.calls == ["_plan", "_upload"]
    assert srv.dev_bytes == a.dev_bytes > 0 and len(srv.cache) == 1
    used = srv.device_bytes()
    b = Request(kind="allreduce", P=8, hierarchy=[2, 4], bytes_per_rank=8 * 1024 * 4, dtype="f32")
    srv.submit(b)
    assert _step(srv) == [b] and b.cached
    assert len(planned) == 1 and srv.pool.calls == ["_plan", "_upload"]     # no planning, no upload
    assert b.send_ptrs == a.send_ptrs and b.recv_ptrs == a.recv_ptrs        # the resident buffers
    assert srv.device_bytes() == used and srv.plan_cache_hits == 1 and srv.plan_cache_misses == 1
    # another shape (another root) is planned anew
    c = Request(kind="allreduce", P=8, hierarchy=[2, 4], bytes_per_rank=8 * 1024 * 4, dtype="f32", root=3)
    srv.submit(c)
    assert _step(srv) == [c] and not c.cached and len(planned) == 2 and srv.plan_cache_misses == 2
    srv.close()
    assert srv.device_bytes() == 0 and srv.arena.used == 0


def test_budget_evicts_idle_plans():
    srv = Server(8 << 20, slots=2, device="cpu")
    srv.pool = _Pool()
    reqs = [Request(kind="allgather", P=8, hierarchy=[2, 4], bytes_per_rank=(96 + 32 * k) * 1024, dtype="f32")
            for k in range(12)]
    for r in reqs:                       # one at a time: each finishes before the next arrives
        srv.submit(r)
        assert _step(srv) == [r]
        assert srv.device_bytes() <= srv.budget
    assert len(srv.cache) < len(reqs)    # older idle plans were evicted for the newer ones
    assert all(not r.cached and not r.error for r in reqs)
    srv.close()
    assert srv.device_bytes() == 0


def test_request_beyond_budget_is_refused():
    srv = Server(1 << 20, slots=1, device="cpu")
    srv.pool = _Pool()
    r = Request(kind="allreduce", P=8, hierarchy=[2, 4], bytes_per_rank=1 << 20, dtype="f32")
    srv.submit(r)
    for _ in range(3):
        _step(srv)
    assert srv.waiting and srv.waiting[0] is r        # its buffers never fit: it waits, FIFO
    assert srv.plan_cache_misses == 0                  # retries of the waiting request count nothing


def test_planned_request_waits_for_memory_held_by_others():
    """A planned request whose tables do not fit next to buffers that other
    admitted requests hold waits for them (it is not refused while they can
    still move), and the requests behind it that fit are uploaded."""
    srv = Server(64 << 20, slots=2, device="cpu")
    srv.pool = _Pool()
    a = Request(kind="allreduce", P=8, hierarchy=[2, 4], bytes_per_rank=8 * 1024 * 4, dtype="f32")
    b = Request(kind="allgather", P=8, hierarchy=[2, 4], bytes_per_rank=8 * 1024 * 4, dtype="f32")
    srv.submit(a)
    srv.submit(b)
    with srv.lock:
        srv._admit()
    srv.planning = srv._collect(srv.planning, srv.to_upload.append)
    assert list(srv.to_upload) == [a, b]
    srv.budget = srv.arena.used + b.dev_bytes            # room for b's tables only
    srv._reserve_uploads()
    assert [r for _, r in srv.uploading] == [b] and list(srv.to_upload) == [a] and not a.error
    srv.uploading = srv._collect(srv.uploading, srv.ready.append)
    srv._reserve_uploads()                               # b is ready and will free memory: a waits
    assert list(srv.to_upload) == [a] and not a.error
    srv._finish(srv.ready.popleft(), time.perf_counter())   # b done; its plan is kept idle
    srv._reserve_uploads()                               # evicting b's idle plan makes room for a
    assert [r for _, r in srv.uploading] == [a] and not a.error
