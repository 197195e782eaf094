"""Admission order of the serving loop, on the host (a server on the CPU
admits, plans and memoizes but launches nothing).  Requests are admitted in
arrival order; while the head waits for memory, small requests behind it may
pass it -- each at most ``bypass_frac`` of the budget, together at most
``bypass_cap_frac`` -- but only while the head could not fit even without
them, so the head waits at most for those short requests to drain."""
import time

from paper_2408_05962_gb300.serving import Request, Server

from .test_serving_cache import _Pool

MiB = 1 << 20


def _ag(need_mib: float) -> Request:
    """An All-gather over 8 ranks whose buffers take ``need_mib`` MiB in all
    (d values sent and p*d received on each of the 8 ranks; its plan needs no
    relay buffers, so its device tables are small next to the buffers)."""
    return Request(kind="allgather", P=8, hierarchy=[2, 4], bytes_per_rank=int(need_mib * MiB) // 9 // 128 * 128,
                   dtype="f32")


def _advance(srv):
    """Admit, plan and 'upload' (on the host); returns the requests that
    became ready (they stay running until finished by the test)."""
    with srv.lock:
        srv._admit()
    srv.planning = srv._collect(srv.planning, srv.to_upload.append)
    srv._reserve_uploads()
    srv.uploading = srv._collect(srv.uploading, srv._on_uploaded)
    out = list(srv.ready)
    srv.ready.clear()
    return out


def _server(budget_mib, **kw):
    srv = Server(budget_mib * MiB, slots=2, device="cpu", **kw)
    srv.pool = _Pool()
    return srv


def test_small_requests_pass_a_waiting_head_within_the_caps():
    srv = _server(1024, bypass_frac=1 / 16, bypass_cap_frac=1 / 8, cache_entries=0)
    hold = _ag(640)
    srv.submit(hold)
    assert _advance(srv) == [hold]                    # running: holds 640 MiB
    head, small1, big, small2, small3 = _ag(512), _ag(48), _ag(200), _ag(48), _ag(48)
    for r in (head, small1, big, small2, small3):
        srv.submit(r)
    ready = _advance(srv)
    # 64 MiB each at most, 128 MiB together: two small requests pass, the
    # large one behind the head does not, the third small one exceeds the cap
    assert ready == [small1, small2]
    assert list(srv.waiting) == [head, big, small3]
    assert srv.bypassed == 2 and srv.bypass_held >= 2 * 48 * MiB
    srv._finish(small1, time.perf_counter())          # a passed request drains: the cap has room again
    assert _advance(srv) == [small3]
    srv._finish(hold, time.perf_counter())            # the head fits now; the large one follows it in order
    assert _advance(srv) == [head, big] and not srv.waiting
    for r in (head, big, small2, small3):
        srv._finish(r, time.perf_counter())
    srv.close()
    assert srv.device_bytes() == 0 and srv.bypass_held == 0


def test_no_request_passes_a_head_that_fits_without_the_passed_ones():
    srv = _server(1024, bypass_frac=1 / 8, bypass_cap_frac=1 / 4, cache_entries=0)
    mid, hold = _ag(300), _ag(500)
    srv.submit(mid)
    srv.submit(hold)
    assert _advance(srv) == [mid, hold]               # 800 MiB held
    head = _ag(600)
    srv.submit(head)
    smalls = [_ag(100) for _ in range(2)]
    for r in smalls:
        srv.submit(r)
    assert _advance(srv) == smalls                    # 1000 MiB of buffers held; the head needs 600
    srv._finish(hold, time.perf_counter())            # 500 MiB: the head would fit without the passed ones
    late = _ag(16)
    srv.submit(late)
    assert _advance(srv) == []                        # so nothing passes it any more
    assert list(srv.waiting) == [head, late]
    srv._finish(smalls[0], time.perf_counter())
    srv._finish(smalls[1], time.perf_counter())
    assert _advance(srv) == [head, late]              # the passed requests drained: the head goes first
    for r in (mid, head, late):
        srv._finish(r, time.perf_counter())
    srv.close()
    assert srv.device_bytes() == 0


def test_bypass_off_is_first_in_first_out():
    srv = _server(1024, bypass_frac=0, cache_entries=0)
    hold = _ag(640)
    srv.submit(hold)
    assert _advance(srv) == [hold]
    head, small = _ag(512), _ag(16)
    srv.submit(head)
    srv.submit(small)
    assert _advance(srv) == [] and list(srv.waiting) == [head, small]
    srv._finish(hold, time.perf_counter())
    assert _advance(srv) == [head, small]
    srv._finish(head, time.perf_counter())
    srv._finish(small, time.perf_counter())
    srv.close()
    assert srv.device_bytes() == 0


def test_evicted_plans_are_destroyed_off_the_polling_loop(monkeypatch):
    destroyed = []
    srv = _server(1024, cache_entries=2)
    reqs = [_ag(8 + k) for k in range(5)]             # five shapes, two idle plans kept
    for r in reqs:
        srv.submit(r)
        assert _advance(srv) == [r]
        orig = r.comm.destroy
        r.comm.destroy = (lambda o=orig, c=r.comm: (destroyed.append(c), o())[1])
        srv._finish(r, time.perf_counter())
    srv.reaper.shutdown()                             # wait for the reaper thread
    assert srv.evicted == 3 and len(destroyed) == 3 and len(srv.cache) == 2


def test_idle_plans_stay_when_evicting_them_would_not_make_room():
    srv = _server(1024, bypass_frac=1 / 16, bypass_cap_frac=1 / 8)
    small = _ag(60)
    srv.submit(small)
    assert _advance(srv) == [small]
    srv._finish(small, time.perf_counter())           # idle, memoized: about 60 MiB
    assert len(srv.cache) == 1 and srv.cache.nbytes > 60 * MiB - (1 << 20)
    hold = _ag(640)
    srv.submit(hold)
    assert _advance(srv) == [hold]                    # running
    head = _ag(512)
    srv.submit(head)
    assert _advance(srv) == [] and list(srv.waiting) == [head]
    assert len(srv.cache) == 1 and srv.evicted == 0   # 640 + 512 > 1024 even without it: kept
    again = _ag(60)                                   # the same shape passes the head on its resident plan
    srv.submit(again)
    assert _advance(srv) == [again] and again.cached and again.send_ptrs == small.send_ptrs
    assert srv.bypass_held > 0 and srv.cache.nbytes == 0
    srv._finish(again, time.perf_counter())
    assert srv.bypass_held == 0 and len(srv.cache) == 1
    srv._finish(hold, time.perf_counter())            # now evicting the idle plans makes room for the head
    assert _advance(srv) == [head] and srv.evicted >= 1
    srv._finish(head, time.perf_counter())
    srv.close()
    assert srv.device_bytes() == 0 and srv.cache.nbytes == 0
