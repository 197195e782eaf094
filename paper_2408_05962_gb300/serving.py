"""Serving loop with continuous batching over the C ABI.

Requests (a collective kind, P virtual ranks, hierarchy, per-rank size,
payload) arrive at any time.  The server

* admits a request when its buffers fit in the device-memory budget (one
  device arena, first-fit; FIFO, so a large request is never starved by later
  small ones), keeping buffers and step tables on the device;
* plans admitted requests on a pool of host threads (the native factorizer
  and the table upload; ctypes releases the GIL during the calls);
* launches planned requests on whichever of its ``slots`` CUDA streams is
  free -- each request alone (``group_max`` 1), or up to ``group_max``
  waiting requests together as one grouped persistent launch
  (``hiccl_group``); requests that arrive while others run take the next free
  slot, and launches on different slots overlap on the device;
* retires a launch when its event completes, freeing its memory and recording
  each request's latency (completion observed minus arrival).

Planning uses stripe 1 and pipeline 1 for every request: on one GPU every
level is HBM, and the cost of planning is paid per request.
"""
from __future__ import annotations

import bisect
import threading
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

from . import hiccl as H
from .collectives import buffer_lengths

_ESIZE_TORCH = {"f32": 4, "i32": 4, "bf16": 2}


class DeviceArena:
    """First-fit sub-allocator over one device tensor of ``nbytes``."""

    def __init__(self, nbytes: int, device, align: int = 256):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.base = int(self.buf.data_ptr())
        self.size = nbytes
        self.align = align
        self.free_list = [(0, nbytes)]          # sorted (offset, size)
        self.used = 0

    def alloc(self, nbytes: int):
        n = (nbytes + self.align - 1) // self.align * self.align
        for k, (off, size) in enumerate(self.free_list):
            if size >= n:
                if size == n:
                    self.free_list.pop(k)
                else:
                    self.free_list[k] = (off + n, size - n)
                self.used += n
                return off, n
        return None

    def free(self, off: int, n: int):
        k = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(k, (off, n))
        self.used -= n
        # merge with neighbours
        if k + 1 < len(self.free_list) and off + n == self.free_list[k + 1][0]:
            self.free_list[k] = (off, n + self.free_list[k + 1][1])
            self.free_list.pop(k + 1)
        if k > 0 and self.free_list[k - 1][0] + self.free_list[k - 1][1] == self.free_list[k][0]:
            self.free_list[k - 1] = (self.free_list[k - 1][0], self.free_list[k - 1][1] + self.free_list[k][1])
            self.free_list.pop(k)


@dataclass
class Request:
    kind: str
    P: int
    hierarchy: list
    bytes_per_rank: int          # largest per-rank buffer (p*d values)
    dtype: str = "f32"
    root: int = 0
    t_arrival: float = 0.0
    # filled by the server
    id: int = -1
    d: int = 0
    send_ptrs: list = field(default_factory=list)
    recv_ptrs: list = field(default_factory=list)
    region: tuple = ()
    comm: object = None
    hbm_bytes: int = 0
    t_admit: float = 0.0
    t_launch: float = 0.0
    t_done: float = 0.0
    error: str = ""


class Server:
    def __init__(self, budget_bytes: int, slots: int = 8, max_batch: int = 1, planners: int = 4,
                 device="cuda", on_admit=None, on_done=None):
        import torch
        self.device = torch.device(device)
        self.arena = DeviceArena(budget_bytes, self.device)
        self.slots = [{"stream": torch.cuda.Stream(self.device), "event": None, "group": None, "reqs": []}
                      for _ in range(slots)]
        self.max_batch = max_batch
        self.pool = ThreadPoolExecutor(max_workers=planners)
        self.waiting: deque = deque()     # submitted, not admitted
        self.planning: list = []          # (future, request)
        self.ready: deque = deque()       # planned, not launched
        self.done: list = []
        self.on_admit, self.on_done = on_admit, on_done
        self.lock = threading.Lock()
        self.next_id = 0
        self.launches = 0

    # -- requests ---------------------------------------------------------------
    def submit(self, req: Request) -> int:
        with self.lock:
            req.id = self.next_id
            self.next_id += 1
            if not req.t_arrival:
                req.t_arrival = time.perf_counter()
            self.waiting.append(req)
        return req.id

    def _layout(self, req: Request):
        es = _ESIZE_TORCH[req.dtype]
        req.d = req.bytes_per_rank // es // req.P
        ls, lr = buffer_lengths(req.kind, req.P, req.d)
        return ls * es, lr * es

    def _admit(self):
        while self.waiting:
            req = self.waiting[0]
            sb, rb = self._layout(req)
            got = self.arena.alloc(req.P * (sb + rb))
            if got is None:
                return                     # FIFO: wait until memory frees
            self.waiting.popleft()
            off, n = got
            req.region = (off, n)
            base = self.arena.base + off
            req.send_ptrs = [base + r * sb for r in range(req.P)]
            req.recv_ptrs = [base + req.P * sb + r * rb for r in range(req.P)]
            req.t_admit = time.perf_counter()
            if self.on_admit:
                self.on_admit(req)
            self.planning.append((self.pool.submit(self._plan, req, self.max_batch == 1), req))

    @staticmethod
    def _plan(req: Request, upload: bool):
        comm = H.Comm(req.P, req.dtype)
        comm.add_collective(req.kind, req.d, req.send_ptrs, req.recv_ptrs, req.root)
        if upload:     # launched alone: its own table, uploaded here on the planner thread
            comm.init(req.hierarchy, 1, 1)
        else:          # joins a group, which uploads one combined table
            comm.plan(req.hierarchy, 1, 1)
        rd, wr = comm.hbm_bytes()
        req.hbm_bytes = rd + wr
        req.comm = comm

    def _collect_planned(self):
        keep = []
        for fut, req in self.planning:
            if fut.done():
                err = fut.exception()
                if err is not None:
                    req.error = str(err)
                    self._finish(req, time.perf_counter())
                else:
                    self.ready.append(req)
            else:
                keep.append((fut, req))
        self.planning = keep

    def _launch(self):
        for sl in self.slots:
            if not self.ready:
                return
            if sl["event"] is not None:
                continue
            batch = []
            while self.ready and len(batch) < self.max_batch:
                batch.append(self.ready.popleft())
            grp = batch[0].comm if len(batch) == 1 and self.max_batch == 1 else H.Comm.group([r.comm for r in batch])
            now = time.perf_counter()
            for r in batch:
                r.t_launch = now
            grp.start(sl["stream"])
            import torch
            ev = torch.cuda.Event()
            ev.record(sl["stream"])
            sl["event"], sl["group"], sl["reqs"] = ev, grp, batch
            self.launches += 1

    def _retire(self):
        for sl in self.slots:
            ev = sl["event"]
            if ev is None or not ev.query():
                continue
            now = time.perf_counter()
            sl["group"].wait()
            if not (len(sl["reqs"]) == 1 and sl["group"] is sl["reqs"][0].comm):
                sl["group"].destroy()
            for r in sl["reqs"]:
                self._finish(r, now)
            sl["event"], sl["group"], sl["reqs"] = None, None, []

    def _finish(self, req: Request, now: float):
        req.t_done = now
        if self.on_done:
            self.on_done(req)
        if req.comm is not None:
            req.comm.destroy()
            req.comm = None
        if req.region:
            self.arena.free(*req.region)
            req.region = ()
        self.done.append(req)

    def poll(self):
        """One round of progress: retire finished launches, admit and plan
        waiting requests, launch planned ones on free slots."""
        self._retire()
        with self.lock:
            self._admit()
        self._collect_planned()
        self._launch()

    def busy(self) -> bool:
        return bool(self.waiting or self.planning or self.ready or any(s["event"] for s in self.slots))

    def drain(self, timeout_s: float = 600.0):
        t0 = time.perf_counter()
        while self.busy():
            self.poll()
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(0)

    def close(self):
        self.drain()
        self.pool.shutdown()


def latency_stats(done: list) -> dict:
    lat = sorted((r.t_done - r.t_arrival) for r in done if not r.error)
    if not lat:
        return {"n": 0}

    def pct(q):
        return lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))]
    return {"n": len(lat), "p50_ms": pct(0.5) * 1e3, "p99_ms": pct(0.99) * 1e3, "max_ms": lat[-1] * 1e3}
