"""Serving loop with continuous batching over the C ABI.

Requests (a collective kind, P virtual ranks, hierarchy, per-rank size,
payload) arrive at any time.  The server

* admits a request when its buffers fit in the device-memory budget (one
  device arena, first-fit), keeping buffers and step tables on the device.
  Admission is in arrival order, with one exception: while the request at
  the head waits for memory, small requests behind it (buffers of at most
  ``bypass_frac`` of the budget each, together at most ``bypass_cap_frac``)
  may pass it, but only as long as the head could not fit even if every
  request that passed it were gone -- so the head waits at most for those
  short requests to drain, and a large request is never starved by later
  small ones;
* memoizes plans (Sec. 5.2: a schedule is optimized once and reused): a
  finished request leaves its communicator -- step table, counters, relay
  buffers -- and its arena buffers resident, keyed by the request's shape; a
  later request of the same shape takes them over with no factorization, no
  upload and no allocation.  Idle entries are evicted, least recently used
  first, when the budget needs their memory -- and only when evicting them
  makes room: a request that waits for memory held by running requests
  leaves the idle plans in place;
* plans the other admitted requests on a pool of host threads (the native
  factorizer), counts each plan's device footprint (table, counters, relay
  buffers) against the budget together with the buffers, then uploads it on
  the pool;
* launches planned requests on whichever of its ``slots`` CUDA streams is
  free -- each request alone (``group_max`` 1), or up to ``group_max``
  waiting requests together as one grouped persistent launch
  (``hiccl_group``, whose combined table is built on the planner threads);
  requests that arrive while others run take the next free slot, and
  launches on different slots overlap on the device;
* retires a launch when its event completes, recording each request's
  latency (completion observed minus arrival).

Planning uses stripe 1 and pipeline 1 for every request: on one GPU every
level is HBM.  The polling loop yields the interpreter lock once per round
(and, with ``idle_s`` > 0, sleeps that long after a round that changed
nothing), so the planner threads, whose Python parts need the lock between
native calls, run as soon as their native calls return.
"""
from __future__ import annotations

import bisect
import threading
import time
from collections import OrderedDict, deque
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


class PlanCache:
    """Idle memoized plans by request shape, least recently used first.

    An entry is whatever the server stores for a finished request (its
    communicator, arena region, buffer pointers, footprint); ``take`` hands an
    idle entry of a shape to a new request (the oldest of that shape), ``put``
    returns one after use, ``evict_lru`` removes the least recently used idle
    entry of any shape.  Every operation is O(1).  ``nbytes`` is the device
    memory the idle entries hold (each entry's weight as ``put`` was given
    it).  ``hits`` and ``misses`` count admitted requests (the server updates
    them)."""

    def __init__(self, max_entries: int = 4096):
        self.max_entries = max_entries
        self.by_shape = {}             # shape -> deque of serials, oldest first
        self.lru = OrderedDict()       # serial -> (shape, entry, nbytes), oldest first
        self.serial = 0
        self.nbytes = 0
        self.hits = 0
        self.misses = 0

    def __len__(self):
        return len(self.lru)

    def take(self, shape):
        q = self.by_shape.get(shape)
        if not q:
            return None
        _, entry, nb = self.lru.pop(q.popleft())
        self.nbytes -= nb
        if not q:
            del self.by_shape[shape]
        return entry

    def put(self, shape, entry, nbytes: int = 0):
        """Store an idle entry; returns the entries pushed out by the size cap."""
        self.serial += 1
        self.by_shape.setdefault(shape, deque()).append(self.serial)
        self.lru[self.serial] = (shape, entry, nbytes)
        self.nbytes += nbytes
        out = []
        while len(self.lru) > self.max_entries:
            out.append(self.evict_lru())
        return out

    def evict_lru(self):
        if not self.lru:
            return None
        serial, (shape, entry, nb) = self.lru.popitem(last=False)
        self.nbytes -= nb
        q = self.by_shape[shape]
        q.popleft()                    # serials grow, so the oldest overall is the oldest of its shape
        if not q:
            del self.by_shape[shape]
        return entry


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
    dev_bytes: int = 0           # table, counters and relays of its communicator
    cached: bool = False         # served from a memoized plan
    reserved: bool = False       # dev_bytes counted against the budget
    bypass_bytes: int = 0        # device bytes held while admitted past a waiting head
    t_admit: float = 0.0
    t_ready: float = 0.0         # planned and uploaded (or memoized): waiting for a slot
    t_launch: float = 0.0
    t_done: float = 0.0
    error: str = ""


class Server:
    """The serving loop; ``poll`` makes one round of progress.

    budget_bytes bounds the device memory of everything the server keeps:
    the requests' buffers (in one arena of that size) plus the tables,
    counters and relay buffers of their communicators, memoized ones
    included (a grouped launch's combined table is counted while it runs).
    ``cache_entries`` caps the memoized plans (0 disables them);
    ``comm_options`` ({hiccl option: value}) is applied to every request's
    communicator before planning.  ``bypass_frac`` = 0 makes admission
    strictly first in, first out; ``bypass_scan`` bounds how far behind a
    waiting head admission looks.  ``idle_s`` > 0 makes the loop sleep after
    a round that changed nothing (0: it only yields)."""

    def __init__(self, budget_bytes: int, slots: int = 8, max_batch: int = 1, planners: int = 4,
                 device="cuda", on_admit=None, on_done=None, cache_entries: int = 256, comm_options=None,
                 bypass_frac: float = 1 / 64, bypass_cap_frac: float = 1 / 8, bypass_scan: int = 64,
                 idle_s: float = 0.0):
        import torch
        self.device = torch.device(device)
        self.budget = budget_bytes
        self.arena = DeviceArena(budget_bytes, self.device)
        # a server on the CPU admits, plans and memoizes but launches nothing
        # (its host logic is tested that way on machines without a GPU)
        cuda = self.device.type == "cuda"
        self.slots = [{"stream": torch.cuda.Stream(self.device) if cuda else None, "event": None, "group": None,
                       "reqs": [], "group_bytes": 0} for _ in range(slots)]
        self.max_batch = max_batch
        self.pool = ThreadPoolExecutor(max_workers=planners)
        self.reaper = ThreadPoolExecutor(max_workers=1)   # destroys evicted communicators
        self.waiting: deque = deque()     # submitted, not admitted
        self.planning: list = []          # (future, request): host planning
        self.to_upload: deque = deque()   # planned, waiting for device memory
        self.uploading: list = []         # (future, request)
        self.ready: deque = deque()       # on the device, not launched
        self.grouping: list = []          # (future, batch): combined tables being built
        self.grouped: deque = deque()     # (group, device bytes, batch): built, waiting for a slot
        self.done: list = []
        self.on_admit, self.on_done = on_admit, on_done
        self.lock = threading.Lock()
        self.next_id = 0
        self.launches = 0
        # memoized plans apply to requests launched alone; grouped launches
        # build one combined table per group and keep no per-request state
        self.cache = PlanCache(cache_entries if max_batch == 1 else 0)
        self.dev_bytes = 0                # tables, counters, relays of live communicators
        self.comm_options = dict(comm_options or {})
        self.bypass_max = int(budget_bytes * bypass_frac)
        self.bypass_cap = int(budget_bytes * bypass_cap_frac)
        self.bypass_scan = bypass_scan
        self.bypass_held = 0              # device bytes of live requests admitted past a waiting head
        self.bypassed = 0                 # requests admitted past a waiting head
        self.idle_s = idle_s
        self.evicted = 0                  # memoized plans evicted for memory
        self.max_round_s = 0.0            # longest poll round (host stalls)

    @property
    def plan_cache_hits(self):
        return self.cache.hits

    @property
    def plan_cache_misses(self):
        return self.cache.misses

    def device_bytes(self) -> int:
        """Device memory held against the budget (buffers + communicators)."""
        return self.arena.used + self.dev_bytes

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

    @staticmethod
    def _shape(req: Request):
        return (req.kind, req.P, tuple(req.hierarchy), req.d, req.dtype, req.root)

    def _release_entry(self, e):
        """Free a memoized entry: its arena region and its communicator.  The
        entry is idle (no launch uses it), so its region is reusable at once;
        the communicator is destroyed on the reaper thread (its device memory
        is freed in stream order there), so that evicting many plans for one
        large request does not stall the polling loop."""
        self.evicted += 1
        self.dev_bytes -= e["dev_bytes"]
        self.arena.free(*e["region"])
        self.reaper.submit(e["comm"].destroy)

    def _fits(self, extra: int) -> bool:
        return self.arena.used + self.dev_bytes + extra <= self.budget

    def _make_room(self, need: int) -> bool:
        """Evict idle memoized plans (least recently used first) until
        ``need`` more bytes fit in the budget; evicts nothing when even
        every idle plan gone would not make room (memory held by running
        requests must free first, and the idle plans stay reusable)."""
        if self._fits(need):
            return True
        if not self._fits(need - self.cache.nbytes):
            return False
        while not self._fits(need):
            e = self.cache.evict_lru()
            if e is None:
                return False
            self._release_entry(e)
        return True

    def _admit(self):
        """Admit waiting requests in order while their buffers fit (memoized
        shapes take their resident plan).  When the head does not fit, small
        requests behind it may pass it under the rule in the module notes."""
        k = 0
        head_need = None               # buffer bytes of the head, while it waits for memory
        while k < len(self.waiting):
            req = self.waiting[k]
            sb, rb = self._layout(req)
            need = req.P * (sb + rb)
            passing = head_need is not None
            if passing:
                if k >= self.bypass_scan or self._fits(head_need - self.bypass_held - self.cache.nbytes):
                    return             # the head would fit once the requests that passed it drain
                if need > self.bypass_max or self.bypass_held + need > self.bypass_cap:
                    k += 1
                    continue
            if self.max_batch == 1:
                e = self.cache.take(self._shape(req))
                if e is not None:                      # memoized: nothing to plan, upload or allocate
                    self.cache.hits += 1
                    del self.waiting[k]
                    req.comm, req.region = e["comm"], e["region"]
                    req.send_ptrs, req.recv_ptrs = e["send_ptrs"], e["recv_ptrs"]
                    req.hbm_bytes, req.dev_bytes, req.cached = e["hbm_bytes"], e["dev_bytes"], True
                    req.reserved = True
                    if passing:                        # its resident memory is now held past the head
                        self._hold_bypass(req, e["region"][1] + e["dev_bytes"])
                    req.t_admit = req.t_ready = time.perf_counter()
                    if self.on_admit:
                        self.on_admit(req)
                    self.ready.append(req)
                    continue
            if passing:
                # nothing is evicted for a request that passes the head (the
                # head's own attempt already freed what could be freed)
                got = self.arena.alloc(need) if self._fits(need) else None
            else:
                room = self._make_room(need)
                got = self.arena.alloc(need) if room else None
                while room and got is None and len(self.cache):   # fragmentation: free idle regions until it fits
                    self._release_entry(self.cache.evict_lru())
                    got = self.arena.alloc(need)
            if got is None:
                if not passing:
                    if self.bypass_max <= 0:
                        return                 # strictly in order: wait until memory frees
                    head_need = need
                k += 1
                continue
            del self.waiting[k]
            self.cache.misses += 1
            off, n = got
            req.region = (off, n)
            if passing:
                self._hold_bypass(req, n)
            base = self.arena.base + off
            req.send_ptrs = [base + r * sb for r in range(req.P)]
            req.recv_ptrs = [base + req.P * sb + r * rb for r in range(req.P)]
            req.t_admit = time.perf_counter()
            if self.on_admit:
                self.on_admit(req)
            self.planning.append((self.pool.submit(self._plan, req, self.comm_options), req))

    def _hold_bypass(self, req: Request, nbytes: int):
        req.bypass_bytes = nbytes
        self.bypass_held += nbytes
        self.bypassed += 1

    @staticmethod
    def _plan(req: Request, options: dict):
        """Host planning (pool thread): factorize, and note the plan's device footprint."""
        comm = H.Comm(req.P, req.dtype)
        req.comm = comm
        for opt, val in options.items():
            comm.set_option(opt, val)
        comm.add_collective(req.kind, req.d, req.send_ptrs, req.recv_ptrs, req.root)
        comm.plan(req.hierarchy, 1, 1)
        rd, wr = comm.hbm_bytes()
        req.hbm_bytes = rd + wr
        info = comm.plan_info()
        req.dev_bytes = info["table_bytes"] + info["scratch_bytes"]

    @staticmethod
    def _upload(req: Request):
        """Upload of a host plan (pool thread; the plan is not factorized again)."""
        req.comm.init(req.hierarchy, 1, 1)

    def _on_uploaded(self, req: Request):
        req.t_ready = time.perf_counter()
        self.ready.append(req)

    def _collect(self, pending, on_ok):
        keep = []
        for fut, req in pending:
            if fut.done():
                err = fut.exception()
                if err is not None:
                    req.error = str(err)
                    self._finish(req, time.perf_counter())
                else:
                    on_ok(req)
            else:
                keep.append((fut, req))
        return keep

    def _reserve_uploads(self):
        """Count planned requests' tables and relays against the budget and
        upload those that fit (in order, passing over one that does not fit
        yet).  When nothing that holds memory can move -- no launch running,
        nothing uploading, ready or planning -- and no planned request fits,
        the first is refused so that its buffers go to the others."""
        if self.max_batch > 1:                         # group members stay host plans
            while self.to_upload:
                req = self.to_upload.popleft()
                req.dev_bytes = 0
                req.t_ready = time.perf_counter()
                self.ready.append(req)
            return
        kept = deque()
        while self.to_upload:
            req = self.to_upload.popleft()
            if self._make_room(req.dev_bytes):
                self.dev_bytes += req.dev_bytes
                req.reserved = True
                if req.bypass_bytes:
                    req.bypass_bytes += req.dev_bytes
                    self.bypass_held += req.dev_bytes
                self.uploading.append((self.pool.submit(self._upload, req), req))
            else:
                kept.append(req)
        self.to_upload = kept
        if kept and not (self.uploading or self.ready or self.planning or any(s["event"] for s in self.slots)):
            req = self.to_upload.popleft()
            req.error = (f"device footprint ({req.dev_bytes} bytes of tables and relays) does not fit the "
                         f"budget next to the buffers of the waiting requests")
            self._finish(req, time.perf_counter())

    @staticmethod
    def _build_group(batch):
        """Combined table of a batch (pool thread): plan union and upload."""
        grp = H.Comm.group([r.comm for r in batch])
        info = grp.plan_info()
        return grp, info["table_bytes"] + info["scratch_bytes"]

    def _start_on(self, sl, grp, batch, gb):
        """Launch ``grp`` on slot ``sl``; ``gb``: device bytes of a combined
        table (counted since it was built), released when the launch retires."""
        import torch
        sl["group_bytes"] = gb
        now = time.perf_counter()
        for r in batch:
            r.t_launch = now
        grp.start(sl["stream"])
        ev = torch.cuda.Event()
        ev.record(sl["stream"])
        sl["event"], sl["group"], sl["reqs"] = ev, grp, batch
        self.launches += 1

    def _collect_groups(self):
        keep = []
        for fut, batch in self.grouping:
            if not fut.done():
                keep.append((fut, batch))
                continue
            err = fut.exception()
            if err is not None:
                for r in batch:
                    r.error = str(err)
                    self._finish(r, time.perf_counter())
            else:
                grp, gb = fut.result()
                self.dev_bytes += gb           # the combined table is on the device from now on
                self.grouped.append((grp, gb, batch))
        self.grouping = keep

    def _launch(self):
        if self.device.type != "cuda":
            return
        for sl in self.slots:
            if sl["event"] is not None:
                continue
            if self.max_batch == 1:
                if not self.ready:
                    break
                req = self.ready.popleft()
                self._start_on(sl, req.comm, [req], 0)
            elif self.grouped:
                grp, gb, batch = self.grouped.popleft()
                self._start_on(sl, grp, batch, gb)
        # grouped launches: combined tables are built on the planner threads,
        # at most one per slot ahead of the launches
        while self.max_batch > 1 and self.ready and len(self.grouping) + len(self.grouped) < len(self.slots):
            batch = []
            while self.ready and len(batch) < self.max_batch:
                batch.append(self.ready.popleft())
            self.grouping.append((self.pool.submit(self._build_group, batch), batch))

    def _retire(self):
        for sl in self.slots:
            ev = sl["event"]
            if ev is None or not ev.query():
                continue
            now = time.perf_counter()
            sl["group"].wait()
            if not (len(sl["reqs"]) == 1 and sl["group"] is sl["reqs"][0].comm):
                sl["group"].destroy()
            self.dev_bytes -= sl["group_bytes"]
            sl["group_bytes"] = 0
            for r in sl["reqs"]:
                self._finish(r, now)
            sl["event"], sl["group"], sl["reqs"] = None, None, []

    def _finish(self, req: Request, now: float):
        req.t_done = now
        self.bypass_held -= req.bypass_bytes
        req.bypass_bytes = 0
        if self.on_done:
            self.on_done(req)
        if req.comm is not None and req.reserved and not req.error and self.cache.max_entries > 0:
            # memoize: the communicator and its buffers stay resident
            e = {"comm": req.comm, "region": req.region, "send_ptrs": req.send_ptrs, "recv_ptrs": req.recv_ptrs,
                 "hbm_bytes": req.hbm_bytes, "dev_bytes": req.dev_bytes}
            for old in self.cache.put(self._shape(req), e, req.region[1] + req.dev_bytes):
                self._release_entry(old)
        else:
            if req.comm is not None:
                req.comm.destroy()
            if req.reserved:
                self.dev_bytes -= req.dev_bytes
                req.reserved = False
            if req.region:
                self.arena.free(*req.region)
        req.comm = None
        req.region = ()
        self.done.append(req)

    def poll(self):
        """One round of progress: retire finished launches, admit waiting
        requests (memoized plans directly, the others to the planners), upload
        planned ones that fit, launch ready ones on free slots; then yield the
        interpreter lock to the planner threads (for ``idle_s`` after a round
        that changed nothing)."""
        t0 = time.perf_counter()
        before = (len(self.done), len(self.waiting), len(self.planning), len(self.uploading), len(self.ready),
                  len(self.grouping), self.launches)
        self._retire()
        with self.lock:
            self._admit()
        self.planning = self._collect(self.planning, self.to_upload.append)
        self._reserve_uploads()
        self.uploading = self._collect(self.uploading, self._on_uploaded)
        self._collect_groups()
        self._launch()
        after = (len(self.done), len(self.waiting), len(self.planning), len(self.uploading), len(self.ready),
                 len(self.grouping), self.launches)
        self.max_round_s = max(self.max_round_s, time.perf_counter() - t0)
        time.sleep(self.idle_s if after == before else 0)

    def busy(self) -> bool:
        return bool(self.waiting or self.planning or self.to_upload or self.uploading or self.ready
                    or self.grouping or self.grouped or any(s["event"] for s in self.slots))

    def drain(self, timeout_s: float = 600.0):
        t0 = time.perf_counter()
        while self.busy():
            self.poll()
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")

    def close(self):
        """Drain, stop the planners and free every memoized plan."""
        self.drain()
        self.pool.shutdown()
        while len(self.cache):
            self._release_entry(self.cache.evict_lru())
        self.reaper.shutdown()


def latency_stats(done: list) -> dict:
    lat = sorted((r.t_done - r.t_arrival) for r in done if not r.error)
    if not lat:
        return {"n": 0}

    def pct(q):
        return lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))]
    return {"n": len(lat), "p50_ms": pct(0.5) * 1e3, "p99_ms": pct(0.99) * 1e3, "max_ms": lat[-1] * 1e3}


def phase_stats(done: list) -> dict:
    """Where served requests spent their time, as p50 / p99 in ms of each
    phase: waiting for admission (memory), planning and upload, waiting for
    a launch slot, and from launch to observed completion."""
    ok = [r for r in done if not r.error and r.t_launch]
    if not ok:
        return {}
    phases = {"admit_wait": lambda r: r.t_admit - r.t_arrival, "plan_upload": lambda r: r.t_ready - r.t_admit,
              "slot_wait": lambda r: r.t_launch - r.t_ready, "run": lambda r: r.t_done - r.t_launch}
    out = {}
    for name, f in phases.items():
        v = sorted(f(r) for r in ok)
        out[name] = [round(v[int(q * (len(v) - 1) + 0.5)] * 1e3, 3) for q in (0.5, 0.99)]
    return out
