"""Benchmark of the hierarchical collective path on GB300.

Headline workload (one "step"): the seven standard collectives --
Broadcast, Scatter, Gather, All-gather, Reduce-scatter, All-reduce (Listing
2) and All-to-all -- over P = 64 virtual ranks with hierarchy {4,4,4}, 4 MiB
of fp32 per rank (uniform[-1, 1], seed 0), stripe 4, pipeline 8; each
collective is one start of its own persistent communicator.  The seven
starts of a step are captured once in a CUDA graph, each on its own stream
forked from the step's stream (independent collectives started back to back
on separate streams, so that one launch's last work items run beside the
next one's first); the timed region is a series of blocks of K graph
replays (at least one second in all) and the median block gives the step
time (Sec. 6.2 reports the median of its measured rounds).  Beside it: the
same step with the starts in order on one stream ("serial_step"), the same
steps through start / wait on the host ("eager"), and the seven collectives
as one grouped communicator, one launch per step ("grouped_step").

Metric: device-memory GB/s of the schedule (each copy reads its bytes once
and writes them once per destination; an f-input reduce reads f times and
writes once), with the fraction of the measured HBM bandwidth; per
collective GB/s, the semantic-minimum bytes and the paper-style d*p/t are
reported beside it.  The default line also carries, each under its own
timing: the 64 MiB-per-rank All-reduce as FP32, BF16 and FP8 payloads with
their FP64 errors; the batch of 256 mixed collectives (one launch each,
grouped, graph); and a short served run with p50 / p99 latency.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload seven|allreduce64|batch256|serve] [--no-extras]
Under torchrun each rank runs an independent replica on its own GPU
("replicas only": the virtual-rank path does not shard across devices).
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HBM GB/s (% of GB300 peak) per collective; p50/p99 latency of served requests"
KINDS = ("broadcast", "scatter", "gather", "allgather", "reducescatter", "allreduce", "alltoall")
P, HIER, STRIPE, PIPE = 64, [4, 4, 4], 4, 8
BYTES_PER_RANK = 4 << 20
KERNEL_SRC = os.path.join(ROOT, "paper_2408_05962_gb300", "csrc", "hiccl_runtime.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "executor_traffic_seven_p64.txt")


# the two single-GPU workloads: the seven collectives (the headline), and the
# large All-reduce of 64 MiB per rank used for the >= 16 MiB-per-rank bandwidth
WORKLOADS = {
    "seven": {"ranks": 64, "hierarchy": [4, 4, 4], "stripe": 4, "pipeline": 8, "bytes_per_rank": 4 << 20,
              "kinds": KINDS, "data": "uniform[-1,1] fp32, seed 0",
              "name": "seven collectives, P=64 virtual ranks, hierarchy {4,4,4}, 4 MiB fp32 per rank, "
                      "stripe 4, pipeline 8",
              "l2": "working set of one step ~3.5 GB > 129 MB L2; no flush between steps"},
    "allreduce64": {"ranks": 32, "hierarchy": [4, 8], "stripe": 1, "pipeline": 4, "bytes_per_rank": 64 << 20,
                    "kinds": ("allreduce",), "data": "N(0,1) * 10**U(-3,3) per rank fp32, seed 0",
                    "name": "All-reduce (Listing 2), P=32 virtual ranks, hierarchy {4,8}, 64 MiB fp32 per rank, "
                            "stripe 1, pipeline 4",
                    "l2": "working set 4 GiB > 129 MB L2; no flush between steps"},
}


def workload_config(w="seven", world=1, dtype="f32", extra=None):
    """The ``config`` of a line: the same dict in both arms."""
    W = WORKLOADS[w]
    cfg = {"workload": W["name"], "ranks": W["ranks"], "hierarchy": W["hierarchy"], "stripe": W["stripe"],
           "pipeline": W["pipeline"], "bytes_per_rank": W["bytes_per_rank"], "collectives": list(W["kinds"]),
           "inputs": W["data"], "l2": W["l2"], "payload": dtype, "parallelism": f"replicas{world}"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# host placement of the end-to-end buffers
# ---------------------------------------------------------------------------

def parse_cpulist(text):
    """'0-3,8,10-11' -> {0, 1, 2, 3, 8, 10, 11}"""
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def host_node_of(device, sysfs="/sys"):
    """NUMA node of the host side of the GPU's link (sysfs numa_node of its
    PCI function), or None where it is not known."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device)
        bus = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        with open(os.path.join(sysfs, "bus", "pci", "devices", bus, "numa_node")) as f:
            node = int(f.read().strip())
        return node if node >= 0 else None
    except (AttributeError, OSError, ValueError, RuntimeError):
        return None


class cpus_of_node:
    """Context manager: run the calling thread on the CPUs of NUMA node
    `node` (those it may use), so that host memory it first touches is
    allocated there; a no-op for None or an unknown node."""

    def __init__(self, node, sysfs="/sys"):
        self.node, self.sysfs, self.saved = node, sysfs, None

    def __enter__(self):
        if self.node is None or not hasattr(os, "sched_setaffinity"):
            return self
        try:
            with open(os.path.join(self.sysfs, "devices", "system", "node", f"node{self.node}", "cpulist")) as f:
                want = parse_cpulist(f.read())
            allowed = os.sched_getaffinity(0)
            use = want & allowed
            if use and use != allowed:
                os.sched_setaffinity(0, use)
                self.saved = allowed
        except (OSError, ValueError):
            pass
        return self

    def __exit__(self, *exc):
        if self.saved is not None:
            os.sched_setaffinity(0, self.saved)
        return False


def host_copy_rates(h_send, h_recv, bufs, kinds, stream, device):
    """GB/s of one plain pass of the end-to-end leg's copies: every send
    buffer host -> device alone, every receive buffer device -> host alone,
    and both at once on two streams (bytes of both directions over the time
    of both).  The end-to-end figure cannot exceed what the host link gives
    here; None where the measurement fails."""
    import torch
    try:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize(device)
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for k in kinds:
                bufs[k].send.copy_(h_send[k], non_blocking=True)
            ev[1].record(stream)
            for k in kinds:
                h_recv[k].copy_(bufs[k].recv, non_blocking=True)
            ev[2].record(stream)
        ev[2].synchronize()
        hb = sum(t.numel() * t.element_size() for t in h_send.values())
        db = sum(t.numel() * t.element_size() for t in h_recv.values())
        out = {"h2d_gbs": hb / (ev[0].elapsed_time(ev[1]) * 1e6), "d2h_gbs": db / (ev[1].elapsed_time(ev[2]) * 1e6)}
        other = torch.cuda.Stream(device)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize(device)
        e0.record(stream)
        other.wait_event(e0)
        with torch.cuda.stream(stream):
            for k in kinds:
                bufs[k].send.copy_(h_send[k], non_blocking=True)
            e1.record(stream)
        with torch.cuda.stream(other):
            for k in kinds:
                h_recv[k].copy_(bufs[k].recv, non_blocking=True)
            e2.record(other)
        torch.cuda.synchronize(device)
        both = max(e0.elapsed_time(e1), e0.elapsed_time(e2))
        out["both_directions_gbs"] = (hb + db) / (both * 1e6)
        return out
    except Exception:   # a report field only: never fail the benchmark for it
        return {"h2d_gbs": None, "d2h_gbs": None, "both_directions_gbs": None}


# ---------------------------------------------------------------------------
# multi-rank plumbing (replicas): barrier and max over ranks
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(backend):
    import torch.distributed as dist
    world, rank, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return world, rank


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(local_bytes: float, local_seconds: float, device=None):
    """Whole-job (sum of bytes over ranks, max of time over ranks)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local_bytes, local_seconds
    dev = device if (device is not None and dist.get_backend() == "nccl") else torch.device("cpu")
    b = torch.tensor([local_bytes], dtype=torch.float64, device=dev)
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(b.item()), float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("hiccl_runtime.cu", "hiccl_internal.h"):
        with open(os.path.join(ROOT, "paper_2408_05962_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current executor source (else None)."""
    try:
        vals = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("kernel_sha") != kernel_hash():
            return None
        return float(vals["dram_bytes_per_step"])
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the oracle as a CPU baseline / reference arm (bounded sample)
# ---------------------------------------------------------------------------

_ORACLE_CACHE = {}


def _oracle_plan(kind: str, seed: int = 0):
    """The oracle's factorized schedule of one collective of the headline
    workload and its buffers (built once; factorization is initialization,
    not part of a step)."""
    key = (kind, seed)
    if key in _ORACLE_CACHE:
        return _ORACLE_CACHE[key]
    import numpy as np

    from oracle import programs as PR
    from oracle.factorize import factorize
    from synth import uniform_ranks

    d = BYTES_PER_RANK // 4 // P
    x = uniform_ranks(P, d * P, seed=seed)
    prog = PR.BUILDERS[kind](P, d)
    plan = factorize(prog, HIER, STRIPE, PIPE)
    mem = prog.allocate()
    for r in range(P):
        mem[("send", r)][...] = x[r][:mem[("send", r)].shape[0]]
    for k, n in plan.scratch.items():
        mem[k] = np.zeros(n, dtype=np.float32)
    _ORACLE_CACHE[key] = (plan, mem)
    return plan, mem


def _simulate_for(kind: str, budget_s: float, seed: int = 0):
    """Run the oracle's schedule simulator on one collective for about
    ``budget_s`` seconds: complete executions in dependency order, repeated,
    the last one cut off when the time is up.  Returns (schedule bytes, s)."""
    from oracle.simulate import execute_op

    plan, mem = _oracle_plan(kind, seed)
    total_b, t0 = 0, time.perf_counter()
    while True:
        for op in plan.ops:
            execute_op(op, mem)
            total_b += op.n * 4 * (1 + len(op.dsts) if op.kind == "copy" else len(op.srcs) + 1)
            if time.perf_counter() - t0 > budget_s:
                return total_b, time.perf_counter() - t0


def oracle_sample(budget_s: float, seed: int = 0):
    """The oracle's schedule simulator on one thread over the seven
    collectives, ``budget_s`` seconds in all.  Returns (bytes, s, description)."""
    per = budget_s / len(KINDS)
    bs, ts = 0, 0.0
    for kind in KINDS:
        b, t = _simulate_for(kind, per, seed)
        bs += b
        ts += t
    return bs, ts, (f"oracle schedule simulator (NumPy, 1 thread) on each of the seven collectives for "
                    f"{per:.1f} s (complete executions in dependency order, repeated; factorization untimed)")


_BARRIER = None


def _worker_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(job):
    kind, budget_s, seed = job
    _oracle_plan(kind, seed)   # untimed set-up
    _BARRIER.wait()            # every worker simulates in the same time window
    return _simulate_for(kind, budget_s, seed)


def oracle_all_cores(budget_s: float, cores: int, seed: int = 0):
    """The same simulator on ``cores`` worker processes at once (spawned:
    nothing is forked from a process that has used the GPU), worker i
    simulating its own copy of collective i mod 7.  Returns (bytes summed over
    the workers, the longest worker's time, description)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    jobs = [(KINDS[i % len(KINDS)], budget_s, seed) for i in range(cores)]
    with ctx.Pool(cores, initializer=_worker_init, initargs=(barrier,)) as pool:
        res = pool.map(_oracle_worker, jobs, chunksize=1)
    return (sum(b for b, _ in res), max(t for _, t in res),
            f"oracle schedule simulator in {cores} processes at once, process i running its own copy of "
            f"collective i mod 7 for {budget_s:.1f} s (complete executions, repeated; factorization untimed)")


def cpu_baseline(budget_s: float):
    """Single-thread and all-cores legs of the oracle on this host."""
    cores = os.cpu_count() or 1
    b1, t1, d1 = oracle_sample(budget_s)
    out = {"unit": "GB/s", "kind": "oracle", "nproc": cores,
           "single_thread": {"value": b1 / t1 / 1e9, "cores": 1, "sample": d1}}
    try:
        bn, tn, dn = oracle_all_cores(budget_s / 2, cores)
        out.update({"value": bn / tn / 1e9, "cores": cores, "sample": dn})
    except Exception as e:   # a report field only
        out.update({"value": b1 / t1 / 1e9, "cores": 1, "sample": d1, "all_cores_error": repr(e)[:200]})
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if world > 1:
        dist_init("gloo")
        if rank != 0:
            return
    for _ in range(args.warmup):
        oracle_sample(0.5)
    per_step = []
    bs, ts = 0, 0.0
    for _ in range(args.steps):
        b, t, desc = oracle_sample(args.ref_budget)
        bs += b
        ts += t
        per_step.append(t)
    gbs = bs / ts / 1e9
    line = {"metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.median(per_step) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config("seven", world, "f32"), "impl": "reference",
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc,
                             "nproc": os.cpu_count()},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def _fp8_blocks(x):
    """Encode binary32 rows into the FP8 payload (per 128 values: e4m3
    codes of x * (448 / amax), the binary32 scale amax / 448, 12 zero bytes), on the
    GPU with torch's float8_e4m3fn conversion (round to nearest even).
    Input encoding is set-up, not part of the timed path."""
    import torch
    P, n = x.shape
    xb = x.reshape(P, n // 128, 128)
    amax = xb.abs().amax(dim=2, keepdim=True)
    scale = torch.where(amax == 0, torch.ones_like(amax), amax / 448.0)
    inv = torch.where(amax == 0, torch.ones_like(amax), 448.0 / amax)
    q = (xb * inv).clamp(-448.0, 448.0).to(torch.float8_e4m3fn).view(torch.uint8)
    out = torch.zeros(P, n // 128, 144, dtype=torch.uint8, device=x.device)
    out[:, :, :128] = q
    out[:, :, 128:132] = scale.view(torch.uint8).reshape(P, n // 128, 4)
    return out.reshape(P, -1)


def _bf16_rows(x):
    """binary32 rows (host) -> BF16 bit patterns, round to nearest even on the
    upper 16 bits (payload encoding, set-up)."""
    import torch
    t = torch.from_numpy(x).view(torch.int32)
    return ((t + 0x7FFF + ((t >> 16) & 1)) >> 16).to(torch.int16)


def min_bytes(kind: str, P: int, B: int) -> int:
    """HBM bytes a collective cannot avoid on one device: every input byte it
    needs read once and every output byte written once (B = the largest
    per-rank buffer, d*P values; root-only results for Reduce and Gather)."""
    d = B // P
    return {"broadcast": B + P * B, "reduce": P * B + B, "allgather": P * d + P * B,
            "reducescatter": P * B + P * d, "allreduce": 2 * P * B, "allreduce_single": 2 * P * B,
            "scatter": B + P * d, "gather": P * d + B, "alltoall": 2 * P * B}.get(kind, 0)


def _decode_rows(t, dtype):
    """Payload rows (device) -> binary32 values (device)."""
    import torch
    if dtype == "bf16":
        return (t.to(torch.int32) << 16).view(torch.float32)
    blk = t.reshape(t.shape[0], -1, 144)
    codes = blk[:, :, :128].contiguous().view(torch.float8_e4m3fn).to(torch.float32)
    scale = blk[:, :, 128:132].contiguous().view(torch.float32)
    return (codes * scale).reshape(t.shape[0], -1)


def _lowprec_accuracy(b, dtype, xs, device):
    """Error of the reduced-precision All-reduce results, measured after the
    timed region with plain torch arithmetic, per result buffer: relative L2
    and max-norm errors against the FP64 sum of the decoded inputs, and the
    relative L2 error against the FP64 sum of the unquantized binary32
    sources (the worst over the P result buffers is reported)."""
    import torch
    P = b.send.shape[0]
    y64 = torch.zeros(_decode_rows(b.send[:1], dtype).shape[1], dtype=torch.float64, device=device)
    x64 = torch.zeros_like(y64)
    for r in range(P):
        y64 += _decode_rows(b.send[r:r + 1], dtype)[0].double()
        x64 += torch.from_numpy(xs[r]).to(device).double()
    n64, m64, nx = y64.norm(), y64.abs().max(), x64.norm()
    l2, mx, lx = 0.0, 0.0, 0.0
    for r in range(P):
        y = _decode_rows(b.recv[r:r + 1], dtype)[0].double()
        l2 = max(l2, float((y - y64).norm() / n64))
        mx = max(mx, float((y - y64).abs().max() / m64))
        lx = max(lx, float((y - x64).norm() / nx))
    return {"rel_l2_vs_fp64_of_decoded": l2, "rel_max_vs_fp64_of_decoded": mx,
            "rel_l2_vs_fp64_of_unquantized": lx, "bound_rel_l2": 1e-2 if dtype == "bf16" else 6e-2,
            "result_buffers": P}


def _time_blocks(fn, k, min_s, stream):
    """Blocks of ``k`` calls of fn, each bracketed by CUDA events on
    ``stream``, until at least ``min_s`` seconds and three blocks have been
    timed; returns the block times in ms."""
    import torch
    blocks, total = [], 0.0
    while total < min_s or len(blocks) < 3:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        blocks.append(ms)
        total += ms / 1e3
    return blocks


def _make_comm(H, P, dtype, args):
    comm = H.Comm(P, dtype)
    if args.item_bytes:
        comm.set_option(H.OPT_ITEM_BYTES, args.item_bytes)
    if args.order is not None:
        comm.set_option(H.OPT_ORDER, args.order)
    if args.ctas_per_sm:
        comm.set_option(H.OPT_CTAS_PER_SM, args.ctas_per_sm)
    if args.threads:
        comm.set_option(H.OPT_THREADS, args.threads)
    if args.ring > 1:
        comm.set_option(H.OPT_RING, args.ring)
    if args.slot_items:
        comm.set_option(H.OPT_SLOT_ITEMS, args.slot_items)
    return comm


def _graph_of(comms, kinds, device, concurrent=False):
    """One CUDA graph holding one start of the communicator of every name in
    ``kinds`` (names may repeat; a start under capture records only the
    executor launch, and each replay is a complete execution): in order on
    one stream, or (``concurrent``) each on its own stream forked from the
    graph's stream and joined back, as independent collectives started back
    to back on separate streams run -- the launches then overlap on the
    device (one's last work items beside the next one's first) instead of
    each waiting for the previous grid to complete."""
    import torch
    gs = torch.cuda.Stream(device)
    graph = torch.cuda.CUDAGraph()
    side = [torch.cuda.Stream(device) for _ in kinds] if concurrent else []
    with torch.cuda.graph(graph, stream=gs):
        if concurrent:
            for s, kind in zip(side, kinds):
                s.wait_stream(gs)
                comms[kind].start(s)
            for s in side:
                gs.wait_stream(s)
        else:
            for kind in kinds:
                comms[kind].start(gs)
    return graph


def measure_collectives(args, device, world, workload, dtype, xs=None, e2e=True):
    """The headline measurement of a single-GPU workload (the seven
    collectives, or one All-reduce payload of the 64 MiB workload)."""
    import torch

    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    from synth import uniform_ranks

    W = WORKLOADS[workload]
    Pw, hier, stripe, pipe = W["ranks"], W["hierarchy"], W["stripe"], W["pipeline"]
    bpr = args.bytes_per_rank or W["bytes_per_rank"]
    d = bpr // 4 // Pw                            # values per chunk (bytes of fp32 values per rank / P)
    if workload == "seven":
        x = torch.from_numpy(uniform_ranks(Pw, d * Pw, seed=0))
    elif dtype == "bf16":
        x = _bf16_rows(xs)
    elif dtype == "fp8":
        x = None
    else:
        x = torch.from_numpy(xs)
    comms, bufs, nbytes, pbytes, mbytes = {}, {}, {}, {}, {}
    kinds = tuple(args.kinds.split(",")) if args.kinds else W["kinds"]
    tdt = {"f32": torch.float32, "bf16": torch.int16, "fp8": torch.uint8}[dtype]
    for kind in kinds:
        b = C.Buffers(kind, Pw, d, tdt, device)
        if x is None:
            b.send.copy_(_fp8_blocks(torch.from_numpy(xs).to(device)))
        else:
            b.send.copy_(x[:, :b.send.shape[1]].to(device))
        b.recv.zero_()
        comm = _make_comm(H, Pw, dtype, args)
        C.compose(comm, kind, d, b.send_ptrs(), b.recv_ptrs())
        comm.init(hier, stripe, pipe)
        rd, wr = comm.hbm_bytes()
        comms[kind], bufs[kind], nbytes[kind] = comm, b, rd + wr
        pbytes[kind] = H.nbytes(H.DTYPES[dtype], d * Pw)   # the paper's d*p per collective
        mbytes[kind] = min_bytes(kind, Pw, pbytes[kind])
    del x
    stream = torch.cuda.current_stream(device)
    step_bytes = sum(nbytes.values())

    def eager_step(evs=None):
        """All collectives back to back on one stream through start / wait.
        With ``evs`` (one event per collective plus one) each launch is
        bracketed; without, consecutive launches overlap their launch latency
        (programmatic dependent launch)."""
        for i, kind in enumerate(kinds):
            if evs is not None:
                evs[i].record(stream)
            comms[kind].start(stream)
        if evs is not None:
            evs[len(kinds)].record(stream)
        for kind in kinds:
            comms[kind].wait()

    warm = max(args.warmup, 3)
    for _ in range(warm):
        eager_step()
    torch.cuda.synchronize(device)

    # per-collective breakdown (untimed pass, events between the launches)
    per_kind = {kind: [] for kind in kinds}
    for _ in range(10):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(kinds) + 1)]
        eager_step(evs)
        torch.cuda.synchronize(device)
        for i, kind in enumerate(kinds):
            per_kind[kind].append(evs[i].elapsed_time(evs[i + 1]))

    # per-collective steady state: ten starts of one collective in one graph,
    # replayed (consecutive launches overlap as in the step's graph)
    per_kind_graph = {}
    for kind in kinds:
        g1 = _graph_of(comms, (kind,) * 10, device)
        for _ in range(2):
            g1.replay()
        per_kind_graph[kind] = statistics.median(_time_blocks(g1.replay, 3, 0.0, stream)) / 30
        del g1
    torch.cuda.synchronize(device)

    # the same collectives as one grouped communicator (hiccl_group): one
    # persistent launch per step whose tickets interleave the seven by depth
    grouped = None
    if len(kinds) > 1:
        gcomm = H.Comm.group([comms[k] for k in kinds])
        gg = _graph_of({"group": gcomm}, ("group",) * 10, device)
        for _ in range(2):
            gg.replay()
        gms = statistics.median(_time_blocks(gg.replay, 3, 0.0, stream)) / 30
        grouped = {"ms_per_step": gms, "gbs": step_bytes / gms / 1e6, "launches_per_step": 1,
                   "method": "graph of ten starts of the grouped communicator, replayed; median of 3 blocks of 3"}
        del gg
        gcomm.destroy()
        torch.cuda.synchronize(device)

    # the same step with the seven starts in order on one stream, each launch
    # waiting for the previous grid (programmatic dependent launch overlaps
    # only their launch latency)
    serial = None
    if len(kinds) > 1:
        gser = _graph_of(comms, kinds, device)
        for _ in range(warm):
            gser.replay()
        sblocks = _time_blocks(gser.replay, args.steps, 0.25, stream)
        sms = statistics.median(sblocks) / args.steps
        serial = {"ms_per_step": sms, "gbs": step_bytes / sms / 1e6, "launches_per_step": len(kinds),
                  "method": f"graph of one step with the starts in order on one stream; blocks of {args.steps} "
                            "replays until >= 0.25 s, median block"}
        del gser
        torch.cuda.synchronize(device)

    graph = _graph_of(comms, kinds, device, concurrent=len(kinds) > 1)
    for _ in range(warm):
        graph.replay()
    torch.cuda.synchronize(device)

    clocks = ClockSampler(device.index)
    clocks.start()
    time.sleep(0.3)
    barrier(device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    blocks = _time_blocks(graph.replay, args.steps, args.min_seconds, stream)
    wall = time.perf_counter() - t0
    barrier(device)
    clk = clocks.stop()
    # the same steps through start / wait on the host, one block
    torch.cuda.synchronize(device)
    eager_blocks = _time_blocks(eager_step, args.steps, 0.0, stream)
    block_ms = statistics.median(blocks)
    tot_bytes, tot_s = aggregate(step_bytes * args.steps, block_ms / 1e3, device)
    gbs = tot_bytes / tot_s / 1e9
    peak, peak_kind = measured_peak()

    e2e_line = None
    if e2e:
        e2e_line = _end_to_end(comms, bufs, kinds, tdt, step_bytes, args, device, stream)

    coll = {}
    for kind in kinds:
        med = statistics.median(per_kind[kind])
        gm = per_kind_graph[kind]
        coll[kind] = {"ms": med, "gbs": nbytes[kind] / med / 1e6, "frac": nbytes[kind] / med / 1e6 / peak,
                      "graph_ms": gm, "graph_gbs": nbytes[kind] / gm / 1e6, "graph_frac": nbytes[kind] / gm / 1e6 / peak,
                      "dp_over_t_gbs": pbytes[kind] / med / 1e6, "schedule_bytes": nbytes[kind],
                      "min_bytes": mbytes[kind], "min_gbs": mbytes[kind] / med / 1e6,
                      "level_bytes": comms[kind].level_bytes(), "steps": comms[kind].plan_info()["steps"]}
    accuracy = None
    if dtype in ("bf16", "fp8") and "allreduce" in bufs:
        accuracy = _lowprec_accuracy(bufs["allreduce"], dtype, xs, device)
    out = {"value": gbs, "frac": gbs / world / peak, "peak": peak, "peak_kind": peak_kind,
           "ms_per_step": block_ms / args.steps, "blocks": len(blocks), "steps_per_block": args.steps,
           "block_ms": blocks, "timed_s": sum(blocks) / 1e3, "wall_s": wall, "clocks": clk,
           "launches": len(kinds) * args.steps * len(blocks), "step_bytes": step_bytes,
           "eager": {"value": step_bytes * args.steps / (statistics.median(eager_blocks) / 1e3) / 1e9,
                     "ms_per_step": statistics.median(eager_blocks) / args.steps},
           "collectives": coll, "e2e": e2e_line, "accuracy": accuracy, "grouped": grouped, "serial": serial}
    for c in comms.values():
        c.destroy()
    del bufs, graph
    torch.cuda.empty_cache()
    return out


def _end_to_end(comms, bufs, kinds, tdt, step_bytes, args, device, stream):
    """End to end through the public API with host buffers (pinned), placed on
    the NUMA node of the GPU's host link where sysfs names one: every step
    copies each send buffer host -> device, starts and waits on every
    collective, and copies each receive buffer device -> host.  The copies
    overlap the collectives and each other: the uploads run on one stream and
    the downloads on another, ordered only by events -- a collective starts
    once its inputs are uploaded and the previous step's download of its
    receive buffer is done, an upload waits for the previous step's
    collective to have read the buffer -- so one step's downloads overlap the
    next step's uploads (the host link runs both directions at once)."""
    import torch
    numa = host_node_of(device)
    with cpus_of_node(numa):
        h_send = {k: torch.empty(bufs[k].send.shape, dtype=tdt, pin_memory=True) for k in kinds}
        h_recv = {k: torch.empty(bufs[k].recv.shape, dtype=tdt, pin_memory=True) for k in kinds}
        for k in kinds:
            h_send[k].copy_(bufs[k].send)
            h_recv[k].zero_()
    h2d = sum(t.numel() * t.element_size() for t in h_send.values())
    d2h = sum(t.numel() * t.element_size() for t in h_recv.values())
    e2e_steps = max(1, min(args.steps, 5))
    s_in, s_out = torch.cuda.Stream(device), torch.cuda.Stream(device)
    coll_done = {k: None for k in kinds}   # collective k of the previous step has read its inputs
    d2h_done = {k: None for k in kinds}    # download of k's results of the previous step is done
    t_e2e = 0.0
    for it in range(e2e_steps + 1):      # the first pass is an untimed warm-up
        if it == 1:
            barrier(device)
            torch.cuda.synchronize(device)
            t_e2e = time.perf_counter()
        ev_in = {}
        with torch.cuda.stream(s_in):
            for k in kinds:
                if coll_done[k] is not None:
                    s_in.wait_event(coll_done[k])
                bufs[k].send.copy_(h_send[k], non_blocking=True)
                ev_in[k] = torch.cuda.Event()
                ev_in[k].record(s_in)
        for k in kinds:
            stream.wait_event(ev_in[k])
            if d2h_done[k] is not None:
                stream.wait_event(d2h_done[k])
            comms[k].start(stream)
            coll_done[k] = torch.cuda.Event()
            coll_done[k].record(stream)
            s_out.wait_event(coll_done[k])
            with torch.cuda.stream(s_out):
                h_recv[k].copy_(bufs[k].recv, non_blocking=True)
                d2h_done[k] = torch.cuda.Event()
                d2h_done[k].record(s_out)
        for k in kinds:
            comms[k].wait()
        if it == 0:
            torch.cuda.synchronize(device)
    torch.cuda.synchronize(device)
    e2e_s = time.perf_counter() - t_e2e
    eb, es = aggregate(step_bytes * e2e_steps, e2e_s, device)
    host_link = host_copy_rates(h_send, h_recv, bufs, kinds, s_in, device)
    return {"value": eb / es / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": e2e_steps, "host_numa_node": numa, **host_link}


def measure_allreduce64(args, device, dtypes=("f32", "bf16", "fp8")):
    """The 64 MiB-per-rank All-reduce (P = 32 over {4, 8}, s = 1, m = 4) on
    the same synthetic values as FP32, BF16 and FP8 payloads, each timed on
    its own (graph-replayed blocks, as the headline) with its FP64 errors."""
    from synth import scaled_normal_ranks
    W = WORKLOADS["allreduce64"]
    xs = scaled_normal_ranks(W["ranks"], W["bytes_per_rank"] // 4, seed=0)
    sub = argparse.Namespace(**vars(args))
    sub.kinds, sub.bytes_per_rank, sub.steps, sub.min_seconds = "", 0, 10, 0.25
    out = {}
    for dt in dtypes:
        r = measure_collectives(sub, device, 1, "allreduce64", dt, xs=xs, e2e=False)
        out[dt] = {"gbs": r["value"], "frac": r["frac"], "ms": r["ms_per_step"],
                   "schedule_bytes": r["step_bytes"], "eager_gbs": r["eager"]["value"],
                   **({"accuracy": r["accuracy"]} if r["accuracy"] else {})}
    out["config"] = workload_config("allreduce64", 1, "f32+bf16+fp8")
    return out


def measure_batch(args, device, steps):
    """Batched workload: 256 collectives (All-gather / Reduce-scatter /
    All-reduce drawn uniformly, P from {8, 16, 32} with two-level
    hierarchies, per-rank sizes log-uniform 4 KiB .. 16 MiB, fp32 and bf16
    mixed; synth.batch_mix seed 0), stripe / pipeline / executor knobs chosen
    by the autotuner (one tuning per kind, P, hierarchy, payload and size
    octave).  Timed three ways on one stream: one launch per collective (all
    256 enqueued, then waited), one grouped launch, and the grouped launch
    replayed from a CUDA graph."""
    import torch

    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    from synth import batch_mix

    descs = batch_mix(256, seed=0)
    gen = torch.Generator(device=device)
    gen.manual_seed(0)
    comms, bufs, tuned = [], [], {}
    stream = torch.cuda.current_stream(device)
    total_bytes = 0
    t_setup = time.perf_counter()
    for dsc in descs:
        P, h, dt = dsc["P"], dsc["hierarchy"], dsc["dtype"]
        es = 4 if dt == "f32" else 2
        d = dsc["bytes_per_rank"] // es // P
        b = C.Buffers(dsc["kind"], P, d, torch.float32 if dt == "f32" else torch.bfloat16, device)
        b.send.uniform_(-1.0, 1.0, generator=gen)
        b.recv.zero_()
        key = (dsc["kind"], P, tuple(h), dt, int(math.log2(dsc["bytes_per_rank"])))
        comm = H.Comm(P, dt)
        conf = tuned.get(key)
        if conf:
            comm.set_option(H.OPT_ORDER, conf["order"])
            comm.set_option(H.OPT_ITEM_BYTES, conf["item_bytes"])
        C.compose(comm, dsc["kind"], d, b.send_ptrs(), b.recv_ptrs())
        if conf:
            comm.init(h, conf["stripe"], conf["pipeline"])
        else:
            comm.init(h, h[-1], 4)
            tuned[key] = comm.autotune(stream, tune_method=True)
        rd, wr = comm.hbm_bytes()
        total_bytes += rd + wr
        comms.append(comm)
        bufs.append(b)
    t_setup = time.perf_counter() - t_setup

    def separate():
        for c in comms:
            c.start(stream)
        for c in comms:
            c.wait()

    grp = H.Comm.group(comms)

    def grouped():
        grp.start(stream)
        grp.wait()

    for _ in range(3):
        separate()
        grouped()
    torch.cuda.synchronize(device)
    gs = torch.cuda.Stream(device)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        grp.start(gs)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize(device)
    t_sep = statistics.median(_time_blocks(separate, steps, 0.2, stream)) / steps / 1e3
    t_grp = statistics.median(_time_blocks(grouped, steps, 0.2, stream)) / steps / 1e3
    t_graph = statistics.median(_time_blocks(graph.replay, steps, 0.2, stream)) / steps / 1e3
    out = {"schedule_bytes": total_bytes, "one_launch_each_ms": t_sep * 1e3,
           "grouped_ms": t_grp * 1e3, "graph_ms": t_graph * 1e3,
           "one_launch_each_gbs": total_bytes / t_sep / 1e9, "grouped_gbs": total_bytes / t_grp / 1e9,
           "graph_gbs": total_bytes / t_graph / 1e9, "speedup_vs_one_launch_each": t_sep / t_graph,
           "tuned_configs": len(tuned), "setup_s": t_setup,
           "config": "256 collectives (All-gather/Reduce-scatter/All-reduce), P in {8,16,32}, two-level "
                     "hierarchies, 4 KiB..16 MiB per rank log-uniform, fp32/bf16, one persistent launch "
                     "replayed from a CUDA graph; stripe, pipeline and executor knobs autotuned"}
    for c in comms:
        c.destroy()
    grp.destroy()
    del bufs, graph
    torch.cuda.empty_cache()
    return out


def serve_trace(rate, duration, budget_gb, slots, max_batch, seed=0, shapes=0, **server_kw):
    """Serve one Poisson arrival trace (synth.poisson_requests; ``shapes`` > 0:
    arrivals drawn from that many recurring request shapes) with
    serving.Server; returns its latency and throughput summary."""
    from paper_2408_05962_gb300.serving import Request, Server, latency_stats, phase_stats
    from synth import poisson_requests

    descs = poisson_requests(rate, duration, seed=seed, shapes=shapes)
    srv = Server(budget_gb << 30, slots=slots, max_batch=max_batch, planners=8, **server_kw)
    # as a latency-bound Python service would run: the objects made before
    # serving (this process's earlier measurements, torch's own) are frozen
    # out of the cyclic collector, and the collector is off while requests
    # arrive (reference counting still frees everything acyclic; a full
    # collection over the requests kept for the statistics paused the loop
    # for up to 180 ms in a 60 s run); it collects once the trace is served.
    # Any collection during the trace is recorded
    pauses, t_gc = [], [0.0]

    def on_gc(phase, info):
        if phase == "start":
            t_gc[0] = time.perf_counter()
        else:
            pauses.append((info.get("generation", -1), time.perf_counter() - t_gc[0]))

    gc.collect()
    gc.freeze()
    gc.callbacks.append(on_gc)
    gc.disable()
    try:
        t0 = time.perf_counter()
        k = 0
        while k < len(descs) or srv.busy():
            now = time.perf_counter() - t0
            while k < len(descs) and descs[k]["t"] <= now:
                dsc = descs[k]
                srv.submit(Request(kind=dsc["kind"], P=dsc["P"], hierarchy=dsc["hierarchy"],
                                   bytes_per_rank=dsc["bytes_per_rank"], dtype=dsc["dtype"],
                                   t_arrival=t0 + dsc["t"]))
                k += 1
            srv.poll()
        wall = time.perf_counter() - t0
    finally:
        gc.enable()
        gc.callbacks.remove(on_gc)
    srv.close()
    gc.unfreeze()
    gc.collect()
    done = [r for r in srv.done if not r.error]
    st = latency_stats(done)
    total = sum(r.hbm_bytes for r in done)
    out = {"rate_per_s": rate, "duration_s": duration, "shapes": shapes or "all distinct", "requests": len(descs),
           "completed": len(done),
           "errors": len(srv.done) - len(done), "wall_s": wall, "achieved_req_per_s": len(done) / wall,
           "gbs": total / wall / 1e9, "launches": srv.launches, **st}
    out["phases_p50_p99_ms"] = phase_stats(done)
    out["passed_waiting_head"] = srv.bypassed
    out["plans_evicted"] = srv.evicted
    out["longest_poll_round_ms"] = srv.max_round_s * 1e3
    out["gc_pauses"] = {"count": len(pauses), "longest_ms": max((p for _, p in pauses), default=0.0) * 1e3,
                        "full_collections": sum(1 for g, _ in pauses if g == 2)}
    errs = sorted({r.error for r in srv.done if r.error})
    if errs:
        out["error_messages"] = errs[:3]
    for key in ("plan_cache_hits", "plan_cache_misses"):
        if hasattr(srv, key):
            out[key] = getattr(srv, key)
    return out


def measure_serving_short(args):
    """Config 5's serving loop (concurrent launch slots) for a short run at
    the offered 2000 requests/s and at a sub-saturating 100 requests/s."""
    out = {}
    for rate in (args.rate, args.low_rate):
        out[f"{rate:g}/s"] = serve_trace(rate, args.extras_serve_s, args.budget_gb, 8, 1)
        out[f"{rate:g}/s recurring shapes"] = serve_trace(rate, args.extras_serve_s, args.budget_gb, 8, 1,
                                                          shapes=args.shapes)
    out["config"] = (f"serving: Poisson arrivals of the seven collectives, P in {{8,16,64}}, 1 KiB..256 MiB per "
                     f"rank, fp32/bf16/int32, {args.budget_gb} GB budget, 8 concurrent launch slots, "
                     f"{args.extras_serve_s:g} s of arrivals per rate; 'recurring shapes': the same arrivals drawn "
                     f"from {args.shapes} shapes (memoized plans reused); the 60 s run: --workload serve")
    return out


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist_init("nccl")

    import __graft_entry__
    __graft_entry__.build()

    xs = None
    if args.workload == "allreduce64":
        from synth import scaled_normal_ranks
        xs = scaled_normal_ranks(WORKLOADS["allreduce64"]["ranks"],
                                 (args.bytes_per_rank or WORKLOADS["allreduce64"]["bytes_per_rank"]) // 4, seed=0)
    elif args.dtype != "f32":
        raise SystemExit("the seven-collective workload is fp32")
    r = measure_collectives(args, device, world, args.workload, args.dtype, xs=xs)
    peak = r["peak"]

    extras = {}
    if world == 1 and rank == 0 and args.workload == "seven" and not args.no_extras and not args.kinds:
        t = time.perf_counter()
        extras["allreduce64"] = measure_allreduce64(args, device)
        extras["batch256"] = measure_batch(args, device, 3)
        extras["serving"] = measure_serving_short(args)
        extras["extras_wall_s"] = time.perf_counter() - t

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "seven":
        cpu = cpu_baseline(args.cpu_budget)

    default_run = (args.workload == "seven" and not args.kinds and args.ring == 1 and not args.bytes_per_rank
                   and not args.item_bytes and not args.ctas_per_sm and not args.threads and args.order is None
                   and not args.slot_items)
    # DRAM bytes of an average executor launch of the default workload, from
    # the committed ncu capture (null for other workloads or options, or once
    # the executor sources have changed since the capture)
    step_traffic = recorded_traffic() if default_run else None
    nk = len(r["collectives"])
    traffic = step_traffic / nk if step_traffic else None
    line = {
        "metric": METRIC, "value": r["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic",
        "config": workload_config(args.workload, world, args.dtype,
                                  {**({"ring": args.ring} if args.ring > 1 else {}),
                                   **({"bytes_per_rank": args.bytes_per_rank} if args.bytes_per_rank else {}),
                                   **({"collectives": args.kinds.split(",")} if args.kinds else {})}),
        "timing": {"method": "CUDA graph of one step (one start per collective"
                             + (", each on its own stream forked from the step's stream and joined back"
                                if len(r["collectives"]) > 1 else "")
                             + f"), replayed; blocks of {args.steps} replays bracketed by CUDA events until >= "
                             f"{args.min_seconds:g} s; median block; 'eager': the starts in order on one stream "
                             "through start / wait; per collective: 'ms' from eager starts bracketed by events, "
                             "'graph_ms' from a graph of ten starts of that collective, replayed",
                   "blocks": r["blocks"], "timed_s": r["timed_s"],
                   "block_ms": r["block_ms"], "eager": r["eager"]},
        "roofline": {"bound": "hbm", "achieved": r["value"] / world, "peak": peak, "unit": "GB/s",
                     "frac": r["frac"], "peak_source": r["peak_kind"],
                     "traffic": traffic, "traffic_per_step": step_traffic,
                     "schedule_bytes_per_launch": r["step_bytes"] / nk, "kernel": "hiccl_exec_kernel"},
        "clocks": r["clocks"], "gpu_launches": r["launches"] * world,
        "e2e": r["e2e"], "collectives": r["collectives"], "cpu_baseline": cpu,
    }
    if r["accuracy"]:
        line["accuracy"] = r["accuracy"]
    if r["grouped"]:
        g = dict(r["grouped"])
        g["frac"] = g["gbs"] / world / peak
        line["grouped_step"] = g
    if r["serial"]:
        g = dict(r["serial"])
        g["frac"] = g["gbs"] / world / peak
        line["serial_step"] = g
    if extras:
        line["allreduce64"] = extras["allreduce64"]
        line["batch256"] = extras["batch256"]
        line["serving"] = extras["serving"]
        head = extras["serving"].get(f"{args.rate:g}/s", {})
        line["p50_ms"], line["p99_ms"] = head.get("p50_ms"), head.get("p99_ms")
        line["extras_wall_s"] = extras["extras_wall_s"]
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist_init("nccl")
    import __graft_entry__
    __graft_entry__.build()
    clocks = ClockSampler(local)
    clocks.start()
    b = measure_batch(args, device, args.steps)
    clk = clocks.stop()
    tb, tg = aggregate(b["schedule_bytes"] * args.steps, b["graph_ms"] / 1e3 * args.steps, device)
    peak, peak_kind = measured_peak()
    gbs = tb / tg / 1e9
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": 3, "ms_per_step": b["graph_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": b["config"], "collectives": 256, "parallelism": f"replicas{world}",
                   "tuned_configs": b["tuned_configs"]},
        "roofline": {"bound": "hbm", "achieved": gbs / world, "peak": peak, "unit": "GB/s",
                     "frac": gbs / world / peak, "peak_source": peak_kind, "traffic": None,
                     "kernel": "hiccl_exec_kernel"},
        "clocks": clk, "gpu_launches": args.steps * world, "batch": b,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving workload (config 5): Poisson arrivals (synth.poisson_requests
    seed 0) of the seven collectives, P in {8, 16, 64} ({2,4}, {4,4},
    {4,4,4}), per-rank sizes log-uniform 1 KiB .. 256 MiB, fp32 / bf16 /
    int32, admitted under a 64 GB device-memory budget with continuous
    batching (serving.Server: 8 launch slots, requests overlapping on the
    device; and grouped launches of up to 16 requests on 2 slots).  The same
    arrival trace is also served one launch at a time (1 slot).  Reports p50
    / p99 latency and the aggregate schedule GB/s of each."""
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist_init("nccl")
    import __graft_entry__
    __graft_entry__.build()

    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    for rate in (args.rate, args.low_rate):
        out[f"{rate:g}/s"] = {"batched": serve_trace(rate, args.duration, args.budget_gb, 8, 1),
                              "grouped": serve_trace(rate, args.duration, args.budget_gb, 2, 16),
                              "one_launch_at_a_time": serve_trace(rate, args.duration, args.budget_gb, 1, 1),
                              "batched_recurring_shapes": serve_trace(rate, args.duration, args.budget_gb, 8, 1,
                                                                      shapes=args.shapes)}
    clk = clocks.stop()
    head = out[f"{args.rate:g}/s"]["batched"]
    peak, peak_kind = measured_peak()
    line = {
        "metric": METRIC, "value": head["gbs"], "unit": "GB/s", "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": head["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+bf16+i32", "data": "synthetic",
        "config": {"workload": f"serving: Poisson {args.rate:g} requests/s for {args.duration:g} s of the seven "
                               "collectives, P in {8,16,64}, 1 KiB..256 MiB per rank, fp32/bf16/int32, "
                               f"{args.budget_gb} GB budget, continuous batching", "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "achieved": head["gbs"], "peak": peak, "unit": "GB/s",
                     "frac": head["gbs"] / peak, "peak_source": peak_kind, "traffic": None,
                     "kernel": "hiccl_exec_kernel"},
        "clocks": clk, "serving": out, "p50_ms": head.get("p50_ms"), "p99_ms": head.get("p99_ms"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="steps (graph replays) per timed block")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--min-seconds", type=float, default=1.0, help="length of the timed region (blocks of --steps)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=14.0)
    ap.add_argument("--ref-budget", type=float, default=7.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only (no 64 MiB All-reduce payloads, batch of 256, served run)")
    ap.add_argument("--extras-serve-s", type=float, default=5.0, help="seconds of arrivals per rate in the default line")
    ap.add_argument("--item-bytes", type=int, default=0, help="executor work-item size (0: library default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="executor CTAs per SM (0: library default)")
    ap.add_argument("--workload", default="seven", choices=sorted(WORKLOADS) + ["batch256", "serve"])
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: offered requests per second")
    ap.add_argument("--low-rate", type=float, default=100.0, help="serve: a sub-saturating rate")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--budget-gb", type=int, default=64, help="serve: device-memory budget")
    ap.add_argument("--shapes", type=int, default=64, help="serve: request shapes of the recurring-shape runs")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "fp8"],
                    help="payload of the allreduce64 workload (accumulation is FP32)")
    ap.add_argument("--kinds", default="", help="comma-separated subset of the seven collectives (profiling)")
    ap.add_argument("--threads", type=int, default=0, help="executor threads per CTA (0: library default)")
    ap.add_argument("--order", type=int, default=None, help="work order: 0 pipeline slots, 1 stage depth")
    ap.add_argument("--ring", type=int, default=1, help="ring(n) of the hybrid ring+tree topology (1: tree)")
    ap.add_argument("--slot-items", type=int, default=0, help="items a pipeline slot is spread over (0: library default)")
    ap.add_argument("--bytes-per-rank", type=int, default=0,
                    help="override the workload's per-rank bytes (profiling of a smaller case; 0: the workload's)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
