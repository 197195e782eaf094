"""Benchmark of the hierarchical collective path on GB300.

Workload (one "step"): the seven standard collectives -- Broadcast, Scatter,
Gather, All-gather, Reduce-scatter, All-reduce (Listing 2) and All-to-all --
over P = 64 virtual ranks with hierarchy {4,4,4}, 4 MiB of fp32 per rank
(uniform[-1, 1], seed 0), stripe 4, pipeline 8; each collective is one start
of its own persistent communicator, all seven enqueued back to back.

Metric: device-memory GB/s of the schedule (each copy reads its bytes once
and writes them once per destination; an f-input reduce reads f times and
writes once), summed over the seven collectives and divided by their summed
kernel time, with the fraction of the measured HBM bandwidth; per-collective
GB/s and the paper-style d*p/t are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload seven|allreduce64]
Under torchrun each rank runs an independent replica on its own GPU
("replicas only": the virtual-rank path does not shard across devices).
"""
from __future__ import annotations

import argparse
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
STRIDE = 1          # oracle sample: every STRIDE-th primitive of each collective
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


def workload_config(extra=None, w="seven"):
    W = WORKLOADS[w]
    cfg = {"workload": W["name"], "ranks": W["ranks"], "hierarchy": W["hierarchy"], "stripe": W["stripe"],
           "pipeline": W["pipeline"], "bytes_per_rank": W["bytes_per_rank"], "collectives": list(W["kinds"]),
           "inputs": W["data"], "l2": W["l2"]}
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
    """GB/s of one plain pass of the end-to-end leg's copies, alone: every
    send buffer host -> device, then every receive buffer device -> host
    (CUDA events on one stream).  The end-to-end figure cannot exceed what the
    host link gives here; None where the measurement fails."""
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
        return {"h2d_gbs": hb / (ev[0].elapsed_time(ev[1]) * 1e6), "d2h_gbs": db / (ev[1].elapsed_time(ev[2]) * 1e6)}
    except Exception:   # a report field only: never fail the benchmark for it
        return {"h2d_gbs": None, "d2h_gbs": None}


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


def _oracle_plans(seed: int = 0):
    """The oracle's factorized schedules of the workload and their buffers
    (built once; factorization is initialization, not part of a step)."""
    if seed in _ORACLE_CACHE:
        return _ORACLE_CACHE[seed]
    import numpy as np

    from oracle import programs as PR
    from oracle.factorize import factorize
    from oracle.model import Program
    from synth import uniform_ranks

    d = BYTES_PER_RANK // 4 // P
    x = uniform_ranks(P, d * P, seed=seed)
    out = []
    for kind in KINDS:
        full = PR.BUILDERS[kind](P, d)
        prog = Program(P, full.dtype, dict(full.buffers), [ep[::STRIDE] for ep in full.epochs])
        plan = factorize(prog, HIER, STRIPE, PIPE)
        mem = prog.allocate()
        for r in range(P):
            mem[("send", r)][...] = x[r][:mem[("send", r)].shape[0]]
        for k, n in plan.scratch.items():
            mem[k] = np.zeros(n, dtype=np.float32)
        out.append((kind, plan, mem))
    _ORACLE_CACHE[seed] = out
    return out


def oracle_sample(budget_s: float, seed: int = 0):
    """Simulate the oracle's factorized schedule of the workload (all seven
    collectives) for at most ``budget_s`` seconds in all.
    Returns (schedule bytes simulated, seconds, description)."""
    from oracle.simulate import execute_op

    total_b, total_t = 0, 0.0
    per = budget_s / len(KINDS)
    for kind, plan, mem in _oracle_plans(seed):
        t0 = time.perf_counter()
        for op in plan.ops:
            execute_op(op, mem)
            total_b += op.n * 4 * (1 + len(op.dsts) if op.kind == "copy" else len(op.srcs) + 1)
            if time.perf_counter() - t0 > per:
                break
        total_t += time.perf_counter() - t0
    kept = "every primitive" if STRIDE == 1 else f"every {STRIDE}-th primitive"
    return total_b, total_t, (f"oracle schedule simulator (NumPy, 1 thread) on {kept} of each of the seven "
                              f"collectives, at most {per:.1f} s of simulation each (factorization untimed)")


def run_reference(args):
    world, rank, _ = dist_env()
    if world > 1:
        dist_init("gloo")
        if rank != 0:
            return
    for _ in range(args.warmup):
        oracle_sample(0.5)
    bs, ts = 0, 0.0
    for _ in range(args.steps):
        b, t, desc = oracle_sample(args.ref_budget)
        bs += b
        ts += t
    gbs = bs / ts / 1e9
    line = {"metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ts / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(), "impl": "reference",
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc},
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
    """Error of the reduced-precision All-reduce result, measured after the
    timed region with plain torch arithmetic: relative L2 and max-norm errors
    against the FP64 sum of the decoded inputs, and the relative L2 error
    against the FP64 sum of the unquantized binary32 sources."""
    import torch
    P = b.send.shape[0]
    y64 = torch.zeros(_decode_rows(b.send[:1], dtype).shape[1], dtype=torch.float64, device=device)
    x64 = torch.zeros_like(y64)
    for r in range(P):
        y64 += _decode_rows(b.send[r:r + 1], dtype)[0].double()
        x64 += torch.from_numpy(xs[r]).to(device).double()
    y = _decode_rows(b.recv[:1], dtype)[0].double()
    return {"rel_l2_vs_fp64_of_decoded": float((y - y64).norm() / y64.norm()),
            "rel_max_vs_fp64_of_decoded": float((y - y64).abs().max() / y64.abs().max()),
            "rel_l2_vs_fp64_of_unquantized": float((y - x64).norm() / x64.norm()),
            "bound_rel_l2": 1e-2 if dtype == "bf16" else 6e-2}


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist_init("nccl")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    from synth import uniform_ranks

    W = WORKLOADS[args.workload]
    Pw, hier, stripe, pipe = W["ranks"], W["hierarchy"], W["stripe"], W["pipeline"]
    bpr = args.bytes_per_rank or W["bytes_per_rank"]
    d = bpr // 4 // Pw                            # values per chunk (bytes of fp32 values per rank / P)
    dtype = args.dtype
    if args.workload == "seven":
        if dtype != "f32":
            raise SystemExit("the seven-collective workload is fp32")
        x = torch.from_numpy(uniform_ranks(Pw, d * Pw, seed=0))
    else:
        from synth import scaled_normal_ranks
        xs = scaled_normal_ranks(Pw, d * Pw, seed=0)
        if dtype == "bf16":       # round to nearest even on the upper 16 bits (payload encoding)
            t = torch.from_numpy(xs).view(torch.int32)
            x = ((t + 0x7FFF + ((t >> 16) & 1)) >> 16).to(torch.int16)
        elif dtype == "fp8":      # per-128-value block scales, e4m3 codes (payload encoding on the GPU)
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
        comm = H.Comm(Pw, dtype)
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
        C.compose(comm, kind, d, b.send_ptrs(), b.recv_ptrs())
        comm.init(hier, stripe, pipe)
        rd, wr = comm.hbm_bytes()
        comms[kind], bufs[kind], nbytes[kind] = comm, b, rd + wr
        pbytes[kind] = H.nbytes(H.DTYPES[dtype], d * Pw)   # the paper's d*p per collective
        mbytes[kind] = min_bytes(kind, Pw, pbytes[kind])
    stream = torch.cuda.current_stream(device)
    step_bytes = sum(nbytes.values())

    def one_step(evs=None):
        """All collectives back to back on one stream.  With ``evs`` (one
        event per collective plus one) each launch is bracketed; without,
        consecutive launches overlap their launch latency (programmatic
        dependent launch)."""
        for i, kind in enumerate(kinds):
            if evs is not None:
                evs[i].record(stream)
            comms[kind].start(stream)
        if evs is not None:
            evs[len(kinds)].record(stream)
        for kind in kinds:
            comms[kind].wait()

    for _ in range(max(args.warmup, 3)):
        one_step()
    torch.cuda.synchronize(device)

    # per-collective breakdown (untimed pass, events between the launches)
    per_kind = {kind: [] for kind in kinds}
    for _ in range(min(args.steps, 10)):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(kinds) + 1)]
        one_step(evs)
        torch.cuda.synchronize(device)
        for i, kind in enumerate(kinds):
            per_kind[kind].append(evs[i].elapsed_time(evs[i + 1]))

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step_evs[k][0].record(stream)
        one_step()
        step_evs[k][1].record(stream)
    torch.cuda.synchronize(device)
    wall = time.perf_counter() - t0
    barrier(device)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in step_evs]
    dev_s = sum(step_ms) / 1e3
    tot_bytes, tot_s = aggregate(step_bytes * args.steps, dev_s, device)
    gbs = tot_bytes / tot_s / 1e9
    peak, peak_kind = measured_peak()

    # end to end through the public API with host buffers (pinned), placed on
    # the NUMA node of the GPU's host link where sysfs names one
    numa = host_node_of(device)
    with cpus_of_node(numa):
        h_send = {k: torch.empty(bufs[k].send.shape, dtype=tdt, pin_memory=True) for k in kinds}
        h_recv = {k: torch.empty(bufs[k].recv.shape, dtype=tdt, pin_memory=True) for k in kinds}
        for k in kinds:
            h_send[k].copy_(bufs[k].send)
            h_recv[k].zero_()
    h2d = sum(t.numel() * t.element_size() for t in h_send.values())
    d2h = sum(t.numel() * t.element_size() for t in h_recv.values())
    # copies overlap the collectives: H2D of collective k+1 and D2H of
    # collective k-1 run on their own streams while collective k executes
    e2e_steps = max(1, min(args.steps, 3))
    s_in, s_out = torch.cuda.Stream(device), torch.cuda.Stream(device)
    t_e2e = 0.0
    for it in range(e2e_steps + 1):      # the first pass is an untimed warm-up
        if it == 1:
            barrier(device)
            torch.cuda.synchronize(device)
            t_e2e = time.perf_counter()
        ev_in = {k: torch.cuda.Event() for k in kinds}
        ev_out = {k: torch.cuda.Event() for k in kinds}
        with torch.cuda.stream(s_in):
            for k in kinds:
                bufs[k].send.copy_(h_send[k], non_blocking=True)
                ev_in[k].record(s_in)
        for k in kinds:
            stream.wait_event(ev_in[k])
            comms[k].start(stream)
            ev_out[k].record(stream)
            s_out.wait_event(ev_out[k])
            with torch.cuda.stream(s_out):
                h_recv[k].copy_(bufs[k].recv, non_blocking=True)
        for k in kinds:
            comms[k].wait()
        torch.cuda.synchronize(device)
    e2e_s = time.perf_counter() - t_e2e
    eb, es = aggregate(step_bytes * e2e_steps, e2e_s, device)
    host_link = host_copy_rates(h_send, h_recv, bufs, kinds, s_in, device)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "seven":
        b, t, desc = oracle_sample(args.cpu_budget)
        cpu = {"value": b / t / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc}

    accuracy = None
    if dtype in ("bf16", "fp8") and "allreduce" in bufs:
        accuracy = _lowprec_accuracy(bufs["allreduce"], dtype, xs, device)

    coll = {}
    for kind in kinds:
        med = statistics.median(per_kind[kind])
        coll[kind] = {"ms": med, "gbs": nbytes[kind] / med / 1e6, "frac": nbytes[kind] / med / 1e6 / peak,
                      "dp_over_t_gbs": pbytes[kind] / med / 1e6, "schedule_bytes": nbytes[kind],
                      "min_bytes": mbytes[kind], "min_gbs": mbytes[kind] / med / 1e6,
                      "level_bytes": comms[kind].level_bytes(), "steps": comms[kind].plan_info()["steps"]}
    # DRAM bytes of an average executor launch of the default workload, from
    # the committed ncu capture (null for other workloads or options, or once
    # the executor sources have changed since the capture)
    default_run = (args.workload == "seven" and not args.kinds and args.ring == 1 and not args.bytes_per_rank
                   and not args.item_bytes and not args.ctas_per_sm and not args.threads and args.order is None)
    step_traffic = recorded_traffic() if default_run else None
    traffic = step_traffic / len(kinds) if step_traffic else None
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": statistics.mean(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": workload_config(
            {"parallelism": f"replicas{world}", "payload": dtype, **({"ring": args.ring} if args.ring > 1 else {}),
             **({"bytes_per_rank": bpr} if args.bytes_per_rank else {})},
            args.workload),
        "roofline": {"bound": "hbm", "achieved": gbs / world, "peak": peak, "unit": "GB/s",
                     "frac": gbs / world / peak, "peak_source": peak_kind,
                     "traffic": traffic, "traffic_per_step": step_traffic,
                     "schedule_bytes_per_launch": step_bytes / len(kinds), "kernel": "hiccl_exec_kernel"},
        "clocks": clk, "gpu_launches": len(kinds) * args.steps * world,
        "e2e": {"value": eb / es / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "host_numa_node": numa, **host_link},
        "collectives": coll, "wall_ms_per_step": wall / args.steps * 1e3,
        "cpu_baseline": cpu,
    }
    if accuracy:
        line["accuracy"] = accuracy
    if rank == 0:
        print(json.dumps(line), flush=True)
    for c in comms.values():
        c.destroy()


def run_batch(args):
    """Batched workload: 256 collectives (All-gather / Reduce-scatter /
    All-reduce drawn uniformly, P from {8, 16, 32} with two-level
    hierarchies, per-rank sizes log-uniform 4 KiB .. 16 MiB, fp32 and bf16
    mixed; synth.batch_mix seed 0), stripe / pipeline / executor knobs chosen
    by the autotuner (one tuning per kind, P, hierarchy, payload and size
    octave).  Timed three ways on one stream: one launch per collective (all
    256 enqueued, then waited), one grouped launch, and the grouped launch
    replayed from a CUDA graph."""
    import math

    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist_init("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    from synth import batch_mix

    descs = batch_mix(256, seed=0)
    gen = torch.Generator(device=device)
    gen.manual_seed(0)
    comms, bufs, tuned = [], [], {}
    stream = torch.cuda.current_stream(device)
    total_bytes = 0
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

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(device)
        torch.cuda.synchronize(device)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / 1e3 / k

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t_sep = timed(separate, args.steps)
    t_grp = timed(grouped, args.steps)
    t_graph = timed(graph.replay, args.steps)
    clk = clocks.stop()
    tb, tg = aggregate(total_bytes * args.steps, t_graph * args.steps, device)
    peak, peak_kind = measured_peak()
    gbs = tb / tg / 1e9
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": 3, "ms_per_step": t_graph * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": "256 collectives (All-gather/Reduce-scatter/All-reduce), P in {8,16,32}, "
                               "two-level hierarchies, 4 KiB..16 MiB per rank log-uniform, fp32/bf16, "
                               "one persistent launch replayed from a CUDA graph; stripe, pipeline and "
                               "executor knobs autotuned", "collectives": 256, "parallelism": f"replicas{world}",
                   "tuned_configs": len(tuned)},
        "roofline": {"bound": "hbm", "achieved": gbs / world, "peak": peak, "unit": "GB/s",
                     "frac": gbs / world / peak, "peak_source": peak_kind, "traffic": None,
                     "kernel": "hiccl_exec_kernel"},
        "clocks": clk, "gpu_launches": args.steps * world,
        "batch": {"schedule_bytes": total_bytes, "one_launch_each_ms": t_sep * 1e3,
                  "grouped_ms": t_grp * 1e3, "graph_ms": t_graph * 1e3,
                  "one_launch_each_gbs": total_bytes / t_sep / 1e9, "grouped_gbs": total_bytes / t_grp / 1e9,
                  "graph_gbs": total_bytes / t_graph / 1e9, "speedup_vs_one_launch_each": t_sep / t_graph},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving workload: Poisson arrivals (synth.poisson_requests seed 0) of the
    seven collectives, P in {8, 16, 64} ({2,4}, {4,4}, {4,4,4}), per-rank sizes
    log-uniform 1 KiB .. 256 MiB, fp32 / bf16 / int32, admitted under a 64 GB
    device-memory budget with continuous batching (serving.Server: 8 launch
    slots, requests overlapping on the device; and grouped launches of up to
    16 requests on 2 slots).  The same arrival trace is also served one
    launch at a time (1 slot).  Reports p50 / p99 latency and the aggregate
    schedule GB/s of each."""
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist_init("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_05962_gb300.serving import Request, Server, latency_stats
    from synth import poisson_requests

    def serve(descs, slots, max_batch):
        srv = Server(args.budget_gb << 30, slots=slots, max_batch=max_batch, planners=8)
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
        srv.close()
        done = [r for r in srv.done if not r.error]
        st = latency_stats(done)
        total = sum(r.hbm_bytes for r in done)
        return {"requests": len(descs), "completed": len(done), "errors": len(srv.done) - len(done),
                "wall_s": wall, "achieved_req_per_s": len(done) / wall, "gbs": total / wall / 1e9,
                "launches": srv.launches, **st}

    out = {}
    for rate in (args.rate, args.low_rate):
        descs = poisson_requests(rate, args.duration, seed=0)
        out[f"{rate:g}/s"] = {"batched": serve(descs, 8, 1), "grouped": serve(descs, 2, 16),
                              "one_launch_at_a_time": serve(descs, 1, 1)}
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
        "serving": out, "p50_ms": head.get("p50_ms"), "p99_ms": head.get("p99_ms"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=14.0)
    ap.add_argument("--ref-budget", type=float, default=7.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--item-bytes", type=int, default=0, help="executor work-item size (0: library default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="executor CTAs per SM (0: library default)")
    ap.add_argument("--workload", default="seven", choices=sorted(WORKLOADS) + ["batch256", "serve"])
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: offered requests per second")
    ap.add_argument("--low-rate", type=float, default=100.0, help="serve: a sub-saturating rate")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    ap.add_argument("--budget-gb", type=int, default=64, help="serve: device-memory budget")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "fp8"],
                    help="payload of the allreduce64 workload (accumulation is FP32)")
    ap.add_argument("--kinds", default="", help="comma-separated subset of the seven collectives (profiling)")
    ap.add_argument("--threads", type=int, default=0, help="executor threads per CTA (0: library default)")
    ap.add_argument("--order", type=int, default=None, help="work order: 0 pipeline slots, 1 stage depth")
    ap.add_argument("--ring", type=int, default=1, help="ring(n) of the hybrid ring+tree topology (1: tree)")
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
