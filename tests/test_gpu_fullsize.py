"""Parity at the full workload sizes, in the launch configuration the
benchmark times: the seven collectives of P = 64 virtual ranks over
{4,4,4} with 4 MiB fp32 per rank, stripe 4, pipeline 8, and All-reduce with
P = 32 over {4, 8} at 64 MiB per rank, every result compared in full."""
import numpy as np
import pytest

from oracle import semantics as S
from synth import scaled_normal_ranks, uniform_ranks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _run(kind, P, d, h, s, m, x):
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    bufs = C.Buffers(kind, P, d, torch.float32)
    bufs.send.copy_(torch.from_numpy(x[:, :bufs.ls]))
    bufs.recv.fill_(-3.0)
    comm = H.Comm(P, "f32")
    C.compose(comm, kind, d, bufs.send_ptrs(), bufs.recv_ptrs())
    comm.init(h, s, m)
    comm.start()
    comm.wait()
    out = bufs.recv.cpu().numpy()
    comm.destroy()
    return out


def _expected_seven(kind, xs, d, h):
    P = len(xs)
    if kind == "broadcast":
        exp = S.def_broadcast(xs, 0)
    elif kind == "scatter":
        exp = S.def_scatter(xs, 0)
    elif kind == "gather":
        exp = [None] * P
        exp[0] = np.concatenate([v[:d] for v in xs])
    elif kind == "allgather":
        exp = S.def_allgather([v[:d] for v in xs])
    elif kind == "reducescatter":
        exp = S.def_reducescatter(xs, h)
    elif kind == "allreduce":
        exp = S.def_allreduce(xs, h)
    else:
        exp = S.def_alltoall(xs)
    return exp


def _check(kind, y, exp):
    for r in range(len(exp)):
        if exp[r] is None:
            assert np.all(y[r] == -3.0), (kind, r)
        else:
            assert np.array_equal(y[r].view(np.uint32), exp[r].view(np.uint32)), (kind, r)


SEVEN = ["broadcast", "scatter", "gather", "allgather", "reducescatter", "allreduce", "alltoall"]


@pytest.mark.parametrize("kind", SEVEN)
def test_seven_collectives_full_size(kind):
    P, h = 64, [4, 4, 4]
    d = (4 << 20) // 4 // P
    x = uniform_ranks(P, d * P, seed=1)
    y = _run(kind, P, d, h, 4, 8, x)
    _check(kind, y, _expected_seven(kind, [x[r] for r in range(P)], d, h))


def test_seven_collectives_concurrent_graph_full_size():
    """The benchmark's step as it is timed: the seven communicators' starts
    captured in one CUDA graph, each on its own stream forked from the
    graph's stream (their launches overlap on the device), replayed twice;
    after each replay every receive buffer of every collective equals the
    oracle's in full."""
    import torch

    import bench
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    P, h = 64, [4, 4, 4]
    d = (4 << 20) // 4 // P
    x = uniform_ranks(P, d * P, seed=4)
    xs = [x[r] for r in range(P)]
    dev = torch.device("cuda", 0)
    comms, bufs = {}, {}
    for kind in SEVEN:
        b = C.Buffers(kind, P, d, torch.float32, dev)
        b.send.copy_(torch.from_numpy(x[:, :b.ls]))
        comm = H.Comm(P, "f32")
        C.compose(comm, kind, d, b.send_ptrs(), b.recv_ptrs())
        comm.init(h, 4, 8)
        comms[kind], bufs[kind] = comm, b
    graph = bench._graph_of(comms, SEVEN, dev, concurrent=True)
    exp = {kind: _expected_seven(kind, xs, d, h) for kind in SEVEN}
    for _ in range(2):
        for kind in SEVEN:
            bufs[kind].recv.fill_(-3.0)
        torch.cuda.synchronize(dev)
        graph.replay()
        torch.cuda.synchronize(dev)
        for kind in SEVEN:
            _check(kind, bufs[kind].recv.cpu().numpy(), exp[kind])
    del graph
    for c in comms.values():
        c.destroy()


def test_allreduce_64mib_full():
    """All-reduce at 64 MiB per rank (P = 32 over {4, 8}, stripe 1, pipeline
    16): every receive buffer equals the oracle's fold of all 16,777,216
    values bit for bit."""
    P, h = 32, [4, 8]
    n = 16 << 20                     # 64 MiB of fp32 per rank
    d = n // P
    x = scaled_normal_ranks(P, n, seed=3)
    y = _run("allreduce", P, d, h, 1, 16, x)
    expect = S.nested_fold({r: x[r] for r in range(P)}, h).view(np.uint32)
    for r in range(P):
        assert np.array_equal(y[r].view(np.uint32), expect), r


def test_buffers_beyond_four_gib():
    """Byte offsets past 2**32 (a 4.5 GiB buffer per rank, 1.2 G values):
    a Broadcast over {2, 2} with stripe 2 and pipeline 4 and a Reduce of the
    same size, checked on sampled values (the generators fill the buffers on
    the device; the expected values are formed from the same samples)."""
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    P, h = 4, [2, 2]
    n = (9 << 29) // 4 // P * P              # 4.5 GiB of fp32 per rank
    d = n // P
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    for kind in ("broadcast", "reduce"):
        b = C.Buffers(kind, P, d, torch.float32)
        b.send.uniform_(-1.0, 1.0, generator=g)
        b.recv.fill_(-3.0)
        comm = H.Comm(P, "f32")
        C.compose(comm, kind, d, b.send_ptrs(), b.recv_ptrs())
        comm.init(h, 2, 4)
        comm.start()
        comm.wait()
        rng = np.random.Generator(np.random.PCG64(3))
        idx = np.unique(np.concatenate([rng.integers(0, n, 20000), [0, n - 1, (1 << 30) - 1, 1 << 30, n // 2]]))
        ti = torch.from_numpy(idx).cuda()
        xs = b.send[:, ti].cpu().numpy()
        ys = b.recv[:, ti].cpu().numpy()
        if kind == "broadcast":
            for r in range(P):
                assert np.array_equal(ys[r].view(np.uint32), xs[0].view(np.uint32)), r
        else:
            expect = S.nested_fold({r: xs[r] for r in range(P)}, h)
            assert np.array_equal(ys[0].view(np.uint32), expect.view(np.uint32))
            assert np.all(ys[1:] == -3.0)
        comm.destroy()
        del b
        torch.cuda.empty_cache()


def test_batch256_grouped_graph_full():
    """Config 4 at full size, in the launch configuration the benchmark times:
    the 256 collectives of the batch (All-gather / Reduce-scatter /
    All-reduce, P in {8, 16, 32}, two-level hierarchies, 4 KiB .. 16 MiB per
    rank, fp32 and bf16; synth.batch_mix seed 0), stripe, pipeline and
    executor knobs autotuned per shape, run as one grouped launch replayed
    from a CUDA graph.  Every receive buffer of every collective equals the
    oracle's result for that collective alone, bit for bit."""
    import math

    import torch

    from oracle import lowprec as LP
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    from synth import batch_mix, rng

    descs = batch_mix(256, seed=0)
    stream = torch.cuda.current_stream()
    comms, bufs, tuned = [], [], {}

    def inputs(i, dsc, ls):
        x = rng(7000 + i).uniform(-1.0, 1.0, size=(dsc["P"], ls)).astype(np.float32)
        return x if dsc["dtype"] == "f32" else LP.f32_to_bf16(x)

    for i, dsc in enumerate(descs):
        P, h, dt = dsc["P"], dsc["hierarchy"], dsc["dtype"]
        es = 4 if dt == "f32" else 2
        d = dsc["bytes_per_rank"] // es // P
        b = C.Buffers(dsc["kind"], P, d, torch.float32 if dt == "f32" else torch.int16)
        b.send.view(torch.uint8).copy_(torch.from_numpy(inputs(i, dsc, b.ls).view(np.uint8)))
        b.recv.view(torch.uint8).fill_(0xA5)
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
            tuned[key] = comm.autotune(stream, tune_method=True)   # leaves the communicator on its best knobs
        comms.append(comm)
        bufs.append(b)
    for b in bufs:                               # autotuning ran the collectives: start from sentinels again
        b.recv.view(torch.uint8).fill_(0xA5)
    grp = H.Comm.group(comms)
    gs = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        grp.start(gs)
    graph.replay()
    torch.cuda.synchronize()
    for i, (dsc, b) in enumerate(zip(descs, bufs)):
        P, h, dt = dsc["P"], dsc["hierarchy"], dsc["dtype"]
        x = inputs(i, dsc, b.ls)
        xs = [x[r] for r in range(P)]
        fold_dt = None if dt == "f32" else dt
        if dsc["kind"] == "allgather":
            exp = S.def_allgather(xs)
        elif dsc["kind"] == "reducescatter":
            exp = S.def_reducescatter(xs, h, fold_dt)
        else:
            exp = S.def_allreduce(xs, h, fold_dt)
        got = b.recv.view(torch.uint8).cpu().numpy()
        for r in range(P):
            assert np.array_equal(got[r], exp[r].view(np.uint8)), (i, dsc, r)
    grp.destroy()
    for c in comms:
        c.destroy()
