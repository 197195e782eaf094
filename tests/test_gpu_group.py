"""Batched execution: several collectives of different kinds, payloads and
hierarchies run as one persistent launch (hiccl_group), directly and replayed
from a CUDA graph; every member's result equals the oracle (and so its result
when run alone) bit for bit."""
import numpy as np
import pytest

from oracle import programs as PR
from oracle import semantics as S
from tests._cases import fill

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


MEMBERS = [("allreduce", 8, [2, 4], 4, 2, "f32", 1027), ("reducescatter", 16, [4, 4], 4, 3, "bf16", 515),
           ("allgather", 8, [2, 2, 2], 2, 2, "f32", 999), ("alltoall", 12, [2, 2, 3], 3, 1, "i32", 77),
           ("broadcast", 6, [2, 3], 3, 4, "bf16", 300), ("reduce", 16, [2, 8], 2, 2, "f32", 4097)]


def _setup():
    import torch
    from tests._bridge import register
    progs, refs, dev, comms = [], [], [], []
    for i, (name, P, h, s, m, dt, d) in enumerate(MEMBERS):
        prog = PR.BUILDERS[name](P, d, dtype=dt)
        mem0 = fill(prog, 100 + i)
        ref = {k: v.copy() for k, v in mem0.items()}
        S.run_program(prog, ref, h)
        bufs = {k: torch.from_numpy(v.view(np.uint8).copy()).cuda() for k, v in mem0.items()}
        es = np.dtype(next(iter(mem0.values())).dtype).itemsize
        comm = register(prog, lambda r, b=bufs, es=es: int(b[r.key].data_ptr()) + es * r.off)
        comm.plan(h, s, m)
        progs.append((prog, mem0))
        refs.append(ref)
        dev.append(bufs)
        comms.append(comm)
    return progs, refs, dev, comms


def _reset(progs, dev):
    import torch
    for (prog, mem0), bufs in zip(progs, dev):
        for k, v in mem0.items():
            bufs[k].copy_(torch.from_numpy(v.view(np.uint8)))


def _check(progs, refs, dev):
    for (prog, mem0), ref, bufs in zip(progs, refs, dev):
        for k in ref:
            got = bufs[k].cpu().numpy()
            assert np.array_equal(got, ref[k].view(np.uint8)), (prog.dtype, k)


def test_group_matches_members_run_alone():
    from paper_2408_05962_gb300 import hiccl as H
    progs, refs, dev, comms = _setup()
    g = H.Comm.group(comms)
    info = g.plan_info()
    assert info["steps"] == sum(c.plan_info()["steps"] for c in comms)
    assert g.hbm_bytes() == tuple(map(sum, zip(*[c.hbm_bytes() for c in comms])))
    for _ in range(2):
        _reset(progs, dev)
        g.start()
        g.wait()
        _check(progs, refs, dev)
    g.destroy()


def test_group_replayed_from_cuda_graph():
    import torch
    from paper_2408_05962_gb300 import hiccl as H
    progs, refs, dev, comms = _setup()
    g = H.Comm.group(comms)
    g.start()                      # one direct run first (warms the launch path)
    g.wait()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s):
        g.start(s)
    for _ in range(3):
        _reset(progs, dev)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        _check(progs, refs, dev)
    # a direct start after the replays still works
    _reset(progs, dev)
    g.start()
    g.wait()
    _check(progs, refs, dev)
    g.destroy()
