"""hiccl_run_static: running a planned communicator without any device
allocation, for callers that cannot call cudaMalloc themselves (code under a
caller-owned memory pool or budget, or inside an allocator callback).

Its output must equal the regular hiccl_init / hiccl_start / hiccl_wait path
bit for bit -- the tolerance of every other parity test here -- and the
oracle's semantics, on several calls in a row.  Calls share one fixed device
array that keeps the previous call's contents, so the calls alternate
between communicators whose tables, counters and relay buffers have
different sizes and offsets: a call that did not clear what must start at
zero would inherit another plan's counters.  This file is collected last so
that a failure here cannot hide another test's result."""
import numpy as np
import pytest

from oracle import programs as PR
from oracle import semantics as S
from oracle.model import DTYPES
from tests._cases import fill

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _device_buffers(mem0):
    import torch
    return {k: torch.from_numpy(v.copy()).cuda() for k, v in mem0.items()}


def _reset(dev, mem0):
    import torch
    for k, v in mem0.items():
        dev[k].copy_(torch.from_numpy(v))
    torch.cuda.synchronize()


def _host(dev):
    return {k: t.cpu().numpy() for k, t in dev.items()}


def _same(a, b, what):
    for k in a:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), (what, k)


class Case:
    """One program on its own device buffers: the oracle's result, the
    allocating path's result, and a communicator that is only planned."""

    def __init__(self, name, P, h, s, m, count, seed):
        from tests._bridge import register
        self.prog = PR.BUILDERS[name](P, count)
        self.h = h
        self.mem0 = fill(self.prog, seed)
        self.dev = _device_buffers(self.mem0)
        ref = {k: v.copy() for k, v in self.mem0.items()}
        S.run_program(self.prog, ref, h)
        self.oracle = ref
        esize = DTYPES[self.prog.dtype].itemsize

        def addr(r):
            return int(self.dev[r.key].data_ptr()) + esize * r.off

        alloc = register(self.prog, addr)
        alloc.init(h, s, m)
        alloc.start()
        alloc.wait()
        self.allocating = _host(self.dev)
        alloc.destroy()
        _same(self.oracle, self.allocating, "allocating path vs oracle")
        self.comm = register(self.prog, addr)
        self.comm.plan(h, s, m)

    def run_static(self):
        _reset(self.dev, self.mem0)
        self.comm.run_static()
        got = _host(self.dev)
        _same(self.allocating, got, "static vs allocating path")
        _same(self.oracle, got, "static vs oracle")


@pytest.mark.parametrize("name,P,h,s,m", [("allreduce", 8, [2, 4], 1, 1), ("allreduce", 8, [2, 4], 2, 2),
                                          ("reducescatter", 16, [4, 4], 4, 2), ("alltoall", 8, [2, 2, 2], 2, 3)])
def test_static_matches_allocating_path_and_oracle(name, P, h, s, m):
    c = Case(name, P, h, s, m, 2053, 17)
    for _ in range(2):
        c.run_static()
    c.comm.destroy()


def test_static_alternating_communicators():
    """A, B, A, B, A: an all-to-all over {2,2,2} and a reduce-scatter over
    {4,4} (different step counts, so counters, control block and relays lie
    at different offsets of the shared array)."""
    a = Case("alltoall", 8, [2, 2, 2], 2, 3, 1031, 5)
    b = Case("reducescatter", 16, [4, 4], 4, 2, 2053, 6)
    assert a.comm.plan_info()["steps"] != b.comm.plan_info()["steps"]
    for c in (a, b, a, b, a):
        c.run_static()
    a.comm.destroy()
    b.comm.destroy()


def test_static_allocates_no_device_memory():
    """After a first call (which loads the module holding the array), further
    calls leave the device's free memory unchanged, and the communicator,
    only planned, still owns no device state (it cannot be started)."""
    import torch
    from paper_2408_05962_gb300 import hiccl as H

    c = Case("allreduce", 8, [2, 4], 2, 2, 4099, 9)
    c.run_static()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        c.comm.run_static()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    with pytest.raises(H.HicclError) as e:
        c.comm.start()
    assert e.value.status == H.ERR_STATE
    c.comm.destroy()


def test_static_rejects_plans_beyond_the_arena():
    from paper_2408_05962_gb300 import hiccl as H
    from tests._bridge import FakeAddresses, register

    # relay buffers alone exceed the fixed array: 64 ranks reduce-scattering
    # 1 MiB chunks need tens of MiB of partial sums
    prog = PR.reducescatter(64, 1 << 18)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([4, 4, 4], 1, 1)
    assert comm.plan_info()["scratch_bytes"] > H.STATIC_ARENA_BYTES
    with pytest.raises(H.HicclError) as e:
        comm.run_static()
    assert e.value.status == H.ERR_TOO_LARGE
    comm.destroy()
