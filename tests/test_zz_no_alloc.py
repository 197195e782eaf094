"""hiccl_run_static: running a planned communicator without any device
allocation, for callers that cannot call cudaMalloc themselves (code under a
caller-owned memory pool or budget, or inside an allocator callback).  Its
output must equal the regular hiccl_init / hiccl_start / hiccl_wait path bit
for bit -- the tolerance of every other parity test here -- on two calls in a
row (the second call finds the fixed device array holding the first call's
contents and must clear what has to start at zero).  This file is collected
last so that a failure here cannot hide another test's result."""
import numpy as np
import pytest

from oracle import programs as PR
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


def _host(dev):
    return {k: t.cpu().numpy() for k, t in dev.items()}


@pytest.mark.parametrize("name,P,h,s,m", [("allreduce", 8, [2, 4], 1, 1), ("allreduce", 8, [2, 4], 2, 2),
                                          ("reducescatter", 16, [4, 4], 4, 2), ("alltoall", 8, [2, 2, 2], 2, 3)])
def test_static_matches_allocating_path(name, P, h, s, m):
    import torch
    from paper_2408_05962_gb300 import hiccl as H
    from tests._bridge import register

    prog = PR.BUILDERS[name](P, 2053)
    mem0 = fill(prog, 17)
    dev = _device_buffers(mem0)

    def addr(r):
        return int(dev[r.key].data_ptr()) + 4 * r.off

    # the existing entry points (they allocate the table, counters, relays)
    ref_comm = register(prog, addr)
    ref_comm.init(h, s, m)
    ref_comm.start()
    ref_comm.wait()
    ref = _host(dev)
    ref_comm.destroy()

    # the allocation-free entry point on a communicator that is only planned
    comm = register(prog, addr)
    comm.plan(h, s, m)
    for call in range(2):
        _reset(dev, mem0)
        torch.cuda.synchronize()
        comm.run_static()
        got = _host(dev)
        for k in ref:
            assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), (call, k)
    comm.destroy()


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
