"""A withheld dependency makes the executor's bounded wait run out: the
launch ends by itself, hiccl_wait reports HICCL_ERR_TIMEOUT, and the same
communicator then runs correctly again.  Nothing here faults the GPU: the
fault is a raised counter target set from the host."""
import time

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


def test_withheld_dependency_times_out_and_recovers():
    import torch
    from paper_2408_05962_gb300 import hiccl as H
    from tests._bridge import register

    P, d, h = 8, 4096, [2, 4]
    prog = PR.allreduce(P, d)
    mem0 = fill(prog, 9)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    dev = {k: torch.from_numpy(v.copy()).cuda() for k, v in mem0.items()}
    comm = register(prog, lambda r: int(dev[r.key].data_ptr()) + 4 * r.off)
    comm.set_option(H.OPT_TIMEOUT_NS, 50_000_000)          # 50 ms
    comm.init(h, 2, 2)
    steps = comm.steps()
    victim = next(i for i, st in enumerate(steps) if st["preds"])
    comm.withhold(victim, 1)
    t0 = time.time()
    comm.start()
    with pytest.raises(H.HicclError) as e:
        comm.wait()
    assert e.value.status == H.ERR_TIMEOUT
    assert time.time() - t0 < 20.0
    # the first wait to run out belongs to the victim, to a step staged in the
    # same work item (same pipeline slot), or to one that depends on those;
    # nothing of an earlier slot can be held up
    import re
    reported = int(re.search(r"step (\d+)", e.value.message).group(1))
    assert 0 <= reported < len(steps)
    assert steps[reported]["slot"] >= steps[victim]["slot"]
    # restore: the reset communicator runs correctly
    comm.withhold(victim, 0)
    for k, v in mem0.items():
        dev[k].copy_(torch.from_numpy(v))
    comm.start()
    comm.wait()
    for k in ref:
        assert np.array_equal(dev[k].cpu().numpy().view(np.uint32), ref[k].view(np.uint32)), k
    # a second launch also works (counters re-armed)
    comm.start()
    comm.wait()
    comm.destroy()
