"""Executor trace (HICCL_OPT_TRACE): one record per work item in ticket
order whose four timestamps follow the item's life -- staging began, handed
to the data warps, data done, successors released -- and whose last field
is the first step of the item's record in the uploaded table."""
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("kind,h,s,m", [("allreduce", [4, 4], 2, 2), ("alltoall", [2, 8], 4, 1)])
def test_trace_follows_every_item(kind, h, s, m):
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    P, d = 16, 4096
    b = C.Buffers(kind, P, d, torch.float32, "cuda")
    b.send.uniform_()
    b.recv.zero_()
    c = H.Comm(P, "f32")
    c.set_option(H.OPT_TRACE, 1)
    C.compose(c, kind, d, b.send_ptrs(), b.recv_ptrs())
    c.init(h, s, m)
    for _ in range(2):
        c.start()
        c.wait()
    info = c.plan_info()
    tr = np.array(c.trace(), dtype=np.uint64)
    assert tr.shape == (info["items"], 6)
    assert (tr[:, 0] > 0).all()
    assert (tr[:, 0] <= tr[:, 1]).all() and (tr[:, 1] <= tr[:, 2]).all() and (tr[:, 2] <= tr[:, 3]).all()
    recs, items = c.image()
    first = [struct.unpack_from("<I", recs, int(rec) * 16)[0] for rec in items[:, 0]]
    assert tr[:, 5].tolist() == first
    c.destroy()
