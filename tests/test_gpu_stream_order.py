"""Stream order around executor launches: the executor's launches let the
next kernel of the stream become resident early (programmatic dependent
launch), so these tests check that nothing is read or written out of stream
order -- a kernel writing the send buffers right before a start, a start
right after another collective that produces its inputs, and a kernel
reading the receive buffers right after it."""
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


def test_inputs_written_by_the_previous_kernel_are_seen():
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    P, h, d = 16, [4, 4], 4099
    b = C.Buffers("allreduce", P, d, torch.float32)
    comm = H.Comm(P, "f32")
    C.compose(comm, "allreduce", d, b.send_ptrs(), b.recv_ptrs())
    comm.init(h, 4, 4)
    s = torch.cuda.current_stream()
    prog = PR.allreduce(P, d)
    for it in range(6):
        mem0 = fill(prog, 500 + it)
        host = torch.from_numpy(np.stack([mem0[("send", r)] for r in range(P)]))
        staged = host.cuda()
        torch.cuda.synchronize()
        b.recv.fill_(float(it))            # stale values that must be overwritten
        b.send.copy_(staged)               # kernel writing the inputs, then the start, no sync
        comm.start(s)
        out = b.recv.clone()               # kernel reading the results right after
        comm.wait()
        ref = {k: v.copy() for k, v in mem0.items()}
        S.run_program(prog, ref, h)
        got = out.cpu().numpy()
        for r in range(P):
            assert np.array_equal(got[r].view(np.uint32), ref[("recv", r)].view(np.uint32)), (it, r)


def test_chained_collectives_on_one_stream():
    """Reduce-scatter feeding an All-gather of its results (two communicators,
    consecutive launches without a host synchronization) equals All-reduce."""
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    P, h, d = 8, [2, 4], 2053
    rs = C.Buffers("reducescatter", P, d, torch.float32)
    ag = C.Buffers("allgather", P, d, torch.float32)
    x = fill(PR.allreduce(P, d), 77)
    send = np.stack([x[("send", r)] for r in range(P)])
    rs.send.copy_(torch.from_numpy(send))
    c1 = H.Comm(P, "f32")
    C.compose(c1, "reducescatter", d, rs.send_ptrs(), [int(p) for p in ag.send_ptrs()])
    c1.init(h, 2, 2)
    c2 = H.Comm(P, "f32")
    C.compose(c2, "allgather", d, ag.send_ptrs(), ag.recv_ptrs())
    c2.init(h, 2, 2)
    s = torch.cuda.current_stream()
    for _ in range(3):
        ag.send.zero_()
        ag.recv.zero_()
        c1.start(s)
        c2.start(s)
        c1.wait()
        c2.wait()
    got = ag.recv.cpu().numpy()
    want = S.def_allreduce([send[r] for r in range(P)], h)
    for r in range(P):
        assert np.array_equal(got[r].view(np.uint32), want[r].view(np.uint32)), r


def test_grid_changes_between_starts():
    """One communicator started back to back with its grid changing between
    starts (CTAs per SM 2 -> 1 -> 2), then a CUDA graph captured with the
    last grid and replayed between further starts: work items are numbered
    from one ticket counter over all launches, which the library resets when
    the grid changes, so every result equals the oracle's."""
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    P, h, d = 16, [4, 4], 8195
    b = C.Buffers("allreduce", P, d, torch.float32)
    comm = H.Comm(P, "f32")
    C.compose(comm, "allreduce", d, b.send_ptrs(), b.recv_ptrs())
    comm.init(h, 2, 4)
    prog = PR.allreduce(P, d)
    graph = None
    plan = [(2, False), (1, False), (1, False), (2, False), (2, True), (2, False), (2, True), (2, True)]
    for it, (per_sm, replay) in enumerate(plan):
        mem0 = fill(prog, 700 + it)
        b.send.copy_(torch.from_numpy(np.stack([mem0[("send", r)] for r in range(P)])))
        b.recv.fill_(-1.0)
        torch.cuda.synchronize()
        comm.set_option(H.OPT_CTAS_PER_SM, per_sm)
        if replay:
            if graph is None:
                gs = torch.cuda.Stream()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=gs):
                    comm.start(gs)
            graph.replay()
            torch.cuda.synchronize()
        else:
            comm.start()
            comm.wait()
        ref = {k: v.copy() for k, v in mem0.items()}
        S.run_program(prog, ref, h)
        got = b.recv.cpu().numpy()
        for r in range(P):
            assert np.array_equal(got[r].view(np.uint32), ref[("recv", r)].view(np.uint32)), (it, r)
    comm.destroy()
