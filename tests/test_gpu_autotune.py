"""The autotuner times candidate stripe / pipeline / executor configurations,
leaves the communicator on the fastest, and the tuned communicator still
computes the oracle's result bit for bit."""
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


@pytest.mark.parametrize("name,P,h,dt", [("allreduce", 16, [4, 4], "f32"), ("allgather", 8, [2, 4], "bf16")])
def test_autotune_keeps_results(name, P, h, dt):
    import torch
    from tests._bridge import register
    prog = PR.BUILDERS[name](P, 4096, dtype=dt)
    mem0 = fill(prog, 3)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    bufs = {k: torch.from_numpy(v.view(np.uint8).copy()).cuda() for k, v in mem0.items()}
    es = np.dtype(next(iter(mem0.values())).dtype).itemsize
    comm = register(prog, lambda r: int(bufs[r.key].data_ptr()) + es * r.off)
    comm.init(h, 4, 8)
    best = comm.autotune(tune_method=True)
    assert best["trials"] >= 8
    assert best["stripe"] in (1, 4) and best["pipeline"] in (1, 2, 4, 8)
    assert best["order"] in (0, 1) and best["us"] > 0
    for k, v in mem0.items():
        bufs[k].copy_(torch.from_numpy(v.view(np.uint8)))
    comm.start()
    comm.wait()
    for k in ref:
        assert np.array_equal(bufs[k].cpu().numpy(), ref[k].view(np.uint8)), k
    comm.destroy()
