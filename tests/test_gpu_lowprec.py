"""BF16 and block-scaled FP8-e4m3 payloads on the GPU, through the C ABI.

The executor decodes every input of a reduce step to binary32, folds in the
fixed order and encodes the step's result once (BF16: nearest even; FP8: a
fresh per-128-value scale amax/448 and nearest-even, saturating codes).  The
results must equal the oracle bit for bit, and stay within 1e-2 (BF16) and
6e-2 (FP8) relative L2 error of the FP64 sum of the decoded inputs."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import lowprec as LP
from oracle import programs as PR
from oracle import semantics as S
from tests._cases import fill
from tests._gpu import assert_bit_equal, run_on_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _parity(prog, h, s, m, seed=0, **kw):
    mem0 = fill(prog, seed)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    outs, _ = run_on_gpu(prog, h, s, m, mem0, **kw)
    for out in outs:
        assert_bit_equal(ref, out)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("name", ["allreduce", "reducescatter", "reduce", "allgather", "alltoall",
                                  "broadcast", "allreduce_single"])
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 1, 1), (8, [2, 4], 4, 3), (12, [2, 2, 3], 3, 2),
                                     (16, [4, 4], 4, 2)])
def test_lowprec_collectives(dtype, name, P, h, s, m):
    d = 1027 if dtype == "bf16" else 9      # BF16 ragged tails; FP8 in 128-value blocks
    _parity(PR.BUILDERS[name](P, d, dtype=dtype), h, s, m, seed=P * 3 + s)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_lowprec_wide_fanin_vector_path(dtype):
    """16 inputs per reduce step exceed the shared-memory fold (8) and take the
    vector-load path."""
    d = 515 if dtype == "bf16" else 5
    _parity(PR.allreduce(16, d, dtype=dtype), [16], 1, 2)
    _parity(PR.reducescatter(32, d, dtype=dtype), [2, 16], 2, 1)


def test_bf16_unaligned_element_path():
    _parity(PR.allreduce(8, 333, dtype="bf16"), [2, 4], 2, 2, misalign_elems=3)


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-6), ("bf16", 1e-2), ("fp8", 6e-2)])
def test_config3_allreduce_three_variants(dtype, tol):
    """All-reduce, P = 32 over {4, 8}, the same 16,777,216 values per rank
    (N(0,1) * 10**U(-3,3) per rank) as FP32, BF16 and FP8 payloads, in the
    launch configuration of the benchmark (stripe 1, pipeline 4).  The oracle
    folds all 16,777,216 values; every one of the 32 receive buffers equals it
    byte for byte, and the relative L2 error of each result buffer against
    the FP64 sum of the decoded inputs is within the stated bound."""
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    from synth import scaled_normal_ranks

    P, h = 32, [4, 8]
    n = 16 << 20
    d = n // P
    x = scaled_normal_ranks(P, n, seed=3)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as pool:
        enc = list(pool.map(lambda r: LP.encode(x[r], dtype), range(P)))
    del x
    tdt = {"f32": torch.float32, "bf16": torch.int16, "fp8": torch.uint8}[dtype]
    bufs = C.Buffers("allreduce", P, d, tdt)
    for r in range(P):
        bufs.send[r].view(torch.uint8).copy_(torch.from_numpy(enc[r].view(np.uint8)))
    bufs.recv.zero_()
    comm = H.Comm(P, dtype)
    C.compose(comm, "allreduce", d, bufs.send_ptrs(), bufs.recv_ptrs())
    comm.init(h, 1, 4)
    comm.start()
    comm.wait()
    comm.destroy()
    expect = S.nested_fold({r: enc[r] for r in range(P)}, h, None if dtype == "f32" else dtype)
    ref = S.fsum64([LP.payload_to_f32(e, dtype) for e in enc])
    del enc
    want = expect.view(np.uint8)
    nref = np.linalg.norm(ref)
    for r in range(P):
        got = bufs.recv[r].view(torch.uint8).cpu().numpy()
        assert np.array_equal(got, want), r
        err = float(np.linalg.norm(LP.payload_to_f32(got.view(expect.dtype), dtype).astype(np.float64) - ref) / nref)
        assert err <= tol, (r, err)
