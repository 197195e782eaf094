"""BF16 and block-scaled FP8-e4m3 payloads on the GPU, through the C ABI.

The executor decodes every input of a reduce step to binary32, folds in the
fixed order and encodes the step's result once (BF16: nearest even; FP8: a
fresh per-128-value scale amax/448 and nearest-even, saturating codes).  The
results must equal the oracle bit for bit, and stay within 1e-2 (BF16) and
6e-2 (FP8) relative L2 error of the FP64 sum of the decoded inputs."""
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
    (N(0,1) * 10**U(-3,3) per rank) as FP32, BF16 and FP8 payloads; sampled
    elements (whole FP8 blocks) are compared with the oracle's fold bit for
    bit, and the relative L2 error against the FP64 sum of the decoded inputs
    is within the stated bound."""
    import torch
    from paper_2408_05962_gb300 import collectives as C
    from paper_2408_05962_gb300 import hiccl as H
    from synth import scaled_normal_ranks

    P, h = 32, [4, 8]
    n = 16 << 20
    d = n // P
    x = scaled_normal_ranks(P, n, seed=3)
    enc = [LP.encode(x[r], dtype) for r in range(P)]
    tdt = {"f32": torch.float32, "bf16": torch.int16, "fp8": torch.uint8}[dtype]
    bufs = C.Buffers("allreduce", P, d, tdt)
    host = np.stack([e.view(np.uint8) for e in enc])
    bufs.send.view(torch.uint8).copy_(torch.from_numpy(host))
    bufs.recv.zero_()
    comm = H.Comm(P, dtype)
    C.compose(comm, "allreduce", d, bufs.send_ptrs(), bufs.recv_ptrs())
    comm.init(h, 1, 4)
    comm.start()
    comm.wait()
    y = bufs.recv.view(torch.uint8).cpu().numpy()
    comm.destroy()
    g = np.random.Generator(np.random.PCG64(7))
    if dtype == "fp8":
        blk = np.unique(np.concatenate([g.integers(0, n // 128, 512), np.arange(0, n // 128, d // 128)]))
        vals = {r: enc[r][blk] for r in range(P)}
        expect = S.nested_fold(vals, h, dtype)
        for r in (0, 5, 31):
            got = y[r].view(LP.FP8_BLOCK_DTYPE)[blk]
            assert np.array_equal(got.view(np.uint8), expect.view(np.uint8)), r
        yv = LP.payload_to_f32(expect, dtype)
        ref = S.fsum64([LP.payload_to_f32(v, dtype) for v in vals.values()])
    else:
        idx = np.unique(np.concatenate([g.integers(0, n, 65536), np.arange(0, n, d), [n - 1]]))
        vals = {r: enc[r][idx] for r in range(P)}
        expect = S.nested_fold(vals, h, None if dtype == "f32" else dtype)
        view = np.float32 if dtype == "f32" else np.uint16
        for r in (0, 5, 31):
            got = y[r].view(view)[idx]
            assert np.array_equal(got.view(np.uint8), expect.view(np.uint8)), r
        yv = LP.payload_to_f32(expect, dtype)
        ref = S.fsum64([LP.payload_to_f32(v, dtype) for v in vals.values()])
    err = float(np.linalg.norm(yv - ref) / np.linalg.norm(ref))
    assert err <= tol, err
