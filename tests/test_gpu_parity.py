"""Parity of the CUDA executor with the oracle, through the C ABI.

Copies, int32 and FP32 reductions must be bit-exact against the oracle's
plain semantics (the hierarchical fixed-order sum); guard bands around every
buffer must be untouched."""
import numpy as np
import pytest

from oracle import programs as PR
from oracle import semantics as S
from oracle.hierarchy import all_factorizations
from tests._cases import fill, random_program
from tests._gpu import assert_bit_equal, run_on_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _parity(prog, h, s, m, seed=0, repeats=1, zero_frac=0.0, **kw):
    mem0 = fill(prog, seed, zero_frac)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    outs, comm = run_on_gpu(prog, h, s, m, mem0, repeats=repeats, **kw)
    for out in outs:
        assert_bit_equal(ref, out)
    return comm


COLL = PR.SEVEN + ("reduce", "allreduce_single", "broadcast_ag_scatter", "reduce_gather_rs",
                   "allgather_bcast_gather", "reducescatter_scatter_reduce", "allreduce_bcast_reduce")


@pytest.mark.parametrize("name", COLL)
@pytest.mark.parametrize("dtype", ["f32", "i32"])
@pytest.mark.parametrize("P,h,s,m,d", [(8, [2, 4], 1, 1, 1027), (8, [2, 4], 4, 3, 2053),
                                       (12, [2, 2, 3], 3, 2, 999), (16, [4, 4], 4, 8, 4099)])
def test_collectives_small(name, dtype, P, h, s, m, d):
    """Several 4 KiB segments per piece plus a ragged tail (d not a multiple
    of 4 elements)."""
    _parity(PR.BUILDERS[name](P, d, dtype=dtype), h, s, m, seed=P + s + m)


def test_config1_allreduce_repeated():
    """All-reduce of 65,536 fp32 per rank, P = 8, {2, 4}, s = 1, m = 1
    (Listing 2), uniform[-1, 1] seed 0; started three times on one
    communicator (dependency counters carry over between launches)."""
    from synth import uniform_ranks
    P, d = 8, 65536 // 8
    prog = PR.allreduce(P, d)
    mem0 = prog.allocate()
    x = uniform_ranks(P, d * P, seed=0)
    for r in range(P):
        mem0[("send", r)][...] = x[r]
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, [2, 4])
    outs, _ = run_on_gpu(prog, [2, 4], 1, 1, mem0, repeats=3)
    for out in outs:
        assert_bit_equal(ref, out)


@pytest.mark.parametrize("P", [2, 3, 4, 6, 8])
def test_random_programs(P):
    n = 0
    for h in all_factorizations(P):
        for s in sorted({1, 2, P}):
            for m in (1, 3):
                seed = P * 100 + s * 7 + m + len(h)
                prog = random_program(P, seed, "f32" if (s + m) % 2 else "i32", max_n=3000)
                if S.find_race(prog) is not None:
                    continue
                _parity(prog, h, s, m, seed=seed)
                n += 1
    assert n > 0


def test_unaligned_buffers_use_element_path():
    """Buffers 4 bytes off a 16-byte boundary take the element-wise path."""
    prog = PR.allreduce(8, 1001)
    _parity(prog, [2, 4], 2, 2, misalign_elems=1)
    prog = PR.alltoall(4, 333, dtype="i32")
    _parity(prog, [2, 2], 2, 1, misalign_elems=3)


def test_degenerate_cases():
    # one rank
    _parity(PR.allreduce(1, 100), [1], 1, 1)
    _parity(PR.broadcast(1, 5), [1], 1, 4)
    # trivial levels
    _parity(PR.reducescatter(6, 50), [1, 3, 1, 2], 2, 2)
    # more pipeline channels than elements: empty pieces are skipped
    _parity(PR.allgather(4, 3), [2, 2], 2, 16)
    # a zero-count primitive next to a real one
    from oracle.model import Program
    prog = Program(4)
    a = [prog.buffer(("send", r), 64) for r in range(4)]
    b = [prog.buffer(("recv", r), 64) for r in range(4)]
    prog.multicast(0, [1, 2, 3], 0, a[0], {j: b[j] for j in (1, 2, 3)})
    prog.reduction([0, 1, 2, 3], 2, 64, {i: a[i] for i in range(4)}, b[2])
    _parity(prog, [2, 2], 2, 2)
    # in-place broadcast: the root's source is its destination
    prog = PR.broadcast(8, 100)
    p0 = prog.primitives[0]
    p0.dsts[0] = p0.src
    _parity(prog, [2, 4], 4, 2)


def test_options_do_not_change_results():
    from paper_2408_05962_gb300 import hiccl as H
    prog = PR.allreduce(16, 5000)
    for opts in ({H.OPT_ORDER: 1}, {H.OPT_ITEM_BYTES: 4096}, {H.OPT_ITEM_BYTES: 1 << 20},
                 {H.OPT_CTAS_PER_SM: 1}):
        _parity(prog, [4, 4], 4, 4, options=opts)


OPS_CASES = [(op, dt) for op in ("max", "min") for dt in ("f32", "i32", "bf16")] + [("lor", "i32")]


@pytest.mark.parametrize("op,dtype", OPS_CASES)
@pytest.mark.parametrize("name", ["allreduce", "reduce", "reducescatter"])
@pytest.mark.parametrize("P,h,s,m,d,mis", [(8, [2, 4], 4, 3, 2053, 0), (16, [16], 2, 2, 1031, 0),
                                           (12, [2, 2, 3], 3, 2, 999, 1)])
def test_reduction_operators(op, dtype, name, P, h, s, m, d, mis):
    """Max, min and logical or (Sec. 3.1) through every fold path: shared-memory
    folds (fan-in <= 8, aligned), vector-load folds (fan-in 16) and the
    element path (buffers one element off 16-byte alignment)."""
    _parity(PR.BUILDERS[name](P, d, dtype=dtype, op=op), h, s, m, seed=P + s + m, zero_frac=0.25,
            misalign_elems=mis)


RING_GPU = [(12, [4, 3], 4, 3, 6, 1500), (12, [2, 2, 3], 4, 3, 8, 2053), (16, [4, 4], 16, 1, 4, 999),
            (64, [4, 4, 4], 4, 4, 8, 4096)]


@pytest.mark.parametrize("name", ["allreduce", "reducescatter", "reduce", "broadcast", "allgather", "alltoall"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("P,h,ring,s,m,d", RING_GPU)
def test_ring(name, dtype, P, h, ring, s, m, d):
    """Hybrid ring+tree (Sec. 4.4): the executor reproduces the ring-order
    semantics bit for bit, up to the 64-rank three-level machine."""
    from paper_2408_05962_gb300 import hiccl as H
    prog = PR.BUILDERS[name](P, d, dtype=dtype)
    mem0 = fill(prog, P + ring)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h, ring)
    outs, _ = run_on_gpu(prog, h, s, m, mem0, options={H.OPT_RING: ring})
    assert_bit_equal(ref, outs[0])


@pytest.mark.parametrize("name", ["allreduce", "reducescatter", "reduce"])
@pytest.mark.parametrize("P,h,ring,s,m", [(12, [4, 3], 4, 3, 2), (16, [4, 4], 16, 1, 2)])
def test_ring_fp8(name, P, h, ring, s, m):
    """The ring order with block-scaled FP8 payloads: every chain step
    re-quantizes the partial (a fresh block scale per level, as the tree)."""
    from paper_2408_05962_gb300 import hiccl as H
    prog = PR.BUILDERS[name](P, 3, dtype="fp8")
    mem0 = fill(prog, P + ring)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h, ring)
    outs, _ = run_on_gpu(prog, h, s, m, mem0, options={H.OPT_RING: ring})
    assert_bit_equal(ref, outs[0])
