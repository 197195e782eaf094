"""The library's host factorizer against the oracle, without a GPU.

For every case the same program is given to the oracle and, at fake device
addresses, to the C-ABI library in plan-only mode.  Checked: per-level link
bytes, HBM bytes and the number of stages equal the oracle factorizer's
(same readings of the paper), and the library's own step table -- its
steps, relay offsets and execution order -- interpreted on NumPy buffers
reproduces the oracle's plain semantics bit for bit."""
import numpy as np
import pytest

from oracle import programs as PR
from oracle import semantics as S
from oracle.factorize import factorize
from oracle.hierarchy import all_factorizations
from paper_2408_05962_gb300 import build as B
from tests._bridge import FakeAddresses, interpret, register
from tests._cases import fill, random_program


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _check(prog, h, s, m, seed=0, interpret_steps=True, zero_frac=0.0, ring=1):
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    if ring != 1:
        from paper_2408_05962_gb300 import hiccl as H
        comm.set_option(H.OPT_RING, ring)
    comm.plan(h, s, m)
    plan = factorize(prog, h, s, m, ring)
    assert comm.level_bytes() == plan.level_bytes()
    assert comm.hbm_bytes() == plan.hbm_bytes()
    info = comm.plan_info()
    assert info["stages"] == plan.stages()
    assert info["steps"] == len(plan.ops)
    if interpret_steps:
        mem0 = fill(prog, seed, zero_frac)
        ref = {k: v.copy() for k, v in mem0.items()}
        S.run_program(prog, ref, h, ring)
        got = interpret(comm, fake, {k: v.copy() for k, v in mem0.items()}, prog.dtype)
        for k in ref:
            assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k
    return comm


COLL = PR.SEVEN + ("reduce", "allreduce_single", "broadcast_ag_scatter", "reduce_gather_rs",
                   "allgather_bcast_gather", "reducescatter_scatter_reduce", "allreduce_bcast_reduce")


@pytest.mark.parametrize("name", COLL)
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 1, 1), (8, [2, 4], 4, 3), (12, [2, 2, 3], 3, 2),
                                     (16, [4, 4], 4, 2), (8, [8], 2, 2), (6, [3, 2], 2, 1)])
@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_collectives(name, P, h, s, m, dtype):
    _check(PR.BUILDERS[name](P, 11, dtype=dtype), h, s, m, seed=P * 7 + s)


@pytest.mark.parametrize("P", [2, 3, 4, 6, 8])
def test_random_programs_all_hierarchies(P):
    n = 0
    for h in all_factorizations(P):
        for s in sorted({1, 2, P}):
            for m in (1, 2):
                seed = P * 1000 + s * 10 + m + len(h)
                prog = random_program(P, seed, "f32")
                if S.find_race(prog) is not None:
                    continue
                _check(prog, h, s, m, seed=seed)
                n += 1
    assert n > 0


def test_config1_allreduce_accounting():
    """All-reduce of 65,536 fp32 per rank over {2, 4} as Listing 2 (s = 1,
    m = 1): chunk n = 32 KiB.  Reduce-scatter moves 8 x (2*5n + 3n) = 104n of
    device memory and All-gather 8 x (2n + 4n + 4n) = 80n, its multicast hops
    reading their source once (top hop: 1 read + 1 write; a bottom hop into
    three ranks: 1 read + 3 writes, in both nodes); the top level carries 16n
    (Table 3: 2(p - g)d per node, two nodes) and the bottom level 96n."""
    prog = PR.allreduce(8, 8192)
    comm = _check(prog, [2, 4], 1, 1, interpret_steps=False)
    n = 8192 * 4
    rd, wr = comm.hbm_bytes()
    assert rd + wr == 104 * n + 80 * n
    assert comm.level_bytes() == [16 * n, 96 * n]


def test_config2_shapes_plan():
    """The seven collectives of P = 64, {4,4,4}, 4 MiB per rank, s = 4, m = 8
    plan, and agree with the oracle's accounting (no execution: too large for
    the interpreter)."""
    d = (4 << 20) // 4 // 64
    for name in PR.SEVEN:
        prog = PR.BUILDERS[name](64, d)
        _check(prog, [4, 4, 4], 4, 8, interpret_steps=False)


def test_table_order_and_items():
    prog = PR.allreduce(8, 4096)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([2, 4], 2, 4)
    info = comm.plan_info()
    steps = comm.steps()
    slots = [st["slot"] for st in steps]
    assert slots == sorted(slots)
    for i, st in enumerate(steps):
        for q in st["preds"]:
            assert steps[q]["slot"] < st["slot"]
    assert info["items"] >= 1 and info["slots"] == slots[-1] + 1


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("name", ["allreduce", "reducescatter", "reduce", "allgather", "alltoall", "broadcast"])
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 1, 1), (8, [2, 4], 4, 3), (12, [2, 2, 3], 3, 2)])
def test_lowprec_collectives(dtype, name, P, h, s, m):
    """BF16 and block-scaled FP8 payloads: the library's step table, run by
    the NumPy interpreter with the payloads' decode / fold / encode, equals
    the oracle bit for bit (FP8 counts are 128-value blocks)."""
    d = 37 if dtype == "bf16" else 3
    _check(PR.BUILDERS[name](P, d, dtype=dtype), h, s, m, seed=P + s + m)


def test_fp8_count_must_be_block_multiple():
    from paper_2408_05962_gb300 import hiccl as H
    c = H.Comm(2, "fp8")
    a = [0x100000, 0x200000]
    with pytest.raises(H.HicclError) as e:
        c.add_multicast(a, a, 100, 0, [1])
    assert e.value.status == H.ERR_INVALID
    c.add_multicast(a, [0, 0x300000], 256, 0, [1])
    c.plan([2])
    assert c.hbm_bytes() == (2 * 144, 2 * 144)


@pytest.mark.parametrize("name", ["broadcast", "reduce", "allgather", "reducescatter", "allreduce", "scatter",
                                  "gather", "alltoall", "allreduce_single"])
def test_native_composition_equals_primitive_composition(name):
    """hiccl_add_collective registers the same program as the Table 2
    compositions built primitive by primitive (identical plans: step count,
    HBM and level bytes), and its step table computes the oracle's result."""
    from paper_2408_05962_gb300 import hiccl as H
    P, d, h = 8, 13, [2, 4]
    prog = PR.BUILDERS[name](P, d)
    fake = FakeAddresses(prog)
    ref_comm = register(prog, fake.addr)
    ref_comm.plan(h, 2, 2)
    comm = H.Comm(P, "f32")
    recv = [fake.base[("recv", r)] for r in range(P)]
    send = [fake.base[("send", r)] for r in range(P)]
    comm.add_collective(name, d, send, recv, root=0)
    comm.plan(h, 2, 2)
    assert comm.plan_info()["steps"] == ref_comm.plan_info()["steps"]
    assert comm.hbm_bytes() == ref_comm.hbm_bytes()
    assert comm.level_bytes() == ref_comm.level_bytes()
    mem0 = fill(prog, 4)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    got = interpret(comm, fake, {k: v.copy() for k, v in mem0.items()}, prog.dtype)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k


OPS_CASES = [(op, dt) for op in ("max", "min") for dt in ("f32", "i32", "bf16")] + [("lor", "i32")]


@pytest.mark.parametrize("op,dtype", OPS_CASES)
@pytest.mark.parametrize("name", ["reduce", "reducescatter", "allreduce", "allreduce_single"])
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 1, 1), (8, [2, 4], 4, 3), (12, [2, 2, 3], 3, 2)])
def test_reduction_operators(op, dtype, name, P, h, s, m):
    """Max, min and logical or (Sec. 3.1): the step table carries the
    operator of each reduce and reproduces the oracle bit for bit (inputs
    with a quarter zeros, so that logical or sees both outcomes)."""
    prog = PR.BUILDERS[name](P, 29, dtype=dtype, op=op)
    comm = _check(prog, h, s, m, seed=P + s, zero_frac=0.25)
    ops = {st["op"] for st in comm.steps() if st["kind"] == "reduce"}
    assert ops == {op}


@pytest.mark.parametrize("name,op", [("allreduce", "max"), ("reducescatter", "min"), ("reduce", "max"),
                                     ("allreduce_single", "min")])
def test_native_composition_operator(name, op):
    """hiccl_add_collective passes its operator to every reduction it registers."""
    from paper_2408_05962_gb300 import hiccl as H
    P, d, h = 8, 13, [2, 4]
    prog = PR.BUILDERS[name](P, d, op=op)
    fake = FakeAddresses(prog)
    comm = H.Comm(P, "f32")
    comm.add_collective(name, d, [fake.base[("send", r)] for r in range(P)],
                        [fake.base[("recv", r)] for r in range(P)], root=0, op=op)
    comm.plan(h, 2, 2)
    mem0 = fill(prog, 5)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    got = interpret(comm, fake, {k: v.copy() for k, v in mem0.items()}, prog.dtype)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k


RING_CASES = [(12, [4, 3], 4, 3, 2), (12, [2, 2, 3], 4, 3, 3), (12, [2, 2, 3], 2, 1, 2), (8, [2, 2, 2], 8, 1, 2),
              (16, [4, 4], 4, 4, 4), (12, [3, 2, 2], 6, 2, 1)]


@pytest.mark.parametrize("name", COLL)
@pytest.mark.parametrize("P,h,ring,s,m", RING_CASES)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_ring_collectives(name, P, h, ring, s, m, dtype):
    """ring(n) (Sec. 4.4): the library's plan has the oracle's level bytes,
    HBM bytes and stage count, and its step table reproduces the ring-order
    semantics bit for bit."""
    _check(PR.BUILDERS[name](P, 19, dtype=dtype), h, s, m, seed=P + ring + s, ring=ring)


@pytest.mark.parametrize("P", [4, 6, 8, 12])
def test_ring_random_programs(P):
    from oracle.hierarchy import group_sizes
    n = 0
    for h in all_factorizations(P, max_levels=3):
        for l in range(1, len(h) + 1):
            ring = int(np.prod(h[:l]))
            node = P // ring
            for s in sorted({1, node}):
                prog = random_program(P, P * 31 + l + s, ("f32", "i32")[l % 2])
                if S.find_race(prog) is not None:
                    continue
                _check(prog, h, s, 2, seed=l, ring=ring)
                n += 1
    assert n > 0 and group_sizes


def test_ring_validation():
    from paper_2408_05962_gb300 import hiccl as H
    prog = PR.broadcast(12, 4)
    fake = FakeAddresses(prog)
    for ring, s, ok in ((3, 1, False), (4, 4, False), (4, 3, True), (12, 1, True), (1, 12, True)):
        comm = register(prog, fake.addr)
        comm.set_option(H.OPT_RING, ring)
        if ok:
            comm.plan([4, 3], s, 1)
        else:
            with pytest.raises(H.HicclError) as e:
                comm.plan([4, 3], s, 1)
            assert e.value.status == H.ERR_INVALID
    comm = register(prog, fake.addr)
    with pytest.raises(H.HicclError):
        comm.set_option(H.OPT_RING, 13)


def test_planner_scales_to_a_thousand_ranks():
    """Initialization at scale (the paper reports under six seconds on a
    thousand GPUs, per process): the whole All-gather schedule of 1024
    virtual ranks in 256 nodes of 4 ({256, 4}, stripe 4, pipeline 2) is
    planned in well under a minute on one host core, with the closed-form
    top-level volume (p - g) * d per node."""
    import time
    from paper_2408_05962_gb300 import hiccl as H
    P, d = 1024, 256
    base = 1 << 40
    send = [base + r * (d * 4 + 4096) for r in range(P)]
    recv = [base + (1 << 36) + r * (d * P * 4 + 4096) for r in range(P)]
    comm = H.Comm(P, "f32")
    comm.add_collective("allgather", d, send, recv)
    t0 = time.perf_counter()
    comm.plan([256, 4], 4, 2)
    dt = time.perf_counter() - t0
    info = comm.plan_info()
    assert info["stages"] == 3 and info["steps"] > 0
    assert comm.level_bytes()[0] == 256 * (P - 4) * d * 4
    assert dt < 60.0, dt


@pytest.mark.parametrize("what,needle", [(0, "depends on a later step"), (1, "outside its primitive"),
                                         (2, "do not tile")])
def test_corrupted_tables_are_caught_on_the_host(what, needle):
    """Host-side fault tests: a table with a dependency cycle, an operand
    outside its primitive's buffers, or uncovered segments is rejected by the
    plan check before anything reaches the GPU (and hiccl_init on it is
    refused); the uncorrupted plan passes the same check."""
    from paper_2408_05962_gb300 import hiccl as H
    prog = PR.allreduce(8, 37)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([2, 4], 2, 2)
    comm.validate()
    comm.corrupt(what)
    with pytest.raises(H.HicclError) as e:
        comm.validate()
    assert e.value.status == H.ERR_INVALID
    assert needle in H.hiccl_last_error(comm.handle)


@pytest.mark.parametrize("name", COLL)
def test_every_plan_passes_the_check(name):
    for P, h, s, m in [(8, [2, 4], 4, 3), (12, [2, 2, 3], 3, 2)]:
        prog = PR.BUILDERS[name](P, 11)
        comm = register(prog, FakeAddresses(prog).addr)
        comm.plan(h, s, m)
        comm.validate()


@pytest.mark.parametrize("name", ["allreduce", "reducescatter", "reduce", "allgather"])
@pytest.mark.parametrize("P,h,ring,s,m", [(12, [4, 3], 4, 3, 2), (16, [4, 4], 16, 1, 2), (12, [2, 2, 3], 2, 3, 1)])
def test_ring_fp8_collectives(name, P, h, ring, s, m):
    _check(PR.BUILDERS[name](P, 3, dtype="fp8"), h, s, m, seed=P + ring, ring=ring)


def test_fuzz_random_programs_and_shapes():
    """Seeded sweep beyond the exhaustive small cases: P up to 24, a random
    factorization of P, random stripe, pipeline and (where a level allows
    one) ring, random sparse programs in f32 and i32 -- the library's table
    reproduces the oracle's semantics and accounting in every case."""
    from oracle.hierarchy import ring_level
    g = np.random.Generator(np.random.PCG64(20240805))
    n = 0
    for it in range(240):
        P = int(g.choice([5, 6, 8, 9, 12, 16, 18, 24]))
        hs = all_factorizations(P)
        h = list(hs[int(g.integers(0, len(hs)))])
        s = int(g.integers(1, P + 1))
        m = int(g.integers(1, 5))
        dtype = "f32" if it % 2 == 0 else "i32"
        prog = random_program(P, 5000 + it, dtype, chunks=int(g.integers(1, 4)), max_n=24)
        if S.find_race(prog) is not None:
            continue
        ring = 1
        if it % 3 == 0:   # a ring over the groups of a level, when the stripe fits a node
            def fits(r):
                try:
                    ring_level(h, r)
                except ValueError:
                    return False
                return s <= P // r
            cands = [r for r in range(2, P + 1) if P % r == 0 and fits(r)]
            if cands:
                ring = int(cands[int(g.integers(0, len(cands)))])
        _check(prog, h, s, m, seed=it, ring=ring)
        n += 1
    assert n >= 160


@pytest.mark.parametrize("m", [1, 2, 4, 5, 7])
def test_pipeline_slots_of_fig7(m):
    """Sec. 4.5 / Fig. 7: the m channels of a piece run the same stages, each
    channel one slot behind the previous, so a schedule of S dependent stages
    fills S + m - 1 pipeline slots (warm-up, overlapped middle, wind-down).
    Fig. 6's examples on four nodes of three GPUs with stripe(3): the tree
    over {2,2,3} has S = 4 stages, ring(4) over {4,3} has S = 5 (pipeline-slot
    order, HICCL_OPT_ORDER = 0)."""
    from paper_2408_05962_gb300 import hiccl as H
    for hier, ring, stages in (([2, 2, 3], 1, 4), ([4, 3], 4, 5)):
        prog = PR.broadcast(12, 600, root=0)
        fake = FakeAddresses(prog)
        comm = register(prog, fake.addr)
        comm.set_option(H.OPT_ORDER, 0)
        if ring > 1:
            comm.set_option(H.OPT_RING, ring)
        comm.plan(hier, 3, m)
        info = comm.plan_info()
        assert info["stages"] == stages
        assert info["slots"] == stages + m - 1, (hier, ring, m, info)


@pytest.mark.parametrize("m", [1, 3, 5])
def test_pipeline_slots_of_eq1_eq2(m):
    """Sec. 4.6, Eq. 1: a pipelined ring Broadcast over n nodes with no
    hierarchy inside them takes n + m - 2 inter-node slots (n - 1 hops, each
    channel one slot behind the previous); Eq. 2: the tree over n = 2^L nodes
    has log n levels, i.e. log n + m - 1 slots."""
    import math
    from paper_2408_05962_gb300 import hiccl as H
    for n in (3, 4, 6, 8):
        prog = PR.broadcast(n, 480, root=0)
        fake = FakeAddresses(prog)
        comm = register(prog, fake.addr)
        comm.set_option(H.OPT_ORDER, 0)
        comm.set_option(H.OPT_RING, n)
        comm.plan([n], 1, m)
        info = comm.plan_info()
        assert info["stages"] == n - 1 and info["slots"] == n + m - 2, (n, m, info)
    for n in (2, 4, 8, 16):
        L = int(math.log2(n))
        prog = PR.broadcast(n, 480, root=0)
        fake = FakeAddresses(prog)
        comm = register(prog, fake.addr)
        comm.set_option(H.OPT_ORDER, 0)
        comm.plan([2] * L, 1, m)
        info = comm.plan_info()
        assert info["stages"] == L and info["slots"] == L + m - 1, (n, m, info)


def test_library_fence_is_dependency_not_barrier():
    """Sec. 3.3 / Fig. 4 in the library's table: in the All-reduce program
    (reductions R_0..R_7, fence, multicasts M_0..M_7), a step of M_i depends
    across the fence only on steps of R_i of the same pipeline channel."""
    P, d = 8, 16
    prog = PR.allreduce(P, d)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([2, 4], 1, 2)
    steps = comm.steps()
    crossing = 0
    for st in steps:
        if st["prim"] < P:
            continue
        for q in st["preds"]:
            dep = steps[q]
            if dep["prim"] < P:
                assert dep["prim"] == st["prim"] - P and dep["channel"] == st["channel"], (st, dep)
                crossing += 1
    assert crossing > 0


@pytest.mark.parametrize("name", PR.SEVEN + ("reduce",))
@pytest.mark.parametrize("P,h,s,m,ring", [(8, [2, 4], 4, 3, 1), (12, [2, 2, 3], 3, 5, 1), (12, [4, 3], 3, 4, 4),
                                          (16, [4, 4], 4, 2, 1), (16, [4, 4], 4, 3, 4)])
def test_pipeline_slots_match_the_oracle(name, P, h, s, m, ring):
    """In pipeline-slot order (HICCL_OPT_ORDER = 0) the library's number of
    slots equals the oracle factorizer's (channel c starts at slot c, a step
    runs one slot after its latest predecessor, fences included)."""
    from paper_2408_05962_gb300 import hiccl as H
    prog = PR.BUILDERS[name](P, 48)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.set_option(H.OPT_ORDER, 0)
    if ring > 1:
        comm.set_option(H.OPT_RING, ring)
    comm.plan(h, s, m)
    plan = factorize(prog, h, s, m, ring)
    assert comm.plan_info()["slots"] == plan.slots()
    assert comm.plan_info()["stages"] == plan.stages()
