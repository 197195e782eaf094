"""The executor's table image, decoded on the host (no GPU): every work-item
record built for upload is checked against the library's own step table --
entries and their meta words, dependency counts, inline operand pointers,
run prefix sums, completion targets and successor lists -- so that the
encoding the kernel reads is tested without running the kernel."""
import struct

import numpy as np
import pytest

from oracle import programs as PR
from paper_2408_05962_gb300 import build as B
from paper_2408_05962_gb300 import hiccl as H
from tests._bridge import FakeAddresses, register

PTR_GLOBAL = 0x80000000
SUCC_GLOBAL = 0xFFFFFFFF
PTR_STEP_MAX, PTR_CAP, SUCC_CAP = 64, 160, 128


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _r16(n):
    return (n + 15) & ~15


def _decode(recs, items):
    """Per item: its entries, run prefix sums, runs, inline pointers and
    completion section, from the layout the header documents."""
    out = []
    for rec, nent, nrun, nptr, nsucc, *_ in items.tolist():
        o = rec * 16
        ent = [struct.unpack_from("<4I", recs, o + 16 * k) for k in range(nent)]
        o += nent * 16
        rpre = list(struct.unpack_from(f"<{nrun + 1}I", recs, o))
        o += _r16((nrun + 1) * 4)
        runs = [struct.unpack_from("<IIQQ", recs, o + 24 * k) for k in range(nrun)]
        o += _r16(nrun * 24)
        ptr = list(struct.unpack_from(f"<{nptr}Q", recs, o))
        o += _r16(nptr * 8)
        ncmp = 2 * nent + 1 + (0 if nsucc == SUCC_GLOBAL else nsucc)
        cmp = list(struct.unpack_from(f"<{ncmp}I", recs, o))
        out.append(dict(ent=ent, rpre=rpre, runs=runs, ptr=ptr, cmp=cmp, nsucc=nsucc, nent=nent))
    return out


def _check_image(comm, dtype_code, seg):
    steps = comm.steps()
    N = len(steps)
    recs, items = comm.image()
    assert len(items) == comm.plan_info()["items"]
    succ = [[] for _ in range(N)]
    for i, st in enumerate(steps):
        for q in st["preds"]:
            succ[q].append(i)
    dec = _decode(recs, items)
    # every step is covered by its entries; count them (completion targets)
    cover = np.zeros(N, dtype=np.int64)
    for it in dec:
        for e in it["ent"]:
            cover[e[0]] += 1
    assert (cover > 0).all()
    last_slot = -1
    for it in dec:
        nent, nptr_used = it["nent"], 0
        assert 1 <= nent <= 64
        slots = {steps[e[0]]["slot"] for e in it["ent"]}
        assert len(slots) == 1                         # one pipeline slot per item
        assert min(slots) >= last_slot                 # tickets in slot order
        last_slot = min(slots)
        total_succ = 0
        for k, (step, meta, poff, indeg) in enumerate(it["ent"]):
            st = steps[step]
            ops = [a for (_, a, _) in st["srcs"]] + [a for (_, a, _) in st["dsts"]]
            assert meta & 3 == (0 if st["kind"] == "copy" else 1)
            assert (meta >> 2) & 15 == dtype_code
            assert (meta >> 6) & 1 == int(all(a % 16 == 0 for a in ops))
            if st["kind"] == "reduce":                  # (a copy ignores the operator field)
                assert (meta >> 7) & 7 == H.OPS[st["op"]]
            assert (meta >> 10) & 2047 == len(st["srcs"]) and (meta >> 21) & 2047 == len(st["dsts"])
            assert indeg == len(st["preds"])
            if poff & PTR_GLOBAL:
                # kept global: too many operands, or the item's inline space is used up
                assert len(ops) > PTR_STEP_MAX or nptr_used + len(ops) > PTR_CAP
            else:
                assert poff == nptr_used
                assert it["ptr"][poff:poff + len(ops)] == ops
                nptr_used += len(ops)
            assert it["cmp"][k] == cover[step]          # completion target
            total_succ += len(succ[step])
        assert len(it["ptr"]) == nptr_used
        # runs: prefix sums of their segment counts; first entries in range
        for r, (entry, _, off, nbytes) in enumerate(it["runs"]):
            assert entry < nent and nbytes > 0
            assert it["rpre"][r + 1] - it["rpre"][r] == -(-nbytes // seg)
        assert it["rpre"][0] == 0
        # successor section
        if it["nsucc"] == SUCC_GLOBAL:
            assert total_succ > SUCC_CAP
        else:
            assert it["nsucc"] == total_succ
            soff = it["cmp"][nent:2 * nent + 1]
            lists = it["cmp"][2 * nent + 1:]
            assert soff[0] == 0 and soff[-1] == total_succ
            for k, e in enumerate(it["ent"]):
                assert lists[soff[k]:soff[k + 1]] == sorted(succ[e[0]])


@pytest.mark.parametrize("name", PR.SEVEN + ("reduce",))
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 2, 2), (16, [4, 4], 4, 3), (64, [4, 4, 4], 4, 8)])
def test_table_image_matches_the_step_table(name, P, h, s, m):
    prog = PR.BUILDERS[name](P, 4096 if P == 64 else 700)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan(h, s, m)
    _check_image(comm, H.DTYPES["f32"], 4096)


@pytest.mark.parametrize("dtype,seg", [("bf16", 4096), ("fp8", 4032), ("i32", 4096)])
def test_table_image_payloads_and_operators(dtype, seg):
    for name, op in (("allreduce", "sum"), ("reducescatter", "max" if dtype != "fp8" else "sum")):
        if dtype == "fp8" and name != "allreduce":
            continue
        prog = PR.BUILDERS[name](16, 1024, dtype=dtype, op=op)
        fake = FakeAddresses(prog)
        comm = register(prog, fake.addr)
        comm.plan([4, 4], 2, 2)
        _check_image(comm, H.DTYPES[dtype], seg)


def test_table_image_wide_steps_keep_pointers_global():
    """A 64-way reduce has 65 operands: its pointers stay in the global array."""
    prog = PR.reduce(64, 64)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([64], 1, 1)
    recs, items = comm.image()
    dec = _decode(recs, items)
    wide = [e for it in dec for e in it["ent"] if ((e[1] >> 10) & 2047) + ((e[1] >> 21) & 2047) > PTR_STEP_MAX]
    assert wide and all(e[2] & PTR_GLOBAL for e in wide)
    _check_image(comm, H.DTYPES["f32"], 4096)


@pytest.mark.parametrize("name", PR.SEVEN + ("reduce",))
@pytest.mark.parametrize("P,h,s,m,dtype", [(8, [2, 4], 2, 2, "f32"), (16, [4, 4], 4, 3, "i32"),
                                           (12, [2, 2, 3], 3, 2, "bf16"), (16, [4, 4], 4, 2, "fp8")])
def test_table_image_executed_on_the_host_equals_the_oracle(name, P, h, s, m, dtype):
    """The image, executed segment by segment the way the kernel walks it
    (ticket order is topological), gives the oracle's plain semantics bit
    for bit: runs, segment offsets and record pointers are right."""
    from oracle import semantics as S
    from tests._bridge import interpret_image
    from tests._cases import fill
    d = 3 if dtype == "fp8" else 1500     # FP8 counts are 128-value blocks
    prog = PR.BUILDERS[name](P, d, dtype=dtype)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan(h, s, m)
    mem0 = fill(prog, 7)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    got = interpret_image(comm, fake, {k: v.copy() for k, v in mem0.items()}, dtype)
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k


@pytest.mark.parametrize("name", ["allreduce", "alltoall", "broadcast"])
def test_table_image_executed_three_levels(name):
    """The bench's machine, {4,4,4} with stripe 4 and pipeline 8, at a
    reduced size: merged runs across channels and relays, executed from the
    image, equal the oracle."""
    from oracle import semantics as S
    from tests._bridge import interpret_image
    from tests._cases import fill
    prog = PR.BUILDERS[name](64, 512)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([4, 4, 4], 4, 8)
    mem0 = fill(prog, 3)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, [4, 4, 4])
    got = interpret_image(comm, fake, {k: v.copy() for k, v in mem0.items()}, "f32")
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("name,P,h,s,m,ring", [("allreduce", 16, [4, 4], 4, 3, 1), ("alltoall", 12, [2, 2, 3], 3, 2, 1),
                                               ("allreduce", 12, [4, 3], 3, 2, 4), ("reducescatter", 64, [4, 4, 4], 4, 8, 1),
                                               ("broadcast_ag_scatter", 8, [2, 4], 2, 2, 1)])
def test_table_image_in_random_dependency_order(seed, name, P, h, s, m, ring):
    """Items executed in random orders that only the image's own dependency
    counts, completion targets and successor lists allow -- as concurrent
    CTAs may run them -- still give the oracle's result: the image carries
    every dependency the data needs (tree edges and fences)."""
    from oracle import semantics as S
    from tests._bridge import interpret_image
    from tests._cases import fill
    prog = PR.BUILDERS[name](P, 256)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    if ring > 1:
        comm.set_option(H.OPT_RING, ring)
    comm.plan(h, s, m)
    mem0 = fill(prog, seed)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h, ring)
    got = interpret_image(comm, fake, {k: v.copy() for k, v in mem0.items()}, "f32", seed=seed)
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k


def test_random_order_catches_a_missing_dependency():
    """Sanity of the check above: with one dependency withheld from the
    successor lists the host execution can diverge from the oracle, so the
    random-order test would notice a missing edge."""
    import struct
    from oracle import semantics as S
    from tests import _bridge
    from tests._cases import fill
    prog = PR.BUILDERS["allreduce"](8, 256)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([2, 4], 1, 1)
    recs, items = comm.image()
    # release every step's successors as soon as it is claimed: drop all
    # dependency counts to zero in a copy of the image
    recs = bytearray(recs)
    for rec, nent, *_ in items.tolist():
        for k in range(nent):
            struct.pack_into("<I", recs, rec * 16 + 16 * k + 12, 0)
    orig = comm.image
    comm.image = lambda: (bytes(recs), items)
    try:
        mem0 = fill(prog, 5)
        ref = {k: v.copy() for k, v in mem0.items()}
        S.run_program(prog, ref, [2, 4])
        differs = False
        for seed in range(8):
            got = _bridge.interpret_image(comm, fake, {k: v.copy() for k, v in mem0.items()}, "f32", seed=seed)
            differs |= any(not np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)) for k in ref)
        assert differs
    finally:
        comm.image = orig


class _Members:
    """Fake addresses of several programs in disjoint ranges, resolvable as
    one memory (keys (member, buffer key))."""

    def __init__(self, progs):
        self.fakes, self.base = [], {}
        b = 0x7f0000000000
        for m, prog in enumerate(progs):
            f = FakeAddresses(prog, base=b)
            self.fakes.append(f)
            for k, a in f.base.items():
                self.base[(m, k)] = a
            b = (f.end + (1 << 20)) & ~255

    def resolve(self, addr):
        best = None
        for key, b in self.base.items():
            if b <= addr and (best is None or b > best[1]):
                best = (key, b)
        return best[0], addr - best[1]


@pytest.mark.parametrize("seed", [None, 11, 12])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_group_image_executes_every_member(seed, dtype):
    """hiccl_group's combined table (members interleaved by slot, relays
    moved to disjoint ranges, successor lists shifted), planned on the host:
    executed from its image -- in ticket order or in random dependency
    orders -- every member's buffers equal that member's oracle result."""
    from oracle import semantics as S
    from tests._bridge import interpret_image
    from tests._cases import fill
    shapes = [("allreduce", [4, 4], 2, 3), ("allgather", [2, 8], 4, 2), ("reducescatter", [16], 1, 1),
              ("alltoall", [4, 4], 4, 1)]
    progs = [PR.BUILDERS[name](16, 3 if dtype == "fp8" else 300, dtype=dtype) for name, *_ in shapes]
    mm = _Members(progs)
    members = []
    for prog, fake, (name, h, s, m) in zip(progs, mm.fakes, shapes):
        c = register(prog, fake.addr)
        c.plan(h, s, m)
        members.append(c)
    g = H.Comm.group_plan(members)
    info = g.plan_info()
    assert info["steps"] == sum(c.plan_info()["steps"] for c in members)
    assert info["items"] == sum(c.plan_info()["items"] for c in members)
    mem0, ref = {}, {}
    for i, prog in enumerate(progs):
        m0 = fill(prog, 100 + i)
        r = {k: v.copy() for k, v in m0.items()}
        S.run_program(prog, r, shapes[i][1])
        for k in m0:
            mem0[(i, k)] = m0[k]
            ref[(i, k)] = r[k]
    got = interpret_image(g, mm, {k: v.copy() for k, v in mem0.items()}, dtype, seed=seed)
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k
    with pytest.raises(H.HicclError):
        g.start()                                # planned only: not startable


def test_group_plan_errors():
    """hiccl_group's checks, on the host: unplanned members are refused
    (HICCL_ERR_STATE) and FP8 members cannot join other payloads
    (HICCL_ERR_UNSUPPORTED)."""
    a = PR.BUILDERS["allreduce"](8, 256)
    b = PR.BUILDERS["allreduce"](8, 2, dtype="fp8")
    mm = _Members([a, b])
    ca, cb = register(a, mm.fakes[0].addr), register(b, mm.fakes[1].addr)
    with pytest.raises(H.HicclError) as e:
        H.Comm.group_plan([ca, cb])
    assert e.value.status == H.ERR_STATE
    ca.plan([2, 4], 1, 1)
    cb.plan([2, 4], 1, 1)
    with pytest.raises(H.HicclError) as e:
        H.Comm.group_plan([ca, cb])
    assert e.value.status == H.ERR_UNSUPPORTED
    g = H.Comm.group_plan([ca])
    assert g.plan_info()["steps"] == ca.plan_info()["steps"]


def _items_by_slot(comm):
    """{slot: [bytes of each item]} of a planned communicator's image."""
    steps = comm.steps()
    recs, items = comm.image()
    out = {}
    for it in _decode(recs, items):
        slot = steps[it["ent"][0][0]]["slot"]
        out.setdefault(slot, []).append(sum(r[3] for r in it["runs"]))
    return out, steps


@pytest.mark.parametrize("name,slot_items", [("scatter", 0), ("scatter", 768), ("allreduce", 0), ("broadcast", 0)])
def test_item_sizing(name, slot_items):
    """Items follow the documented sizing: a slot of S bytes is cut at cap =
    S / D rounded up to 4 KiB, within [4 KiB, ITEM_BYTES]; without a device
    D is 304 for S under 12 MiB (one round over a 152-SM GB300's grid) and
    768 above, unless SLOT_ITEMS sets it."""
    P, d = 64, (4 << 20) // 4 // 64
    prog = PR.BUILDERS[name](P, d)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    if slot_items:
        comm.set_option(H.OPT_SLOT_ITEMS, slot_items)
    comm.plan([4, 4, 4], 4, 8)
    by_slot, steps = _items_by_slot(comm)
    slot_bytes = {}
    for st in steps:
        slot_bytes[st["slot"]] = slot_bytes.get(st["slot"], 0) + st["nbytes"]
    seg, item_max = 4096, 49152
    for slot, sizes in by_slot.items():
        S = slot_bytes[slot]
        D = slot_items or (304 if S < (12 << 20) else 768)
        per_item = -(-S // D)                                   # ceil(S / D)
        cap = min(max(-(-per_item // seg) * seg, seg), item_max)
        assert sum(sizes) == S
        assert max(sizes) < cap + seg
        if not slot_items and S < (12 << 20):
            assert len(sizes) <= 304 + 2           # one round (a class change may close one more)
    comm.destroy()


def test_small_slots_take_fewer_items_than_768():
    """A Scatter's 4 MiB relay stage: one round over the grid (at most 304
    items) by default, about 512 items when spread over 768."""
    P, d = 64, (4 << 20) // 4 // 64
    prog = PR.scatter(P, d)
    fake = FakeAddresses(prog)
    counts = []
    for si in (0, 768):
        comm = register(prog, fake.addr)
        if si:
            comm.set_option(H.OPT_SLOT_ITEMS, si)
        comm.plan([4, 4, 4], 4, 8)
        by_slot, _ = _items_by_slot(comm)
        counts.append(len(by_slot[0]))
        comm.destroy()
    assert counts[0] <= 304 < counts[1]
