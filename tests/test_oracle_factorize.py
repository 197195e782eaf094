"""Pins of the oracle's factorizer and schedule simulator (paper Sec. 4):
the worked examples of Sec. 4.3 and Fig. 1, closed-form per-level volumes,
the volumes implied by Table 3, stage counts, and brute-force agreement of
the simulated schedule with the plain semantics over every hierarchy of up to
eight ranks, random roots, leaf subsets, stripe counts and pipeline depths,
executed in random dependency-respecting orders."""
import os
from math import prod

import numpy as np
import pytest

from oracle import programs as PR
from oracle import semantics as S
from oracle.factorize import factorize, piece_bounds
from oracle.hierarchy import all_factorizations, group_sizes, level_of
from oracle.model import Program
from oracle.simulate import simulate
from synth import int_ranks, random_leaf_set, uniform_ranks

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _hops(plan):
    out = set()
    for op in plan.ops:
        if op.kind != "copy" or op.level is None:
            continue
        a = op.srcs[0][0]
        for b, _ in op.dsts:
            out.add((op.level, a, b))
    return out


# ---------------------------------------------------------------------------
# worked examples
# ---------------------------------------------------------------------------

def test_golden_broadcast_2_2_3():
    rows = _read_golden("bcast_2_2_3.txt")
    hops = {(int(r[1]), int(r[2]), int(r[3])) for r in rows if r[0] == "hop"}
    stages = {int(r[1]): int(r[2]) for r in rows if r[0] == "stages"}
    prog = PR.broadcast(12, 6, root=0)
    plan = factorize(prog, [2, 2, 3])
    assert _hops(plan) == hops
    for s, n in stages.items():
        assert factorize(prog, [2, 2, 3], stripe=s).stages() == n


def test_golden_fig1_direct_vs_hierarchical():
    node = [2, 3]                                  # two nodes of three GPUs
    for h, crossing in _read_golden("fig1_direct_vs_hier.txt"):
        h = [int(v) for v in h.split(",")]
        plan = factorize(PR.broadcast(6, 2, root=0), h)
        n = sum(1 for lv, a, b in _hops(plan) if level_of(a, b, node) == 0)
        assert n == int(crossing)


def test_golden_ring_4x3():
    """Sec. 4.4: ring(4) with stripe(3) over {4,3}: the inter-node hops of each
    stripe form the chain N0 -> N1 -> N2 -> N3, and five stages."""
    rows = _read_golden("ring_4x3.txt")
    prog = PR.broadcast(12, 6, root=0)
    for r in rows:
        if r[0] == "stages":
            ring, stripe, n = int(r[1]), int(r[2]), int(r[3])
            assert factorize(prog, [4, 3], stripe=stripe, ring=ring).stages() == n
    plan = factorize(prog, [4, 3], stripe=3, ring=4)
    inter = {(a, b) for lv, a, b in _hops(plan) if lv == 0}
    want = set()
    for r in rows:
        if r[0] == "chain":
            ranks = [int(v) for v in r[1:]]
            want |= set(zip(ranks, ranks[1:]))
    assert inter == want
    # the tree on the same machine: one top-level hop per stripe into every node
    tree = factorize(prog, [4, 3], stripe=3)
    assert {(a, b) for lv, a, b in _hops(tree) if lv == 0} == {(k, k + 3 * i) for k in range(3) for i in (1, 2, 3)}
    assert tree.stages() == 3          # stage 0, the top level, inside the nodes


def test_ring_level_volumes_and_chain_start():
    """A ring over all nodes from node 0 crosses each level as often as the
    tree (consecutive nodes a, a+1 first differ at level l for
    prod(f_0..f_{l-1}) * (f_l - 1) values of a); from another node the chain
    wraps: for {2,2,3} from node 1 it runs N1->N2 (level 0), N2->N3 (level 1),
    N3->N0 (level 0)."""
    d, e = 8, 4
    for h, ring in (([2, 2, 3], 4), ([4, 3], 4), ([2, 3, 2], 2), ([2, 3, 2], 6), ([3, 2, 2], 12)):
        P = prod(h)
        G = group_sizes(h)
        b = d * P * e
        closed = [prod(h[:l]) * (h[l] - 1) * b for l in range(len(h))]
        assert factorize(PR.broadcast(P, d, root=0), h, ring=ring).level_bytes() == closed
        assert factorize(PR.reduce(P, d, root=0), h, ring=ring).level_bytes() == closed
    plan = factorize(PR.broadcast(12, d, root=4), [2, 2, 3], ring=4)
    inter = sorted((lv, a, b) for lv, a, b in _hops(plan) if lv < 2)
    assert inter == [(0, 4, 7), (0, 10, 1), (1, 7, 10)]


def test_ring_rejects_bad_shapes():
    prog = PR.broadcast(12, 2)
    with pytest.raises(ValueError):
        factorize(prog, [4, 3], ring=3)            # 4-rank nodes are not a level of {4,3}
    with pytest.raises(ValueError):
        factorize(prog, [4, 3], stripe=4, ring=4)  # stripe beyond the node
    factorize(prog, [4, 3], stripe=3, ring=4)
    factorize(prog, [4, 3], stripe=4, ring=1)


def test_striped_tree_is_multi_rail():
    """Sec. 4.3: with stripe(3) on {2,2,3} every GPU of the root node sends one
    piece across the top level (g0, g1, g2 -> g6, g7, g8)."""
    plan = factorize(PR.broadcast(12, 6, root=0), [2, 2, 3], stripe=3)
    top = {(a, b) for lv, a, b in _hops(plan) if lv == 0}
    assert top == {(0, 6), (1, 7), (2, 8)}


# ---------------------------------------------------------------------------
# closed-form volumes
# ---------------------------------------------------------------------------

HIERS = [[8], [2, 4], [4, 2], [2, 2, 2], [2, 2, 3], [4, 4, 4], [3, 1, 2], [1, 6]]


@pytest.mark.parametrize("h", HIERS)
@pytest.mark.parametrize("s,m", [(1, 1), (2, 3), (3, 1), (4, 2)])
def test_full_leaf_level_volumes(h, s, m):
    """A multicast (or reduction) of b bytes over all P ranks crosses level l
    prod_{k<l} f_k * (f_l - 1) times: one copy into each sibling subgroup of
    every level-l group, (P-1) copies in all.  Pipelining leaves this
    unchanged.  Striping inside one bottom-level group only re-routes the
    same transfers (Sec. 4.3), except that a root holding a separate
    destination also exchanges the pieces of the branches b > 0 with k_b
    (the branches deliver to "all GPUs but" k_b, the root included)."""
    P = prod(h)
    if s > P:
        pytest.skip("stripe larger than P")
    d = 8
    b = d * P * 4
    L = len(h)
    expect = [prod(h[:l]) * (h[l] - 1) * b for l in range(L)]
    G = group_sizes(h)
    ls = max(l for l in range(L + 1) if G[l] >= s)
    striped = s > 1 and G[ls] < P
    bounds = piece_bounds(d * P, s * m, 4)
    extra = (d * P - bounds[m]) * 4 if striped else 0
    for root in {0, P - 1, P // 2}:
        bc = factorize(PR.broadcast(P, d, root=root), h, s, m).level_bytes()
        rd = factorize(PR.reduce(P, d, root=root), h, s, m).level_bytes()
        inplace = PR.broadcast(P, d, root=root)
        p0 = inplace.primitives[0]
        p0.dsts[root] = p0.src
        ip = factorize(inplace, h, s, m).level_bytes()
        assert sum(ip) == (P - 1) * b
        assert sum(bc) == (P - 1) * b + extra
        assert sum(rd) == (P - 1) * b + extra
        if not striped or ls == L - 1:
            assert ip == expect
            want = list(expect)
            want[L - 1] += extra
            assert bc == want and rd == want, (bc, rd, want)


@pytest.mark.parametrize("n,g", [(2, 2), (2, 4), (4, 4), (3, 2)])
@pytest.mark.parametrize("s", [1, 2])
def test_table3_top_level_volumes(n, g, s):
    """Table 3's bounds divide the per-node top-level volume by the node
    bandwidth kf.  With h = {n, g}, p = n*g and chunk d, the volumes entering
    each node are: All-gather and Reduce-scatter (p-g)d, All-reduce 2(p-g)d,
    All-to-all g(p-g)d, Broadcast dp (every non-root node), Gather (p-g)d
    into the root node; Scatter sends (p-g)d out of the root node."""
    p = n * g
    d = 16
    e = 4

    def per_node_in(plan):
        vol = [0] * n
        for op in plan.ops:
            pairs = ([(op.srcs[0][0], b) for b, _ in op.dsts] if op.kind == "copy"
                     else [(a, op.dsts[0][0]) for a, _ in op.srcs])
            for a, b in pairs:
                if a // g != b // g:
                    vol[b // g] += op.n * e
        return vol

    def per_node_out(plan):
        vol = [0] * n
        for op in plan.ops:
            pairs = ([(op.srcs[0][0], b) for b, _ in op.dsts] if op.kind == "copy"
                     else [(a, op.dsts[0][0]) for a, _ in op.srcs])
            for a, b in pairs:
                if a // g != b // g:
                    vol[a // g] += op.n * e
        return vol

    h = [n, g]
    if s > g:
        pytest.skip()
    assert per_node_in(factorize(PR.allgather(p, d), h, s)) == [(p - g) * d * e] * n
    assert per_node_in(factorize(PR.reducescatter(p, d), h, s)) == [(p - g) * d * e] * n
    assert per_node_in(factorize(PR.allreduce(p, d), h, s)) == [2 * (p - g) * d * e] * n
    assert per_node_in(factorize(PR.alltoall(p, d), h, s)) == [g * (p - g) * d * e] * n
    vin = per_node_in(factorize(PR.broadcast(p, d, root=0), h, s))
    assert vin == [0] + [d * p * e] * (n - 1)
    assert per_node_in(factorize(PR.gather(p, d, root=0), h, s))[0] == (p - g) * d * e
    assert per_node_out(factorize(PR.scatter(p, d, root=0), h, s))[0] == (p - g) * d * e


def test_hierarchical_vs_direct_top_volume():
    """Sec. 2.2: hierarchical factorization minimises top-level traffic; for a
    Broadcast on {n, g} the top level carries (n-1) copies instead of p-g."""
    for n, g in [(2, 3), (4, 4), (2, 8)]:
        p = n * g
        node = [n, g]
        flat = factorize(PR.broadcast(p, 4, root=0), [p])
        hier = factorize(PR.broadcast(p, 4, root=0), node)
        cross = lambda plan: sum(1 for lv, a, b in _hops(plan) if level_of(a, b, node) == 0)
        assert cross(flat) == p - g
        assert cross(hier) == n - 1


# ---------------------------------------------------------------------------
# stages and fences
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("h", [[2, 2, 3], [4, 4, 4], [2, 4], [8]])
def test_stage_counts(h):
    """Without striping a full broadcast has one dependent stage per level;
    striping adds stage 0; pipelining does not change the chain length of a
    channel (Sec. 4.5)."""
    P = prod(h)
    L = sum(1 for f in h if f > 1)
    prog = PR.broadcast(P, 64, root=0)
    assert factorize(prog, h).stages() == L
    assert factorize(prog, h, 1, 4).stages() == L
    g = group_sizes(h)[-2]
    if len(h) > 1:
        assert factorize(prog, h, g).stages() == L + 1


def test_fence_is_dependency_not_barrier():
    """Sec. 3.3 / Fig. 4: in the All-reduce program, multicast M_i depends on
    reduction R_i only (per pipeline channel), not on the other R_j."""
    P, d = 8, 16
    plan = factorize(PR.allreduce(P, d), [2, 4], 1, 2)
    for op in plan.ops:
        if op.epoch != 1:
            continue
        for j in op.deps:
            dep = plan.ops[j]
            if dep.epoch == 0:
                assert dep.prim == op.prim - P          # M_i -> R_i
                assert dep.channel == op.channel


def test_piece_bounds_properties():
    for count in [0, 1, 3, 4, 17, 1000, 4097]:
        for parts in [1, 2, 3, 8, 32]:
            for q in [4, 8, 128]:
                b = piece_bounds(count, parts, q)
                assert b[0] == 0 and b[-1] == count
                assert all(b[i] <= b[i + 1] for i in range(parts))
                assert all(v % q == 0 for v in b[:-1] if v != count)


# ---------------------------------------------------------------------------
# simulator == semantics, brute force over small configurations
# ---------------------------------------------------------------------------

from tests._cases import fill as _init, random_program as _random_program  # noqa: E402


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 8])
def test_simulator_matches_semantics(P):
    cases = 0
    for h in all_factorizations(P):
        for s in sorted({1, 2, P} & set(range(1, P + 1))):
            for m in (1, 3):
                for dtype in ("f32", "i32"):
                    seed = hash((P, tuple(h), s, m, dtype)) % 100000
                    prog = _random_program(P, seed, dtype)
                    if S.find_race(prog) is not None:
                        continue
                    mem0 = _init(prog, seed)
                    ref = {k: v.copy() for k, v in mem0.items()}
                    S.run_program(prog, ref, h)
                    plan = factorize(prog, h, s, m)
                    got = {k: v.copy() for k, v in mem0.items()}
                    simulate(plan, got, order_seed=seed)
                    for k in ref:
                        assert np.array_equal(ref[k], got[k]), (h, s, m, dtype, k)
                    cases += 1
    assert cases > 0


def _rings(h):
    """Every ring(n) that matches a level of h: n = f_0 * ... * f_{l-1}."""
    return sorted({prod(h[:l]) for l in range(len(h) + 1)})


@pytest.mark.parametrize("P", [2, 4, 6, 8, 12])
def test_ring_simulator_matches_semantics(P):
    """Every ring of every hierarchy: the simulated schedule (random
    dependency-respecting order) reproduces the ring-order semantics bit for
    bit, for random programs, roots and leaf sets."""
    cases = 0
    for h in all_factorizations(P, max_levels=3):
        node_sizes = group_sizes(h)
        for ring in _rings(h):
            N = P // ring
            for s in sorted({1, 2, N} & set(range(1, (N if ring > 1 else P) + 1))):
                for m in (1, 2):
                    dtype = ("f32", "i32", "bf16")[(P + ring + s + m) % 3]
                    seed = hash((P, tuple(h), ring, s, m)) % 100000
                    prog = _random_program(P, seed, dtype)
                    if S.find_race(prog) is not None:
                        continue
                    mem0 = _init(prog, seed)
                    ref = {k: v.copy() for k, v in mem0.items()}
                    S.run_program(prog, ref, h, ring)
                    got = {k: v.copy() for k, v in mem0.items()}
                    simulate(factorize(prog, h, s, m, ring), got, order_seed=seed)
                    for k in ref:
                        assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), (h, ring, s, m, k)
                    cases += 1
    assert cases > 0 and node_sizes


@pytest.mark.parametrize("name", PR.SEVEN + ("reduce", "allreduce_single"))
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 1, 1), (8, [2, 4], 4, 3), (12, [2, 2, 3], 3, 2),
                                     (16, [4, 4], 4, 2), (8, [2, 2, 2], 2, 4)])
def test_collectives_simulated(name, P, h, s, m):
    d = 13
    prog = PR.BUILDERS[name](P, d)
    x = uniform_ranks(P, d * P, seed=2)
    mem0 = prog.allocate()
    for r in range(P):
        mem0[("send", r)][...] = x[r][:mem0[("send", r)].shape[0]]
        mem0[("recv", r)][...] = np.float32(-7.0)              # guard value
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    plan = factorize(prog, h, s, m)
    got = {k: v.copy() for k, v in mem0.items()}
    simulate(plan, got, order_seed=P + s + m)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), (name, k)



@pytest.mark.parametrize("op,dtype", [("max", "f32"), ("min", "i32"), ("lor", "i32"), ("max", "bf16")])
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 1, 1), (8, [2, 4], 4, 2), (12, [2, 2, 3], 3, 2)])
def test_other_ops_simulated(op, dtype, P, h, s, m):
    d = 24
    for prog in (PR.allreduce(P, d, dtype=dtype, op=op), PR.reduce(P, d, root=P - 1, dtype=dtype, op=op)):
        mem0 = _init_ops(prog, 3)
        ref = {k: v.copy() for k, v in mem0.items()}
        S.run_program(prog, ref, h)
        got = {k: v.copy() for k, v in mem0.items()}
        simulate(factorize(prog, h, s, m), got, order_seed=s + m)
        for k in ref:
            assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k


def _init_ops(prog, seed):
    from tests._cases import fill
    mem = fill(prog, seed)
    if prog.dtype == "i32":                      # small values with zeros, for lor
        g = np.random.Generator(np.random.PCG64(seed))
        for v in mem.values():
            v[...] = g.integers(-2, 3, size=v.shape)
    return mem


@pytest.mark.parametrize("m", [1, 2, 5])
def test_oracle_slots_of_fig7_and_eq1(m):
    """Sec. 4.5 / Fig. 7 and Eq. 1: S dependent stages over m channels fill
    S + m - 1 slots -- the tree and ring(4) examples of Fig. 6 (S = 4, 5) and
    a ring over n single-GPU nodes (S = n - 1, Eq. 1's n + m - 2)."""
    prog = PR.broadcast(12, 600, root=0)
    assert factorize(prog, [2, 2, 3], 3, m).slots() == 4 + m - 1
    assert factorize(prog, [4, 3], 3, m, ring=4).slots() == 5 + m - 1
    for n in (3, 4, 6):
        assert factorize(PR.broadcast(n, 480, root=0), [n], 1, m, ring=n).slots() == n + m - 2
