"""Pins of the oracle's plain semantics (paper Sec. 3, Table 2) against brute
force, closed forms and textbook error bounds -- nothing here re-uses the
oracle's own formulas to produce an expected value."""
import itertools
import math

import numpy as np
import pytest

from oracle import programs as PR
from oracle import semantics as S
from oracle.hierarchy import all_factorizations, level_of
from synth import int_ranks, uniform_ranks

U32 = 1 << 32


def _wrap(v: int) -> int:
    v %= U32
    return v - U32 if v >= 1 << 31 else v


def _brute_sum(rows, idx):
    return _wrap(sum(int(r[idx]) for r in rows))


# ---------------------------------------------------------------------------
# collective definitions vs. element-by-element brute force (int32, wrapping)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 8])
def test_definitions_bruteforce_int(P):
    d = 3
    x = list(int_ranks(P, d * P, seed=P))
    h = [P]
    root = P // 2
    y = S.def_broadcast(x, root)
    for r in range(P):
        for k in range(d * P):
            assert int(y[r][k]) == int(x[root][k])
    y = S.def_reduce(x, root, h)
    assert all(y[r] is None for r in range(P) if r != root)
    for k in range(d * P):
        assert int(y[root][k]) == _brute_sum(x, k)
    y = S.def_allgather([v[:d] for v in x])
    for r in range(P):
        for i in range(P):
            for k in range(d):
                assert int(y[r][i * d + k]) == int(x[i][k])
    y = S.def_reducescatter(x, h)
    for j in range(P):
        for k in range(d):
            assert int(y[j][k]) == _brute_sum(x, j * d + k)
    y = S.def_allreduce(x, h)
    for r in range(P):
        for k in range(d * P):
            assert int(y[r][k]) == _brute_sum(x, k)
    y = S.def_scatter(x, root)
    for j in range(P):
        for k in range(d):
            assert int(y[j][k]) == int(x[root][j * d + k])
    y = S.def_gather([v[:d] for v in x], root)
    for i in range(P):
        for k in range(d):
            assert int(y[root][i * d + k]) == int(x[i][k])
    y = S.def_alltoall(x)
    for i in range(P):
        for j in range(P):
            for k in range(d):
                assert int(y[j][i * d + k]) == int(x[i][j * d + k])


# ---------------------------------------------------------------------------
# the fixed-order sum
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("P", [2, 4, 6, 8, 12])
def test_fold_exact_on_integers(P):
    """Integer-valued float32 inputs whose partial sums stay below 2**24 are
    summed exactly in any order: every hierarchy gives the exact sum."""
    g = np.random.Generator(np.random.PCG64(P))
    x = g.integers(-1000, 1000, size=(P, 257)).astype(np.float32)
    exact = x.astype(np.int64).sum(axis=0)
    for h in all_factorizations(P):
        got = S.nested_fold({r: x[r] for r in range(P)}, h)
        assert got.dtype == np.float32
        assert np.array_equal(got.astype(np.int64), exact)


def test_fold_grouping_hand_example():
    """Four ranks holding 2**24, 1, 1, 1 (float32, round to nearest even).

    A flat left fold ({4}) adds 1 to 2**24 three times; each intermediate
    2**24 + 1 is a tie that rounds to the even 2**24, so the result is 2**24.
    With {2,2} the groups are (2**24 + 1) -> 2**24 and (1 + 1) = 2, and
    2**24 + 2 is representable: 16777218.  With {1,4} (a trivial top level)
    the result equals the flat fold.  A plausible mistake (flat summation,
    wrong group boundaries, pairwise tree) changes one of these."""
    x = {0: np.array([2.0 ** 24], np.float32), 1: np.array([1.0], np.float32),
         2: np.array([1.0], np.float32), 3: np.array([1.0], np.float32)}
    assert float(S.nested_fold(x, [4])[0]) == 16777216.0
    assert float(S.nested_fold(x, [2, 2])[0]) == 16777218.0
    assert float(S.nested_fold(x, [1, 4])[0]) == 16777216.0
    # the group order matters too: the big value in the last group
    y = {0: x[3], 1: x[2], 2: x[1], 3: x[0]}
    # ((1+1)+1) + 2**24 = 3 + 2**24 = 16777219 -> rounds to 16777220 (tie to even)
    assert float(S.nested_fold(y, [4])[0]) == 16777220.0
    # {2,2}: (1+1) + (1 + 2**24 -> 2**24) = 2 + 2**24 = 16777218
    assert float(S.nested_fold(y, [2, 2])[0]) == 16777218.0


def test_fold_sparse_leaves_skip_empty_groups():
    """A leaf set that leaves a subgroup empty folds only the non-empty ones;
    with integer data the result is the exact sum of the leaves."""
    x = {r: np.array([float(r + 1)], np.float32) for r in (1, 5, 6)}
    assert float(S.nested_fold(x, [2, 4])[0]) == 2.0 + 6.0 + 7.0
    assert float(S.nested_fold({3: x[1]}, [2, 2])[0]) == 2.0


@pytest.mark.parametrize("P", [3, 8, 16])
def test_fold_error_bound(P):
    """|fold - exact| <= gamma_{P-1} * sum|x| (recursive summation, any order;
    Higham, Accuracy and Stability, Sec. 4.2), with u = 2**-24."""
    x = uniform_ranks(P, 4096, seed=7 + P)
    u = 2.0 ** -24
    gamma = (P - 1) * u / (1 - (P - 1) * u)
    absum = np.abs(x.astype(np.float64)).sum(axis=0)
    for h in all_factorizations(P)[:6]:
        got = S.nested_fold({r: x[r] for r in range(P)}, h).astype(np.float64)
        for k in range(0, 4096, 97):
            exact = math.fsum(float(v) for v in x[:, k])
            assert abs(got[k] - exact) <= gamma * absum[k] + 1e-30


def test_fold_flat_is_sequential_scalar_fold():
    """With h = {P} the fold is the plain rank-order left fold, here done one
    float32 scalar at a time."""
    P = 7
    x = uniform_ranks(P, 64, seed=3)
    got = S.nested_fold({r: x[r] for r in range(P)}, [P])
    for k in range(64):
        acc = np.float32(x[0, k])
        for r in range(1, P):
            acc = np.float32(acc + np.float32(x[r, k]))
        assert got[k] == acc


def test_level_of():
    h = [2, 2, 3]
    assert level_of(0, 6, h) == 0
    assert level_of(0, 3, h) == 1
    assert level_of(6, 9, h) == 1
    assert level_of(9, 11, h) == 2
    assert level_of(4, 4, h) is None


# ---------------------------------------------------------------------------
# Table 2 compositions vs. the direct definitions
# ---------------------------------------------------------------------------

def _run(builder, P, d, h, x, dtype="f32", **kw):
    prog = builder(P, d, dtype=dtype, **kw)
    mem = prog.allocate()
    for r in range(P):
        if ("send", r) in mem:
            mem[("send", r)][...] = x[r][:mem[("send", r)].shape[0]]
    S.run_program(prog, mem, h)
    return prog, mem


CASES = [(4, [2, 2]), (6, [2, 3]), (8, [2, 4]), (8, [2, 2, 2]), (5, [5])]


@pytest.mark.parametrize("P,h", CASES)
@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_single_step_compositions(P, h, dtype):
    d = 5
    x = uniform_ranks(P, d * P, seed=11) if dtype == "f32" else int_ranks(P, d * P, seed=11)
    xs = [x[r] for r in range(P)]
    root = P - 1

    def recv(mem):
        return [mem[("recv", r)] for r in range(P)]

    _, m = _run(PR.broadcast, P, d, h, xs, dtype, root=root)
    assert all(np.array_equal(a, b) for a, b in zip(recv(m), S.def_broadcast(xs, root)))
    _, m = _run(PR.reduce, P, d, h, xs, dtype, root=root)
    assert np.array_equal(recv(m)[root], S.def_reduce(xs, root, h)[root])
    assert all(not recv(m)[r].any() for r in range(P) if r != root)
    _, m = _run(PR.allgather, P, d, h, xs, dtype)
    assert all(np.array_equal(a, b) for a, b in zip(recv(m), S.def_allgather([v[:d] for v in xs])))
    _, m = _run(PR.reducescatter, P, d, h, xs, dtype)
    assert all(np.array_equal(a, b) for a, b in zip(recv(m), S.def_reducescatter(xs, h)))
    for b in (PR.allreduce_single, PR.allreduce):
        _, m = _run(b, P, d, h, xs, dtype)
        assert all(np.array_equal(a, b2) for a, b2 in zip(recv(m), S.def_allreduce(xs, h)))
    _, m = _run(PR.scatter, P, d, h, xs, dtype, root=root)
    assert all(np.array_equal(a, b) for a, b in zip(recv(m), S.def_scatter(xs, root)))
    _, m = _run(PR.gather, P, d, h, xs, dtype, root=root)
    assert np.array_equal(recv(m)[root], S.def_gather([v[:d] for v in xs], root)[root])
    _, m = _run(PR.alltoall, P, d, h, xs, dtype)
    assert all(np.array_equal(a, b) for a, b in zip(recv(m), S.def_alltoall(xs)))


@pytest.mark.parametrize("P,h", CASES)
def test_multi_step_equivalences(P, h):
    """Table 2 (Multiple): each two-step form equals its single-step form,
    bit for bit in FP32 (the fixed-order sum does not depend on the root)."""
    d = 4
    x = uniform_ranks(P, d * P, seed=5)
    xs = [x[r] for r in range(P)]
    root = 1 % P

    def recv(mem):
        return [mem[("recv", r)] for r in range(P)]

    pairs = [
        (PR.broadcast_ag_scatter, PR.broadcast, {"root": root}, None),
        (PR.reduce_gather_rs, PR.reduce, {"root": root}, root),
        (PR.allgather_bcast_gather, PR.allgather, {"root": root}, None),
        (PR.reducescatter_scatter_reduce, PR.reducescatter, {"root": root}, None),
        (PR.allreduce_bcast_reduce, PR.allreduce_single, {"root": root}, None),
        (PR.allreduce, PR.allreduce_single, {}, None),
    ]
    for multi, single, kw, only in pairs:
        _, a = _run(multi, P, d, h, xs, **kw)
        kw1 = kw if single in (PR.broadcast, PR.reduce) else {}
        _, b = _run(single, P, d, h, xs, **kw1)
        ranks = [only] if only is not None else range(P)
        for r in ranks:
            assert np.array_equal(recv(a)[r], recv(b)[r]), (multi.__name__, r)


def test_race_detection():
    from oracle.model import Program
    P = 4
    prog = Program(P)
    a = prog.buffer(("a", 0), 8)
    b = [prog.buffer(("b", r), 8) for r in range(P)]
    prog.multicast(0, [1, 2], 8, a, {1: b[1], 2: b[2]})
    prog.multicast(3, [2], 4, b[3], {2: b[2].shift(4)})      # overlaps b[2][4:8]
    assert S.find_race(prog) == (0, 0, 1)
    prog2 = Program(P)
    a = prog2.buffer(("a", 0), 8)
    b = [prog2.buffer(("b", r), 8) for r in range(P)]
    prog2.multicast(0, [1, 2], 8, a, {1: b[1], 2: b[2]})
    prog2.fence()
    prog2.multicast(3, [2], 4, b[3], {2: b[2].shift(4)})
    assert S.find_race(prog2) is None
    for name in ("allreduce", "alltoall", "allgather", "reducescatter", "broadcast_ag_scatter"):
        assert S.find_race(PR.BUILDERS[name](P, 3)) is None
    # read/write race: one primitive reads what another writes in the same epoch
    prog3 = Program(P)
    b = [prog3.buffer(("b", r), 8) for r in range(P)]
    prog3.multicast(0, [1], 4, b[0], {1: b[1]})
    prog3.multicast(1, [2], 4, b[1], {2: b[2]})
    assert S.find_race(prog3) is not None


# ---------------------------------------------------------------------------
# other reduction operators (Sec. 3.1: sum, max, logical or, ...)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("op", ["max", "min", "lor"])
@pytest.mark.parametrize("P,h", [(4, [2, 2]), (8, [2, 4]), (6, [3, 2]), (5, [5])])
def test_other_ops_bruteforce(op, P, h):
    """max / min are order-free: the fold equals the plain elementwise max /
    min over ranks (brute force); logical or of two or more contributions is
    1 exactly where some rank is nonzero."""
    g = np.random.Generator(np.random.PCG64(P))
    xi = g.integers(-3, 4, size=(P, 40)).astype(np.int32)        # many zeros for lor
    xi[:, :5] = 0
    got = S.nested_fold({r: xi[r] for r in range(P)}, h, None, op)
    for k in range(40):
        col = [int(xi[r, k]) for r in range(P)]
        want = {"max": max(col), "min": min(col), "lor": int(any(v != 0 for v in col))}[op]
        assert int(got[k]) == want
    if op != "lor":
        xf = uniform_ranks(P, 40, seed=P)
        gotf = S.nested_fold({r: xf[r] for r in range(P)}, h, None, op)
        assert np.array_equal(gotf, xf.max(axis=0) if op == "max" else xf.min(axis=0))


def test_single_leaf_reduction_omits_the_operation():
    """Sec. 3.1: a reduction with one leaf is point-to-point; the operation
    is omitted (a logical or of one nonzero value is the value itself)."""
    x = {3: np.array([5, 0, -2], np.int32)}
    assert list(S.nested_fold(x, [2, 2], None, "lor")) == [5, 0, -2]


def test_ring_order_fold():
    """Sec. 4.4 ring order on three single-rank nodes (hierarchy {3},
    ring(3)) with x = (1e8, -1e8, 1) in binary32, where -1e8 + 1 and 1 + 1e8
    round back to -1e8 and 1e8: the chain from the root's node folds from its
    far end backwards.  Root 0: x0 + (x1 + x2) = 0; root 1: x1 + (x2 + x0) = 0;
    root 2: x2 + (x0 + x1) = 1; the tree (ring(1)) gives (x0 + x1) + x2 = 1."""
    x = {0: np.array([1e8], np.float32), 1: np.array([-1e8], np.float32), 2: np.array([1.0], np.float32)}
    assert float(S.nested_fold(x, [3])[0]) == 1.0
    assert [float(S.nested_fold(x, [3], ring=3, root=r)[0]) for r in range(3)] == [0.0, 0.0, 1.0]
    # nodes of two ranks ({2,2}, ring(2)), root in node 1: (x2 + x3) + (x0 + x1)
    y = {0: np.array([1.0], np.float32), 1: np.array([1e8], np.float32),
         2: np.array([-1e8], np.float32), 3: np.array([1.0], np.float32)}
    assert float(S.nested_fold(y, [2, 2], ring=2, root=3)[0]) == 0.0      # -1e8 + 1e8
    assert float(S.nested_fold(y, [2, 2], ring=2, root=0)[0]) == 0.0      # 1e8 + -1e8
    # a node with one contributing subgroup still folds the incoming partial
    z = {1: np.array([3.0], np.float32), 2: np.array([4.0], np.float32)}
    assert float(S.nested_fold(z, [2, 2], ring=2, root=0)[0]) == 7.0


@pytest.mark.parametrize("h,ring", [([2, 4], 2), ([2, 2, 2], 4), ([4, 2], 8), ([2, 3], 2)])
def test_ring_fold_int32_equals_tree(h, ring):
    """Wrapping int32 addition is order-free: every ring order gives the tree's sum."""
    P = int(np.prod(h))
    x = int_ranks(P, 64, seed=ring)
    for root in range(P):
        vals = {r: x[r] for r in range(P)}
        assert np.array_equal(S.nested_fold(vals, h, ring=ring, root=root), S.nested_fold(vals, h))
