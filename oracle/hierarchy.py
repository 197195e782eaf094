"""Group arithmetic of a hierarchy vector (paper Sec. 4.2).

A hierarchy is a list of integer factors h = [f_0, ..., f_{L-1}] whose product
is the number of ranks P, listed from the top (coarsest) level down.  Ranks are
numbered so that at every level a group is a contiguous block of ranks: the
group at level l holding rank r starts at r - r % G[l] and has G[l] ranks,
where G[l] = f_l * f_{l+1} * ... * f_{L-1} (G[0] = P, G[L] = 1).  A level-l
group is split into f_l subgroups of G[l+1] ranks each (Sec. 4.2, Fig. 5).

Level indices in this package count from the top: level 0 is the first factor
(the paper calls the top level "Level L" and the leaf level "Level 1").
"""
from __future__ import annotations

from math import prod


def check(hierarchy, P: int) -> list[int]:
    """The hierarchy vector as a list of factors whose product is P (Sec. 4.1,
    the hierarchy argument of init)."""
    h = [int(f) for f in hierarchy]
    if not h or any(f < 1 for f in h) or prod(h) != P:
        raise ValueError(f"hierarchy {hierarchy} does not factor P={P}")
    return h


def group_sizes(hierarchy) -> list[int]:
    """G[l] for l = 0..L; G[0] = P and G[L] = 1 (Sec. 4.2)."""
    h = list(hierarchy)
    return [prod(h[l:]) for l in range(len(h) + 1)]


def level_of(a: int, b: int, hierarchy) -> int | None:
    """The level at which ranks a and b first fall into different subgroups,
    i.e. the hierarchy level whose link a transfer a -> b crosses.  None when
    a == b (a local, in-memory transfer).  Sec. 4.2."""
    if a == b:
        return None
    G = group_sizes(hierarchy)
    for l in range(len(hierarchy)):
        if a // G[l + 1] != b // G[l + 1]:
            return l
    raise AssertionError("unreachable")


def ring_level(hierarchy, ring: int) -> int:
    """Level whose groups are the conceptual nodes of ``ring(n)`` (Sec. 4.4).

    Reading: the ring chains the n groups of P/n ranks, which must be the
    groups of one level of the hierarchy, i.e. n = f_0 * ... * f_{l-1} for
    some l; the ring replaces the tree above that level and the tree
    factorizes inside each node.  ``ring(1)`` is the plain tree (l = 0)."""
    G = group_sizes(hierarchy)
    n = int(ring)
    for l, g in enumerate(G):
        if n >= 1 and g * n == G[0]:
            return l
    raise ValueError(f"ring({ring}) does not match a level of hierarchy {list(hierarchy)}")


def all_factorizations(P: int, max_levels: int = 4) -> list[list[int]]:
    """Every ordered factorization of P into factors >= 2, plus [P] itself:
    the hierarchies Sec. 4.1 allows for P ranks."""
    out = []

    def rec(rest, acc):
        if rest == 1:
            if acc:
                out.append(list(acc))
            return
        if len(acc) >= max_levels:
            return
        for f in range(2, rest + 1):
            if rest % f == 0:
                rec(rest // f, acc + [f])

    if P == 1:
        return [[1]]
    rec(P, [])
    return out
