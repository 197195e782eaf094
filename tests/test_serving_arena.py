"""Host logic of the serving loop's device arena (first fit, 256-byte
aligned, neighbours merged on free), exercised on a CPU tensor: live
regions never overlap, the free list stays sorted and coalesced, the byte
count is exact, and freeing everything restores one free block."""
import numpy as np

from paper_2408_05962_gb300.serving import DeviceArena


def _check(a, live):
    spans = sorted(live.values())
    for (o1, n1), (o2, _) in zip(spans, spans[1:]):
        assert o1 + n1 <= o2                                   # no overlap
    assert all(o % a.align == 0 and n % a.align == 0 for o, n in spans)
    assert a.used == sum(n for _, n in spans)
    fl = a.free_list
    assert fl == sorted(fl)
    for (o1, n1), (o2, _) in zip(fl, fl[1:]):
        assert o1 + n1 < o2                                    # merged: no touching free blocks
    assert a.used + sum(n for _, n in fl) == a.size
    for o, n in fl:                                            # free and live are disjoint
        assert all(o + n <= lo or lo + ln <= o for lo, ln in spans)


def test_arena_random_alloc_free():
    g = np.random.Generator(np.random.PCG64(7))
    a = DeviceArena(1 << 20, "cpu")
    live, k = {}, 0
    for it in range(3000):
        if live and (g.random() < 0.45 or a.used > (3 << 18)):
            key = list(live)[int(g.integers(0, len(live)))]
            a.free(*live.pop(key))
        else:
            got = a.alloc(int(g.integers(1, 40000)))
            if got is not None:
                live[k] = got
                k += 1
        _check(a, live)
    for key in list(live):
        a.free(*live.pop(key))
    _check(a, live)
    assert a.free_list == [(0, 1 << 20)] and a.used == 0


def test_arena_first_fit_and_full():
    a = DeviceArena(4096, "cpu")
    x = a.alloc(1000)          # rounds up to 1024
    y = a.alloc(1024)
    z = a.alloc(2048)
    assert (x, y, z) == ((0, 1024), (1024, 1024), (2048, 2048))
    assert a.alloc(1) is None  # full
    a.free(*y)
    assert a.alloc(2000) is None and a.alloc(512) == (1024, 512)   # first fit in the hole
    a.free(*x)
    assert a.alloc(1024) == (0, 1024)
