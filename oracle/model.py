"""Data model of a composed collective (paper Sec. 3, Listing 1).

A program holds named per-rank buffers and a sequence of epochs.  Each epoch
is a set of primitives registered between two fences; all primitives of an
epoch run concurrently (Sec. 3.2) and a fence orders the epochs (Sec. 3.3).

* ``Multicast(root i, leaves j, count d)``: the root's source range is
  replicated into every leaf's destination range (Sec. 3.1, M(i, j, d)).
* ``Reduction(leaves i, root j, count d)``: the leaves' source ranges are
  summed into the root's destination range (Sec. 3.1, R(i, j, d, op)); the op
  is sum.

A location is a ``Ref(key, off)``: an element offset into a named buffer.  The
keys of user buffers are tuples such as ``("send", r)``; the factorizer's
relay buffers use ``("scratch", k)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .lowprec import FP8_BLOCK_DTYPE

# storage of one counted unit: a value, or for FP8 a 144-byte block of 128
# values and their scale (counts of FP8 programs are in blocks)
DTYPES = {
    "f32": np.dtype(np.float32),
    "i32": np.dtype(np.int32),
    "bf16": np.dtype(np.uint16),     # bit patterns; see lowprec
    "fp8": FP8_BLOCK_DTYPE,          # 128 e4m3 codes + binary32 scale; see lowprec
}

# units per piece-boundary quantum: 16 bytes of values, one FP8 block
QUANTUM = {"f32": 4, "i32": 4, "bf16": 8, "fp8": 1}


@dataclass(frozen=True)
class Ref:
    """A location: an element offset into a named buffer (the paper's
    ``sendbuf + offset`` of Listing 1)."""
    key: tuple
    off: int

    def shift(self, k: int) -> "Ref":
        """The location ``k`` elements further (pointer arithmetic of Listing 1)."""
        return Ref(self.key, self.off + k)


@dataclass
class Multicast:
    """M(i, j, d) of Sec. 3.1: root i's source range replicated into every
    leaf's destination range."""
    root: int
    leaves: tuple
    count: int
    src: Ref                      # the root's source range
    dsts: dict                    # leaf rank -> Ref of its destination range

    kind = "multicast"


@dataclass
class Reduction:
    """R(i, j, d, op) of Sec. 3.1: the leaves' source ranges combined into
    the root's destination range."""
    leaves: tuple
    root: int
    count: int
    srcs: dict                    # leaf rank -> Ref of its source range
    dst: Ref                      # the root's destination range
    op: str = "sum"               # sum | max | min | lor

    kind = "reduction"


@dataclass
class Program:
    """A composed collective (Sec. 3.2, Listing 1): buffers and epochs of
    primitives separated by fences."""
    P: int
    dtype: str = "f32"
    buffers: dict = field(default_factory=dict)     # key -> length (elements)
    epochs: list = field(default_factory=lambda: [[]])

    # -- registration (Listing 1) ------------------------------------------
    def buffer(self, key, length: int) -> Ref:
        """A named per-rank buffer of ``n`` units (a user buffer of Listing 1)."""
        self.buffers[key] = int(length)
        return Ref(key, 0)

    def multicast(self, root: int, leaves, count: int, src: Ref, dsts: dict) -> None:
        """Register M(root, leaves, count) in the current epoch (Sec. 3.1)."""
        self.epochs[-1].append(Multicast(int(root), tuple(sorted(int(j) for j in leaves)),
                                         int(count), src, dict(dsts)))

    def reduction(self, leaves, root: int, count: int, srcs: dict, dst: Ref, op: str = "sum") -> None:
        """Register R(leaves, root, count, op) in the current epoch (Sec. 3.1)."""
        self.epochs[-1].append(Reduction(tuple(sorted(int(i) for i in leaves)), int(root),
                                         int(count), dict(srcs), dst, op))

    def fence(self) -> None:
        """Close the current epoch (Sec. 3.3)."""
        self.epochs.append([])

    @property
    def primitives(self):
        """All primitives with their epoch indices, in registration order."""
        return [p for ep in self.epochs for p in ep]

    def allocate(self, fill=None) -> dict:
        """Zero-filled NumPy arrays for every user buffer."""
        dt = DTYPES[self.dtype]
        return {k: np.zeros(n, dtype=dt) for k, n in self.buffers.items()}
