"""CPU oracle for the hierarchical collective path (HiCCL, arXiv 2408.05962).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow reference that the
CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import it. The product
library never imports, links or calls anything here, and nothing here imports
the product package; the two share only the seeded input generators in
``synth``.

Contents (each function cites the passage of the paper it restates):

* ``hierarchy``  -- group arithmetic of the hierarchy vector (Sec. 4.2).
* ``semantics``  -- primitive semantics (Sec. 3.1) with the sum, max, min and
  logical-or operators, the collective definitions of Table 2, the
  hierarchical fixed-order fold and its ring order (Sec. 4.4), FP64 reference
  sums, a race check (Sec. 3.2).
* ``programs``   -- the collectives of Table 2 (single and multiple steps) and
  the All-reduce program of Listing 2, composed from primitives.
* ``factorize``  -- the optimizer of Sec. 4: striping (4.3), ring (4.4), tree
  (4.2) and pipelining (4.5), emitting point-to-point copy / reduce
  operations with their levels and dependencies, plus per-level and HBM
  byte accounting.
* ``simulate``   -- executes a factorized plan on NumPy buffers.
* ``lowprec``    -- BF16 rounding and FP8-e4m3 block-scaled encoding used for
  the reduced-precision payloads.

Where the paper is silent the oracle follows one stated reading; the readings
are listed in the module docstrings. Parity status: every function here is
pinned by a ``-m "not gpu"`` test against brute force, closed forms, the
paper's worked examples or invariants (see ``tests/test_oracle_*.py``).
"""
