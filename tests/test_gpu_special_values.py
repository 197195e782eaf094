"""NaN and infinity in the payloads: the executor and the oracle agree on
every value that is not NaN bit for bit and on the positions of the NaNs
(the bits of a NaN are not specified: GPU arithmetic returns the canonical
NaN, NumPy propagates an operand's payload)."""
import numpy as np
import pytest

from oracle import lowprec as LP
from oracle import programs as PR
from oracle import semantics as S
from tests._cases import fill
from tests._gpu import run_on_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _values(buf, dtype):
    if dtype == "f32":
        return np.asarray(buf, np.float32)
    return LP.payload_to_f32(buf, dtype)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("name", ["allreduce", "reduce", "broadcast"])
def test_nan_and_infinity(dtype, name):
    P, h, s, m = 8, [2, 4], 2, 2
    d = 1027 if dtype != "fp8" else 3
    prog = PR.BUILDERS[name](P, d, dtype=dtype)
    mem0 = fill(prog, 9)
    g = np.random.Generator(np.random.PCG64(5))
    for r in range(P):
        key = ("send", r)
        x = _values(mem0[key], dtype).copy()
        idx = g.choice(x.size, size=6, replace=False)
        x[idx[:2]] = np.nan
        x[idx[2]] = np.inf
        x[idx[3]] = -np.inf
        x[idx[4]] = np.float32(3.0e38)          # sums overflow to infinity
        mem0[key][...] = LP.encode(x, dtype) if dtype != "f32" else x
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    outs, _ = run_on_gpu(prog, h, s, m, mem0)
    got = outs[0]
    for k in ref:
        a, b = _values(ref[k], dtype), _values(got[k], dtype)
        assert np.array_equal(np.isnan(a), np.isnan(b)), k
        ok = ~np.isnan(a)
        assert np.array_equal(a[ok].view(np.uint32), b[ok].view(np.uint32)), k
        if dtype == "fp8":                       # the block scales too
            assert np.array_equal(ref[k]["s"].view(np.uint32), got[k]["s"].view(np.uint32)), k
