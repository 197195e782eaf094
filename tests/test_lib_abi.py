"""The C-ABI library builds, loads without a GPU, and exports every function
that include/hiccl.h declares; argument validation and the state machine work
without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2408_05962_gb300 import build as B
from paper_2408_05962_gb300 import hiccl as H

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hiccl.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hiccl_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    lib = ctypes.CDLL(H.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    for n in declared_functions():
        assert hasattr(H, n), n


def _comm(P=4, dt="f32"):
    return H.Comm(P, dt)


def test_validation_errors():
    c = _comm(4)
    base = [0x1000 * (r + 1) for r in range(4)]
    with pytest.raises(H.HicclError) as e:
        c.add_multicast(base, base, 8, 7, [1])            # root out of range
    assert e.value.status == H.ERR_INVALID
    with pytest.raises(H.HicclError) as e:
        c.add_multicast(base, base, 8, 0, [1, 1])         # duplicate leaf
    assert e.value.status == H.ERR_INVALID
    c.add_multicast(base, base, 8, 0, [])                 # no leaf: nothing registered
    with pytest.raises(H.HicclError) as e:
        c.add_reduction(base, base, 8, [], 0)             # a reduction needs a leaf
    assert e.value.status == H.ERR_INVALID
    with pytest.raises(H.HicclError) as e:
        c.add_multicast([0] * 4, base, 8, 0, [1])         # null root buffer
    assert e.value.status == H.ERR_INVALID
    with pytest.raises(H.HicclError) as e:
        c.add_multicast([b + 2 for b in base], base, 8, 0, [1])   # misaligned f32
    assert e.value.status == H.ERR_INVALID
    c.add_multicast(base, [b + 0x100000 for b in base], 8, 0, [1, 2])
    for h, s, m in [([3], 1, 1), ([2, 2], 0, 1), ([2, 2], 5, 1), ([2, 2], 1, 0), ([0, 4], 1, 1)]:
        with pytest.raises(H.HicclError) as e:
            c.plan(h, s, m)
        assert e.value.status == H.ERR_INVALID, (h, s, m)
    c.plan([2, 2], 2, 2)
    with pytest.raises(H.HicclError) as e:
        c.add_fence()                                     # composition closed
    assert e.value.status == H.ERR_STATE
    with pytest.raises(H.HicclError) as e:
        c.start()                                         # planned, not initialized
    assert e.value.status == H.ERR_STATE
    with pytest.raises(H.HicclError) as e:
        c.wait()
    assert e.value.status == H.ERR_STATE


def test_race_rejected():
    c = _comm(4)
    a = [0x100000 * (r + 1) for r in range(4)]
    c.add_multicast(a, a, 16, 0, [1, 2])
    c.add_multicast([x + 0x10000 for x in a], [a[0], a[1] + 32, 0, 0], 4, 1, [1])  # overlaps rank 1's recv
    with pytest.raises(H.HicclError) as e:
        c.plan([2, 2])
    assert e.value.status == H.ERR_RACE
    c2 = _comm(4)
    c2.add_multicast(a, a, 16, 0, [1, 2])
    c2.add_fence()
    c2.add_multicast([x + 0x10000 for x in a], [a[0], a[1] + 32, 0, 0], 4, 1, [1])
    c2.plan([2, 2])


def test_reduction_operators_checked():
    c = _comm(2)
    a = [0x1000, 0x2000]
    with pytest.raises(H.HicclError) as e:
        H.hiccl_add_reduction(c.handle, a, a, 4, [0, 1], 0, 2, op=7)
    assert e.value.status == H.ERR_INVALID
    with pytest.raises(H.HicclError) as e:           # logical or on floats
        H.hiccl_add_reduction(c.handle, a, a, 4, [0, 1], 0, 2, op=H.LOR)
    assert e.value.status == H.ERR_UNSUPPORTED
    for op in (H.SUM, H.MAX, H.MIN):
        H.hiccl_add_reduction(c.handle, a, a, 4, [0, 1], 0, 2, op=op)
        c.add_fence()
    f8 = H.Comm(2, "fp8")
    with pytest.raises(H.HicclError) as e:
        H.hiccl_add_reduction(f8.handle, a, a, 128, [0, 1], 0, 2, op=H.MAX)
    assert e.value.status == H.ERR_UNSUPPORTED
    i32 = H.Comm(2, "i32")
    H.hiccl_add_reduction(i32.handle, a, a, 4, [0, 1], 0, 2, op=H.LOR)


def test_options():
    c = _comm(2)
    c.set_option(H.OPT_TIMEOUT_NS, 5_000_000)
    c.set_option(H.OPT_CTAS_PER_SM, 3)
    c.set_option(H.OPT_ITEM_BYTES, 65536)
    c.set_option(H.OPT_ORDER, 1)
    with pytest.raises(H.HicclError):
        c.set_option(H.OPT_CTAS_PER_SM, 0)
    with pytest.raises(H.HicclError):
        c.set_option(99, 1)


def test_empty_program_plans():
    c = _comm(3)
    c.plan([3])
    info = c.plan_info()
    assert info["steps"] == 0 and info["items"] == 0
    assert c.level_bytes() == [0]


_NOMEM_CHILD = r"""
import resource, sys
sys.path.insert(0, sys.argv[1])
from paper_2408_05962_gb300 import hiccl as H
H.lib()                                   # load before the limit
lim = int(sys.argv[2])
resource.setrlimit(resource.RLIMIT_AS, (lim, lim))
P, d = 1024, 1024
base = 1 << 40
send = [base + r * (d * P * 4 + 4096) for r in range(P)]
recv = [base + (1 << 38) + r * (d * P * 4 + 4096) for r in range(P)]
c = H.Comm(P, "f32")
c.add_collective("allreduce", d, send, recv)
try:
    c.plan([32, 32], 32, 4)               # needs several GB of host memory
    print("planned")
except H.HicclError as e:
    print("status", e.status, e.message)
"""


def test_host_memory_exhaustion_is_a_status_not_an_abort():
    """No call of the C ABI lets a C++ exception escape: planning a schedule
    of hundreds of millions of operands under a 1.5 GB address-space limit
    returns HICCL_ERR_NOMEM (the process does not abort)."""
    import subprocess
    import sys
    pytest.importorskip("resource")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    limit = 1536 << 20
    r = subprocess.run([sys.executable, "-c", _NOMEM_CHILD, root, str(limit)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    out = r.stdout.strip().splitlines()[-1]
    assert out.startswith(f"status {H.ERR_NOMEM} "), out


def test_static_size_check_precedes_any_cuda_call():
    """hiccl_run_static rejects a plan larger than its fixed device array
    before any CUDA call: on a host without a GPU it still answers
    HICCL_ERR_TOO_LARGE (a CUDA call there would fail with HICCL_ERR_CUDA)."""
    import torch

    from oracle import programs as PR
    from tests._bridge import FakeAddresses, register
    if torch.cuda.is_available():
        pytest.skip("checks the order of the checks on a host without a GPU")
    prog = PR.reducescatter(64, 1 << 18)
    fake = FakeAddresses(prog)
    comm = register(prog, fake.addr)
    comm.plan([4, 4, 4], 1, 1)
    with pytest.raises(H.HicclError) as e:
        comm.run_static()
    assert e.value.status == H.ERR_TOO_LARGE
    comm.destroy()
