"""Thin ctypes binding of the C ABI in ``include/hiccl.h``.

Argument marshalling only: the module-level ``hiccl_*`` functions carry the
C names and signatures (pointer arrays become Python sequences of ints,
tensors or None) and raise ``HicclError`` on a non-OK status.  ``Comm`` is a
small object wrapper over the same calls.  Every step of a collective runs in
the CUDA library; there is no Python or CPU execution path, and loading fails
loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhiccl.so")

F32, I32, BF16, FP8E4M3 = 0, 1, 2, 3
DTYPES = {"f32": F32, "i32": I32, "bf16": BF16, "fp8": FP8E4M3}
ESIZE = {F32: 4, I32: 4, BF16: 2}
FP8_BLOCK, FP8_BLOCK_BYTES = 128, 144     # FP8 payload: 128 e4m3 codes + binary32 scale + 12 zero bytes


def nbytes(dtype: int, elems: int) -> int:
    """Bytes of ``elems`` values of a payload (FP8: whole 128-value blocks)."""
    if dtype == FP8E4M3:
        if elems % FP8_BLOCK:
            raise ValueError("FP8 counts must be multiples of 128")
        return elems // FP8_BLOCK * FP8_BLOCK_BYTES
    return elems * ESIZE[dtype]


SUM, MAX, MIN, LOR = 0, 1, 2, 3
OPS = {"sum": SUM, "max": MAX, "min": MIN, "lor": LOR}
OP_NAMES = {v: k for k, v in OPS.items()}

OK, ERR_INVALID, ERR_STATE, ERR_RACE, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_TOO_LARGE = range(9)
STATUS_NAMES = ["OK", "INVALID", "STATE", "RACE", "NOMEM", "CUDA", "TIMEOUT", "UNSUPPORTED", "TOO_LARGE"]
STATIC_ARENA_BYTES = 16 << 20

COLLECTIVES = {"broadcast": 0, "reduce": 1, "allgather": 2, "reducescatter": 3, "allreduce": 4,
               "scatter": 5, "gather": 6, "alltoall": 7, "allreduce_single": 8}

(OPT_TIMEOUT_NS, OPT_CTAS_PER_SM, OPT_ITEM_BYTES, OPT_ORDER, OPT_THREADS, OPT_TRACE, OPT_SLOT_ITEMS,
 OPT_RING) = range(8)


class HicclError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"HICCL_ERR_{name}: {message}")
        self.status = status
        self.message = message


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_ulonglong) for n in
                ("steps", "copy_steps", "reduce_steps", "items", "edges", "stages",
                 "scratch_bytes", "table_bytes", "slots", "runs")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("stripe", ctypes.c_int), ("pipeline", ctypes.c_int), ("order", ctypes.c_int),
                ("threads", ctypes.c_int), ("item_bytes", ctypes.c_ulonglong), ("us", ctypes.c_float),
                ("trials", ctypes.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class StepDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("level", ctypes.c_int), ("nsrc", ctypes.c_int),
                ("ndst", ctypes.c_int), ("npreds", ctypes.c_int), ("prim", ctypes.c_int),
                ("branch", ctypes.c_int), ("channel", ctypes.c_int), ("op", ctypes.c_int),
                ("reserved", ctypes.c_int), ("nbytes", ctypes.c_ulonglong), ("slot", ctypes.c_ulonglong)]


_lib = None

_SIGS = {
    "hiccl_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "hiccl_add_multicast": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t,
                                           ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "hiccl_add_reduction": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int]),
    "hiccl_add_fence": (ctypes.c_int, [ctypes.c_void_p]),
    "hiccl_add_collective": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_int, ctypes.c_int]),
    "hiccl_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int]),
    "hiccl_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int]),
    "hiccl_start": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hiccl_wait": (ctypes.c_int, [ctypes.c_void_p]),
    "hiccl_level_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]),
    "hiccl_hbm_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong),
                                       ctypes.POINTER(ctypes.c_ulonglong)]),
    "hiccl_debug_image": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_size_t), ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_size_t)]),
    "hiccl_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]),
    "hiccl_get_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.POINTER(StepDesc),
                                      ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_ulonglong),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_ulonglong)]),
    "hiccl_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong]),
    "hiccl_debug_withhold": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_int]),
    "hiccl_validate": (ctypes.c_int, [ctypes.c_void_p]),
    "hiccl_debug_corrupt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hiccl_run_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hiccl_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(TuneResult)]),
    "hiccl_group": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "hiccl_group_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "hiccl_get_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]),
    "hiccl_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hiccl_destroy": (None, [ctypes.c_void_p]),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2408_05962_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError(f"cannot take the address of {type(x)}")


def _ptr_array(seq: Sequence, n: int):
    if len(seq) != n:
        raise ValueError(f"need {n} per-rank pointers, got {len(seq)}")
    return (ctypes.c_void_p * n)(*[_addr(v) or None for v in seq])


def _check(comm, st: int):
    if st != OK:
        msg = lib().hiccl_last_error(comm).decode() if comm else ""
        raise HicclError(st, msg)


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---- the C names ------------------------------------------------------------

def hiccl_create(nranks: int, dtype: int | str = F32):
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    out = ctypes.c_void_p()
    st = lib().hiccl_create(int(nranks), dt, ctypes.byref(out))
    if st != OK:
        raise HicclError(st, "hiccl_create")
    return out.value


def hiccl_add_multicast(comm, send, recv, count: int, root: int, leaves: Sequence[int], nranks: int):
    lv = (ctypes.c_int * len(leaves))(*leaves)
    _check(comm, lib().hiccl_add_multicast(comm, _ptr_array(send, nranks), _ptr_array(recv, nranks),
                                           int(count), int(root), lv, len(leaves)))


def hiccl_add_reduction(comm, send, recv, count: int, leaves: Sequence[int], root: int, nranks: int,
                        op: int = SUM):
    lv = (ctypes.c_int * len(leaves))(*leaves)
    _check(comm, lib().hiccl_add_reduction(comm, _ptr_array(send, nranks), _ptr_array(recv, nranks),
                                           int(count), lv, len(leaves), int(root), int(op)))


def hiccl_add_fence(comm):
    _check(comm, lib().hiccl_add_fence(comm))


def hiccl_add_collective(comm, kind, d: int, send, recv, nranks: int, root: int = 0, op=SUM):
    k = COLLECTIVES[kind] if isinstance(kind, str) else int(kind)
    o = OPS[op] if isinstance(op, str) else int(op)
    _check(comm, lib().hiccl_add_collective(comm, k, int(d), _ptr_array(send, nranks), _ptr_array(recv, nranks),
                                            int(root), o))


def hiccl_init(comm, hierarchy: Sequence[int], stripe: int = 1, pipeline: int = 1):
    h = (ctypes.c_int * len(hierarchy))(*hierarchy)
    _check(comm, lib().hiccl_init(comm, h, len(hierarchy), int(stripe), int(pipeline)))


def hiccl_plan(comm, hierarchy: Sequence[int], stripe: int = 1, pipeline: int = 1):
    h = (ctypes.c_int * len(hierarchy))(*hierarchy)
    _check(comm, lib().hiccl_plan(comm, h, len(hierarchy), int(stripe), int(pipeline)))


def hiccl_start(comm, stream=None):
    s = _stream_handle(stream)
    _check(comm, lib().hiccl_start(comm, ctypes.c_void_p(s) if s else None))


def hiccl_wait(comm):
    _check(comm, lib().hiccl_wait(comm))


def hiccl_level_bytes(comm, nlevels: int) -> list:
    arr = (ctypes.c_ulonglong * nlevels)()
    _check(comm, lib().hiccl_level_bytes(comm, arr, nlevels))
    return [int(v) for v in arr]


def hiccl_hbm_bytes(comm) -> tuple:
    r, w = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    _check(comm, lib().hiccl_hbm_bytes(comm, ctypes.byref(r), ctypes.byref(w)))
    return int(r.value), int(w.value)


def hiccl_plan_info(comm) -> dict:
    info = PlanInfo()
    _check(comm, lib().hiccl_plan_info(comm, ctypes.byref(info)))
    return info.as_dict()


def hiccl_debug_image(comm):
    """(records, items): the host-built table image of a planned communicator
    as bytes and a (nitems, 8) uint32 array of item descriptors (rec, nent,
    nrun, nptr, nsucc, pad...)."""
    import numpy as np
    rb, ni = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(comm, lib().hiccl_debug_image(comm, None, 0, ctypes.byref(rb), None, 0, ctypes.byref(ni)))
    recs = (ctypes.c_ubyte * max(rb.value, 1))()
    items = (ctypes.c_uint32 * max(8 * ni.value, 1))()
    _check(comm, lib().hiccl_debug_image(comm, recs, rb.value, ctypes.byref(rb), items, 32 * ni.value,
                                         ctypes.byref(ni)))
    return bytes(recs)[:rb.value], np.frombuffer(bytes(items), dtype=np.uint32)[:8 * ni.value].reshape(-1, 8)


def hiccl_get_step(comm, index: int) -> dict:
    d = StepDesc()
    _check(comm, lib().hiccl_get_step(comm, int(index), ctypes.byref(d), None, None, None, None, None,
                                      None, None))
    ns, nd, npd = d.nsrc, d.ndst, d.npreds
    sa, ss, sr = (ctypes.c_ulonglong * ns)(), (ctypes.c_int * ns)(), (ctypes.c_int * ns)()
    da, ds, dr = (ctypes.c_ulonglong * nd)(), (ctypes.c_int * nd)(), (ctypes.c_int * nd)()
    pr = (ctypes.c_ulonglong * max(npd, 1))()
    _check(comm, lib().hiccl_get_step(comm, int(index), ctypes.byref(d), sa, ss, sr, da, ds, dr, pr))
    return {
        "kind": "copy" if d.kind == 0 else "reduce", "level": d.level, "nbytes": int(d.nbytes),
        "prim": d.prim, "branch": d.branch, "channel": d.channel, "slot": int(d.slot),
        "op": OP_NAMES[d.op],
        "srcs": [(int(sr[k]), int(sa[k]), bool(ss[k])) for k in range(ns)],
        "dsts": [(int(dr[k]), int(da[k]), bool(ds[k])) for k in range(nd)],
        "preds": [int(pr[k]) for k in range(npd)],
    }


def hiccl_set_option(comm, opt: int, value: int):
    _check(comm, lib().hiccl_set_option(comm, int(opt), int(value)))


def hiccl_validate(comm):
    _check(comm, lib().hiccl_validate(comm))


def hiccl_debug_corrupt(comm, what: int):
    _check(comm, lib().hiccl_debug_corrupt(comm, int(what)))


def hiccl_debug_withhold(comm, index: int, extra: int):
    _check(comm, lib().hiccl_debug_withhold(comm, int(index), int(extra)))


def hiccl_run_static(comm, stream=None):
    """Run a planned communicator from the library's fixed device array
    (no device allocation; blocks until the run is done)."""
    s = _stream_handle(stream)
    st = lib().hiccl_run_static(comm, ctypes.c_void_p(s) if s else None)
    if st != OK:
        raise HicclError(st, "hiccl_run_static")


def hiccl_get_trace(comm, nitems: int):
    """Per-item executor timestamps of the last start: a list of
    (staging began, handed to data warps, data done, successors released, SM,
    first step)."""
    cap = 6 * int(nitems)
    buf = (ctypes.c_ulonglong * max(cap, 1))()
    n = ctypes.c_size_t()
    _check(comm, lib().hiccl_get_trace(comm, buf, cap, ctypes.byref(n)))
    v = [int(x) for x in buf[:n.value]]
    return [tuple(v[i:i + 6]) for i in range(0, len(v), 6)]


def hiccl_autotune(comm, stream=None, flags: int = 0) -> dict:
    """Time candidate configurations and keep the fastest (see the header)."""
    s = _stream_handle(stream)
    r = TuneResult()
    _check(comm, lib().hiccl_autotune(comm, ctypes.c_void_p(s) if s else None, int(flags), ctypes.byref(r)))
    return r.as_dict()


def hiccl_group(comms: Sequence) -> int:
    """A communicator running the given planned communicators in one launch."""
    arr = (ctypes.c_void_p * len(comms))(*[c.handle if isinstance(c, Comm) else c for c in comms])
    out = ctypes.c_void_p()
    st = lib().hiccl_group(arr, len(comms), ctypes.byref(out))
    if st != OK:
        raise HicclError(st, "hiccl_group")
    return out.value


def hiccl_group_plan(comms: Sequence) -> int:
    """The same combined table as hiccl_group, planned on the host only."""
    arr = (ctypes.c_void_p * len(comms))(*[c.handle if isinstance(c, Comm) else c for c in comms])
    out = ctypes.c_void_p()
    st = lib().hiccl_group_plan(arr, len(comms), ctypes.byref(out))
    if st != OK:
        raise HicclError(st, "hiccl_group_plan")
    return out.value


def hiccl_last_error(comm) -> str:
    return lib().hiccl_last_error(comm).decode()


def hiccl_destroy(comm):
    lib().hiccl_destroy(comm)


# ---- object wrapper -------------------------------------------------------------

class Comm:
    """A communicator (the paper's persistent ``Comm<T>``, Listing 2)."""

    def __init__(self, nranks: int, dtype: int | str = "f32", _handle=None):
        self.P = int(nranks)
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.handle = _handle if _handle is not None else hiccl_create(self.P, self.dtype)
        self.nlevels = None

    @classmethod
    def group(cls, comms: Sequence["Comm"]) -> "Comm":
        """One communicator executing all of ``comms`` in a single launch."""
        return cls(comms[0].P, comms[0].dtype, _handle=hiccl_group(comms))

    @classmethod
    def group_plan(cls, comms: Sequence["Comm"]) -> "Comm":
        """The group's combined table, planned on the host only (inspection)."""
        return cls(comms[0].P, comms[0].dtype, _handle=hiccl_group_plan(comms))

    def add_multicast(self, send, recv, count, root, leaves):
        hiccl_add_multicast(self.handle, send, recv, count, root, list(leaves), self.P)

    def add_reduction(self, send, recv, count, leaves, root, op="sum"):
        hiccl_add_reduction(self.handle, send, recv, count, list(leaves), root, self.P,
                            OPS[op] if isinstance(op, str) else int(op))

    def add_fence(self):
        hiccl_add_fence(self.handle)

    def add_collective(self, kind, d, send, recv, root=0, op="sum"):
        hiccl_add_collective(self.handle, kind, d, send, recv, self.P, root, op)

    def init(self, hierarchy, stripe=1, pipeline=1):
        hiccl_init(self.handle, list(hierarchy), stripe, pipeline)
        self.nlevels = len(hierarchy)

    def plan(self, hierarchy, stripe=1, pipeline=1):
        hiccl_plan(self.handle, list(hierarchy), stripe, pipeline)
        self.nlevels = len(hierarchy)

    def start(self, stream=None):
        hiccl_start(self.handle, stream)

    def wait(self):
        hiccl_wait(self.handle)

    def level_bytes(self):
        return hiccl_level_bytes(self.handle, self.nlevels)

    def hbm_bytes(self):
        return hiccl_hbm_bytes(self.handle)

    def plan_info(self):
        return hiccl_plan_info(self.handle)

    def image(self):
        return hiccl_debug_image(self.handle)

    def step(self, i):
        return hiccl_get_step(self.handle, i)

    def steps(self):
        return [self.step(i) for i in range(self.plan_info()["steps"])]

    def autotune(self, stream=None, tune_method: bool = False):
        return hiccl_autotune(self.handle, stream, 1 if tune_method else 0)

    def trace(self):
        return hiccl_get_trace(self.handle, self.plan_info()["items"])

    def run_static(self, stream=None):
        hiccl_run_static(self.handle, stream)

    def set_option(self, opt, value):
        hiccl_set_option(self.handle, opt, value)

    def validate(self):
        hiccl_validate(self.handle)

    def corrupt(self, what):
        hiccl_debug_corrupt(self.handle, what)

    def withhold(self, index, extra):
        hiccl_debug_withhold(self.handle, index, extra)

    def destroy(self):
        if self.handle:
            hiccl_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
