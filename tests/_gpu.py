"""Run an oracle-described program through the C ABI on the GPU."""
from __future__ import annotations

import numpy as np

GUARD = 64          # guard elements before and after every buffer


def torch_dtype(dtype: str):
    import torch
    return {"f32": torch.float32, "i32": torch.int32, "bf16": torch.int16, "fp8": torch.uint8}[dtype]


def run_on_gpu(prog, h, s, m, mem0: dict, repeats: int = 1, misalign_elems: int = 0, options=None,
               reset_between=True, check_guards=True):
    """Execute ``prog`` on device copies of ``mem0``; returns (host results,
    communicator).  Every buffer sits between guard bands that must survive."""
    import torch

    from tests._bridge import register

    dev = torch.device("cuda:0")
    tdt = torch_dtype(prog.dtype)
    dev_bufs, base_addr = {}, {}
    esize = np.dtype(mem0[next(iter(mem0))].dtype).itemsize   # FP8: one 144-byte block
    sentinel = {}
    for kidx, (key, arr) in enumerate(mem0.items()):
        n = arr.shape[0]
        host = np.empty(n + 2 * GUARD + misalign_elems, dtype=arr.dtype)
        g = np.random.Generator(np.random.PCG64(1000 + kidx))
        host.view(np.uint8)[...] = g.integers(0, 256, size=host.nbytes, dtype=np.uint8)
        host[GUARD + misalign_elems:GUARD + misalign_elems + n] = arr
        sentinel[key] = host.copy()
        t = torch.from_numpy(host.view(np.uint8).copy()).to(dev)
        dev_bufs[key] = t
        base_addr[key] = int(t.data_ptr()) + (GUARD + misalign_elems) * esize

    comm = register(prog, lambda ref: base_addr[ref.key] + ref.off * esize)
    for opt, val in (options or {}).items():
        comm.set_option(opt, val)
    comm.init(h, s, m)
    results = []
    for rep in range(repeats):
        if rep and reset_between:
            for key, t in dev_bufs.items():
                t.copy_(torch.from_numpy(sentinel[key].view(np.uint8)))
        comm.start()
        comm.wait()
        torch.cuda.synchronize()
        out = {}
        for key, t in dev_bufs.items():
            host = t.cpu().numpy().view(mem0[key].dtype)
            if check_guards:
                lo = GUARD + misalign_elems
                n = mem0[key].shape[0]
                ref = sentinel[key]
                assert np.array_equal(host[:lo].view(np.uint8), ref[:lo].view(np.uint8)), ("guard before", key)
                assert np.array_equal(host[lo + n:].view(np.uint8), ref[lo + n:].view(np.uint8)), ("guard after", key)
            out[key] = host[GUARD + misalign_elems:GUARD + misalign_elems + mem0[key].shape[0]].copy()
        results.append(out)
    return results, comm


def assert_bit_equal(ref: dict, got: dict):
    for k in ref:
        a, b = ref[k], got[k]
        assert a.shape == b.shape, k
        if not np.array_equal(a.view(np.uint8), b.view(np.uint8)):
            bad = np.nonzero(a.view(np.uint8) != b.view(np.uint8))[0]
            raise AssertionError(f"{k}: {len(bad)} bytes differ, first at byte {bad[0]}")
