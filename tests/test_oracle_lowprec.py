"""Pins of the reduced-precision payload formats (BF16, FP8 e4m3 with
per-128-element block scales) and of their fixed-order reduction, against
the formats' definitions, exhaustive enumeration, brute-force nearest values
and error bounds."""
import math

import numpy as np
import pytest

from oracle import lowprec as LP
from oracle import programs as PR
from oracle import semantics as S
from oracle.factorize import factorize
from oracle.simulate import simulate
from synth import scaled_normal_ranks, uniform_ranks


# ---- BF16 -----------------------------------------------------------------------

def test_bf16_hand_values():
    one = np.float32(1.0)
    # 1 + 2**-8 is halfway between 1 and 1 + 2**-7: ties to the even mantissa (1.0)
    assert LP.f32_to_bf16(np.array([1 + 2.0 ** -8], np.float32))[0] == 0x3F80
    # 1 + 3 * 2**-8 is halfway between 1 + 2**-7 (odd) and 1 + 2**-6 (even)
    assert LP.f32_to_bf16(np.array([1 + 3 * 2.0 ** -8], np.float32))[0] == 0x3F82
    # just above the halfway point rounds up
    assert LP.f32_to_bf16(np.array([np.nextafter(np.float32(1 + 2.0 ** -8), np.float32(2))], np.float32))[0] == 0x3F81
    assert LP.f32_to_bf16(np.array([-2.0], np.float32))[0] == 0xC000
    assert float(LP.bf16_to_f32(np.array([0x4049], np.uint16))[0]) == 3.140625
    assert np.isnan(LP.bf16_to_f32(LP.f32_to_bf16(np.array([np.nan], np.float32))))[0]


def test_bf16_roundtrip_exhaustive():
    h = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    f = LP.bf16_to_f32(h)
    ok = ~np.isnan(f)
    assert np.array_equal(LP.f32_to_bf16(f)[ok], h[ok])


def test_bf16_nearest_bruteforce():
    g = np.random.Generator(np.random.PCG64(1))
    x = (g.standard_normal(20000) * 10.0 ** g.uniform(-5, 5, 20000)).astype(np.float32)
    r = LP.f32_to_bf16(x)
    y = LP.bf16_to_f32(r).astype(np.float64)
    for d in (-1, 1):
        nb = LP.bf16_to_f32((r.astype(np.int64) + d).astype(np.uint16)).astype(np.float64)
        assert np.all(np.abs(y - x) <= np.abs(nb - x))


# ---- FP8 e4m3 -------------------------------------------------------------------

def test_e4m3_definition_values():
    v = LP.E4M3_VALUES
    assert v[0x00] == 0.0 and v[0x80] == 0.0 and math.copysign(1, v[0x80]) == -1
    assert v[0x38] == 1.0                      # exponent 7 = bias, mantissa 0
    assert v[0x7E] == 448.0                    # largest finite
    assert v[0x08] == 2.0 ** -6                # smallest normal
    assert v[0x01] == 2.0 ** -9                # smallest subnormal
    assert v[0x07] == 7 * 2.0 ** -9
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    assert np.sum(np.isnan(v)) == 2
    fin = v[:0x7F]
    assert np.all(np.diff(fin) > 0)            # codes 0..0x7E increase


def test_e4m3_encode_roundtrip_and_ties():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF, 0x80)], np.uint8)
    assert np.array_equal(LP.e4m3_encode(LP.e4m3_decode(codes)), codes)
    # midpoints between consecutive codes go to the even code
    pos = LP.E4M3_VALUES[:0x7F].astype(np.float64)
    for c in range(0x7E):
        mid = np.float32((pos[c] + pos[c + 1]) / 2)
        if float(mid) != (pos[c] + pos[c + 1]) / 2:
            continue                           # midpoint not exact in binary32
        got = int(LP.e4m3_encode(np.array([mid]))[0])
        assert got == (c if c % 2 == 0 else c + 1), c
    # saturation of finite values beyond 448, sign kept
    assert list(LP.e4m3_encode(np.array([449.0, 1e30, -500.0], np.float32))) == [0x7E, 0x7E, 0xFE]


def test_e4m3_nearest_bruteforce():
    g = np.random.Generator(np.random.PCG64(2))
    x = (g.standard_normal(20000) * 10.0 ** g.uniform(-4, 2.6, 20000)).astype(np.float32)
    q = LP.e4m3_encode(x)
    y = LP.e4m3_decode(q).astype(np.float64)
    fin = LP.E4M3_VALUES[:0x7F].astype(np.float64)
    allv = np.concatenate([fin, -fin])
    best = np.min(np.abs(allv[None, :] - np.clip(x, -448, 448)[:, None].astype(np.float64)), axis=1)
    assert np.allclose(np.abs(y - np.clip(x, -448, 448)), best, rtol=0, atol=0)


def test_fp8_block_quantize_bounds():
    x = scaled_normal_ranks(1, 128 * 256, seed=3)[0]
    b = LP.fp8_quantize(x)
    assert b.dtype.itemsize == 144 and b.shape == (256,)
    xb = x.reshape(-1, 128)
    amax = np.abs(xb).max(axis=1)
    assert np.array_equal(b["s"], (amax / np.float32(448)).astype(np.float32))
    inv = (np.float32(448) / amax).astype(np.float32)
    assert np.array_equal(b["q"], LP.e4m3_encode((xb * inv[:, None]).astype(np.float32)))
    assert np.all(np.abs(LP.e4m3_decode(b["q"])).max(axis=1) == 448.0)   # the max element maps to +-448
    y = LP.fp8_dequantize(b).reshape(-1, 128)
    err = np.abs(y.astype(np.float64) - xb)
    bound = np.maximum(2.0 ** -4 * np.abs(xb), 2.0 ** -10 * b["s"][:, None]) * (1 + 1e-6)
    assert np.all(err <= bound)
    z = LP.fp8_quantize(np.zeros(128, np.float32))
    assert z["s"][0] == 1.0 and not z["q"].any()
    assert not b["pad"].any()


# ---- reductions of BF16 / FP8 payloads ----------------------------------------------

def _rel_l2(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("dtype,tol", [("bf16", 1e-2), ("fp8", 6e-2)])
def test_lowprec_allreduce_error_vs_fp64(dtype, tol):
    """The fixed-order reduction of the reduced-precision payloads stays within
    the stated relative error of the FP64 sum of the (dequantized) inputs on
    data spanning six decades across ranks."""
    P, h = 32, [4, 8]
    n = 128 * 64
    x = scaled_normal_ranks(P, n, seed=4)
    enc = [LP.encode(x[r], dtype) for r in range(P)]
    ref = S.fsum64([LP.payload_to_f32(e, dtype) for e in enc])
    y = LP.payload_to_f32(S.nested_fold({r: enc[r] for r in range(P)}, h, dtype), dtype)
    assert _rel_l2(y, ref) <= tol


def test_lowprec_fold_levels_round():
    """BF16: each tree level rounds once.  Ranks 0..3 hold 1, 2**-8, 2**-8,
    2**-8 over {2,2}: group 0 folds 1 + 2**-8 = 1.00390625 -> rounds (tie) to
    1.0; group 1 folds 2**-7 exactly; the top folds 1 + 2**-7 = 1.0078125,
    representable.  A flat fold {4} rounds once at the end: 1 + 3*2**-8 ->
    1.015625 (tie to even)."""
    vals = [1.0, 2.0 ** -8, 2.0 ** -8, 2.0 ** -8]
    x = {r: LP.f32_to_bf16(np.array([v], np.float32)) for r, v in enumerate(vals)}
    assert float(LP.bf16_to_f32(S.nested_fold(x, [2, 2], "bf16"))[0]) == 1.0078125
    assert float(LP.bf16_to_f32(S.nested_fold(x, [4], "bf16"))[0]) == 1.015625


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("name", ["allreduce", "reducescatter", "reduce", "allgather", "alltoall"])
@pytest.mark.parametrize("P,h,s,m", [(8, [2, 4], 1, 1), (8, [2, 4], 4, 2), (12, [2, 2, 3], 3, 2)])
def test_lowprec_simulated_equals_semantics(dtype, name, P, h, s, m):
    d = 24 if dtype == "bf16" else 2          # FP8 counts are 128-value blocks
    prog = PR.BUILDERS[name](P, d, dtype=dtype)
    from tests._cases import fill
    mem0 = fill(prog, 8)
    ref = {k: v.copy() for k, v in mem0.items()}
    S.run_program(prog, ref, h)
    got = {k: v.copy() for k, v in mem0.items()}
    simulate(factorize(prog, h, s, m), got, order_seed=s + m)
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k


def test_fp8_block_amax_ignores_nan():
    """A NaN value stays a NaN code without poisoning its block: the scale
    comes from the largest magnitude that is not NaN, and a block of NaNs
    only keeps scale 1."""
    x = np.linspace(-2.0, 3.0, 128, dtype=np.float32)
    x[5] = np.nan
    b = LP.fp8_quantize(x)
    assert b["s"][0] == np.float32(np.float32(3.0) / np.float32(448.0))
    y = LP.fp8_dequantize(b)
    assert np.isnan(y[5]) and np.sum(np.isnan(y)) == 1
    assert float(y[-1]) == 3.0
    allnan = LP.fp8_quantize(np.full(128, np.nan, np.float32))
    assert allnan["s"][0] == 1.0 and np.all(np.isnan(LP.fp8_dequantize(allnan)))
