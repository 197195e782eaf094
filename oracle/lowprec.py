"""Reduced-precision payloads: BF16 and block-scaled FP8-e4m3 (test
infrastructure only).

Formats, written from their definitions:

* **BF16**: the upper 16 bits of an IEEE binary32.  Encoding rounds the
  binary32 value to nearest, ties to even, on bit 16; NaNs stay NaN (quiet).
* **FP8 e4m3** (OCP 8-bit floating point, E4M3): 1 sign bit, 4 exponent bits
  with bias 7, 3 mantissa bits; exponent field 0 holds subnormals
  m/8 * 2**-6; no infinities; S.1111.111 is NaN, so the largest finite value
  is 1.75 * 2**8 = 448.  Encoding rounds to nearest, ties to even, and
  saturates finite values beyond 448 to +-448.
* **FP8 block** (this library's payload layout): 128 e4m3 codes followed by
  their binary32 scale and 12 zero bytes -- 144 bytes per 128 elements.  The
  value of code q is decode(q) * scale.  Quantizing a block of binary32
  values x: amax = max|x| over the values that are not NaN (0 when there are
  none); scale = amax / 448 and inv = 448 / amax (binary32 divisions; both 1
  when amax is 0); codes = encode(x * inv) (binary32 multiply: one
  reciprocal per block rather than a division per value), so a NaN value
  stays a NaN code and does not poison its block.

Reduction of these payloads (the reading of "FP32 accumulation"): every
input of a reduce step is decoded to binary32, the inputs are folded in the
fixed order with binary32 adds, and the result is encoded once (BF16: rounded;
FP8: a fresh block scale and codes).  A tree level is one reduce step, so
partial sums are rounded to the payload at each hierarchy level.
"""
from __future__ import annotations

import numpy as np

FP8_BLOCK = 128
FP8_BLOCK_BYTES = 144
FP8_MAX = 448.0

# one 144-byte FP8 block as a NumPy structured element
FP8_BLOCK_DTYPE = np.dtype([("q", np.uint8, (FP8_BLOCK,)), ("s", "<f4"), ("pad", np.uint8, (12,))])
assert FP8_BLOCK_DTYPE.itemsize == FP8_BLOCK_BYTES


# ---------------------------------------------------------------------------
# BF16
# ---------------------------------------------------------------------------

def bf16_to_f32(h: np.ndarray) -> np.ndarray:
    """BF16 bit patterns -> binary32 values (a BF16 value is the upper half of
    a binary32)."""
    return (np.asarray(h, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def f32_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round binary32 to BF16, nearest-even; NaN -> quiet NaN."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    nan = np.isnan(np.asarray(x, dtype=np.float32))
    r = np.where(nan, (u >> 16) | 0x40, r)
    return r.astype(np.uint16)


# ---------------------------------------------------------------------------
# FP8 e4m3
# ---------------------------------------------------------------------------

def _e4m3_table() -> np.ndarray:
    """binary32 value of each of the 256 codes (NaN for S.1111.111)."""
    vals = np.empty(256, dtype=np.float32)
    for c in range(256):
        s = -1.0 if c & 0x80 else 1.0
        e = (c >> 3) & 0xF
        m = c & 0x7
        if e == 0xF and m == 0x7:
            vals[c] = np.nan
        elif e == 0:
            vals[c] = s * (m / 8.0) * 2.0 ** -6
        else:
            vals[c] = s * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


E4M3_VALUES = _e4m3_table()
_POS = E4M3_VALUES[:0x7F]          # codes 0x00..0x7E: the non-negative finite values, increasing


def e4m3_decode(q: np.ndarray) -> np.ndarray:
    """e4m3 codes -> binary32 values, from the code table of the format's
    definition."""
    return E4M3_VALUES[np.asarray(q, dtype=np.uint8)]


def e4m3_encode(x: np.ndarray) -> np.ndarray:
    """binary32 -> e4m3 code: nearest, ties to the even code, saturating."""
    x = np.asarray(x, dtype=np.float32)
    a = np.abs(x).astype(np.float64)
    sign = np.where(np.signbit(x), 0x80, 0).astype(np.uint8)
    # candidate codes: the largest representable magnitude <= a, and the next one
    lo = np.searchsorted(_POS, a, side="right") - 1          # 0..0x7E
    lo = np.clip(lo, 0, 0x7E)
    hi = np.clip(lo + 1, 0, 0x7E)
    vlo = _POS[lo].astype(np.float64)
    vhi = _POS[hi].astype(np.float64)
    dlo = a - vlo
    dhi = vhi - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi != lo) & (lo % 2 == 1))
    code = np.where(pick_hi, hi, lo).astype(np.uint8)
    code = np.where(a >= FP8_MAX, 0x7E, code).astype(np.uint8)   # saturate
    out = (code | sign).astype(np.uint8)
    return np.where(np.isnan(x), np.uint8(0x7F) | sign, out).astype(np.uint8)


# ---------------------------------------------------------------------------
# FP8 blocks
# ---------------------------------------------------------------------------

def fp8_quantize(x: np.ndarray) -> np.ndarray:
    """binary32 values (length a multiple of 128) -> array of FP8 blocks."""
    x = np.asarray(x, dtype=np.float32).reshape(-1, FP8_BLOCK)
    out = np.zeros(x.shape[0], dtype=FP8_BLOCK_DTYPE)
    amax = np.max(np.where(np.isnan(x), np.float32(0), np.abs(x)), axis=1)
    zero = amax == 0
    safe = np.where(zero, np.float32(1.0), amax).astype(np.float32)
    scale = np.where(zero, np.float32(1.0), (safe / np.float32(FP8_MAX)).astype(np.float32)).astype(np.float32)
    inv = np.where(zero, np.float32(1.0), (np.float32(FP8_MAX) / safe).astype(np.float32)).astype(np.float32)
    out["s"] = scale
    with np.errstate(invalid="ignore", over="ignore"):    # infinite or NaN values stay so
        out["q"] = e4m3_encode((x * inv[:, None]).astype(np.float32))
    return out


def fp8_dequantize(b: np.ndarray) -> np.ndarray:
    """array of FP8 blocks -> binary32 values."""
    b = np.asarray(b, dtype=FP8_BLOCK_DTYPE)
    with np.errstate(invalid="ignore", over="ignore"):
        return (e4m3_decode(b["q"]) * b["s"][:, None]).astype(np.float32).reshape(-1)


# ---------------------------------------------------------------------------
# the fold hooks for semantics.nested_fold and the simulator
# ---------------------------------------------------------------------------

def to_acc(v: np.ndarray, dtype: str) -> np.ndarray:
    """Payload -> binary32 accumulation values (every input of a reduce step
    is decoded before the fold)."""
    if dtype == "bf16":
        return bf16_to_f32(v)
    if dtype == "fp8":
        return fp8_dequantize(v)
    return v


def from_acc(a: np.ndarray, dtype: str) -> np.ndarray:
    """binary32 accumulation values -> payload (one encoding per reduce
    step)."""
    if dtype == "bf16":
        return f32_to_bf16(a)
    if dtype == "fp8":
        return fp8_quantize(a)
    return a


def payload_to_f32(v: np.ndarray, dtype: str) -> np.ndarray:
    """Values a payload buffer represents, as binary32."""
    if dtype in ("bf16", "fp8"):
        return to_acc(v, dtype)
    return np.asarray(v, dtype=np.float32)


def encode(x: np.ndarray, dtype: str) -> np.ndarray:
    """binary32 values -> payload buffer."""
    if dtype == "bf16":
        return f32_to_bf16(x)
    if dtype == "fp8":
        return fp8_quantize(x)
    return np.asarray(x, dtype=np.float32)
