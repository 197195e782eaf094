"""Pins of the oracle's FP64 error reference and of its FP8 block quantizer
against exact rational arithmetic.

Both are checked here with ``fractions.Fraction``, from the definitions of
the formats alone -- none of the oracle's NumPy code is reused:

* binary32: round to nearest, ties to even, with 24 significand bits for
  normal numbers and a fixed quantum of 2**-149 below 2**-126;
* e4m3: the non-negative finite values are (m/8) * 2**-6 for exponent field
  0 and (1 + m/8) * 2**(e-7) otherwise, except e = 15, m = 7 (NaN); encoding
  takes the nearest value, ties to the even code, and saturates at 448;
* the block payload (the library's reading of "per-block scaled" FP8):
  scale = fl32(amax / 448), codes = encode(fl32(x * fl32(448 / amax))).

The hand-chosen blocks contain values whose codes differ between that
multiply-by-reciprocal form and a division by the scale, fl32(x / scale), so
a quantizer that divides fails here.
"""
from __future__ import annotations

import math
import struct
from fractions import Fraction as Q

import numpy as np
import pytest

from oracle import lowprec as LP
from oracle import semantics as S

# ---------------------------------------------------------------------------
# exact models of the formats
# ---------------------------------------------------------------------------


def _f32_bits(u: int) -> float:
    return struct.unpack("<f", struct.pack("<I", u))[0]


def rne_binary32(q: Q) -> Q:
    """The binary32 value nearest to the rational q (ties to an even
    significand); no overflow handling (the cases stay far below 2**128)."""
    if q == 0:
        return Q(0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Q(2) ** e > a:
        e -= 1
    while Q(2) ** (e + 1) <= a:
        e += 1
    quantum = Q(2) ** (max(e, -126) - 23)
    n = a / quantum
    whole = n.numerator // n.denominator
    frac = n - whole
    if frac > Q(1, 2) or (frac == Q(1, 2) and whole % 2 == 1):
        whole += 1
    return sign * whole * quantum


E4M3_POS = []
for _c in range(0x7F):
    _e, _m = (_c >> 3) & 0xF, _c & 0x7
    E4M3_POS.append(Q(_m, 8) * Q(1, 64) if _e == 0 else (1 + Q(_m, 8)) * Q(2) ** (_e - 7))


def e4m3_code(y: Q) -> int:
    """Nearest e4m3 code (ties to the even code), saturating at 448."""
    sign = 0x80 if y < 0 else 0
    a = abs(y)
    if a >= 448:
        return 0x7E | sign
    best = min(range(0x7F), key=lambda c: (abs(a - E4M3_POS[c]), c & 1))
    return best | sign


def exact_block(xs):
    """(scale, codes, division-form codes) of one block of binary32 values."""
    mags = [abs(Q(float(v))) for v in xs]
    # the sign of a product or quotient with a positive factor is the sign of
    # x, signed zeros included
    signs = [0x80 if math.copysign(1.0, float(v)) < 0 else 0 for v in xs]
    amax = max(mags)
    if amax == 0:
        return Q(1), signs, None
    scale = rne_binary32(amax / 448)
    inv = rne_binary32(Q(448) / amax)
    codes = [e4m3_code(rne_binary32(a * inv)) | s for a, s in zip(mags, signs)]
    div = [e4m3_code(rne_binary32(a / scale)) | s for a, s in zip(mags, signs)]
    return scale, codes, div


# ---------------------------------------------------------------------------
# the rational models themselves, against facts of the formats
# ---------------------------------------------------------------------------

def test_exact_models_against_format_facts():
    assert rne_binary32(Q(1, 3)) == Q(_f32_bits(0x3EAAAAAB))
    assert rne_binary32(Q(1) + Q(1, 2 ** 24)) == 1                    # tie -> even significand
    assert rne_binary32(Q(1) + Q(3, 2 ** 24)) == 1 + Q(2, 2 ** 23)    # tie -> even, upwards
    assert rne_binary32(Q(3, 2 ** 150)) == Q(2, 2 ** 149)             # subnormal quantum, tie to even
    assert E4M3_POS[0x38] == 1 and E4M3_POS[0x7E] == 448 and E4M3_POS[0x01] == Q(1, 2 ** 9)
    assert E4M3_POS[0x08] == Q(1, 64) and all(E4M3_POS[c] < E4M3_POS[c + 1] for c in range(0x7E))
    assert e4m3_code(Q(17, 16)) == 0x38          # midpoint of 1 and 1.125 -> even code (1.0)
    assert e4m3_code(Q(19, 16)) == 0x3A          # midpoint of 1.125 and 1.25 -> even code (1.25)
    assert e4m3_code(Q(-500)) == 0xFE


# ---------------------------------------------------------------------------
# FP8 block quantizer
# ---------------------------------------------------------------------------

# (amax, values whose multiply-form and division-form codes differ), found by
# scanning binary32 neighbours of e4m3 midpoints with the rational model
SPLIT_BLOCKS = [
    (0x40400000, [0x3CB92492]),                                   # amax 3.0
    (0x42F6CCCD, [0x3E95D7C6, 0x3EA778AF, 0x3EDC5B6F, 0x3F6DFC58]),  # amax 123.4
    (0x3F547AE1, [0x3B010177, 0x3B102ECF, 0x3BCCE434]),             # amax 0.83
    (0x3FD9999A, [0x3B93A83A, 0x3BC24925]),                         # amax 1.7
]


def _block(amax_bits, special_bits, seed):
    """128 binary32 values: the amax (once, negated at the end), the
    special values with both signs, and seeded values below amax."""
    amax = np.uint32(amax_bits).view(np.float32)
    g = np.random.Generator(np.random.PCG64(seed))
    x = (g.uniform(-1.0, 1.0, 128) * float(amax) * 0.999).astype(np.float32)
    x[0] = amax
    x[127] = -amax
    for i, b in enumerate(special_bits):
        v = np.uint32(b).view(np.float32)
        x[1 + 2 * i] = v
        x[2 + 2 * i] = -v
    return x


@pytest.mark.parametrize("k", range(len(SPLIT_BLOCKS)))
def test_fp8_quantize_matches_exact_codes(k):
    amax_bits, special = SPLIT_BLOCKS[k]
    x = _block(amax_bits, special, seed=k)
    scale, codes, div = exact_block(x)
    got = LP.fp8_quantize(x)
    assert Q(float(got["s"][0])) == scale
    assert [int(c) for c in got["q"][0]] == codes
    # the block really separates the two forms: a quantizer dividing by the
    # scale gives other codes at the hand-chosen positions
    split = [i for i in range(128) if codes[i] != div[i]]
    assert set(range(1, 1 + 2 * len(special))) <= set(split)


def test_fp8_quantize_exact_on_ties_subnormals_and_zero():
    # values landing exactly on e4m3 midpoints after scaling by 448/amax = 1
    # (amax = 448): ties go to the even code
    x = np.zeros(128, np.float32)
    mids = [float((E4M3_POS[c] + E4M3_POS[c + 1]) / 2) for c in range(0x7E)]
    x[:126] = np.array(mids, np.float32)
    x[126] = 448.0
    x[127] = -0.0
    scale, codes, _ = exact_block(x)
    got = LP.fp8_quantize(x)
    assert Q(float(got["s"][0])) == scale == 1
    assert [int(c) for c in got["q"][0]] == codes
    # a block spanning 2**-20 .. amax: small values fall into e4m3 subnormals or flush to zero
    g = np.random.Generator(np.random.PCG64(11))
    y = (np.sign(g.uniform(-1, 1, 128)) * 2.0 ** g.uniform(-20, 0, 128)).astype(np.float32)
    y[0] = 1.0
    scale, codes, _ = exact_block(y)
    got = LP.fp8_quantize(y)
    assert Q(float(got["s"][0])) == scale
    assert [int(c) for c in got["q"][0]] == codes
    assert any(c & 0x7F in range(1, 8) for c in codes) and any(c & 0x7F == 0 for c in codes)
    # an all-zero block: scale 1, zero codes (sign kept)
    z = np.zeros(128, np.float32)
    z[3] = -0.0
    got = LP.fp8_quantize(z)
    assert got["s"][0] == 1.0 and int(got["q"][0][3]) == 0x80 and int(got["q"][0].sum()) == 0x80


def test_fp8_dequantize_exact():
    """decode(code) * scale is one binary32 product, exact for these scales."""
    x = _block(0x42F6CCCD, SPLIT_BLOCKS[1][1], seed=5)
    b = LP.fp8_quantize(x)
    scale = Q(float(b["s"][0]))
    want = [rne_binary32((E4M3_POS[c & 0x7F]) * scale * (-1 if c & 0x80 else 1)) for c in b["q"][0]]
    got = LP.fp8_dequantize(b)
    assert [Q(float(v)) for v in got] == want


# ---------------------------------------------------------------------------
# the FP64 reference sum
# ---------------------------------------------------------------------------

def test_fsum64_cancellation_needs_a_binary64_accumulator():
    """1 + 2**-40 - 1 is 2**-40 in binary64 (exact at every step) but 0 with
    a binary32 accumulator; 2**24 + 1 + 1 is 2**24 + 2 in binary64 but 2**24
    in binary32 (each +1 is a tie that rounds back to even)."""
    v = [np.array([1.0, 2.0 ** 24], np.float32), np.array([2.0 ** -40, 1.0], np.float32),
         np.array([-1.0, 1.0], np.float32)]
    got = S.fsum64(v)
    assert got.dtype == np.float64
    assert got[0] == 2.0 ** -40 and got[1] == 2.0 ** 24 + 2


def test_fsum64_integer_sums_are_exact():
    """Integer-valued binary32 inputs up to 2**24 over 64 ranks: every
    partial sum is an integer below 2**31, exact in binary64, so the result
    equals the int64 sum (a binary32 accumulator drops low bits past 2**24)."""
    g = np.random.Generator(np.random.PCG64(3))
    ints = g.integers(-(2 ** 24), 2 ** 24, size=(64, 4096))
    got = S.fsum64([ints[r].astype(np.float32) for r in range(64)])
    assert np.array_equal(got, ints.sum(axis=0).astype(np.float64))
    assert np.any(np.abs(ints.cumsum(axis=0)) > 2 ** 24)


def test_fsum64_within_the_binary64_bound_of_the_exact_sum():
    """|fsum64 - exact| <= gamma_{n-1} * sum|x| with gamma_k = k u / (1 - k u),
    u = 2**-53 (Higham, recursive summation), element by element against
    math.fsum (correctly rounded) on data spanning six decades; a binary32
    accumulator (u = 2**-24) breaks the bound."""
    g = np.random.Generator(np.random.PCG64(9))
    n = 32
    x = (g.standard_normal((n, 2000)) * 10.0 ** g.uniform(-3, 3, (n, 1))).astype(np.float32)
    got = S.fsum64([x[r] for r in range(n)])
    u = 2.0 ** -53
    gam = (n - 1) * u / (1 - (n - 1) * u)
    worst32 = 0.0
    for j in range(x.shape[1]):
        col = [float(v) for v in x[:, j]]
        exact = math.fsum(col)
        bound = gam * math.fsum(abs(v) for v in col)
        assert abs(got[j] - exact) <= bound + 1e-300, j
        acc32 = np.float32(0)
        for v in x[:, j]:
            acc32 = np.float32(acc32 + v)
        worst32 = max(worst32, abs(float(acc32) - exact) / max(bound, 1e-300))
    assert worst32 > 1.0
