"""Accuracy of the float-pair square root the float64 step uses for its LLF
speed (sqrt_pair in csrc/rsst_math_fp64.cuh), emulated on the CPU in numpy
float32 with the same steps: the double split from its bit pattern into the
leading 24 and trailing 29 significant bits, a reciprocal-square-root seed
(here with a deliberate relative error up to 2^-22, worse than the
hardware's), one Newton step with the square split exactly by an FMA, and
the 2^k rescaling.  The device self-test checks the same bound against
CUDA's sqrt."""
import struct

import numpy as np

F32 = np.float32


def _fmaf(a, b, c):
    # the product of two floats is exact in float64; one rounding to float32
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _float(i):
    return struct.unpack("<f", struct.pack("<I", i & 0xFFFFFFFF))[0]


def sqrt_pair(x, seed_err):
    ix = _bits(x)
    be = ix >> 52
    e = be - 1023
    odd = e & 1
    h = F32(_float(((127 + odd) << 23) | ((ix >> 29) & 0x7FFFFF)))
    l = F32(F32(ix & 0x1FFFFFFF) * F32(_float((75 + odd) << 23)))
    r = F32(F32(1.0 / np.sqrt(np.float64(h))) * F32(1.0 + seed_err))
    s0 = F32(h * r)
    p = F32(s0 * s0)
    d = F32(F32(F32(h - p) - _fmaf(s0, s0, -p)) + l)
    c0 = F32(d * F32(F32(0.5) * r))
    k = (e - odd) >> 1
    return np.float64(s0) * 2.0 ** k, np.float64(c0) * 2.0 ** k


def test_float_pair_sqrt_within_2_to_minus_41():
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(20000):
        x = float(2.0 ** rng.uniform(-200.0, 200.0))
        s, c = sqrt_pair(x, rng.uniform(-1.0, 1.0) * 2.0 ** -22)
        worst = max(worst, abs((s + c) - np.sqrt(x)) / np.sqrt(x))
    assert worst < 2.0 ** -41, worst


def test_split_is_exact_to_float_rounding_of_the_tail():
    """h + l reproduces the double's value 2^(-2k) x to 2^-48."""
    rng = np.random.default_rng(8)
    for _ in range(2000):
        x = float(2.0 ** rng.uniform(-100.0, 100.0))
        ix = _bits(x)
        e = (ix >> 52) - 1023
        odd = e & 1
        h = np.float64(_float(((127 + odd) << 23) | ((ix >> 29) & 0x7FFFFF)))
        l = np.float64(F32(F32(ix & 0x1FFFFFFF) * F32(_float((75 + odd) << 23))))
        y = x * 2.0 ** -(e - odd)
        assert abs((h + l) - y) <= 2.0 ** -48 * y


def _two_sum_pair(sv, cv, sa, ca):
    t = F32(sv + sa)
    bv = F32(t - sv)
    lo = F32(F32(F32(sv - F32(t - bv)) + F32(sa - bv)) + F32(cv + ca))
    h = F32(t + lo)
    return h, F32(lo - F32(h - t))


def _f2d_bits(f):
    b = struct.unpack("<I", struct.pack("<f", float(f)))[0]
    E = (b >> 23) & 0xFF
    sign = (b >> 31) << 63
    ex = 0 if E == 0 else ((0x7FF if E == 255 else E + 896) << 52)
    mant = 0 if E == 0 else (b & 0x7FFFFF) << 29
    return struct.unpack("<d", struct.pack("<Q", sign | ex | mant))[0]


def test_llf_speed_pair_sum_max_and_conversion():
    """c_tot = |V| + a/xi from the two float-pair roots (two-sum, normalised),
    the larger of two sides picked by comparing pairs, and the pair turned
    back into a double by bit assembly: within 2^-41 of the float64 value."""
    rng = np.random.default_rng(9)
    for _ in range(5000):
        sides = []
        for _side in range(2):
            v2 = float(rng.uniform(0.0, 4.0)) * 10.0 ** rng.integers(-8, 3)
            a2x = float(rng.uniform(0.01, 10.0))
            sv, cv = sqrt_pair(v2, rng.uniform(-1, 1) * 2.0 ** -22)
            sa, ca = sqrt_pair(a2x, rng.uniform(-1, 1) * 2.0 ** -22)
            h, l = _two_sum_pair(F32(sv), F32(cv), F32(sa), F32(ca))
            assert abs(float(l)) <= 0.5 * float(np.spacing(h))          # normalised
            sides.append((h, l, np.sqrt(v2) + np.sqrt(a2x)))
        (hL, lL, cL), (hR, lR, cR) = sides
        left = hL > hR or (hL == hR and lL >= lR)
        alpha = _f2d_bits(hL if left else hR) + _f2d_bits(lL if left else lR)
        assert abs(alpha - max(cL, cR)) <= 2.0 ** -41 * max(cL, cR)
    for f in (1.5, -0.25, 0.0, 3.0e-39, float("inf")):
        want = 0.0 if f == 3.0e-39 else f
        assert _f2d_bits(F32(f)) == want
