"""Pins of the constants of the kernels' FP64 exponential (Tang's
table-driven method): every table entry and constant in exp64.cuh must be
the correctly rounded double of its mathematical value, recomputed here in
60-digit decimal arithmetic."""
import math
import os
import re
import struct
from decimal import Decimal, getcontext
from fractions import Fraction

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "paper_1310_5182_gb300", "csrc", "exp64.cuh")).read()
getcontext().prec = 60
LN2 = Decimal(2).ln()


def nearest(x) -> float:
    """Correctly rounded double of an exact rational or decimal."""
    return float(Fraction(x))


def const(name):
    m = re.search(rf"{name}\s*=\s*([0-9a-fx.p+-]+);", SRC)
    assert m, name
    return float.fromhex(m.group(1))


def test_table_is_2_pow_k_over_64():
    body = SRC[SRC.index("#define LAGP_EXP64_TABLE"):SRC.index("static __device__")]
    vals = [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]\d+", body)]
    assert len(vals) == 64
    for k, v in enumerate(vals):
        assert v == nearest(Decimal(2) ** (Decimal(k) / 64)), k


def test_reduction_constants():
    assert const("EXP64_INV_L") == nearest(64 / LN2)
    hi, lo = const("EXP64_L_HI"), const("EXP64_L_LO")
    L = Fraction(LN2 / 64)
    # L_HI: at most 36 significant bits, so N * L_HI is exact for |N| < 2^17
    m, e = math.frexp(hi)
    assert (Fraction(m) * 2 ** 36).denominator == 1
    assert abs(Fraction(hi) - L) < Fraction(1, 2 ** 36) * Fraction(hi)
    assert lo == nearest(L - Fraction(hi))
    assert const("EXP64_SHIFT") == 1.5 * 2.0 ** 52
    for k in range(2, 7):
        assert const(f"EXP64_C{k}") == nearest(Fraction(1, math.factorial(k))), k
    bits = int(re.search(r"EXP64_FAST_MAX_BITS\s*=\s*(0x[0-9a-fA-F]+)LL", SRC).group(1), 16)
    assert struct.unpack("<d", struct.pack("<Q", bits))[0] == 700.0


def test_polynomial_degree_suffices():
    # |r| <= ln2/128 after reduction; the degree-6 Taylor remainder is below
    # r^7/7! * e^|r|, far under half an ulp of exp(r) ~ 1
    r = math.log(2) / 128 * (1 + 1e-12)
    assert r ** 7 / math.factorial(7) * math.exp(r) < 2.0 ** -60
