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


NT = 1024  # table entries


def test_table_is_2_pow_k_over_1024():
    assert re.search(r"EXP64_TABLE_SIZE\s*=\s*1024;", SRC)
    body = SRC[SRC.index("#define LAGP_EXP64_TABLE"):SRC.index("static __device__")]
    vals = [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]\d+", body)]
    assert len(vals) == NT
    for k, v in enumerate(vals):
        assert v == nearest(Decimal(2) ** (Decimal(k) / NT)), k


def test_reduction_constants():
    assert const("EXP64_INV_L") == nearest(NT / LN2)
    hi, lo = const("EXP64_L_HI"), const("EXP64_L_LO")
    L = Fraction(LN2 / NT)
    # L_HI: at most 33 significant bits, so N * L_HI is exact for |N| < 2^20
    # (|a| <= 700 gives |N| <= 700 * 1024 / ln 2 < 2^20)
    m, e = math.frexp(hi)
    assert (Fraction(m) * 2 ** 33).denominator == 1
    assert 700 * NT / math.log(2) < 2 ** 20
    assert abs(Fraction(hi) - L) < Fraction(1, 2 ** 33) * Fraction(hi)
    assert lo == nearest(L - Fraction(hi))
    assert const("EXP64_SHIFT") == 1.5 * 2.0 ** 52
    for k in range(2, 5):
        assert const(f"EXP64_C{k}") == nearest(Fraction(1, math.factorial(k))), k
    assert "EXP64_C5" not in SRC
    bits = int(re.search(r"EXP64_FAST_MAX_BITS\s*=\s*(0x[0-9a-fA-F]+)LL", SRC).group(1), 16)
    assert struct.unpack("<d", struct.pack("<Q", bits))[0] == 700.0


def test_polynomial_degree_suffices():
    # |r| <= ln2/2048 after reduction; the degree-4 Taylor remainder is below
    # r^5/5! * e^|r|, far under half an ulp of exp(r) ~ 1
    r = math.log(2) / (2 * NT) * (1 + 1e-12)
    assert r ** 5 / math.factorial(5) * math.exp(r) < 2.0 ** -60
