"""Accuracy of the kernels' FP64 exponential (Tang's table-driven method)
against CUDA's exp and against exact values (60-digit decimal)."""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def ulp(x: float) -> float:
    return math.ulp(x)


@pytest.fixture(scope="module")
def L():
    from paper_1310_5182_gb300 import lagp
    return lagp


def test_exp64_against_cuda_and_exact(L):
    rng = np.random.default_rng(11)
    a = np.concatenate([
        -rng.uniform(0, 1, 200_000),            # kernel values near 1 (close points)
        -rng.exponential(5.0, 200_000),          # typical -||x-x'||^2/d
        -rng.uniform(0, 700, 100_000),           # whole fast range
        rng.uniform(-700, 700, 50_000),          # positive side as well
        -np.abs(rng.standard_normal(1000)) * 1e-300,  # tiny (and subnormal) arguments
        np.array([0.0, -0.0, -1e-320, -700.0, 700.0, -700.0000001, -708.0, -745.0, -800.0,
                  709.0, -np.inf, np.inf, np.nan]),
    ])
    at = torch.from_numpy(a).cuda()
    tang, lib = (t.cpu().numpy() for t in L.exp64_check(at))
    # special cases
    assert tang[np.isnan(a)].size == 1 and np.isnan(tang[np.isnan(a)]).all()
    assert tang[a == -np.inf][0] == 0.0 and tang[a == np.inf][0] == np.inf
    fin = np.isfinite(a)
    # within 2 ulp of CUDA's exp everywhere
    diff = np.abs(tang[fin] - lib[fin])
    tol = 2 * np.array([ulp(float(v)) for v in lib[fin]])
    assert (diff <= tol).all(), a[fin][diff > tol][:10]
    # within 1 ulp of the exact value on a sample
    getcontext().prec = 40
    idx = rng.choice(np.flatnonzero(fin), 3000, replace=False)
    worst = 0.0
    for i in idx:
        exact = Decimal(float(a[i])).exp()
        e = float(exact)
        if e == 0.0 or not math.isfinite(e):
            continue
        err = abs(Decimal(float(tang[i])) - exact) / Decimal(ulp(e))
        worst = max(worst, float(err))
    assert worst <= 1.0, worst


def test_double_float_split_and_exp(L):
    """The FP32-bulk search's double-float arithmetic: the split of a double
    into hi + lo on the integer pipe (hi the round-to-nearest FP32 value, the
    pair within 2^-47 of the double), and Tang's exponential in double-float
    against the exact exponential of hi + lo (60-digit decimal) for the
    kernel values' range a in [-87, 0]."""
    rng = np.random.default_rng(12)
    mags = np.concatenate([rng.uniform(-1, 1, 20_000), rng.uniform(-3, 3, 5_000) * 10.0 ** rng.integers(-20, 20, 5_000),
                           np.array([0.0, -0.0, 1.0, -1.0, 0.5, 1e-30, -1e-30, 3e38, -3e38])])
    sp, _ = (t.cpu().numpy() for t in L.df_check(torch.from_numpy(mags).cuda()))
    hi, lo = sp[:, 0].astype(np.float64), sp[:, 1].astype(np.float64)
    big = np.abs(mags) >= 2.0 ** -74
    assert np.all(np.abs(hi + lo - mags)[big] <= 2.0 ** -47 * np.abs(mags[big]))
    # hi is the FP32 value of the double rounded to nearest (ties away from
    # zero, where numpy rounds ties to even: exact ties need 29 trailing zero bits)
    f32 = mags.astype(np.float32).astype(np.float64)
    assert np.mean(hi[big] == f32[big]) > 0.999
    assert np.all(np.abs(hi - f32)[big] <= np.spacing(np.abs(f32[big]).astype(np.float32)).astype(np.float64))
    assert sp[np.flatnonzero(mags == 0.0)].tolist() == [[0.0, 0.0], [0.0, 0.0]]
    # exponential
    a = np.concatenate([-rng.uniform(0, 1, 20_000), -rng.exponential(5.0, 20_000), -rng.uniform(0, 87, 20_000),
                        np.array([0.0, -1e-30, -86.99, -87.5, -100.0, -1000.0])])
    sp, ex = (t.cpu().numpy() for t in L.df_check(torch.from_numpy(a).cuda()))
    val = ex[:, 0].astype(np.float64) + ex[:, 1].astype(np.float64)
    assert np.all(val[a < -87.0] == 0.0)
    getcontext().prec = 60
    idx = np.concatenate([rng.choice(np.flatnonzero(a >= -87.0), 4000, replace=False), np.arange(len(a) - 6, len(a) - 3)])
    worst, worst_abs = 0.0, 0.0
    for i in idx:
        x = Decimal(float(sp[i, 0])) + Decimal(float(sp[i, 1]))  # the argument the pair holds
        exact = x.exp()
        got = Decimal(float(ex[i, 0])) + Decimal(float(ex[i, 1]))
        if a[i] >= -70.0:
            # N ln2/1024 is carried to ~2^-48 relative, so the reduced argument's
            # absolute error, and the result's relative error, grow like |a| 2^-48;
            # the kernel values e^-a then keep an absolute error below e^-1 2^-48
            worst = max(worst, float(abs(got - exact) / exact) / max(1.0, abs(float(x))))
        else:
            # below e^-70 ~ 2^-101 the low word leaves FP32's normal range and
            # the pair keeps FP32 precision (such kernel values are negligible
            # beside the O(1) terms of every sum they enter)
            worst_abs = max(worst_abs, float(abs(got - exact)))
    # a few units of 2^-48 times max(1, |a|) (the reduction's and the table's roundings)
    assert worst <= 2.0 ** -45, worst
    assert worst_abs <= 2.0 ** -120, worst_abs
