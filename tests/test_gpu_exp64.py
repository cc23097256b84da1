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
