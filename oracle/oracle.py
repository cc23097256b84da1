"""ctypes wrapper around the plain FP64 C oracle (lagp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py.  The CUDA library never imports it.

All inputs are numpy arrays; floating inputs are converted to float64 (exact
for float32 data), integer inputs to int32.  Functions follow the paper's
notation: X (N x p design), Y (N responses), Xref (M x p reference
locations), n0/n/N' design sizes, d lengthscale, g nugget.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lagp_oracle.c")
_LIB = os.path.join(_HERE, "liblagp_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOTPD = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liblagp_oracle.so (gcc, FP64, no FMA
    contraction, OpenMP over locations).  Returns the library path."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lagp_oracle.h"))
        ):
            return _LIB
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64, I32, D = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_separable.argtypes = [P, ctypes.c_int]
        lib.orc_knn.argtypes = [P, I64, ctypes.c_int, P, I64, P, I32, P]
        lib.orc_alc_select.argtypes = [P, I64, ctypes.c_int, P, I64, P, P, I32, I32, P, I32, P, D,
                                       P, P, I32, P, P, P]
        lib.orc_alc_scores.argtypes = [P, I64, ctypes.c_int, P, P, I32, P, I32, D, D, P, P]
        lib.orc_partitioned_inverse.argtypes = [P, I64, ctypes.c_int, P, I32, I32, D, D, P]
        lib.orc_predict.argtypes = [P, P, I64, ctypes.c_int, P, I64, P, P, I32, P, D, P, P, P, P]
        lib.orc_llik.argtypes = [P, P, I64, ctypes.c_int, I64, P, P, I32, P, D, P, P, P, P]
        lib.orc_mle.argtypes = [P, P, I64, ctypes.c_int, I64, P, P, I32, P, D, D, D, I32, P, P,
                                P, P, P]
        lib.orc_predict_grad.argtypes = [P, P, I64, ctypes.c_int, P, I64, P, P, I32, P, D, P, P,
                                         P, P, P, P]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != ORC_OK:
        raise ValueError(f"oracle {what}: invalid arguments (code {rc})")


def set_separable(theta=None):
    """Separable lengthscales theta (p values) for the search and prediction
    correlations, or None for the isotropic form (see lagp_oracle.h)."""
    if theta is None:
        _check(_load().orc_set_separable(None, 0), "set_separable")
        return
    t = _f64(np.asarray(theta, dtype=np.float64))
    _check(_load().orc_set_separable(_ptr(t), len(t)), "set_separable")


def set_threads(n: int) -> int:
    """OpenMP threads for the per-location loops; returns the count in effect."""
    return int(_load().orc_set_threads(int(n)))


def _per_loc(v, M, dtype, default):
    if v is None:
        return np.full(M, default, dtype=dtype)
    v = np.asarray(v, dtype=dtype)
    return np.ascontiguousarray(np.broadcast_to(v, (M,)).copy())


def knn(X, Xref, Np_max, Np=None):
    """Exact N'-nearest neighbours, rows sorted by (d2, row); -1 padded."""
    X, Xref = _f64(X), _f64(Xref)
    N, p = X.shape
    M = Xref.shape[0]
    Npa = None if Np is None else _i32(np.broadcast_to(Np, (M,)))
    idx = np.empty((M, Np_max), dtype=np.int32)
    _check(_load().orc_knn(_ptr(X), N, p, _ptr(Xref), M, _ptr(Npa), int(Np_max), _ptr(idx)), "knn")
    return idx


def alc_select(X, Xref, idx, n0, n, d, g, Np=None, nmax=None, topk=0):
    """Greedy ALC search.  Returns dict(sel, alc, status[, top_idx, top_val])."""
    X, Xref, idx = _f64(X), _f64(Xref), _i32(idx)
    N, p = X.shape
    M, Npmax = idx.shape
    n_arr = _per_loc(n, M, np.int32, 0)
    nmax = int(n_arr.max()) if nmax is None else int(nmax)
    if M == 0:
        nmax = max(nmax, n0)
    Npa = None if Np is None else _i32(np.broadcast_to(Np, (M,)))
    d_arr = _per_loc(d, M, np.float64, 0.0)
    sel = np.empty((M, nmax), dtype=np.int32)
    alc = np.empty((M, nmax), dtype=np.float64)
    status = np.empty(M, dtype=np.int32)
    ti = tv = None
    if topk > 0:
        ti = np.empty((M, nmax, topk), dtype=np.int32)
        tv = np.empty((M, nmax, topk), dtype=np.float64)
    _check(_load().orc_alc_select(_ptr(X), N, p, _ptr(Xref), M, _ptr(idx), _ptr(Npa), Npmax,
                                  int(n0), _ptr(n_arr), nmax, _ptr(d_arr), float(g), _ptr(sel),
                                  _ptr(alc), int(topk), _ptr(ti), _ptr(tv), _ptr(status)),
           "alc_select")
    out = dict(sel=sel, alc=alc, status=status)
    if topk > 0:
        out.update(top_idx=ti, top_val=tv)
    return out


def alc_scores(X, x, design, cands, d, g):
    """(three-term Eq. dxy, simplified) ALC of each candidate row."""
    X, x = _f64(X), _f64(x)
    design, cands = _i32(design), _i32(cands)
    N, p = X.shape
    d3 = np.empty(len(cands))
    ds = np.empty(len(cands))
    rc = _load().orc_alc_scores(_ptr(X), N, p, _ptr(x), _ptr(design), len(design), _ptr(cands),
                                len(cands), float(d), float(g), _ptr(d3), _ptr(ds))
    if rc != ORC_OK:
        raise ValueError(f"oracle alc_scores failed ({rc})")
    return d3, ds


def partitioned_inverse(X, design, n0, d, g):
    X, design = _f64(X), _i32(design)
    N, p = X.shape
    n = len(design)
    out = np.empty((n, n))
    rc = _load().orc_partitioned_inverse(_ptr(X), N, p, _ptr(design), int(n0), n, float(d),
                                         float(g), _ptr(out))
    if rc != ORC_OK:
        raise ValueError(f"oracle partitioned_inverse failed ({rc})")
    return out


def predict(X, Y, Xref, sel, n, d, g):
    """Local predictive mean, scale s2 and degrees of freedom (Eqs. predgp/preds2)."""
    X, Y, Xref, sel = _f64(X), _f64(Y), _f64(Xref), _i32(sel)
    N, p = X.shape
    M, nmax = sel.shape
    n_arr = _per_loc(n, M, np.int32, nmax)
    d_arr = _per_loc(d, M, np.float64, 0.0)
    mean, s2, df = np.empty(M), np.empty(M), np.empty(M)
    status = np.empty(M, dtype=np.int32)
    _check(_load().orc_predict(_ptr(X), _ptr(Y), N, p, _ptr(Xref), M, _ptr(sel), _ptr(n_arr), nmax,
                               _ptr(d_arr), float(g), _ptr(mean), _ptr(s2), _ptr(df),
                               _ptr(status)), "predict")
    return dict(mean=mean, s2=s2, df=df, status=status)


def llik(X, Y, sel, n, d, g):
    """Log-likelihood of Eq. (gpk) and its first two d-derivatives."""
    X, Y, sel = _f64(X), _f64(Y), _i32(sel)
    N, p = X.shape
    M, nmax = sel.shape
    n_arr = _per_loc(n, M, np.int32, nmax)
    d_arr = _per_loc(d, M, np.float64, 0.0)
    l, dl, d2l = np.empty(M), np.empty(M), np.empty(M)
    status = np.empty(M, dtype=np.int32)
    _check(_load().orc_llik(_ptr(X), _ptr(Y), N, p, M, _ptr(sel), _ptr(n_arr), nmax, _ptr(d_arr),
                            float(g), _ptr(l), _ptr(dl), _ptr(d2l), _ptr(status)), "llik")
    return dict(llik=l, dllik=dl, d2llik=d2l, status=status)


def mle(X, Y, sel, n, d0, g, dmin, dmax, max_iter):
    """Per-location Newton MLE of d (Fig. 1 step 3)."""
    X, Y, sel = _f64(X), _f64(Y), _i32(sel)
    N, p = X.shape
    M, nmax = sel.shape
    n_arr = _per_loc(n, M, np.int32, nmax)
    d = _per_loc(d0, M, np.float64, 0.0)
    l, dl, d2l = np.empty(M), np.empty(M), np.empty(M)
    it = np.empty(M, dtype=np.int32)
    status = np.empty(M, dtype=np.int32)
    _check(_load().orc_mle(_ptr(X), _ptr(Y), N, p, M, _ptr(sel), _ptr(n_arr), nmax, _ptr(d),
                           float(g), float(dmin), float(dmax), int(max_iter), _ptr(l), _ptr(dl),
                           _ptr(d2l), _ptr(it), _ptr(status)), "mle")
    return dict(d=d, llik=l, dllik=dl, d2llik=d2l, iters=it, status=status)


def predict_grad(X, Y, Xref, sel, n, d, g):
    """Analytic d/dd and d/dg of the predictive mean and s2, and dllik/dg."""
    X, Y, Xref, sel = _f64(X), _f64(Y), _f64(Xref), _i32(sel)
    N, p = X.shape
    M, nmax = sel.shape
    n_arr = _per_loc(n, M, np.int32, nmax)
    d_arr = _per_loc(d, M, np.float64, 0.0)
    outs = [np.empty(M) for _ in range(5)]
    status = np.empty(M, dtype=np.int32)
    _check(_load().orc_predict_grad(_ptr(X), _ptr(Y), N, p, _ptr(Xref), M, _ptr(sel), _ptr(n_arr),
                                    nmax, _ptr(d_arr), float(g), *[_ptr(o) for o in outs],
                                    _ptr(status)), "predict_grad")
    keys = ["dmean_dd", "dmean_dg", "ds2_dd", "ds2_dg", "dllik_dg"]
    r = dict(zip(keys, outs))
    r["status"] = status
    return r


def run_pipeline(X, Y, Xref, n0, n, Np, d, g, mle_args=None, Np_arr=None, rounds=1):
    """kNN -> ALC search -> (MLE) -> predict for every location (FP64),
    Fig. 1.  With mle_args, steps 2-3 (search at the current d, then the MLE
    of d on that design from the current d) run `rounds` times (step 4);
    rounds=2 is the two-stage scheme."""
    M = len(Xref)
    n_arr = _per_loc(n, M, np.int32, 0)
    Np_max = int(np.max(Np_arr)) if Np_arr is not None else int(Np)
    idx = knn(X, Xref, Np_max, Np_arr)
    dd = _per_loc(d, M, np.float64, 0.0)
    out = dict(idx=idx, rounds=[])
    for _ in range(rounds if mle_args is not None else 1):
        s = alc_select(X, Xref, idx, n0, n_arr, dd, g, Np=Np_arr)
        out.update(sel=s["sel"], alc=s["alc"], sel_status=s["status"])
        if mle_args is not None:
            r = mle(X, Y, s["sel"], n_arr, dd, g, *mle_args)
            out["rounds"].append(dict(sel=s["sel"], d_in=dd, d=r["d"]))
            dd = r["d"]
            out["mle"] = r
    out.update(predict(X, Y, Xref, s["sel"], n_arr, dd, g))
    out["d"] = dd
    return out
