"""Thin Python binding of liblagp.so (C ABI declared in include/lagp.h).

Argument marshalling only: every step of local approximate GP regression runs
in the library's CUDA kernels.  Device arrays are PyTorch CUDA tensors (memory
and streams come from PyTorch); work is enqueued on the current PyTorch
stream of the tensors' device.  There is no CPU fallback: if liblagp.so is
missing or cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblagp.so")

LAGP_OK, LAGP_EINVAL, LAGP_ENOTPD, LAGP_ECUDA, LAGP_ETIMEOUT, LAGP_ENOMEM = range(6)
LAGP_F64, LAGP_F32 = 0, 1
LAGP_PREC_F64, LAGP_PREC_F32BULK, LAGP_PREC_F64SCHUR, LAGP_PREC_F32BULK_F64 = 0, 1, 2, 3
_PREC = {"f64": LAGP_PREC_F64, "f32bulk": LAGP_PREC_F32BULK, "f64schur": LAGP_PREC_F64SCHUR,
         "f32bulk_f64": LAGP_PREC_F32BULK_F64}


class LagpError(RuntimeError):
    def __init__(self, fn, code, msg):
        self.code = code
        super().__init__(f"{fn} failed: {_STATUS.get(code, code)}: {msg}")


_STATUS = {0: "LAGP_OK", 1: "LAGP_EINVAL", 2: "LAGP_ENOTPD", 3: "LAGP_ECUDA", 4: "LAGP_ETIMEOUT",
           5: "LAGP_ENOMEM"}


class lagp_tuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("rescore_max", ctypes.c_int32), ("rescore_rel", ctypes.c_double),
                ("knn_path", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.lagp_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P]
    lib.lagp_destroy.argtypes = [P]
    lib.lagp_set_stream.argtypes = [P, P]
    lib.lagp_last_error.argtypes = [P]
    lib.lagp_last_error.restype = ctypes.c_char_p
    lib.lagp_status_string.argtypes = [ctypes.c_int]
    lib.lagp_status_string.restype = ctypes.c_char_p
    lib.lagp_get_tuning.argtypes = [P, ctypes.POINTER(lagp_tuning)]
    lib.lagp_set_tuning.argtypes = [P, ctypes.POINTER(lagp_tuning)]
    lib.lagp_launch_count.argtypes = [P]
    lib.lagp_launch_count.restype = I64
    lib.lagp_knn.argtypes = [P, P, I64, I32, ctypes.c_int, P, I64, P, I32, P, P]
    lib.lagp_alc_select.argtypes = [P, P, I64, I32, ctypes.c_int, P, I64, P, P, I32, I32, P, I32, P,
                                    D, ctypes.c_int, P, P, P]
    lib.lagp_predict.argtypes = [P, P, P, I64, I32, ctypes.c_int, P, I64, P, P, I32, P, D, P, P, P, P]
    lib.lagp_alc_predict.argtypes = [P, P, P, I64, I32, ctypes.c_int, P, I64, P, P, I32, I32, P, I32,
                                     P, D, ctypes.c_int, P, P, P, P, P, P]
    lib.lagp_predict_noalloc.argtypes = lib.lagp_predict.argtypes
    lib.lagp_mle_step.argtypes = [P, P, P, I64, I32, ctypes.c_int, I64, P, P, I32, P, D, D, D, I32,
                                  P, P, P, P, P]
    lib.lagp_predict_grad.argtypes = [P, P, P, I64, I32, ctypes.c_int, P, I64, P, P, I32, P, D, P, P,
                                      P, P, P, P, P]
    lib.lagp_autotune.argtypes = [P, P, I64, I32, ctypes.c_int, P, I64, P, P, I32, I32, P, I32, P, D,
                                  ctypes.c_int, P, P, P]
    lib.lagp_agp.argtypes = [P, P, P, I64, I32, ctypes.c_int, P, I64, P, I32, I32, P, I32, D, D,
                             ctypes.c_int, ctypes.c_int, D, D, I32, P, P, P, P, P]
    lib.lagp_alc_work.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
    lib.lagp_mle_work.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
    lib.lagp_alc_eval.argtypes = [P, P, I64, I32, ctypes.c_int, P, P, I32, P, I64, D, D, P, P]
    lib.lagp_scale_inputs.argtypes = [P, P, I64, I32, ctypes.c_int, P, P]
    lib.lagp_exp64_check.argtypes = [P, P, I64, P, P]
    lib.lagp_df_check.argtypes = [P, P, I64, P, P]
    lib.lagp_knn_tc_dist.argtypes = [P, P, I64, I32, ctypes.c_int, P, I64, P]
    lib.lagp_knn_stats.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I32)]
    lib.lagp_knn_tc_stall.argtypes = [P]
    for f in ("lagp_create", "lagp_destroy", "lagp_set_stream", "lagp_get_tuning", "lagp_set_tuning",
              "lagp_knn", "lagp_alc_select", "lagp_alc_predict", "lagp_predict", "lagp_predict_noalloc",
              "lagp_mle_step",
              "lagp_predict_grad", "lagp_autotune",
              "lagp_agp", "lagp_alc_work", "lagp_mle_work", "lagp_exp64_check", "lagp_df_check", "lagp_alc_eval",
              "lagp_scale_inputs", "lagp_knn_tc_dist", "lagp_knn_stats", "lagp_knn_tc_stall"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


_lib = _load()
_ctx_lock = threading.Lock()
_ctxs: dict[int, ctypes.c_void_p] = {}


def library():
    """The loaded ctypes library handle."""
    return _lib


def context(device: int | torch.device | None = None):
    """The library context for a CUDA device, bound to PyTorch's current
    stream on that device."""
    if device is None:
        device = torch.cuda.current_device()
    dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    with _ctx_lock:
        ctx = _ctxs.get(idx)
        if ctx is None:
            ctx = ctypes.c_void_p()
            stream = torch.cuda.current_stream(idx).cuda_stream
            rc = _lib.lagp_create(ctypes.byref(ctx), idx, ctypes.c_void_p(stream))
            if rc != LAGP_OK:
                raise LagpError("lagp_create", rc, "could not create a context")
            _ctxs[idx] = ctx
    _check(_lib.lagp_set_stream(ctx, ctypes.c_void_p(torch.cuda.current_stream(idx).cuda_stream)),
           ctx, "lagp_set_stream")
    return ctx


def _check(rc, ctx, fn):
    if rc != LAGP_OK:
        msg = _lib.lagp_last_error(ctx) if ctx else b""
        raise LagpError(fn, rc, (msg or b"").decode())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return LAGP_F64
    if t.dtype == torch.float32:
        return LAGP_F32
    raise TypeError(f"coordinates must be float64 or float32, not {t.dtype}")


def _dev(t: torch.Tensor, name, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _opt_i32(v, M, device, name, uniform=None):
    """None -> NULL pointer; array -> int32 CUDA tensor of length M.  A plain
    integer equal to `uniform` (the value the C API assumes for NULL) also
    becomes NULL, so that no device copy is made for it."""
    if v is None:
        return None, None
    if uniform is not None and isinstance(v, (int, np.integer)) and int(v) == int(uniform):
        return None, None
    t = torch.as_tensor(v, dtype=torch.int32, device=device)
    if t.dim() == 0:
        t = t.expand(M)
    t = t.contiguous()
    if t.numel() != M:
        raise ValueError(f"{name} must have M = {M} entries")
    return t, ctypes.c_void_p(t.data_ptr())


def _per_loc_f64(v, M, device):
    if isinstance(v, (int, float, np.floating, np.integer)):
        return torch.full((M,), float(v), dtype=torch.float64, device=device)
    t = torch.as_tensor(v, dtype=torch.float64, device=device)
    if t.dim() == 0:
        t = t.expand(M)
    return t.contiguous().clone() if t.numel() == M else _bad(f"expected M = {M} values")


def _bad(msg):
    raise ValueError(msg)


def _ptr_or_null(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def get_tuning(device=None) -> lagp_tuning:
    ctx = context(device)
    t = lagp_tuning()
    _check(_lib.lagp_get_tuning(ctx, ctypes.byref(t)), ctx, "lagp_get_tuning")
    return t


def set_tuning(device=None, **fields):
    ctx = context(device)
    t = get_tuning(device)
    for k, v in fields.items():
        setattr(t, k, v)
    _check(_lib.lagp_set_tuning(ctx, ctypes.byref(t)), ctx, "lagp_set_tuning")


def lagp_autotune(X, Xref, idx, n0, n, d, g, prec="f32bulk", Y=None, Nprime=None, n_max=None):
    """Time the ALC search on a sample of this problem for each admissible
    resident-CTA count (and, for the FP32-bulk form, re-score batch size) and
    record the fastest on the context.  Returns dict(ctas_per_sm,
    rescore_max)."""
    ctx = context(X.device)
    N, p = X.shape
    M, Npmax = idx.shape
    if n_max is None and isinstance(n, (int, np.integer)):
        n_max = int(n)
    nt, npp = _opt_i32(n, M, X.device, "n", uniform=n_max)
    if n_max is None:  # per-location n without n_max: one device sync
        n_max = int(nt.max().item()) if M else 1
    Npt, Npp = _opt_i32(Nprime, M, X.device, "Nprime", uniform=Npmax)
    dt = _per_loc_f64(d, M, X.device)
    best, best_b = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(_lib.lagp_autotune(ctx, _dev(X, "X"), N, p, _dtype_code(X), _dev(Xref, "Xref", X.dtype), M,
                              _dev(idx, "idx", torch.int32), Npp, Npmax, int(n0), npp, int(n_max),
                              _dev(dt, "d"), float(g), _PREC[prec],
                              None if Y is None else _dev(Y, "Y", X.dtype), ctypes.byref(best),
                              ctypes.byref(best_b)),
           ctx, "lagp_autotune")
    return {"ctas_per_sm": int(best.value), "rescore_max": int(best_b.value)}


def launch_count(device=None) -> int:
    return int(_lib.lagp_launch_count(context(device)))


def alc_work(device=None) -> dict:
    """FP32-bulk search work counters since the last read (then reset):
    locations, contenders re-scored in FP64 (n_c), sum n_c*j, sum n_c*j^2."""
    ctx = context(device)
    out = (ctypes.c_uint64 * 4)()
    _check(_lib.lagp_alc_work(ctx, out), ctx, "lagp_alc_work")
    return dict(locations=int(out[0]), rescored=int(out[1]), rescored_j=int(out[2]),
                rescored_j2=int(out[3]))


def mle_work(device=None) -> dict:
    """Newton MLE work counters since the last read (then reset): the sums of
    n^3 over likelihood evaluations and over derivative evaluations."""
    ctx = context(device)
    out = (ctypes.c_uint64 * 2)()
    _check(_lib.lagp_mle_work(ctx, out), ctx, "lagp_mle_work")
    return dict(llik_n3=int(out[0]), derivs_n3=int(out[1]))


def exp64_check(a: torch.Tensor):
    """The library's FP64 exp (Tang's table-driven method) and CUDA's exp at
    the values of the FP64 device tensor a.  Returns (tang, lib)."""
    pa = _dev(a, "a", torch.float64)
    ctx = context(a.device)
    t, l = torch.empty_like(a), torch.empty_like(a)
    _check(_lib.lagp_exp64_check(ctx, pa, a.numel(), ctypes.c_void_p(t.data_ptr()),
                                 ctypes.c_void_p(l.data_ptr())), ctx, "lagp_exp64_check")
    return t, l


def df_check(a: torch.Tensor):
    """The double-float split of the FP64 device tensor a and the
    double-float exp of it.  Returns (split, ex), each [n, 2] float32 (hi, lo)."""
    pa = _dev(a, "a", torch.float64)
    ctx = context(a.device)
    sp = torch.empty((a.numel(), 2), dtype=torch.float32, device=a.device)
    ex = torch.empty_like(sp)
    _check(_lib.lagp_df_check(ctx, pa, a.numel(), ctypes.c_void_p(sp.data_ptr()),
                              ctypes.c_void_p(ex.data_ptr())), ctx, "lagp_df_check")
    return sp, ex


def lagp_knn(X: torch.Tensor, Xref: torch.Tensor, Nprime_max: int, Nprime=None):
    """a1: exact N'-nearest neighbours.  Returns (idx [M, Nprime_max] int32,
    status [M] int32)."""
    ctx = context(X.device)
    N, p = X.shape
    M = Xref.shape[0]
    if Xref.dtype != X.dtype or Xref.shape[1] != p:
        raise ValueError("Xref must match X in dtype and p")
    Npt, Npp = _opt_i32(Nprime, M, X.device, "Nprime", uniform=Nprime_max)
    idx = torch.empty((M, Nprime_max), dtype=torch.int32, device=X.device)
    status = torch.empty(M, dtype=torch.int32, device=X.device)
    if M:
        _check(_lib.lagp_knn(ctx, _dev(X, "X"), N, p, _dtype_code(X), _dev(Xref, "Xref"), M, Npp,
                             int(Nprime_max), _dev(idx, "idx"), _dev(status, "status")),
               ctx, "lagp_knn")
    return idx, status


def lagp_knn_tc_dist(X: torch.Tensor, Xref: torch.Tensor) -> torch.Tensor:
    """Diagnostic: the squared distances of the kNN screen's tensor-core
    collection pass, |y_m|^2 + |y_r|^2 - 2 y_m . y_r on centred FP32
    coordinates (FP16 split products, FP32 accumulation).  Returns [M, N]
    float32."""
    ctx = context(X.device)
    N, p = X.shape
    M = Xref.shape[0]
    if Xref.dtype != X.dtype or Xref.shape[1] != p:
        raise ValueError("Xref must match X in dtype and p")
    out = torch.empty((M, N), dtype=torch.float32, device=X.device)
    _check(_lib.lagp_knn_tc_dist(ctx, _dev(X, "X"), N, p, _dtype_code(X), _dev(Xref, "Xref"), M,
                                 _dev(out, "out")), ctx, "lagp_knn_tc_dist")
    return out


def knn_tc_stall(device=None):
    """Test hook: the next tensor-core kNN pass on this device's context stops
    feeding its pipeline, so that its bounded waits run out (see lagp.h)."""
    ctx = context(device)
    _check(_lib.lagp_knn_tc_stall(ctx), ctx, "lagp_knn_tc_stall")


def knn_stats(device=None) -> dict:
    """Of the last lagp_knn call: locations recomputed by the exact retry of
    the screen, and whether the tensor-core pass gave up on a wait."""
    ctx = context(device)
    n, f = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(_lib.lagp_knn_stats(ctx, ctypes.byref(n), ctypes.byref(f)), ctx, "lagp_knn_stats")
    return {"retried": int(n.value), "tc_failed": int(f.value)}


def lagp_alc_select(X, Xref, idx, n0, n, d, g, prec="f32bulk", Nprime=None, n_max=None,
                    want_alc=False):
    """a2..a6: greedy ALC local designs.  n, d: scalars or per-location
    arrays.  Returns dict(sel [M, n_max], status [M], alc [M, n_max] or None)."""
    ctx = context(X.device)
    N, p = X.shape
    M, Npmax = idx.shape
    if n_max is None and isinstance(n, (int, np.integer)):
        n_max = int(n)
    nt, npp = _opt_i32(n, M, X.device, "n", uniform=n_max)
    if n_max is None:  # per-location n without n_max: one device sync
        n_max = int(nt.max().item()) if M else 1
    Npt, Npp = _opt_i32(Nprime, M, X.device, "Nprime", uniform=Npmax)
    dt = _per_loc_f64(d, M, X.device)
    sel = torch.empty((M, n_max), dtype=torch.int32, device=X.device)
    status = torch.empty(M, dtype=torch.int32, device=X.device)
    alc = torch.empty((M, n_max), dtype=torch.float64, device=X.device) if want_alc else None
    if M:
        _check(_lib.lagp_alc_select(ctx, _dev(X, "X"), N, p, _dtype_code(X), _dev(Xref, "Xref"), M,
                                    _dev(idx, "idx", torch.int32), Npp, Npmax, int(n0), npp,
                                    int(n_max), _dev(dt, "d"), float(g), _PREC[prec],
                                    _dev(sel, "sel"), _ptr_or_null(alc), _dev(status, "status")),
               ctx, "lagp_alc_select")
    return dict(sel=sel, status=status, alc=alc)


def lagp_alc_predict(X, Y, Xref, idx, n0, n, d, g, prec="f32bulk", Nprime=None, n_max=None,
                     want_alc=False):
    """a2..a7 fused: greedy ALC designs and the local predictive equations on
    them in one kernel.  Returns dict(sel, status, alc, mean, s2, df)."""
    ctx = context(X.device)
    N, p = X.shape
    M, Npmax = idx.shape
    if n_max is None and isinstance(n, (int, np.integer)):
        n_max = int(n)
    nt, npp = _opt_i32(n, M, X.device, "n", uniform=n_max)
    if n_max is None:  # per-location n without n_max: one device sync
        n_max = int(nt.max().item()) if M else 1
    Npt, Npp = _opt_i32(Nprime, M, X.device, "Nprime", uniform=Npmax)
    dt = _per_loc_f64(d, M, X.device)
    sel = torch.empty((M, n_max), dtype=torch.int32, device=X.device)
    status = torch.empty(M, dtype=torch.int32, device=X.device)
    alc = torch.empty((M, n_max), dtype=torch.float64, device=X.device) if want_alc else None
    out = {k: torch.empty(M, dtype=torch.float64, device=X.device) for k in ("mean", "s2", "df")}
    if M:
        _check(_lib.lagp_alc_predict(ctx, _dev(X, "X"), _dev(Y, "Y", X.dtype), N, p, _dtype_code(X),
                                     _dev(Xref, "Xref", X.dtype), M, _dev(idx, "idx", torch.int32), Npp,
                                     Npmax, int(n0), npp, int(n_max), _dev(dt, "d"), float(g),
                                     _PREC[prec], _dev(sel, "sel"), _ptr_or_null(alc),
                                     _dev(out["mean"], "mean"), _dev(out["s2"], "s2"),
                                     _dev(out["df"], "df"), _dev(status, "status")),
               ctx, "lagp_alc_predict")
    out.update(sel=sel, status=status, alc=alc)
    return out


def lagp_scale_inputs(X, theta):
    """Inputs scaled for separable lengthscales theta (p values): X_i /
    sqrt(theta_i), FP64.  Search and predict on the scaled inputs with d = 1
    evaluate exp(-sum_i (x_i - x'_i)^2 / theta_i)."""
    ctx = context(X.device)
    N, p = X.shape
    th = torch.as_tensor(theta, dtype=torch.float64, device=X.device).contiguous()
    if th.numel() != p:
        raise ValueError(f"theta must have p = {p} values")
    out = torch.empty((N, p), dtype=torch.float64, device=X.device)
    _check(_lib.lagp_scale_inputs(ctx, _dev(X, "X"), N, p, _dtype_code(X), _dev(th, "theta"),
                                  _dev(out, "Xs")), ctx, "lagp_scale_inputs")
    return out


def lagp_alc_eval(X, x, design, cands, d, g):
    """The ALC criterion (Eq. dxy, simplified) of every candidate row at one
    location x (p values) for the given design rows.  Returns (delta [Nc],
    status [1])."""
    ctx = context(X.device)
    N, p = X.shape
    xd = torch.as_tensor(x, dtype=torch.float64, device=X.device).contiguous()
    if xd.numel() != p:
        raise ValueError(f"x must have p = {p} values")
    design = torch.as_tensor(design, dtype=torch.int32, device=X.device).contiguous()
    cands = torch.as_tensor(cands, dtype=torch.int32, device=X.device).contiguous()
    delta = torch.empty(cands.numel(), dtype=torch.float64, device=X.device)
    status = torch.empty(1, dtype=torch.int32, device=X.device)
    _check(_lib.lagp_alc_eval(ctx, _dev(X, "X"), N, p, _dtype_code(X), _dev(xd, "x"),
                              _dev(design, "design"), design.numel(), _dev(cands, "cands"), cands.numel(),
                              float(d), float(g), _dev(delta, "delta"), _dev(status, "status")),
           ctx, "lagp_alc_eval")
    return delta, status


def lagp_predict(X, Y, Xref, sel, n, d, g):
    """a7: local predictive mean, scale and degrees of freedom."""
    ctx = context(X.device)
    N, p = X.shape
    M, n_max = sel.shape
    nt, npp = _opt_i32(n, M, X.device, "n", uniform=n_max)
    dt = _per_loc_f64(d, M, X.device)
    out = {k: torch.empty(M, dtype=torch.float64, device=X.device) for k in ("mean", "s2", "df")}
    status = torch.empty(M, dtype=torch.int32, device=X.device)
    if M:
        _check(_lib.lagp_predict(ctx, _dev(X, "X"), _dev(Y, "Y", X.dtype), N, p, _dtype_code(X),
                                 _dev(Xref, "Xref", X.dtype), M, _dev(sel, "sel", torch.int32), npp,
                                 n_max, _dev(dt, "d"), float(g), _dev(out["mean"], "mean"),
                                 _dev(out["s2"], "s2"), _dev(out["df"], "df"), _dev(status, "status")),
               ctx, "lagp_predict")
    out["status"] = status
    return out


def lagp_predict_noalloc(X, Y, Xref, sel, n, d, g, out=None):
    """a7 through the entry point that allocates no device memory (scratch in
    a fixed 2 MiB array inside the library; n_max <= 64).  For callers that
    cannot allocate, pass preallocated `out` = dict(mean, s2, df (float64 [M])
    and status (int32 [M])) and an int32 `n` / float64 `d` tensor of length M,
    so that this wrapper allocates nothing either."""
    ctx = context(X.device)
    N, p = X.shape
    M, n_max = sel.shape
    nt, npp = _opt_i32(n, M, X.device, "n", uniform=n_max)
    dt = d if (isinstance(d, torch.Tensor) and d.dtype == torch.float64 and d.is_cuda
               and d.numel() == M and d.is_contiguous()) else _per_loc_f64(d, M, X.device)
    if out is None:
        out = {k: torch.empty(M, dtype=torch.float64, device=X.device) for k in ("mean", "s2", "df")}
        out["status"] = torch.empty(M, dtype=torch.int32, device=X.device)
    _check(_lib.lagp_predict_noalloc(ctx, _dev(X, "X"), _dev(Y, "Y", X.dtype), N, p, _dtype_code(X),
                                     _dev(Xref, "Xref", X.dtype), M, _dev(sel, "sel", torch.int32),
                                     npp, n_max, _dev(dt, "d"), float(g), _dev(out["mean"], "mean"),
                                     _dev(out["s2"], "s2"), _dev(out["df"], "df"),
                                     _dev(out["status"], "status")),
           ctx, "lagp_predict_noalloc")
    return out


def lagp_mle_step(X, Y, sel, n, d0, g, dmin, dmax, max_iter):
    """a8: per-location Newton MLE of d.  Returns dict(d, llik, dllik,
    d2llik, iters, status)."""
    ctx = context(X.device)
    N, p = X.shape
    M, n_max = sel.shape
    nt, npp = _opt_i32(n, M, X.device, "n", uniform=n_max)
    d = _per_loc_f64(d0, M, X.device)
    out = {k: torch.empty(M, dtype=torch.float64, device=X.device) for k in ("llik", "dllik", "d2llik")}
    iters = torch.empty(M, dtype=torch.int32, device=X.device)
    status = torch.empty(M, dtype=torch.int32, device=X.device)
    if M:
        _check(_lib.lagp_mle_step(ctx, _dev(X, "X"), _dev(Y, "Y", X.dtype), N, p, _dtype_code(X), M,
                                  _dev(sel, "sel", torch.int32), npp, n_max, _dev(d, "d"), float(g),
                                  float(dmin), float(dmax), int(max_iter), _dev(out["llik"], "llik"),
                                  _dev(out["dllik"], "dllik"), _dev(out["d2llik"], "d2llik"),
                                  _dev(iters, "iters"), _dev(status, "status")),
               ctx, "lagp_mle_step")
    out.update(d=d, iters=iters, status=status)
    return out


def lagp_predict_grad(X, Y, Xref, sel, n, d, g):
    """Adjoint: d/dd, d/dg of mean, s2 and the log-likelihood, per location."""
    ctx = context(X.device)
    N, p = X.shape
    M, n_max = sel.shape
    nt, npp = _opt_i32(n, M, X.device, "n", uniform=n_max)
    dt = _per_loc_f64(d, M, X.device)
    keys = ("dmean_dd", "dmean_dg", "ds2_dd", "ds2_dg", "dllik_dd", "dllik_dg")
    out = {k: torch.empty(M, dtype=torch.float64, device=X.device) for k in keys}
    status = torch.empty(M, dtype=torch.int32, device=X.device)
    if M:
        _check(_lib.lagp_predict_grad(ctx, _dev(X, "X"), _dev(Y, "Y", X.dtype), N, p, _dtype_code(X),
                                      _dev(Xref, "Xref", X.dtype), M, _dev(sel, "sel", torch.int32),
                                      npp, n_max, _dev(dt, "d"), float(g),
                                      *[_dev(out[k], k) for k in keys], _dev(status, "status")),
               ctx, "lagp_predict_grad")
    out["status"] = status
    return out


def lagp_agp(X, Y, Xref, n0, n, Nprime, d0, g, prec="f32bulk", mle=None, rounds=1, device=0):
    """The whole method on HOST arrays (numpy or CPU tensors): kNN -> ALC ->
    MLE (when mle = (dmin, dmax, max_iter) is given; search and MLE repeated
    `rounds` times, rounds=2 being the two-stage scheme) -> predict.  Inputs
    are copied to the GPU and results back inside the call.  Returns numpy
    arrays."""
    ctx = context(device)
    X = np.ascontiguousarray(X)
    if X.dtype not in (np.float64, np.float32):
        raise TypeError("X must be float64 or float32")
    Y = np.ascontiguousarray(Y, dtype=X.dtype)
    Xref = np.ascontiguousarray(Xref, dtype=X.dtype)
    N, p = X.shape
    M = Xref.shape[0]
    # per-location sizes and the outputs in pinned host memory (torch's caching
    # host allocator): the library's copies to and from them run at full rate
    pinned = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    n_arr = pinned(M, torch.int32)
    n_arr[:] = np.broadcast_to(np.asarray(n, np.int32), (M,))
    Np_arr = pinned(M, torch.int32)
    Np_arr[:] = np.broadcast_to(np.asarray(Nprime, np.int32), (M,))
    out = {k: pinned(M, torch.float64) for k in ("mean", "s2", "df", "d")}
    status = pinned(M, torch.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    dmin, dmax, it = mle if mle is not None else (1e-3, 20.0, 0)
    _check(_lib.lagp_agp(ctx, ptr(X), ptr(Y), N, p, LAGP_F64 if X.dtype == np.float64 else LAGP_F32,
                         ptr(Xref), M, ptr(Np_arr), int(Np_arr.max()) if M else 1, int(n0), ptr(n_arr),
                         int(n_arr.max()) if M else int(n0), float(d0), float(g), _PREC[prec],
                         int(rounds) if mle is not None else 0, float(dmin), float(dmax), int(it),
                         ptr(out["mean"]), ptr(out["s2"]), ptr(out["df"]), ptr(out["d"]), ptr(status)),
           ctx, "lagp_agp")
    out["status"] = status
    return out
