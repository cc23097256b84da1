"""lagp_predict_noalloc: the prediction entry point that allocates no device
memory, for callers that cannot call cudaMalloc (an allocator of their own
owns the device memory, a memory budget is fixed at start-up, or the path
cannot take cudaMalloc's implicit synchronisation).  Its scratch is a fixed
array inside the library shared by every call, so this file checks it on two
calls in a row, each against the ordinary lagp_predict on the same inputs,
with the tolerance the parity tests use (relative 1e-6, or 16 eps cond(K_n)
times the quantity's scale).  It also checks the per-location failure
statuses against lagp_predict's (the paths where a stale matrix from the
previous call could leak into the output) and the values directly against
the FP64 oracle.  The file is collected last on purpose."""
import os

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _tolerances(X, Y, sel, n_arr, d, g):
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    d = np.broadcast_to(np.asarray(d, np.float64), (sel.shape[0],))
    am, a2 = [], []
    for m in range(sel.shape[0]):
        rows = sel[m, :int(n_arr[m])]
        A = X[rows]
        K = np.exp(-((A[:, None] - A[None]) ** 2).sum(-1) / d[m]) + g * np.eye(len(rows))
        c = np.linalg.cond(K)
        psi = Y[rows] @ np.linalg.solve(K, Y[rows])
        am.append(16 * EPS * c * np.abs(Y[rows]).max())
        a2.append(16 * EPS * c * psi / len(rows))
    return np.array(am), np.array(a2)


def _case(L, w, n_arr, d):
    dev = torch.device("cuda", 0)
    X = torch.from_numpy(w.X).to(dev)
    Y = torch.from_numpy(w.Y).to(dev)
    Xr = torch.from_numpy(w.Xref).to(dev)
    Np = int(w.Np[0])
    idx, _ = L.lagp_knn(X, Xr, Np)
    sel = L.lagp_alc_select(X, Xr, idx, w.n0, n_arr, d, w.g, prec="f32bulk")["sel"]
    return X, Y, Xr, sel


def _compare(a, b, w, sel, n_arr, d):
    for k in ("mean", "s2", "df", "status"):
        a[k] = a[k].cpu().numpy()
        b[k] = b[k].cpu().numpy()
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal(a["df"], b["df"])
    am, a2 = _tolerances(w.X, w.Y, sel, n_arr, d, w.g)
    assert np.all(np.abs(a["mean"] - b["mean"]) <= np.maximum(1e-6 * np.abs(b["mean"]), am))
    assert np.all(np.abs(a["s2"] - b["s2"]) <= np.maximum(1e-6 * np.abs(b["s2"]), a2))


def test_predict_noalloc_matches_predict_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5182_gb300 as L

    # first call: the 2-d toy, n = 50 everywhere, FP64 inputs
    w1 = W.toy2d(seed=31, N=5_000, M=150, Np=400, n=50)
    X, Y, Xr, sel = _case(L, w1, 50, w1.d)
    got = L.lagp_predict_noalloc(X, Y, Xr, sel, 50, w1.d, w1.g)
    ref = L.lagp_predict(X, Y, Xr, sel, 50, w1.d, w1.g)
    torch.cuda.synchronize()
    _compare(got, ref, w1, sel.cpu().numpy(), np.full(150, 50), w1.d)
    assert (ref["status"] == 0).all()

    # second call in a row: different sizes, ragged n, FP32 inputs, more
    # locations than the entry point's 64 persistent CTAs
    w2 = W.borehole(seed=32, N=20_000, M=333, Np=300, dtype=np.float32, g=1e-5)
    n_arr = np.random.default_rng(33).integers(7, 65, 333).astype(np.int32)
    X, Y, Xr, sel = _case(L, w2, n_arr, w2.d)
    got = L.lagp_predict_noalloc(X, Y, Xr, sel, n_arr, w2.d, w2.g)
    ref = L.lagp_predict(X, Y, Xr, sel, n_arr, w2.d, w2.g)
    torch.cuda.synchronize()
    _compare(got, ref, w2, sel.cpu().numpy(), n_arr, w2.d)
    assert (ref["status"] == 0).all()


def test_predict_noalloc_failure_statuses_and_oracle():
    """Failed locations between valid ones, right after a call that filled
    the scratch: a design row out of range, n = 0, d <= 0 (LAGP_EINVAL) and
    a repeated design row with no nugget (LAGP_ENOTPD) must get the same
    status and NaN outputs as lagp_predict; the valid locations must match
    the FP64 oracle's predictions within the parity bar."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5182_gb300 as L
    from oracle import oracle as O
    O.build()
    O.set_threads(os.cpu_count() or 1)

    w = W.borehole(seed=35, N=20_000, M=8, Np=200, n=8)
    X, Y, Xr, sel = _case(L, w, 8, w.d)
    sel_np = sel.cpu().numpy().copy()
    n_arr = np.full(8, 8, np.int32)
    d = np.full(8, w.d)
    g = 0.0
    sel_np[0, 3] = w.N + 5          # row out of range
    n_arr[1] = 0                    # empty design
    d[2] = -1.0                     # non-positive lengthscale
    sel_np[3, 1] = sel_np[3, 0]     # repeated row, no nugget: K_n singular
    sel_bad = torch.from_numpy(sel_np).cuda()
    got = L.lagp_predict_noalloc(X, Y, Xr, sel_bad, n_arr, d, g)
    ref = L.lagp_predict(X, Y, Xr, sel_bad, n_arr, d, g)
    torch.cuda.synchronize()
    st_g, st_r = got["status"].cpu().numpy(), ref["status"].cpu().numpy()
    assert np.array_equal(st_g, st_r), (st_g, st_r)
    assert list(st_g[:4]) == [1, 1, 1, 2] and (st_g[4:] == 0).all()
    for k in ("mean", "s2", "df"):
        a_, b_ = got[k].cpu().numpy(), ref[k].cpu().numpy()
        assert np.isnan(a_[:4]).all() and np.isnan(b_[:4]).all()
    ok = np.arange(4, 8)
    orc = O.predict(w.X, w.Y, w.Xref[ok], sel_np[ok], n_arr[ok], d[ok], g)
    am, a2 = _tolerances(w.X, w.Y, sel_np[ok], n_arr[ok], d[ok], g)
    mg, sg = got["mean"].cpu().numpy()[ok], got["s2"].cpu().numpy()[ok]
    assert np.all(np.abs(mg - orc["mean"]) <= np.maximum(1e-6 * np.abs(orc["mean"]), am))
    assert np.all(np.abs(sg - orc["s2"]) <= np.maximum(1e-6 * np.abs(orc["s2"]), a2))


def test_predict_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5182_gb300 as L

    w = W.toy2d(seed=34, N=2_000, M=4, Np=100, n=65)
    X, Y, Xr, sel = _case(L, w, 65, w.d)
    with pytest.raises(L.LagpError, match="n_max must be in"):
        L.lagp_predict_noalloc(X, Y, Xr, sel, 65, w.d, w.g)
    # an infinite nugget is rejected like lagp_predict rejects it
    with pytest.raises(L.LagpError, match="g must be finite"):
        L.lagp_predict_noalloc(X, Y, Xr, sel[:, :64].contiguous(), 64, w.d, float("inf"))
