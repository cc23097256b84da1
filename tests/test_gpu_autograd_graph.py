"""GPU: the adjoint behind torch.autograd (against five-point finite
differences of the forward kernels), and the search captured in a CUDA graph
(replays identical to eager calls)."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5182_gb300 as lib
    return lib


def _setup(L, seed=51):
    w = W.toy2d(seed=seed, N=4000, M=24, Np=200, n=25)
    dev = torch.device("cuda", 0)
    X, Y, Xr = (torch.from_numpy(a).to(dev) for a in (w.X, w.Y, w.Xref))
    idx, _ = L.lagp_knn(X, Xr, 200)
    sel = L.lagp_alc_select(X, Xr, idx, 6, 25, w.d, w.g, prec="f64")["sel"]
    return w, X, Y, Xr, sel


def _fd5(f, x, h):
    return (8 * (f(x + h) - f(x - h)) - (f(x + 2 * h) - f(x - 2 * h))) / (12 * h)


def test_local_gp_gradients_match_finite_differences(L):
    w, X, Y, Xr, sel = _setup(L)
    d = torch.full((24,), 0.4, dtype=torch.float64, device=X.device, requires_grad=True)
    g = torch.tensor(2e-4, dtype=torch.float64, device=X.device, requires_grad=True)
    wm = torch.linspace(0.5, 1.5, 24, dtype=torch.float64, device=X.device)
    mean, s2 = L.local_gp(d, g, X, Y, Xr, sel, 25)
    (wm * mean + 3.0 * s2).sum().backward()

    def objective(dd, gg):
        m, s = L.local_gp(dd, gg, X, Y, Xr, sel, 25)
        return (wm * m + 3.0 * s).sum().item()

    with torch.no_grad():
        for i in (0, 7, 23):
            def fi(t):
                dd = d.detach().clone()
                dd[i] = t
                return objective(dd, g.item())
            fd = _fd5(fi, 0.4, 1e-3 * 0.4)
            assert abs(d.grad[i].item() - fd) <= 1e-6 * max(1.0, abs(fd))
        fdg = _fd5(lambda t: objective(d.detach(), t), 2e-4, 1e-2 * 2e-4)
        assert abs(g.grad.item() - fdg) <= 1e-5 * max(1.0, abs(fdg))


def test_local_loglik_gradients(L):
    from oracle import oracle as O
    w, X, Y, Xr, sel = _setup(L, seed=52)
    d = torch.linspace(0.2, 1.2, 24, dtype=torch.float64, device=X.device).requires_grad_(True)
    ll = L.local_loglik(d, w.g, X, Y, Xr, sel, 25)
    ll.sum().backward()
    ref = O.llik(w.X, w.Y, sel.cpu().numpy(), 25, d.detach().cpu().numpy(), w.g)
    np.testing.assert_allclose(ll.detach().cpu().numpy(), ref["llik"], rtol=1e-9)
    np.testing.assert_allclose(d.grad.cpu().numpy(), ref["dllik"], rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("prec", ["f32bulk", "f32bulk_f64", "f64", "f64schur"])
def test_search_captured_in_cuda_graph(L, prec):
    """kNN and the fused search+prediction, captured once and replayed: the
    persistent kernels and their work counters (reset by captured memsets)
    give the same designs and predictions as eager calls."""
    w = W.borehole(seed=53, N=20_000, M=300, Np=400, n=30)
    dev = torch.device("cuda", 0)
    X, Y, Xr = (torch.from_numpy(a).to(dev) for a in (w.X, w.Y, w.Xref))
    # per-location arguments as device tensors made before capture (a Python
    # scalar would need a host-to-device copy inside the capture)
    n_t = torch.full((w.M,), 30, dtype=torch.int32, device=dev)
    d_t = torch.full((w.M,), w.d, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        idx, _ = L.lagp_knn(X, Xr, 400)  # warm: workspaces are sized outside capture
        eager = L.lagp_alc_predict(X, Y, Xr, idx, 6, n_t, d_t, w.g, prec=prec, n_max=30)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        idx_g, _ = L.lagp_knn(X, Xr, 400)
        out_g = L.lagp_alc_predict(X, Y, Xr, idx_g, 6, n_t, d_t, w.g, prec=prec, n_max=30)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(idx_g, idx)
        assert torch.equal(out_g["sel"], eager["sel"])
        assert torch.equal(out_g["mean"], eager["mean"])
        assert torch.equal(out_g["s2"], eager["s2"])


def test_uneven_mle_pipeline_captured_in_cuda_graph(L):
    """The whole MLE pipeline of the batched uneven configuration (kNN ->
    FP32-bulk search -> Newton MLE of d -> prediction, per-location n and N'
    drawn as in the 1M-point workload, on a smaller design), captured once
    and replayed twice: every output bitwise the eager calls'."""
    w = W.borehole(seed=57, N=60_000, M=400, n_range=(30, 100), Np_range=(500, 2000), dtype=np.float32,
                   mle=(1e-3, 20.0, 10))
    dev = torch.device("cuda", 0)
    X, Y, Xr = (torch.from_numpy(a).to(dev) for a in (w.X, w.Y, w.Xref))
    n_t, Np_t = torch.from_numpy(w.n).to(dev), torch.from_numpy(w.Np).to(dev)
    Npm, nmax = int(w.Np.max()), int(w.n.max())

    def pipeline():
        idx, _ = L.lagp_knn(X, Xr, Npm, Nprime=Np_t)
        s = L.lagp_alc_select(X, Xr, idx, w.n0, n_t, w.d, w.g, prec="f32bulk", Nprime=Np_t, n_max=nmax,
                             want_alc=True)
        m = L.lagp_mle_step(X, Y, s["sel"], n_t, w.d, w.g, *w.mle)
        pr = L.lagp_predict(X, Y, Xr, s["sel"], n_t, m["d"], w.g)
        return dict(idx=idx, sel=s["sel"], alc=s["alc"], d=m["d"], iters=m["iters"], mean=pr["mean"],
                    s2=pr["s2"], st=torch.stack([s["status"], m["status"], pr["status"]]))

    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        eager = pipeline()  # (workspaces sized outside the capture)
    torch.cuda.synchronize()
    assert (eager["st"] == 0).all()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        got = pipeline()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for k in eager:
            assert torch.equal(torch.nan_to_num(got[k], nan=-7.0), torch.nan_to_num(eager[k], nan=-7.0)), k


def test_autotune_picks_a_grid_and_results_do_not_depend_on_it(L):
    """The autotuner times every admissible resident-CTA count and re-score
    batch; the designs and predictions must not depend on either (one
    persistent CTA per location at a time; a contender's arithmetic follows
    the step's contender count, not its batch), and the tuned choice must be
    the one later calls use."""
    w = W.toy2d(seed=54, N=20_000, M=700, Np=600, n=25)  # many contenders a step
    dev = torch.device("cuda", 0)
    X, Y, Xr = (torch.from_numpy(a).to(dev) for a in (w.X, w.Y, w.Xref))
    idx, _ = L.lagp_knn(X, Xr, 600)
    before = L.lagp_alc_predict(X, Y, Xr, idx, 6, 25, w.d, w.g, want_alc=True)
    best = L.lagp_autotune(X, Xr, idx, 6, 25, w.d, w.g, prec="f32bulk", Y=Y)
    assert 1 <= best["ctas_per_sm"] <= 4 and best["rescore_max"] in (4, 8, 16)
    after = L.lagp_alc_predict(X, Y, Xr, idx, 6, 25, w.d, w.g, want_alc=True)
    for k in ("sel", "mean", "s2", "alc"):
        assert torch.equal(torch.nan_to_num(before[k]), torch.nan_to_num(after[k])), k
    try:
        for cps in (1, 3):
            for b in (1, 3, 8, 16):
                L.set_tuning(ctas_per_sm=cps, rescore_max=b)
                out = L.lagp_alc_predict(X, Y, Xr, idx, 6, 25, w.d, w.g, want_alc=True)
                for k in ("sel", "mean", "s2", "alc"):
                    assert torch.equal(torch.nan_to_num(before[k]), torch.nan_to_num(out[k])), (cps, b, k)
    finally:
        L.set_tuning(ctas_per_sm=0, rescore_max=0)