"""The kNN screen's collection pass on the tensor cores (tcgen05, FP16 split
products, FP32 accumulation).

  * the values it computes, s = |y_q|^2 + |y_x|^2 - 2 y_q . y_x on the centred
    FP32 coordinates, against the FP64 squared distance of the same centred
    coordinates: within the pass's error bound E_tc (the bound the exactness
    argument of the screen uses), at sizes spanning several 128-row design
    blocks with a ragged tail and one to several query blocks per CTA;
  * the neighbour sets through the tensor-core pass against the CUDA-core
    pass (both exact: bit-identical), the tensor-core pass sending hardly
    more locations to the exact retry than the CUDA-core one.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -24 * (1 + 2.0 ** -27)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5182_gb300 as lib
    return lib


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def centred(X, Xr):
    """fl32(x - c) with c the midrange of each coordinate over X and Xr, and
    the half-width B, as the screen computes them."""
    A = np.concatenate([X, Xr]).astype(np.float64)
    lo, hi = A.min(0), A.max(0)
    c = 0.5 * lo + 0.5 * hi
    B = np.max(np.maximum(hi - c, c - lo) + 2.0 ** -52 * np.maximum(np.abs(lo), np.abs(hi)))
    B *= 1 + 2.0 ** -50
    y = (A - c).astype(np.float32)
    return y[:len(X)], y[len(X):], B


def e_tc(p, B):
    """The pass's error bound (coordinates scaled by 2^-e <= 1/B, S = 2^e):
    the FP16 splits and the dropped low products, the FP32 norms and their
    splits, and 64 ulps of 2^-24 per tensor-core instruction (K / 16 of them)
    on the sum of the magnitudes 4 p S^2."""
    K = (3 * p + 4 + 15) // 16 * 16
    S = 2.0 ** math.frexp(B)[1]
    gp = p * U / (1 - p * U)
    return S * S * (4 * p * 2.0 ** -21 + 2 * (gp * p + 2.0 ** -22 * p + 2.0 ** -25)
                    + 64.0 * (K // 16) * 2.0 ** -24 * 4 * p * (1 + 2.0 ** -9))


@pytest.mark.parametrize("p,N,M,dtype", [(8, 3_001, 300, np.float64), (2, 1_000, 37, np.float64),
                                         (1, 513, 5, np.float64), (3, 2_050, 211, np.float32),
                                         (20, 700, 40, np.float64), (8, 300, 19_511, np.float64)])
def test_tc_values_within_bound(L, p, N, M, dtype):
    """(8, 300, 19511): more than 128 x SMs locations, so several query blocks
    of 128 per CTA."""
    rng = np.random.default_rng(100 + p)
    X = rng.uniform(-3, 5, (N, p)).astype(dtype)
    Xr = rng.uniform(-3, 5, (M, p)).astype(dtype)
    s = L.lagp_knn_tc_dist(dev(X), dev(Xr)).cpu().numpy().astype(np.float64)
    yx, yq, B = centred(X, Xr)
    ref = ((yq.astype(np.float64)[:, None, :] - yx.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    err = np.abs(s - ref)
    bound = e_tc(p, B)
    print(f"p={p}: max |s - ref| = {err.max():.3e} = {err.max() / (4 * p * B * B):.2e} x 4pB^2, "
          f"bound {bound / (4 * p * B * B):.2e} x 4pB^2")
    assert np.isfinite(s).all()
    assert err.max() <= bound


@pytest.mark.parametrize("case", ["borehole_100k", "toy2d_full", "ragged", "lattice_ties"])
def test_tc_and_cuda_core_paths_agree(L, case):
    rng = np.random.default_rng(31)
    Np_arr = None
    if case == "borehole_100k":   # the benchmark's design with a sample of its locations
        w = W.c2_borehole_100k(M=600)
        X, Xr, Npm = w.X, w.Xref, 1000
    elif case == "toy2d_full":
        w = W.c1_toy2d_fp64()
        X, Xr, Npm = w.X, w.Xref, 1000
    elif case == "ragged":
        X = rng.uniform(0, 1, (7_001, 8))
        Xr = rng.uniform(0, 1, (29, 8))
        Np_arr = rng.integers(1, 513, 29).astype(np.int32)
        Npm = 512
    else:
        g = np.arange(40, dtype=np.float64)
        X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
        X = np.concatenate([X, X[:50]])
        Xr = np.array([[10.0, 10.0], [0.0, 0.0], [20.5, 20.5], [39.0, 12.0]])
        Npm = 300
    L.set_tuning(knn_path=0)
    idx_tc, st_tc = L.lagp_knn(dev(X), dev(Xr), Npm, Nprime=Np_arr)
    stats = L.knn_stats()
    L.set_tuning(knn_path=1)
    try:
        idx_cc, st_cc = L.lagp_knn(dev(X), dev(Xr), Npm, Nprime=Np_arr)
        stats_cc = L.knn_stats()
    finally:
        L.set_tuning(knn_path=0)
    print(case, "retried: tensor cores", stats["retried"], "CUDA cores", stats_cc["retried"], "of", len(Xr))
    assert np.array_equal(st_tc.cpu().numpy(), st_cc.cpu().numpy())
    assert np.array_equal(idx_tc.cpu().numpy(), idx_cc.cpu().numpy())
    assert stats["tc_failed"] == 0
    # the sampled threshold sends the same few locations to the exact retry
    # (the wider tensor-core margin adds at most a few overflows)
    assert stats["retried"] <= stats_cc["retried"] + max(1, len(Xr) // 100), (stats, stats_cc)


def test_bounded_wait_reports_and_retries(L):
    """Failure detection without a GPU fault: the test hook stops the
    pass's producer after the first design block, the MMA thread's bounded
    wait on the next block runs out (2 s), the pass reports it, and the exact
    retry recomputes every location: the neighbour sets are unchanged."""
    rng = np.random.default_rng(41)
    X = rng.uniform(0, 1, (5_000, 8))
    Xr = rng.uniform(0, 1, (40, 8))
    ref, st_ref = L.lagp_knn(dev(X), dev(Xr), 200)
    assert L.knn_stats()["tc_failed"] == 0
    L.knn_tc_stall()
    idx, st = L.lagp_knn(dev(X), dev(Xr), 200)
    stats = L.knn_stats()
    assert stats["tc_failed"] == 1
    assert stats["retried"] == len(Xr)
    assert np.array_equal(st.cpu().numpy(), st_ref.cpu().numpy())
    assert np.array_equal(idx.cpu().numpy(), ref.cpu().numpy())
    # the hook is spent: the next call is normal again
    L.lagp_knn(dev(X), dev(Xr), 200)
    assert L.knn_stats()["tc_failed"] == 0


@pytest.mark.parametrize("M", [1, 3, 18, 21])
def test_retry_teams_match_oracle(L, M):
    """The exact retry of a block with at most four flagged queries runs each
    one's sweep on a team of warps (8, 4 or 2 of them, the rows of every tile
    split between them) instead of one warp.  The stall hook flags every
    query, so that M = 1 and 3 give one block of one and three flagged
    queries, M = 18 and 21 a full block (one warp per two queries) and one of
    two and five (teams of four; one warp each).  Ragged N' and a duplicated
    design row put ties at the thresholds.  The neighbour sets equal the
    oracle's bit for bit."""
    from oracle import oracle as orc
    orc.build()
    rng = np.random.default_rng(47)
    X = rng.uniform(0, 1, (6_000, 8))
    X[4_000:4_010] = X[17]  # equal distances at every query
    Xr = rng.uniform(0, 1, (M, 8))
    Np = rng.integers(150, 301, M).astype(np.int32)
    L.knn_tc_stall()
    idx, st = L.lagp_knn(dev(X), dev(Xr), 300, Nprime=Np)
    stats = L.knn_stats()
    assert stats["tc_failed"] == 1
    assert stats["retried"] == M
    assert (st.cpu().numpy() == 0).all()
    ref = orc.knn(X, Xr, 300, Np=Np)
    assert np.array_equal(idx.cpu().numpy(), ref)


def test_non_finite_rows_both_paths(L):
    """Design rows with NaN or infinite coordinates never enter a candidate
    set on either path; the two paths agree bit for bit (statuses too)."""
    rng = np.random.default_rng(43)
    X = rng.uniform(0, 1, (6_000, 8))
    X[[3, 500, 4_999], 2] = np.nan
    X[[10, 2_000], 5] = np.inf
    X[[77], 0] = -np.inf
    Xr = rng.uniform(0, 1, (33, 8))
    L.set_tuning(knn_path=0)
    idx_tc, st_tc = L.lagp_knn(dev(X), dev(Xr), 300)
    L.set_tuning(knn_path=1)
    try:
        idx_cc, st_cc = L.lagp_knn(dev(X), dev(Xr), 300)
    finally:
        L.set_tuning(knn_path=0)
    bad = {3, 500, 4_999, 10, 2_000, 77}
    assert not bad & set(idx_tc.cpu().numpy().ravel().tolist())
    assert np.array_equal(idx_tc.cpu().numpy(), idx_cc.cpu().numpy())
    assert np.array_equal(st_tc.cpu().numpy(), st_cc.cpu().numpy())
    assert (st_tc.cpu().numpy() == 0).all()
