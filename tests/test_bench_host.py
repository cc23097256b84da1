"""Host-side arithmetic of bench.py: the work and flop counts behind its
cand_evals_per_sec and roofline figures, pinned against values computed a
different way (the candidate-evaluation counts of the paper's search, Fig. 1
step 2, and itemised per-step sums)."""
import numpy as np

import bench


def test_candidate_evaluations_per_location():
    # E = sum_{j=n0}^{n-1} (N' - j): at step j the N' - j unchosen candidates
    # of the N' nearest neighbours are scored (the seeds are the first n0)
    for n0, n, Np in [(6, 50, 1000), (6, 50, 2000), (6, 60, 1500), (6, 100, 2000), (1, 2, 3)]:
        E = 0
        chosen = set(range(n0))
        for j in range(n0, n):
            E += Np - len(chosen)
            chosen.add(j)
        assert bench.work_per_location(n0, n, Np) == E
    assert bench.work_per_location(6, 50, 1000) == 42_790


def test_fp32_screen_flops_hand_count():
    # n = 3, N' = 5, p = 1: after step 0 four candidates take 0 + 3 + 8 flops,
    # after step 1 three take 2 + 3 + 8; the last step has no bulk pass
    assert bench.fp32_flops_per_location(3, 5, 1) == 4 * 11 + 3 * 13
    assert bench.fp32_flops_per_location(1, 5, 1) == 0


def test_fp64_flops_closed_form_matches_itemised_sum():
    # the closed form over the work counters (sums of n_c, n_c j, n_c j^2)
    # against the per-contender and per-step counts added one by one
    rng = np.random.default_rng(3)
    p, n, M = 8, 50, 7
    for fused in (False, True):
        e = 2 if fused else 1
        work = {"rescored": 0, "rescored_j": 0, "rescored_j2": 0}
        total = 0
        for _ in range(M):
            for j in range(n):
                ncon = int(rng.integers(1, 9))
                work["rescored"] += ncon
                work["rescored_j"] += ncon * j
                work["rescored_j2"] += ncon * j * j
                kernel_values = (j + 1) * (p + 2 * p + 1 + bench.EXP_FLOPS)
                contraction = 2 * j * (j + e)
                total += ncon * (kernel_values + contraction + 2 * j + 12)
                total += j + j * (j + 1) + 2 * j * e + 10
        assert bench.fp64_flops(work, M, n, p, fused) == total


def test_exp_flop_count():
    # the table-driven exp: seven fused multiply-adds (2 flops each), one
    # subtract and one multiply
    assert bench.EXP_FLOPS == 7 * 2 + 1 + 1
