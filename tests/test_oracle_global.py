"""Pins of the oracle's global search (Sec. 4.1, Alg. global_search) against what the algorithm
fixes, with every fitness value recomputed independently (periodic-image recount, Eq. sro and
Eq. fitness_function in exact rational arithmetic):

  * the pool of an iteration is the solutions kept from the previous one plus fresh random
    configurations, and the refined set is its best n_refine by (F^2, pool index);
  * the kept solutions are the best n_keep refined ones of the previous iteration (the worst
    fraction p_a = 1 - n_keep / n_refine is discarded);
  * a refinement (Alg. parallel_mc) never raises F^2, so the best F^2 never rises across iterations;
  * the result is ranked best first and its counts and F^2 are those of its configurations;
  * on the 16-site binary BCC cell the search reaches the exhaustive minimum (B2 target: F = 0,
    met by exactly two arrangements);
  * with one iteration the search reduces to independent parallel Monte Carlo runs from fresh
    configurations (the library routine the refinement step names).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import independent as ind


def exact_f2(kind, M, n_per, cnt, target, w):
    n = [int(x) for x in n_per]
    N = sum(n)
    f2 = Fraction(0)
    for k in range(M):
        Z = ind.SHELL_Z[kind][k]
        for i in range(len(n)):
            for j in range(len(n)):
                alpha = 1 - Fraction(int(cnt[k, i, j]) * N, Z * n[i] * n[j])
                e = alpha - Fraction(float(target[k, i, j]))
                f2 += Fraction(float(w[k])) * e * e
    return f2


def double_f2(kind, M, n_per, cnt, target, w):
    """F^2 in binary64 with the documented rounding order (the precision the ranking decides in)."""
    n = [int(x) for x in n_per]
    N = sum(n)
    s = 0.0
    for k in range(M):
        Z = ind.SHELL_Z[kind][k]
        for i in range(len(n)):
            for j in range(len(n)):
                Q = float(N) / ((float(Z) * float(n[i])) * float(n[j]))
                e = (1.0 - float(cnt[k, i, j]) * Q) - float(target[k, i, j])
                s = s + float(w[k]) * (e * e)
    return s


def close(x, exact):
    return abs(Fraction(float(x)) - exact) <= Fraction(1, 10 ** 12) * max(exact, Fraction(1, 10 ** 6))


CASES = [
    # kind, L, M, n_per, P, n_refine, n_keep, G, T, d, target scale
    (ind.FCC, (2, 2, 2), 2, [8, 8, 8, 8], 8, 0, -1, 3, 8, 4, 0.0),
    (ind.BCC, (3, 2, 2), 3, [9, 9, 6], 10, 6, 3, 3, 12, 3, 0.4),
    (ind.FCC, (2, 3, 2), 1, [20, 28], 9, 5, 1, 4, 4, 5, 0.3),
]


def run_case(case, seed=5):
    kind, L, M, n_per, P, PL, R, G, T, d, scale = case
    S = len(n_per)
    rng = np.random.default_rng(seed)
    target = scale * rng.uniform(-1, 1, (M, S, S))
    w = rng.uniform(0.5, 1.5, M)
    out = oracle.global_search(kind, L, M, n_per, w, target, n_solutions=P, n_refine=PL, n_keep=R,
                               iterations=G, tasks=T, depth_limit=d, seed=seed, check=True)
    return (kind, L, M, n_per, w, target), out


@pytest.mark.parametrize("case", range(len(CASES)))
def test_pool_selection_keep_and_discard(case):
    (kind, L, M, n_per, w, target), (types, cnt, f2, log, totals) = run_case(CASES[case])
    P = CASES[case][4]
    PL = log.shape[1]
    R = CASES[case][6] if CASES[case][6] >= 0 else PL // 2
    S = len(n_per)
    N = sum(n_per)
    prev_ranked = None
    for g in range(log.shape[0]):
        n_kept = 0 if g == 0 else R
        # Independent fitness of every pool entry: kept ones carry the previous ranked F^2,
        # fresh ones are recounted from their seeded initial configuration.
        pool_f2 = []
        for i in range(P):
            if i < n_kept:
                pool_f2.append(float(prev_ranked[i]))
            else:
                t = oracle.init_config(N, n_per, oracle.fresh_seed(5, g, i - n_kept))
                assert np.bincount(t, minlength=S).tolist() == list(n_per)
                c = ind.counts_by_images(kind, L, M, S, t)
                pool_f2.append(double_f2(kind, M, n_per, c, target, w))
                assert close(pool_f2[-1], exact_f2(kind, M, n_per, c, target, w))
        expect = sorted(range(P), key=lambda i: (pool_f2[i], i))[:PL]
        assert log["origin"][g].tolist() == expect, g
        for r in range(PL):
            assert log["f2_in"][g, r] == pool_f2[expect[r]], (g, r)
            assert log["f2_out"][g, r] <= log["f2_in"][g, r] * (1 + 1e-12)   # up to the key's rounding
        ranked_slots = sorted(range(PL), key=lambda r: (log["f2_out"][g, r], r))
        prev_ranked = [log["f2_out"][g, r] for r in ranked_slots]
    assert f2.tolist() == prev_ranked
    assert totals[0] == int(log["steps"].sum()) and totals[2] == int(log["accepted"].sum())
    assert totals[1] == totals[0] * CASES[case][8]
    for r in range(PL):
        assert np.bincount(types[r], minlength=S).tolist() == list(n_per)
        c = ind.counts_by_images(kind, L, M, S, types[r])
        assert np.array_equal(cnt[r], c)
        assert close(f2[r], exact_f2(kind, M, n_per, c, target, w))


def test_best_never_rises_across_iterations():
    (_, _, _, _, _, _), (_, _, f2, log, _) = run_case((ind.BCC, (3, 3, 2), 2, [12, 12, 12], 12, 0, -1, 5, 6, 2, 0.5))
    best = log["f2_out"].min(axis=1)
    assert all(best[g + 1] <= best[g] * (1 + 1e-12) for g in range(len(best) - 1))
    assert f2[0] == best[-1]


def test_reaches_exhaustive_minimum_on_binary_bcc():
    kind, L, M, S = ind.BCC, (2, 2, 2), 3, 2
    n_per = [8, 8]
    w = np.ones(M)
    b2 = np.array([[[1.0, -1.0], [-1.0, 1.0]], [[-1.0, 1.0], [1.0, -1.0]], [[-1.0, 1.0], [1.0, -1.0]]])
    zero = set()
    for ones in itertools.combinations(range(16), 8):
        t = np.zeros(16, np.uint8)
        t[list(ones)] = 1
        if exact_f2(kind, M, n_per, ind.counts_by_images(kind, L, M, S, t), b2, w) == 0:
            zero.add(ones)
    assert len(zero) == 2
    types, _, f2, _, _ = oracle.global_search(kind, L, M, n_per, w, b2, n_solutions=8, iterations=4, tasks=16,
                                              depth_limit=10, seed=3)
    assert f2[0] == 0.0
    assert tuple(np.flatnonzero(types[0] == 1)) in zero


def test_one_iteration_is_independent_parallel_mc_runs():
    kind, L, M, n_per = ind.FCC, (2, 2, 3), 2, [12, 12, 12, 12]
    S = len(n_per)
    N = sum(n_per)
    rng = np.random.default_rng(8)
    target = 0.3 * rng.uniform(-1, 1, (M, S, S))
    w = np.ones(M)
    types, cnt, f2, log, _ = oracle.global_search(kind, L, M, n_per, w, target, n_solutions=6, iterations=1,
                                                  tasks=16, depth_limit=6, seed=11)
    refined = {}
    for r in range(6):
        t0 = oracle.init_config(N, n_per, oracle.fresh_seed(11, 0, int(log["origin"][0, r])))
        c0 = oracle.counts(kind, L, M, S, t0)
        t1, c1, res, _ = oracle.search(kind, L, M, n_per, w, target, t0, c0, K=16, max_steps=1 << 30,
                                       depth_limit=6, seed=11, chain=r)
        refined[r] = (t1, c1, res["f2"])
        assert res["f2"] == log["f2_out"][0, r] and res["steps"] == log["steps"][0, r]
    ranked = sorted(range(6), key=lambda r: (refined[r][2], r))
    for pos, r in enumerate(ranked):
        assert np.array_equal(types[pos], refined[r][0]) and np.array_equal(cnt[pos], refined[r][1])


def test_fresh_seed_is_philox_counter_four():
    r = oracle.philox4x32_10((7, 3, 0, 4), (0x9ABCDEF0, 0x12345678))
    assert oracle.fresh_seed(0x123456789ABCDEF0, 3, 7) == (int(r[1]) << 32) | int(r[0])
