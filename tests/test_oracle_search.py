"""Pins for the oracle's Monte Carlo search (Alg. parallel_mc, Sec. 4.2; Sec. 4.6.3-4.6.4):
incremental counts equal a full recount after every step, each accepted step lowers F^2, the
best-of-K choice equals an independent brute force over the K candidates, multi-accepted swaps do
not interact, resume is exact, and the result is never below the exhaustive optimum."""
import itertools
import os

import numpy as np
import pytest

import oracle
from tests import independent as ind

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def philox_kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("row", philox_kat_rows())
def test_philox_known_answers(row):
    ctr, key, want = row
    assert list(oracle.philox4x32_10(ctr, key)) == want


def setup(kind, L, M, S, seed, target_scale=0.3):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    n_per = rng.multinomial(N - 2 * S, np.ones(S) / S) + 2
    types = oracle.init_config(N, n_per, seed)
    cnt = oracle.counts(kind, L, M, S, types)
    w = rng.uniform(0.5, 1.5, M)
    target = rng.uniform(-target_scale, target_scale, (M, S, S))
    target = 0.5 * (target + target.transpose(0, 2, 1))
    return N, n_per, types, cnt, w, target


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kind,L,M,S,K", [(ind.FCC, (3, 3, 3), 3, 4, 16), (ind.BCC, (4, 4, 3), 2, 5, 32),
                                          (ind.FCC, (2, 2, 2), 5, 3, 8)])
def test_trajectory_counts_stay_exact(mode, kind, L, M, S, K):
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 3)
    ty, c, res, _ = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=K, max_steps=60,
                                  accept_mode=mode, seed=5, check=True)
    assert res["status"] == 0
    assert np.array_equal(c, oracle.counts(kind, L, M, S, ty))
    assert np.array_equal(np.bincount(ty, minlength=S), n_per)     # composition is conserved
    assert res["trials"] == res["steps"] * K
    _, f2 = oracle.alpha_f2(kind, L, M, n_per, w, target, c)
    assert res["f2"] == f2


def brute_force_step(kind, L, M, S, n_per, w, target, types, pairs):
    """F^2 after each candidate swap, by full independent recount (Eq. sro + Eq. fitness_function)."""
    out = []
    for a, b in pairs:
        t2 = types.copy()
        t2[a], t2[b] = t2[b], t2[a]
        cnt = ind.counts_by_images(kind, L, M, S, t2)
        out.append(ind.f2_eq_fitness(ind.alpha_eq_sro(kind, L, M, n_per, cnt), target, w))
    return np.array(out)


def test_best_of_k_choice_matches_brute_force():
    kind, L, M, S, K = ind.FCC, (2, 2, 3), 3, 3, 12
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 8, target_scale=0.6)
    checked = 0
    for step in range(6):
        pairs = oracle.draw_pairs(N, 21, 0, step, 1, K)
        f2_now = ind.f2_eq_fitness(ind.alpha_eq_sro(kind, L, M, n_per, ind.counts_by_images(kind, L, M, S, types)),
                                   target, w)
        f2_new = brute_force_step(kind, L, M, S, n_per, w, target, types, pairs)
        moved = np.array([a != b and types[a] != types[b] for a, b in pairs])
        dF = np.where(moved, f2_new - f2_now, 0.0)
        best = int(np.argmin(dF))
        order = np.sort(np.unique(np.round(dF, 9)))
        ty, c, res, acc = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=K, max_steps=1,
                                        seed=21, step0=step, log=True)
        clear_gap = len(order) < 2 or order[1] - order[0] > 1e-9
        if dF[best] < -1e-9 and clear_gap:
            assert res["accepted"] == 1
            assert tuple(acc[0]) == tuple(pairs[best])
            checked += 1
        if dF.min() > 1e-9:
            assert res["accepted"] == 0
            checked += 1
        types, cnt = ty, c
    assert checked >= 4


def test_accepted_steps_lower_the_objective():
    kind, L, M, S = ind.BCC, (5, 5, 5), 2, 4
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 4)
    prev = None
    ty, c = types, cnt
    for chunk in range(20):
        ty2, c2, res, _ = oracle.search(kind, L, M, n_per, w, target, ty, c, K=16, max_steps=1, seed=9,
                                        step0=chunk, accept_mode=chunk % 2)
        if prev is not None:
            if res["accepted"] > 0:
                assert res["f2"] < prev
            else:
                assert res["f2"] == prev
        prev = res["f2"]
        ty, c = ty2, c2


def test_multi_accept_swaps_do_not_interact():
    kind, L, M, S = ind.FCC, (6, 6, 6), 3, 4
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 6, target_scale=0.8)
    nbr = oracle.neighbours(kind, L, M)
    ty, c, res, acc = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=256, max_steps=1,
                                    accept_mode=1, seed=3, log=True)
    assert res["accepted"] > 1
    sites = acc.reshape(-1)
    assert len(set(sites.tolist())) == len(sites)
    for i in range(len(acc)):
        for j in range(i + 1, len(acc)):
            for u in acc[i]:
                for v in acc[j]:
                    assert v not in nbr[u]
    # The combined move equals the sum of the separate deltas (they do not interact).
    assert np.array_equal(c, oracle.counts(kind, L, M, S, ty))


def test_max_accept_caps_swaps_per_step():
    kind, L, M, S = ind.FCC, (6, 6, 6), 3, 4
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 6, target_scale=0.8)
    _, _, res, _ = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=256, max_steps=3,
                                 accept_mode=1, max_accept=2, seed=3)
    assert 0 < res["accepted"] <= 6


@pytest.mark.parametrize("mode", [0, 1])
def test_resume_is_exact(mode):
    kind, L, M, S = ind.BCC, (4, 4, 4), 3, 3
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 12)
    ty_a, c_a, r_a, _ = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=8, max_steps=40, seed=2,
                                      accept_mode=mode)
    ty_1, c_1, r_1, _ = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=8, max_steps=17, seed=2,
                                      accept_mode=mode)
    ty_b, c_b, r_b, _ = oracle.search(kind, L, M, n_per, w, target, ty_1, c_1, K=8, max_steps=23, seed=2,
                                      step0=17, depth0=r_1["depth"], accept_mode=mode)
    assert np.array_equal(ty_a, ty_b) and np.array_equal(c_a, c_b)
    assert r_a["f2"] == r_b["f2"] and r_a["depth"] == r_b["depth"]
    assert r_a["accepted"] == r_1["accepted"] + r_b["accepted"]


def test_depth_limit_stops_after_consecutive_failures():
    kind, L, M, S = ind.FCC, (3, 3, 3), 3, 3
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 2)
    _, _, res, _ = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=4, max_steps=100000,
                                 depth_limit=5, seed=1)
    assert res["depth"] == 5
    assert res["steps"] < 100000


def test_search_never_beats_exhaustive_minimum_and_finds_b2():
    """BCC 2x2x2, 8 A + 8 B: the B2 target is met (F = 0) only by the two B2 arrangements."""
    kind, L, M, S = ind.BCC, (2, 2, 2), 3, 2
    n_per = [8, 8]
    w = np.ones(M)
    b2 = np.array([[[1.0, -1.0], [-1.0, 1.0]], [[-1.0, 1.0], [1.0, -1.0]], [[-1.0, 1.0], [1.0, -1.0]]])
    f2_all = []
    zero = []
    for ones in itertools.combinations(range(16), 8):
        t = np.zeros(16, np.uint8)
        t[list(ones)] = 1
        _, f2 = oracle.alpha_f2(kind, L, M, n_per, w, b2, oracle.counts(kind, L, M, S, t))
        f2_all.append(f2)
        if f2 == 0.0:
            zero.append(ones)
    assert len(zero) == 2
    f2_min = min(f2_all)
    for seed in range(1, 6):
        types = oracle.init_config(16, n_per, seed)
        cnt = oracle.counts(kind, L, M, S, types)
        _, _, res, _ = oracle.search(kind, L, M, n_per, w, b2, types, cnt, K=16, max_steps=200, seed=seed,
                                     depth_limit=20)
        assert res["f2"] >= f2_min


def test_multi_accept_group_top_keeps_group_winners():
    """With group_top = 1 the walk only sees the best eligible candidate of each group of
    group_size consecutive candidates (checked against keys from the oracle's delta)."""
    kind, L, M, S = ind.FCC, (6, 6, 6), 3, 4
    N, n_per, types, cnt, w, target = setup(kind, L, M, S, 6, target_scale=0.8)
    K, G = 256, 32
    pairs = oracle.draw_pairs(N, 3, 0, 0, 1, K)
    key, _, null = oracle.delta_swap(kind, L, M, n_per, w, target, types, cnt, pairs)
    winners = set()
    for g in range(K // G):
        cand = [c for c in range(g * G, (g + 1) * G) if not null[c] and key[c] < 0]
        if cand:
            winners.add(min(cand, key=lambda c: (key[c], c)))
    _, _, res, acc = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=K, max_steps=1, accept_mode=1,
                                   seed=3, group_size=G, group_top=1, log=True)
    assert 0 < res["accepted"] <= len(winners)
    assert {tuple(x) for x in acc} <= {tuple(pairs[c]) for c in winners}
    # group_top >= group_size keeps everything: same as the plain rule.
    a = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=K, max_steps=3, accept_mode=1, seed=3)
    b = oracle.search(kind, L, M, n_per, w, target, types, cnt, K=K, max_steps=3, accept_mode=1, seed=3,
                      group_size=G, group_top=G)
    assert np.array_equal(a[0], b[0]) and a[2]["f2"] == b[2]["f2"]
