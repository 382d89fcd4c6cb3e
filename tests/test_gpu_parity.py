"""GPU parity: every libhea entry point against the CPU oracle on the same seeded inputs.

Counts, configurations, step/accept tallies and the FP64 objective are compared bit for bit (the
objective arithmetic is fixed operation by operation, so the tolerance is zero).  Sizes span
several CTA tiles with ragged tails, the degenerate cases of the method (null moves, a-b bonds,
cells of two conventional cells where one site is reached by several shell vectors, absent
species in the initial composition) and the full-size workloads.
"""
import numpy as np
import pytest

import oracle
from paper_2411_18906_gb300 import workloads
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

FCC, BCC = workloads.FCC, workloads.BCC


def random_objective(M, S, rng, scale=0.3, symmetric=False):
    w = rng.uniform(0.3, 1.7, M)
    t = rng.uniform(-scale, scale, (M, S, S))
    if symmetric:
        t = 0.5 * (t + t.transpose(0, 2, 1))
    return w, t


def composition(N, S, rng, lo=1):
    return list(rng.multinomial(N - lo * S, np.ones(S) / S) + lo)


# ------------------------------------------------------------------------------------------------
# Initial configuration
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,L,n_per,seed", [
    (FCC, (4, 4, 4), [64, 64, 64, 64], 1),
    (BCC, (20, 20, 20), [3200] * 5, 3),
    (FCC, (40, 40, 40), workloads.composition_counts(256000, [0.4, 0.2, 0.2, 0.2]), 1),
    (BCC, (3, 2, 2), [0, 12, 0, 12], 5),                  # absent species
    (FCC, (3, 5, 7), [420], 2),                            # one species
    (FCC, (5, 5, 3), [38, 37, 37, 37, 37, 37, 37, 40], 9),  # eight species, ragged
    (BCC, (4, 4, 4), [13] * 9 + [11], 4),                  # more than eight species
    (FCC, (64, 64, 64), [262144] * 4, 6),                   # ~256 keys per 12-bit bin: buffer overflow path
])
def test_init_config_matches_oracle(kind, L, n_per, seed):
    got = G.gpu_init(kind, L, 1, n_per, seed)
    want = oracle.init_config(len(got), n_per, seed)
    assert np.array_equal(got, want)


# ------------------------------------------------------------------------------------------------
# Full recount
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,L,M,S,n_cfg", [
    (FCC, (2, 2, 2), 5, 3, 3), (BCC, (2, 2, 2), 5, 4, 3),        # shells wrap: multiplicities
    (FCC, (3, 5, 7), 3, 4, 5), (BCC, (7, 3, 5), 4, 6, 4),        # ragged, several tiles
    (FCC, (9, 8, 7), 5, 8, 2), (BCC, (11, 9, 6), 2, 2, 7),
    (FCC, (4, 4, 4), 3, 4, 1), (BCC, (20, 20, 20), 2, 5, 6),
    (FCC, (40, 40, 40), 3, 4, 1),
])
def test_counts_match_oracle(kind, L, M, S, n_cfg):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(N + 31 * S + n_cfg)
    batch = np.stack([oracle.init_config(N, composition(N, S, rng), 100 + c) for c in range(n_cfg)])
    got = G.gpu_counts(kind, L, M, S, batch)
    for c in range(n_cfg):
        assert np.array_equal(got[c], oracle.counts(kind, L, M, S, batch[c])), c


def test_counts_thousand_configs_full_size():
    """BCC 20^3, 5 species: 1000 seeded configurations in one call.  A sample is checked against
    the oracle; every configuration satisfies sum_j N_ij = N_i Z_k and symmetry."""
    kind, L, M, S = BCC, (20, 20, 20), 2, 5
    N = 16000
    n_per = workloads.equiatomic(N, S)
    batch = np.stack([G.gpu_init(kind, L, M, n_per, seed) for seed in range(1, 1001)])
    got = G.gpu_counts(kind, L, M, S, batch)
    Z = [8, 6]
    for k in range(M):
        assert np.all(got[:, k].sum(axis=2) == np.array(n_per)[None, :] * Z[k])
        assert np.all(got[:, k] == got[:, k].transpose(0, 2, 1))
    for c in (0, 1, 499, 998, 999):
        assert np.array_equal(got[c], oracle.counts(kind, L, M, S, batch[c]))


def test_counts_ignore_out_of_range_species():
    kind, L, M, S = FCC, (3, 3, 3), 2, 3
    N = 108
    t = oracle.init_config(N, [36, 36, 36], 3)
    t2 = t.copy()
    t2[::7] = 200                                   # not a species
    got = G.gpu_counts(kind, L, M, S, t2)[0]
    # Pairs touching the marked sites are dropped; everything else is counted.
    nbr = oracle.neighbours(kind, L, M)
    Z, _, _ = oracle.shells(kind, M)
    want = np.zeros((M, S, S), np.int64)
    for s in range(N):
        if t2[s] >= S:
            continue
        start = 0
        for k in range(M):
            for n in nbr[s, start:start + Z[k]]:
                if t2[n] < S:
                    want[k, t2[s], t2[n]] += 1
            start += Z[k]
    assert np.array_equal(got, want)


# ------------------------------------------------------------------------------------------------
# alpha and F^2
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,L,M,S", [(FCC, (4, 4, 4), 3, 4), (BCC, (5, 3, 4), 5, 7), (FCC, (2, 2, 2), 1, 2)])
def test_alpha_f2_bit_exact(kind, L, M, S):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(11 * S)
    n_per = composition(N, S, rng)
    t = oracle.init_config(N, n_per, 7)
    cnt = oracle.counts(kind, L, M, S, t)
    w, target = random_objective(M, S, rng)
    a_g, f2_g = G.gpu_alpha(kind, L, M, n_per, w, target, cnt)
    a_o, f2_o = oracle.alpha_f2(kind, L, M, n_per, w, target, cnt)
    assert np.array_equal(a_g, a_o)
    assert f2_g == f2_o


# ------------------------------------------------------------------------------------------------
# Delta of candidate swaps
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,L,M,S,seed", [(FCC, (2, 2, 2), 5, 3, 1), (BCC, (2, 2, 2), 5, 4, 2),
                                             (FCC, (4, 4, 4), 3, 4, 3), (BCC, (20, 20, 20), 2, 5, 4),
                                             (FCC, (5, 4, 6), 4, 8, 5), (BCC, (3, 4, 5), 3, 2, 6)])
def test_delta_swap_bit_exact(kind, L, M, S, seed):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    n_per = composition(N, S, rng)
    t = oracle.init_config(N, n_per, seed)
    cnt = oracle.counts(kind, L, M, S, t)
    w, target = random_objective(M, S, rng)
    nbr = oracle.neighbours(kind, L, M)
    pairs = [tuple(x) for x in rng.integers(0, N, (700, 2))]
    pairs += [(a, int(nbr[a, rng.integers(0, nbr.shape[1])])) for a in rng.integers(0, N, 300)]
    pairs += [(0, 0), (N - 1, N - 1), (0, N - 1)]
    pairs = np.array(pairs, np.int64)
    k_g, d_g = G.gpu_delta(kind, L, M, n_per, w, target, t, cnt, pairs)
    k_o, d_o, _ = oracle.delta_swap(kind, L, M, n_per, w, target, t, cnt, pairs)
    assert np.array_equal(d_g, d_o)
    assert np.array_equal(k_g.view(np.uint64), k_o.view(np.uint64))


# ------------------------------------------------------------------------------------------------
# Search trajectories
# ------------------------------------------------------------------------------------------------
def run_both(kind, L, M, S, n_per, w, target, seed_cfg, **kw):
    t = oracle.init_config(oracle.num_sites(kind, L), n_per, seed_cfg)
    cnt = oracle.counts(kind, L, M, S, t)
    tg, cg, rg = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, **kw)
    to, co, ro, _ = oracle.search(kind, L, M, n_per, w, target, t, cnt, **kw)
    return (tg, cg, rg), (to, co, ro)


def assert_same(g, o):
    tg, cg, rg = g
    to, co, ro = o
    assert rg["status"] == ro["status"] == 0
    for f in ("steps", "trials", "accepted", "depth"):
        assert rg[f] == ro[f], f
    assert np.array_equal(cg, co)
    assert np.array_equal(tg, to)
    assert rg["f2"] == ro["f2"] and rg["f"] == ro["f"]


def fcc256_spec():
    spec = workloads.fcc_256()
    return spec.kind, spec.L, spec.M, spec.S, spec.n_per, spec.weights(), spec.targets()


def test_search_fcc256_full_budget_best_of_32():
    """FCC 4x4x4, 4 species, shells 1-3, target 0: 1e5 trials at K = 32 (3125 steps)."""
    kind, L, M, S, n_per, w, target = fcc256_spec()
    g, o = run_both(kind, L, M, S, n_per, w, target, 1, K=32, max_steps=3125, seed=1)
    assert_same(g, o)
    assert g[2]["trials"] == 100000


def test_search_bcc16k_full_budget_best_of_256():
    """BCC 20x20x20, 5 x 3200, shells 1-2, target 0: 39,063 steps at K = 256 (10,000,128 trials)."""
    spec = workloads.bcc_16k()
    g, o = run_both(spec.kind, spec.L, spec.M, spec.S, spec.n_per, spec.weights(), spec.targets(), spec.seed, K=256,
                    max_steps=39063, seed=1)
    assert_same(g, o)
    assert g[2]["trials"] == 10_000_128


@pytest.mark.parametrize("kind,L,M,S,K,steps,seed", [
    (FCC, (2, 2, 2), 5, 3, 8, 300, 1), (BCC, (2, 2, 2), 5, 2, 16, 300, 2),
    (FCC, (3, 5, 4), 3, 5, 64, 400, 3), (BCC, (5, 5, 5), 4, 6, 100, 300, 4),
    (FCC, (6, 6, 6), 2, 8, 256, 200, 5), (BCC, (20, 20, 20), 2, 5, 256, 150, 6),
    (FCC, (4, 4, 4), 1, 2, 1, 2000, 7), (BCC, (8, 8, 8), 3, 4, 700, 60, 8),
])
def test_search_best_of_k_bit_exact(kind, L, M, S, K, steps, seed):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    n_per = composition(N, S, rng)
    w, target = random_objective(M, S, rng, scale=0.6)
    g, o = run_both(kind, L, M, S, n_per, w, target, seed, K=K, max_steps=steps, seed=seed + 10, chain=seed)
    assert_same(g, o)


@pytest.mark.parametrize("kind,L,M,S,K,steps,max_acc,seed", [
    (FCC, (6, 6, 6), 3, 4, 256, 30, 0, 1), (BCC, (9, 9, 9), 2, 5, 512, 20, 0, 2),
    (FCC, (3, 3, 3), 5, 3, 64, 60, 0, 3), (BCC, (10, 10, 10), 3, 6, 256, 25, 5, 4),
    (FCC, (10, 10, 10), 3, 4, 1024, 10, 0, 5),
    (BCC, (16, 16, 16), 2, 4, 2048, 3, 0, 6),     # ranked lists longer than the pairwise walk holds
])
def test_search_multi_accept_bit_exact(kind, L, M, S, K, steps, max_acc, seed):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    n_per = composition(N, S, rng)
    w, target = random_objective(M, S, rng, scale=0.8, symmetric=True)
    g, o = run_both(kind, L, M, S, n_per, w, target, seed, K=K, max_steps=steps, accept_mode=1,
                    max_accept=max_acc, seed=seed + 20)
    assert_same(g, o)
    if N < 1000:
        return      # closed neighbourhoods of 5 shells cover most of a tiny cell
    # Several swaps in one step: the first step alone accepts more than one.
    t = oracle.init_config(N, n_per, seed)
    cnt = oracle.counts(kind, L, M, S, t)
    _, _, r1 = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, K=K, max_steps=1, accept_mode=1,
                            max_accept=max_acc, seed=seed + 20)
    assert r1["accepted"] > 1


def test_search_threshold_accepts_bounded_uphill():
    kind, L, M, S = FCC, (3, 3, 3), 3, 3
    rng = np.random.default_rng(9)
    n_per = composition(108, S, rng)
    w, target = random_objective(M, S, rng)
    for mode in (0, 1):
        g, o = run_both(kind, L, M, S, n_per, w, target, 9, K=16, max_steps=200, threshold=1e-3,
                        accept_mode=mode, seed=4)
        assert_same(g, o)


def test_search_depth_limit_and_resume():
    kind, L, M, S = BCC, (6, 6, 6), 3, 4
    rng = np.random.default_rng(13)
    n_per = composition(432, S, rng)
    w, target = random_objective(M, S, rng)
    g, o = run_both(kind, L, M, S, n_per, w, target, 2, K=8, max_steps=100000, depth_limit=6, seed=3)
    assert_same(g, o)
    assert g[2]["depth"] == 6 and g[2]["steps"] < 100000
    # Resume: 37 + 63 steps equal 100 straight steps.
    t = oracle.init_config(432, n_per, 2)
    cnt = oracle.counts(kind, L, M, S, t)
    ta, ca, ra = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, K=8, max_steps=100, seed=3)
    t1, c1, r1 = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, K=8, max_steps=37, seed=3)
    tb, cb, rb = G.gpu_search(kind, L, M, n_per, w, target, t1, c1, K=8, max_steps=63, seed=3, step0=37,
                              depth0=r1["depth"])
    assert np.array_equal(ta, tb) and np.array_equal(ca, cb) and ra["f2"] == rb["f2"]


def test_search_zero_steps_and_single_candidate():
    kind, L, M, S, n_per, w, target = fcc256_spec()
    g, o = run_both(kind, L, M, S, n_per, w, target, 1, K=1, max_steps=0, seed=1)
    assert_same(g, o)
    g, o = run_both(kind, L, M, S, n_per, w, target, 1, K=1, max_steps=5000, seed=2)
    assert_same(g, o)


def test_search_time_budget_reports_timeout():
    kind, L, M, S = BCC, (20, 20, 20), 2, 5
    n_per = workloads.equiatomic(16000, S)
    t = oracle.init_config(16000, n_per, 1)
    cnt = oracle.counts(kind, L, M, S, t)
    tg, cg, rg = G.gpu_search(kind, L, M, n_per, np.ones(M), np.zeros((M, S, S)), t, cnt, K=256,
                              max_steps=2**31, seed=1, timeout_us=2000)
    assert rg["status"] == 4                       # HEA_ETIMEOUT
    assert 0 < rg["steps"] < 2**31
    # The state it stopped in is consistent.
    assert np.array_equal(cg, oracle.counts(kind, L, M, S, tg))
    to, co, ro, _ = oracle.search(kind, L, M, n_per, np.ones(M), np.zeros((M, S, S)), t, cnt, K=256,
                                  max_steps=rg["steps"], seed=1)
    assert np.array_equal(tg, to)


def test_search_rejects_species_out_of_range_on_device():
    kind, L, M, S, n_per, w, target = fcc256_spec()
    t = oracle.init_config(256, n_per, 1)
    cnt = oracle.counts(kind, L, M, S, t)
    t[17] = 9
    tg, cg, rg = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, K=4, max_steps=10, seed=1)
    assert rg["status"] == 1 and rg["steps"] == 0


def test_search_annealed_target_fcc_4000():
    entry = workloads.annealed_targets()["fcc_4sp_40_20_20_20"]
    kind, L, M, S = FCC, (10, 10, 10), 3, 4
    n_per = entry["n_per"]
    target = np.array(entry["alpha"])
    for mode, K in ((0, 128), (1, 256)):
        g, o = run_both(kind, L, M, S, n_per, np.ones(M), target, 5, K=K, max_steps=200, accept_mode=mode, seed=8)
        assert_same(g, o)


# ------------------------------------------------------------------------------------------------
# Batched search
# ------------------------------------------------------------------------------------------------
def test_batch_matches_independent_oracle_runs():
    rng = np.random.default_rng(77)
    cells, params, oracle_out = [], [], []
    specs = [(FCC, (4, 4, 4), 3, 4), (BCC, (5, 4, 3), 2, 3), (FCC, (2, 3, 2), 5, 5), (BCC, (8, 8, 8), 1, 6),
             (FCC, (7, 6, 5), 3, 8), (BCC, (2, 2, 2), 3, 2), (FCC, (12, 12, 12), 2, 4), (BCC, (20, 20, 20), 2, 5)]
    for c, (kind, L, M, S) in enumerate(specs):
        N = oracle.num_sites(kind, L)
        n_per = composition(N, S, rng)
        w, target = random_objective(M, S, rng, scale=0.5)
        t = oracle.init_config(N, n_per, 40 + c)
        cnt = oracle.counts(kind, L, M, S, t)
        kw = dict(K=int(rng.choice([16, 64, 256])), max_steps=int(rng.integers(50, 150)),
                  accept_mode=int(c % 2), seed=90 + c, chain=c)
        cells.append((kind, L, M, n_per, w, target, t, cnt))
        params.append(kw)
        oracle_out.append(oracle.search(kind, L, M, n_per, w, target, t, cnt, **kw))
    ts, cs, rs = G.gpu_search_batch(cells, params)
    for c in range(len(cells)):
        to, co, ro, _ = oracle_out[c]
        assert_same((ts[c], cs[c], rs[c]), (to, co, ro))


# ------------------------------------------------------------------------------------------------
# Full-size single chain in the benchmark's launch configuration
# ------------------------------------------------------------------------------------------------
def test_fcc_256k_multi_accept_matches_oracle_prefix():
    """FCC 40^3, 40/20/20/20, shells 1-3, annealed target, multi-accept at the benchmark's K:
    a prefix of the trajectory bit-exact against the oracle."""
    spec = workloads.fcc_256k()
    from bench import SEARCH_K
    g, o = run_both(spec.kind, spec.L, spec.M, spec.S, spec.n_per, spec.weights(), spec.targets(), spec.seed,
                    K=SEARCH_K, max_steps=12, accept_mode=1, seed=1)
    assert_same(g, o)


@pytest.mark.parametrize("kind,L,M,S,K,G,top,steps", [
    (FCC, (8, 8, 8), 3, 4, 256, 32, 1, 40), (BCC, (10, 10, 10), 2, 5, 512, 64, 2, 30),
    (FCC, (5, 6, 7), 3, 6, 1024, 256, 4, 15), (BCC, (4, 4, 4), 5, 3, 96, 17, 1, 50),
])
def test_search_multi_accept_group_rule_bit_exact(kind, L, M, S, K, G, top, steps):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(K + G)
    n_per = composition(N, S, rng)
    w, target = random_objective(M, S, rng, scale=0.8, symmetric=True)
    g, o = run_both(kind, L, M, S, n_per, w, target, 3, K=K, max_steps=steps, accept_mode=1, group_size=G,
                    group_top=top, seed=11)
    assert_same(g, o)


@pytest.mark.parametrize("mode,K", [(0, 512), (1, 512), (1, 2048)])
def test_search_massive_key_ties_from_ordered_start(mode, K):
    """B2-ordered BCC 8^3 with a zero target: swaps with identical surroundings have bit-identical
    keys, so hundreds of candidates tie and are ordered by k alone (large overlap clusters)."""
    kind, L, M, S = BCC, (8, 8, 8), 3, 2
    pos = oracle.positions(kind, L)
    t = (pos[:, 0] % 2).astype(np.uint8)
    n_per = [512, 512]
    cnt = oracle.counts(kind, L, M, S, t)
    w, target = np.ones(M), np.zeros((M, S, S))
    tg, cg, rg = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, K=K, max_steps=6, accept_mode=mode, seed=3)
    to, co, ro, _ = oracle.search(kind, L, M, n_per, w, target, t, cnt, K=K, max_steps=6, accept_mode=mode, seed=3)
    assert_same((tg, cg, rg), (to, co, ro))
    assert ro["accepted"] > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_two_bit_species_storage_half_million_sites(mode):
    """FCC 50^3 (500,000 sites, 4 species): the cell fits one CTA's shared memory only at 2 bits per
    site; a prefix of the trajectory bit-exact against the oracle."""
    kind, L, M, S = FCC, (50, 50, 50), 3, 4
    N = oracle.num_sites(kind, L)
    entry = workloads.annealed_targets()["pool_fcc_4sp"][2]
    n_per = workloads.composition_counts(N, entry["fractions"])
    g, o = run_both(kind, L, M, S, n_per, np.ones(M), np.array(entry["alpha"]), 5, K=256, max_steps=8,
                    accept_mode=mode, seed=4)
    assert_same(g, o)
    assert o[2]["accepted"] > 0


# ------------------------------------------------------------------------------------------------
# Threads per CTA (a launch shape: results must not depend on it)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("threads", [128, 512])
@pytest.mark.parametrize("kind,L,M,S,K,mode,steps,seed", [
    (FCC, (4, 4, 4), 3, 4, 32, 0, 400, 1), (BCC, (20, 20, 20), 2, 5, 1024, 0, 60, 2),
    (FCC, (6, 6, 6), 3, 4, 256, 1, 30, 3), (BCC, (10, 10, 10), 3, 6, 700, 1, 20, 4),
    (FCC, (3, 3, 3), 5, 3, 64, 1, 60, 5), (BCC, (16, 16, 16), 2, 4, 2048, 1, 3, 6),
])
def test_search_threads_per_cta_bit_exact(threads, kind, L, M, S, K, mode, steps, seed):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    n_per = composition(N, S, rng)
    w, target = random_objective(M, S, rng, scale=0.7, symmetric=mode == 1)
    t = oracle.init_config(N, n_per, seed)
    cnt = oracle.counts(kind, L, M, S, t)
    kw = dict(K=K, max_steps=steps, accept_mode=mode, seed=seed + 30)
    o = oracle.search(kind, L, M, n_per, w, target, t, cnt, **kw)[:3]
    g = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, threads=threads, **kw)
    assert_same(g, o)


def test_batch_mixed_threads_per_cta():
    rng = np.random.default_rng(5)
    cells, params, want = [], [], []
    for c, (kind, L, M, S, threads) in enumerate([(FCC, (4, 4, 4), 3, 4, 128), (BCC, (6, 5, 4), 2, 3, 512),
                                                  (FCC, (5, 5, 5), 2, 5, 256), (BCC, (8, 8, 8), 3, 4, 128),
                                                  (FCC, (3, 4, 5), 3, 6, 512), (BCC, (3, 3, 3), 1, 2, 0)]):
        N = oracle.num_sites(kind, L)
        n_per = composition(N, S, rng)
        w, target = random_objective(M, S, rng, scale=0.5)
        t = oracle.init_config(N, n_per, 60 + c)
        cnt = oracle.counts(kind, L, M, S, t)
        kw = dict(K=int(rng.choice([32, 128, 512])), max_steps=80, accept_mode=c % 2, seed=70 + c, chain=c)
        cells.append((kind, L, M, n_per, w, target, t, cnt))
        params.append(dict(kw, threads=threads))
        want.append(oracle.search(kind, L, M, n_per, w, target, t, cnt, **kw)[:3])
    ts, cs, rs = G.gpu_search_batch(cells, params)
    for c in range(len(cells)):
        assert_same((ts[c], cs[c], rs[c]), want[c])
