"""GPU parity of the cooperative search (one chain over many CTAs) against the CPU oracle and
against the single-CTA search: best-of-K is the plain best-of-K over all K candidates; the
multi-accept walk sees the group_top best eligible candidates of each CTA's slice."""
import numpy as np
import pytest

import oracle
from paper_2411_18906_gb300 import hea, workloads
from tests import gpu_util as G
from tests.test_gpu_parity import assert_same, composition, random_objective

pytestmark = pytest.mark.gpu

FCC, BCC = workloads.FCC, workloads.BCC


def both(kind, L, M, S, n_per, w, target, seed_cfg, ctas, **kw):
    N = oracle.num_sites(kind, L)
    t = oracle.init_config(N, n_per, seed_cfg)
    cnt = oracle.counts(kind, L, M, S, t)
    g = G.gpu_search_coop(kind, L, M, n_per, w, target, t, cnt, ctas, **kw)
    o = oracle.search(kind, L, M, n_per, w, target, t, cnt, **kw)[:3]
    return g, o, t, cnt


@pytest.mark.parametrize("kind,L,M,S,ctas,Kc,steps", [
    (FCC, (6, 6, 6), 3, 4, 2, 64, 60), (BCC, (10, 10, 10), 2, 5, 8, 32, 60),
    (FCC, (4, 4, 4), 3, 4, 16, 16, 80), (BCC, (5, 4, 3), 5, 3, 3, 100, 50),
])
def test_coop_best_of_k_bit_exact(kind, L, M, S, ctas, Kc, steps):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(ctas * Kc)
    n_per = composition(N, S, rng)
    w, target = random_objective(M, S, rng, scale=0.6)
    g, o, t, cnt = both(kind, L, M, S, n_per, w, target, 2, ctas, K=ctas * Kc, max_steps=steps, seed=3)
    assert_same(g, o)
    # Identical to the single-CTA kernel with the same K.
    ts, cs, rs = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, K=ctas * Kc, max_steps=steps, seed=3)
    assert np.array_equal(ts, g[0]) and rs["f2"] == g[2]["f2"]


@pytest.mark.parametrize("kind,L,M,S,ctas,Kc,top,steps", [
    (FCC, (8, 8, 8), 3, 4, 4, 128, 1, 30), (BCC, (10, 10, 10), 2, 5, 8, 64, 2, 30),
    (FCC, (6, 7, 8), 3, 6, 6, 96, 4, 25), (BCC, (6, 6, 6), 3, 4, 2, 256, 3, 25),
    (FCC, (9, 9, 9), 3, 4, 16, 64, 4, 80),      # long walks over many batches and steps
])
def test_coop_multi_accept_bit_exact(kind, L, M, S, ctas, Kc, top, steps):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(ctas + Kc + top)
    n_per = composition(N, S, rng)
    w, target = random_objective(M, S, rng, scale=0.8, symmetric=True)
    kw = dict(K=ctas * Kc, max_steps=steps, accept_mode=1, group_size=Kc, group_top=top, seed=5)
    g, o, t, cnt = both(kind, L, M, S, n_per, w, target, 4, ctas, **kw)
    assert_same(g, o)
    ts, cs, rs = G.gpu_search(kind, L, M, n_per, w, target, t, cnt, **kw)
    assert np.array_equal(ts, g[0]) and rs["f2"] == g[2]["f2"]


@pytest.mark.parametrize("ctas,Kc,top", [(4, 16, 2), (2, 32, 4), (8, 8, 3), (3, 40, 4)])
def test_coop_dense_conflicts_few_records(ctas, Kc, top):
    """FCC 4x4x4 with shells 1-3: the closed neighbourhood of a site covers 43 of the 256 sites, so
    a handful of published records conflict in more pairs than the fast walk's edge list holds
    (2 per record); the walk must fall back to the conflict matrix."""
    spec = workloads.fcc_256()
    entry = workloads.annealed_targets()["pool_fcc_4sp"][0]
    n_per = workloads.composition_counts(spec.N, entry["fractions"])
    target = np.array(entry["alpha"])
    kw = dict(K=ctas * Kc, max_steps=100, accept_mode=1, group_size=Kc, group_top=top, seed=6)
    g, o, t, cnt = both(spec.kind, spec.L, spec.M, len(n_per), n_per, spec.weights(), target, 3, ctas, **kw)
    assert_same(g, o)


def test_coop_rejects_bad_splits():
    G.ensure_built()
    lat = hea.Lattice(FCC, (4, 4, 4), 3)
    obj = hea.Objective([64] * 4, np.ones(3), np.zeros((3, 4, 4)))
    import torch
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    res = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for ctas, kw in [(3, dict(K=64)), (2, dict(K=64, accept_mode=1, group_size=16, group_top=1)),
                     (2, dict(K=64, accept_mode=1, group_size=32, group_top=9))]:
        with pytest.raises(hea.HeaError) as e:
            hea.hea_search_coop(lat, obj, hea.search_params(max_steps=1, **kw), ctas, buf, buf, res, buf)
        assert e.value.status == hea.HEA_EINVAL
    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(hea.HeaError):
        hea.hea_search_coop(lat, obj, hea.search_params(64, 1), 2, buf, buf, res, small)
    # more merged records than the walk holds (ctas * group_top > 640)
    with pytest.raises(hea.HeaError) as e:
        hea.hea_search_coop(lat, obj, hea.search_params(200 * 4, 1, accept_mode=1, group_size=4, group_top=4), 200,
                            buf, buf, res, torch.zeros(hea.hea_search_coop_workspace_bytes(200), dtype=torch.uint8,
                                                       device="cuda"))
    assert e.value.status == hea.HEA_EINVAL and "640" in str(e.value)
    # the withholding test aid belongs to cooperative searches only, and must name one of the CTAs
    with pytest.raises(hea.HeaError) as e:
        hea.hea_search(lat, obj, hea.search_params(64, 1, test_withhold_cta=1), buf, buf, res)
    assert e.value.status == hea.HEA_EINVAL
    with pytest.raises(hea.HeaError) as e:
        hea.hea_search_coop(lat, obj, hea.search_params(64, 1, test_withhold_cta=3), 2, buf, buf, res, buf)
    assert e.value.status == hea.HEA_EINVAL


def test_coop_time_budget():
    kind, L, M, S = BCC, (20, 20, 20), 2, 5
    n_per = workloads.equiatomic(16000, S)
    t = oracle.init_config(16000, n_per, 1)
    cnt = oracle.counts(kind, L, M, S, t)
    ctas = min(16, G.sm_count())
    tg, cg, rg = G.gpu_search_coop(kind, L, M, n_per, np.ones(M), np.zeros((M, S, S)), t, cnt, ctas,
                                   K=ctas * 64, max_steps=2**31, seed=1, timeout_us=3000)
    assert rg["status"] == hea.HEA_ETIMEOUT and 0 < rg["steps"] < 2**31
    assert np.array_equal(cg, oracle.counts(kind, L, M, S, tg))


@pytest.mark.parametrize("top", [1, 2])
def test_coop_fcc_256k_all_sms_prefix(top):
    """FCC 40^3 with the annealed target on every SM in the benchmark's launch configuration
    (candidates per CTA and published candidates per CTA from bench.py, and one other): a prefix of
    the trajectory bit-exact against the oracle."""
    from bench import COOP_KC, COOP_TOP
    spec = workloads.fcc_256k()
    ctas = G.sm_count()
    Kc = COOP_KC
    kw = dict(K=ctas * Kc, max_steps=6, accept_mode=1, group_size=Kc, group_top=(COOP_TOP if top == 1 else top),
              seed=1)
    g, o, _, _ = both(spec.kind, spec.L, spec.M, spec.S, spec.n_per, spec.weights(), spec.targets(), spec.seed,
                      ctas, **kw)
    assert_same(g, o)
    assert g[2]["accepted"] > 6


@pytest.mark.parametrize("mode", [0, 1])
def test_coop_wait_for_a_withheld_cta_runs_out(mode):
    """One CTA never publishes its records: every other CTA's wait for them is bounded (here 20 ms),
    the search ends with HEA_ESYNC after no completed step, the state written back is the input state,
    and the GPU context stays usable (the next search on the same workspace is bit-exact)."""
    import time
    import torch
    kind, L, M, S = FCC, (8, 8, 8), 3, 4
    N = oracle.num_sites(kind, L)
    n_per = workloads.equiatomic(N, S)
    w, target = np.ones(M), np.zeros((M, S, S))
    t = oracle.init_config(N, n_per, 3)
    cnt = oracle.counts(kind, L, M, S, t)
    ctas = min(8, G.sm_count())
    kw = dict(K=ctas * 64, max_steps=50, accept_mode=mode, seed=7)
    if mode == 1:
        kw.update(group_size=64, group_top=2)
    G.ensure_built()
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    ws = torch.zeros(hea.hea_search_coop_workspace_bytes(ctas), dtype=torch.uint8, device="cuda")
    tg, cg = G.dev(t), G.dev(cnt)
    res = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hea.hea_search_coop(lat, obj, hea.search_params(**kw, sync_wait_us=20000, test_withhold_cta=4), ctas, tg, cg,
                        res, ws)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    r = hea.decode_results(res.cpu().numpy())[0]
    assert r["status"] == hea.HEA_ESYNC and r["steps"] == 0 and r["accepted"] == 0
    assert elapsed < 1.5
    assert np.array_equal(tg.cpu().numpy(), t) and np.array_equal(cg.cpu().numpy(), cnt)
    # the same workspace, no CTA withheld: identical to the oracle
    hea.hea_search_coop(lat, obj, hea.search_params(**kw), ctas, tg, cg, res, ws)
    torch.cuda.synchronize()
    o = oracle.search(kind, L, M, n_per, w, target, t, cnt, **kw)[:3]
    assert_same((tg.cpu().numpy(), cg.cpu().numpy(), hea.decode_results(res.cpu().numpy())[0]), o)


def test_coop_fcc_256k_bench_trajectory_checkpoints():
    """The benchmark's launch (FCC 40^3, annealed target, one CTA per SM, bench.py's candidates and
    published records per CTA, seed 1) over its whole trajectory: from checkpoints at steps 100 and
    300, just before the last step that accepts a swap (where keys are tiny and intervals matter
    most) and 3 steps before the end, 3 GPU steps and 3 oracle steps (resumed with step0 / depth0)
    agree bit for bit; the full run ends in a state whose counts are its recount."""
    from bench import COOP_KC, COOP_TOP, TRIALS_PER_STEP
    spec = workloads.fcc_256k()
    ctas = G.sm_count()
    K = ctas * COOP_KC
    total = TRIALS_PER_STEP // K
    base = dict(K=K, accept_mode=1, group_size=COOP_KC, group_top=COOP_TOP, seed=spec.seed)
    args = (spec.kind, spec.L, spec.M, spec.n_per, spec.weights(), spec.targets())
    t0 = oracle.init_config(spec.N, spec.n_per, spec.seed)
    c0 = oracle.counts(spec.kind, spec.L, spec.M, spec.S, t0)
    tf, cf, rf = G.gpu_search_coop(*args, t0, c0, ctas, max_steps=total, **base)
    assert rf["status"] == 0 and rf["steps"] == total and rf["accepted"] > 0
    assert np.array_equal(cf, oracle.counts(spec.kind, spec.L, spec.M, spec.S, tf))
    _, f2 = oracle.alpha_f2(spec.kind, spec.L, spec.M, spec.n_per, spec.weights(), spec.targets(), cf)
    assert rf["f2"] == f2
    last = total - rf["depth"] - 1          # last step that accepted a swap
    for s in sorted({100, 300, max(1, last - 1), total - 3}):
        ts, cs, rs = G.gpu_search_coop(*args, t0, c0, ctas, max_steps=s, **base)
        kw = dict(base, max_steps=3, step0=s, depth0=rs["depth"])
        g = G.gpu_search_coop(*args, ts, cs, ctas, **kw)
        o = oracle.search(*args, ts, cs, **kw)[:3]
        assert_same(g, o)
        if s == total - 3:
            assert np.array_equal(g[0], tf) and np.array_equal(g[1], cf)


@pytest.mark.parametrize("mode,top", [(0, 1), (1, 1), (1, 3)])
def test_coop_massive_key_ties_from_ordered_start(mode, top):
    """B2-ordered BCC 8^3 with a zero target on 8 CTAs: swaps with identical surroundings have
    bit-identical keys in different CTAs, so the fixed-point intervals of the published records
    overlap and their order falls back to binary64 keys and k; bit-exact against the oracle."""
    kind, L, M, S = BCC, (8, 8, 8), 3, 2
    pos = oracle.positions(kind, L)
    t = (pos[:, 0] % 2).astype(np.uint8)
    n_per = [512, 512]
    cnt = oracle.counts(kind, L, M, S, t)
    w, target = np.ones(M), np.zeros((M, S, S))
    ctas, Kc = 8, 64
    kw = dict(K=ctas * Kc, max_steps=6, accept_mode=mode, seed=3)
    if mode == 1:
        kw.update(group_size=Kc, group_top=top)
    g = G.gpu_search_coop(kind, L, M, n_per, w, target, t, cnt, ctas, **kw)
    o = oracle.search(kind, L, M, n_per, w, target, t, cnt, **kw)[:3]
    assert_same(g, o)
    assert o[2]["accepted"] > 0


@pytest.mark.parametrize("Kc,top", [(2500, 1), (1500, 3)])
def test_coop_slices_scored_in_chunks(Kc, top):
    """A CTA's slice larger than one scoring pass (1024 candidates) is scored in chunks with the best
    candidates so far carried between them: bit-exact against the oracle's group rule."""
    kind, L, M, S = FCC, (8, 8, 8), 3, 4
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(Kc)
    n_per = composition(N, S, rng)
    w, target = random_objective(M, S, rng, scale=0.8, symmetric=True)
    ctas = 8
    kw = dict(K=ctas * Kc, max_steps=8, accept_mode=1, group_size=Kc, group_top=top, seed=13)
    g, o, _, _ = both(kind, L, M, S, n_per, w, target, 6, ctas, **kw)
    assert_same(g, o)
    assert o[2]["accepted"] > 0
