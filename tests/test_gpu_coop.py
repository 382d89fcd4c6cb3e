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
