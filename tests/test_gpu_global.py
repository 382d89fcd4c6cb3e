"""GPU parity of the global search (Sec. 4.1, Alg. global_search) against the oracle: the final
ranked set (configurations, counts, F^2), the per-iteration log (selected pool index, F^2 before
and after every refinement, its steps and accepted swaps) and the totals, bit for bit.  At the
presets' full sizes (Sec. 2.1) the result is checked by properties that hold at any size and by
replaying sampled refinements in the oracle."""
import numpy as np
import pytest

import oracle
from paper_2411_18906_gb300 import workloads
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

FCC, BCC = workloads.FCC, workloads.BCC


def objective(M, S, seed, scale):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 1.5, M), scale * rng.uniform(-1, 1, (M, S, S))


def compare(case, seed, **kw):
    kind, L, M, n_per, scale = case
    w, target = objective(M, len(n_per), seed, scale)
    got = G.gpu_global_search(kind, L, M, n_per, w, target, seed=seed, **kw)
    okw = dict(kw)
    want = oracle.global_search(kind, L, M, n_per, w, target, seed=seed, **okw)
    types, cnt, f2, log, res = got
    wt, wc, wf, wl, wtot = want
    for name in ("origin", "f2_in", "f2_out", "steps", "accepted"):
        assert np.array_equal(log[name], wl[name]), name
    assert np.array_equal(types, wt) and np.array_equal(cnt, wc) and np.array_equal(f2, wf)
    assert (res["steps"], res["trials"], res["accepted"]) == wtot
    assert res["iterations"] == kw["iterations"] and res["status"] == 0
    assert res["best_f2"] == wf[0] and res["best_f"] == np.sqrt(wf[0])
    return got


@pytest.mark.parametrize("case,kw", [
    ((FCC, (2, 2, 2), 2, [8, 8, 8, 8], 0.0), dict(n_solutions=8, iterations=3, tasks=8, depth_limit=4)),
    ((BCC, (3, 2, 2), 3, [9, 9, 6], 0.4), dict(n_solutions=10, n_refine=6, n_keep=3, iterations=3, tasks=12,
                                               depth_limit=3)),
    ((FCC, (2, 3, 2), 1, [20, 28], 0.3), dict(n_solutions=9, n_refine=5, n_keep=1, iterations=4, tasks=4,
                                              depth_limit=5)),
    ((FCC, (4, 4, 4), 3, [64] * 4, 0.0), dict(n_solutions=16, iterations=3, tasks=32, depth_limit=8)),
    ((BCC, (5, 4, 3), 2, [30, 40, 50], 0.5), dict(n_solutions=20, n_refine=12, n_keep=6, iterations=3, tasks=64,
                                                  depth_limit=6, accept_mode=1)),
    ((FCC, (3, 3, 3), 3, [30, 20, 25, 33], 0.2), dict(n_solutions=7, n_refine=7, n_keep=0, iterations=2, tasks=300,
                                                      depth_limit=3)),
])
def test_global_search_matches_oracle(case, kw):
    compare(case, 5, **kw)


def test_single_solution_and_single_iteration():
    compare((BCC, (2, 2, 2), 2, [8, 8], 0.5), 2, n_solutions=1, iterations=1, tasks=16, depth_limit=4)
    compare((FCC, (2, 2, 2), 1, [16, 16], 0.0), 3, n_solutions=5, n_refine=1, n_keep=0, iterations=3, tasks=8,
            depth_limit=2)


def check_properties(spec, gp_kw, got, replay_max_trials):
    types, cnt, f2, log, res = got
    S = spec.S
    w, target = spec.weights(), spec.targets()
    PL = log.shape[1]
    R = PL // 2
    assert np.all(np.diff(f2) >= 0)
    for r in range(PL):
        assert np.bincount(types[r], minlength=S).tolist() == list(spec.n_per)
    # counts and F^2 of every returned configuration, against the oracle
    for r in range(PL):
        c = oracle.counts(spec.kind, spec.L, spec.M, S, types[r])
        assert np.array_equal(c, cnt[r]), r
        assert oracle.alpha_f2(spec.kind, spec.L, spec.M, spec.n_per, w, target, c)[1] == f2[r]
    # a refinement accepts only swaps whose key D < 0, so F^2 does not rise beyond the rounding of
    # the key (a swap whose exact change is 0 may be taken on a key that rounded below 0)
    assert np.all(log["f2_out"] <= log["f2_in"] * (1 + 1e-12))
    for g in range(1, log.shape[0]):
        prev = np.sort(log["f2_out"][g - 1], kind="stable")
        kept = log["origin"][g] < R
        assert kept.sum() == R and np.array_equal(np.sort(log["f2_in"][g][kept]), prev[:R])
    best = log["f2_out"].min(axis=1)
    assert np.all(best[1:] <= best[:-1] * (1 + 1e-12)) and res["best_f2"] == f2[0] == best[-1]
    assert res["trials"] == res["steps"] * gp_kw["tasks"]
    assert res["steps"] == int(log["steps"].sum()) and res["accepted"] == int(log["accepted"].sum())
    # replay the cheapest fresh refinement of the first iteration in the oracle
    g = 0
    r = int(np.argmin(log["steps"][g]))
    if log["steps"][g, r] * gp_kw["tasks"] <= replay_max_trials:
        t0 = oracle.init_config(spec.N, spec.n_per, oracle.fresh_seed(1, g, int(log["origin"][g, r])))
        c0 = oracle.counts(spec.kind, spec.L, spec.M, S, t0)
        assert oracle.alpha_f2(spec.kind, spec.L, spec.M, spec.n_per, w, target, c0)[1] == log["f2_in"][g, r]
        _, _, rr, _ = oracle.search(spec.kind, spec.L, spec.M, spec.n_per, w, target, t0, c0, K=gp_kw["tasks"],
                                    max_steps=1 << 30, depth_limit=gp_kw["depth_limit"], seed=1, chain=g * 65536 + r)
        assert rr["f2"] == log["f2_out"][g, r] and rr["steps"] == log["steps"][g, r]
        assert rr["accepted"] == log["accepted"][g, r]


@pytest.mark.parametrize("preset", ["performance", "precision"])
@pytest.mark.parametrize("which", ["fcc_256", "bcc_16k"])
def test_presets_full_size(preset, which):
    spec = getattr(workloads, which)()
    kw = dict(workloads.GLOBAL_PRESETS[preset])
    got = G.gpu_global_search(spec.kind, spec.L, spec.M, spec.n_per, spec.weights(), spec.targets(), seed=1, **kw)
    check_properties(spec, kw, got, replay_max_trials=400_000)


def test_performance_preset_fcc_256_matches_oracle_exactly():
    spec = workloads.fcc_256()
    kw = dict(workloads.GLOBAL_PRESETS["performance"])
    kw.update(n_solutions=16, iterations=3)
    compare((spec.kind, spec.L, spec.M, spec.n_per, 0.0), 1, **kw)
