"""The serving loop: request recipe on CPU; on the GPU, continuous batching keeps every result
identical to the same request served alone, and admission never exceeds the memory budget."""
import numpy as np
import pytest

from paper_2411_18906_gb300 import serve, workloads


def test_poisson_request_recipe():
    reqs = serve.poisson_requests(2000, rate_per_s=50.0, seed=3)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 50) < 0.002
    sizes = np.array([r.cell.N for r in reqs])
    assert sizes.min() >= 500 and sizes.max() == 256000
    assert 0.17 < np.mean(sizes == 256000) < 0.30
    for r in reqs[:200]:
        assert sum(r.cell.n_per) == r.cell.N and r.cell.S in (4, 5) and r.cell.M == 3
        assert r.cell.targets().shape == (3, r.cell.S, r.cell.S)


def _small_requests(n, spread_s):
    pool = workloads.annealed_targets()
    rng = np.random.default_rng(5)
    out = []
    for rid in range(n):
        kind = rid % 2
        L = (4 + rid % 3, 4, 5) if kind == workloads.FCC else (6, 5 + rid % 2, 6)
        N = workloads.BASIS_SITES[kind] * L[0] * L[1] * L[2]
        S = 4 + rid % 2
        entry = pool[f"pool_{'fcc' if kind == 0 else 'bcc'}_{S}sp"][rid % 8]
        cell = workloads.CellSpec(kind, L, 3, workloads.composition_counts(N, entry["fractions"]), seed=500 + rid,
                                  target=np.array(entry["alpha"]))
        out.append(serve.Request(rid, float(rng.uniform(0, spread_s)), cell, K=128, max_trials=128 * 400,
                                 depth_limit=0 if rid % 3 else 10, accept_mode=rid % 2, seed=900 + rid))
    return out


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    reqs = _small_requests(16, spread_s=0.01)
    mixed = serve.Server(slots=16, keep_types=True).run(reqs)
    srv = serve.Server(slots=16, keep_types=True)
    assert len(mixed) == 16
    for r in reqs:
        r_alone = serve.Request(r.rid, 0.0, r.cell, r.K, r.max_trials, r.depth_limit, r.accept_mode, r.seed)
        alone = srv.run([r_alone])[0]
        m = mixed[r.rid]
        assert m.result == alone.result
        assert np.array_equal(m.types, alone.types)
    assert srv.max_inflight == 1


@pytest.mark.gpu
def test_admission_respects_memory_budget():
    reqs = _small_requests(12, spread_s=0.0)
    need = max(r.device_bytes() for r in reqs)
    srv = serve.Server(hbm_budget_bytes=2 * need + 10, slots=8)
    done = srv.run(reqs)
    assert len(done) == 12 and all(c.result["status"] == 0 for c in done)
    assert srv.max_reserved <= 2 * need + 10 and srv.max_inflight <= 2
    with pytest.raises(ValueError):
        serve.Server(hbm_budget_bytes=need // 2).run(reqs[:1])
