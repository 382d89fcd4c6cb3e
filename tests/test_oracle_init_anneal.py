"""Pins for the oracle's initial configuration (exact composition, the documented ordering rule
restated with numpy) and for the annealed-target recipe (energy changes of the delta rule equal
full-energy recomputes exactly; the stored targets are reproducible)."""
import numpy as np
import pytest

import oracle
from paper_2411_18906_gb300 import workloads
from tests import independent as ind


@pytest.mark.parametrize("N,n_per,seed", [(256, [64, 64, 64, 64], 1), (1000, [400, 200, 200, 200], 7),
                                          (17, [17], 3), (50, [0, 25, 25], 9)])
def test_init_composition_and_ordering_rule(N, n_per, seed):
    types = oracle.init_config(N, n_per, seed)
    assert np.array_equal(np.bincount(types, minlength=len(n_per)), n_per)
    # Restated: site i keyed by (r0 << 32 | i), r0 = Philox(counter (i,0,0,0), key (lo, hi of seed)).
    keys = []
    for i in range(N):
        r = oracle.philox4x32_10([i, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        keys.append((int(r[0]) << 32) | i)
    order = np.argsort(np.array(keys, dtype=np.uint64), kind="stable")
    want = np.zeros(N, np.uint8)
    want[order] = np.repeat(np.arange(len(n_per)), n_per).astype(np.uint8)
    assert np.array_equal(types, want)


def test_init_is_roughly_uniform():
    N, n_per = 4000, [1000, 1000, 1000, 1000]
    types = oracle.init_config(N, n_per, 5)
    cnt = oracle.counts(ind.FCC, (10, 10, 10), 1, 4, types)
    alpha, _ = oracle.alpha_f2(ind.FCC, (10, 10, 10), 1, n_per, [1.0], np.zeros((1, 4, 4)), cnt)
    assert np.abs(alpha).max() < 0.1     # a random arrangement has alpha near 0 (Sec. 4.3)


def test_swap_energy_change_is_exact():
    kind, L, S = ind.FCC, (4, 4, 4), 3
    N = 256
    n_per = workloads.composition_counts(N, [0.5, 0.3, 0.2])
    types = oracle.init_config(N, n_per, 4)
    rng = np.random.default_rng(1)
    eps = np.round(rng.uniform(-0.05, 0.05, (S, S)) * 2**30) / 2**30
    eps = np.triu(eps) + np.triu(eps, 1).T
    cnt = oracle.counts(kind, L, 1, S, types)
    pairs = rng.integers(0, N, (50, 2))
    _, dN, _ = oracle.delta_swap(kind, L, 1, n_per, [1.0], np.zeros((1, S, S)), types, cnt, pairs)
    e0 = oracle.energy(kind, L, types, eps)
    for c, (a, b) in enumerate(pairs):
        t2 = types.copy()
        t2[a], t2[b] = t2[b], t2[a]
        dE = 0.5 * float((dN[c, 0] * eps).sum())
        assert dE == oracle.energy(kind, L, t2, eps) - e0


def test_anneal_orders_and_lowers_energy():
    kind, L = ind.FCC, (6, 6, 6)
    n_per = workloads.composition_counts(864, [0.4, 0.3, 0.3])
    types, eps, alpha, taken = oracle.anneal(kind, L, n_per, seed=3, T=300.0, sweeps=30, M_out=3)
    rand = oracle.init_config(864, n_per, 3)
    assert oracle.energy(kind, L, types, eps) < oracle.energy(kind, L, rand, eps)
    assert taken > 0 and np.abs(alpha).max() > 0.1
    assert np.array_equal(np.bincount(types, minlength=3), n_per)


def test_stored_fcc_target_is_reproducible():
    entry = workloads.annealed_targets()["fcc_4sp_40_20_20_20"]
    L = tuple(entry["cell"])
    _, eps, alpha, taken = oracle.anneal(ind.FCC, L, entry["n_per"], entry["seed"], T=entry["T"],
                                         sweeps=entry["sweeps"], M_out=3)
    assert taken == entry["accepted_moves"]
    assert np.array_equal(alpha, np.array(entry["alpha"]))
    assert np.array_equal(eps, np.array(entry["eps"]))
