"""GPU parity of the two full-recount kernels (Sec. 4.3, Eq. sro counts) against the oracle:
neighbour gathers (configurations staged whole, staged in slabs with halos, or read through the
cache) and bit planes (popcount of species planes), bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2411_18906_gb300 import hea, workloads
from tests import gpu_util as G
from tests.test_gpu_parity import composition

pytestmark = pytest.mark.gpu

FCC, BCC = workloads.FCC, workloads.BCC


def run_method(kind, L, M, S, batch, method):
    import torch
    G.ensure_built()
    lat = hea.Lattice(kind, L, M)
    tb = np.ascontiguousarray(batch, dtype=np.uint8).reshape(-1, lat.N)
    t = G.dev(tb)
    counts = torch.full((tb.shape[0], M, S, S), -7, dtype=torch.int32, device="cuda")
    hea.hea_sro_counts_method(lat, tb.shape[0], t, S, counts, method)
    torch.cuda.synchronize()
    return counts.cpu().numpy()


def random_batch(kind, L, S, n_cfg, seed):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    return np.stack([oracle.init_config(N, composition(N, S, rng), seed + c) for c in range(n_cfg)])


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("kind,L,M,S,n_cfg", [
    (FCC, (3, 3, 3), 2, 3, 5), (BCC, (20, 20, 20), 2, 5, 70), (FCC, (5, 6, 7), 5, 4, 3),
    (BCC, (4, 4, 4), 5, 6, 4), (FCC, (2, 2, 2), 3, 2, 3), (BCC, (9, 7, 5), 3, 6, 2),
    (FCC, (64, 3, 2), 3, 4, 2), (BCC, (33, 5, 4), 4, 5, 2),
])
def test_recount_kernels_match_oracle(kind, L, M, S, n_cfg, method):
    batch = random_batch(kind, L, S, n_cfg, 7 * S + M)
    got = run_method(kind, L, M, S, batch, method)
    for c in range(n_cfg):
        assert np.array_equal(got[c], oracle.counts(kind, L, M, S, batch[c])), c


def test_gather_staged_in_slabs_with_halos():
    """BCC 30^3 (54,000 sites: more than one CTA stages at once) x 100 configurations: slabs of planes
    with halo planes on both sides."""
    kind, L, M, S = BCC, (30, 30, 30), 3, 4
    batch = random_batch(kind, L, S, 100, 5)
    got = run_method(kind, L, M, S, batch, 1)
    for c in (0, 37, 99):
        assert np.array_equal(got[c], oracle.counts(kind, L, M, S, batch[c])), c


def test_gather_through_cache_single_large_cell():
    """FCC 40^3 (256,000 sites), one configuration: sites in chunks read through the cache."""
    spec = workloads.fcc_256k()
    batch = oracle.init_config(spec.N, spec.n_per, 3)[None]
    got = run_method(spec.kind, spec.L, spec.M, spec.S, batch, 1)
    assert np.array_equal(got[0], oracle.counts(spec.kind, spec.L, spec.M, spec.S, batch[0]))


def test_methods_agree_and_refuse_inapplicable():
    kind, L, M, S = BCC, (20, 20, 20), 2, 5
    batch = random_batch(kind, L, S, 64, 11)
    a, b, c = (run_method(kind, L, M, S, batch, m) for m in (0, 1, 2))
    assert np.array_equal(a, b) and np.array_equal(b, c)
    G.ensure_built()
    import torch
    lat = hea.Lattice(FCC, (65, 2, 2), 2)        # rows of 65 cells: no bit planes
    buf = torch.zeros(lat.N * 8, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(2 * 4 * 4, dtype=torch.int32, device="cuda")
    with pytest.raises(hea.HeaError) as e:
        hea.hea_sro_counts_method(lat, 1, buf, 4, cnt, 2)
    assert e.value.status == hea.HEA_EINVAL
    with pytest.raises(hea.HeaError):
        hea.hea_sro_counts_method(lat, 1, buf, 4, cnt, 3)


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("kind,L,M,S", [(FCC, (3, 3, 3), 2, 3), (BCC, (6, 5, 4), 3, 5)])
def test_out_of_range_species_not_counted(kind, L, M, S, method):
    """Sites holding a value >= S drop out of every pair, in both kernels (the bit-plane kernel
    then counts every pair instead of taking the last species from the row sums)."""
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(5 * S + M)
    t = oracle.init_config(N, composition(N, S, rng), 3)
    t2 = t.copy()
    t2[::7] = 200                                   # not a species
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
    got = run_method(kind, L, M, S, np.stack([t2, t]), method)
    assert np.array_equal(got[0], want)
    assert np.array_equal(got[1], oracle.counts(kind, L, M, S, t))
