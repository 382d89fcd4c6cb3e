"""Pins for the oracle's pair counts, alpha and F^2: hand-derived closed forms of ordered
structures, invariants that hold for any configuration, an independent periodic-image recount,
and exhaustive enumeration of a 16-site binary cell."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from tests import independent as ind

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def closed_form(name):
    with open(GOLDEN) as fh:
        return json.load(fh)[name]


def ordered_types(kind, L, rule):
    pos = ind.positions(kind, L)
    if rule == "B2":
        return (pos[:, 0] % 2).astype(np.uint8)              # sublattice (1,1,1) -> B
    if rule == "L10":
        return (pos[:, 2] % 2).astype(np.uint8)              # odd half-unit z -> B
    if rule == "L12":
        corner = (pos % 2 == 0).all(axis=1)
        return np.where(corner, 1, 0).astype(np.uint8)        # corners -> B
    raise ValueError(rule)


@pytest.mark.parametrize("name,kind,L,rule", [
    ("B2_bcc", ind.BCC, (4, 4, 4), "B2"), ("B2_bcc", ind.BCC, (2, 3, 2), "B2"),
    ("L10_fcc", ind.FCC, (4, 4, 4), "L10"), ("L10_fcc", ind.FCC, (3, 2, 5), "L10"),
    ("L12_fcc", ind.FCC, (4, 4, 4), "L12"), ("L12_fcc", ind.FCC, (2, 2, 3), "L12")])
def test_closed_form_alpha(name, kind, L, rule):
    cf = closed_form(name)
    types = ordered_types(kind, L, rule)
    n_per = np.bincount(types, minlength=2)
    cnt = oracle.counts(kind, L, 3, 2, types)
    alpha, f2 = oracle.alpha_f2(kind, L, 3, n_per, np.ones(3), np.zeros((3, 2, 2)), cnt)
    np.testing.assert_allclose(alpha, np.array(cf["alpha"]), rtol=0, atol=1e-14)
    # F^2 against the zero target is the plain sum of squares of the closed form.
    assert abs(f2 - float((np.array(cf["alpha"]) ** 2).sum())) < 1e-12


@pytest.mark.parametrize("kind,L,M,S,seed", [(ind.FCC, (3, 4, 2), 5, 4, 1), (ind.BCC, (4, 3, 3), 5, 5, 2),
                                             (ind.FCC, (5, 5, 5), 3, 6, 3), (ind.BCC, (2, 2, 2), 4, 3, 4)])
def test_invariants_random_configs(kind, L, M, S, seed):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    n_per = rng.multinomial(N - S, np.ones(S) / S) + 1
    types = oracle.init_config(N, n_per, seed)
    cnt = oracle.counts(kind, L, M, S, types).astype(np.int64)
    Z = ind.SHELL_Z[kind][:M]
    for k in range(M):
        assert np.array_equal(cnt[k].sum(axis=1), n_per * Z[k])     # sum_j N_ij = N_i Z_k
        assert np.array_equal(cnt[k], cnt[k].T)                      # N_ij = N_ji
        assert cnt[k].sum() == N * Z[k]
    alpha, _ = oracle.alpha_f2(kind, L, M, n_per, np.ones(M), np.zeros((M, S, S)), cnt)
    c = n_per / N
    for k in range(M):
        np.testing.assert_allclose(alpha[k] @ c, 0.0, atol=1e-12)    # sum_j c_j alpha_ij = 0
        np.testing.assert_allclose(c @ alpha[k], 0.0, atol=1e-12)    # sum_i c_i alpha_ij = 0
        np.testing.assert_allclose(alpha[k], alpha[k].T, atol=1e-13)  # alpha_ij = alpha_ji


@pytest.mark.parametrize("kind,L,M,S", [(ind.FCC, (2, 2, 2), 5, 3), (ind.FCC, (3, 2, 2), 4, 4),
                                        (ind.BCC, (2, 2, 3), 5, 2), (ind.BCC, (3, 3, 2), 3, 5)])
def test_counts_match_independent_image_recount(kind, L, M, S):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(N * 7 + S)
    types = rng.integers(0, S, N).astype(np.uint8)
    got = oracle.counts(kind, L, M, S, types)
    want = ind.counts_by_images(kind, L, M, S, types)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kind,L,M", [(ind.FCC, (3, 3, 3), 3), (ind.BCC, (3, 2, 4), 3)])
def test_alpha_and_f2_match_equations(kind, L, M):
    N = oracle.num_sites(kind, L)
    S = 4
    rng = np.random.default_rng(5)
    n_per = rng.multinomial(N - S, np.ones(S) / S) + 1
    types = oracle.init_config(N, n_per, 11)
    cnt = oracle.counts(kind, L, M, S, types)
    w = rng.uniform(0.1, 2.0, M)
    target = rng.uniform(-0.5, 0.5, (M, S, S))
    alpha, f2 = oracle.alpha_f2(kind, L, M, n_per, w, target, cnt)
    want_alpha = ind.alpha_eq_sro(kind, L, M, n_per, cnt)
    np.testing.assert_allclose(alpha, want_alpha, rtol=0, atol=1e-13)
    assert abs(f2 - ind.f2_eq_fitness(want_alpha, target, w)) <= 1e-12 * max(1.0, f2)


def test_exhaustive_16_site_bcc_binary():
    """All C(16,8) = 12,870 arrangements of 8 A + 8 B on BCC 2x2x2."""
    kind, L, M, S = ind.BCC, (2, 2, 2), 3, 2
    N = 16
    total_ab = np.zeros(M, np.int64)
    minus_one = 0
    for ones in itertools.combinations(range(N), 8):
        types = np.zeros(N, np.uint8)
        types[list(ones)] = 1
        cnt = oracle.counts(kind, L, M, S, types)
        total_ab += cnt[:, 0, 1]
        if cnt[0, 0, 1] == 8 * 8:        # alpha_AB^(1) = 1 - N_AB * 16 / (8 * 8 * 8) = -1
            minus_one += 1
    # Every (site, vector) partner is a distinct non-self site, so each contributes in
    # C(14, 7) = 3432 arrangements: sum = 12870 * N_A * Z_k * N_B / (N - 1).
    assert list(total_ab) == [439296, 329472, 658944]
    assert minus_one == 2   # the two B2 variants


@pytest.mark.parametrize("kind,L,M,S", [(ind.FCC, (4, 5, 3), 3, 4), (ind.BCC, (6, 4, 5), 2, 5),
                                        (ind.FCC, (2, 3, 2), 5, 6), (ind.BCC, (3, 3, 4), 5, 3)])
def test_half_vectors_and_row_sums_give_the_counts(kind, L, M, S):
    """The bit-plane recount's algebra, checked on the oracle's neighbour lists: the vector -v counts
    (j, i) where v counts (i, j), so N_ij = sum over the lexicographically positive half of each
    shell's vectors of c_ij + c_ji; each row of N^(k) sums to N_i Z_k, which gives the last species."""
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(3 * M + S)
    t = rng.integers(0, S, N).astype(np.uint8)
    Z, _, vecs = oracle.shells(kind, M)
    nbr = oracle.neighbours(kind, L, M)
    pos = oracle.positions(kind, L)
    period = 2 * np.array(L)
    # the neighbour columns follow the shell vectors
    for s in (0, N // 2, N - 1):
        for v in range(len(vecs)):
            assert np.array_equal((pos[s] + vecs[v]) % period, pos[nbr[s, v]] % period)
    want = oracle.counts(kind, L, M, S, t)
    n_i = np.bincount(t, minlength=S)
    start = 0
    for k in range(M):
        vk = vecs[start:start + Z[k]]
        half = [start + v for v in range(Z[k]) if tuple(vk[v]) > (0, 0, 0)]
        assert len(half) * 2 == Z[k]
        c = np.zeros((S, S), np.int64)
        for v in half:
            np.add.at(c, (t, t[nbr[:, v]]), 1)
        got = np.zeros((S, S), np.int64)
        got[:S - 1, :S - 1] = (c + c.T)[:S - 1, :S - 1]
        for i in range(S - 1):
            got[i, S - 1] = n_i[i] * Z[k] - got[i, :S - 1].sum()
            got[S - 1, i] = got[i, S - 1]
        got[S - 1, S - 1] = n_i[S - 1] * Z[k] - got[S - 1, :S - 1].sum()
        assert np.array_equal(got, want[k]), k
        start += Z[k]
