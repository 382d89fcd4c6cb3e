"""Pins for the oracle's incremental swap delta (Sec. 4.5) and swap key: N + dN equals a full
recount of the swapped configuration (including a-b bonds and small periodic cells where b is
reached by several vectors), and the key equals the change of F^2 computed from scratch."""
import numpy as np
import pytest

import oracle
from tests import independent as ind


def random_state(kind, L, M, S, seed):
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(seed)
    n_per = rng.multinomial(N - S, np.ones(S) / S) + 1
    types = oracle.init_config(N, n_per, seed)
    w = rng.uniform(0.2, 2.0, M)
    target = rng.uniform(-0.4, 0.4, (M, S, S))
    return N, n_per, types, w, target, rng


def pair_list(kind, L, M, N, rng, n_random=60):
    nbr = oracle.neighbours(kind, L, M)
    pairs = [(a, b) for a, b in rng.integers(0, N, (n_random, 2))]
    for _ in range(n_random):                      # neighbours: a-b bonds in every shell
        a = int(rng.integers(0, N))
        pairs.append((a, int(nbr[a, rng.integers(0, nbr.shape[1])])))
    pairs += [(3, 3), (0, N - 1)]
    return np.array(pairs, np.int64)


@pytest.mark.parametrize("kind,L,M,S,seed", [(ind.FCC, (2, 2, 2), 5, 3, 1), (ind.FCC, (3, 4, 3), 3, 4, 2),
                                             (ind.BCC, (2, 2, 2), 5, 4, 3), (ind.BCC, (4, 3, 5), 2, 5, 4),
                                             (ind.FCC, (2, 3, 2), 4, 6, 5)])
def test_delta_equals_full_recount(kind, L, M, S, seed):
    N, n_per, types, w, target, rng = random_state(kind, L, M, S, seed)
    cnt = oracle.counts(kind, L, M, S, types)
    pairs = pair_list(kind, L, M, N, rng)
    key, dN, null = oracle.delta_swap(kind, L, M, n_per, w, target, types, cnt, pairs)
    _, f2_before = oracle.alpha_f2(kind, L, M, n_per, w, target, cnt)
    for c, (a, b) in enumerate(pairs):
        t2 = types.copy()
        t2[a], t2[b] = t2[b], t2[a]
        after = oracle.counts(kind, L, M, S, t2)
        assert np.array_equal(cnt + dN[c], after), (c, a, b)
        for k in range(M):
            assert np.array_equal(dN[c][k], dN[c][k].T)
        assert null[c] == (a == b or types[a] == types[b])
        if null[c]:
            assert key[c] == 0.0 and not np.signbit(key[c])
            continue
        # Key against the change of F^2 from two independent full evaluations (Eq. fitness_function).
        f2_after = ind.f2_eq_fitness(ind.alpha_eq_sro(kind, L, M, n_per, after), target, w)
        f2_prev = ind.f2_eq_fitness(ind.alpha_eq_sro(kind, L, M, n_per, cnt), target, w)
        scale = max(f2_after, f2_prev, 1e-300)
        assert abs(key[c] - (f2_after - f2_prev)) <= 1e-12 * scale
        _, f2_o = oracle.alpha_f2(kind, L, M, n_per, w, target, after)
        assert abs(key[c] - (f2_o - f2_before)) <= 1e-12 * scale


def test_delta_matches_g_vector_rule_on_a_bond():
    """dN[A][A] = 2 g[A], dN[B][B] = -2 g[B], dN[A][B] = g[B] - g[A] with g = h_b - h_a (bond a-b
    excluded), checked by counting h_a and h_b directly from the neighbour table."""
    kind, L, M, S = ind.FCC, (3, 3, 3), 3, 3
    N = oracle.num_sites(kind, L)
    types = oracle.init_config(N, [36, 36, 36], 9)
    nbr = oracle.neighbours(kind, L, M)
    Z, _, _ = oracle.shells(kind, M)
    cnt = oracle.counts(kind, L, M, S, types)
    for a in range(0, N, 7):
        b = int(nbr[a, 0])                      # a shell-1 neighbour of a
        A, B = int(types[a]), int(types[b])
        if A == B:
            continue
        _, dN, _ = oracle.delta_swap(kind, L, M, [36, 36, 36], np.ones(M), np.zeros((M, S, S)), types, cnt,
                                     np.array([[a, b]]))
        start = 0
        for k in range(M):
            cols = slice(start, start + Z[k])
            start += Z[k]
            ha = np.bincount([types[t] for t in nbr[a, cols] if t != b], minlength=S)
            hb = np.bincount([types[t] for t in nbr[b, cols] if t != a], minlength=S)
            g = hb - ha
            assert g.sum() == (Z[k] - np.sum(nbr[b, cols] == a)) - (Z[k] - np.sum(nbr[a, cols] == b))
            assert dN[0, k, A, A] == 2 * g[A]
            assert dN[0, k, B, B] == -2 * g[B]
            assert dN[0, k, A, B] == g[B] - g[A] == dN[0, k, B, A]


def test_symmetric_screen_covers_every_changed_entry():
    """The symmetric FP32 screen adds (A, A), (B, B), 2 (A, B) and 2 (A, y), 2 (B, y) for the other
    species y: with symmetric coefficients this equals the sum over every ordered entry of
    dN (a dN + b), exactly (rational arithmetic), because the count changes of a swap are symmetric
    and vanish outside rows and columns A and B."""
    from fractions import Fraction
    kind, L, M, S = ind.FCC, (3, 4, 3), 3, 4
    N = oracle.num_sites(kind, L)
    rng = np.random.default_rng(17)
    t = rng.integers(0, S, N).astype(np.uint8)
    n_per = np.bincount(t, minlength=S)
    cnt = oracle.counts(kind, L, M, S, t)
    pairs = rng.integers(0, N, (200, 2))
    _, dN, null = oracle.delta_swap(kind, L, M, n_per, np.ones(M), np.zeros((M, S, S)), t, cnt, pairs)
    a = [[[Fraction(int(x), 97) for x in row] for row in rng.integers(1, 50, (S, S))] for _ in range(M)]
    b = [[[Fraction(int(x), 89) for x in row] for row in rng.integers(-40, 40, (S, S))] for _ in range(M)]
    for k in range(M):
        for i in range(S):
            for j in range(i):
                a[k][i][j] = a[k][j][i]
                b[k][i][j] = b[k][j][i]
    term = lambda k, i, j: dN_k[i, j] * (a[k][i][j] * dN_k[i, j] + b[k][i][j])
    checked = 0
    for p in range(len(pairs)):
        if null[p]:
            continue
        A, B = int(t[pairs[p, 0]]), int(t[pairs[p, 1]])
        full = half = Fraction(0)
        for k in range(M):
            dN_k = dN[p, k].astype(np.int64)
            assert np.array_equal(dN_k, dN_k.T)
            full += sum(term(k, i, j) for i in range(S) for j in range(S))
            half += term(k, A, A) + term(k, B, B) + 2 * term(k, A, B)
            half += sum(2 * (term(k, A, y) + term(k, B, y)) for y in range(S) if y not in (A, B))
        assert full == half
        checked += 1
    assert checked > 100
