"""Pin of the oracle's accept decision against the paper's rule (Alg. parallel_mc and
Alg. serial_mc compare fitness values: a swap improves when F(new) < F(current)).

The oracle decides on its swap key D (a binary64 FMA chain, Sec. 4.5).  Here the change of F^2 is
computed independently and exactly: counts of the swapped configuration from a periodic-image
recount (tests/independent.py), alpha from Eq. sro and F^2 from Eq. fitness_function in rational
arithmetic (targets and weights taken as the exact values of their binary64 encodings).  Whenever
the exact change clears 1e-12 F^2, the sign of D must be its sign; D must also stay within 1e-12 F^2
of it.  States include ones close to their target, where keys are small differences of large terms."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import independent as ind


def exact_f2(kind, M, n_per, cnt, target, w):
    n = [int(x) for x in n_per]
    N = sum(n)
    f2 = Fraction(0)
    for k in range(M):
        Z = ind.SHELL_Z[kind][k]
        wk = Fraction(float(w[k]))
        for i in range(len(n)):
            for j in range(len(n)):
                alpha = 1 - Fraction(int(cnt[k, i, j]) * N, Z * n[i] * n[j])
                e = alpha - Fraction(float(target[k, i, j]))
                f2 += wk * e * e
    return f2


def swapped(types, a, b):
    t = types.copy()
    t[a], t[b] = t[b], t[a]
    return t


def states():
    """(kind, L, M, n_per, types, w, target): random targets, and targets taken from a nearby
    configuration (a few swaps away) so that the current F^2 is small."""
    out = []
    for kind, L, M, S, seed in [(ind.FCC, (3, 3, 3), 3, 4, 11), (ind.BCC, (4, 4, 3), 2, 3, 12),
                                (ind.FCC, (2, 3, 3), 4, 5, 13), (ind.BCC, (3, 3, 3), 3, 4, 14)]:
        N = oracle.num_sites(kind, L)
        rng = np.random.default_rng(seed)
        n_per = rng.multinomial(N - S, np.ones(S) / S) + 1
        types = oracle.init_config(N, n_per, seed)
        w = rng.uniform(0.3, 2.0, M)
        out.append((kind, L, M, n_per, types, w, rng.uniform(-0.5, 0.5, (M, S, S))))
        near = types.copy()
        for a, b in rng.integers(0, N, (3, 2)):
            near = swapped(near, a, b)
        cnt_near = oracle.counts(kind, L, M, S, near)
        target = ind.alpha_eq_sro(kind, L, M, n_per, cnt_near) + rng.uniform(-1e-3, 1e-3, (M, S, S))
        out.append((kind, L, M, n_per, types, w, target))
    return out


@pytest.mark.parametrize("case", range(8))
def test_accept_sign_matches_exact_fitness_change(case):
    kind, L, M, n_per, types, w, target = states()[case]
    S = len(n_per)
    N = len(types)
    rng = np.random.default_rng(100 + case)
    nbr = oracle.neighbours(kind, L, M)
    pairs = [tuple(p) for p in rng.integers(0, N, (50, 2))]
    pairs += [(int(a), int(nbr[a, rng.integers(0, nbr.shape[1])])) for a in rng.integers(0, N, 30)]
    pairs = [(a, b) for a, b in pairs if a != b and types[a] != types[b]]
    cnt = oracle.counts(kind, L, M, S, types)
    key, _, null = oracle.delta_swap(kind, L, M, n_per, w, target, types, cnt, np.array(pairs, np.int64))
    f2_before = exact_f2(kind, M, n_per, ind.counts_by_images(kind, L, M, S, types), target, w)
    decided = 0
    for c, (a, b) in enumerate(pairs):
        assert not null[c]
        after = ind.counts_by_images(kind, L, M, S, swapped(types, a, b))
        diff = exact_f2(kind, M, n_per, after, target, w) - f2_before
        scale = max(float(f2_before), float(f2_before + diff), 1e-300)
        assert abs(key[c] - float(diff)) <= 1e-12 * scale, (c, key[c], float(diff))
        if abs(diff) > Fraction(1e-12) * Fraction(scale):
            decided += 1
            assert (key[c] < 0.0) == (diff < 0), (c, key[c], float(diff))
            assert (key[c] > 0.0) == (diff > 0), (c, key[c], float(diff))
    assert decided >= 0.9 * len(pairs)
