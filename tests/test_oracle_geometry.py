"""Pins for the oracle's lattice geometry: textbook coordination numbers and radii, the index
layout, and neighbours checked against an independent periodic-image search."""
import numpy as np
import pytest

import oracle
from tests import independent as ind


@pytest.mark.parametrize("kind", [ind.FCC, ind.BCC])
def test_shell_coordination_numbers_and_radii(kind):
    Z, r2, vecs = oracle.shells(kind, 5)
    assert list(Z) == ind.SHELL_Z[kind]
    assert list(r2) == ind.SHELL_R2[kind]
    start = 0
    for k in range(5):
        v = vecs[start:start + Z[k]]
        start += Z[k]
        assert np.all((v * v).sum(axis=1) == r2[k])
        # Shells are centrosymmetric: -d is in the shell whenever d is.
        assert {tuple(x) for x in v} == {tuple(-x) for x in v}
        # Lexicographic order inside the shell.
        assert [tuple(x) for x in v] == sorted(tuple(x) for x in v)


@pytest.mark.parametrize("kind,L", [(ind.FCC, (2, 3, 4)), (ind.BCC, (3, 2, 5)), (ind.FCC, (5, 4, 3))])
def test_positions_follow_documented_layout(kind, L):
    pos = oracle.positions(kind, L)
    assert np.array_equal(pos, ind.positions(kind, L))
    assert len({tuple(p) for p in pos}) == len(pos)


@pytest.mark.parametrize("kind,L,M", [(ind.FCC, (2, 2, 2), 5), (ind.FCC, (3, 2, 4), 5),
                                      (ind.BCC, (2, 2, 2), 5), (ind.BCC, (3, 4, 2), 5)])
def test_neighbours_match_periodic_image_search(kind, L, M):
    nbr = oracle.neighbours(kind, L, M)
    Z, _, _ = oracle.shells(kind, M)
    mult = ind.shell_multiplicity(kind, L, M)
    N = nbr.shape[0]
    start = 0
    for k in range(M):
        block = nbr[:, start:start + Z[k]]
        start += Z[k]
        got = np.zeros((N, N), np.int64)
        for s in range(N):
            for t in block[s]:
                got[s, t] += 1
        assert np.array_equal(got, mult[k]), f"shell {k + 1}"
    # No site is its own neighbour for L >= 2 (shell radii up to 5 fit inside the period).
    assert not np.any(nbr == np.arange(N)[:, None])
