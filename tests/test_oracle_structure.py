"""Pins of the oracle's mapping of an external structure onto the lattice (Sec. 2.3, application
workflow) and CPU checks of the structure file readers.  Positions come from textbook geometry
(tests/independent.py), are shuffled, displaced, shifted by whole periods and offset; the mapping
must return the original arrangement, report every defect, and the extracted alpha must equal the
closed forms of ordered structures."""
import os

import numpy as np
import pytest

import oracle
from paper_2411_18906_gb300 import structure
from tests import independent as ind


def synthetic(kind, L, S, a, seed, noise=0.15, origin=(0.0, 0.0, 0.0)):
    """(xyz, species, true types): every site once, in random order, displaced by up to `noise`
    half units per axis, shifted by random whole periods, offset by origin."""
    rng = np.random.default_rng(seed)
    P = ind.positions(kind, L).astype(np.float64)
    N = len(P)
    types = rng.integers(0, S, N).astype(np.uint8)
    period = 2.0 * np.asarray(L)
    shift = rng.integers(-2, 3, (N, 3)) * period
    half = P + rng.uniform(-noise, noise, (N, 3)) + shift
    xyz = half * (a / 2.0) + np.asarray(origin)
    order = rng.permutation(N)
    return xyz[order], types[order], types


@pytest.mark.parametrize("kind,L,S,a", [(ind.FCC, (3, 2, 4), 4, 3.59), (ind.BCC, (4, 3, 2), 5, 2.87),
                                        (ind.FCC, (2, 2, 2), 2, 1.0), (ind.BCC, (5, 5, 5), 3, 3.3)])
def test_round_trip_identity(kind, L, S, a):
    xyz, sp, truth = synthetic(kind, L, S, a, 3, origin=(1.5, -2.25, 0.125))
    types, rep = oracle.map_structure(kind, L, S, xyz, sp, a, origin=(1.5, -2.25, 0.125), tol=0.3)
    assert rep.tolist() == [0, 0, 0, 0]
    assert np.array_equal(types, truth)


def test_defects_are_reported():
    kind, L, S, a = ind.FCC, (3, 3, 2), 3, 3.6
    xyz, sp, _ = synthetic(kind, L, S, a, 5, noise=0.05)
    xyz = xyz.copy()
    sp = sp.copy()
    xyz[0] += np.array([0.6, 0.0, 0.0]) * a / 2      # 0.6 half units off: off-lattice, its site empty
    xyz[1] = xyz[2]                                   # two atoms on one site, atom 1's site empty
    sp[3] = 7                                         # species beyond S
    _, rep = oracle.map_structure(kind, L, S, xyz, sp, a, tol=0.3)
    assert rep.tolist() == [1, 1, 2, 1]


def test_extracted_alpha_matches_closed_forms():
    """B2 (BCC A50B50 by sublattice) and L1_2 (FCC A3B, B on the cube corners)."""
    P = ind.positions(ind.BCC, (3, 3, 3))
    b2 = (P[:, 0] % 2).astype(np.uint8)
    xyz = P * 1.5
    types, rep = oracle.map_structure(ind.BCC, (3, 3, 3), 2, xyz[::-1], b2[::-1], 3.0)
    assert rep.tolist() == [0, 0, 0, 0]
    cnt = oracle.counts(ind.BCC, (3, 3, 3), 3, 2, types)
    alpha, _ = oracle.alpha_f2(ind.BCC, (3, 3, 3), 3, [27, 27], np.ones(3), np.zeros((3, 2, 2)), cnt)
    assert np.array_equal(alpha[0], [[1.0, -1.0], [-1.0, 1.0]])
    assert np.array_equal(alpha[1], [[-1.0, 1.0], [1.0, -1.0]])
    P = ind.positions(ind.FCC, (2, 2, 2))
    l12 = ((P[:, 0] % 2 == 0) & (P[:, 1] % 2 == 0) & (P[:, 2] % 2 == 0)).astype(np.uint8)   # B at corners
    types, rep = oracle.map_structure(ind.FCC, (2, 2, 2), 2, P * 2.0, l12, 4.0)
    assert rep.tolist() == [0, 0, 0, 0]
    cnt = oracle.counts(ind.FCC, (2, 2, 2), 2, 2, types)
    alpha, _ = oracle.alpha_f2(ind.FCC, (2, 2, 2), 2, [24, 8], np.ones(2), np.zeros((2, 2, 2)), cnt)
    assert abs(alpha[0, 0, 1] + 1 / 3) < 1e-15 and abs(alpha[0, 1, 0] + 1 / 3) < 1e-15
    assert abs(alpha[0, 0, 0] - 1 / 9) < 1e-15 and alpha[0, 1, 1] == 1.0
    assert abs(alpha[1, 1, 1] + 3) < 1e-15 and abs(alpha[1, 0, 1] - 1) < 1e-15


def test_lammps_and_xyz_files_round_trip(tmp_path):
    kind, L, S, a = ind.BCC, (3, 2, 2), 3, 2.9
    xyz, sp, truth = synthetic(kind, L, S, a, 9, noise=0.0)
    xyz = np.mod(xyz, np.asarray(L) * a)     # inside the box, as a simulation would write it
    st = structure.Structure(xyz, sp, np.zeros(3), np.asarray(L, np.float64) * a)
    path = os.path.join(tmp_path, "cell.data")
    structure.write_lammps_data(path, st, masses=[55.845, 54.938, 51.996])
    back = structure.read_lammps_data(path)
    assert np.array_equal(back.species, sp) and np.allclose(back.xyz, xyz, atol=1e-9)
    assert np.allclose(back.box_hi, st.box_hi)
    types, rep = oracle.map_structure(kind, L, S, back.xyz, back.species, a)
    assert rep.tolist() == [0, 0, 0, 0] and np.array_equal(types, truth)
    st.labels = ["Fe", "Mn", "Cr"]
    path = os.path.join(tmp_path, "cell.xyz")
    structure.write_xyz(path, st)
    back = structure.read_xyz(path, labels=["Fe", "Mn", "Cr"], box_hi=st.box_hi)
    assert np.array_equal(back.species, sp) and np.allclose(back.xyz, xyz, atol=1e-9)
    with open(path) as fh:
        text = fh.read()
    with open(path, "w") as fh:
        fh.write(text.replace("Fe ", "Ni "))
    with pytest.raises(ValueError):
        structure.read_xyz(path, labels=["Fe", "Mn", "Cr"])
