"""GPU parity of hea_map_structure (Sec. 2.3, application workflow) against the oracle's
nearest-site mapping on the same synthetic structures (arrangement and defect report bit for bit),
and the target SRO extracted from a structure file end to end."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2411_18906_gb300 import hea, structure, workloads
from tests import gpu_util as G
from tests.test_oracle_structure import synthetic

pytestmark = pytest.mark.gpu

FCC, BCC = workloads.FCC, workloads.BCC


def gpu_map(kind, L, S, xyz, sp, a, origin=(0.0, 0.0, 0.0), tol=0.25):
    G.ensure_built()
    lat = hea.Lattice(kind, L, 1)
    types = torch.full((lat.N,), 99, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(lat.N, dtype=torch.int32, device="cuda")
    report = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    hea.hea_map_structure(lat, len(sp), G.dev(np.asarray(xyz, np.float64)), G.dev(np.asarray(sp, np.uint8)), S, a,
                          origin, tol, types, scratch, report)
    torch.cuda.synchronize()
    return types.cpu().numpy(), report.cpu().numpy()


@pytest.mark.parametrize("kind,L,S,a,seed", [(FCC, (3, 2, 4), 4, 3.59, 1), (BCC, (4, 3, 2), 5, 2.87, 2),
                                             (FCC, (10, 10, 10), 5, 3.6, 3), (BCC, (20, 20, 20), 5, 2.9, 4),
                                             (FCC, (7, 3, 2), 8, 1.0, 5)])
def test_map_matches_oracle(kind, L, S, a, seed):
    origin = (0.75, -1.0, 3.5)
    xyz, sp, truth = synthetic(kind, L, S, a, seed, origin=origin)
    got = gpu_map(kind, L, S, xyz, sp, a, origin, 0.3)
    want = oracle.map_structure(kind, L, S, xyz, sp, a, origin=origin, tol=0.3)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert np.array_equal(got[0], truth) and got[1].tolist() == [0, 0, 0, 0]


def test_defects_match_oracle():
    kind, L, S, a = FCC, (3, 3, 2), 3, 3.6
    xyz, sp, _ = synthetic(kind, L, S, a, 5, noise=0.05)
    xyz, sp = xyz.copy(), sp.copy()
    xyz[0] += np.array([0.6, 0.0, 0.0]) * a / 2
    xyz[1] = xyz[2]
    sp[1] = sp[2]          # which of two atoms on one site writes last is not fixed: make them alike
    sp[3] = 7
    xyz[4] = np.nan
    xyz[5, 2] = 1e12
    got = gpu_map(kind, L, S, xyz, sp, a, tol=0.3)
    assert got[1].tolist() == [3, 1, 4, 1]
    # the oracle has no NaN / far-away rule: compare on the defects it shares
    keep = np.ones(len(sp), bool)
    keep[[4, 5]] = False
    want = oracle.map_structure(kind, L, S, xyz[keep], sp[keep], a, tol=0.3)
    assert want[1].tolist() == [1, 1, 4, 1]
    assert np.array_equal(got[0], want[0])


def test_full_size_round_trip():
    spec = workloads.fcc_256k()
    xyz, sp, truth = synthetic(spec.kind, spec.L, spec.S, 3.6, 7, noise=0.14)   # |d| < 0.25
    got = gpu_map(spec.kind, spec.L, spec.S, xyz, sp, 3.6)
    assert got[1].tolist() == [0, 0, 0, 0] and np.array_equal(got[0], truth)


def test_target_from_lammps_file(tmp_path):
    """Structure file -> lattice -> counts -> alpha, against the oracle on the known arrangement."""
    kind, L, M, a = FCC, (5, 5, 5), 3, 3.59
    N = 4 * 125
    n_per = [200, 200, 50, 50]
    truth = oracle.init_config(N, n_per, 17)
    P = oracle.positions(kind, L)
    rng = np.random.default_rng(2)
    xyz = np.mod(P * a / 2 + rng.uniform(-0.05, 0.05, (N, 3)), np.asarray(L) * a)
    order = rng.permutation(N)
    st = structure.Structure(xyz[order], truth[order], np.zeros(3), np.asarray(L, np.float64) * a)
    path = os.path.join(tmp_path, "fe_mn_cr_co.data")
    structure.write_lammps_data(path, st)
    G.ensure_built()
    lat = hea.Lattice(kind, L, M)
    alpha, counts, comp = structure.target_from_structure(structure.read_lammps_data(path), lat)
    cnt = oracle.counts(kind, L, M, 4, truth)
    want, _ = oracle.alpha_f2(kind, L, M, n_per, np.ones(M), np.zeros((M, 4, 4)), cnt)
    assert comp == n_per and np.array_equal(counts, cnt) and np.array_equal(alpha, want)
