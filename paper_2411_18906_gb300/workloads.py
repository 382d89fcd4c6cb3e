"""Seeded synthetic workload generators shared by the tests and the benchmark.

This module holds the input recipes only: lattice sizes, integer compositions, weights, seeds,
request mixes.  It contains none of the method's arithmetic (no counting, no SRO, no objective,
no random-swap draws); those live in the CUDA library and, independently, in the CPU oracle.

The workloads mirror the paper's benchmark shapes (Table 1: FCC/BCC supercells S = A * L^3 with
three coordination shells) at the sizes used for measurement.
"""
from dataclasses import dataclass, field
import json
import math
import os
from typing import List, Optional

import numpy as np

FCC, BCC = 0, 1
BASIS_SITES = {FCC: 4, BCC: 2}
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def composition_counts(N: int, fractions) -> List[int]:
    """Integer species counts summing to N, by the largest-remainder rule (ties to lower index)."""
    f = np.asarray(fractions, dtype=np.float64)
    f = f / f.sum()
    raw = f * N
    base = np.floor(raw).astype(np.int64)
    rem = raw - base
    short = N - int(base.sum())
    order = sorted(range(len(f)), key=lambda i: (-rem[i], i))
    for i in order[:short]:
        base[i] += 1
    return [int(x) for x in base]


def equiatomic(N: int, S: int) -> List[int]:
    return composition_counts(N, [1.0] * S)


@dataclass
class CellSpec:
    kind: int
    L: tuple
    M: int
    n_per: List[int]
    seed: int
    target: Optional[np.ndarray] = None   # [M][S][S]; None = all zero
    w: Optional[np.ndarray] = None        # [M]; None = all one

    @property
    def S(self) -> int:
        return len(self.n_per)

    @property
    def N(self) -> int:
        return BASIS_SITES[self.kind] * self.L[0] * self.L[1] * self.L[2]

    def weights(self) -> np.ndarray:
        return np.ones(self.M) if self.w is None else np.asarray(self.w, np.float64)

    def targets(self) -> np.ndarray:
        if self.target is None:
            return np.zeros((self.M, self.S, self.S))
        return np.asarray(self.target, np.float64).reshape(self.M, self.S, self.S)


def fcc_256():
    """FCC 4x4x4 (256 sites), 4 species equiatomic, shells 1-3, target 0, unit weights."""
    return CellSpec(FCC, (4, 4, 4), 3, equiatomic(256, 4), seed=1)


def bcc_16k(seed: int = 1):
    """BCC 20x20x20 (16,000 sites), 5 species equiatomic, shells 1-2, target 0."""
    return CellSpec(BCC, (20, 20, 20), 2, equiatomic(16000, 5), seed=seed)


def annealed_targets():
    """Stored annealed target SRO matrices (written by oracle/make_annealed_targets.py)."""
    path = os.path.join(DATA_DIR, "annealed_targets.json")
    with open(path) as fh:
        return json.load(fh)


def fcc_256k():
    """FCC 40x40x40 (256,000 sites), 40/20/20/20 at.%, shells 1-3, annealed nonzero target."""
    n_per = composition_counts(256000, [0.4, 0.2, 0.2, 0.2])
    entry = annealed_targets()["fcc_4sp_40_20_20_20"]
    return CellSpec(FCC, (40, 40, 40), 3, n_per, seed=1, target=np.array(entry["alpha"]))


def lattice_dims_for(kind: int, n_target: float, rng: np.random.Generator):
    """Lx, Ly, Lz >= 2 whose site count A*Lx*Ly*Lz is nearest to n_target (non-cubic allowed)."""
    A = BASIS_SITES[kind]
    cells = max(8.0, n_target / A)
    best = None
    base = max(2, int(round(cells ** (1.0 / 3.0))))
    for lx in range(max(2, base - 3), base + 4):
        for ly in range(max(2, base - 3), base + 4):
            lz = max(2, int(round(cells / (lx * ly))))
            for z in (lz - 1, lz, lz + 1):
                if z < 2:
                    continue
                err = abs(A * lx * ly * z - n_target)
                key = (err, abs(lx - ly) + abs(ly - z), lx, ly, z)
                if best is None or key < best:
                    best = key
    _, _, lx, ly, lz = best
    dims = [lx, ly, lz]
    rng.shuffle(dims)
    return tuple(int(d) for d in dims)


def dirichlet_composition(rng: np.random.Generator, S: int, lo=0.05, hi=0.35, alpha=5.0):
    """Dirichlet(alpha * 1) fractions, rejection-sampled until every fraction lies in [lo, hi]."""
    if S * hi < 1.0 - 1e-12:
        raise ValueError("no composition fits the clip")
    while True:
        f = rng.dirichlet([alpha] * S)
        if f.min() >= lo and f.max() <= hi:
            return f


def batch_cells(n_cells: int = 512, seed: int = 1, n_lo: float = 500, n_hi: float = 32000,
                target_pool=None):
    """The batched workload: independent cells, lattice FCC or BCC at random, sizes log-uniform,
    3-6 species, Dirichlet(5) compositions clipped to 5-35 at.%, 1-3 shells.  Targets are drawn
    from the stored annealed pool entry matching (lattice, species count)."""
    rng = np.random.default_rng(seed)
    pool = annealed_targets() if target_pool is None else target_pool
    cells = []
    for c in range(n_cells):
        kind = int(rng.integers(0, 2))
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        L = lattice_dims_for(kind, n_target, rng)
        S = int(rng.integers(3, 7))
        M = int(rng.integers(1, 4))
        N = BASIS_SITES[kind] * L[0] * L[1] * L[2]
        key = f"pool_{'fcc' if kind == FCC else 'bcc'}_{S}sp"
        entries = pool[key]
        entry = entries[int(rng.integers(0, len(entries)))]
        n_per = composition_counts(N, entry["fractions"])
        target = np.array(entry["alpha"])[:M]
        cells.append(CellSpec(kind, L, M, n_per, seed=1000 + c, target=target))
    return cells


# Global-search parameter presets (Sec. 2.1, parameter optimization): solutions, global
# iterations, tasks (candidate swaps per Monte Carlo step) and search depth.
GLOBAL_PRESETS = {
    "precision": dict(n_solutions=128, iterations=10, tasks=256, depth_limit=10),
    "performance": dict(n_solutions=64, iterations=6, tasks=64, depth_limit=8),
}
