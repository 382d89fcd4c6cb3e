"""Writes paper_2411_18906_gb300/data/annealed_targets.json -- calls only the oracle.

The annealed-target recipe (an input generator): a ~4,000-site cell of the workload's lattice and
composition is annealed by seeded Metropolis swaps with symmetric shell-1 pair energies
eps_ij ~ U[-0.05, 0.05] eV at T = 800 K for 200 sweeps, and the Warren-Cowley alpha of the final
state for shells 1-3 (Sec. 4.3, Eq. sro) becomes the target.  The paper obtains its targets from an
external MC-MD run (Sec. 4.7); this recipe stands in for that step with synthetic pair energies.

Entries:
  fcc_4sp_40_20_20_20   FCC 10x10x10, 40/20/20/20 at.%   (the 256,000-site FCC workload's target)
  pool_<lat>_<S>sp      8 entries each for lat in {fcc, bcc}, S in 3..6, compositions drawn from
                        Dirichlet(5) clipped to 5-35 at.% (the batched and served workloads)

Run:  python -m oracle.make_annealed_targets
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2411_18906_gb300 import workloads  # noqa: E402

OUT = os.path.join(os.path.dirname(HERE), "paper_2411_18906_gb300", "data", "annealed_targets.json")

CELL = {workloads.FCC: (10, 10, 10), workloads.BCC: (13, 13, 12)}
T_KELVIN = 800.0
SWEEPS = 200
M_OUT = 3
POOL_PER_KEY = 8


def anneal_entry(kind, fractions, seed):
    L = CELL[kind]
    N = oracle.num_sites(kind, L)
    n_per = workloads.composition_counts(N, fractions)
    types, eps, alpha, taken = oracle.anneal(kind, L, n_per, seed, T=T_KELVIN, sweeps=SWEEPS, M_out=M_OUT)
    return {
        "kind": "fcc" if kind == workloads.FCC else "bcc",
        "cell": list(L),
        "n_per": n_per,
        "fractions": [float(x) for x in fractions],
        "seed": seed,
        "T": T_KELVIN,
        "sweeps": SWEEPS,
        "accepted_moves": taken,
        "eps": eps.tolist(),
        "alpha": alpha.tolist(),
    }


def main():
    out = {"_recipe": __doc__.strip().splitlines()[0],
           "_command": "python -m oracle.make_annealed_targets"}
    out["fcc_4sp_40_20_20_20"] = anneal_entry(workloads.FCC, [0.4, 0.2, 0.2, 0.2], seed=7)
    rng = np.random.default_rng(2411)
    for kind in (workloads.FCC, workloads.BCC):
        for S in (3, 4, 5, 6):
            key = f"pool_{'fcc' if kind == workloads.FCC else 'bcc'}_{S}sp"
            entries = []
            for e in range(POOL_PER_KEY):
                frac = workloads.dirichlet_composition(rng, S)
                entries.append(anneal_entry(kind, frac, seed=100 * S + 10 * kind + e + 1))
                print(key, e, flush=True)
            out[key] = entries
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
