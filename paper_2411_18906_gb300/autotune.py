"""Autotuner for the batched search: picks the candidates-per-step K and the threads per CTA of
each cell-size bucket.

For a fixed trial budget per cell, K trades steps (each with a fixed barrier/accept cost) against
per-step work, and the CTA's thread count trades parallel scoring against the per-step
synchronisation; the best pair depends on the cell size and the GPU.  The tuner times
hea_search_batch on a sample of the workload's cells for every (K, threads) pair of a candidate
grid, per size bucket, skipping pairs whose candidate slots do not fit shared memory, and keeps the
pair with the highest trials/s.  The report says whether the chosen K lies strictly inside the
feasible K range (bracketed).  Results are cached per (GPU name, budget, grid) in a JSON file.
"""
import json
import os
import time

import numpy as np

from . import hea

CANDIDATE_K = (128, 256, 512, 1024, 2048, 3072, 4096)
CANDIDATE_THREADS = (128, 256, 512)
BUCKETS = ((0, 4000), (4000, 12000), (12000, 1 << 30))   # sites


def bucket_of(n_sites: int) -> int:
    for b, (lo, hi) in enumerate(BUCKETS):
        if lo <= n_sites < hi:
            return b
    return len(BUCKETS) - 1


def _cache_path():
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "hea_gb300_autotune.json")


def _time_batch(torch, cells, K, trials, accept_mode, threads=0, repeats=2):
    """Seconds of one hea_search_batch over `cells` (list of (Lattice, Objective, types, counts));
    None when the candidate slots do not fit a CTA's shared memory."""
    n = len(cells)
    params = [hea.search_params(K, max(1, trials // K), accept_mode=accept_mode, seed=7 + i, threads=threads)
              for i in range(n)]
    res = torch.zeros(n * hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    best = None
    for _ in range(repeats):
        ts = [t.clone() for _, _, t, _ in cells]
        cs = [c.clone() for _, _, _, c in cells]
        try:
            plan = hea.BatchPlan([l for l, _, _, _ in cells], [o for _, o, _, _ in cells], params, ts, cs, res)
        except hea.HeaError as e:
            if e.status == hea.HEA_ENOMEM:
                return None
            raise
        plan_dev = torch.from_numpy(plan.host).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hea.hea_search_batch(plan.host, plan_dev)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best


def _fits(torch, cells, K, threads, trials, accept_mode):
    """True when a batch plan of `cells` with K candidates and `threads` per CTA fits shared memory
    (planned on the host; nothing is launched)."""
    params = [hea.search_params(K, max(1, trials // K), accept_mode=accept_mode, seed=1, threads=threads)
              for _ in cells]
    res = torch.zeros(len(cells) * hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    try:
        hea.BatchPlan([l for l, _, _, _ in cells], [o for _, o, _, _ in cells], params, [t for _, _, t, _ in cells],
                      [c for _, _, _, c in cells], res)
    except hea.HeaError as e:
        if e.status == hea.HEA_ENOMEM:
            return False
        raise
    return True


def tune(cells, trials: int, accept_mode: int = 0, sample: int = 48, use_cache: bool = True):
    """cells: list of (Lattice, Objective, types tensor, counts tensor).  Returns
    ({bucket: (K, threads)}, report)."""
    import torch
    gpu = torch.cuda.get_device_name(0)
    key = f"v4|{gpu}|{trials}|{accept_mode}|{len(cells)}|{CANDIDATE_K}|{CANDIDATE_THREADS}"
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        return {int(b): tuple(k) for b, k in cache[key]["choice"].items()}, cache[key]["report"]
    by_bucket = {}
    for cell in cells:
        by_bucket.setdefault(bucket_of(cell[0].N), []).append(cell)
    rng = np.random.default_rng(0)
    choice, report = {}, {}
    for b, members in sorted(by_bucket.items()):
        pick = [members[i] for i in rng.choice(len(members), size=min(sample, len(members)), replace=False)]
        rates = {}
        for K in CANDIDATE_K:
            for threads in CANDIDATE_THREADS:
                dt = _time_batch(torch, pick, K, trials, accept_mode, threads)
                if dt is not None:
                    rates[(K, threads)] = len(pick) * (trials // K) * K / dt
        # the fastest pair on the sample whose candidate slots fit every cell of the bucket
        best = None
        for pair in sorted(rates, key=rates.get, reverse=True):
            if _fits(torch, members, pair[0], pair[1], trials, accept_mode):
                best = pair
                break
        if best is None:
            raise RuntimeError(f"no candidate (K, threads) fits every cell of size bucket {b}")
        feasible = sorted({k for k, _ in rates})
        choice[b] = best
        report[str(b)] = {"sites": list(BUCKETS[b]), "cells_sampled": len(pick),
                          "trials_per_s": {f"{k}x{t}": v for (k, t), v in rates.items()},
                          "K": best[0], "threads": best[1], "K_tested": feasible,
                          "bracketed": feasible[0] < best[0] < feasible[-1],
                          # the grid goes on past the chosen K, but no larger K fits a CTA's shared memory
                          "at_shared_memory_limit": best[0] == feasible[-1] and max(CANDIDATE_K) > feasible[-1]}
    if use_cache:
        cache[key] = {"choice": {str(b): list(k) for b, k in choice.items()}, "report": report}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return choice, report
