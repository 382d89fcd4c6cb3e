"""Continuous-batching request server for structure generation on one GPU.

A request asks for a configuration of a given lattice, size, composition and target SRO.  The
server admits requests as they arrive, as long as a stream slot is free and the device memory
they need fits the HBM budget; every admitted request runs the whole hot path on its own CUDA
stream (initial configuration, full recount, search) through libhea, so requests that arrive
while others are on the GPU start at once and overlap with them on the device.  State (species,
counts, result) stays device-resident; only the small search result is copied back.  Each
request's randomness depends only on its own seed, so its result is the same alone and in any mix.

Latency = result ready on the host - arrival time.  Completion is detected by polling CUDA events.
"""
from dataclasses import dataclass, field
import math
import time
from typing import Dict, List, Optional

import numpy as np

from . import hea, workloads


@dataclass
class Request:
    rid: int
    arrival: float               # seconds from the start of the run
    cell: workloads.CellSpec
    K: int = 256
    max_trials: int = 1_000_000
    depth_limit: int = 10
    accept_mode: int = 0
    seed: int = 1

    def device_bytes(self) -> int:
        S, M = self.cell.S, self.cell.M
        return self.cell.N + 4 * M * S * S + hea.RESULT_BYTES + 1024


@dataclass
class Completed:
    rid: int
    arrival: float
    admitted: float
    done: float
    result: dict
    types: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _Slot:
    def __init__(self, torch, device):
        self.stream = torch.cuda.Stream(device=device)
        self.event = torch.cuda.Event()
        self.request = None
        self.buffers = None
        self.admitted = 0.0


class Server:
    """Admits requests by free slots and an HBM budget; runs each on its own stream."""

    def __init__(self, hbm_budget_bytes: int = 8 << 30, slots: int = 64, device: int = 0, keep_types=False):
        import torch
        self.torch = torch
        self.device = device
        self.budget = int(hbm_budget_bytes)
        self.reserved = 0
        self.keep_types = keep_types
        self.max_reserved = 0
        self.max_inflight = 0
        self.slots = [_Slot(torch, device) for _ in range(slots)]
        self._lat: Dict[tuple, hea.Lattice] = {}

    def _lattice(self, cell):
        key = (cell.kind, tuple(cell.L), cell.M)
        if key not in self._lat:
            self._lat[key] = hea.Lattice(cell.kind, cell.L, cell.M)
        return self._lat[key]

    def _launch(self, slot: _Slot, req: Request):
        torch = self.torch
        cell = req.cell
        lat = self._lattice(cell)
        obj = hea.Objective(cell.n_per, cell.weights(), cell.targets())
        with torch.cuda.stream(slot.stream):
            types = torch.empty(cell.N, dtype=torch.uint8, device=self.device)
            counts = torch.empty((cell.M, cell.S, cell.S), dtype=torch.int32, device=self.device)
            res = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device=self.device)
        steps = max(1, req.max_trials // req.K)
        params = hea.search_params(req.K, steps, accept_mode=req.accept_mode, depth_limit=req.depth_limit,
                                   seed=req.seed)
        s = slot.stream
        hea.hea_init_config(lat, cell.n_per, cell.seed, types, s)
        hea.hea_sro_counts(lat, 1, types, cell.S, counts, s)
        hea.hea_search(lat, obj, params, types, counts, res, s)
        host = torch.empty(hea.RESULT_BYTES, dtype=torch.uint8).pin_memory()
        with torch.cuda.stream(s):
            host.copy_(res, non_blocking=True)
        slot.event.record(s)
        slot.request = req
        slot.buffers = (types, counts, res, host, obj)

    def run(self, requests: List[Request], poll_s: float = 2e-5) -> List[Completed]:
        """Serves `requests` (their arrival times in seconds from now) and returns completions."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if r.device_bytes() > self.budget:
                raise ValueError(f"request {r.rid} needs more device memory than the whole budget")
        waiting: List[Request] = []
        done: List[Completed] = []
        t0 = time.perf_counter()
        i = 0
        while len(done) < len(requests):
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= now:
                waiting.append(pending[i])
                i += 1
            # Completions free slots and memory.
            for slot in self.slots:
                if slot.request is not None and slot.event.query():
                    req = slot.request
                    types, counts, res, host, _ = slot.buffers
                    t_done = time.perf_counter() - t0
                    result = hea.decode_results(host.numpy())[0]
                    done.append(Completed(req.rid, req.arrival, slot.admitted, t_done, result,
                                          types.cpu().numpy() if self.keep_types else None))
                    self.reserved -= req.device_bytes()
                    slot.request = None
                    slot.buffers = None
            # Admission: first come, first served, while a slot is free and the budget allows.
            while waiting:
                req = waiting[0]
                free = next((s for s in self.slots if s.request is None), None)
                if free is None or self.reserved + req.device_bytes() > self.budget:
                    break
                waiting.pop(0)
                self.reserved += req.device_bytes()
                self.max_reserved = max(self.max_reserved, self.reserved)
                self.max_inflight = max(self.max_inflight, 1 + sum(s.request is not None for s in self.slots))
                free.admitted = time.perf_counter() - t0
                self._launch(free, req)
            if i < len(pending) and not waiting and all(s.request is None for s in self.slots):
                # Idle: sleep until the next arrival.
                delay = pending[i].arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(min(delay, 0.01))
            else:
                time.sleep(poll_s)
        return sorted(done, key=lambda c: c.rid)


def poisson_requests(n: int, rate_per_s: float = 50.0, seed: int = 1, n_lo: float = 1000, n_hi: float = 256000,
                     frac_max: float = 0.2, pool=None) -> List[Request]:
    """The served workload: Poisson arrivals, sizes log-uniform in [n_lo, n_hi] atoms with a
    fraction frac_max at exactly n_hi (FCC 40^3), FCC/BCC at random, 4-5 species, targets from
    the stored annealed pool; K = 256, depth limit 10, at most 1e6 trials per request."""
    rng = np.random.default_rng(seed)
    pool = workloads.annealed_targets() if pool is None else pool
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        kind = int(rng.integers(0, 2))
        S = int(rng.integers(4, 6))
        if rng.random() < frac_max:
            kind, L = workloads.FCC, (40, 40, 40)
        else:
            n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
            L = workloads.lattice_dims_for(kind, n_target, rng)
        N = workloads.BASIS_SITES[kind] * L[0] * L[1] * L[2]
        key = f"pool_{'fcc' if kind == workloads.FCC else 'bcc'}_{S}sp"
        entry = pool[key][int(rng.integers(0, len(pool[key])))]
        n_per = workloads.composition_counts(N, entry["fractions"])
        cell = workloads.CellSpec(kind, L, 3, n_per, seed=10_000 + rid, target=np.array(entry["alpha"]))
        out.append(Request(rid, t, cell, seed=20_000 + rid))
    return out


def latency_summary(done: List[Completed]) -> dict:
    lat = np.array([c.latency for c in done])
    wall = max(c.done for c in done) - min(c.arrival for c in done)
    trials = sum(c.result["trials"] for c in done)
    return {"requests": len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()), "requests_per_s": len(done) / wall,
            "trials_per_s": trials / wall}


def _run_alone(torch, req: Request, lat_cache: dict, coop_ctas: int = 0):
    """One request on the current stream, device-timed (ms): init, recount, search.  With coop_ctas
    the search runs as one cooperative chain over that many CTAs (best-of-K only)."""
    cell = req.cell
    key = (cell.kind, tuple(cell.L), cell.M)
    if key not in lat_cache:
        lat_cache[key] = hea.Lattice(cell.kind, cell.L, cell.M)
    lat = lat_cache[key]
    obj = hea.Objective(cell.n_per, cell.weights(), cell.targets())
    types = torch.empty(cell.N, dtype=torch.uint8, device="cuda")
    counts = torch.empty((cell.M, cell.S, cell.S), dtype=torch.int32, device="cuda")
    res = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    params = hea.search_params(req.K, max(1, req.max_trials // req.K), accept_mode=req.accept_mode,
                               depth_limit=req.depth_limit, seed=req.seed)
    ws = torch.zeros(hea.hea_search_coop_workspace_bytes(coop_ctas), dtype=torch.uint8, device="cuda") \
        if coop_ctas else None
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hea.hea_init_config(lat, cell.n_per, cell.seed, types)
    hea.hea_sro_counts(lat, 1, types, cell.S, counts)
    if coop_ctas:
        hea.hea_search_coop(lat, obj, params, coop_ctas, types, counts, res, ws)
    else:
        hea.hea_search(lat, obj, params, types, counts, res)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1), hea.decode_results(res.cpu().numpy())[0], types


def sequential_baseline(requests: List[Request]) -> dict:
    """The same requests served one at a time by single chains, first come first served: each
    request's device time alone, then the FIFO latencies those service times give under the same
    arrival times."""
    import torch
    cache = {}
    service = []
    for req in sorted(requests, key=lambda r: r.arrival):
        ms, _, _ = _run_alone(torch, req, cache)
        service.append((req.arrival, ms / 1e3))
    free_at = 0.0
    lat = []
    for arrival, s in service:
        start = max(arrival, free_at)
        free_at = start + s
        lat.append(free_at - arrival)
    lat = np.array(lat)
    svc = np.array([s for _, s in service])
    wall = free_at - service[0][0]
    return {"requests": len(service), "mean_service_s": float(svc.mean()), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "requests_per_s": len(service) / wall,
            "utilisation_at_arrival_rate": float(svc.sum() / (service[-1][0] - service[0][0]))}


def coop_vs_single(requests: List[Request], ctas: int = 128) -> dict:
    """The first 256,000-site request alone: single-CTA chain vs one cooperative chain over `ctas`
    CTAs (K = 256 splits into ctas slices of K / ctas candidates; identical results)."""
    import torch
    req = next((r for r in requests if r.cell.N == 256000), None)
    if req is None or req.K % ctas != 0:
        return {"skipped": "no 256k request or K not a multiple of the CTA count"}
    cache = {}
    ms1, r1, t1 = _run_alone(torch, req, cache)
    ms2, r2, t2 = _run_alone(torch, req, cache, coop_ctas=ctas)
    return {"rid": req.rid, "K": req.K, "single_cta_ms": ms1, "coop_ms": ms2, "coop_ctas": ctas,
            "identical": bool(torch.equal(t1, t2) and r1["f2"] == r2["f2"] and r1["steps"] == r2["steps"]),
            "steps": r1["steps"],
            "note": "with K = 256 each CTA scores 2 candidates per step; the per-step exchange between CTAs "
                    "then costs more than the scoring it spreads"}
