"""Benchmark of the SRO-targeted swap search on one GB300 (or N replicas under torchrun).

One step = the whole hot path once on the 256,000-site FCC workload (40x40x40 conventional cells,
species 40/20/20/20 at.%, shells 1-3, nonzero annealed target, unit weights):
  initial configuration -> full pair recount -> alpha and F^2 -> 1e8 candidate swaps scored by
  the persistent search (non-overlapping multi-swap accept, K candidates per step).
The metric is swap trials per second (a trial = one scored candidate).  Inputs are synthetic
(seeded); the cell is device-resident when the timed region starts.  L2 is flushed (256 MiB write)
between timed steps, outside the per-step event pairs.

`--impl reference` times the plain CPU oracle on the same workload (bounded sample per step).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2411_18906_gb300 import workloads  # noqa: E402

METRIC = "Δ-SRO swap trials/s at 256k-atom FCC; batched cells/s; p99 serve latency"
SEARCH_K = 256           # candidates per step of the single-CTA chain (parity tests, CPU sample)
COOP_KC = 512            # candidates per CTA per step of the cooperative chain
COOP_TOP = 1             # best eligible candidates per CTA that enter the multi-accept walk
TRIALS_PER_STEP = 100_000_000
WORKLOAD = "FCC 40x40x40 (256,000 sites), 4 species 40/20/20/20, shells 1-3, annealed target, " \
           "1e8 swap trials per step, multi-accept, one chain over all SMs (512 candidates per CTA per " \
           "search step, best 1 per CTA walked)"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def replica_seed(rank):
    """Each rank runs an independent chain (replicas: no data-path collective)."""
    return 1 + rank


def aggregate_ranks(dist, total_ms, search_ms, trials_local, device):
    """Max over ranks of the timed device time (and of the search part); whole-job throughput =
    the trials of all ranks over that time.  dist = None for a single process."""
    import torch
    t = torch.tensor([total_ms, search_ms], dtype=torch.float64, device=device)
    n = torch.tensor([float(trials_local)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    total_ms, search_ms = float(t[0]), float(t[1])
    return total_ms, search_ms, float(n[0]) / (total_ms / 1000.0)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_inputs():
    spec = workloads.fcc_256k()
    return spec


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2411_18906_gb300 import build as hbuild
    from paper_2411_18906_gb300 import hea

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    hbuild.build()
    spec = workload_inputs()
    lat = hea.Lattice(spec.kind, spec.L, spec.M)
    obj = hea.Objective(spec.n_per, spec.weights(), spec.targets())
    N, S, M = lat.N, spec.S, spec.M
    ctas = torch.cuda.get_device_properties(local).multi_processor_count
    coop_kc, coop_top = args.coop_kc, args.coop_top
    K = ctas * coop_kc
    steps_per_call = max(1, args.trials // K)
    trials_per_step = steps_per_call * K
    workspace = torch.zeros(hea.hea_search_coop_workspace_bytes(ctas), dtype=torch.uint8, device="cuda")

    def search(step_seed):
        params = hea.search_params(K, steps_per_call, accept_mode=1, group_size=coop_kc, group_top=coop_top,
                                   seed=step_seed)
        hea.hea_search_coop(lat, obj, params, ctas, types, counts, result, workspace, stream)

    stream = torch.cuda.current_stream()
    types = torch.empty(N, dtype=torch.uint8, device="cuda")
    counts = torch.empty((M, S, S), dtype=torch.int32, device="cuda")
    alpha = torch.empty((M, S, S), dtype=torch.float64, device="cuda")
    f2 = torch.empty(1, dtype=torch.float64, device="cuda")
    result = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    seed = replica_seed(rank)

    def one_step(step_seed):
        hea.hea_init_config(lat, spec.n_per, step_seed, types, stream)
        hea.hea_sro_counts(lat, 1, types, S, counts, stream)
        hea.hea_sro_alpha(lat, obj, counts, alpha, f2, stream)
        search(step_seed)

    for w in range(args.warmup):
        one_step(seed)
    torch.cuda.synchronize()
    res_warm = hea.decode_results(result.cpu().numpy())[0]
    if res_warm["status"] != 0 or res_warm["trials"] != trials_per_step:
        raise RuntimeError(f"warm-up search did not complete its budget: {res_warm}")

    sampler = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    search_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(s & 0xFF)  # evict L2 between timed steps (outside the event pair)
        starts[s].record(stream)
        hea.hea_init_config(lat, spec.n_per, seed, types, stream)
        hea.hea_sro_counts(lat, 1, types, S, counts, stream)
        hea.hea_sro_alpha(lat, obj, counts, alpha, f2, stream)
        search_start[s].record(stream)
        search(seed)
        stops[s].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [starts[s].elapsed_time(stops[s]) for s in range(args.steps)]
    search_ms = [search_start[s].elapsed_time(stops[s]) for s in range(args.steps)]
    total_ms = float(sum(step_ms))
    res = hea.decode_results(result.cpu().numpy())[0]
    if res["status"] != 0:
        raise RuntimeError(f"search status {res['status']}")
    # Max over ranks of the timed device time.
    total_ms, search_total_ms, value = aggregate_ranks(dist if world > 1 else None, total_ms, float(sum(search_ms)),
                                                        trials_per_step * args.steps, "cuda")

    # End to end through the public API with host buffers: initial structure copied in from pinned
    # memory, recount, alpha, search, final structure + counts + result copied back.
    host_in = torch.from_numpy(oracle_free_initial(spec, N)).pin_memory()
    host_types = torch.empty(N, dtype=torch.uint8).pin_memory()
    host_counts = torch.empty((M, S, S), dtype=torch.int32).pin_memory()
    host_res = torch.empty(hea.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for s in range(e2e_steps):
        flush.fill_(s & 0xFF)
        e0.record(stream)
        types.copy_(host_in, non_blocking=True)
        hea.hea_sro_counts(lat, 1, types, S, counts, stream)
        hea.hea_sro_alpha(lat, obj, counts, alpha, f2, stream)
        search(seed)
        host_types.copy_(types, non_blocking=True)
        host_counts.copy_(counts, non_blocking=True)
        host_res.copy_(result, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_value = trials_per_step * e2e_steps / (e2e_ms / 1000.0)

    peaks, peak_kind = load_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", SM_MAX_MHZ)
    # Dominant kernel: the persistent search.  Algorithmic work per trial: 2 (1 + Z_tot) species
    # bytes gathered from shared memory (Z_tot = 42); peak = one 32-lane shared-memory wavefront
    # per SM per clock at the maximum SM clock, 1 useful byte per lane, all 152 SMs.
    z_tot = 12 + 6 + 24
    bytes_per_trial = 2 * (1 + z_tot)
    search_s = (search_total_ms / args.steps) / 1000.0
    achieved_gbs = trials_per_step * bytes_per_trial / search_s / 1e9
    peak_gbs = SM_COUNT * 32 * peaks.get("sm_max_mhz", SM_MAX_MHZ) * 1e6 / 1e9
    roofline = {"bound": "alu", "kernel": f"coop_kernel (one chain, {ctas} CTAs)",
                "achieved": round(achieved_gbs, 3), "peak": round(peak_gbs, 1), "unit": "GB/s",
                "frac": achieved_gbs / peak_gbs, "traffic": None,
                "peak_source": "shared-memory gather issue rate: 152 SMs x 32 lanes x max SM clock "
                               f"({peak_kind} peaks file for the clock)",
                "search_ms_per_step": search_total_ms / args.steps}

    line = {
        "metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8+i32+f64", "data": "synthetic",
        "config": {"workload": (WORKLOAD if args.trials == TRIALS_PER_STEP else
                                WORKLOAD.replace("1e8 swap trials", f"{trials_per_step} swap trials")).replace(
                                    "512 candidates per CTA", f"{coop_kc} candidates per CTA").replace(
                                    "best 1 per CTA", f"best {coop_top} per CTA"),
                   "sites": N, "trials_per_step": trials_per_step, "K": K, "ctas": ctas, "search_steps": steps_per_call,
                   "accept_mode": "multi", "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "trials/s", "h2d_bytes_per_step": N,
                "d2h_bytes_per_step": N + 4 * M * S * S + hea.RESULT_BYTES},
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
        "final": {"F": res["f"], "accepted": res["accepted"], "search_steps": res["steps"]},
        "wall_s": wall,
    }
    if rank == 0 and world == 1 and not args.no_secondary:
        line["batched"] = run_batched(torch, hea)
        line["recount"] = run_recount(torch, hea)
        line["serve"] = run_serving(args.serve_requests)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_steps, ctas, coop_kc, coop_top)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batched(torch, hea, n_cells=512, trials=1_000_000, steps=3, warmup=1):
    """Batched workload: n_cells independent cells (FCC or BCC, 500-32,000 sites, 3-6 species,
    1-3 shells, annealed targets) searched together, 1e6 trials each, best-of-K; the whole step
    (initial configuration, recount and the batched search of every cell) is one captured CUDA
    graph, replayed per timed step.  K per size bucket comes from the autotuner."""
    from paper_2411_18906_gb300 import autotune
    cells = workloads.batch_cells(n_cells, seed=1)
    prep = []
    for c in cells:
        lat = hea.Lattice(c.kind, c.L, c.M)
        obj = hea.Objective(c.n_per, c.weights(), c.targets())
        t = torch.empty(c.N, dtype=torch.uint8, device="cuda")
        k = torch.empty((c.M, c.S, c.S), dtype=torch.int32, device="cuda")
        hea.hea_init_config(lat, c.n_per, c.seed, t)
        hea.hea_sro_counts(lat, 1, t, c.S, k)
        prep.append((lat, obj, t, k))
    torch.cuda.synchronize()
    choice, report = autotune.tune(prep, trials=100_000, accept_mode=0)
    params = []
    for i, (lat, _, _, _) in enumerate(prep):
        K = choice[autotune.bucket_of(lat.N)]
        params.append(hea.search_params(K, max(1, trials // K), accept_mode=0, seed=3000 + i, chain=i))
    res = torch.zeros(n_cells * hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan = hea.BatchPlan([p[0] for p in prep], [p[1] for p in prep], params, [p[2] for p in prep],
                         [p[3] for p in prep], res)
    plan_dev = torch.from_numpy(plan.host).cuda()

    def step():
        for (lat, obj, t, k), c in zip(prep, cells):
            hea.hea_init_config(lat, c.n_per, c.seed, t)
            hea.hea_sro_counts(lat, 1, t, c.S, k)
        hea.hea_search_batch(plan.host, plan_dev)

    step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
            step()
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = hea.decode_results(res.cpu().numpy())
    trials_total = sum(r["trials"] for r in out)
    return {"metric": "batched cells/s", "value": n_cells / (ms / 1000.0), "unit": "cells/s",
            "ms_per_step": ms, "cells": n_cells, "trials_per_cell": trials, "trials_per_s": trials_total / (ms / 1e3),
            "accept_mode": "best-of-K", "K_by_bucket": {str(b): k for b, k in choice.items()},
            "autotune": report, "graph": "one CUDA graph per step (init + recount per cell, one batched search)",
            "mean_F": float(np.mean([r["f"] for r in out])),
            "status_ok": all(r["status"] == 0 for r in out)}


def run_recount(torch, hea, n_configs=1000):
    """Full recount throughput: 1000 seeded BCC 20x20x20 configurations (5 species, shells 1-2) in
    one call; HBM roofline = configuration bytes read + count bytes written."""
    spec = workloads.bcc_16k()
    lat = hea.Lattice(spec.kind, spec.L, spec.M)
    N, S, M = lat.N, spec.S, spec.M
    types = torch.empty((n_configs, N), dtype=torch.uint8, device="cuda")
    for i in range(n_configs):
        hea.hea_init_config(lat, spec.n_per, i + 1, types[i])
    counts = torch.empty((n_configs, M, S, S), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        hea.hea_sro_counts(lat, n_configs, types, S, counts)
    torch.cuda.synchronize()
    times = []
    for r in range(5):
        flush.fill_(r)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        hea.hea_sro_counts(lat, n_configs, types, S, counts)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1000.0)
    t = float(np.median(times))
    peaks, kind = load_peaks()
    nbytes = n_configs * N + n_configs * M * S * S * 4
    visits = n_configs * N * (8 + 6)
    return {"metric": "pair-counts/s (full recount, 1000 x BCC 20^3)", "value": visits / t, "unit": "pair visits/s",
            "seconds": t, "roofline": {"bound": "hbm", "achieved": nbytes / t / 1e9, "peak": peaks["hbm_gbs"],
                                        "unit": "GB/s", "frac": nbytes / t / 1e9 / peaks["hbm_gbs"],
                                        "peak_source": kind}}


def run_serving(n_requests=300, rate=50.0):
    """Served workload: Poisson arrivals (50/s), 1k-256k sites (20% at 256k), 4-5 species, K = 256,
    depth limit 10, at most 1e6 trials per request, continuous batching on per-request streams."""
    from paper_2411_18906_gb300 import serve
    reqs = serve.poisson_requests(n_requests, rate, seed=1)
    srv = serve.Server(hbm_budget_bytes=16 << 30, slots=64)
    done = srv.run(reqs)
    out = serve.latency_summary(done)
    out.update({"metric": "serve latency", "unit": "s", "rate_per_s": rate, "max_inflight": srv.max_inflight,
                "status_ok": all(c.result["status"] == 0 for c in done)})
    return out


def oracle_free_initial(spec, N):
    """A seeded random initial structure built on the host with numpy (input only)."""
    rng = np.random.default_rng(spec.seed + 12345)
    t = np.repeat(np.arange(spec.S, dtype=np.uint8), spec.n_per)
    rng.shuffle(t)
    return t


# ------------------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ------------------------------------------------------------------------------------------------
def cpu_baseline(n_steps, ctas=SM_COUNT, coop_kc=COOP_KC, coop_top=COOP_TOP):
    """The plain serial oracle on a bounded sample of the same workload: init, recount, then n_steps
    search steps with the benchmark's candidate set and accept rule (K = ctas x 512 candidates per
    step, the best 2 eligible of every 512 walked).  Returns trials/s of the search part."""
    import oracle
    spec = workload_inputs()
    N = spec.N
    K = ctas * coop_kc
    t0 = time.perf_counter()
    types = oracle.init_config(N, spec.n_per, spec.seed)
    cnt = oracle.counts(spec.kind, spec.L, spec.M, spec.S, types)
    t1 = time.perf_counter()
    _, _, res, _ = oracle.search(spec.kind, spec.L, spec.M, spec.n_per, spec.weights(), spec.targets(), types, cnt,
                                 K=K, max_steps=n_steps, accept_mode=1, group_size=coop_kc, group_top=coop_top,
                                 seed=spec.seed)
    t2 = time.perf_counter()
    trials = res["trials"]
    return {"value": trials / (t2 - t1), "unit": "trials/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_steps} search steps x K={K} ({trials} trials) of the 256,000-site FCC workload from "
                      f"a fresh random start (same candidates and accept rule as the GPU run); init + recount "
                      f"took {t1 - t0:.2f} s (not in value)",
            "seconds": t2 - t0}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(max(1, args.cpu_steps // 2)))
    wall = time.perf_counter() - t0
    value = float(np.mean([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+i32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sites": 256000, "K": SM_COUNT * COOP_KC, "accept_mode": "multi",
                       "parallelism": "CPU oracle, 1 thread"},
            "cpu_baseline": {"value": value, "unit": "trials/s", "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"] if vals else ""},
            "e2e": {"value": value, "unit": "trials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-steps", type=int, default=12, help="oracle search steps in the CPU sample")
    ap.add_argument("--trials", type=int, default=TRIALS_PER_STEP,
                    help="swap trials per step (workload size; the headline workload is 1e8)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the batched, recount and serving measurements")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--coop-kc", type=int, default=COOP_KC, help="candidates per CTA per search step")
    ap.add_argument("--coop-top", type=int, default=COOP_TOP, help="best eligible candidates per CTA walked")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
