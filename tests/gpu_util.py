"""Helpers for the GPU parity tests: run libhea calls on torch CUDA buffers and return numpy."""
import numpy as np
import torch

from paper_2411_18906_gb300 import build as hbuild
from paper_2411_18906_gb300 import hea

_built = False


def ensure_built():
    global _built
    if not _built:
        hbuild.build()
        hea.lib()
        _built = True


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_init(kind, L, M, n_per, seed):
    ensure_built()
    lat = hea.Lattice(kind, L, M)
    types = torch.empty(lat.N, dtype=torch.uint8, device="cuda")
    hea.hea_init_config(lat, n_per, seed, types)
    torch.cuda.synchronize()
    return types.cpu().numpy()


def gpu_counts(kind, L, M, S, types_batch):
    ensure_built()
    lat = hea.Lattice(kind, L, M)
    tb = np.ascontiguousarray(types_batch, dtype=np.uint8).reshape(-1, lat.N)
    t = dev(tb)
    counts = torch.full((tb.shape[0], M, S, S), -7, dtype=torch.int32, device="cuda")
    hea.hea_sro_counts(lat, tb.shape[0], t, S, counts)
    torch.cuda.synchronize()
    return counts.cpu().numpy()


def gpu_alpha(kind, L, M, n_per, w, target, cnt):
    ensure_built()
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    S = len(n_per)
    alpha = torch.empty((M, S, S), dtype=torch.float64, device="cuda")
    f2 = torch.empty(1, dtype=torch.float64, device="cuda")
    hea.hea_sro_alpha(lat, obj, dev(np.asarray(cnt, np.int32)), alpha, f2)
    torch.cuda.synchronize()
    return alpha.cpu().numpy(), float(f2.cpu().numpy()[0])


def gpu_delta(kind, L, M, n_per, w, target, types, cnt, pairs):
    ensure_built()
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    S = len(n_per)
    p = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    K = p.shape[0]
    key = torch.empty(K, dtype=torch.float64, device="cuda")
    dN = torch.empty((K, M, S, S), dtype=torch.int32, device="cuda")
    hea.hea_delta_swap(lat, obj, dev(np.asarray(types, np.uint8)), dev(np.asarray(cnt, np.int32)), dev(p), K, key, dN)
    torch.cuda.synchronize()
    return key.cpu().numpy(), dN.cpu().numpy()


def gpu_search(kind, L, M, n_per, w, target, types, cnt, **kw):
    ensure_built()
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    t = dev(np.asarray(types, np.uint8))
    c = dev(np.asarray(cnt, np.int32))
    res = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    hea.hea_search(lat, obj, hea.search_params(**kw), t, c, res)
    torch.cuda.synchronize()
    return t.cpu().numpy(), c.cpu().numpy(), hea.decode_results(res.cpu().numpy())[0]


def gpu_search_batch(cells, params):
    """cells: list of (kind, L, M, n_per, w, target, types, counts); params: list of search_params kwargs."""
    ensure_built()
    lats, objs, ts, cs, ps = [], [], [], [], []
    for (kind, L, M, n_per, w, target, types, cnt), kw in zip(cells, params):
        lats.append(hea.Lattice(kind, L, M))
        objs.append(hea.Objective(n_per, w, target))
        ts.append(dev(np.asarray(types, np.uint8)))
        cs.append(dev(np.asarray(cnt, np.int32)))
        ps.append(hea.search_params(**kw))
    n = len(cells)
    res = torch.zeros(n * hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan = hea.BatchPlan(lats, objs, ps, ts, cs, res)
    plan_dev = dev(plan.host)
    hea.hea_search_batch(plan.host, plan_dev)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in ts], [c.cpu().numpy() for c in cs], hea.decode_results(res.cpu().numpy())


def sm_count():
    return torch.cuda.get_device_properties(0).multi_processor_count


def gpu_search_coop(kind, L, M, n_per, w, target, types, cnt, ctas, **kw):
    ensure_built()
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    t = dev(np.asarray(types, np.uint8))
    c = dev(np.asarray(cnt, np.int32))
    res = torch.zeros(hea.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ws = torch.zeros(hea.hea_search_coop_workspace_bytes(ctas), dtype=torch.uint8, device="cuda")
    hea.hea_search_coop(lat, obj, hea.search_params(**kw), ctas, t, c, res, ws)
    torch.cuda.synchronize()
    return t.cpu().numpy(), c.cpu().numpy(), hea.decode_results(res.cpu().numpy())[0]


def gpu_global_search(kind, L, M, n_per, w, target, **kw):
    """hea_global_search on fresh torch buffers; kw as hea.global_params.  Returns (types, counts,
    f2, log, result dict) as numpy."""
    ensure_built()
    lat = hea.Lattice(kind, L, M)
    obj = hea.Objective(n_per, w, target)
    gp = hea.global_params(**kw)
    S = len(n_per)
    PL, G = gp.n_refine, gp.iterations
    types = torch.empty((PL, lat.N), dtype=torch.uint8, device="cuda")
    counts = torch.empty((PL, M, S, S), dtype=torch.int32, device="cuda")
    f2 = torch.empty(PL, dtype=torch.float64, device="cuda")
    log = torch.zeros(G * PL * hea.GLOBAL_LOG_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    res = torch.zeros(ctypes_sizeof_global_result(), dtype=torch.uint8, device="cuda")
    ws = torch.empty(hea.hea_global_search_workspace_bytes(lat, obj, gp), dtype=torch.uint8, device="cuda")
    hea.hea_global_search(lat, obj, gp, types, counts, f2, log, res, ws)
    torch.cuda.synchronize()
    lg = np.frombuffer(log.cpu().numpy().tobytes(), dtype=hea.GLOBAL_LOG_DTYPE).reshape(G, PL)
    return (types.cpu().numpy(), counts.cpu().numpy(), f2.cpu().numpy(), lg,
            hea.decode_global_result(res.cpu().numpy()))


def ctypes_sizeof_global_result():
    import ctypes
    return ctypes.sizeof(hea.hea_global_result)
