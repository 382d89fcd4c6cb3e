"""Python binding of libhea (include/hea.h): the same entry points, argument marshalling only.

Device buffers are torch CUDA tensors (PyTorch supplies device memory and streams); every step of
the computation runs in libhea's CUDA kernels.  There is no CPU fallback: importing works without
a GPU, but the library must be built (``paper_2411_18906_gb300.build``) and every compute call
needs a CUDA device.
"""
import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhea.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hea.h")

HEA_OK, HEA_EINVAL, HEA_ENOMEM, HEA_ECUDA, HEA_ETIMEOUT, HEA_EMISMATCH, HEA_ESYNC = range(7)
HEA_FCC, HEA_BCC = 0, 1

_lib = None


class HeaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libhea status {status}: {message}")
        self.status = status


class hea_objective(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("M", ctypes.c_int), ("n_per", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("target", ctypes.c_void_p)]


class hea_search_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("accept_mode", ctypes.c_int32), ("max_steps", ctypes.c_int64),
                ("depth_limit", ctypes.c_int32), ("max_accept", ctypes.c_int32), ("threshold", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("chain", ctypes.c_uint32), ("step0", ctypes.c_uint32),
                ("depth0", ctypes.c_int32), ("group_size", ctypes.c_int32), ("group_top", ctypes.c_int32),
                ("sync_wait_us", ctypes.c_int32), ("timeout_us", ctypes.c_int64), ("test_withhold_cta", ctypes.c_int32),
                ("threads", ctypes.c_int32)]


class hea_search_result(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("trials", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("status", ctypes.c_int32), ("f2", ctypes.c_double),
                ("f", ctypes.c_double)]


class hea_global_params(ctypes.Structure):
    _fields_ = [("n_solutions", ctypes.c_int32), ("n_refine", ctypes.c_int32), ("n_keep", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("tasks", ctypes.c_int32), ("depth_limit", ctypes.c_int32),
                ("max_steps", ctypes.c_int64), ("seed", ctypes.c_uint64), ("accept_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class hea_global_result(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("trials", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("iterations", ctypes.c_int32), ("status", ctypes.c_int32), ("best_f2", ctypes.c_double),
                ("best_f", ctypes.c_double)]


# hea_global_log as a numpy record type.
GLOBAL_LOG_DTYPE = np.dtype([("origin", np.int32), ("pad", np.int32), ("f2_in", np.float64),
                             ("f2_out", np.float64), ("steps", np.int64), ("accepted", np.int64)])

RESULT_BYTES = ctypes.sizeof(hea_search_result)
RESULT_FIELDS = [f for f, _ in hea_search_result._fields_]


def declared_symbols():
    """Names of the functions declared in include/hea.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(hea_[a-z_0-9]+)\s*\(", text)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhea is not built ({LIB_PATH} missing); run paper_2411_18906_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
        sig = {
            "hea_build_lattice": (i32, [i32, i32, i32, i32, i32, ctypes.POINTER(P)]),
            "hea_lattice_destroy": (None, [P]),
            "hea_num_sites": (i64, [P]),
            "hea_num_shells": (i32, [P]),
            "hea_shell_size": (i32, [P, i32]),
            "hea_init_config": (i32, [P, i32, P, u64, P, P]),
            "hea_sro_counts": (i32, [P, i32, P, i32, P, P]),
            "hea_sro_counts_method": (i32, [P, i32, P, i32, P, i32, P]),
            "hea_sro_alpha": (i32, [P, ctypes.POINTER(hea_objective), P, P, P, P]),
            "hea_delta_swap": (i32, [P, ctypes.POINTER(hea_objective), P, P, P, i64, P, P, P]),
            "hea_search": (i32, [P, ctypes.POINTER(hea_objective), ctypes.POINTER(hea_search_params), P, P, P, P]),
            "hea_search_batch_plan_bytes": (sz, [i32]),
            "hea_search_batch_plan": (i32, [i32, P, P, P, P, P, P, P]),
            "hea_search_batch": (i32, [P, P, P]),
            "hea_search_coop_workspace_bytes": (sz, [i32]),
            "hea_search_coop_max_ctas": (i32, [P, ctypes.POINTER(hea_objective), ctypes.POINTER(hea_search_params),
                                               i32]),
            "hea_search_coop": (i32, [P, ctypes.POINTER(hea_objective), ctypes.POINTER(hea_search_params), i32, P, P,
                                      P, P, sz, P]),
            "hea_search_coop_noalloc": (i32, [P, ctypes.POINTER(hea_objective), ctypes.POINTER(hea_search_params),
                                              i32, P, P, P, P]),
            "hea_probe_smem_gather": (i32, [i32, i32, i64, P, P]),
            "hea_map_structure": (i32, [P, i64, P, P, i32, ctypes.c_double, P, ctypes.c_double, P, P, P, P]),
            "hea_global_search_workspace_bytes": (sz, [P, ctypes.POINTER(hea_objective),
                                                       ctypes.POINTER(hea_global_params)]),
            "hea_global_search": (i32, [P, ctypes.POINTER(hea_objective), ctypes.POINTER(hea_global_params), P, P, P,
                                        P, P, P, sz, P]),
            "hea_last_error": (ctypes.c_char_p, []),
            "hea_status_string": (ctypes.c_char_p, [i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != HEA_OK:
        raise HeaError(status, lib().hea_last_error().decode())


def _ptr(t):
    """Device pointer of a torch tensor, host pointer of a numpy array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Objective:
    """Host-side hea_objective with its arrays kept alive."""

    def __init__(self, n_per, w, target):
        self.n_per = np.ascontiguousarray(n_per, dtype=np.int64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        S = len(self.n_per)
        M = len(self.w)
        self.target = np.ascontiguousarray(target, dtype=np.float64).reshape(M, S, S)
        self.c = hea_objective(S, M, self.n_per.ctypes.data, self.w.ctypes.data, self.target.ctypes.data)

    @property
    def S(self):
        return self.c.S

    @property
    def M(self):
        return self.c.M


class Lattice:
    """Owns an hea_lattice handle."""

    def __init__(self, kind, L, n_shells):
        self.kind, self.L, self.M = int(kind), tuple(int(x) for x in L), int(n_shells)
        h = ctypes.c_void_p()
        _check(lib().hea_build_lattice(self.kind, *self.L, self.M, ctypes.byref(h)))
        self.handle = h

    @property
    def N(self):
        return int(lib().hea_num_sites(self.handle))

    def shell_size(self, k):
        return int(lib().hea_shell_size(self.handle, k))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.hea_lattice_destroy(h)
            self.handle = None


def hea_build_lattice(kind, Lx, Ly, Lz, n_shells):
    return Lattice(kind, (Lx, Ly, Lz), n_shells)


def hea_init_config(lat, n_per, seed, types, stream=None):
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    _check(lib().hea_init_config(lat.handle, len(n), _ptr(n), int(seed), _ptr(types), _stream(stream)))


def hea_sro_counts(lat, n_configs, types, S, counts, stream=None):
    _check(lib().hea_sro_counts(lat.handle, int(n_configs), _ptr(types), int(S), _ptr(counts), _stream(stream)))


def hea_sro_counts_method(lat, n_configs, types, S, counts, method, stream=None):
    _check(lib().hea_sro_counts_method(lat.handle, int(n_configs), _ptr(types), int(S), _ptr(counts), int(method),
                                       _stream(stream)))


def hea_sro_alpha(lat, obj, counts, alpha, f2, stream=None):
    _check(lib().hea_sro_alpha(lat.handle, ctypes.byref(obj.c), _ptr(counts), _ptr(alpha), _ptr(f2),
                               _stream(stream)))


def hea_delta_swap(lat, obj, types, counts, pairs, K, key, dcounts=None, stream=None):
    _check(lib().hea_delta_swap(lat.handle, ctypes.byref(obj.c), _ptr(types), _ptr(counts), _ptr(pairs), int(K),
                                _ptr(key), _ptr(dcounts), _stream(stream)))


def search_params(K, max_steps, accept_mode=0, depth_limit=0, max_accept=0, threshold=0.0, seed=1, chain=0,
                  step0=0, depth0=0, group_size=0, group_top=0, timeout_us=0, sync_wait_us=0, test_withhold_cta=0,
                  threads=0):
    return hea_search_params(K, accept_mode, max_steps, depth_limit, max_accept, threshold, seed, chain, step0,
                             depth0, group_size, group_top, sync_wait_us, timeout_us, test_withhold_cta, threads)


def hea_search(lat, obj, params, types, counts, result, stream=None):
    """`result` is a device buffer of RESULT_BYTES bytes (e.g. a uint8 tensor)."""
    _check(lib().hea_search(lat.handle, ctypes.byref(obj.c), ctypes.byref(params), _ptr(types), _ptr(counts),
                            _ptr(result), _stream(stream)))


def hea_search_coop_workspace_bytes(ctas):
    return int(lib().hea_search_coop_workspace_bytes(int(ctas)))


def hea_search_coop_max_ctas(lat, obj, params, ctas):
    return int(lib().hea_search_coop_max_ctas(lat.handle, ctypes.byref(obj.c), ctypes.byref(params), int(ctas)))


def hea_search_coop(lat, obj, params, ctas, types, counts, result, workspace, stream=None):
    """`workspace` is a device buffer of at least hea_search_coop_workspace_bytes(ctas) bytes."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().hea_search_coop(lat.handle, ctypes.byref(obj.c), ctypes.byref(params), int(ctas), _ptr(types),
                                 _ptr(counts), _ptr(result), _ptr(workspace), nbytes, _stream(stream)))


def hea_search_coop_noalloc(lat, obj, params, ctas, types, counts, result, stream=None):
    """hea_search_coop with the library's fixed exchange area (no device memory from the caller)."""
    _check(lib().hea_search_coop_noalloc(lat.handle, ctypes.byref(obj.c), ctypes.byref(params), int(ctas),
                                         _ptr(types), _ptr(counts), _ptr(result), _stream(stream)))


def decode_results(raw):
    """Host bytes of hea_search_result[n] -> list of dicts."""
    b = bytes(np.ascontiguousarray(raw, dtype=np.uint8))
    n = len(b) // RESULT_BYTES
    out = []
    for i in range(n):
        r = hea_search_result.from_buffer_copy(b[i * RESULT_BYTES:(i + 1) * RESULT_BYTES])
        out.append({f: getattr(r, f) for f in RESULT_FIELDS})
    return out


def hea_search_batch_plan_bytes(n):
    return int(lib().hea_search_batch_plan_bytes(int(n)))


class BatchPlan:
    """Host plan written by hea_search_batch_plan, with every array it references kept alive."""

    def __init__(self, lats, objs, params, types, counts, results):
        n = len(lats)
        self.n = n
        self._objs = objs
        self.lat_arr = (ctypes.c_void_p * n)(*[l.handle.value for l in lats])
        self.obj_arr = (hea_objective * n)(*[o.c for o in objs])
        self.par_arr = (hea_search_params * n)(*params)
        self.typ_arr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in types])
        self.cnt_arr = (ctypes.c_void_p * n)(*[c.data_ptr() for c in counts])
        self.host = np.zeros(hea_search_batch_plan_bytes(n), np.uint8)
        _check(lib().hea_search_batch_plan(n, self.lat_arr, self.obj_arr, self.par_arr, self.typ_arr, self.cnt_arr,
                                           _ptr(results), _ptr(self.host)))


def hea_search_batch(plan_host, plan_dev, stream=None):
    _check(lib().hea_search_batch(_ptr(plan_host), _ptr(plan_dev), _stream(stream)))


def global_params(n_solutions, iterations, tasks, depth_limit, n_refine=0, n_keep=-1, max_steps=1 << 30, seed=1,
                  accept_mode=0):
    """hea_global_params; n_refine 0 = all n_solutions, n_keep -1 = n_refine // 2 (p_a = 1/2)."""
    PL = n_refine if n_refine > 0 else n_solutions
    R = n_keep if n_keep >= 0 else PL // 2
    return hea_global_params(n_solutions, PL, R, iterations, tasks, depth_limit, max_steps, seed, accept_mode, 0)


def hea_global_search_workspace_bytes(lat, obj, params):
    return int(lib().hea_global_search_workspace_bytes(lat.handle, ctypes.byref(obj.c), ctypes.byref(params)))


def hea_global_search(lat, obj, params, types, counts, f2, log, result, workspace, stream=None):
    """`result` is a device buffer of sizeof(hea_global_result) bytes; `log` a device buffer of
    iterations * n_refine GLOBAL_LOG_DTYPE records or None; `workspace` 256-byte aligned."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().hea_global_search(lat.handle, ctypes.byref(obj.c), ctypes.byref(params), _ptr(types), _ptr(counts),
                                   _ptr(f2), _ptr(log), _ptr(result), _ptr(workspace), nbytes, _stream(stream)))


def decode_global_result(raw):
    r = hea_global_result.from_buffer_copy(bytes(np.ascontiguousarray(raw, dtype=np.uint8)))
    return {f: getattr(r, f) for f, _ in hea_global_result._fields_}


def hea_map_structure(lat, n, xyz, species, S, a, origin, tol, types, scratch, report, stream=None):
    """xyz, species, types, scratch, report: device tensors; origin: 3 floats (host)."""
    o = np.ascontiguousarray(origin, dtype=np.float64)
    _check(lib().hea_map_structure(lat.handle, int(n), _ptr(xyz), _ptr(species), int(S), float(a), _ptr(o),
                                   float(tol), _ptr(types), _ptr(scratch), _ptr(report), _stream(stream)))


def hea_probe_smem_gather(mode, ctas, iters, sink, stream=None):
    _check(lib().hea_probe_smem_gather(int(mode), int(ctas), int(iters), _ptr(sink), _stream(stream)))
