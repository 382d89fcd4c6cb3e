"""CPU oracle for the SRO-targeted swap search -- TEST INFRASTRUCTURE ONLY.

A plain, slow, serial C++ implementation (hea_oracle.cpp) of what the GPU path computes:
Warren-Cowley pair counts and alpha (Sec. 4.3, Eq. sro), the fitness (Sec. 4.4,
Eq. fitness_function), the incremental swap delta (Sec. 4.5) and the parallel Monte Carlo
search with depth termination (Sec. 4.2, Alg. parallel_mc; Sec. 4.6.4), the global search over a
ranked pool of solutions (Sec. 4.1, Alg. global_search), the mapping of an external structure onto
the lattice (Sec. 2.3), plus the annealed-target input recipe.  Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this
package; the CUDA library neither imports nor links it.

Every function here is argument marshalling around the C entry points.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

FCC, BCC = 0, 1


class SearchParams(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("accept_mode", ctypes.c_int32),
        ("max_steps", ctypes.c_int64),
        ("depth_limit", ctypes.c_int32),
        ("max_accept", ctypes.c_int32),
        ("threshold", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("chain", ctypes.c_uint32),
        ("step0", ctypes.c_uint32),
        ("depth0", ctypes.c_int32),
        ("group_size", ctypes.c_int32),
        ("group_top", ctypes.c_int32),
        ("check", ctypes.c_int32),
    ]


class GlobalParams(ctypes.Structure):
    _fields_ = [
        ("n_solutions", ctypes.c_int32),
        ("n_refine", ctypes.c_int32),
        ("n_keep", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("tasks", ctypes.c_int32),
        ("depth_limit", ctypes.c_int32),
        ("max_steps", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("accept_mode", ctypes.c_int32),
        ("check", ctypes.c_int32),
    ]


GLOBAL_LOG_DTYPE = np.dtype([("origin", np.int32), ("pad", np.int32), ("f2_in", np.float64),
                             ("f2_out", np.float64), ("steps", np.int64), ("accepted", np.int64)])


class SearchResult(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("trials", ctypes.c_int64),
        ("accepted", ctypes.c_int64),
        ("depth", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("f2", ctypes.c_double),
        ("f", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, u32, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        _lib.or_philox4x32_10.argtypes = [P, P, P]
        _lib.or_philox4x32_10.restype = None
        _lib.or_shells.argtypes = [i32, i32, P, P, P]
        _lib.or_shells.restype = i32
        _lib.or_num_sites.argtypes = [i32, i32, i32, i32]
        _lib.or_num_sites.restype = i64
        _lib.or_positions.argtypes = [i32, i32, i32, i32, P]
        _lib.or_positions.restype = i32
        _lib.or_neighbours.argtypes = [i32, i32, i32, i32, i32, P]
        _lib.or_neighbours.restype = i32
        _lib.or_init_config.argtypes = [i64, i32, P, u64, P]
        _lib.or_init_config.restype = i32
        _lib.or_counts.argtypes = [i32, i32, i32, i32, i32, i32, P, P]
        _lib.or_counts.restype = i32
        _lib.or_alpha_f2.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P, P, P, P]
        _lib.or_alpha_f2.restype = i32
        _lib.or_delta_swap.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P, P, P, P, i64, P, P, P]
        _lib.or_delta_swap.restype = i32
        _lib.or_draw_pairs.argtypes = [i64, u64, u32, u32, i64, i32, P]
        _lib.or_draw_pairs.restype = i32
        _lib.or_search.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P,
                                   ctypes.POINTER(SearchParams), P, P, ctypes.POINTER(SearchResult), P]
        _lib.or_search.restype = i32
        _lib.or_map_structure.argtypes = [i32, i32, i32, i32, i32, i64, P, P, dbl, P, dbl, P, P]
        _lib.or_map_structure.restype = i32
        _lib.or_fresh_seed.argtypes = [u64, u32, u32]
        _lib.or_fresh_seed.restype = u64
        _lib.or_global_search.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P, ctypes.POINTER(GlobalParams),
                                          P, P, P, P, P]
        _lib.or_global_search.restype = i32
        _lib.or_anneal.argtypes = [i32, i32, i32, i32, i32, P, u64, dbl, i32, i32, P, P, P, P]
        _lib.or_anneal.restype = i32
        _lib.or_energy.argtypes = [i32, i32, i32, i32, i32, P, P]
        _lib.or_energy.restype = dbl
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def shells(kind, M):
    """(Z[M], r2[M], vectors[sum Z, 3]) for shells 1..M."""
    Z = np.zeros(M, np.int32)
    r2 = np.zeros(M, np.int32)
    vecs = np.zeros((200, 3), np.int32)
    n = lib().or_shells(kind, M, _ptr(Z), _ptr(r2), _ptr(vecs))
    if n < 0:
        raise ValueError("bad lattice kind or shell count")
    return Z, r2, vecs[:n].copy()


def num_sites(kind, L):
    return int(lib().or_num_sites(kind, *L))


def positions(kind, L):
    N = num_sites(kind, L)
    pos = np.zeros((N, 3), np.int32)
    _check(lib().or_positions(kind, *L, _ptr(pos)), "positions")
    return pos


def neighbours(kind, L, M):
    N = num_sites(kind, L)
    Z, _, _ = shells(kind, M)
    nbr = np.zeros((N, int(Z.sum())), np.int64)
    _check(lib().or_neighbours(kind, *L, M, _ptr(nbr)), "neighbours")
    return nbr


def init_config(N, n_per, seed):
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    types = np.zeros(N, np.uint8)
    _check(lib().or_init_config(N, len(n), _ptr(n), seed, _ptr(types)), "init_config")
    return types


def counts(kind, L, M, S, types):
    t = np.ascontiguousarray(types, dtype=np.uint8)
    out = np.zeros((M, S, S), np.int32)
    _check(lib().or_counts(kind, *L, M, S, _ptr(t), _ptr(out)), "counts")
    return out


def alpha_f2(kind, L, M, n_per, w, target, cnt):
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    S = len(n)
    w = np.ascontiguousarray(w, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64).reshape(M, S, S)
    c = np.ascontiguousarray(cnt, dtype=np.int32).reshape(M, S, S)
    alpha = np.zeros((M, S, S), np.float64)
    f2 = np.zeros(1, np.float64)
    _check(lib().or_alpha_f2(kind, *L, M, S, _ptr(n), _ptr(w), _ptr(t), _ptr(c), _ptr(alpha), _ptr(f2)),
           "alpha_f2")
    return alpha, float(f2[0])


def delta_swap(kind, L, M, n_per, w, target, types, cnt, pairs):
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    S = len(n)
    w = np.ascontiguousarray(w, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64).reshape(M, S, S)
    ty = np.ascontiguousarray(types, dtype=np.uint8)
    c = np.ascontiguousarray(cnt, dtype=np.int32).reshape(M, S, S)
    p = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    K = p.shape[0]
    key = np.zeros(K, np.float64)
    dN = np.zeros((K, M, S, S), np.int32)
    null = np.zeros(K, np.uint8)
    _check(lib().or_delta_swap(kind, *L, M, S, _ptr(n), _ptr(w), _ptr(t), _ptr(ty), _ptr(c), _ptr(p), K,
                               _ptr(key), _ptr(dN), _ptr(null)), "delta_swap")
    return key, dN, null.astype(bool)


def draw_pairs(N, seed, chain, step0, n_steps, K):
    out = np.zeros((n_steps * K, 2), np.int64)
    _check(lib().or_draw_pairs(N, seed, chain, step0, n_steps, K, _ptr(out)), "draw_pairs")
    return out


def search(kind, L, M, n_per, w, target, types, cnt, *, K, max_steps, accept_mode=0, depth_limit=0,
           max_accept=0, threshold=0.0, seed=1, chain=0, step0=0, depth0=0, group_size=0, group_top=0,
           check=False, log=False, timeout_us=0):
    """Runs the search in place on copies; returns (types, counts, result dict, accepted pairs or None)."""
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    S = len(n)
    w = np.ascontiguousarray(w, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64).reshape(M, S, S)
    ty = np.array(types, dtype=np.uint8, copy=True)
    c = np.array(cnt, dtype=np.int32, copy=True).reshape(M, S, S)
    p = SearchParams(K, accept_mode, max_steps, depth_limit, max_accept, threshold, seed, chain, step0,
                     depth0, group_size, group_top, 1 if check else 0)
    r = SearchResult()
    acc = np.zeros((max(1, K * max_steps), 2), np.int64) if log else None
    rc = lib().or_search(kind, *L, M, S, _ptr(n), _ptr(w), _ptr(t), ctypes.byref(p), _ptr(ty), _ptr(c),
                         ctypes.byref(r), _ptr(acc))
    if rc == 1:
        raise ValueError("oracle search: invalid arguments")
    res = {f: getattr(r, f) for f, _ in SearchResult._fields_}
    if log:
        acc = acc[: res["accepted"]].copy()
    return ty, c, res, acc


def map_structure(kind, L, S, xyz, species, a, origin=(0.0, 0.0, 0.0), tol=0.25):
    """External structure onto the lattice by nearest site; returns (types[N], report[4]:
    off-lattice atoms, multiply taken sites, empty sites, bad species)."""
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    types = np.zeros(num_sites(kind, L), np.uint8)
    report = np.zeros(4, np.int64)
    _check(lib().or_map_structure(kind, *L, S, x.shape[0], _ptr(x), _ptr(sp), a, _ptr(o), tol, _ptr(types),
                                  _ptr(report)), "map_structure")
    return types, report


def fresh_seed(seed, g, j):
    """Seed of fresh solution j of global-search iteration g."""
    return int(lib().or_fresh_seed(seed, g, j))


def global_search(kind, L, M, n_per, w, target, *, n_solutions, n_refine=0, n_keep=-1, iterations, tasks,
                  depth_limit, max_steps=1 << 30, seed=1, accept_mode=0, check=False):
    """Alg. global_search; returns (types[P_ls][N], counts[P_ls][M][S][S], f2[P_ls], log[G][P_ls],
    totals (steps, trials, accepted)).  n_refine 0 = all P solutions; n_keep -1 = n_refine // 2."""
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    S = len(n)
    N = num_sites(kind, L)
    w = np.ascontiguousarray(w, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64).reshape(M, S, S)
    PL = n_refine if n_refine > 0 else n_solutions
    R = n_keep if n_keep >= 0 else PL // 2
    gp = GlobalParams(n_solutions, PL, R, iterations, tasks, depth_limit, max_steps, seed, accept_mode,
                      1 if check else 0)
    types = np.zeros((PL, N), np.uint8)
    cnt = np.zeros((PL, M, S, S), np.int32)
    f2 = np.zeros(PL, np.float64)
    log = np.zeros((iterations, PL), GLOBAL_LOG_DTYPE)
    totals = np.zeros(3, np.int64)
    _check(lib().or_global_search(kind, *L, M, S, _ptr(n), _ptr(w), _ptr(t), ctypes.byref(gp), _ptr(types),
                                  _ptr(cnt), _ptr(f2), _ptr(log), _ptr(totals)), "global_search")
    return types, cnt, f2, log, tuple(int(x) for x in totals)


def anneal(kind, L, n_per, seed, T=800.0, sweeps=200, M_out=3):
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    S = len(n)
    N = num_sites(kind, L)
    types = np.zeros(N, np.uint8)
    eps = np.zeros((S, S), np.float64)
    alpha = np.zeros((M_out, S, S), np.float64)
    taken = np.zeros(1, np.int64)
    _check(lib().or_anneal(kind, *L, S, _ptr(n), seed, T, sweeps, M_out, _ptr(types), _ptr(eps), _ptr(alpha),
                           _ptr(taken)), "anneal")
    return types, eps, alpha, int(taken[0])


def energy(kind, L, types, eps):
    ty = np.ascontiguousarray(types, dtype=np.uint8)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    return float(lib().or_energy(kind, *L, e.shape[0], _ptr(ty), _ptr(e)))
