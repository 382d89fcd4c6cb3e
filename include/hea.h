/*
 * hea.h -- C ABI of libhea: GPU (sm_103a) hot path of the short-range-order (SRO) targeted
 * structure search of Niu & Liu, "Short-Range Order Based Ultra Fast Large-Scale Modeling of
 * High-Entropy Alloys" (arXiv 2411.18906).
 *
 * The library computes, on one GPU:
 *   - a seeded random initial configuration with an exact composition           (Sec. 4.1)
 *   - Warren-Cowley pair counts N_ij^(k) and alpha_ij^(k) = 1 - P_ij^(k) / c_j   (Sec. 4.3, Eq. sro)
 *   - the fitness F = sqrt(sum_k w_k sum_ij (alpha - alpha_target)^2)           (Sec. 4.4, Eq. fitness_function)
 *   - the incremental change of the counts and of F^2 for candidate swaps       (Sec. 4.5; Sec. 4.6.2)
 *   - the parallel Monte Carlo search: K random two-atom swaps per step, best-of-K
 *     (or non-overlapping multi-swap) accept, depth counter, step budget       (Sec. 4.2, Alg. parallel_mc;
 *                                                                               Sec. 4.6.3-4.6.4)
 *
 * Conventions shared by every call:
 *   - Pointers marked "device" are CUDA device (or managed) memory owned by the caller; pointers
 *     marked "host" are ordinary host memory read during the call only.  The library keeps no
 *     pointer after a call returns and never allocates device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Device work
 *     is asynchronous on that stream; outputs are valid after the stream is synchronised.
 *   - Every call returns a hea_status.  Argument errors are detected on the host before any launch
 *     and leave outputs untouched; hea_last_error() then returns a message (thread-local).
 *     Conditions met on the device (a search that ran out of its time budget) are reported in the
 *     status field of hea_search_result.
 *   - Geometry: integer coordinates in half lattice units.  FCC sites are the points with X+Y+Z
 *     even, BCC sites the points whose three coordinates share one parity; the period along each
 *     axis is 2*L.  Site index = ((b * Lz + cz) * Ly + cy) * Lx + cx with the basis (sublattice)
 *     b in the order FCC (0,0,0),(0,1,1),(1,0,1),(1,1,0); BCC (0,0,0),(1,1,1).  Shell k (1-based)
 *     is the k-th smallest neighbour distance: FCC Z = 12, 6, 24, 12, 24; BCC Z = 8, 6, 12, 24, 8.
 *   - Counts are int32 arrays [M][S][S] (row-major shell k, species i, species j); N_ij^(k) counts
 *     ordered (site, shell vector) pairs, so row i sums to N_i * Z_k.
 *   - Objective arithmetic (IEEE binary64, shared exactly with the reference definition):
 *       Q = N / ((Z_k * N_i) * N_j), e = (1 - n * Q) - t, F^2 = sum over (k,i,j) row-major of
 *       w_k * (e * e); swap key D = change of F^2 = sum over (k,i,j) row-major of
 *       fma(dN, fma(a, dN, b), D) with a = w_k * (Q * Q) and b = -2 * (w_k * (Q * e)).
 */
#ifndef HEA_H
#define HEA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every declaration below is exported from libhea.so even though the library is built with
 * hidden default visibility. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef enum {
    HEA_OK = 0,
    HEA_EINVAL = 1,    /* invalid argument (shape, range, composition, null pointer) */
    HEA_ENOMEM = 2,    /* problem does not fit the on-chip (shared-memory) budget of a kernel */
    HEA_ECUDA = 3,     /* a CUDA runtime call failed (no device, launch error) */
    HEA_ETIMEOUT = 4,  /* a search stopped at its time budget (reported in hea_search_result) */
    HEA_EMISMATCH = 5, /* reserved (no call returns it) */
    HEA_ESYNC = 6      /* a cooperative search stopped because a wait for another CTA's records ran out
                          (reported in hea_search_result) */
} hea_status;

typedef enum { HEA_FCC = 0, HEA_BCC = 1 } hea_kind;

/* Opaque, host-side lattice description (no device memory behind it). */
typedef struct hea_lattice hea_lattice;

/* Maximum sizes accepted by the calls below. */
#define HEA_MAX_SPECIES 8
#define HEA_MAX_SHELLS 5
#define HEA_MAX_SITES (1 << 30)

/*
 * Builds the periodic FCC/BCC supercell of Lx x Ly x Lz conventional cells (Table 1 caption:
 * S = A * L^3 with A = 4 for fcc and 2 for bcc; non-cubic cells allowed) with shells 1..n_shells.
 * Requires Lx, Ly, Lz >= 2 (no site is its own neighbour) and 1 <= n_shells <= 5.
 * Host only.  *out receives a handle to release with hea_lattice_destroy.
 */
hea_status hea_build_lattice(int kind, int Lx, int Ly, int Lz, int n_shells, hea_lattice** out);
void hea_lattice_destroy(hea_lattice* lat);
int64_t hea_num_sites(const hea_lattice* lat);
int hea_num_shells(const hea_lattice* lat);
/* Coordination number Z_k of shell k (1-based); 0 when k is out of range. */
int hea_shell_size(const hea_lattice* lat, int k);

/*
 * Initial configuration (Sec. 4.1: the first candidate solutions are generated entirely at
 * random) with exactly n_per[s] sites of species s.  Sites are ordered by the unique 64-bit key
 * (r0 << 32 | i), r0 the first word of Philox4x32-10 with key (lo32(seed), hi32(seed)) and counter
 * (i, 0, 0, 0); the site of rank r gets species s with cum[s] <= r < cum[s+1].
 *   n_per   host int64[S], each >= 0, summing to N
 *   types   device uint8[N], overwritten
 * Errors: HEA_EINVAL for a bad composition or S outside [1, 255].
 */
hea_status hea_init_config(const hea_lattice* lat, int S, const int64_t* n_per, uint64_t seed, uint8_t* types,
                           void* stream);

/*
 * Full recount of the Warren-Cowley pair counts N_ij^(k) (Sec. 4.3) for n_configs
 * configurations of the same lattice.
 *   types   device uint8[n_configs][N], species in [0, S)
 *   counts  device int32[n_configs][M][S][S], overwritten
 * Errors: HEA_EINVAL for S outside [1, 8] or n_configs < 1.  Species values >= S are not checked
 * on the device; their pairs are not counted.
 */
hea_status hea_sro_counts(const hea_lattice* lat, int n_configs, const uint8_t* types, int S, int32_t* counts,
                          void* stream);

/*
 * hea_sro_counts with a chosen kernel (same arguments, results and errors):
 *   method 0  automatic (bit planes for batches of at least 64 configurations when they apply)
 *   method 1  neighbour gathers: per site, its shell histograms from species staged in shared memory,
 *             summed per centre species across each warp
 *   method 2  bit planes: per species one bit per site; N_ij^(k) = sum over shell-k vectors of
 *             popcount(plane_i AND shifted plane_j), one CTA per configuration; needs Lx <= 64 and
 *             2 <= S <= 6 (HEA_EINVAL otherwise)
 */
hea_status hea_sro_counts_method(const hea_lattice* lat, int n_configs, const uint8_t* types, int S, int32_t* counts,
                                 int method, void* stream);

/* Objective of Eq. fitness_function; all arrays in host memory, read during the call only. */
typedef struct {
    int S;                 /* species, 2..8 */
    int M;                 /* shells, must equal the lattice's n_shells */
    const int64_t* n_per;  /* int64[S] composition, each >= 1, summing to N */
    const double* w;       /* double[M] shell weights w_k, finite, >= +0 */
    const double* target;  /* double[M][S][S] target alpha (may be asymmetric), finite */
} hea_objective;

/*
 * alpha_ij^(k) (Eq. sro) and F^2 (Eq. fitness_function, squared) from device counts.
 *   counts  device int32[M][S][S];  alpha device double[M][S][S];  f2 device double[1]
 */
hea_status hea_sro_alpha(const hea_lattice* lat, const hea_objective* obj, const int32_t* counts, double* alpha,
                         double* f2, void* stream);

/*
 * Scores K candidate swaps against one state (Sec. 4.5, Sec. 4.6.2): for each pair (a, b) the
 * exact change dN of the counts and the key D = change of F^2.  Bonds between a and b keep their
 * unordered species pair and contribute nothing.  A null move (a == b or equal species) gets
 * D = +0.0 and dN = 0.
 *   types   device uint8[N];  counts device int32[M][S][S] (must be the counts of types)
 *   pairs   device int64[K][2], each in [0, N)
 *   key     device double[K]
 *   dcounts device int32[K][M][S][S] or NULL
 * Errors: HEA_EINVAL for K < 1 or a bad objective.  Out-of-range pairs are not checked on the
 * device; their key is set to NaN.
 */
hea_status hea_delta_swap(const hea_lattice* lat, const hea_objective* obj, const uint8_t* types,
                          const int32_t* counts, const int64_t* pairs, int64_t K, double* key, int32_t* dcounts,
                          void* stream);

/* Parameters of the parallel Monte Carlo search (Alg. parallel_mc; Sec. 4.6.4). */
typedef struct {
    int32_t K;            /* candidate swaps (tasks) per step: 1..4096 per CTA, further limited by
                             shared memory (about 60 bytes per candidate next to the cell;
                             HEA_ENOMEM when it does not fit) */
    int32_t accept_mode;  /* 0: best-of-K (argmin over (D, k)); 1: non-overlapping multi-accept */
    int64_t max_steps;    /* step budget (>= 0) */
    int32_t depth_limit;  /* stop once this many consecutive steps accepted nothing (0 = off) */
    int32_t max_accept;   /* multi-accept: at most this many swaps per step (0 = unlimited) */
    double threshold;     /* 0: accept only D < 0; > 0 also accepts non-null moves with D <= threshold */
    uint64_t seed;        /* Philox key */
    uint32_t chain;       /* chain id (third Philox counter word) */
    uint32_t step0;       /* counter of the first step (resume: previous step0 + steps) */
    int32_t depth0;       /* depth counter at entry (resume) */
    int32_t group_size;   /* multi-accept: candidate k belongs to group k / group_size (0 = one group of K) */
    int32_t group_top;    /* multi-accept: only the group_top best eligible candidates (by (D, k)) of each
                             group enter the walk (0 = all eligible candidates) */
    int32_t sync_wait_us; /* cooperative search: limit of each wait for another CTA's records, in
                             microseconds (0 = 2,000,000); ignored by the other searches */
    int64_t timeout_us;   /* wall-clock budget measured on the device, 0 = none */
    int32_t test_withhold_cta; /* testing aid of the cooperative search: 1 + the index of a CTA that
                                  never publishes its records, so that the others' bounded waits run
                                  out and the search ends with HEA_ESYNC (0 = none; must be 0 elsewhere) */
    int32_t threads;      /* threads per CTA of hea_search and hea_search_batch: 0 (= 256), 128, 256 or 512
                             (results do not depend on it); must be 0 for the cooperative searches */
} hea_search_params;

/* Written by the search on the device (device or host-mapped pinned memory). */
typedef struct {
    int64_t steps;     /* steps executed */
    int64_t trials;    /* candidates scored = steps * K */
    int64_t accepted;  /* swaps applied */
    int32_t depth;     /* depth counter at exit */
    int32_t status;    /* HEA_OK; HEA_ETIMEOUT when the time budget ended the search; HEA_ESYNC when a
                          cooperative search stopped because a wait for another CTA ran out */
    double f2;         /* F^2 of the final state (canonical order) */
    double f;          /* sqrt(F^2) */
} hea_search_result;

/*
 * Runs the search on one chain in a single persistent CTA (one step = K Philox-drawn swaps
 * scored in parallel, then the accept step; candidate k of step s draws Philox with key
 * (lo32(seed), hi32(seed)) and counter (k, s, chain, 1): a = r0 * N >> 32, b = r1 * N >> 32).
 *   types   device uint8[N], in/out;  counts device int32[M][S][S], in/out (counts of types)
 *   result  device (or host-mapped) hea_search_result
 * Errors: HEA_EINVAL for bad parameters; HEA_ENOMEM when the cell and K do not fit the CTA's
 * shared memory (about 400,000 sites at 4 bits per site, minus the candidate buffers).
 */
hea_status hea_search(const hea_lattice* lat, const hea_objective* obj, const hea_search_params* params,
                      uint8_t* types, int32_t* counts, hea_search_result* result, void* stream);

/*
 * Batched search: n independent cells (any lattice, size, species and shell count) in one call,
 * one CTA per cell, cells ordered largest first.  Two steps, so that the launch itself reads only
 * device memory (and can be captured in a CUDA graph):
 *   1. hea_search_batch_plan() validates every cell and writes a plan of hea_search_batch_plan_bytes(n)
 *      bytes into host memory `plan_host`;
 *   2. the caller copies those bytes to device memory `plan_dev` and calls hea_search_batch().
 * plan_host must stay unchanged between the two calls; plan_dev must hold the copied plan until
 * the launched work completes.
 *   lats[n], objs[n], params[n]     host arrays
 *   types[n], counts[n]             host arrays of device pointers (as for hea_search)
 *   results                         device hea_search_result[n]
 */
size_t hea_search_batch_plan_bytes(int n);
hea_status hea_search_batch_plan(int n, const hea_lattice* const* lats, const hea_objective* objs,
                                 const hea_search_params* params, uint8_t* const* types, int32_t* const* counts,
                                 hea_search_result* results, void* plan_host);
hea_status hea_search_batch(const void* plan_host, const void* plan_dev, void* stream);

/*
 * Cooperative search: one chain run by `ctas` co-resident CTAs, one per SM, each holding a copy
 * of the cell in shared memory.  The K candidates of a step are split into ctas equal slices;
 * each CTA scores its slice and publishes its best candidates (records) through `workspace`, every
 * CTA reads all records once each CTA's tag for the step is visible, and every CTA applies the same
 * accepted swaps.  Results are those of hea_search with the same parameters:
 *   best-of-K (accept_mode 0): identical to hea_search for any K;
 *   multi-accept (accept_mode 1): requires group_size = K / ctas, 1 <= group_top <= 4 and
 *   ctas * group_top <= 640, and is then identical to hea_search with those group parameters.
 *   workspace        device memory of at least hea_search_coop_workspace_bytes(ctas) bytes,
 *                    16-byte aligned, owned by the caller; its first (header and tag) bytes are
 *                    zeroed on `stream` before the launch; calls that share a workspace must not
 *                    overlap
 * Errors: HEA_EINVAL for bad parameters or a short workspace; HEA_ENOMEM when `ctas` CTAs with
 * this cell cannot all be resident (see hea_search_coop_max_ctas).  Each wait for another CTA's
 * records is bounded (params->sync_wait_us, default 2 s); a wait that runs out ends the search with
 * status HEA_ESYNC in the result (the state written back is the one before the unfinished step).
 */
size_t hea_search_coop_workspace_bytes(int ctas);
/* Most CTAs that can be co-resident for this problem with `ctas`-way splitting (0 on error). */
int hea_search_coop_max_ctas(const hea_lattice* lat, const hea_objective* obj, const hea_search_params* params,
                             int ctas);
hea_status hea_search_coop(const hea_lattice* lat, const hea_objective* obj, const hea_search_params* params,
                           int ctas, uint8_t* types, int32_t* counts, hea_search_result* result, void* workspace,
                           size_t workspace_bytes, void* stream);

/*
 * hea_search_coop without caller memory, for callers that cannot allocate device memory (a
 * process whose device memory belongs to another runtime's allocator, a plugin host that forbids
 * cudaMalloc, a deployment with a fixed device-memory budget).  The paper has no counterpart: the
 * exchange area of the cooperative search lives in a fixed array of HEA_NOALLOC_SCRATCH_BYTES
 * bytes inside the library's device image, held by every GPU that loads the library until the
 * process exits.  Nothing is allocated.
 *   - ctas must be at most HEA_NOALLOC_MAX_CTAS; larger requests return HEA_EINVAL before any
 *     launch.
 *   - The array is shared by every call on a device and keeps the last call's contents; each call
 *     clears the header and tag words on `stream` before launching.  Calls that overlap on the GPU
 *     race on the array: serialise them.
 *   - The first call on a device (with that device current) looks up the array's address once per
 *     CUDA context; make that first call before any stream capture.  After a device reset the next
 *     call looks the address up again.
 * Other arguments, results and errors: as hea_search_coop.
 */
#define HEA_NOALLOC_MAX_CTAS 512
#define HEA_NOALLOC_SCRATCH_BYTES 344064
hea_status hea_search_coop_noalloc(const hea_lattice* lat, const hea_objective* obj, const hea_search_params* params,
                                   int ctas, uint8_t* types, int32_t* counts, hea_search_result* result, void* stream);

/* Message for the last error returned on the calling thread ("" if none). */
/*
 * External structure onto the lattice (Sec. 2.3, application workflow: a structure relaxed or
 * simulated by an external tool is analysed to give the target SRO of a larger search; follow
 * with hea_sro_counts and hea_sro_alpha).  Atom i at Cartesian position xyz[i] (length unit of
 * the cubic lattice constant a; the cell's origin at origin[]) goes to the nearest lattice site:
 * X = round(2 (x - origin_x) / a) taken modulo 2 Lx, likewise Y and Z, which is a site when its
 * parities match the lattice (FCC: X + Y + Z even; BCC: all three equal).  types[site] receives
 * species[i].  Counted in report (device int64[4], overwritten):
 *   report[0]  atoms farther than tol half-lattice units (tol * a / 2) from that point, or whose
 *              rounded point is not a site of this lattice (left unassigned)
 *   report[1]  sites taken by more than one atom
 *   report[2]  sites taken by no atom (their types entry is 0)
 *   report[3]  atoms whose species is outside 0..S-1
 * The mapping is valid when all four are 0.
 *   xyz      device double[n][3];  species device uint8[n]
 *   types    device uint8[N], out
 *   scratch  device int32[N] (per-site claim counts)
 *   origin   host double[3]
 * Errors: HEA_EINVAL for n < 1, S outside 1..255, a <= 0, tol outside [0, 0.5] or non-finite
 * origin; positions beyond 2^30 half units of the origin count as off-lattice.
 */
hea_status hea_map_structure(const hea_lattice* lat, int64_t n, const double* xyz, const uint8_t* species, int S,
                             double a, const double* origin, double tol, uint8_t* types, int32_t* scratch,
                             int64_t* report, void* stream);

/*
 * Global search (Sec. 4.1, Alg. global_search; the parameter ranges and the precision and
 * performance presets are those of Sec. 2.1, parameter optimization): a pool of solutions ranked by
 * fitness, the best refined by the parallel Monte Carlo search, the worst fraction discarded.
 * Iteration g (0-based) of G:
 *   1. pool = the n_keep solutions kept from iteration g-1 (none when g = 0), best first, then
 *      P - (kept) fresh random configurations; fresh one j starts from the initial configuration
 *      of hea_init_config with the 64-bit seed (r1 << 32) | r0 of Philox counter (j, g, 0, 4)
 *      under the key (lo32(seed), hi32(seed));
 *   2. F^2 of every fresh solution from a full recount;
 *   3. the n_refine best of the pool by (F^2, pool index) are selected ("top solutions");
 *   4. selected solution r is refined by the search of hea_search (K = tasks, accept_mode,
 *      depth_limit, max_steps, seed, chain g * 65536 + r, step0 0, depth0 0);
 *   5. the refined solutions are ranked by (F^2, r) and the best n_keep are kept; the others are
 *      discarded (the fraction p_a = 1 - n_keep / n_refine; n_keep <= n_refine / 2 keeps at most
 *      half, so at least half of every later refined set is new).
 * The output is iteration G-1's refined set, ranked best first.  Every step runs on the device
 * on `stream` (no host synchronisation inside the call, so it can be captured in a CUDA graph).
 */
typedef struct {
    int32_t n_solutions;  /* P: solutions ranked per iteration, 1..4096 */
    int32_t n_refine;     /* solutions refined per iteration, 1..P */
    int32_t n_keep;       /* refined solutions kept for the next iteration, 0..n_refine/2 */
    int32_t iterations;   /* G: 1..65536 */
    int32_t tasks;        /* candidate swaps per Monte Carlo step, 1..4096 */
    int32_t depth_limit;  /* a refinement ends after this many consecutive steps without an accepted swap, >= 1 */
    int64_t max_steps;    /* step cap of one refinement, 1..2^32 */
    uint64_t seed;        /* Philox key of the fresh solutions and of every refinement */
    int32_t accept_mode;  /* 0: best-of-K (Alg. parallel_mc); 1: non-overlapping multi-accept */
    int32_t reserved;     /* must be 0 */
} hea_global_params;

/* One record per (iteration, refined slot). */
typedef struct {
    int32_t origin;    /* pool index the slot was selected from (below the kept count: kept solution of that rank) */
    int32_t pad;
    double f2_in;      /* F^2 before the refinement */
    double f2_out;     /* F^2 after the refinement */
    int64_t steps;     /* Monte Carlo steps of the refinement */
    int64_t accepted;  /* swaps it accepted */
} hea_global_log;

typedef struct {
    int64_t steps;       /* Monte Carlo steps, summed over every refinement */
    int64_t trials;      /* candidates scored, summed */
    int64_t accepted;    /* swaps accepted, summed */
    int32_t iterations;  /* iterations run (= G) */
    int32_t status;      /* HEA_OK */
    double best_f2;      /* F^2 of the best solution */
    double best_f;       /* sqrt(best_f2) */
} hea_global_result;

/* Workspace for hea_global_search: the pool (P configurations with their counts and F^2), the
 * selection order and the refinement descriptors.  0 for invalid arguments. */
size_t hea_global_search_workspace_bytes(const hea_lattice* lat, const hea_objective* obj,
                                         const hea_global_params* params);

/*
 *   types      device uint8[n_refine][N], out: the final refined set, best first
 *   counts     device int32[n_refine][M][S][S], out: their counts
 *   f2         device double[n_refine], out: their F^2
 *   log        device hea_global_log[G][n_refine], out (NULL = not written)
 *   result     device (or host-mapped) hea_global_result, out
 *   workspace  device memory of at least hea_global_search_workspace_bytes() bytes, 256-byte
 *              aligned, owned by the caller; calls sharing a workspace must not overlap
 * Errors: HEA_EINVAL for parameters outside the ranges above or a short or misaligned workspace;
 * HEA_ENOMEM when a cell with `tasks` candidate slots does not fit one CTA (as for hea_search).
 */
hea_status hea_global_search(const hea_lattice* lat, const hea_objective* obj, const hea_global_params* params,
                             uint8_t* types, int32_t* counts, double* f2, hea_global_log* log,
                             hea_global_result* result, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Measurement aid (not part of the search): the single-byte shared-memory gather rate of this GPU,
 * the ceiling of the swap scoring's neighbour gathers.  Launches `ctas` CTAs of 512 threads, each
 * holding a 64 KiB buffer in shared memory; every thread performs iters * 8 one-byte loads.
 *   mode 0: random addresses (as the scoring's gathers are);  mode 1: lane l reads bank l.
 *   sink: device uint64[2], caller-zeroed; sink[1] counts finished CTAs.
 * Time the call with events; bytes gathered = ctas * 512 * 8 * iters.
 */
hea_status hea_probe_smem_gather(int mode, int ctas, int64_t iters, uint64_t* sink, void* stream);

const char* hea_last_error(void);
const char* hea_status_string(int status);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* HEA_H */
