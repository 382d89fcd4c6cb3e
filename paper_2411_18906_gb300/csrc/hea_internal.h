// hea_internal.h -- descriptors shared between libhea's host entry points and its kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include "hea.h"

namespace hea {

constexpr int kChainThreads = 256;   // threads of a single-CTA search chain (default)
constexpr int kChainMaxThreads = 512;
constexpr int kCoopThreads = 512;    // threads of each CTA of a cooperative chain
constexpr int kMaxK = 4096;          // candidates per CTA per step (cooperative multi-accept: per chunk)
constexpr int kGlobalMaxSolutions = 4096;  // global search: largest pool
constexpr int kCoopMaxKc = 1 << 20;  // cooperative multi-accept: candidates per CTA per step
constexpr int kCoopMaxTop = 4;       // records (best eligible candidates) per CTA per step
constexpr int kPairWalkMax = 640;    // longest ranked list the pairwise multi-accept walk handles
constexpr uint32_t kSearchSmemLimit = 227 * 1024;

// Everything one search chain needs, passed by value (single chain) or from device memory
// (batched search).  Objective tables are copied in so a launch reads no host memory.
struct ChainDesc {
    int32_t kind, Lx, Ly, Lz, M, S, N, bits;  // bits: species storage, 8, 4 or 2 per site
    int32_t K, accept_mode, depth_limit, max_accept;
    uint32_t chain, step0;
    int32_t depth0, group_size, group_top, ctas;
    int32_t pair_cap, pad2;   // multi-accept: longest ranked list the pairwise walk can hold
    int64_t max_steps;
    int64_t timeout_ns;
    uint64_t seed;
    double threshold;
    int64_t n_per[8];
    double w[5];
    double target[5 * 8 * 8];
    uint8_t* types;
    int32_t* counts;
    hea_search_result* result;
    void* workspace;        // cooperative chain: exchange area (see CoopHeader)
    uint32_t smem_bytes;
    int32_t qcap;           // candidate slots in shared memory
    int64_t wait_ns;        // cooperative chain: limit of each wait for the other CTAs' records
    int32_t withhold;       // cooperative chain, testing aid: 1 + index of a CTA that never publishes (0 = none)
    int32_t nrec;           // cooperative chain: most records merged per step (ctas * records per CTA)
    int32_t chunk;          // cooperative multi-accept: candidates scored per pass (the slice is scored in chunks)
    int32_t threads;        // threads per CTA of the single-CTA and batched chains
};

// Shared-memory layout of one search CTA (offsets in bytes from the dynamic smem base).
struct ChainLayout {
    uint32_t types, cnt, Q, tgt, ca, cb, fa, fb, fQ, fe0, dn, tiny, beta, vec, slot;
    uint32_t qk, qa, qb, qlo, qhi, qD, qkey, qg, order, acc, bitmap, fw;
    // cooperative chain only: fixed-point coefficient tables, per-slot fixed-point keys, walk data
    uint32_t fA, fB, qfix, qeps, qflag, walk;
    uint32_t total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// The site grid that finds conflicting candidates: at most 2048 bins (list heads), then per site
// its next pointer and its packed bin coordinates.
constexpr uint32_t kConflictBins = 2048;

// Scratch shared by the conflict grid (before the walk's batches) and the batch data.
__host__ __device__ inline uint32_t scratch_bytes(int n, uint32_t E) {
    const uint32_t batch = align_up(32 * ((E + 3) & ~3u), 16) + 2 * 32 * 32 * 4 + 4 * 32 * 4;
    const uint32_t hash = 4 * kConflictBins + 8 * 2 * (uint32_t)n;   // heads, next pointers, site bins
    return batch > hash ? batch : hash;
}

// Bytes of the pairwise-walk data for a ranked list of up to n candidates: per candidate its
// nonzero count changes (2 bytes each, M (4S - 4) at most), its count, its two sites' coordinates
// (6 int16), its row of the conflict matrix (ceil(n / 32) words) and its sites and species; then
// the scratch of one batch of 32 candidates.
__host__ __device__ inline uint32_t pair_walk_bytes(int n, int M, int S) {
    const uint32_t mp = (uint32_t)(M * (4 * S - 4));
    const uint32_t nw = (uint32_t)((n + 31) / 32);
    const uint32_t E = (uint32_t)(M * S * S);
    return align_up((uint32_t)n * 2 * mp, 16) + align_up((uint32_t)n, 16) + align_up((uint32_t)n * 12, 16) +
           align_up((uint32_t)n * 4 * nw, 16) + align_up((uint32_t)n * 10, 16) +
           // batch scratch of the walk: dense count changes (int8 [32][E rounded up to 4]), cross
           // terms and their bounds (float [32][32] each), estimates, their bounds and the conflict
           // information of the batch's candidates ([32] each)
           scratch_bytes(n, E);
}

// qcap: candidate slots (the candidates a CTA scores per step, or the merged records of a
// cooperative chain, whichever is larger).  pair_cap: longest ranked list the pairwise walk
// handles (0 = always the bitmap walk); its data shares memory with the site bitmap.
__host__ __device__ inline ChainLayout chain_layout(int N, int M, int S, int qcap, int bits, int accept_mode,
                                                   int pair_cap = 0) {
    ChainLayout L{};
    const uint32_t E = (uint32_t)(M * S * S);
    const uint32_t C = (uint32_t)qcap;
    uint32_t o = 0;
    L.types = o;
    o = align_up(o + (bits == 8 ? (uint32_t)N : (bits == 4 ? (uint32_t)(N + 1) / 2 : (uint32_t)(N + 3) / 4)), 16);
    L.cnt = o;    o = align_up(o + 4 * E, 16);
    L.Q = o;      o = align_up(o + 8 * E, 16);
    L.tgt = o;    o = align_up(o + 8 * E, 16);
    L.ca = o;     o = align_up(o + 8 * E, 16);
    L.cb = o;     o = align_up(o + 8 * E, 16);
    L.fa = o;     o = align_up(o + 4 * E, 16);
    L.fb = o;     o = align_up(o + 4 * E, 16);
    L.fQ = o;     o = align_up(o + 4 * E, 16);
    L.fe0 = o;    o = align_up(o + 4 * E, 16);
    L.dn = o;     o = align_up(o + 4 * E, 16);
    L.tiny = o;   o = align_up(o + 4 * E, 16);
    L.beta = o;   o = align_up(o + 4 * E, 16);
    L.vec = o;    o = align_up(o + 4 * 96, 16);
    L.slot = o;   o = align_up(o + 2 * 5 * 28, 16);
    L.fw = o;     o = align_up(o + 4 * E, 16);
    L.qk = o;     o = align_up(o + 4 * C, 16);
    L.qa = o;     o = align_up(o + 4 * C, 16);
    L.qb = o;     o = align_up(o + 4 * C, 16);
    L.qlo = o;    o = align_up(o + 4 * C, 16);
    L.qhi = o;    o = align_up(o + 4 * C, 16);
    L.qD = o;     o = align_up(o + 8 * C, 16);
    L.qkey = o;   o = align_up(o + 8 * C, 16);
    L.qg = o;     o = align_up(o + 8 * C * (uint32_t)M, 16);
    L.order = o;  o = align_up(o + 4 * C, 16);
    L.acc = o;    o = align_up(o + 4 * C, 16);
    if (accept_mode == 1) {
        L.bitmap = o;
        const uint32_t bm = 4 * (uint32_t)((N + 31) / 32);
        const uint32_t pw = pair_cap > 0 ? pair_walk_bytes(pair_cap, M, S) : 0u;
        o = align_up(o + (bm > pw ? bm : pw), 16);
    } else {
        L.bitmap = o;
    }
    L.total = o;
    return L;
}

// Data of the multi-accept walk of a cooperative chain over at most `nrec` ranked candidates (E
// entries, rows of Ep = E rounded up to 4): dense count changes int8 [nrec][Ep], sites u32
// [nrec][2], species u8 [nrec][2], positions int16 [nrec][6], the conflict matrix u32
// [nrec][ceil(nrec / 32)], per-entry totals int32 [Ep], accepted-record and scratch masks u32
// [2][ceil(nrec / 32)], conflicting pairs u32 [2 nrec], two occupancy bitmaps of hashed conventional cells (kCoopCellBits bits
// each), suspect sites u16 [2 nrec], then one batch of 32: rows float [32][Ws] x 2 (Ws: Ep padded
// to 4 mod 8), cross terms, their bounds and three prefix-sum tables float [32][33] x 5, keys and
// bounds float [32] x 2, conflict masks u32 [32] x 2.  The device-side pointers (coop_walk_arrays)
// follow this order.
constexpr int kCoopCellBits = 16;
constexpr uint32_t kCoopCellWords = (1u << kCoopCellBits) / 32u;

__host__ __device__ inline uint32_t coop_walk_bytes(int nrec, int E) {
    const uint32_t n = (uint32_t)nrec, Ep = ((uint32_t)E + 3u) & ~3u;
    const uint32_t Ws = (Ep % 8u == 4u) ? Ep : Ep + 4u;   // batch row stride (floats)
    const uint32_t nw = (n + 31u) / 32u;
    return align_up(n * Ep, 16) + align_up(8 * n, 16) + align_up(2 * n, 16) + align_up(12 * n, 16) +
           align_up(4 * n * nw, 16) + align_up(4 * Ep, 16) + align_up(8 * nw, 16) + align_up(8 * n, 16) +
           2 * 4 * kCoopCellWords +
           align_up(4 * n, 16) + 2 * 4 * 32 * Ws +
           5 * 4 * 32 * 33 + 2 * 4 * 32 + 2 * 4 * 32;
}

// Shared memory of a cooperative chain: the arrays of a chain (without the single-chain walk
// data) followed by the fixed-point tables, per-slot keys and the walk data.
__host__ __device__ inline ChainLayout coop_layout(int N, int M, int S, int qcap, int bits, int accept_mode, int nrec) {
    ChainLayout L = chain_layout(N, M, S, qcap, bits, 0, 0);
    const uint32_t E = (uint32_t)(M * S * S), C = (uint32_t)qcap;
    uint32_t o = L.total;
    L.fA = o;     o = align_up(o + 8 * E, 16);
    L.fB = o;     o = align_up(o + 8 * E, 16);
    L.qfix = o;   o = align_up(o + 8 * C, 16);
    L.qeps = o;   o = align_up(o + 8 * C, 16);
    L.qflag = o;  o = align_up(o + 4 * C, 16);
    L.walk = o;
    if (accept_mode == 1) o = align_up(o + coop_walk_bytes(nrec, (int)E), 16);
    L.total = o;
    return L;
}

// Exchange area of a cooperative chain (caller-provided device memory): a header, then for each
// of two step parities and each CTA a tag word, then for each parity and CTA up to kCoopMaxTop
// candidate records.  CTA r publishes step s (counted from 0 in each launch) by writing its records
// and the tag ((s + 1) << 32) | (stop << 16) | count, then adding 1 (release) to the arrival
// counter of the step's parity.  A CTA reads the records of step s once that counter reaches
// ctas * (s / 2 + 1) (acquire): one polling thread per CTA on one word.  Only CTA 0 sets `stop`
// (time budget spent), so every CTA takes the same stop decision for the same step.
struct CoopHeader {
    int32_t error;              // a wait for another CTA's records ran out
    uint32_t arrive[2];         // CTAs that published, per step parity (cumulative over the launch)
    int32_t pad[13];
};

struct CoopRecord {
    double D;        // binary64 key (best-of-K: always; multi-accept: when flags & 1)
    float lo, hi;    // FP32 interval around the key (multi-accept)
    uint32_t k, a, b, flags;
    uint64_t g[5];   // per-shell swap vectors (biased bytes)
};

// Byte offsets inside the exchange area of a chain of `ctas` CTAs.
__host__ __device__ inline size_t coop_tags_offset() { return sizeof(CoopHeader); }
__host__ __device__ inline size_t coop_records_offset(int ctas) {
    return (coop_tags_offset() + 2 * sizeof(unsigned long long) * (size_t)ctas + 63) / 64 * 64;
}
__host__ __device__ inline size_t coop_workspace_bytes(int ctas) {
    return coop_records_offset(ctas) + 2 * (size_t)ctas * kCoopMaxTop * sizeof(CoopRecord);
}

// Global search workspace: the pool (P configurations, counts, F^2), the selection order, the
// refinement descriptors and results; each part 256-byte aligned.
struct GlobalLayout {
    size_t types, counts, f2, order, descs, results, total;
};
inline GlobalLayout global_layout(int P, int PL, int64_t N, int E) {
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    GlobalLayout L{};
    L.types = 0;
    L.counts = up((size_t)P * (size_t)N);
    L.f2 = L.counts + up((size_t)P * E * sizeof(int32_t));
    L.order = L.f2 + up((size_t)P * sizeof(double));
    L.descs = L.order + up((size_t)P * sizeof(int32_t));
    L.results = L.descs + up((size_t)PL * sizeof(ChainDesc));
    L.total = L.results + up((size_t)PL * sizeof(hea_search_result));
    return L;
}

// Records `message` as the calling thread's hea_last_error() text and returns `status`.
hea_status set_last_error(hea_status status, const char* message);

// Launchers implemented in the .cu files.
cudaError_t launch_init_config(int kind, int Lx, int Ly, int Lz, int S, const int64_t* cum, uint64_t seed,
                               uint8_t* types, cudaStream_t stream);
cudaError_t launch_init_fresh(int kind, int Lx, int Ly, int Lz, int S, const int64_t* cum, uint64_t seed,
                              uint32_t g, uint32_t j0, int n, uint8_t* types, cudaStream_t stream);
cudaError_t launch_sro_counts(int kind, int Lx, int Ly, int Lz, int M, int S, int n_configs, const uint8_t* types,
                              int32_t* counts, int method, cudaStream_t stream);
bool sro_counts_planes_apply(int kind, int Lx, int Ly, int Lz, int M, int S);
cudaError_t launch_sro_alpha(const ChainDesc& d, const int32_t* counts, double* alpha, double* f2,
                             cudaStream_t stream, int n_configs = 1);
cudaError_t launch_delta_swap(const ChainDesc& d, const uint8_t* types, const int32_t* counts,
                              const int64_t* pairs, int64_t K, double* key, int32_t* dcounts, cudaStream_t stream);
cudaError_t launch_search_fcc(const ChainDesc& d, cudaStream_t stream);
cudaError_t launch_search_bcc(const ChainDesc& d, cudaStream_t stream);
cudaError_t launch_search_batch_fcc(const ChainDesc* descs_dev, int n, uint32_t smem_max, int threads,
                                    cudaStream_t stream);
cudaError_t launch_search_batch_bcc(const ChainDesc* descs_dev, int n, uint32_t smem_max, int threads,
                                    cudaStream_t stream);
cudaError_t launch_search_coop_fcc(const ChainDesc& d, cudaStream_t stream);
cudaError_t launch_search_coop_bcc(const ChainDesc& d, cudaStream_t stream);
cudaError_t launch_map_structure(int kind, int Lx, int Ly, int Lz, int64_t n, const double* xyz, const uint8_t* species,
                                 int S, double a, const double* origin, double tol, uint8_t* types, int32_t* scratch,
                                 int64_t* report, cudaStream_t stream);
cudaError_t launch_smem_gather_probe(int mode, int ctas, int64_t iters, unsigned long long* sink,
                                     cudaStream_t stream);
cudaError_t launch_global_select(const double* pool_f2, int P, int PL, int32_t* order, hea_global_log* log,
                                 cudaStream_t stream);
cudaError_t launch_global_rank(const hea_search_result* res, int PL, int32_t* order, hea_global_log* log,
                               hea_global_result* total, cudaStream_t stream);
cudaError_t launch_global_gather(const uint8_t* src_types, const int32_t* src_counts, const double* src_f2,
                                 const hea_search_result* src_res, const int32_t* order, int n, uint8_t* dst_types,
                                 int32_t* dst_counts, double* dst_f2, int64_t N, int E, cudaStream_t stream);
cudaError_t launch_global_descs(const ChainDesc& d, ChainDesc* descs, int n, uint8_t* types, int32_t* counts,
                                hea_search_result* results, int64_t N, int E, uint32_t chain_base,
                                cudaStream_t stream);
cudaError_t launch_global_finish(const double* best_f2, int G, hea_global_result* total, cudaStream_t stream);
int coop_max_ctas_fcc(const ChainDesc& d);
int coop_max_ctas_bcc(const ChainDesc& d);

}  // namespace hea
