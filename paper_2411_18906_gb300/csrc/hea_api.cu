// hea_api.cu -- the C entry points of libhea (declared in include/hea.h): argument validation on
// the host, descriptor set-up, kernel launches.  No device memory is allocated here.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "hea_device.cuh"
#include "hea_internal.h"

struct hea_lattice {
    int kind, Lx, Ly, Lz, M;
    int64_t N;
    int Z[hea::kMaxShells];
};

namespace {

thread_local char g_err[512] = "";

hea_status fail(hea_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

hea_status ok() {
    g_err[0] = '\0';
    return HEA_OK;
}

hea_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ok();
    return fail(HEA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

hea_status check_objective(const hea_lattice* lat, const hea_objective* obj) {
    if (!obj) return fail(HEA_EINVAL, "objective is NULL");
    if (obj->S < 2 || obj->S > HEA_MAX_SPECIES) return fail(HEA_EINVAL, "S = %d outside [2, %d]", obj->S, HEA_MAX_SPECIES);
    if (obj->M != lat->M) return fail(HEA_EINVAL, "objective M = %d but lattice has %d shells", obj->M, lat->M);
    if (!obj->n_per || !obj->w || !obj->target) return fail(HEA_EINVAL, "objective array is NULL");
    int64_t total = 0;
    for (int i = 0; i < obj->S; ++i) {
        if (obj->n_per[i] < 1) return fail(HEA_EINVAL, "species %d has %lld sites; alpha needs N_i >= 1", i, (long long)obj->n_per[i]);
        total += obj->n_per[i];
    }
    if (total != lat->N) return fail(HEA_EINVAL, "composition sums to %lld, lattice has %lld sites", (long long)total, (long long)lat->N);
    for (int k = 0; k < obj->M; ++k)
        if (!std::isfinite(obj->w[k]) || std::signbit(obj->w[k])) return fail(HEA_EINVAL, "weight w[%d] must be finite and >= +0", k);
    for (int e = 0; e < obj->M * obj->S * obj->S; ++e)
        if (!std::isfinite(obj->target[e])) return fail(HEA_EINVAL, "target[%d] is not finite", e);
    return ok();
}

void fill_desc(const hea_lattice* lat, const hea_objective* obj, hea::ChainDesc* d) {
    std::memset(d, 0, sizeof *d);
    d->kind = lat->kind;
    d->Lx = lat->Lx;
    d->Ly = lat->Ly;
    d->Lz = lat->Lz;
    d->M = lat->M;
    d->S = obj->S;
    d->N = (int32_t)lat->N;
    for (int i = 0; i < obj->S; ++i) d->n_per[i] = obj->n_per[i];
    for (int k = 0; k < obj->M; ++k) d->w[k] = obj->w[k];
    for (int e = 0; e < obj->M * obj->S * obj->S; ++e) d->target[e] = obj->target[e];
}

hea_status check_params(const hea_lattice* lat, const hea_search_params* p) {
    if (!p) return fail(HEA_EINVAL, "search params are NULL");
    if (p->K < 1) return fail(HEA_EINVAL, "K = %d < 1", p->K);
    if (p->accept_mode != 0 && p->accept_mode != 1) return fail(HEA_EINVAL, "accept_mode must be 0 or 1");
    if (p->max_steps < 0) return fail(HEA_EINVAL, "max_steps < 0");
    if ((uint64_t)p->step0 + (uint64_t)p->max_steps > (1ull << 32)) return fail(HEA_EINVAL, "step0 + max_steps exceeds the 32-bit step counter");
    if (p->depth_limit < 0 || p->max_accept < 0 || p->depth0 < 0) return fail(HEA_EINVAL, "negative depth_limit, max_accept or depth0");
    if (p->group_size < 0 || p->group_top < 0) return fail(HEA_EINVAL, "negative group_size or group_top");
    if (!(p->threshold >= 0.0) || !std::isfinite(p->threshold)) return fail(HEA_EINVAL, "threshold must be finite and >= 0");
    if (p->threads != 0 && p->threads != 128 && p->threads != 256 && p->threads != 512)
        return fail(HEA_EINVAL, "threads = %d must be 0, 128, 256 or 512", p->threads);
    if (p->sync_wait_us < 0) return fail(HEA_EINVAL, "sync_wait_us < 0");
    if (p->test_withhold_cta < 0) return fail(HEA_EINVAL, "test_withhold_cta < 0");
    if (p->timeout_us < 0) return fail(HEA_EINVAL, "timeout_us < 0");
    (void)lat;
    return ok();
}

// Chooses 8-, 4- or (at most 4 species) 2-bit species storage so that the chain's shared memory (the cell plus `qcap`
// candidate slots) fits one CTA, preferring room for the pairwise multi-accept walk over ranked
// lists of up to `walk_cap` candidates.
hea_status place_chain(const hea_lattice* lat, int S, const hea_search_params* p, int qcap, hea::ChainDesc* d,
                       int walk_cap = -1) {
    const int E = lat->M * S * S;
    int cap = walk_cap < 0 ? qcap : walk_cap;
    if (cap > hea::kPairWalkMax) cap = hea::kPairWalkMax;
    if (E > 255 || p->accept_mode != 1) cap = 0;
    // The pairwise walk keeps site positions as int16 half-unit coordinates.
    if (2 * std::max(lat->Lx, std::max(lat->Ly, lat->Lz)) > 32767) cap = 0;
    for (int pc : {cap, 0}) {
        for (int bits : {8, 4, 2}) {
            if (bits == 2 && S > 4) continue;
            const hea::ChainLayout L = hea::chain_layout((int)lat->N, lat->M, S, qcap, bits, p->accept_mode, pc);
            if (L.total + 2048 <= hea::kSearchSmemLimit) {
                d->bits = bits;
                d->smem_bytes = L.total;
                d->qcap = qcap;
                d->pair_cap = pc;
                return ok();
            }
        }
    }
    return fail(HEA_ENOMEM, "cell of %lld sites with %d candidate slots does not fit one CTA's shared memory",
                (long long)lat->N, qcap);
}

// Cooperative chain: K = ctas * Kc; multi-accept needs group_size = Kc and 1 <= group_top <= 4.
hea_status check_coop(const hea_search_params* p, int ctas, int* Kc_out, int* top_out) {
    if (p->threads != 0) return fail(HEA_EINVAL, "threads must be 0 for a cooperative search (512 threads per CTA)");
    if (ctas < 1 || ctas > 65535) return fail(HEA_EINVAL, "ctas = %d outside [1, 65535]", ctas);
    if (p->K % ctas != 0) return fail(HEA_EINVAL, "K = %d is not a multiple of ctas = %d", p->K, ctas);
    const int Kc = p->K / ctas;
    const int most = (p->accept_mode == 1) ? hea::kCoopMaxKc : hea::kMaxK;
    if (Kc > most) return fail(HEA_EINVAL, "K / ctas = %d exceeds %d", Kc, most);
    int top = 1;
    if (p->accept_mode == 1) {
        if (p->group_size != Kc)
            return fail(HEA_EINVAL, "cooperative multi-accept needs group_size = K / ctas = %d (got %d)", Kc, p->group_size);
        if (p->group_top < 1 || p->group_top > hea::kCoopMaxTop)
            return fail(HEA_EINVAL, "cooperative multi-accept needs 1 <= group_top <= %d", hea::kCoopMaxTop);
        top = p->group_top;
        if (ctas * top > hea::kPairWalkMax)
            return fail(HEA_EINVAL, "cooperative multi-accept merges ctas * group_top = %d records; at most %d", ctas * top,
                        hea::kPairWalkMax);
    }
    *Kc_out = Kc;
    *top_out = top;
    return ok();
}

void fill_params(const hea_search_params* p, hea::ChainDesc* d) {
    d->K = p->K;
    d->accept_mode = p->accept_mode;
    d->depth_limit = p->depth_limit;
    d->max_accept = p->max_accept;
    d->chain = p->chain;
    d->step0 = p->step0;
    d->depth0 = p->depth0;
    d->group_size = p->group_size;
    d->group_top = p->group_top;
    d->max_steps = p->max_steps;
    d->timeout_ns = p->timeout_us * 1000;
    d->seed = p->seed;
    d->threshold = p->threshold;
    d->wait_ns = (p->sync_wait_us > 0 ? (int64_t)p->sync_wait_us : 2000000ll) * 1000;
    d->withhold = p->test_withhold_cta;
    d->threads = p->threads > 0 ? p->threads : hea::kChainThreads;
}

// Cooperative chain: the chain arrays, the fixed-point tables and the walk over `nrec` merged
// records in one CTA's shared memory.  Multi-accept scores a CTA's slice in chunks (the best
// candidates so far are carried from chunk to chunk), so the candidate slots hold one chunk plus
// the carried ones: the largest chunk of 1024, 512 or 256 (at most Kc) that fits, with the widest
// species storage (8, 4, or for at most 4 species 2 bits per site).  Best-of-K scores the slice at
// once.
hea_status place_coop(const hea_lattice* lat, int S, const hea_search_params* p, int Kc, int ctas, int top,
                      hea::ChainDesc* d) {
    const int nrec = ctas * top;
    const int chunks[3] = {1024, 512, 256};
    for (int ci = 0; ci < 3; ++ci) {
        const int chunk = (p->accept_mode == 1) ? std::min(Kc, chunks[ci]) : Kc;
        if (p->accept_mode == 1 && ci > 0 && chunk == std::min(Kc, chunks[ci - 1])) continue;
        const int qcap = std::max((p->accept_mode == 1) ? chunk + top : chunk, nrec);
        for (int bits : {8, 4, 2}) {
            if (bits == 2 && S > 4) continue;
            const hea::ChainLayout L = hea::coop_layout((int)lat->N, lat->M, S, qcap, bits, p->accept_mode, nrec);
            if (L.total + 2048 <= hea::kSearchSmemLimit) {
                d->bits = bits;
                d->smem_bytes = L.total;
                d->qcap = qcap;
                d->pair_cap = 0;
                d->nrec = nrec;
                d->chunk = chunk;
                return ok();
            }
        }
        if (p->accept_mode != 1) break;
    }
    return fail(HEA_ENOMEM, "cell of %lld sites with %d merged records does not fit one CTA's shared memory",
                (long long)lat->N, nrec);
}

// Global search: parameter ranges (see hea.h) and the search parameters of every refinement.
hea_status check_global(const hea_lattice* lat, const hea_objective* obj, const hea_global_params* gp,
                        hea_search_params* sp) {
    if (!lat || !gp) return fail(HEA_EINVAL, "NULL argument");
    hea_status st = check_objective(lat, obj);
    if (st != HEA_OK) return st;
    if (gp->n_solutions < 1 || gp->n_solutions > hea::kGlobalMaxSolutions)
        return fail(HEA_EINVAL, "n_solutions = %d outside [1, %d]", gp->n_solutions, hea::kGlobalMaxSolutions);
    if (gp->n_refine < 1 || gp->n_refine > gp->n_solutions)
        return fail(HEA_EINVAL, "n_refine = %d outside [1, n_solutions = %d]", gp->n_refine, gp->n_solutions);
    if (gp->n_keep < 0 || 2 * gp->n_keep > gp->n_refine)
        return fail(HEA_EINVAL, "n_keep = %d outside [0, n_refine / 2]", gp->n_keep);
    if (gp->iterations < 1 || gp->iterations > 65536) return fail(HEA_EINVAL, "iterations = %d outside [1, 65536]", gp->iterations);
    if (gp->tasks < 1 || gp->tasks > hea::kMaxK) return fail(HEA_EINVAL, "tasks = %d outside [1, %d]", gp->tasks, hea::kMaxK);
    if (gp->depth_limit < 1) return fail(HEA_EINVAL, "depth_limit must be >= 1");
    if (gp->max_steps < 1 || gp->max_steps > (int64_t)1 << 32) return fail(HEA_EINVAL, "max_steps outside [1, 2^32]");
    if (gp->accept_mode != 0 && gp->accept_mode != 1) return fail(HEA_EINVAL, "accept_mode must be 0 or 1");
    if (gp->reserved != 0) return fail(HEA_EINVAL, "reserved field must be 0");
    std::memset(sp, 0, sizeof *sp);
    sp->K = gp->tasks;
    sp->accept_mode = gp->accept_mode;
    sp->max_steps = gp->max_steps;
    sp->depth_limit = gp->depth_limit;
    sp->seed = gp->seed;
    return check_params(lat, sp);
}

// Plan = header + descriptors sorted into launch groups by (lattice kind, threads per CTA), each
// group largest work first.
constexpr int kThreadChoices = 3;   // 128, 256, 512 threads per CTA
int thread_group(int threads) { return threads <= 128 ? 0 : (threads <= 256 ? 1 : 2); }
struct PlanHeader {
    uint64_t magic;
    int32_t n;
    int32_t pad;
    int32_t n_group[2][kThreadChoices];     // cells per (kind, threads) group
    uint32_t smem_max[2][kThreadChoices];   // dynamic shared memory per group
};
constexpr uint64_t kPlanMagic = 0x6865615F706C616EULL;  // "hea_plan"

size_t plan_offset() { return hea::align_up(sizeof(PlanHeader), 256); }

}  // namespace

namespace hea {
hea_status set_last_error(hea_status status, const char* message) { return fail(status, "%s", message); }
}  // namespace hea

extern "C" {

const char* hea_last_error(void) { return g_err; }

const char* hea_status_string(int status) {
    switch (status) {
        case HEA_OK: return "ok";
        case HEA_EINVAL: return "invalid argument";
        case HEA_ENOMEM: return "does not fit on chip";
        case HEA_ECUDA: return "CUDA error";
        case HEA_ETIMEOUT: return "time budget reached";
        case HEA_EMISMATCH: return "consistency check failed";
        case HEA_ESYNC: return "a wait for another CTA ran out";
        default: return "unknown status";
    }
}

hea_status hea_build_lattice(int kind, int Lx, int Ly, int Lz, int n_shells, hea_lattice** out) {
    if (!out) return fail(HEA_EINVAL, "out is NULL");
    *out = nullptr;
    if (kind != HEA_FCC && kind != HEA_BCC) return fail(HEA_EINVAL, "kind must be HEA_FCC or HEA_BCC");
    if (Lx < 2 || Ly < 2 || Lz < 2) return fail(HEA_EINVAL, "each of Lx, Ly, Lz must be >= 2");
    if (n_shells < 1 || n_shells > HEA_MAX_SHELLS) return fail(HEA_EINVAL, "n_shells must be in [1, %d]", HEA_MAX_SHELLS);
    const int64_t N = (int64_t)(kind == HEA_FCC ? 4 : 2) * Lx * Ly * Lz;
    if (N > HEA_MAX_SITES) return fail(HEA_EINVAL, "%lld sites exceed the limit of %d", (long long)N, HEA_MAX_SITES);
    hea_lattice* lat = new (std::nothrow) hea_lattice;
    if (!lat) return fail(HEA_ENOMEM, "host allocation failed");
    lat->kind = kind;
    lat->Lx = Lx;
    lat->Ly = Ly;
    lat->Lz = Lz;
    lat->M = n_shells;
    lat->N = N;
    constexpr hea::ShellTable fcc = hea::build_shell_table(hea::kFCC);
    constexpr hea::ShellTable bcc = hea::build_shell_table(hea::kBCC);
    for (int k = 0; k < hea::kMaxShells; ++k) lat->Z[k] = (kind == HEA_FCC) ? fcc.z[k] : bcc.z[k];
    *out = lat;
    return ok();
}

void hea_lattice_destroy(hea_lattice* lat) { delete lat; }

int64_t hea_num_sites(const hea_lattice* lat) { return lat ? lat->N : -1; }

int hea_num_shells(const hea_lattice* lat) { return lat ? lat->M : -1; }

int hea_shell_size(const hea_lattice* lat, int k) {
    if (!lat || k < 1 || k > lat->M) return 0;
    return lat->Z[k - 1];
}

hea_status hea_init_config(const hea_lattice* lat, int S, const int64_t* n_per, uint64_t seed, uint8_t* types,
                           void* stream) {
    if (!lat || !n_per || !types) return fail(HEA_EINVAL, "NULL argument");
    if (S < 1 || S > 255) return fail(HEA_EINVAL, "S = %d outside [1, 255]", S);
    std::vector<int64_t> cum(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        if (n_per[s] < 0) return fail(HEA_EINVAL, "n_per[%d] < 0", s);
        cum[s + 1] = cum[s] + n_per[s];
    }
    if (cum[S] != lat->N) return fail(HEA_EINVAL, "composition sums to %lld, lattice has %lld sites", (long long)cum[S], (long long)lat->N);
    if (S > 8 && lat->N > (1 << 16)) return fail(HEA_EINVAL, "more than 8 species is supported only up to 65536 sites");
    return cuda_status(hea::launch_init_config(lat->kind, lat->Lx, lat->Ly, lat->Lz, S, cum.data(), seed, types,
                                               as_stream(stream)),
                       "hea_init_config launch");
}

hea_status hea_sro_counts_method(const hea_lattice* lat, int n_configs, const uint8_t* types, int S, int32_t* counts,
                                 int method, void* stream) {
    if (!lat || !types || !counts) return fail(HEA_EINVAL, "NULL argument");
    if (S < 1 || S > HEA_MAX_SPECIES) return fail(HEA_EINVAL, "S = %d outside [1, %d]", S, HEA_MAX_SPECIES);
    if (n_configs < 1 || n_configs > 65535) return fail(HEA_EINVAL, "n_configs = %d outside [1, 65535]", n_configs);
    if (method < 0 || method > 2) return fail(HEA_EINVAL, "method = %d outside [0, 2]", method);
    if (method == 2 && !hea::sro_counts_planes_apply(lat->kind, lat->Lx, lat->Ly, lat->Lz, lat->M, S))
        return fail(HEA_EINVAL, "the bit-plane recount needs Lx <= 64, 2 <= S <= 6 and its planes in shared memory");
    return cuda_status(hea::launch_sro_counts(lat->kind, lat->Lx, lat->Ly, lat->Lz, lat->M, S, n_configs, types,
                                              counts, method, as_stream(stream)),
                       "hea_sro_counts launch");
}

hea_status hea_sro_counts(const hea_lattice* lat, int n_configs, const uint8_t* types, int S, int32_t* counts,
                          void* stream) {
    return hea_sro_counts_method(lat, n_configs, types, S, counts, 0, stream);
}

hea_status hea_sro_alpha(const hea_lattice* lat, const hea_objective* obj, const int32_t* counts, double* alpha,
                         double* f2, void* stream) {
    if (!lat || !counts || !alpha || !f2) return fail(HEA_EINVAL, "NULL argument");
    hea_status st = check_objective(lat, obj);
    if (st != HEA_OK) return st;
    hea::ChainDesc d;
    fill_desc(lat, obj, &d);
    return cuda_status(hea::launch_sro_alpha(d, counts, alpha, f2, as_stream(stream)), "hea_sro_alpha launch");
}

hea_status hea_delta_swap(const hea_lattice* lat, const hea_objective* obj, const uint8_t* types,
                          const int32_t* counts, const int64_t* pairs, int64_t K, double* key, int32_t* dcounts,
                          void* stream) {
    if (!lat || !types || !counts || !pairs || !key) return fail(HEA_EINVAL, "NULL argument");
    if (K < 1 || K > (int64_t)1 << 31) return fail(HEA_EINVAL, "K = %lld outside [1, 2^31]", (long long)K);
    hea_status st = check_objective(lat, obj);
    if (st != HEA_OK) return st;
    hea::ChainDesc d;
    fill_desc(lat, obj, &d);
    return cuda_status(hea::launch_delta_swap(d, types, counts, pairs, K, key, dcounts, as_stream(stream)),
                       "hea_delta_swap launch");
}

hea_status hea_search(const hea_lattice* lat, const hea_objective* obj, const hea_search_params* params,
                      uint8_t* types, int32_t* counts, hea_search_result* result, void* stream) {
    if (!lat || !types || !counts || !result) return fail(HEA_EINVAL, "NULL argument");
    hea_status st = check_objective(lat, obj);
    if (st != HEA_OK) return st;
    st = check_params(lat, params);
    if (st != HEA_OK) return st;
    if (params->K > hea::kMaxK) return fail(HEA_EINVAL, "K = %d exceeds %d for a single-CTA chain", params->K, hea::kMaxK);
    if (params->test_withhold_cta != 0) return fail(HEA_EINVAL, "test_withhold_cta applies to cooperative searches only");
    hea::ChainDesc d;
    fill_desc(lat, obj, &d);
    fill_params(params, &d);
    st = place_chain(lat, obj->S, params, params->K, &d);
    if (st != HEA_OK) return st;
    d.types = types;
    d.counts = counts;
    d.result = result;
    d.ctas = 1;
    const cudaError_t e = (d.kind == HEA_FCC) ? hea::launch_search_fcc(d, as_stream(stream))
                                              : hea::launch_search_bcc(d, as_stream(stream));
    return cuda_status(e, "hea_search launch");
}

size_t hea_search_batch_plan_bytes(int n) {
    if (n < 1) return 0;
    return plan_offset() + sizeof(hea::ChainDesc) * (size_t)n;
}

hea_status hea_search_batch_plan(int n, const hea_lattice* const* lats, const hea_objective* objs,
                                 const hea_search_params* params, uint8_t* const* types, int32_t* const* counts,
                                 hea_search_result* results, void* plan_host) {
    if (n < 1 || n > 65535) return fail(HEA_EINVAL, "n = %d outside [1, 65535]", n);
    if (!lats || !objs || !params || !types || !counts || !results || !plan_host) return fail(HEA_EINVAL, "NULL argument");
    std::vector<hea::ChainDesc> descs((size_t)n);
    for (int c = 0; c < n; ++c) {
        if (!lats[c] || !types[c] || !counts[c]) return fail(HEA_EINVAL, "cell %d: NULL lattice or buffer", c);
        hea_status st = check_objective(lats[c], &objs[c]);
        if (st == HEA_OK) st = check_params(lats[c], &params[c]);
        if (st == HEA_OK && params[c].K > hea::kMaxK) st = fail(HEA_EINVAL, "K = %d exceeds %d", params[c].K, hea::kMaxK);
        if (st == HEA_OK && params[c].test_withhold_cta != 0)
            st = fail(HEA_EINVAL, "test_withhold_cta applies to cooperative searches only");
        if (st == HEA_OK) {
            fill_desc(lats[c], &objs[c], &descs[c]);
            fill_params(&params[c], &descs[c]);
            st = place_chain(lats[c], objs[c].S, &params[c], params[c].K, &descs[c]);
            descs[c].ctas = 1;
        }
        if (st != HEA_OK) {
            char msg[512];
            std::snprintf(msg, sizeof msg, "cell %d: %s", c, g_err);
            return fail(st, "%s", msg);
        }
        descs[c].types = types[c];
        descs[c].counts = counts[c];
        descs[c].result = results + c;
    }
    // Largest cells first, so that the hardware block scheduler hands the longest chains out first.
    std::stable_sort(descs.begin(), descs.end(), [](const hea::ChainDesc& a, const hea::ChainDesc& b) {
        if (a.kind != b.kind) return a.kind < b.kind;
        if (a.threads != b.threads) return a.threads < b.threads;
        return (int64_t)a.N * a.K > (int64_t)b.N * b.K;
    });
    PlanHeader h{};
    h.magic = kPlanMagic;
    h.n = n;
    for (const auto& d : descs) {
        const int g = thread_group(d.threads);
        h.n_group[d.kind][g] += 1;
        h.smem_max[d.kind][g] = std::max(h.smem_max[d.kind][g], d.smem_bytes);
    }
    std::memset(plan_host, 0, plan_offset());
    std::memcpy(plan_host, &h, sizeof h);
    std::memcpy(static_cast<char*>(plan_host) + plan_offset(), descs.data(), sizeof(hea::ChainDesc) * descs.size());
    return ok();
}

hea_status hea_search_batch(const void* plan_host, const void* plan_dev, void* stream) {
    if (!plan_host || !plan_dev) return fail(HEA_EINVAL, "NULL plan");
    PlanHeader h;
    std::memcpy(&h, plan_host, sizeof h);
    if (h.magic != kPlanMagic || h.n < 1) return fail(HEA_EINVAL, "plan_host is not a plan written by hea_search_batch_plan");
    const hea::ChainDesc* descs = reinterpret_cast<const hea::ChainDesc*>(static_cast<const char*>(plan_dev) + plan_offset());
    cudaStream_t s = as_stream(stream);
    static const int threads_of[kThreadChoices] = {128, 256, 512};
    int first = 0;
    for (int kind = 0; kind < 2; ++kind)
        for (int g = 0; g < kThreadChoices; ++g) {
            const int cnt = h.n_group[kind][g];
            if (cnt == 0) continue;
            const cudaError_t e = (kind == HEA_FCC)
                                      ? hea::launch_search_batch_fcc(descs + first, cnt, h.smem_max[kind][g], threads_of[g], s)
                                      : hea::launch_search_batch_bcc(descs + first, cnt, h.smem_max[kind][g], threads_of[g], s);
            hea_status st = cuda_status(e, "hea_search_batch launch");
            if (st != HEA_OK) return st;
            first += cnt;
        }
    return ok();
}

size_t hea_search_coop_workspace_bytes(int ctas) { return ctas < 1 ? 0 : hea::coop_workspace_bytes(ctas); }

int hea_search_coop_max_ctas(const hea_lattice* lat, const hea_objective* obj, const hea_search_params* params,
                             int ctas) {
    if (!lat) return 0;
    if (check_objective(lat, obj) != HEA_OK || check_params(lat, params) != HEA_OK) return 0;
    int Kc = 0, top = 1;
    if (check_coop(params, ctas, &Kc, &top) != HEA_OK) return 0;
    hea::ChainDesc d;
    fill_desc(lat, obj, &d);
    fill_params(params, &d);
    if (place_coop(lat, obj->S, params, Kc, ctas, top, &d) != HEA_OK) return 0;
    return (d.kind == HEA_FCC) ? hea::coop_max_ctas_fcc(d) : hea::coop_max_ctas_bcc(d);
}

hea_status hea_search_coop(const hea_lattice* lat, const hea_objective* obj, const hea_search_params* params,
                           int ctas, uint8_t* types, int32_t* counts, hea_search_result* result, void* workspace,
                           size_t workspace_bytes, void* stream) {
    if (!lat || !types || !counts || !result || !workspace) return fail(HEA_EINVAL, "NULL argument");
    hea_status st = check_objective(lat, obj);
    if (st != HEA_OK) return st;
    st = check_params(lat, params);
    if (st != HEA_OK) return st;
    int Kc = 0, top = 1;
    st = check_coop(params, ctas, &Kc, &top);
    if (st != HEA_OK) return st;
    if (workspace_bytes < hea::coop_workspace_bytes(ctas))
        return fail(HEA_EINVAL, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
                    hea::coop_workspace_bytes(ctas));
    if (reinterpret_cast<uintptr_t>(workspace) % 16 != 0) return fail(HEA_EINVAL, "workspace is not 16-byte aligned");
    if (params->test_withhold_cta > ctas) return fail(HEA_EINVAL, "test_withhold_cta names a CTA beyond ctas");
    hea::ChainDesc d;
    fill_desc(lat, obj, &d);
    fill_params(params, &d);
    st = place_coop(lat, obj->S, params, Kc, ctas, top, &d);
    if (st != HEA_OK) return st;
    const int most = (d.kind == HEA_FCC) ? hea::coop_max_ctas_fcc(d) : hea::coop_max_ctas_bcc(d);
    if (most < 1) return fail(HEA_ECUDA, "no CUDA device for a cooperative launch");
    if (ctas > most) return fail(HEA_ENOMEM, "%d CTAs cannot be co-resident with %u bytes of shared memory each (at most %d)",
                                 ctas, d.smem_bytes, most);
    d.types = types;
    d.counts = counts;
    d.result = result;
    d.ctas = ctas;
    d.workspace = workspace;
    const cudaError_t e = (d.kind == HEA_FCC) ? hea::launch_search_coop_fcc(d, as_stream(stream))
                                              : hea::launch_search_coop_bcc(d, as_stream(stream));
    return cuda_status(e, "hea_search_coop launch");
}

hea_status hea_probe_smem_gather(int mode, int ctas, int64_t iters, uint64_t* sink, void* stream) {
    if (mode != 0 && mode != 1) return fail(HEA_EINVAL, "mode must be 0 (random) or 1 (one bank per lane)");
    if (ctas < 1 || ctas > 65535 || iters < 1 || !sink) return fail(HEA_EINVAL, "bad ctas, iters or sink");
    return cuda_status(hea::launch_smem_gather_probe(mode, ctas, iters, reinterpret_cast<unsigned long long*>(sink),
                                                     as_stream(stream)),
                       "hea_probe_smem_gather launch");
}

hea_status hea_map_structure(const hea_lattice* lat, int64_t n, const double* xyz, const uint8_t* species, int S,
                             double a, const double* origin, double tol, uint8_t* types, int32_t* scratch,
                             int64_t* report, void* stream) {
    if (!lat || !xyz || !species || !origin || !types || !scratch || !report) return fail(HEA_EINVAL, "NULL argument");
    if (n < 1) return fail(HEA_EINVAL, "n = %lld < 1", (long long)n);
    if (S < 1 || S > 255) return fail(HEA_EINVAL, "S = %d outside [1, 255]", S);
    if (!(a > 0.0) || !std::isfinite(a)) return fail(HEA_EINVAL, "lattice constant a must be finite and > 0");
    if (!(tol >= 0.0 && tol <= 0.5)) return fail(HEA_EINVAL, "tol must be in [0, 0.5] half-lattice units");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(origin[c])) return fail(HEA_EINVAL, "origin is not finite");
    return cuda_status(hea::launch_map_structure(lat->kind, lat->Lx, lat->Ly, lat->Lz, n, xyz, species, S, a, origin,
                                                 tol, types, scratch, report, as_stream(stream)),
                       "hea_map_structure launch");
}

size_t hea_global_search_workspace_bytes(const hea_lattice* lat, const hea_objective* obj,
                                         const hea_global_params* params) {
    hea_search_params sp;
    if (check_global(lat, obj, params, &sp) != HEA_OK) return 0;
    const hea::GlobalLayout L = hea::global_layout(params->n_solutions, params->n_refine, lat->N,
                                                   lat->M * obj->S * obj->S);
    return L.total;
}

hea_status hea_global_search(const hea_lattice* lat, const hea_objective* obj, const hea_global_params* gp,
                             uint8_t* types, int32_t* counts, double* f2, hea_global_log* log,
                             hea_global_result* result, void* workspace, size_t workspace_bytes, void* stream) {
    if (!types || !counts || !f2 || !result || !workspace) return fail(HEA_EINVAL, "NULL argument");
    hea_search_params sp;
    hea_status st = check_global(lat, obj, gp, &sp);
    if (st != HEA_OK) return st;
    const int P = gp->n_solutions, PL = gp->n_refine, R = gp->n_keep, G = gp->iterations, S = obj->S;
    const int64_t N = lat->N;
    const int E = lat->M * S * S;
    const hea::GlobalLayout L = hea::global_layout(P, PL, N, E);
    if (workspace_bytes < L.total)
        return fail(HEA_EINVAL, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(HEA_EINVAL, "workspace is not 256-byte aligned");
    hea::ChainDesc d;
    fill_desc(lat, obj, &d);
    fill_params(&sp, &d);
    st = place_chain(lat, S, &sp, sp.K, &d);
    if (st != HEA_OK) return st;
    d.ctas = 1;
    std::vector<int64_t> cum(S + 1, 0);
    for (int s = 0; s < S; ++s) cum[s + 1] = cum[s] + obj->n_per[s];

    char* ws = static_cast<char*>(workspace);
    uint8_t* pool_types = reinterpret_cast<uint8_t*>(ws + L.types);
    int32_t* pool_counts = reinterpret_cast<int32_t*>(ws + L.counts);
    double* pool_f2 = reinterpret_cast<double*>(ws + L.f2);
    int32_t* order = reinterpret_cast<int32_t*>(ws + L.order);
    hea::ChainDesc* descs = reinterpret_cast<hea::ChainDesc*>(ws + L.descs);
    hea_search_result* res = reinterpret_cast<hea_search_result*>(ws + L.results);
    cudaStream_t s = as_stream(stream);

    cudaError_t e = cudaMemsetAsync(result, 0, sizeof *result, s);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        const int kept = (g == 0) ? 0 : R;
        const int fresh = P - kept;
        hea_global_log* lg = log ? log + (size_t)g * PL : nullptr;
        // 1-2: fresh random solutions after the kept ones, their counts and F^2.
        if (fresh > 0) {
            e = hea::launch_init_fresh(lat->kind, lat->Lx, lat->Ly, lat->Lz, S, cum.data(), gp->seed, (uint32_t)g, 0u,
                                       fresh, pool_types + (size_t)kept * N, s);
            if (e == cudaSuccess)
                e = hea::launch_sro_counts(lat->kind, lat->Lx, lat->Ly, lat->Lz, lat->M, S, fresh,
                                           pool_types + (size_t)kept * N, pool_counts + (size_t)kept * E, 0, s);
            if (e == cudaSuccess) e = hea::launch_sro_alpha(d, pool_counts + (size_t)kept * E, nullptr, pool_f2 + kept, s, fresh);
        }
        // 3: the best n_refine into the output slots.
        if (e == cudaSuccess) e = hea::launch_global_select(pool_f2, P, PL, order, lg, s);
        if (e == cudaSuccess)
            e = hea::launch_global_gather(pool_types, pool_counts, pool_f2, nullptr, order, PL, types, counts, f2, N, E, s);
        // 4: one refinement chain per slot.
        if (e == cudaSuccess) e = hea::launch_global_descs(d, descs, PL, types, counts, res, N, E, (uint32_t)g * 65536u, s);
        if (e == cudaSuccess)
            e = (d.kind == HEA_FCC) ? hea::launch_search_batch_fcc(descs, PL, d.smem_bytes, d.threads, s)
                                    : hea::launch_search_batch_bcc(descs, PL, d.smem_bytes, d.threads, s);
        // 5: rank the refined set, keep it in rank order at the front of the pool.
        if (e == cudaSuccess) e = hea::launch_global_rank(res, PL, order, lg, result, s);
        if (e == cudaSuccess)
            e = hea::launch_global_gather(types, counts, nullptr, res, order, PL, pool_types, pool_counts, pool_f2, N, E, s);
    }
    if (e == cudaSuccess)
        e = hea::launch_global_gather(pool_types, pool_counts, pool_f2, nullptr, nullptr, PL, types, counts, f2, N, E, s);
    if (e == cudaSuccess) e = hea::launch_global_finish(pool_f2, G, result, s);
    return cuda_status(e, "hea_global_search launch");
}

}  // extern "C"
