// hea_counts.cu -- initial configuration, full Warren-Cowley recount and alpha / F^2 kernels.
#include <cstdint>
#include <cuda_runtime.h>

#include "hea_device.cuh"
#include "hea_internal.h"

namespace hea {

static __constant__ ShellTable c_shells[2] = {build_shell_table(kFCC), build_shell_table(kBCC)};

// ------------------------------------------------------------------------------------------------
// Initial configuration (Sec. 4.1: random first solutions) with an exact composition.
// Site i has the unique key (r0 << 32 | i), r0 = Philox(i, 0, 0, 0).  The site of rank r gets
// species s with cum[s] <= r < cum[s+1], i.e. the number of thresholds T_s (the key of rank
// cum[s], s = 1..S-1) that its key reaches.  The thresholds are found by an MSB-first radix
// select, 8 bits per pass, all S-1 of them in the same passes; keys are regenerated each pass.
// One CTA per cell.
// ------------------------------------------------------------------------------------------------
struct Cum {
    int64_t v[256];
};

__device__ __forceinline__ uint64_t site_key(uint32_t i, uint32_t k0, uint32_t k1) {
    const Rand4 r = philox(i, 0u, 0u, 0u, k0, k1);
    return ((uint64_t)r.r0 << 32) | (uint64_t)i;
}

constexpr int kInitThreads = 1024;
constexpr int kInitMaxThresholds = 7;   // species 2..8 use the fast path

__global__ void __launch_bounds__(kInitThreads) init_config_kernel(uint32_t N, int S, const Cum cum, uint32_t k0,
                                                                   uint32_t k1, uint8_t* __restrict__ types) {
    __shared__ uint32_t hist[kInitMaxThresholds][256];
    __shared__ uint64_t prefix[kInitMaxThresholds];
    __shared__ uint64_t remaining[kInitMaxThresholds];
    __shared__ int active[kInitMaxThresholds];
    const int nt = S - 1;
    const int tid = threadIdx.x;
    if (tid < nt) {
        const int64_t rank = cum.v[tid + 1];
        active[tid] = rank < (int64_t)N;
        prefix[tid] = 0;
        remaining[tid] = (uint64_t)rank;
    }
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int i = tid; i < kInitMaxThresholds * 256; i += blockDim.x) (&hist[0][0])[i] = 0;
        __syncthreads();
        for (uint32_t i = tid; i < N; i += blockDim.x) {
            const uint64_t key = site_key(i, k0, k1);
            const uint32_t digit = (uint32_t)(key >> shift) & 0xFFu;
            for (int s = 0; s < nt; ++s) {
                if (!active[s]) continue;
                if (pass > 0 && (key >> (shift + 8)) != (prefix[s] >> (shift + 8))) continue;
                atomicAdd(&hist[s][digit], 1u);
            }
        }
        __syncthreads();
        if (tid < nt && active[tid]) {
            uint64_t acc = 0;
            for (int dgt = 0; dgt < 256; ++dgt) {
                const uint64_t c = hist[tid][dgt];
                if (remaining[tid] < acc + c) {
                    prefix[tid] |= (uint64_t)dgt << shift;
                    remaining[tid] -= acc;
                    break;
                }
                acc += c;
            }
        }
        __syncthreads();
    }
    for (uint32_t i = tid; i < N; i += blockDim.x) {
        const uint64_t key = site_key(i, k0, k1);
        int sp = 0;
        for (int s = 0; s < nt; ++s) sp += (active[s] && key >= prefix[s]) ? 1 : 0;
        types[i] = (uint8_t)sp;
    }
}

// Many species (S > 8): each site ranks itself against all keys (quadratic; small cells only).
__global__ void init_config_rank_kernel(uint32_t N, int S, const Cum cum, uint32_t k0, uint32_t k1,
                                        uint8_t* __restrict__ types) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint64_t mine = site_key(i, k0, k1);
    uint32_t rank = 0;
    for (uint32_t j = 0; j < N; ++j) rank += site_key(j, k0, k1) < mine ? 1u : 0u;
    int sp = 0;
    while (sp + 1 < S && (int64_t)rank >= cum.v[sp + 1]) ++sp;
    types[i] = (uint8_t)sp;
}

cudaError_t launch_init_config(int kind, int Lx, int Ly, int Lz, int S, const int64_t* cum_host, uint64_t seed,
                               uint8_t* types, cudaStream_t stream) {
    const uint32_t N = (uint32_t)((kind == kFCC ? 4 : 2) * (int64_t)Lx * Ly * Lz);
    Cum cum{};
    for (int s = 0; s <= S && s < 256; ++s) cum.v[s] = cum_host[s];
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    if (S <= kInitMaxThresholds + 1) {
        init_config_kernel<<<1, kInitThreads, 0, stream>>>(N, S, cum, k0, k1, types);
    } else {
        init_config_rank_kernel<<<(N + 255) / 256, 256, 0, stream>>>(N, S, cum, k0, k1, types);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Full recount of N_ij^(k) (Sec. 4.3).  Each thread takes sites, builds the per-shell neighbour
// histogram of its site (8-bit fields per species, neighbours found from coordinates), and adds
// the S fields of each shell to a CTA histogram in shared memory; the CTA histogram is flushed
// to global memory with one atomic per nonzero bin.  grid.y indexes configurations.
// ------------------------------------------------------------------------------------------------
constexpr int kCountThreads = 256;

template <int KIND, int M>
__global__ void __launch_bounds__(kCountThreads) sro_counts_kernel(Geo g, int S, const uint8_t* __restrict__ types,
                                                                   int32_t* __restrict__ counts) {
    extern __shared__ int32_t hist[];
    const int E = M * S * S;
    for (int e = threadIdx.x; e < E; e += blockDim.x) hist[e] = 0;
    __syncthreads();
    const uint8_t* t = types + (size_t)blockIdx.y * (size_t)g.N;
    auto onehot = [&](uint32_t n) -> uint64_t {
        const int y = __ldg(t + n);
        return y < S ? (1ull << (8 * y)) : 0ull;
    };
    for (uint32_t site = blockIdx.x * blockDim.x + threadIdx.x; site < (uint32_t)g.N;
         site += gridDim.x * blockDim.x) {
        const int A = __ldg(t + site);
        if (A >= S) continue;
        uint64_t h[M];
        neighbour_histogram<KIND, M>(g, site, 0xFFFFFFFFu, onehot, h);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            int32_t* row = hist + (k * S + A) * S;
            for (int y = 0; y < S; ++y) {
                const int c = hist_field(h[k], y);
                if (c) atomicAdd(row + y, c);
            }
        }
    }
    __syncthreads();
    int32_t* out = counts + (size_t)blockIdx.y * (size_t)E;
    for (int e = threadIdx.x; e < E; e += blockDim.x)
        if (hist[e]) atomicAdd(out + e, hist[e]);
}

template <int KIND, int M>
static cudaError_t launch_counts_t(const Geo& g, int S, int n_configs, const uint8_t* types, int32_t* counts,
                                   cudaStream_t stream) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    const int per_cfg = (g.N + kCountThreads - 1) / kCountThreads;
    // Enough CTAs to fill the GPU a few times over, but at least one site per thread.
    int bx = per_cfg;
    const int want = (sms * 8 + n_configs - 1) / n_configs;
    if (bx > want) bx = want < 1 ? 1 : want;
    dim3 grid(bx, n_configs);
    const size_t smem = sizeof(int32_t) * M * S * S;
    sro_counts_kernel<KIND, M><<<grid, kCountThreads, smem, stream>>>(g, S, types, counts);
    return cudaGetLastError();
}

cudaError_t launch_sro_counts(int kind, int Lx, int Ly, int Lz, int M, int S, int n_configs, const uint8_t* types,
                              int32_t* counts, cudaStream_t stream) {
    const Geo g = make_geo(kind, Lx, Ly, Lz);
    cudaError_t err = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_configs * M * S * S, stream);
    if (err != cudaSuccess) return err;
#define HEA_COUNTS_CASE(KD, MM) \
    if (kind == KD && M == MM) return launch_counts_t<KD, MM>(g, S, n_configs, types, counts, stream);
    HEA_COUNTS_CASE(kFCC, 1) HEA_COUNTS_CASE(kFCC, 2) HEA_COUNTS_CASE(kFCC, 3) HEA_COUNTS_CASE(kFCC, 4)
    HEA_COUNTS_CASE(kFCC, 5) HEA_COUNTS_CASE(kBCC, 1) HEA_COUNTS_CASE(kBCC, 2) HEA_COUNTS_CASE(kBCC, 3)
    HEA_COUNTS_CASE(kBCC, 4) HEA_COUNTS_CASE(kBCC, 5)
#undef HEA_COUNTS_CASE
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------------
// alpha_ij^(k) = 1 - n Q (Eq. sro, Q = N / ((Z_k N_i) N_j)) and F^2 = sum over (k,i,j) row-major of
// w_k e^2, e = alpha - t (Eq. fitness_function).  One CTA; the sum runs serially in row-major order.
// ------------------------------------------------------------------------------------------------
__global__ void sro_alpha_kernel(const ChainDesc d, const int32_t* __restrict__ counts, double* __restrict__ alpha,
                                 double* __restrict__ f2) {
    __shared__ double term[kMaxEntries];
    const int S = d.S, M = d.M, E = M * S * S;
    const ShellTable& T = c_shells[d.kind];
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int k = e / (S * S), i = (e / S) % S, j = e % S;
        const double den = __dmul_rn(__dmul_rn((double)T.z[k], (double)d.n_per[i]), (double)d.n_per[j]);
        const double Q = __ddiv_rn((double)d.N, den);
        const double a = __dsub_rn(1.0, __dmul_rn((double)counts[e], Q));
        alpha[e] = a;
        const double err = __dsub_rn(a, d.target[e]);
        term[e] = __dmul_rn(d.w[k], __dmul_rn(err, err));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int e = 0; e < E; ++e) s = __dadd_rn(s, term[e]);
        f2[0] = s;
    }
}

cudaError_t launch_sro_alpha(const ChainDesc& d, const int32_t* counts, double* alpha, double* f2,
                             cudaStream_t stream) {
    sro_alpha_kernel<<<1, 128, 0, stream>>>(d, counts, alpha, f2);
    return cudaGetLastError();
}

}  // namespace hea
