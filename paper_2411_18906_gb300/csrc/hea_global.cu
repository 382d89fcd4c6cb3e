// hea_global.cu -- pool kernels of the global search (Sec. 4.1, Alg. global_search): ranking by
// (F^2, index), moving solutions between the pool and the refined set, the descriptors of the
// refinement chains and the totals.  The pool is small (at most 4096 solutions), so ranking is a
// one-CTA all-pairs count: entry i's rank is the number of entries ordered before it.
#include <cstdint>
#include <cuda_runtime.h>

#include "hea_internal.h"

namespace hea {

constexpr int kPoolThreads = 1024;

// Rank of entry i: #{j : key_j < key_i, or key_j == key_i and j < i}.  Keys are finite F^2 values.
__device__ __forceinline__ int pool_rank(const double* key, int n, int i) {
    const double ki = key[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        const double kj = key[j];
        rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
    }
    return rank;
}

// Step 3: the n_refine best pool entries; order[rank] = pool index.
__global__ void __launch_bounds__(kPoolThreads) global_select_kernel(const double* __restrict__ pool_f2, int P, int PL,
                                                                     int32_t* __restrict__ order,
                                                                     hea_global_log* __restrict__ log) {
    __shared__ double key[kGlobalMaxSolutions];
    for (int i = threadIdx.x; i < P; i += blockDim.x) key[i] = pool_f2[i];
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int r = pool_rank(key, P, i);
        if (r < PL) {
            order[r] = i;
            if (log) {
                log[r].origin = i;
                log[r].pad = 0;
                log[r].f2_in = key[i];
            }
        }
    }
}

// Step 5: ranks the refined slots by (F^2, slot) into order[], logs each slot and adds the
// refinements' steps, trials and accepted swaps to the totals.
__global__ void __launch_bounds__(kPoolThreads) global_rank_kernel(const hea_search_result* __restrict__ res, int PL,
                                                                   int32_t* __restrict__ order,
                                                                   hea_global_log* __restrict__ log,
                                                                   hea_global_result* __restrict__ total) {
    __shared__ double key[kGlobalMaxSolutions];
    __shared__ unsigned long long part[3][kPoolThreads / 32];
    unsigned long long st = 0, tr = 0, ac = 0;
    for (int r = threadIdx.x; r < PL; r += blockDim.x) {
        key[r] = res[r].f2;
        st += (unsigned long long)res[r].steps;
        tr += (unsigned long long)res[r].trials;
        ac += (unsigned long long)res[r].accepted;
        if (log) {
            log[r].f2_out = res[r].f2;
            log[r].steps = res[r].steps;
            log[r].accepted = res[r].accepted;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        st += __shfl_xor_sync(0xFFFFFFFFu, st, o);
        tr += __shfl_xor_sync(0xFFFFFFFFu, tr, o);
        ac += __shfl_xor_sync(0xFFFFFFFFu, ac, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        part[0][warp] = st;
        part[1][warp] = tr;
        part[2][warp] = ac;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < PL; r += blockDim.x) order[pool_rank(key, PL, r)] = r;
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0, c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += part[0][w];
            b += part[1][w];
            c += part[2][w];
        }
        total->steps += (int64_t)a;
        total->trials += (int64_t)b;
        total->accepted += (int64_t)c;
    }
}

// dst slot r <- src slot order[r] (order NULL: r): N species bytes, E counts and F^2 (from
// src_f2, or from the search results when src_f2 is NULL).  One CTA per destination slot.
__global__ void global_gather_kernel(const uint8_t* __restrict__ src_types, const int32_t* __restrict__ src_counts,
                                     const double* __restrict__ src_f2, const hea_search_result* __restrict__ src_res,
                                     const int32_t* __restrict__ order, uint8_t* __restrict__ dst_types,
                                     int32_t* __restrict__ dst_counts, double* __restrict__ dst_f2, int64_t N, int E) {
    const int r = blockIdx.x;
    const int s = order ? order[r] : r;
    const uint8_t* src = src_types + (size_t)s * N;
    uint8_t* dst = dst_types + (size_t)r * N;
    if ((((uintptr_t)src | (uintptr_t)dst) & 15u) == 0) {
        const int64_t n16 = N >> 4;
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = s4[i];
        for (int64_t i = (n16 << 4) + threadIdx.x; i < N; i += blockDim.x) dst[i] = src[i];
    } else {
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) dst[i] = src[i];
    }
    for (int e = threadIdx.x; e < E; e += blockDim.x) dst_counts[(size_t)r * E + e] = src_counts[(size_t)s * E + e];
    if (threadIdx.x == 0) dst_f2[r] = src_f2 ? src_f2[s] : src_res[s].f2;
}

// Step 4's chains: descriptor r = the template with slot r's buffers and chain chain_base + r.
__global__ void global_descs_kernel(const __grid_constant__ ChainDesc d, ChainDesc* __restrict__ descs,
                                    uint8_t* types, int32_t* counts, hea_search_result* results, int64_t N, int E,
                                    uint32_t chain_base) {
    const int r = blockIdx.x;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&d);
    uint32_t* dst = reinterpret_cast<uint32_t*>(descs + r);
    for (int w = threadIdx.x; w < (int)(sizeof(ChainDesc) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    if (threadIdx.x == 0) {
        descs[r].types = types + (size_t)r * N;
        descs[r].counts = counts + (size_t)r * E;
        descs[r].result = results + r;
        descs[r].chain = chain_base + (uint32_t)r;
    }
}

__global__ void global_finish_kernel(const double* __restrict__ best_f2, int G, hea_global_result* __restrict__ total) {
    total->iterations = G;
    total->status = HEA_OK;
    total->best_f2 = best_f2[0];
    total->best_f = __dsqrt_rn(best_f2[0]);
}

cudaError_t launch_global_select(const double* pool_f2, int P, int PL, int32_t* order, hea_global_log* log,
                                 cudaStream_t stream) {
    global_select_kernel<<<1, kPoolThreads, 0, stream>>>(pool_f2, P, PL, order, log);
    return cudaGetLastError();
}

cudaError_t launch_global_rank(const hea_search_result* res, int PL, int32_t* order, hea_global_log* log,
                               hea_global_result* total, cudaStream_t stream) {
    global_rank_kernel<<<1, kPoolThreads, 0, stream>>>(res, PL, order, log, total);
    return cudaGetLastError();
}

cudaError_t launch_global_gather(const uint8_t* src_types, const int32_t* src_counts, const double* src_f2,
                                 const hea_search_result* src_res, const int32_t* order, int n, uint8_t* dst_types,
                                 int32_t* dst_counts, double* dst_f2, int64_t N, int E, cudaStream_t stream) {
    global_gather_kernel<<<n, 256, 0, stream>>>(src_types, src_counts, src_f2, src_res, order, dst_types, dst_counts,
                                                dst_f2, N, E);
    return cudaGetLastError();
}

cudaError_t launch_global_descs(const ChainDesc& d, ChainDesc* descs, int n, uint8_t* types, int32_t* counts,
                                hea_search_result* results, int64_t N, int E, uint32_t chain_base,
                                cudaStream_t stream) {
    global_descs_kernel<<<n, 128, 0, stream>>>(d, descs, types, counts, results, N, E, chain_base);
    return cudaGetLastError();
}

cudaError_t launch_global_finish(const double* best_f2, int G, hea_global_result* total, cudaStream_t stream) {
    global_finish_kernel<<<1, 1, 0, stream>>>(best_f2, G, total);
    return cudaGetLastError();
}

}  // namespace hea
