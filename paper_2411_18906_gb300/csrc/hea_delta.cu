// hea_delta.cu -- hea_delta_swap: exact count change and key of caller-given candidate swaps
// (Sec. 4.5, Sec. 4.6.2), one thread per pair, species read from global memory.
#include "hea_search.cuh"

namespace hea {

template <int KIND, int M>
__global__ void __launch_bounds__(256) delta_swap_kernel(const __grid_constant__ ChainDesc d,
                                                         const uint8_t* __restrict__ types,
                                                         const int32_t* __restrict__ counts,
                                                         const int64_t* __restrict__ pairs, int64_t K,
                                                         double* __restrict__ key, int32_t* __restrict__ dcounts) {
    __shared__ double s_ca[kMaxEntries], s_cb[kMaxEntries];
    const int S = d.S, E = M * S * S;
    const ShellTable& TAB = c_shells[KIND];
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int k = e / (S * S), i = (e / S) % S, j = e % S;
        const double w = d.w[k];
        const double den = __dmul_rn(__dmul_rn((double)TAB.z[k], (double)d.n_per[i]), (double)d.n_per[j]);
        const double Q = __ddiv_rn((double)d.N, den);
        const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)counts[e], Q)), d.target[e]);
        s_ca[e] = __dmul_rn(w, __dmul_rn(Q, Q));
        s_cb[e] = __dmul_rn(-2.0, __dmul_rn(w, __dmul_rn(Q, err)));
    }
    __syncthreads();
    const Geo g = make_geo(KIND, d.Lx, d.Ly, d.Lz);
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    const int64_t a64 = pairs[2 * c], b64 = pairs[2 * c + 1];
    int32_t* dc = dcounts ? dcounts + c * E : nullptr;
    if (a64 < 0 || a64 >= d.N || b64 < 0 || b64 >= d.N) {
        key[c] = CUDART_NAN;
        if (dc)
            for (int e = 0; e < E; ++e) dc[e] = 0;
        return;
    }
    const uint32_t a = (uint32_t)a64, b = (uint32_t)b64;
    auto onehot = [&](uint32_t n) -> uint64_t {
        const int y = __ldg(types + n);
        return y < S ? (1ull << (8 * y)) : 0ull;
    };
    const int A = __ldg(types + a), B = __ldg(types + b);
    if (a == b || A == B || A >= S || B >= S) {
        key[c] = 0.0;
        if (dc)
            for (int e = 0; e < E; ++e) dc[e] = 0;
        return;
    }
    uint64_t ha[M], hb[M];
    neighbour_histogram_upto<KIND, M>(g, a, b, onehot, ha, M);
    neighbour_histogram_upto<KIND, M>(g, b, a, onehot, hb, M);
    uint64_t gb[M];
#pragma unroll
    for (int k = 0; k < M; ++k) gb[k] = pack_g(ha[k], hb[k]);
    key[c] = exact_key(M, S, s_ca, s_cb, A, B, gb);
    if (dc) {
        for (int e = 0; e < E; ++e) {
            const int k = e / (S * S), i = (e / S) % S, j = e % S;
            dc[e] = entry_delta(gb[k], A, B, i, j);
        }
    }
}

cudaError_t launch_delta_swap(const ChainDesc& d, const uint8_t* types, const int32_t* counts,
                              const int64_t* pairs, int64_t K, double* key, int32_t* dcounts, cudaStream_t stream) {
    const int blocks = (int)((K + 255) / 256);
#define HEA_DELTA_CASE(KD, MM)                                                                               \
    if (d.kind == KD && d.M == MM) {                                                                         \
        delta_swap_kernel<KD, MM><<<blocks, 256, 0, stream>>>(d, types, counts, pairs, K, key, dcounts); \
        return cudaGetLastError();                                                                           \
    }
    HEA_DELTA_CASE(kFCC, 1) HEA_DELTA_CASE(kFCC, 2) HEA_DELTA_CASE(kFCC, 3) HEA_DELTA_CASE(kFCC, 4)
    HEA_DELTA_CASE(kFCC, 5) HEA_DELTA_CASE(kBCC, 1) HEA_DELTA_CASE(kBCC, 2) HEA_DELTA_CASE(kBCC, 3)
    HEA_DELTA_CASE(kBCC, 4) HEA_DELTA_CASE(kBCC, 5)
#undef HEA_DELTA_CASE
    return cudaErrorInvalidValue;
}

}  // namespace hea
