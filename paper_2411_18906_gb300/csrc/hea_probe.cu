// hea_probe.cu -- measurement aid: the rate at which all SMs gather single bytes from shared
// memory, the ceiling of the swap scoring (each scored candidate gathers the species bytes of its
// two sites' neighbours from the cell held in shared memory).  Over a 64 KiB buffer:
//   mode 0: each thread follows 8 independent linear congruential streams of random byte
//           addresses (lanes collide in banks as random addresses do);
//   mode 1: each iteration picks a random 1 KiB row; lane l reads byte 4l of each of its eight
//           128-byte segments (lane l always in bank l: one wavefront per warp-wide load).
#include <cstdint>
#include <cuda_runtime.h>

#include "hea_internal.h"

namespace hea {

constexpr int kProbeThreads = 512;
constexpr uint32_t kProbeBytes = 64 * 1024;

template <int MODE>
__global__ void __launch_bounds__(kProbeThreads) smem_gather_probe(int64_t iters, uint32_t seed,
                                                                   unsigned long long* __restrict__ sink) {
    extern __shared__ __align__(16) uint8_t buf[];
    uint32_t* w = reinterpret_cast<uint32_t*>(buf);
    for (uint32_t i = threadIdx.x; i < kProbeBytes / 4; i += blockDim.x) w[i] = i * 2654435761u + seed;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    uint32_t x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (blockIdx.x * blockDim.x + threadIdx.x) * 8u + (uint32_t)j + seed;
    uint32_t acc = 0;
    for (int64_t it = 0; it < iters; ++it) {
        if (MODE == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                x[j] = x[j] * 1664525u + 1013904223u;
                acc += buf[x[j] >> 16];
            }
        } else {
            // one random row of 8 x 128 bytes per iteration; lane l reads byte 4l of each 128
            x[0] = x[0] * 1664525u + 1013904223u;
            const uint8_t* row = buf + (((x[0] >> 16) & (kProbeBytes - 1024u)) | (lane << 2));
#pragma unroll
            for (int j = 0; j < 8; ++j) acc += row[128 * j];
        }
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;   // keeps the loads live; practically never taken
    if (threadIdx.x == 0) atomicAdd(&sink[1], 1ull);
}

cudaError_t launch_smem_gather_probe(int mode, int ctas, int64_t iters, unsigned long long* sink,
                                     cudaStream_t stream) {
    cudaError_t e;
    if (mode == 0) {
        e = cudaFuncSetAttribute(smem_gather_probe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeBytes);
        if (e == cudaSuccess) smem_gather_probe<0><<<ctas, kProbeThreads, kProbeBytes, stream>>>(iters, 12345u, sink);
    } else {
        e = cudaFuncSetAttribute(smem_gather_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeBytes);
        if (e == cudaSuccess) smem_gather_probe<1><<<ctas, kProbeThreads, kProbeBytes, stream>>>(iters, 12345u, sink);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e;
    }
    return cudaGetLastError();
}

}  // namespace hea
