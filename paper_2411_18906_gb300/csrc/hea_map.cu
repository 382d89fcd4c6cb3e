// hea_map.cu -- an external structure onto the lattice (Sec. 2.3, application workflow): each
// atom is rounded to the nearest half-unit lattice point, which must be a site of the lattice;
// per-site claim counts find sites taken twice or not at all.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "hea_internal.h"

namespace hea {

struct MapGeom {
    int kind, L[3];
    double inv_half;  // 2 / a
    double origin[3];
    double tol2;      // squared tolerance in half units
};

__device__ __forceinline__ long long wrap_ll(long long x, long long p) {
    const long long r = x % p;
    return r < 0 ? r + p : r;
}

__global__ void map_atoms_kernel(const MapGeom g, int64_t n, const double* __restrict__ xyz,
                                 const uint8_t* __restrict__ species, int S, uint8_t* __restrict__ types,
                                 int32_t* __restrict__ claims, unsigned long long* __restrict__ report) {
    unsigned long long off = 0, bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        long long P[3];
        double d2 = 0.0;
        bool ok = true;
        for (int c = 0; c < 3; ++c) {
            const double u = (xyz[3 * i + c] - g.origin[c]) * g.inv_half;
            if (!(fabs(u) < 1073741824.0)) {   // also false for NaN
                ok = false;
                P[c] = 0;
                continue;
            }
            const double r = rint(u);
            d2 += (u - r) * (u - r);
            P[c] = wrap_ll((long long)r, 2LL * g.L[c]);
        }
        if (ok && d2 > g.tol2) ok = false;
        int b = 0;
        if (ok) {
            const int px = (int)(P[0] & 1), py = (int)(P[1] & 1), pz = (int)(P[2] & 1);
            if (g.kind == HEA_FCC) {
                if (((px + py + pz) & 1) != 0) ok = false;
                // basis (0,0,0), (0,1,1), (1,0,1), (1,1,0): the odd x-parity picks 2 or 3
                b = px ? (py ? 3 : 2) : (py ? 1 : 0);
            } else {
                if (px != py || py != pz) ok = false;
                b = px;
            }
        }
        if (!ok) {
            ++off;
            continue;
        }
        const uint8_t sp = species[i];
        if (sp >= S) ++bad;
        const int64_t site = (((int64_t)b * g.L[2] + (P[2] >> 1)) * g.L[1] + (P[1] >> 1)) * g.L[0] + (P[0] >> 1);
        atomicAdd(&claims[site], 1);
        types[site] = sp;
    }
    if (off) atomicAdd(&report[0], off);
    if (bad) atomicAdd(&report[3], bad);
}

__global__ void map_sites_kernel(int64_t N, const int32_t* __restrict__ claims, uint8_t* __restrict__ types,
                                 unsigned long long* __restrict__ report) {
    unsigned long long twice = 0, empty = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = claims[s];
        if (c > 1) ++twice;
        if (c == 0) {
            ++empty;
            types[s] = 0;
        }
    }
    if (twice) atomicAdd(&report[1], twice);
    if (empty) atomicAdd(&report[2], empty);
}

cudaError_t launch_map_structure(int kind, int Lx, int Ly, int Lz, int64_t n, const double* xyz, const uint8_t* species,
                                 int S, double a, const double* origin, double tol, uint8_t* types, int32_t* scratch,
                                 int64_t* report, cudaStream_t stream) {
    const int64_t N = (int64_t)(kind == HEA_FCC ? 4 : 2) * Lx * Ly * Lz;
    MapGeom g{};
    g.kind = kind;
    g.L[0] = Lx;
    g.L[1] = Ly;
    g.L[2] = Lz;
    g.inv_half = 2.0 / a;
    for (int c = 0; c < 3; ++c) g.origin[c] = origin[c];
    g.tol2 = tol * tol;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int32_t) * (size_t)N, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(report, 0, 4 * sizeof(int64_t), stream);
    if (e != cudaSuccess) return e;
    auto blocks = [](int64_t m) { return (int)std::min<int64_t>((m + 255) / 256, 152 * 16); };
    unsigned long long* rep = reinterpret_cast<unsigned long long*>(report);
    map_atoms_kernel<<<blocks(n), 256, 0, stream>>>(g, n, xyz, species, S, types, scratch, rep);
    map_sites_kernel<<<blocks(N), 256, 0, stream>>>(N, scratch, types, rep);
    return cudaGetLastError();
}

}  // namespace hea
