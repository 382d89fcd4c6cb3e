// hea_counts.cu -- initial configuration, full Warren-Cowley recount and alpha / F^2 kernels.
#include <cstdint>
#include <cuda_runtime.h>

#include "hea_device.cuh"
#include "hea_internal.h"

namespace hea {

static __constant__ ShellTable c_shells[2] = {build_shell_table(kFCC), build_shell_table(kBCC)};

// The lexicographically positive half of every shell's vectors (the shells are centrosymmetric).
struct HalfShells {
    int first[kMaxShells + 1];   // index of the first half vector of shell k
    signed char v[48][3];
};

__host__ __device__ constexpr HalfShells build_half_shells(int kind) {
    const ShellTable t = build_shell_table(kind);
    HalfShells h{};
    int n = 0;
    for (int k = 0; k < kMaxShells; ++k) {
        h.first[k] = n;
        for (int v = t.first[k]; v < t.first[k + 1]; ++v) {
            const int x = t.v[v][0], y = t.v[v][1], z = t.v[v][2];
            if (x > 0 || (x == 0 && (y > 0 || (y == 0 && z > 0)))) {
                h.v[n][0] = t.v[v][0];
                h.v[n][1] = t.v[v][1];
                h.v[n][2] = t.v[v][2];
                ++n;
            }
        }
    }
    h.first[kMaxShells] = n;
    return h;
}

static __constant__ HalfShells c_half[2] = {build_half_shells(kFCC), build_half_shells(kBCC)};
static_assert(2 * build_half_shells(kFCC).first[kMaxShells] == build_shell_table(kFCC).first[kMaxShells],
              "every FCC shell splits into two halves");
static_assert(2 * build_half_shells(kBCC).first[kMaxShells] == build_shell_table(kBCC).first[kMaxShells],
              "every BCC shell splits into two halves");

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

constexpr int kInitBins = 4096;    // first pass: histogram of the top 12 key bits
constexpr int kInitBinCap = 256;   // keys of one threshold's bin kept for the exact selection

__device__ void init_config_block(uint32_t N, int S, const Cum& cum, uint32_t k0, uint32_t k1,
                                  uint8_t* __restrict__ types) {
    __shared__ uint32_t hist[kInitMaxThresholds][256];
    __shared__ uint64_t prefix[kInitMaxThresholds];
    __shared__ uint64_t remaining[kInitMaxThresholds];
    __shared__ int active[kInitMaxThresholds];
    // bin counts, then (same memory) the keys of each threshold's bin
    __shared__ __align__(16) uint64_t bins_raw[kInitBins / 2];
    __shared__ uint32_t bin_of[kInitMaxThresholds], in_bin[kInitMaxThresholds];
    __shared__ int overflow;
    const int nt = S - 1;
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid < nt) {
        const int64_t rank = cum.v[tid + 1];
        active[tid] = rank < (int64_t)N;
        prefix[tid] = 0;
        remaining[tid] = (uint64_t)rank;
        in_bin[tid] = 0;
    }
    if (tid == 0) overflow = 0;
    // Two sweeps find the thresholds exactly: the bin (top 12 key bits) holding each threshold's
    // rank, then the keys of that bin, ranked among themselves.  A bin with more keys than the
    // buffer holds (never for random keys at these sizes) sends the block to the radix select below.
    uint32_t* bins = reinterpret_cast<uint32_t*>(bins_raw);
    for (int b = tid; b < kInitBins; b += T) bins[b] = 0u;
    __syncthreads();
    for (uint32_t i = tid; i < N; i += T) atomicAdd(&bins[(uint32_t)(site_key(i, k0, k1) >> 52)], 1u);
    __syncthreads();
    if (tid < 32) {
        // one warp: running prefix over the bins, 32 at a time; each threshold finds its bin
        uint64_t base = 0;
        for (int b0 = 0; b0 < kInitBins; b0 += 32) {
            const uint32_t cnt = bins[b0 + tid];
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (tid >= o) incl += t;
            }
            const uint64_t lo = base + (incl - cnt), hi = base + incl;   // ranks [lo, hi) in bin b0 + tid
            for (int s = 0; s < nt; ++s)
                if (active[s] && remaining[s] >= lo && remaining[s] < hi) {
                    bin_of[s] = (uint32_t)(b0 + tid);
                    prefix[s] = remaining[s] - lo;   // rank inside the bin (reused below)
                }
            base += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
    }
    __syncthreads();
    uint64_t* keys = bins_raw;   // [nt][kInitBinCap]
    for (uint32_t i = tid; i < N; i += T) {
        const uint64_t key = site_key(i, k0, k1);
        const uint32_t b = (uint32_t)(key >> 52);
        for (int s = 0; s < nt; ++s)
            if (active[s] && b == bin_of[s]) {
                const uint32_t x = atomicAdd(&in_bin[s], 1u);
                if (x < (uint32_t)kInitBinCap) keys[s * kInitBinCap + x] = key;
                else overflow = 1;
            }
    }
    __syncthreads();
    if (!overflow) {
        for (int s = 0; s < nt; ++s) {
            if (!active[s]) continue;
            const uint32_t n = in_bin[s];
            const uint64_t want = prefix[s];
            for (uint32_t x = tid; x < n; x += T) {
                const uint64_t kx = keys[s * kInitBinCap + x];
                uint32_t r = 0;
                for (uint32_t y = 0; y < n; ++y) r += keys[s * kInitBinCap + y] < kx ? 1u : 0u;
                if (r == want) remaining[s] = kx;   // the threshold key (unique: keys are distinct)
            }
        }
        __syncthreads();
        if (tid < nt && active[tid]) prefix[tid] = remaining[tid];
        __syncthreads();
    } else {
        if (tid < nt) {
            prefix[tid] = 0;
            remaining[tid] = (uint64_t)cum.v[tid + 1];
        }
        __syncthreads();
    }
    for (int pass = 0; pass < (overflow ? 8 : 0); ++pass) {
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

__global__ void __launch_bounds__(kInitThreads) init_config_kernel(uint32_t N, int S, const Cum cum, uint32_t k0,
                                                                   uint32_t k1, uint8_t* __restrict__ types) {
    init_config_block(N, S, cum, k0, k1, types);
}

// Fresh solutions of global-search iteration g (Sec. 4.1): configuration j (one CTA each) is the
// initial configuration with the seed (r1 << 32) | r0 of Philox counter (j0 + j, g, 0, 4) under
// the search's key; configurations are stored back to back (N bytes each).
__global__ void __launch_bounds__(kInitThreads) init_fresh_kernel(uint32_t N, int S, const Cum cum, uint32_t k0,
                                                                  uint32_t k1, uint32_t g, uint32_t j0,
                                                                  uint8_t* __restrict__ types) {
    const Rand4 r = philox(j0 + blockIdx.x, g, 0u, 4u, k0, k1);
    init_config_block(N, S, cum, r.r0, r.r1, types + (size_t)blockIdx.x * N);
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

cudaError_t launch_init_fresh(int kind, int Lx, int Ly, int Lz, int S, const int64_t* cum_host, uint64_t seed,
                              uint32_t g, uint32_t j0, int n, uint8_t* types, cudaStream_t stream) {
    const uint32_t N = (uint32_t)((kind == kFCC ? 4 : 2) * (int64_t)Lx * Ly * Lz);
    if (S > kInitMaxThresholds + 1 || n < 1) return cudaErrorInvalidValue;
    Cum cum{};
    for (int s = 0; s <= S; ++s) cum.v[s] = cum_host[s];
    init_fresh_kernel<<<n, kInitThreads, 0, stream>>>(N, S, cum, (uint32_t)(seed & 0xFFFFFFFFu),
                                                       (uint32_t)(seed >> 32), g, j0, types);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Full recount of N_ij^(k) (Sec. 4.3): the number of ordered (site, shell vector) pairs whose sites
// hold species i and j.  Two kernels:
//
//  * counts_gather_kernel: each thread builds the per-shell neighbour histogram of one site (8-bit
//    fields per species, neighbours from coordinates) from species staged in shared memory -- the
//    whole configuration when it fits, else a slab of conventional-cell planes with a halo -- or
//    read through the cache when staging would leave too few CTAs.  A warp groups its lanes by the
//    centre species (__match_any_sync) and sums each histogram field over the group
//    (__reduce_add_sync) into a warp-private histogram: no atomics in the site loop.
//  * counts_planes_kernel (rows of at most 64 cells, at most 6 species, one configuration per CTA):
//    per species y a bit plane P_y (one 64-bit word per row of x-consecutive cells of one
//    sublattice); the vector d maps row r of sublattice b to row r' of sublattice b' shifted by
//    dcx cells along x, so sum_x [type = i][type(+d) = j] = popc(P_i[r] & rot(P_j[r'], dcx)).
//    N_ij = N_ji (the shells are centrosymmetric), so only i <= j is counted.
// grid.y (gather) or grid.x (planes) indexes configurations.
// ------------------------------------------------------------------------------------------------
constexpr int kCountThreads = 256;
constexpr int kCountStageMax = 48 * 1024;   // bytes of species staged per CTA

template <int KIND, int M, bool STAGED>
__global__ void __launch_bounds__(kCountThreads) counts_gather_kernel(Geo g, Geo gt, int S, int tz, int hz,
                                                                      const uint8_t* __restrict__ types,
                                                                      int32_t* __restrict__ counts) {
    extern __shared__ __align__(16) uint8_t sm[];
    constexpr int B = KIND == kFCC ? 4 : 2;
    const int E = M * S * S;
    const int LxLy = g.LxLy, zt = tz + 2 * hz;
    const int cfg = blockIdx.y, z0 = STAGED ? blockIdx.x * tz : 0;
    const int tz_here = STAGED ? min(tz, g.Lz - z0) : 0;
    const uint8_t* t = types + (size_t)cfg * (size_t)g.N;
    const int nwarp = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t staged = STAGED ? (uint32_t)(B * zt * LxLy) : 0u;
    int32_t* wh = reinterpret_cast<int32_t*>(sm + align_up(staged, 16));
    for (int i = threadIdx.x; i < nwarp * E; i += blockDim.x) wh[i] = 0;
    if (STAGED) {
        // planes z0 - hz .. z0 + tz + hz - 1 (periodic) of every sublattice, 16 bytes at a time when
        // the planes are 16-byte aligned
        const bool vec = ((reinterpret_cast<uintptr_t>(t) | (uintptr_t)LxLy | (uintptr_t)g.V) & 15u) == 0u;
        for (int bp = 0; bp < B * zt; ++bp) {
            const int b = bp / zt, p = bp - b * zt;
            int zs = z0 - hz + p;
            zs += (zs < 0) ? g.Lz : 0;
            zs -= (zs >= g.Lz) ? g.Lz : 0;
            const uint8_t* src = t + (size_t)b * g.V + (size_t)zs * LxLy;
            uint8_t* dst = sm + (size_t)bp * LxLy;
            if (vec) {
                for (int i = threadIdx.x; i < LxLy / 16; i += blockDim.x)
                    reinterpret_cast<uint4*>(dst)[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
            } else {
                for (int i = threadIdx.x; i < LxLy; i += blockDim.x) dst[i] = __ldg(src + i);
            }
        }
    }
    __syncthreads();
    // staged: the sites of this tile (sublattice b, planes z0 .. z0 + tz_here - 1); through the cache:
    // sites [blockIdx.x * tz, + tz) of the configuration (tz is then a count of sites)
    const int n_here = STAGED ? B * tz_here * LxLy : max(0, min(tz, g.N - (int)blockIdx.x * tz));
    const Divider dPlane = make_divider((uint32_t)(max(1, tz_here) * LxLy));
    auto onehot = [&](uint32_t n) -> uint64_t {
        const int y = STAGED ? sm[n] : __ldg(t + n);
        return y < S ? (1ull << (8 * y)) : 0ull;
    };
    for (int base = warp * 32; base < n_here; base += blockDim.x) {
        const int i = base + lane;
        int A = 0xFF;
        uint64_t h[M];
#pragma unroll
        for (int k = 0; k < M; ++k) h[k] = 0ull;
        if (i < n_here) {
            int X, Y, Z;
            uint32_t own;
            if (STAGED) {
                const uint32_t b = divide((uint32_t)i, dPlane);
                const uint32_t rem = (uint32_t)i - b * (uint32_t)(tz_here * LxLy);
                const uint32_t czl = divide(rem, g.dLxLy);
                const uint32_t rem2 = rem - czl * (uint32_t)LxLy;
                const uint32_t cy = divide(rem2, g.dLx), cx = rem2 - cy * (uint32_t)g.Lx;
                int ox, oy, oz;
                if (KIND == kFCC) {
                    ox = (int)(b >> 1);
                    oy = (int)(b & 1);
                    oz = ox ^ oy;
                } else {
                    ox = oy = oz = (int)b;
                }
                const int czs = (int)czl + hz;   // plane in the staged layout
                own = b * (uint32_t)gt.V + (uint32_t)czs * (uint32_t)LxLy + cy * (uint32_t)g.Lx + cx;
                X = 2 * (int)cx + ox;
                Y = 2 * (int)cy + oy;
                Z = 2 * czs + oz;
            } else {
                own = (uint32_t)blockIdx.x * (uint32_t)tz + (uint32_t)i;
                site_coords<KIND>(g, own, X, Y, Z);
            }
            A = STAGED ? sm[own] : __ldg(t + own);
            if (A < S)
                neighbour_histogram_at<KIND, M, false, uint64_t>(STAGED ? gt : g, X, Y, Z, 0u, onehot, h, M);
            else
                A = 0xFF;
        }
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, A);
        const int leader = __ffs(grp) - 1;
#pragma unroll
        for (int k = 0; k < M; ++k)
            for (int y = 0; y < S; ++y) {
                const unsigned v = __reduce_add_sync(grp, (unsigned)hist_field(h[k], y));
                if (lane == leader && A != 0xFF && v) wh[warp * E + (k * S + A) * S + y] += (int)v;
            }
    }
    __syncthreads();
    int32_t* out = counts + (size_t)cfg * (size_t)E;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        int sum = 0;
        for (int w = 0; w < nwarp; ++w) sum += wh[w * E + e];
        if (sum) atomicAdd(out + e, sum);
    }
}

// Rotation of the low `Lx` bits of w so that bit x of the result is bit (x + s) mod Lx of w
// (|s| <= 2 < 2 Lx).
template <typename W>
__device__ __forceinline__ W rot_row(W w, int s, int Lx, W mask) {
    s += (s < 0) ? Lx : 0;
    s -= (s >= Lx) ? Lx : 0;
    if (s == 0) return w;
    return ((w >> s) | (w << (Lx - s))) & mask;
}

__device__ __forceinline__ int popc_w(uint32_t w) { return __popc(w); }
__device__ __forceinline__ int popc_w(uint64_t w) { return __popcll(w); }

// Target row and x shift of shell vector V from row (b, cz, cy).
template <int KIND>
__device__ __forceinline__ int vector_row(const signed char* V, int b, int cz, int cy, int Ly, int Lz, int& dcx) {
    int ox, oy, oz;
    if (KIND == kFCC) {
        ox = b >> 1;
        oy = b & 1;
        oz = ox ^ oy;
    } else {
        ox = oy = oz = b;
    }
    const int hx = ox + V[0], hy = oy + V[1], hzz = oz + V[2];
    dcx = hx >> 1;   // floor division by 2
    const int dcy = hy >> 1, dcz = hzz >> 1;
    const int px = hx & 1, py = hy & 1;
    const int b2 = (KIND == kFCC) ? 2 * px + py : px;
    int cy2 = cy + dcy, cz2 = cz + dcz;
    cy2 += (cy2 < 0) ? Ly : 0;
    cy2 -= (cy2 >= Ly) ? Ly : 0;
    cz2 += (cz2 < 0) ? Lz : 0;
    cz2 -= (cz2 >= Lz) ? Lz : 0;
    return (b2 * Lz + cz2) * Ly + cy2;
}

// One configuration per CTA.  With every species in [0, S), only the pairs of the first S - 1
// species are counted, over half of each shell's vectors: the vector -v counts (j, i) where v
// counts (i, j), so N_ij = sum over the half of c_ij + c_ji; every row of N^(k) sums to
// N_i Z_k, which gives the pairs with the last species.  A configuration holding any other value
// counts every pair over every vector (values >= S are then not counted).
template <int KIND, int S, typename W>
__global__ void __launch_bounds__(kCountThreads) counts_planes_kernel(Geo g, int M, const uint8_t* __restrict__ types,
                                                                      int32_t* __restrict__ counts) {
    extern __shared__ __align__(16) uint8_t planes_raw[];
    __shared__ int invalid;
    W* planes = reinterpret_cast<W*>(planes_raw);   // [S][R], one word per row (rows of at most 8 sizeof(W) cells)
    constexpr int B = KIND == kFCC ? 4 : 2;
    constexpr int NP = S * (S + 1) / 2;
    constexpr int SM1 = S - 1, NSYM = SM1 * (SM1 + 1) / 2;
    const int Lx = g.Lx, Ly = g.Ly, Lz = g.Lz, R = B * Ly * Lz, E = M * S * S;
    const uint8_t* t = types + (size_t)blockIdx.x * (size_t)g.N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const W mask = (Lx == 8 * (int)sizeof(W)) ? ~W(0) : (W)((W(1) << Lx) - W(1));
    int32_t* wh = reinterpret_cast<int32_t*>(planes + (size_t)S * R);   // [nwarp][E], then [nwarp][S]
    int32_t* wn = wh + nwarp * E;
    for (int i = threadIdx.x; i < nwarp * (E + S); i += blockDim.x) wh[i] = 0;
    if (threadIdx.x == 0) invalid = 0;
    __syncthreads();
    // bit planes: one thread per row (rows are x-contiguous: ((b Lz + cz) Ly + cy) Lx), read four
    // cells at a time when rows start on 4-byte boundaries
    bool bad = false;
    const bool words = (Lx % 4 == 0) && ((reinterpret_cast<uintptr_t>(t) & 3u) == 0u);
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        W pl[S];
#pragma unroll
        for (int y = 0; y < S; ++y) pl[y] = W(0);
        auto cell = [&](int v, int x) {
            const W bit = W(1) << x;
#pragma unroll
            for (int y = 0; y < S; ++y)
                if (v == y) pl[y] |= bit;
            bad = bad || v >= S;
        };
        if (words) {
            const uint32_t* row = reinterpret_cast<const uint32_t*>(t + (size_t)r * Lx);
            for (int x4 = 0; x4 < Lx / 4; ++x4) {
                const uint32_t w4 = __ldg(row + x4);
#pragma unroll
                for (int q = 0; q < 4; ++q) cell((int)((w4 >> (8 * q)) & 0xFFu), 4 * x4 + q);
            }
        } else {
            const uint8_t* row = t + (size_t)r * Lx;
            for (int x = 0; x < Lx; ++x) cell(__ldg(row + x), x);
        }
#pragma unroll
        for (int y = 0; y < S; ++y) planes[(size_t)y * R + r] = pl[y];
    }
    if (bad) invalid = 1;
    __syncthreads();
    const ShellTable& TAB = c_shells[KIND];
    const HalfShells& HALF = c_half[KIND];
    const Divider dLy = make_divider((uint32_t)Ly), dLz = make_divider((uint32_t)Lz);
    auto row_of = [&](int r, int& b, int& cz, int& cy) {
        const uint32_t t2 = divide((uint32_t)r, dLy);
        cy = r - (int)t2 * Ly;
        b = (int)divide(t2, dLz);
        cz = (int)t2 - b * Lz;
    };
    if (!invalid) {
        int ni[S];
#pragma unroll
        for (int a = 0; a < S; ++a) ni[a] = 0;
        for (int k = 0; k < M; ++k) {
            int sym[NSYM];
#pragma unroll
            for (int x = 0; x < NSYM; ++x) sym[x] = 0;
            for (int r = threadIdx.x; r < R; r += blockDim.x) {
                int b, cz, cy;
                row_of(r, b, cz, cy);
                W own[SM1];
#pragma unroll
                for (int a = 0; a < SM1; ++a) own[a] = planes[(size_t)a * R + r];
                if (k == 0) {
#pragma unroll
                    for (int a = 0; a < SM1; ++a) ni[a] += popc_w(own[a]);
                    ni[SM1] += popc_w(planes[(size_t)SM1 * R + r]);
                }
                for (int v = HALF.first[k]; v < HALF.first[k + 1]; ++v) {
                    int dcx;
                    const int r2 = vector_row<KIND>(HALF.v[v], b, cz, cy, Ly, Lz, dcx);
                    W nb[SM1];
#pragma unroll
                    for (int y = 0; y < SM1; ++y) nb[y] = rot_row<W>(planes[(size_t)y * R + r2], dcx, Lx, mask);
                    int x = 0;
#pragma unroll
                    for (int a = 0; a < SM1; ++a) {
                        sym[x++] += 2 * popc_w((W)(own[a] & nb[a]));
#pragma unroll
                        for (int y = a + 1; y < SM1; ++y) sym[x++] += popc_w((W)(own[a] & nb[y])) + popc_w((W)(own[y] & nb[a]));
                    }
                }
            }
            int x = 0;
#pragma unroll
            for (int a = 0; a < SM1; ++a)
#pragma unroll
                for (int y = a; y < SM1; ++y) {
                    const unsigned sum = __reduce_add_sync(0xFFFFFFFFu, (unsigned)sym[x++]);
                    if (lane == 0) wh[warp * E + (k * S + a) * S + y] = (int)sum;
                }
        }
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const unsigned sum = __reduce_add_sync(0xFFFFFFFFu, (unsigned)ni[a]);
            if (lane == 0) wn[warp * S + a] = (int)sum;
        }
        __syncthreads();
        int32_t* out = counts + (size_t)blockIdx.x * (size_t)E;
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            int nt[S], n[S][S];
#pragma unroll
            for (int a = 0; a < S; ++a) {
                nt[a] = 0;
                for (int w = 0; w < nwarp; ++w) nt[a] += wn[w * S + a];
            }
#pragma unroll
            for (int a = 0; a < SM1; ++a)
#pragma unroll
                for (int y = a; y < SM1; ++y) {
                    int sum = 0;
                    for (int w = 0; w < nwarp; ++w) sum += wh[w * E + (k * S + a) * S + y];
                    n[a][y] = sum;
                    n[y][a] = sum;
                }
            const int Z = TAB.z[k];
            int last = nt[SM1] * Z;
#pragma unroll
            for (int a = 0; a < SM1; ++a) {
                int rest = nt[a] * Z;
#pragma unroll
                for (int y = 0; y < SM1; ++y) rest -= n[a][y];
                n[a][SM1] = rest;
                n[SM1][a] = rest;
                last -= rest;
            }
            n[SM1][SM1] = last;
#pragma unroll
            for (int a = 0; a < S; ++a)
#pragma unroll
                for (int y = 0; y < S; ++y) out[(k * S + a) * S + y] = n[a][y];
        }
        return;
    }
    // some value outside [0, S): every vector, every pair i <= j of valid species
    for (int base = warp * 32; base < R; base += blockDim.x) {
        const int r = base + lane;
        const bool act = r < R;
        int b = 0, cz = 0, cy = 0;
        if (act) row_of(r, b, cz, cy);
        W own[S];
#pragma unroll
        for (int a = 0; a < S; ++a) own[a] = act ? planes[(size_t)a * R + r] : W(0);
        for (int k = 0; k < M; ++k) {
            int acc[NP];
#pragma unroll
            for (int x = 0; x < NP; ++x) acc[x] = 0;
            for (int v = TAB.first[k]; v < TAB.first[k + 1]; ++v) {
                int dcx = 0;
                const int r2 = act ? vector_row<KIND>(TAB.v[v], b, cz, cy, Ly, Lz, dcx) : 0;
                W nb[S];
#pragma unroll
                for (int y = 0; y < S; ++y) nb[y] = act ? rot_row<W>(planes[(size_t)y * R + r2], dcx, Lx, mask) : W(0);
                int x = 0;
#pragma unroll
                for (int a = 0; a < S; ++a)
#pragma unroll
                    for (int y = a; y < S; ++y) acc[x++] += popc_w((W)(own[a] & nb[y]));
            }
            int x = 0;
#pragma unroll
            for (int a = 0; a < S; ++a)
#pragma unroll
                for (int y = a; y < S; ++y) {
                    const unsigned sum = __reduce_add_sync(0xFFFFFFFFu, (unsigned)acc[x++]);
                    if (lane == 0 && sum) {
                        wh[warp * E + (k * S + a) * S + y] += (int)sum;
                        if (y != a) wh[warp * E + (k * S + y) * S + a] += (int)sum;
                    }
                }
        }
    }
    __syncthreads();
    int32_t* out = counts + (size_t)blockIdx.x * (size_t)E;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        int sum = 0;
        for (int w = 0; w < nwarp; ++w) sum += wh[w * E + e];
        out[e] = sum;
    }
}

template <int KIND, int M>
static cudaError_t launch_gather_t(const Geo& g, int S, int n_configs, const uint8_t* types, int32_t* counts,
                                   cudaStream_t stream) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    constexpr int B = KIND == kFCC ? 4 : 2;
    const int reach = build_shell_table(KIND).reach[M - 1];
    const int hz = (reach + 1) / 2;
    const size_t hist = sizeof(int32_t) * (kCountThreads / 32) * M * S * S;
    // whole configurations when they fit; else slabs of tz planes with hz halo planes on each side
    int tz = g.Lz, h = 0;
    if ((size_t)g.N > (size_t)kCountStageMax) {
        h = hz;
        tz = (int)((size_t)kCountStageMax / ((size_t)B * g.LxLy)) - 2 * h;
    }
    const int tiles = tz >= 1 ? (g.Lz + tz - 1) / tz : 0;
    if (tz >= 1 && (size_t)tiles * n_configs >= (size_t)sms) {
        const Geo gt = make_geo(KIND, g.Lx, g.Ly, tz + 2 * h);
        const size_t smem = align_up((uint32_t)(B * (tz + 2 * h) * g.LxLy), 16) + hist;
        if (smem > 48 * 1024) {
            const cudaError_t err = cudaFuncSetAttribute(counts_gather_kernel<KIND, M, true>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) {
                (void)cudaGetLastError();
                return err;
            }
        }
        counts_gather_kernel<KIND, M, true><<<dim3(tiles, n_configs), kCountThreads, smem, stream>>>(
            g, gt, S, tz, h, types, counts);
    } else {
        // through the cache, chunks of sites: enough CTAs to fill the GPU a few times over
        int chunk = kCountThreads * 8;
        while (chunk > kCountThreads && (size_t)((g.N + chunk - 1) / chunk) * n_configs < (size_t)(4 * sms)) chunk /= 2;
        counts_gather_kernel<KIND, M, false><<<dim3((g.N + chunk - 1) / chunk, n_configs), kCountThreads, hist,
                                               stream>>>(g, g, S, chunk, 0, types, counts);
    }
    return cudaGetLastError();
}

template <int KIND, int S, typename W>
static cudaError_t launch_planes_w(const Geo& g, int M, int n_configs, const uint8_t* types, int32_t* counts,
                                   cudaStream_t stream) {
    constexpr int B = KIND == kFCC ? 4 : 2;
    const size_t smem = sizeof(W) * S * B * g.Ly * g.Lz + sizeof(int32_t) * (kCountThreads / 32) * (M * S * S + S);
    cudaError_t err = cudaFuncSetAttribute(counts_planes_kernel<KIND, S, W>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) {
        (void)cudaGetLastError();
        return err;
    }
    counts_planes_kernel<KIND, S, W><<<n_configs, kCountThreads, smem, stream>>>(g, M, types, counts);
    return cudaGetLastError();
}

template <int KIND, int S>
static cudaError_t launch_planes_t(const Geo& g, int M, int n_configs, const uint8_t* types, int32_t* counts,
                                   cudaStream_t stream) {
    if (g.Lx <= 32) return launch_planes_w<KIND, S, uint32_t>(g, M, n_configs, types, counts, stream);
    return launch_planes_w<KIND, S, uint64_t>(g, M, n_configs, types, counts, stream);
}

// Shared memory of the bit-plane kernel, or 0 when it does not apply.
static size_t planes_smem(int kind, int Lx, int Ly, int Lz, int M, int S) {
    if (Lx > 64 || S < 2 || S > 6) return 0;
    const int B = kind == kFCC ? 4 : 2;
    const size_t smem = sizeof(uint64_t) * S * B * Ly * Lz + sizeof(int32_t) * (kCountThreads / 32) * (M * S * S + S);
    return smem <= 200 * 1024 ? smem : 0;
}

bool sro_counts_planes_apply(int kind, int Lx, int Ly, int Lz, int M, int S) {
    return planes_smem(kind, Lx, Ly, Lz, M, S) != 0;
}

cudaError_t launch_sro_counts(int kind, int Lx, int Ly, int Lz, int M, int S, int n_configs, const uint8_t* types,
                              int32_t* counts, int method, cudaStream_t stream) {
    const Geo g = make_geo(kind, Lx, Ly, Lz);
    const bool planes = (method == 2) || (method == 0 && planes_smem(kind, Lx, Ly, Lz, M, S) != 0 && n_configs >= 64);
    if (planes) {
#define HEA_PLANES_CASE(KD, SS) \
    if (kind == KD && S == SS) return launch_planes_t<KD, SS>(g, M, n_configs, types, counts, stream);
        HEA_PLANES_CASE(kFCC, 2) HEA_PLANES_CASE(kFCC, 3) HEA_PLANES_CASE(kFCC, 4) HEA_PLANES_CASE(kFCC, 5)
        HEA_PLANES_CASE(kFCC, 6) HEA_PLANES_CASE(kBCC, 2) HEA_PLANES_CASE(kBCC, 3) HEA_PLANES_CASE(kBCC, 4)
        HEA_PLANES_CASE(kBCC, 5) HEA_PLANES_CASE(kBCC, 6)
#undef HEA_PLANES_CASE
        return cudaErrorInvalidValue;
    }
    cudaError_t err = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_configs * M * S * S, stream);
    if (err != cudaSuccess) return err;
#define HEA_COUNTS_CASE(KD, MM) \
    if (kind == KD && M == MM) return launch_gather_t<KD, MM>(g, S, n_configs, types, counts, stream);
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
// One CTA per configuration: counts, alpha and f2 of configuration c at offsets c * E, c * E, c.
__global__ void sro_alpha_kernel(const __grid_constant__ ChainDesc d, const int32_t* __restrict__ counts,
                                 double* __restrict__ alpha, double* __restrict__ f2) {
    __shared__ double term[kMaxEntries];
    const int S = d.S, M = d.M, E = M * S * S;
    const ShellTable& T = c_shells[d.kind];
    counts += (size_t)blockIdx.x * E;
    if (alpha) alpha += (size_t)blockIdx.x * E;
    f2 += blockIdx.x;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int k = e / (S * S), i = (e / S) % S, j = e % S;
        const double den = __dmul_rn(__dmul_rn((double)T.z[k], (double)d.n_per[i]), (double)d.n_per[j]);
        const double Q = __ddiv_rn((double)d.N, den);
        const double a = __dsub_rn(1.0, __dmul_rn((double)counts[e], Q));
        if (alpha) alpha[e] = a;
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
                             cudaStream_t stream, int n_configs) {
    sro_alpha_kernel<<<n_configs, 128, 0, stream>>>(d, counts, alpha, f2);
    return cudaGetLastError();
}

}  // namespace hea
