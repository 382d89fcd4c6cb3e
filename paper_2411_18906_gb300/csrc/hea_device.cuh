// hea_device.cuh -- device-side building blocks of libhea (sm_103a): Philox4x32-10, lattice
// shells, neighbour indexing computed on the fly from half-unit coordinates, packed species
// storage.  Written for this library; it shares nothing with the CPU reference.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace hea {

constexpr int kFCC = 0;
constexpr int kBCC = 1;
constexpr int kMaxSpecies = 8;
constexpr int kMaxShells = 5;
constexpr int kMaxEntries = kMaxShells * kMaxSpecies * kMaxSpecies;  // M*S*S

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  Ten rounds of
//   (x0, x1, x2, x3) -> (mulhi(B, x2) ^ x1 ^ k0, B*x2, mulhi(A, x0) ^ x3 ^ k1, A*x0)
// with A = 0xD2511F53, B = 0xCD9E8D57, and the key advanced by the Weyl increments
// (0x9E3779B9, 0xBB67AE85) after every round.
// ------------------------------------------------------------------------------------------------
struct Rand4 {
    uint32_t r0, r1, r2, r3;
};

__device__ __forceinline__ Rand4 philox(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo_a = 0xD2511F53u * x0;
        const uint32_t hi_a = __umulhi(0xD2511F53u, x0);
        const uint32_t lo_b = 0xCD9E8D57u * x2;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, x2);
        x0 = hi_b ^ x1 ^ k0;
        x1 = lo_b;
        x2 = hi_a ^ x3 ^ k1;
        x3 = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Rand4{x0, x1, x2, x3};
}

// ------------------------------------------------------------------------------------------------
// Coordination shells.  A half-unit integer vector joins two FCC sites iff its coordinate sum is
// even, and two BCC sites iff its three coordinates share one parity.  Shell k is the k-th
// smallest |d|^2 among such vectors; the table is built at compile time.
// ------------------------------------------------------------------------------------------------
struct ShellTable {
    int z[kMaxShells];          // vectors in shell k
    int first[kMaxShells + 1];  // index of the first vector of shell k
    int radius2[kMaxShells];    // |d|^2 of shell k, half units^2
    int reach[kMaxShells];      // largest |component| over shells 0..k
    signed char v[96][3];
};

__host__ __device__ constexpr bool joins_sites(int kind, int x, int y, int z) {
    return kind == kFCC ? (((x + y + z) & 1) == 0) : (((x & 1) == (y & 1)) && ((y & 1) == (z & 1)));
}

__host__ __device__ constexpr ShellTable build_shell_table(int kind) {
    ShellTable t{};
    int found = 0;
    int n = 0;
    int reach = 0;
    for (int r2 = 1; r2 <= 16 && found < kMaxShells; ++r2) {
        int here = 0;
        for (int x = -4; x <= 4; ++x)
            for (int y = -4; y <= 4; ++y)
                for (int z = -4; z <= 4; ++z)
                    if (x * x + y * y + z * z == r2 && joins_sites(kind, x, y, z)) {
                        if (here == 0) t.first[found] = n;
                        t.v[n][0] = (signed char)x;
                        t.v[n][1] = (signed char)y;
                        t.v[n][2] = (signed char)z;
                        const int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y, az = z < 0 ? -z : z;
                        reach = ax > reach ? ax : reach;
                        reach = ay > reach ? ay : reach;
                        reach = az > reach ? az : reach;
                        ++n;
                        ++here;
                    }
        if (here > 0) {
            t.z[found] = here;
            t.radius2[found] = r2;
            t.reach[found] = reach;
            ++found;
        }
    }
    t.first[kMaxShells] = n;
    return t;
}

// Largest |component| of a vector in shells 1..M (at most 3 for M <= 5).
template <int KIND, int M>
__host__ __device__ constexpr int shell_reach() {
    return build_shell_table(KIND).reach[M - 1];
}

template <int KIND, int M>
__host__ __device__ constexpr int shell_total() {
    return build_shell_table(KIND).first[M];
}

// ------------------------------------------------------------------------------------------------
// Cell geometry.  Site index = b * V + (cz * Ly + cy) * Lx + cx (V = Lx*Ly*Lz cells).
// Half-unit position (X, Y, Z) = (2cx + ox_b, 2cy + oy_b, 2cz + oz_b); for FCC the basis index is
// b = 2*(X&1) + (Y&1), for BCC b = X&1.
// ------------------------------------------------------------------------------------------------
// Unsigned division by a runtime constant d for dividends n < 2^31 (Granlund-Montgomery):
// n / d = umulhi(n, m) >> s with l = ceil(log2 d), m = ceil(2^(31+l) / d), s = l - 1; d = 1 uses
// s = -1 (quotient n).  m < 2^32 because d > 2^(l-1).
struct Divider {
    uint32_t m;
    int s;
};

__host__ __device__ inline Divider make_divider(uint32_t d) {
    if (d <= 1) return Divider{0u, -1};
    int l = 0;
    while ((1ull << l) < (uint64_t)d) ++l;
    const uint64_t p = 1ull << (31 + l);
    const uint64_t m = p / d + ((p % d) != 0 ? 1ull : 0ull);
    return Divider{(uint32_t)m, l - 1};
}

__device__ __forceinline__ uint32_t divide(uint32_t n, const Divider& v) {
    return v.s < 0 ? n : (__umulhi(n, v.m) >> v.s);
}

struct Geo {
    int Lx, Ly, Lz;
    int V;     // cells
    int LxLy;
    int N;     // sites
    Divider dV, dLxLy, dLx;
};

__host__ __device__ inline Geo make_geo(int kind, int Lx, int Ly, int Lz) {
    Geo g;
    g.Lx = Lx;
    g.Ly = Ly;
    g.Lz = Lz;
    g.V = Lx * Ly * Lz;
    g.LxLy = Lx * Ly;
    g.N = (kind == kFCC ? 4 : 2) * g.V;
    g.dV = make_divider((uint32_t)g.V);
    g.dLxLy = make_divider((uint32_t)g.LxLy);
    g.dLx = make_divider((uint32_t)Lx);
    return g;
}

template <int KIND>
__device__ __forceinline__ void site_coords(const Geo& g, uint32_t idx, int& X, int& Y, int& Z) {
    const uint32_t b = divide(idx, g.dV);
    const uint32_t cell = idx - b * (uint32_t)g.V;
    const uint32_t cz = divide(cell, g.dLxLy);
    const uint32_t rem = cell - cz * (uint32_t)g.LxLy;
    const uint32_t cy = divide(rem, g.dLx);
    const uint32_t cx = rem - cy * (uint32_t)g.Lx;
    int ox, oy, oz;
    if (KIND == kFCC) {
        ox = (int)(b >> 1);
        oy = (int)(b & 1);
        oz = ox ^ oy;
    } else {
        ox = oy = oz = (int)b;
    }
    X = 2 * (int)cx + ox;
    Y = 2 * (int)cy + oy;
    Z = 2 * (int)cz + oz;
}

// Per-axis index contributions for offsets -R..R around one site: the neighbour at offset
// (dx, dy, dz) has index x[dx+R] + y[dy+R] + z[dz+R].
template <int KIND, int R>
struct AxisTable {
    int x[2 * R + 1], y[2 * R + 1], z[2 * R + 1];

    __device__ __forceinline__ void build(const Geo& g, int X, int Y, int Z) {
        const int PX = 2 * g.Lx, PY = 2 * g.Ly, PZ = 2 * g.Lz;
#pragma unroll
        for (int d = -R; d <= R; ++d) {
            int xs = X + d, ys = Y + d, zs = Z + d;
            if (d < 0) {
                xs += (xs < 0) ? PX : 0;
                ys += (ys < 0) ? PY : 0;
                zs += (zs < 0) ? PZ : 0;
            } else if (d > 0) {
                xs -= (xs >= PX) ? PX : 0;
                ys -= (ys >= PY) ? PY : 0;
                zs -= (zs >= PZ) ? PZ : 0;
            }
            if (KIND == kFCC) {
                x[d + R] = (xs >> 1) + (xs & 1) * 2 * g.V;
                y[d + R] = (ys >> 1) * g.Lx + (ys & 1) * g.V;
            } else {
                x[d + R] = (xs >> 1) + (xs & 1) * g.V;
                y[d + R] = (ys >> 1) * g.Lx;
            }
            z[d + R] = (zs >> 1) * g.LxLy;
        }
    }
};

// ------------------------------------------------------------------------------------------------
// Species storage in shared memory: 8, 4 or 2 bits per site (2 only for at most 4 species); with
// fewer than 8 bits, site i sits in bits BITS * (i mod 8/BITS) of byte i / (8/BITS).
// ------------------------------------------------------------------------------------------------
template <int BITS>
struct Packing {
    static constexpr uint32_t per = 8 / BITS;                  // sites per byte
    static constexpr int lg = BITS == 8 ? 0 : (BITS == 4 ? 1 : 2);
    static constexpr uint32_t mask = (1u << BITS) - 1u;
};

template <int BITS>
__device__ __forceinline__ int load_species(const uint8_t* s, uint32_t i) {
    if (BITS == 8) return s[i];
    using P = Packing<BITS>;
    return (s[i >> P::lg] >> ((i & (P::per - 1u)) * BITS)) & P::mask;
}

template <int BITS>
__device__ __forceinline__ void store_species(uint8_t* s, uint32_t i, int v) {
    if (BITS == 8) {
        s[i] = (uint8_t)v;
    } else {
        using P = Packing<BITS>;
        const uint32_t sh = (i & (P::per - 1u)) * BITS;
        const uint32_t byte = i >> P::lg;
        s[byte] = (uint8_t)((s[byte] & ~(P::mask << sh)) | ((uint32_t)v << sh));
    }
}

template <int BITS>
__host__ __device__ constexpr uint32_t species_bytes(uint32_t N) {
    return BITS == 8 ? N : (BITS == 4 ? (N + 1) / 2 : (N + 3) / 4);
}

template <int KIND>
struct ShellsOf {
    static constexpr ShellTable table = build_shell_table(KIND);
};

// One-hot species increment of the neighbour reached by shell vector V (a compile-time index, so
// the offsets are immediates and the axis table stays in registers).  H is the accumulator type
// (32 bits hold four 8-bit species fields, 64 bits eight); with EXCL the neighbour `excl` is skipped.
template <int KIND, int R, int V, bool EXCL, typename H, typename OneHot>
__device__ __forceinline__ H vector_increment(const AxisTable<KIND, R>& ax, uint32_t excl, OneHot& onehot) {
    constexpr int dx = ShellsOf<KIND>::table.v[V][0] + R;
    constexpr int dy = ShellsOf<KIND>::table.v[V][1] + R;
    constexpr int dz = ShellsOf<KIND>::table.v[V][2] + R;
    const uint32_t n = (uint32_t)(ax.x[dx] + ax.y[dy] + ax.z[dz]);
    const H inc = onehot(n);
    if (EXCL) return (n != excl) ? inc : (H)0;
    return inc;
}

template <int KIND, int R, int FIRST, bool EXCL, typename H, typename OneHot, int... I>
__device__ __forceinline__ H shell_sum(const AxisTable<KIND, R>& ax, uint32_t excl, OneHot& onehot,
                                       std::integer_sequence<int, I...>) {
    return ((H)0 + ... + vector_increment<KIND, R, FIRST + I, EXCL, H>(ax, excl, onehot));
}

template <int KIND, int R, int K, bool EXCL, typename H, typename OneHot>
__device__ __forceinline__ H shell_histogram(const AxisTable<KIND, R>& ax, uint32_t excl, OneHot& onehot) {
    constexpr int first = ShellsOf<KIND>::table.first[K];
    constexpr int z = ShellsOf<KIND>::table.z[K];
    return shell_sum<KIND, R, first, EXCL, H>(ax, excl, onehot, std::make_integer_sequence<int, z>{});
}

template <int KIND, int R, int MX, bool EXCL, typename H, typename OneHot, int... K>
__device__ __forceinline__ void all_shells(const AxisTable<KIND, R>& ax, uint32_t excl, OneHot& onehot, H (&h)[MX],
                                           int M, std::integer_sequence<int, K...>) {
    ((h[K] = (K < M) ? shell_histogram<KIND, R, K, EXCL, H>(ax, excl, onehot) : (H)0), ...);
}

// Neighbour histogram of the site at half-unit position (X, Y, Z) for shells 1..M (M <= MX):
// h[k] holds 8-bit counts per species (field y at bits 8y..8y+7; Z_k <= 24 fits); with EXCL the
// neighbour `excl` is skipped.  `onehot(n)` returns 1 << (8 * species(n)) (type H), or 0 for a site
// that must not be counted.
template <int KIND, int MX, bool EXCL, typename H, typename OneHot>
__device__ __forceinline__ void neighbour_histogram_at(const Geo& g, int X, int Y, int Z, uint32_t excl,
                                                       OneHot onehot, H (&h)[MX], int M) {
    constexpr int R = shell_reach<KIND, MX>();
    AxisTable<KIND, R> ax;
    ax.build(g, X, Y, Z);
    all_shells<KIND, R, MX, EXCL, H>(ax, excl, onehot, h, M, std::make_integer_sequence<int, MX>{});
}

// Species packed BITS < 8 to a byte (site i in bits BITS (i mod 8/BITS) of byte i / (8/BITS)) with
// Lx a multiple of 8/BITS: every y and z index term is then a multiple of 8/BITS, so the byte and
// the bit offset of a neighbour split into per-axis parts, and a gather is two additions, a load,
// a shift and a mask.
template <int KIND, int R, int BITS>
struct PackedAxisTable {
    static constexpr int lg = BITS == 4 ? 1 : 2;   // log2 of the sites per byte
    int bx[2 * R + 1], sx[2 * R + 1], by[2 * R + 1], bz[2 * R + 1];

    __device__ __forceinline__ void build(const Geo& g, int X, int Y, int Z) {
        AxisTable<KIND, R> ax;
        ax.build(g, X, Y, Z);
#pragma unroll
        for (int d = 0; d < 2 * R + 1; ++d) {
            bx[d] = ax.x[d] >> lg;
            sx[d] = (ax.x[d] & ((1 << lg) - 1)) * BITS;
            by[d] = ax.y[d] >> lg;
            bz[d] = ax.z[d] >> lg;
        }
    }
};

template <int KIND, int R, int BITS, int V, typename H>
__device__ __forceinline__ H packed_increment(const PackedAxisTable<KIND, R, BITS>& ax, const uint8_t* __restrict__ types) {
    constexpr int dx = ShellsOf<KIND>::table.v[V][0] + R;
    constexpr int dy = ShellsOf<KIND>::table.v[V][1] + R;
    constexpr int dz = ShellsOf<KIND>::table.v[V][2] + R;
    const uint32_t y = ((uint32_t)types[ax.bx[dx] + ax.by[dy] + ax.bz[dz]] >> ax.sx[dx]) & ((1u << BITS) - 1u);
    return (H)1 << (8 * y);
}

template <int KIND, int R, int BITS, int FIRST, typename H, int... I>
__device__ __forceinline__ H packed_shell_sum(const PackedAxisTable<KIND, R, BITS>& ax, const uint8_t* __restrict__ types,
                                              std::integer_sequence<int, I...>) {
    return ((H)0 + ... + packed_increment<KIND, R, BITS, FIRST + I, H>(ax, types));
}

template <int KIND, int R, int BITS, int MX, typename H, int... K>
__device__ __forceinline__ void packed_all_shells(const PackedAxisTable<KIND, R, BITS>& ax, const uint8_t* __restrict__ types,
                                                  H (&h)[MX], int M, std::integer_sequence<int, K...>) {
    ((h[K] = (K < M) ? packed_shell_sum<KIND, R, BITS, ShellsOf<KIND>::table.first[K], H>(
                           ax, types, std::make_integer_sequence<int, ShellsOf<KIND>::table.z[K]>{})
                     : (H)0),
     ...);
}

// Full neighbour histogram (no site skipped) of the site at (X, Y, Z) from packed species; needs
// BITS < 8 and Lx a multiple of 8 / BITS.
template <int KIND, int MX, int BITS, typename H>
__device__ __forceinline__ void neighbour_histogram_packed(const Geo& g, int X, int Y, int Z,
                                                           const uint8_t* __restrict__ types, H (&h)[MX], int M) {
    constexpr int R = shell_reach<KIND, MX>();
    PackedAxisTable<KIND, R, BITS> ax;
    ax.build(g, X, Y, Z);
    packed_all_shells<KIND, R, BITS, MX, H>(ax, types, h, M, std::make_integer_sequence<int, MX>{});
}

// The same for a site index, 64-bit fields, skipping `excl`.
template <int KIND, int MX, typename OneHot>
__device__ __forceinline__ void neighbour_histogram_upto(const Geo& g, uint32_t site, uint32_t excl, OneHot onehot,
                                                         uint64_t (&h)[MX], int M) {
    int X, Y, Z;
    site_coords<KIND>(g, site, X, Y, Z);
    neighbour_histogram_at<KIND, MX, true, uint64_t>(g, X, Y, Z, excl, onehot, h, M);
}

// Full histogram (no site skipped) of a site index, 64-bit fields, compile-time shell count.
template <int KIND, int M, typename OneHot>
__device__ __forceinline__ void neighbour_histogram(const Geo& g, uint32_t site, uint32_t excl, OneHot onehot,
                                                    uint64_t (&h)[M]) {
    int X, Y, Z;
    site_coords<KIND>(g, site, X, Y, Z);
    (void)excl;
    neighbour_histogram_at<KIND, M, false, uint64_t>(g, X, Y, Z, 0u, onehot, h, M);
}

__device__ __forceinline__ int hist_field(uint64_t h, int y) { return (int)((h >> (8 * y)) & 0xFFu); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace hea
