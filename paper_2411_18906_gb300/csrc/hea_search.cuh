// hea_search.cuh -- swap scoring (Sec. 4.5, Sec. 4.6.2) and the parallel Monte Carlo search
// (Alg. parallel_mc; Sec. 4.6.3 selection; Sec. 4.6.4 convergence) for sm_103a.
//
// A chain's cell lives in shared memory (8 or 4 bits per site) next to its counts and the
// per-entry objective coefficients.  A step:
//   1. every thread draws candidates (Philox), builds the per-shell neighbour histograms of both
//      sites (neighbours computed from coordinates) and the swap vector g = h_b - h_a, and
//      evaluates an FP32 estimate of the swap key with a rigorous interval [lo, hi] around the
//      exact binary64 key;
//   2. decisions the intervals settle are taken on them; the exact binary64 key (the same FMA
//      chain as the reference definition) is computed only where an interval straddles the
//      acceptance threshold or overlaps another contender's interval, so every decision equals
//      the one the exact keys give;
//   3. best-of-K: argmin over (D, k); multi-accept: eligible candidates ranked by (D, k) and walked
//      by one warp with a neighbourhood bitmap and a re-check against the running counts;
//   4. the accepted swap(s) update species, counts and coefficients in place.
// One CTA runs a chain (run_chain); the cooperative chain over a grid of CTAs (hea_coop.cuh)
// reuses the scoring and the exact keys.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "hea_device.cuh"
#include "hea_internal.h"

namespace hea {

static __constant__ ShellTable c_shells[2] = {build_shell_table(kFCC), build_shell_table(kBCC)};

// Absolute floor of the FP32 key bound (see score_float) and 2^-23, the unit of its relative part.
constexpr float kAbsBound = 7.52316385e-37f;   // 2^-120
constexpr float kTwoUlp = 1.1920928955078125e-07f;  // 2^-23
constexpr float kBetaScale = 3.814697265625e-06f;  // 2^-18

struct ChainShared {
    int qn;          // queued candidates
    int n_elig;      // multi-accept: eligible candidates
    int n_acc;       // swaps accepted this step
    int stop;
    int bad;
    int use_filter;
    int depth;
    int status;
    int win_q;       // best-of-K: slot of the winner (-1 none)
    int sync_ok;
    int batch_n;     // walk: accepted candidates of the current batch
    int walk_done;   // walk: max_accept reached
    uint32_t taken[kPairWalkMax / 32];   // walk: accepted set of the ranked list
    float umin;      // min over candidates of the upper bound on D
    // cooperative chain
    int fixF, fixFa;         // fixed-point scales of the step's b coefficients and of the a coefficients
    int n_amb;               // candidates whose order against the current winner the intervals leave open
    int sync_fail;           // a wait for another CTA's records ran out
    int pub_stop;            // stop bit of CTA 0's record for this step
    int n_pairs;             // walk: suspects / conflicting records / batches holding unsure candidates
    int n_edges;             // walk: conflicting record pairs
    int win_elig;            // best-of-K: winner eligible (1), not (0), or decided on its binary64 key (-1)
    int asym;                // set-up: Q or the target is not symmetric
    unsigned long long maxb; // max |b| over the entries (binary64 bits)
    unsigned int wmax;       // walk: bound on the running |b| (binary32 bits)
    long long red_l[32];
    int64_t steps;
    int64_t accepted;
    uint64_t t0;
    float red_f[32];
    double red_d[32];
    uint32_t red_k[32];
    int red_q[32];
};

// Per-shell swap vector g = h_b - h_a (Sec. 4.5), packed as one biased byte per species:
// byte y holds 64 + h_b[y] - h_a[y] (every histogram byte is <= 24, so no borrow crosses bytes).
constexpr uint64_t kGBias = 0x4040404040404040ull;

__device__ __forceinline__ uint64_t pack_g(uint64_t ha, uint64_t hb) { return (hb + kGBias) - ha; }

__device__ __forceinline__ int g_of(uint64_t gb, int y) { return (int)((gb >> (8 * y)) & 0xFFu) - 64; }

// Delta of entry (k,i,j) for a swap of species A (site a) and B (site b):
//   dN_ij = [i==A] g_j - [i==B] g_j + [j==A] g_i - [j==B] g_i.
__device__ __forceinline__ int entry_delta(uint64_t gb, int A, int B, int i, int j) {
    int d = 0;
    if (i == A || i == B) {
        const int gj = g_of(gb, j);
        d += (i == A) ? gj : -gj;
    }
    if (j == A || j == B) {
        const int gi = g_of(gb, i);
        d += (j == A) ? gi : -gi;
    }
    return d;
}

// Exact key: change of F^2, D <- fma(dN, fma(a, dN, b), D) over (k,i,j) row-major; entries with
// dN = 0 leave D unchanged bit for bit and are skipped.
static __device__ double exact_key(int M, int S, const double* __restrict__ ca, const double* __restrict__ cb, int A,
                                   int B, const uint64_t* gb) {
    double D = 0.0;
    for (int k = 0; k < M; ++k) {
        const uint64_t g_k = gb[k];
        for (int i = 0; i < S; ++i) {
            const bool row = (i == A || i == B);
            for (int j = 0; j < S; ++j) {
                if (!row && j != A && j != B) continue;
                const int d = entry_delta(g_k, A, B, i, j);
                if (d == 0) continue;
                const int e = (k * S + i) * S + j;
                const double x = (double)d;
                D = __fma_rn(x, __fma_rn(ca[e], x, cb[e]), D);
            }
        }
    }
    return D;
}

// Exact key against the running counts: coefficients recomputed in binary64 from cnt with the
// arithmetic of the step-start coefficients.
static __device__ double exact_key_running(int M, int S, const int32_t* cnt, const double* Q, const double* tgt,
                                           const double* ca, const double* w, int A, int B, const uint64_t* gb) {
    double D = 0.0;
    for (int k = 0; k < M; ++k) {
        const uint64_t g_k = gb[k];
        for (int i = 0; i < S; ++i) {
            const bool row = (i == A || i == B);
            for (int j = 0; j < S; ++j) {
                if (!row && j != A && j != B) continue;
                const int dl = entry_delta(g_k, A, B, i, j);
                if (dl == 0) continue;
                const int e = (k * S + i) * S + j;
                const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)cnt[e], Q[e])), tgt[e]);
                const double b = __dmul_rn(-2.0, __dmul_rn(w[k], __dmul_rn(Q[e], err)));
                const double x = (double)dl;
                D = __fma_rn(x, __fma_rn(ca[e], x, b), D);
            }
        }
    }
    return D;
}

// FP32 estimate of the key and a bound on its distance to the exact binary64 key.  Both evaluate
// D = sum_e d_e (a_e d_e + b_e) from the same binary64 coefficients a, b; the estimate uses their
// binary32 roundings and the chain acc <- fma(d, fma(a', d, b'), acc).  With u = 2^-24 and n <= E
// nonzero terms, rounding a and b, the inner and the outer fma each contribute at most u per term
// magnitude plus u |partial sum|, so the estimate is within (n + 2) u (1 + 2 (n + 2) u) S + n 48 2^-150
// of the real value, S = sum |d| (|a| |d| + |b|) (itself underestimated by at most (n + 2) u in FP32);
// the binary64 chain is within (n + 1) 2^-53 S of it.  For E <= 320 the distance is below
// (E + 3) u S + 2^-136, and the bound used, (E + 4) 2^-23 S + 2^-120, is twice that.
__device__ __forceinline__ void score_float(int M, int S, const float* __restrict__ fa, const float* __restrict__ fb,
                                            int A, int B, const uint64_t* gb, float rel, float& D, float& err) {
    float acc = 0.f, mag = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxShells; ++k) {
        if (k >= M) break;
        const uint64_t g_k = gb[k];
        const int base = k * S * S;
        const int gA = g_of(g_k, A);
        const int gB = g_of(g_k, B);
        for (int y = 0; y < S; ++y) {
            const int gy = g_of(g_k, y);
            // Row A: dN_Ay = g_y + [y==A] g_A - [y==B] g_A; row B: dN_By = -g_y + [y==A] g_B - [y==B] g_B.
            const int dA = gy + (y == A ? gA : 0) - (y == B ? gA : 0);
            const int dB = -gy + (y == A ? gB : 0) - (y == B ? gB : 0);
            if (dA != 0) {
                const int e = base + A * S + y;
                const float x = (float)dA, ax = fabsf(x);
                acc = fmaf(x, fmaf(fa[e], x, fb[e]), acc);
                mag = fmaf(ax, fmaf(fabsf(fa[e]), ax, fabsf(fb[e])), mag);
            }
            if (dB != 0) {
                const int e = base + B * S + y;
                const float x = (float)dB, ax = fabsf(x);
                acc = fmaf(x, fmaf(fa[e], x, fb[e]), acc);
                mag = fmaf(ax, fmaf(fabsf(fa[e]), ax, fabsf(fb[e])), mag);
            }
            if (y != A && y != B && gy != 0) {
                // Columns A and B of row y: dN_yA = g_y, dN_yB = -g_y.
                const float x = (float)gy, ax = fabsf(x);
                const int eA = base + y * S + A, eB = base + y * S + B;
                acc = fmaf(x, fmaf(fa[eA], x, fb[eA]), acc);
                acc = fmaf(-x, fmaf(fa[eB], -x, fb[eB]), acc);
                mag = fmaf(ax, fmaf(fabsf(fa[eA]), ax, fabsf(fb[eA])), mag);
                mag = fmaf(ax, fmaf(fabsf(fa[eB]), ax, fabsf(fb[eB])), mag);
            }
        }
    }
    D = acc;
    err = fmaf(mag, rel, kAbsBound);
}

// The same estimate and bound when the coefficient tables are symmetric (a_ijk = a_jik and
// b_ijk = b_jik bit for bit): the counts stay symmetric, so (i, j) and (j, i) change alike and
// each pair enters once with weight 2 (the doubling is exact; the sum S and every term's relative
// rounding are unchanged, and fewer terms are added).
__device__ __forceinline__ void score_float_sym(int M, int S, const float* __restrict__ fa,
                                                const float* __restrict__ fb, int A, int B, const uint64_t* gb,
                                                float rel, float& D, float& err) {
    float acc = 0.f, mag = 0.f;
    auto term = [&](int e, float x, float wgt) {
        const float ax = fabsf(x);
        acc = fmaf(wgt * x, fmaf(fa[e], x, fb[e]), acc);
        mag = fmaf(wgt * ax, fmaf(fabsf(fa[e]), ax, fabsf(fb[e])), mag);
    };
#pragma unroll
    for (int k = 0; k < kMaxShells; ++k) {
        if (k >= M) break;
        const uint64_t g_k = gb[k];
        const int base = k * S * S;
        const int gA = g_of(g_k, A), gB = g_of(g_k, B);
        if (gA != 0) term(base + A * S + A, (float)(2 * gA), 1.0f);       // dN_AA = 2 g_A
        if (gB != 0) term(base + B * S + B, (float)(-2 * gB), 1.0f);      // dN_BB = -2 g_B
        if (gB != gA) term(base + A * S + B, (float)(gB - gA), 2.0f);     // dN_AB = dN_BA = g_B - g_A
        for (int y = 0; y < S; ++y) {
            if (y == A || y == B) continue;
            const int gy = g_of(g_k, y);
            if (gy == 0) continue;
            term(base + A * S + y, (float)gy, 2.0f);    // dN_Ay = dN_yA = g_y
            term(base + B * S + y, (float)(-gy), 2.0f); // dN_By = dN_yB = -g_y
        }
    }
    D = acc;
    err = fmaf(mag, rel, kAbsBound);
}

__device__ __forceinline__ bool eligible(double D, bool null_move, double threshold) {
    if (null_move) return false;
    if (D < 0.0) return true;
    return threshold > 0.0 && D <= threshold;
}

// Eligibility from an interval [lo, hi] around the key: 1 eligible, 0 not, -1 undecided.
// thr_lo / thr_hi are the binary32 neighbours below / above the threshold (both 0 for 0).
__device__ __forceinline__ int eligible_interval(float lo, float hi, bool positive_thr, float thr_lo, float thr_hi) {
    if (positive_thr) return (hi <= thr_lo) ? 1 : ((lo > thr_hi) ? 0 : -1);
    return (hi < 0.f) ? 1 : ((lo >= 0.f) ? 0 : -1);
}

// Coefficients during the multi-accept walk.  At the start of a step entry e has the binary64
// error e0 and coefficient b0, the FP32 copies fe0 = fl(e0) and fb = fl(b0), and dn = 0.  After the
// walk changes its count by dn, the running values are e = e0 - dn Q and b = -2 (w (Q e)); in FP32
// e_f = fe0 - dn fQ and fb = -2 (fw (fQ e_f)).  With u = 2^-24 these are within
// 2 w Q (5 u (|e0| + |dn Q|)) + 2 w Q 2^-51 (2 + |t| + |e0|) of the real values, and the binary64
// coefficient the exact running key uses is within 2 w Q 2^-50 (1 + |n Q| + |t| + |e|) of them.
// beta_e = 2 w Q 2^-20 (|fe0| + |dn fQ|) + tiny_e, with the count-independent
// tiny_e = 2 w Q 2^-46 (4 + 2 N / N_j + 2 |t|) (|n Q| <= N / N_j, |e| <= 1 + N / N_j + |t|), bounds
// the distance of fb to both; at the start of a step beta_e = 2^-23 |fb| + tiny_e.
constexpr float kTwoPow20 = 9.5367431640625e-07f;   // 2^-20

__device__ __forceinline__ void running_coefficient(int e, int dn, float w, const float* fQ, const float* fe0,
                                                    const float* tiny, float* fb, float* beta) {
    const float dq = (float)dn * fQ[e];
    const float ef = fe0[e] - dq;
    fb[e] = -2.0f * (w * (fQ[e] * ef));
    beta[e] = fmaf(2.0f * w * fQ[e], kTwoPow20 * (fabsf(fe0[e]) + fabsf(dq)), tiny[e]);
}

__device__ __forceinline__ bool better(double D1, uint32_t k1, double D2, uint32_t k2) {
    return D1 < D2 || (D1 == D2 && k1 < k2);
}

// Order-preserving integer image of a key (no NaNs; -0 and +0 map to the same value), so that the
// ranking loops compare integers instead of binary64 values.
__device__ __forceinline__ uint64_t order_key(double D) {
    long long bits = __double_as_longlong(D);
    if ((bits & 0x7FFFFFFFFFFFFFFFll) == 0) bits = 0;
    return bits < 0 ? ~(uint64_t)bits : ((uint64_t)bits | 0x8000000000000000ull);
}

__device__ __forceinline__ bool better_key(uint64_t K1, uint32_t k1, uint64_t K2, uint32_t k2) {
    return K1 < K2 || (K1 == K2 && k1 < k2);
}

// Site index of the point at half-unit position (X, Y, Z) + the shell vector packed in `pv`
// (signed bytes dx, dy, dz).
__device__ __forceinline__ int unpack_comp(uint32_t pv, int c) { return (int)(int8_t)((pv >> (8 * c)) & 0xFFu); }

template <int KIND>
__device__ __forceinline__ uint32_t neighbour_at(const Geo& g, int X, int Y, int Z, uint32_t pv) {
    int x = X + unpack_comp(pv, 0), y = Y + unpack_comp(pv, 1), z = Z + unpack_comp(pv, 2);
    const int PX = 2 * g.Lx, PY = 2 * g.Ly, PZ = 2 * g.Lz;
    x += (x < 0) ? PX : 0;
    x -= (x >= PX) ? PX : 0;
    y += (y < 0) ? PY : 0;
    y -= (y >= PY) ? PY : 0;
    z += (z < 0) ? PZ : 0;
    z -= (z >= PZ) ? PZ : 0;
    const int b = (KIND == kFCC) ? 2 * (x & 1) + (y & 1) : (x & 1);
    return (uint32_t)(b * g.V + (z >> 1) * g.LxLy + (y >> 1) * g.Lx + (x >> 1));
}

// Sets (or clears) the bits of the closed shell neighbourhood of `site` in the walk bitmap; the
// calling lanes split the Z_tot + 1 sites between them.  `vec` is the shell-vector table in
// shared memory.
template <int KIND, bool SET>
__device__ __forceinline__ void mark_neighbourhood(const Geo& g, uint32_t site, int ztot, int lane, int lanes,
                                                   const uint32_t* vec, uint32_t* bitmap) {
    int X, Y, Z;
    site_coords<KIND>(g, site, X, Y, Z);
    for (int v = lane; v <= ztot; v += lanes) {
        const uint32_t s = (v == 0) ? site : neighbour_at<KIND>(g, X, Y, Z, vec[v - 1]);
        if (SET)
            atomicOr(&bitmap[s >> 5], 1u << (s & 31));
        else
            atomicAnd(&bitmap[s >> 5], ~(1u << (s & 31)));
    }
}

// Pointers into a chain's shared memory.
struct ChainSmem {
    uint8_t* types;
    int32_t* cnt;
    double *Q, *tgt, *ca, *cb;
    float *fa, *fb, *fQ, *fe0, *tiny, *beta;
    int32_t* dn;
    uint32_t* vec;
    uint16_t* slot;
    uint32_t *qk, *qa, *qb;
    float *qlo, *qhi;
    double* qD;
    uint64_t* qkey;
    uint64_t* qg;
    float* fw;
    uint32_t *order, *acc, *bitmap;
    long long *fA, *fB, *qfix, *qeps;
    uint32_t* qflag;
    uint8_t* walk;

    __device__ ChainSmem(uint8_t* smem, const ChainLayout& L) {
        fA = reinterpret_cast<long long*>(smem + L.fA);
        fB = reinterpret_cast<long long*>(smem + L.fB);
        qfix = reinterpret_cast<long long*>(smem + L.qfix);
        qeps = reinterpret_cast<long long*>(smem + L.qeps);
        qflag = reinterpret_cast<uint32_t*>(smem + L.qflag);
        walk = smem + L.walk;
        types = smem + L.types;
        cnt = reinterpret_cast<int32_t*>(smem + L.cnt);
        Q = reinterpret_cast<double*>(smem + L.Q);
        tgt = reinterpret_cast<double*>(smem + L.tgt);
        ca = reinterpret_cast<double*>(smem + L.ca);
        cb = reinterpret_cast<double*>(smem + L.cb);
        fa = reinterpret_cast<float*>(smem + L.fa);
        fb = reinterpret_cast<float*>(smem + L.fb);
        fQ = reinterpret_cast<float*>(smem + L.fQ);
        fe0 = reinterpret_cast<float*>(smem + L.fe0);
        tiny = reinterpret_cast<float*>(smem + L.tiny);
        beta = reinterpret_cast<float*>(smem + L.beta);
        dn = reinterpret_cast<int32_t*>(smem + L.dn);
        vec = reinterpret_cast<uint32_t*>(smem + L.vec);
        slot = reinterpret_cast<uint16_t*>(smem + L.slot);
        qk = reinterpret_cast<uint32_t*>(smem + L.qk);
        qa = reinterpret_cast<uint32_t*>(smem + L.qa);
        qb = reinterpret_cast<uint32_t*>(smem + L.qb);
        qlo = reinterpret_cast<float*>(smem + L.qlo);
        qhi = reinterpret_cast<float*>(smem + L.qhi);
        qD = reinterpret_cast<double*>(smem + L.qD);
        qkey = reinterpret_cast<uint64_t*>(smem + L.qkey);
        qg = reinterpret_cast<uint64_t*>(smem + L.qg);
        fw = reinterpret_cast<float*>(smem + L.fw);
        order = reinterpret_cast<uint32_t*>(smem + L.order);
        acc = reinterpret_cast<uint32_t*>(smem + L.acc);
        bitmap = reinterpret_cast<uint32_t*>(smem + L.bitmap);
    }
};

// Per-chain constants derived from the descriptor.
struct ChainCtx {
    Geo g;
    int M, S, E, K, ztot;
    uint32_t N;
    double thr;
    uint32_t seed_lo, seed_hi;
    bool use_filter;
    float rel;   // (E + 4) 2^-23: relative part of the FP32 key bound
    int qcap;    // candidate slots in shared memory
    int r2max;   // |d|^2 of shell M, half units^2
    bool alias;  // some axis has at most reach(M) + 1 cells: two shell vectors may reach the same site
    bool packed; // species below 8 bits and Lx a multiple of the sites per byte (split gathers)
    bool sym;    // Q and the target symmetric bit for bit: every coefficient table stays symmetric
    bool pos_thr;            // threshold > 0
    float thr_lo, thr_hi;    // binary32 neighbours of the threshold
};

// ---- set-up: species (validated against S), counts, coefficients, shell vectors ----------------
template <int KIND, int BITS>
__device__ void chain_setup(const ChainDesc& d, ChainSmem& m, ChainShared& sh, ChainCtx& c, bool clear_bitmap = true) {
    const int tid = threadIdx.x, T = blockDim.x;
    c.g = make_geo(KIND, d.Lx, d.Ly, d.Lz);
    c.M = d.M;
    c.S = d.S;
    c.E = d.M * d.S * d.S;
    c.K = d.K;
    c.N = (uint32_t)d.N;
    c.thr = d.threshold;
    c.seed_lo = (uint32_t)(d.seed & 0xFFFFFFFFu);
    c.seed_hi = (uint32_t)(d.seed >> 32);
    c.rel = (float)(c.E + 4) * kTwoUlp;
    c.qcap = d.qcap;
    c.r2max = c_shells[KIND].radius2[d.M - 1];
    c.alias = min(d.Lx, min(d.Ly, d.Lz)) <= c_shells[KIND].reach[d.M - 1] + 1;
    c.packed = BITS < 8 && d.Lx % (8 / BITS) == 0;
    c.pos_thr = d.threshold > 0.0;
    {
        float f = (float)d.threshold;
        c.thr_lo = ((double)f > d.threshold) ? nextafterf(f, -CUDART_INF_F) : f;
        c.thr_hi = ((double)f < d.threshold) ? nextafterf(f, CUDART_INF_F) : f;
    }
    const ShellTable& TAB = c_shells[KIND];
    c.ztot = TAB.first[c.M];
    const int S = c.S, E = c.E;
    const uint32_t N = c.N;
    if (tid == 0) {
        sh.bad = 0;
        sh.use_filter = 1;
        sh.depth = d.depth0;
        sh.status = HEA_OK;
        sh.steps = 0;
        sh.accepted = 0;
        sh.stop = (d.max_steps <= 0);
        sh.t0 = globaltimer_ns();
    }
    __syncthreads();
    if (BITS == 8) {
        for (uint32_t i = tid; i < N; i += T) {
            const uint8_t v = d.types[i];
            if (v >= S) sh.bad = 1;
            m.types[i] = v;
        }
    } else {
        constexpr uint32_t per = 8 / BITS;
        for (uint32_t i = tid; i < species_bytes<BITS>(N); i += T) {
            uint32_t packed = 0;
#pragma unroll
            for (uint32_t j = 0; j < per; ++j) {
                const uint8_t v = (per * i + j < N) ? d.types[per * i + j] : 0;
                if (v >= S) sh.bad = 1;
                packed |= (uint32_t)(v & ((1u << BITS) - 1u)) << (BITS * j);
            }
            m.types[i] = (uint8_t)packed;
        }
    }
    {
        const int P = 4 * S - 4;   // entries a swap touches per shell
        for (int f = tid; f < c.M * P; f += T) m.slot[f] = (uint16_t)(((f / P) << 8) | (f % P));
    }
    for (int v = tid; v < c.ztot; v += T)
        m.vec[v] = (uint32_t)(uint8_t)TAB.v[v][0] | ((uint32_t)(uint8_t)TAB.v[v][1] << 8) |
                   ((uint32_t)(uint8_t)TAB.v[v][2] << 16);
    for (int e = tid; e < E; e += T) {
        const int k = e / (S * S), i = (e / S) % S, j = e % S;
        const double w = d.w[k];
        const double den = __dmul_rn(__dmul_rn((double)TAB.z[k], (double)d.n_per[i]), (double)d.n_per[j]);
        const double Q = __ddiv_rn((double)d.N, den);
        const int n = d.counts[e];
        const double t = d.target[e];
        const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)n, Q)), t);
        const double a = __dmul_rn(w, __dmul_rn(Q, Q));
        const double b = __dmul_rn(-2.0, __dmul_rn(w, __dmul_rn(Q, err)));
        m.cnt[e] = n;
        m.Q[e] = Q;
        m.tgt[e] = t;
        m.ca[e] = a;
        m.cb[e] = b;
        m.fa[e] = (float)a;
        m.fb[e] = (float)b;
        m.fQ[e] = (float)Q;
        m.fw[e] = (float)w;
        m.fe0[e] = (float)err;
        m.dn[e] = 0;
        m.tiny[e] = (float)(2.0 * w * Q * 1.4210854715202004e-14 * (4.0 + 2.0 * (double)d.N / (double)d.n_per[j] + 2.0 * fabs(t)));
        m.beta[e] = fmaf(kTwoUlp, fabsf(m.fb[e]), m.tiny[e]);
        // The FP32 estimate needs every |a| dN^2 and |b| dN to stay far inside the float range;
        // |e| <= 1 + N / N_j + |t| bounds b over the whole search.
        const double zz = 2.0 * TAB.z[k];
        const double bmax = 2.0 * w * Q * (1.0 + (double)d.N / (double)d.n_per[j] + fabs(t));
        if (!(a * zz * zz < 1e30) || !(bmax * zz < 1e30)) sh.use_filter = 0;
    }
    if (d.accept_mode == 1 && clear_bitmap)
        for (uint32_t i = tid; i < (N + 31) / 32; i += T) m.bitmap[i] = 0;
    if (tid == 0) sh.asym = 0;
    __syncthreads();
    for (int e = tid; e < E; e += T) {
        const int k = e / (S * S), i = (e / S) % S, j = e % S;
        const int f = (k * S + j) * S + i;
        if (__double_as_longlong(m.Q[e]) != __double_as_longlong(m.Q[f]) ||
            __double_as_longlong(m.tgt[e]) != __double_as_longlong(m.tgt[f]))
            sh.asym = 1;
    }
    __syncthreads();
    c.use_filter = sh.use_filter != 0;
    c.sym = sh.asym == 0;
}

// Minimum-image squared length (half units^2) of a displacement between two sites of the cell.
__device__ __forceinline__ int min_image_r2(int dx, int dy, int dz, const Geo& g) {
    const int PX = 2 * g.Lx, PY = 2 * g.Ly, PZ = 2 * g.Lz;
    dx = dx < 0 ? -dx : dx;
    dy = dy < 0 ? -dy : dy;
    dz = dz < 0 ? -dz : dz;
    dx = min(dx, PX - dx);
    dy = min(dy, PY - dy);
    dz = min(dz, PZ - dz);
    return dx * dx + dy * dy + dz * dz;
}

// ---- 1. score candidates k in [k_begin, k_end) of step `step`; queue the ones that may matter ----
// Returns this thread's minimum of the upper bounds (null moves count as 0).
template <int KIND, int BITS>
__device__ float score_range(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c, uint32_t step,
                             uint32_t k_begin, uint32_t k_end) {
    constexpr int MX = kMaxShells;
    const int M = c.M;
    auto onehot = [&](uint32_t n) -> uint64_t { return 1ull << (8 * load_species<BITS>(m.types, n)); };
    float my_umin = CUDART_INF_F;
    for (uint32_t kk = k_begin + threadIdx.x; kk < k_end; kk += blockDim.x) {
        const Rand4 r = philox(kk, step, d.chain, 1u, c.seed_lo, c.seed_hi);
        const uint32_t a = __umulhi(r.r0, c.N), b = __umulhi(r.r1, c.N);
        const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
        if (a == b || A == B) {
            my_umin = fminf(my_umin, 0.f);
            if (c.thr > 0.0) {
                const int slot = atomicAdd(&sh.qn, 1);
                m.qk[slot] = kk;
                m.qa[slot] = a;
                m.qb[slot] = b;
                m.qlo[slot] = 0.f;
                m.qhi[slot] = 0.f;
                for (int k = 0; k < M; ++k) m.qg[slot * M + k] = kGBias;
            }
            continue;
        }
        // Histograms of both sites.  b can be a shell neighbour of a only when their minimum-image
        // squared distance is at most r2 of shell M; otherwise no neighbour needs skipping.  With at
        // most four species the 8-bit fields fit one 32-bit word.
        // Outside small cells a shell vector from a reaches b only when it equals their minimum-image
        // displacement, so a near pair is handled by taking the partner's species out of the one
        // shell whose radius is their distance; this keeps every candidate on one code path (a lane
        // on a separate path stalls its warp and fetches cold code).  Small cells (two vectors may
        // reach the same site) skip every vector that reaches the partner.
        int Xa, Ya, Za, Xb, Yb, Zb;
        site_coords<KIND>(c.g, a, Xa, Ya, Za);
        site_coords<KIND>(c.g, b, Xb, Yb, Zb);
        const int r2ab = min_image_r2(Xb - Xa, Yb - Ya, Zb - Za, c.g);
        const bool near = r2ab <= c.r2max;
        const bool skip = near && c.alias;
        uint64_t gb[MX];
        if (c.S <= 4) {
            auto onehot32 = [&](uint32_t n) -> uint32_t { return 1u << (8 * load_species<BITS>(m.types, n)); };
            uint32_t ha[MX], hb[MX];
            if (skip) {
                neighbour_histogram_at<KIND, MX, true, uint32_t>(c.g, Xa, Ya, Za, b, onehot32, ha, M);
                neighbour_histogram_at<KIND, MX, true, uint32_t>(c.g, Xb, Yb, Zb, a, onehot32, hb, M);
            } else {
                bool done = false;
                if constexpr (BITS < 8) {
                    if (c.packed && M <= 3) {
                        // shells 1-3 only: axis tables of reach 2 and no code for shells 4-5
                        uint32_t h3a[3], h3b[3];
                        neighbour_histogram_packed<KIND, 3, BITS, uint32_t>(c.g, Xa, Ya, Za, m.types, h3a, M);
                        neighbour_histogram_packed<KIND, 3, BITS, uint32_t>(c.g, Xb, Yb, Zb, m.types, h3b, M);
#pragma unroll
                        for (int k = 0; k < MX; ++k) {
                            ha[k] = k < 3 ? h3a[k < 3 ? k : 0] : 0u;
                            hb[k] = k < 3 ? h3b[k < 3 ? k : 0] : 0u;
                        }
                        done = true;
                    } else if (c.packed) {
                        neighbour_histogram_packed<KIND, MX, BITS, uint32_t>(c.g, Xa, Ya, Za, m.types, ha, M);
                        neighbour_histogram_packed<KIND, MX, BITS, uint32_t>(c.g, Xb, Yb, Zb, m.types, hb, M);
                        done = true;
                    }
                }
                if (!done) {
                    neighbour_histogram_at<KIND, MX, false, uint32_t>(c.g, Xa, Ya, Za, 0u, onehot32, ha, M);
                    neighbour_histogram_at<KIND, MX, false, uint32_t>(c.g, Xb, Yb, Zb, 0u, onehot32, hb, M);
                }
                if (near) {
#pragma unroll
                    for (int k = 0; k < MX; ++k)
                        if (k < M && c_shells[KIND].radius2[k] == r2ab) {
                            ha[k] -= 1u << (8 * B);
                            hb[k] -= 1u << (8 * A);
                        }
                }
            }
#pragma unroll
            for (int k = 0; k < MX; ++k) gb[k] = pack_g(ha[k], hb[k]);
        } else {
            uint64_t ha[MX], hb[MX];
            if (skip) {
                neighbour_histogram_at<KIND, MX, true, uint64_t>(c.g, Xa, Ya, Za, b, onehot, ha, M);
                neighbour_histogram_at<KIND, MX, true, uint64_t>(c.g, Xb, Yb, Zb, a, onehot, hb, M);
            } else {
                neighbour_histogram_at<KIND, MX, false, uint64_t>(c.g, Xa, Ya, Za, 0u, onehot, ha, M);
                neighbour_histogram_at<KIND, MX, false, uint64_t>(c.g, Xb, Yb, Zb, 0u, onehot, hb, M);
                if (near) {
#pragma unroll
                    for (int k = 0; k < MX; ++k)
                        if (k < M && c_shells[KIND].radius2[k] == r2ab) {
                            ha[k] -= 1ull << (8 * B);
                            hb[k] -= 1ull << (8 * A);
                        }
                }
            }
#pragma unroll
            for (int k = 0; k < MX; ++k) gb[k] = pack_g(ha[k], hb[k]);
        }
        float lo = -CUDART_INF_F, hi = CUDART_INF_F;
        if (c.use_filter) {
            // g = 0 in every shell (the two sites see the same species counts): no count changes,
            // and the key is exactly 0 (the binary64 chain skips every entry)
            bool zero = true;
#pragma unroll
            for (int k = 0; k < MX; ++k) zero = zero && (k >= M || gb[k] == kGBias);
            if (zero) {
                lo = 0.f;
                hi = 0.f;
            } else {
                float Dt, err;
                if (c.sym)
                    score_float_sym(M, c.S, m.fa, m.fb, A, B, gb, c.rel, Dt, err);
                else
                    score_float(M, c.S, m.fa, m.fb, A, B, gb, c.rel, Dt, err);
                hi = __fadd_ru(Dt, err);
                lo = __fadd_rd(Dt, -err);
            }
            my_umin = fminf(my_umin, hi);
            if (c.pos_thr ? (lo > c.thr_hi) : (lo >= 0.f)) continue;   // cannot be accepted
        }
        const int slot = atomicAdd(&sh.qn, 1);
        m.qk[slot] = kk;
        m.qa[slot] = a;
        m.qb[slot] = b;
        m.qlo[slot] = lo;
        m.qhi[slot] = hi;
#pragma unroll
        for (int k = 0; k < MX; ++k)
            if (k < M) m.qg[slot * M + k] = gb[k];
    }
    return my_umin;
}

__device__ __forceinline__ float block_min(float v, ChainShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if (lane == 0) sh.red_f[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float u = CUDART_INF_F;
        for (int w = 0; w < nw; ++w) u = fminf(u, sh.red_f[w]);
        sh.umin = u;
    }
    __syncthreads();
    return sh.umin;
}

// ---- best-of-K: exact keys of the contenders, block argmin over (D, k) --------------------------
// A contender is a queued candidate with lo <= min(umin, threshold): the argmin, whenever it is
// acceptable, is one of them.  Sets sh.win_q to the best slot, or -1.
template <int BITS>
// need_key = false (single chain): with exactly one contender the argmin needs no key, and its
// eligibility is taken from its FP32 interval when that settles it (sh.win_elig 1 / 0; -1: the
// caller decides on the binary64 key in m.qD).
__device__ void best_of_queue(ChainSmem& m, ChainShared& sh, const ChainCtx& c, float umin, bool need_key = true) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double tau = c.use_filter ? fmin((double)umin, c.thr) : CUDART_INF;
    double bD = CUDART_INF;
    uint32_t bk = 0xFFFFFFFFu;
    int bq = -1;
    const int qn = sh.qn;
    if (threadIdx.x == 0) sh.win_elig = -1;
    if (!need_key && c.use_filter) {
        int mine = 0, mq = -1;
        for (int q = threadIdx.x; q < qn; q += blockDim.x)
            if (!((double)m.qlo[q] > tau)) {
                ++mine;
                mq = q;
            }
        const int holders = __syncthreads_count(mine > 0);
        const int several = __syncthreads_or(mine > 1);
        if (holders == 1 && !several) {
            if (mine == 1) {
                sh.win_q = mq;
                const int v = eligible_interval(m.qlo[mq], m.qhi[mq], c.pos_thr, c.thr_lo, c.thr_hi);
                if (v >= 0) {
                    sh.win_elig = v;
                } else {
                    const uint32_t a = m.qa[mq], b = m.qb[mq];
                    const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
                    m.qD[mq] = (a == b || A == B) ? 0.0 : exact_key(c.M, c.S, m.ca, m.cb, A, B, m.qg + mq * c.M);
                }
            }
            __syncthreads();
            return;
        }
        if (holders == 0) {
            if (threadIdx.x == 0) sh.win_q = -1;
            __syncthreads();
            return;
        }
    }
    for (int q = threadIdx.x; q < qn; q += blockDim.x) {
        if (c.use_filter && (double)m.qlo[q] > tau) continue;
        const uint32_t a = m.qa[q], b = m.qb[q];
        const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
        const double D = (a == b || A == B) ? 0.0 : exact_key(c.M, c.S, m.ca, m.cb, A, B, m.qg + q * c.M);
        m.qD[q] = D;
        if (better(D, m.qk[q], bD, bk)) {
            bD = D;
            bk = m.qk[q];
            bq = q;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oD = __shfl_xor_sync(0xFFFFFFFFu, bD, o);
        const uint32_t ok = __shfl_xor_sync(0xFFFFFFFFu, bk, o);
        const int oq = __shfl_xor_sync(0xFFFFFFFFu, bq, o);
        if (better(oD, ok, bD, bk)) {
            bD = oD;
            bk = ok;
            bq = oq;
        }
    }
    if (lane == 0) {
        sh.red_d[warp] = bD;
        sh.red_k[warp] = bk;
        sh.red_q[warp] = bq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double D = CUDART_INF;
        uint32_t k = 0xFFFFFFFFu;
        int q = -1;
        for (int w = 0; w < nw; ++w)
            if (better(sh.red_d[w], sh.red_k[w], D, k)) {
                D = sh.red_d[w];
                k = sh.red_k[w];
                q = sh.red_q[w];
            }
        sh.win_q = q;
    }
    __syncthreads();
}

// Applies the swap in slot q (known acceptable) to species, counts and coefficients.
template <int BITS>
__device__ void apply_slot(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c, int q) {
    const uint32_t a = m.qa[q], b = m.qb[q];
    const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
    const int S = c.S;
    for (int e = threadIdx.x; e < c.E; e += blockDim.x) {
        const int k = e / (S * S), i = (e / S) % S, j = e % S;
        const int dl = entry_delta(m.qg[q * c.M + k], A, B, i, j);
        if (dl == 0) continue;
        const int n = m.cnt[e] + dl;
        m.cnt[e] = n;
        const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)n, m.Q[e])), m.tgt[e]);
        const double bcoef = __dmul_rn(-2.0, __dmul_rn(d.w[k], __dmul_rn(m.Q[e], err)));
        m.cb[e] = bcoef;
        m.fb[e] = (float)bcoef;
        m.fe0[e] = (float)err;
        m.beta[e] = fmaf(kTwoUlp, fabsf(m.fb[e]), m.tiny[e]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        store_species<BITS>(m.types, a, B);
        store_species<BITS>(m.types, b, A);
        sh.n_acc = 1;
    }
}

// Sorts idx[0, n) ascending under `less` (a strict total order on the indices) with an
// all-ascending bitonic network (each merge starts with a flip); positions >= n act as +infinity,
// so n need not be a power of two.  Every thread of the CTA must call it.
template <typename Less>
__device__ void block_sort(uint32_t* idx, int n, Less less) {
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    const int P = 1 << lg;
    for (int ls = 1; ls <= lg; ++ls) {
        const int size = 1 << ls, half = size >> 1;
        for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
            const int i = ((t >> (ls - 1)) << ls) | (t & (half - 1));
            const int j = i ^ (size - 1);
            if (j < n) {
                const uint32_t a = idx[i], b = idx[j];
                if (less(b, a)) {
                    idx[i] = b;
                    idx[j] = a;
                }
            }
        }
        __syncthreads();
        for (int lst = ls - 2; lst >= 0; --lst) {
            const int stride = 1 << lst;
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int i = ((t >> lst) << (lst + 1)) | (t & (stride - 1));
                const int j = i + stride;
                if (j < n) {
                    const uint32_t a = idx[i], b = idx[j];
                    if (less(b, a)) {
                        idx[i] = b;
                        idx[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Order-preserving compaction of src[0, n) where keep(s) into dst; returns the count (all threads).
template <typename Keep>
__device__ int block_compact(const uint32_t* src, int n, uint32_t* dst, Keep keep, ChainShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int base = 0;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const bool k = (s < n) && keep(s);
        const uint32_t ball = __ballot_sync(0xFFFFFFFFu, k);
        if (lane == 0) sh.red_k[warp] = __popc(ball);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < nw; ++w) {
                const int cw = (int)sh.red_k[w];
                sh.red_k[w] = (uint32_t)acc;
                acc += cw;
            }
            sh.red_q[0] = acc;
        }
        __syncthreads();
        const uint32_t v = (s < n) ? src[s] : 0u;
        if (k) dst[base + (int)sh.red_k[warp] + __popc(ball & ((1u << lane) - 1u))] = v;
        base += sh.red_q[0];
        __syncthreads();
    }
    return base;
}

// ---- multi-accept: eligible candidates of slots [0, n) ranked by (D, k) into m.order ------------
// Eligibility is decided on the interval where it can be and on the exact key otherwise; among the
// eligible, a candidate gets its exact key when its interval overlaps another one's.  Ranking by
// (exact key, or the interval midpoint; k) is then the ranking by (D, k): disjoint intervals order
// their keys, overlapping ones are ordered by exact keys.  With group_top > 0 only the group_top
// best of each group (k / group_size) stay.  Sets sh.n_elig.
template <int BITS>
__device__ void rank_eligible(ChainSmem& m, ChainShared& sh, const ChainCtx& c, int n, int group_size,
                              int group_top, bool single_group) {
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid == 0) sh.n_elig = 0;
    __syncthreads();
    for (int q = tid; q < n; q += T) {
        const uint32_t a = m.qa[q], b = m.qb[q];
        const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
        if (a == b || A == B) continue;   // null moves are never accepted
        int v = eligible_interval(m.qlo[q], m.qhi[q], c.pos_thr, c.thr_lo, c.thr_hi);
        bool exact = false;
        if (v < 0) {
            m.qD[q] = exact_key(c.M, c.S, m.ca, m.cb, A, B, m.qg + q * c.M);
            v = eligible(m.qD[q], false, c.thr) ? 1 : 0;
            exact = true;
        }
        if (v == 1) {
            if (!exact) m.qD[q] = 0.5 * ((double)m.qlo[q] + (double)m.qhi[q]);
            m.acc[atomicAdd(&sh.n_elig, 1)] = (uint32_t)q | (exact ? 0x80000000u : 0u);
        }
    }
    __syncthreads();
    const int ne = sh.n_elig;
    // Overlaps: sorted by lower bound, interval s overlaps another iff the largest upper bound
    // before it reaches its lower bound or its successor's lower bound is within it.
    for (int s = tid; s < ne; s += T) m.order[s] = m.acc[s];
    __syncthreads();
    block_sort(m.order, ne, [&](uint32_t x, uint32_t y) {
        const uint32_t qx = x & 0x7FFFFFFFu, qy = y & 0x7FFFFFFFu;
        return m.qlo[qx] < m.qlo[qy] || (m.qlo[qx] == m.qlo[qy] && qx < qy);
    });
    float* pm = reinterpret_cast<float*>(m.qkey);   // prefix maxima of the upper bounds (ping-pong)
    float* pm2 = pm + c.qcap;
    for (int s = tid; s < ne; s += T) pm[s] = m.qhi[m.order[s] & 0x3FFFFFFFu];
    __syncthreads();
    for (int dd = 1; dd < ne; dd <<= 1) {
        for (int s = tid; s < ne; s += T) pm2[s] = (s >= dd) ? fmaxf(pm[s], pm[s - dd]) : pm[s];
        __syncthreads();
        float* tmp = pm;
        pm = pm2;
        pm2 = tmp;
    }
    // Cluster starts (bit 30): no earlier interval reaches this one.  Clusters are contiguous in
    // this order and strictly ordered against each other.
    for (int s = tid; s < ne; s += T) {
        const uint32_t q = m.order[s] & 0x3FFFFFFFu;
        const bool start = (s == 0) || (pm[s - 1] < m.qlo[q]);
        if (start) m.order[s] |= 0x40000000u;
    }
    __syncthreads();
    for (int s = tid; s < ne; s += T) {
        const uint32_t x = m.order[s] & ~0x40000000u;
        if (x & 0x80000000u) continue;   // already exact
        const uint32_t q = x & 0x7FFFFFFFu;
        const bool before = (s > 0) && (pm[s - 1] >= m.qlo[q]);
        const bool after = (s + 1 < ne) && (m.qlo[m.order[s + 1] & 0x3FFFFFFFu] <= m.qhi[q]);
        if (before || after) {
            const int A = load_species<BITS>(m.types, m.qa[q]), B = load_species<BITS>(m.types, m.qb[q]);
            m.qD[q] = exact_key(c.M, c.S, m.ca, m.cb, A, B, m.qg + q * c.M);
        }
    }
    __syncthreads();
    for (int s = tid; s < ne; s += T) {
        const uint32_t q = m.acc[s] & 0x7FFFFFFFu;
        m.acc[s] = q;
        m.qkey[q] = order_key(m.qD[q]);
    }
    __syncthreads();
    int keep = ne;
    if (single_group) {
        // The order by lower bound, with every cluster sorted by (key, k), is the order by (D, k).
        if (tid == 0) sh.red_k[0] = 0u;
        __syncthreads();
        for (int s = tid; s < ne; s += T) {
            if ((m.order[s] & 0x40000000u) == 0u) continue;
            int e = s + 1;
            while (e < ne && (m.order[e] & 0x40000000u) == 0u) ++e;
            if (e - s > 1) atomicMax(&sh.red_k[0], (uint32_t)(e - s));
            if (e - s > 1 && e - s <= 32) {
                for (int x = s; x < e; ++x) m.order[x] &= 0x3FFFFFFFu;
                for (int x = s + 1; x < e; ++x) {
                    const uint32_t v = m.order[x];
                    int y = x - 1;
                    while (y >= s && better_key(m.qkey[v], m.qk[v], m.qkey[m.order[y]], m.qk[m.order[y]])) {
                        m.order[y + 1] = m.order[y];
                        --y;
                    }
                    m.order[y + 1] = v;
                }
            }
        }
        __syncthreads();
        for (int s = tid; s < ne; s += T) m.order[s] &= 0x3FFFFFFFu;
        __syncthreads();
        if (sh.red_k[0] > 32u)
            block_sort(m.order, ne, [&](uint32_t x, uint32_t y) {
                return better_key(m.qkey[x], m.qk[x], m.qkey[y], m.qk[y]);
            });
        if (group_top > 0 && keep > group_top) keep = group_top;
    } else {
        // Ranking by (group, key, k); the group rule keeps the first group_top of every group.
        const uint32_t G = (uint32_t)(group_size > 0 ? group_size : c.K);
        block_sort(m.acc, ne, [&](uint32_t x, uint32_t y) {
            const uint32_t gx = m.qk[x] / G, gy = m.qk[y] / G;
            return gx < gy || (gx == gy && better_key(m.qkey[x], m.qk[x], m.qkey[y], m.qk[y]));
        });
        keep = block_compact(m.acc, ne, m.order, [&](int s) {
            return s < group_top || (m.qk[m.acc[s - group_top]] / G != m.qk[m.acc[s]] / G);
        }, sh);
        block_sort(m.order, keep, [&](uint32_t x, uint32_t y) {
            return better_key(m.qkey[x], m.qk[x], m.qkey[y], m.qk[y]);
        });
    }
    if (tid == 0) sh.n_elig = keep;
    __syncthreads();
}

// The entries a swap of species A and B can change, per shell: row A, row B (S entries each), then
// columns A and B of the S - 2 other rows.  Slot s of shell k -> entry (k, i, j).
__device__ __forceinline__ void swap_entry(int S, int A, int B, int s, int& i, int& j) {
    if (s < S) {
        i = A;
        j = s;
    } else if (s < 2 * S) {
        i = B;
        j = s - S;
    } else {
        int t = s - 2 * S;
        if (t >= S - 2) t -= S - 2;
        const int lo = A < B ? A : B, hi = A < B ? B : A;
        int r = t;
        r += (r >= lo) ? 1 : 0;
        r += (r >= hi) ? 1 : 0;
        i = r;
        j = (s < 3 * S - 2) ? A : B;
    }
}

// ---- multi-accept walk over m.order[0, ne) by warp 0 (sequential by definition) ----------------
// Each re-check against the running counts is an FP32 estimate over the lanes with a rigorous
// bound (the FP32 bound above plus beta for the running coefficients); the exact binary64 key is
// computed only when the bound cannot decide eligibility.
template <int KIND, int BITS>
__device__ void walk_bitmap(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c, int ne) {
    const int lane = threadIdx.x & 31;
    for (uint32_t i = threadIdx.x; i < (c.N + 31) / 32; i += blockDim.x) m.bitmap[i] = 0;
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        const int S = c.S, M = c.M, SS = S * S;
        const int P = 4 * S - 4;   // entries a swap touches per shell
        int n_acc = 0;
        for (int r = 0; r < ne; ++r) {
            if (d.max_accept > 0 && n_acc >= d.max_accept) break;
            const uint32_t q = m.order[r];
            const uint32_t a = m.qa[q], b = m.qb[q];
            const bool blocked = ((m.bitmap[a >> 5] >> (a & 31)) & 1u) | ((m.bitmap[b >> 5] >> (b & 31)) & 1u);
            if (blocked) continue;
            const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
            const uint64_t* gq = m.qg + q * M;
            bool take = true;   // before the first accept the running state is the step-start state
            if (n_acc > 0) {
                float acc = 0.f, err = 0.f;
                for (int f = lane; f < M * P; f += 32) {
                    const int v = m.slot[f], k = v >> 8;
                    int i, j;
                    swap_entry(S, A, B, v & 0xFF, i, j);
                    const int dl = entry_delta(gq[k], A, B, i, j);
                    if (dl == 0) continue;
                    const int e = k * SS + i * S + j;
                    const float x = (float)dl, ax = fabsf(x);
                    acc = fmaf(x, fmaf(m.fa[e], x, m.fb[e]), acc);
                    err = fmaf(ax, fmaf(c.rel * fabsf(m.fa[e]), ax, fmaf(c.rel, fabsf(m.fb[e]), m.beta[e])), err);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                    err += __shfl_xor_sync(0xFFFFFFFFu, err, o);
                }
                // A few extra relative ulps cover the rounding of the lane sums.
                err = fmaf(err, 1.0f + 64.0f * kTwoUlp, kAbsBound);
                int verdict = eligible_interval(__fadd_rd(acc, -err), __fadd_ru(acc, err), c.pos_thr, c.thr_lo, c.thr_hi);
                if (verdict < 0) {
                    double Dp = 0.0;
                    if (lane == 0) Dp = exact_key_running(M, S, m.cnt, m.Q, m.tgt, m.ca, d.w, A, B, gq);
                    Dp = __shfl_sync(0xFFFFFFFFu, Dp, 0);
                    verdict = eligible(Dp, false, c.thr) ? 1 : 0;
                }
                take = verdict == 1;
            }
            if (!take) continue;
            __syncwarp();
            for (int f = lane; f < M * P; f += 32) {
                const int v = m.slot[f], k = v >> 8;
                int i, j;
                swap_entry(S, A, B, v & 0xFF, i, j);
                const int dl = entry_delta(gq[k], A, B, i, j);
                if (dl == 0) continue;
                const int e = k * SS + i * S + j;
                m.cnt[e] += dl;
                m.dn[e] += dl;
                running_coefficient(e, m.dn[e], (float)d.w[k], m.fQ, m.fe0, m.tiny, m.fb, m.beta);
            }
            mark_neighbourhood<KIND, true>(c.g, a, c.ztot, lane, 32, m.vec, m.bitmap);
            mark_neighbourhood<KIND, true>(c.g, b, c.ztot, lane, 32, m.vec, m.bitmap);
            if (lane == 0) {
                store_species<BITS>(m.types, a, B);
                store_species<BITS>(m.types, b, A);
                m.acc[n_acc] = q;
            }
            ++n_acc;
            __syncwarp();
        }
        if (lane == 0) sh.n_acc = n_acc;
    }
    __syncthreads();
}

// ---- multi-accept walk, pairwise form (ranked list of at most d.pair_cap candidates) ----------
// Prepared in parallel: every candidate's nonzero count changes (entry, dN), its sites' positions,
// and the conflict matrix (candidates i < r conflict when a site of one lies in the closed shell
// neighbourhood of a site of the other: the minimum-image squared distance is at most r2 of
// shell M, which for cells of at least two conventional cells per axis is the same relation).
// Warp 0 then walks the list: conflicts are one AND with the accepted set, re-checks read the
// prepared lists, and no site bitmap is needed.
struct PairWalk {
    uint16_t* list;    // [ne][MP]: entry | (dN & 0xFF) << 8
    uint8_t* nlist;    // [ne]
    int16_t* pos;      // [ne][6]: X, Y, Z of a, then of b
    uint32_t* conf;    // [ne][nw]
    uint32_t* site;    // [ne][2]: a, b
    uint8_t* spec;     // [ne][2]: species of a and of b
    int8_t* dense;     // [32][Ep]: count changes of the batch's candidates (row stride Ep = E rounded up to 4)
    float* X;          // [32][32]: cross terms sum_e a_e dN_i dN_j of the batch (i < j)
    float* Xe;         // [32][32]: their bounds
    float* bD;         // [32]: re-check estimates at the start of the batch
    float* bE;         // [32]: their bounds
    uint32_t* bPrior;  // [32]: 1 when a swap accepted in an earlier batch conflicts
    uint32_t* bMask;   // [32]: earlier candidates of the same batch it conflicts with
};

__device__ __forceinline__ PairWalk pair_walk_arrays(uint32_t* base, int pair_cap, int M, int S) {
    const uint32_t mp = (uint32_t)(M * (4 * S - 4));
    const uint32_t nw = (uint32_t)((pair_cap + 31) / 32);
    uint8_t* p = reinterpret_cast<uint8_t*>(base);
    PairWalk w;
    w.list = reinterpret_cast<uint16_t*>(p);
    p += align_up((uint32_t)pair_cap * 2 * mp, 16);
    w.nlist = p;
    p += align_up((uint32_t)pair_cap, 16);
    w.pos = reinterpret_cast<int16_t*>(p);
    p += align_up((uint32_t)pair_cap * 12, 16);
    w.conf = reinterpret_cast<uint32_t*>(p);
    p += align_up((uint32_t)pair_cap * 4 * nw, 16);
    w.site = reinterpret_cast<uint32_t*>(p);
    w.spec = p + (size_t)pair_cap * 8;
    p += align_up((uint32_t)pair_cap * 10, 16);
    w.dense = reinterpret_cast<int8_t*>(p);
    p += align_up(32u * (((uint32_t)(M * S * S) + 3u) & ~3u), 16);
    w.X = reinterpret_cast<float*>(p);
    w.Xe = w.X + 32 * 32;
    w.bD = w.Xe + 32 * 32;
    w.bE = w.bD + 32;
    w.bPrior = reinterpret_cast<uint32_t*>(w.bE + 32);
    w.bMask = w.bPrior + 32;
    return w;
}

// Exact key against the running counts when some accepted swaps of the current batch are not yet
// applied: count of entry e = cnt[e] + sum of the pending candidates' changes (dense rows).
static __device__ double exact_key_pending(int M, int S, const int32_t* cnt, const double* Q, const double* tgt,
                                           const double* ca, const double* w, int A, int B, const uint64_t* gb,
                                           const int8_t* dense, int E, const int* pend, int npend) {
    double D = 0.0;
    for (int k = 0; k < M; ++k) {
        const uint64_t g_k = gb[k];
        for (int i = 0; i < S; ++i) {
            const bool row = (i == A || i == B);
            for (int j = 0; j < S; ++j) {
                if (!row && j != A && j != B) continue;
                const int dl = entry_delta(g_k, A, B, i, j);
                if (dl == 0) continue;
                const int e = (k * S + i) * S + j;
                int n = cnt[e];
                for (int p = 0; p < npend; ++p) n += dense[pend[p] * E + e];
                const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)n, Q[e])), tgt[e]);
                const double b = __dmul_rn(-2.0, __dmul_rn(w[k], __dmul_rn(Q[e], err)));
                const double x = (double)dl;
                D = __fma_rn(x, __fma_rn(ca[e], x, b), D);
            }
        }
    }
    return D;
}

// Replaces the species of site i; safe against other threads writing other sites of the same word.
template <int BITS>
__device__ __forceinline__ void store_species_atomic(uint8_t* s, uint32_t i, int v) {
    if (BITS == 8) {
        s[i] = (uint8_t)v;
    } else {
        using P = Packing<BITS>;
        const uint32_t byte = i >> P::lg;
        uint32_t* word = reinterpret_cast<uint32_t*>(s + (byte & ~3u));
        const uint32_t sh = (byte & 3u) * 8 + (i & (P::per - 1u)) * BITS;
        atomicAnd(word, ~(P::mask << sh));
        atomicOr(word, (uint32_t)v << sh);
    }
}

__device__ __forceinline__ int wrap_min_image(int dx, int period) {
    // dx in (-period, period) -> representative with |dx| <= period / 2
    if (dx > period / 2) dx -= period;
    if (dx < -(period / 2)) dx += period;
    return dx;
}

template <int KIND, int BITS>
__device__ void walk_pairs(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c, int ne) {
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
    const int S = c.S, M = c.M, SS = S * S, P = 4 * S - 4, MP = M * P;
    const int nw = (ne + 31) / 32;
    PairWalk w = pair_walk_arrays(m.bitmap, d.pair_cap, M, S);
    // 1. Per candidate: its list of nonzero count changes and its sites' positions.
    for (int r = tid; r < ne; r += T) {
        const uint32_t q = m.order[r];
        const uint32_t a = m.qa[q], b = m.qb[q];
        const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
        int n = 0;
        for (int f = 0; f < MP; ++f) {
            const int v = m.slot[f], k = v >> 8;
            int i, j;
            swap_entry(S, A, B, v & 0xFF, i, j);
            const int dl = entry_delta(m.qg[q * M + k], A, B, i, j);
            if (dl == 0) continue;
            w.list[r * MP + n++] = (uint16_t)((k * SS + i * S + j) | ((dl & 0xFF) << 8));
        }
        w.nlist[r] = (uint8_t)n;
        w.site[2 * r] = a;
        w.site[2 * r + 1] = b;
        w.spec[2 * r] = (uint8_t)A;
        w.spec[2 * r + 1] = (uint8_t)B;
        int X, Y, Z;
        site_coords<KIND>(c.g, a, X, Y, Z);
        w.pos[r * 6 + 0] = (int16_t)X;
        w.pos[r * 6 + 1] = (int16_t)Y;
        w.pos[r * 6 + 2] = (int16_t)Z;
        site_coords<KIND>(c.g, b, X, Y, Z);
        w.pos[r * 6 + 3] = (int16_t)X;
        w.pos[r * 6 + 4] = (int16_t)Y;
        w.pos[r * 6 + 5] = (int16_t)Z;
    }
    __syncthreads();
    // 2. Conflict matrix rows: bit i of row r (i < r) when candidates i and r conflict.  The 2 ne
    // sites are put in a grid of at most 2048 bins, each at least 4 half units wide (more than any
    // shell radius), kept as linked lists; a site can only conflict with sites of its own and the 26
    // neighbouring bins, which are tested by minimum-image distance.
    const int r2max = c_shells[KIND].radius2[M - 1];
    const int PX = 2 * c.g.Lx, PY = 2 * c.g.Ly, PZ = 2 * c.g.Lz;
    {
        uint32_t* head = reinterpret_cast<uint32_t*>(w.dense);   // the batch scratch, unused until the batches
        uint32_t* next = head + kConflictBins;
        uint32_t* sbin = next + 2 * ne;
        int nbx = max(1, PX / 4), nby = max(1, PY / 4), nbz = max(1, PZ / 4);
        while (nbx * nby * nbz > (int)kConflictBins) {
            if (nbx >= nby && nbx >= nbz) nbx = (nbx + 1) / 2;
            else if (nby >= nbz) nby = (nby + 1) / 2;
            else nbz = (nbz + 1) / 2;
        }
        for (int x = tid; x < nbx * nby * nbz; x += T) head[x] = 0u;
        for (int x = tid; x < ne * nw; x += T) w.conf[x] = 0u;
        __syncthreads();
        for (int s2 = tid; s2 < 2 * ne; s2 += T) {
            const int16_t* P3 = w.pos + (s2 >> 1) * 6 + 3 * (s2 & 1);
            const int bx = P3[0] * nbx / PX, by = P3[1] * nby / PY, bz = P3[2] * nbz / PZ;
            sbin[s2] = (uint32_t)bx | ((uint32_t)by << 11) | ((uint32_t)bz << 22);
            next[s2] = atomicExch(&head[(bz * nby + by) * nbx + bx], (uint32_t)s2 + 1u);
        }
        __syncthreads();
        // One task per (site, layer of 9 neighbouring bins).
        for (int t = tid; t < 2 * ne * 3; t += T) {
            const int s2 = t / 3, lz = t - 3 * s2;
            const int r = s2 >> 1;
            const int16_t* P3 = w.pos + r * 6 + 3 * (s2 & 1);
            const int X = P3[0], Y = P3[1], Z = P3[2];
            const uint32_t bb = sbin[s2];
            int cz = (int)(bb >> 22) + lz - 1;
            cz += (cz < 0) ? nbz : 0;
            cz -= (cz >= nbz) ? nbz : 0;
#pragma unroll
            for (int q9 = 0; q9 < 9; ++q9) {
                int cx = (int)(bb & 2047u) + (q9 % 3) - 1, cy = (int)((bb >> 11) & 2047u) + q9 / 3 - 1;
                cx += (cx < 0) ? nbx : 0;
                cx -= (cx >= nbx) ? nbx : 0;
                cy += (cy < 0) ? nby : 0;
                cy -= (cy >= nby) ? nby : 0;
                for (uint32_t x = head[(cz * nby + cy) * nbx + cx]; x != 0u; x = next[x - 1]) {
                    const int t2 = (int)x - 1, i = t2 >> 1;
                    if (i >= r) continue;
                    const int16_t* Q3 = w.pos + i * 6 + 3 * (t2 & 1);
                    const int dx = wrap_min_image(X - Q3[0], PX);
                    const int dy = wrap_min_image(Y - Q3[1], PY);
                    const int dz = wrap_min_image(Z - Q3[2], PZ);
                    if (dx * dx + dy * dy + dz * dz <= r2max) atomicOr(&w.conf[r * nw + (i >> 5)], 1u << (i & 31));
                }
            }
        }
    }
    for (int x = tid; x < nw; x += T) sh.taken[x] = 0u;
    __syncthreads();
    // 3. The walk, in batches of up to 32 ranked candidates.  For each batch, in parallel: the dense
    // count changes of its candidates, their re-check estimates against the running state at the
    // start of the batch (one warp per candidate), and the cross terms X(i, j) = sum_e a_e dN_i dN_j.
    // Accepting candidate i changes every coefficient b_e by 2 a_e dN_i (exact algebra), so the key
    // of a later candidate j moves by exactly 2 X(i, j): warp 0 then decides the batch in order with
    // scalar corrections, each decision on an interval whose bound covers the estimate, the cross
    // terms and their roundings (the exact binary64 key when it cannot decide).  The accepted swaps
    // are applied to counts, species and FP32 coefficients in parallel at the end of the batch.
    const int E = c.E, Ep = (E + 3) & ~3, warp = tid >> 5, nwarps = T >> 5;
    if (tid == 0) {
        sh.n_acc = 0;
        sh.walk_done = 0;
    }
    __syncthreads();
    for (int r0 = 0; r0 < ne; r0 += 32) {
        if (sh.walk_done) break;
        const int nb = min(32, ne - r0);
        const int acc_before = sh.n_acc;
        // P1: dense count changes of the batch.
        for (int x = tid; x < nb * Ep / 4; x += T) reinterpret_cast<uint32_t*>(w.dense)[x] = 0u;
        __syncthreads();
        for (int x = tid; x < nb * MP; x += T) {
            const int j = x / MP, f = x - j * MP;
            if (f < w.nlist[r0 + j]) {
                const uint32_t v = w.list[(r0 + j) * MP + f];
                w.dense[j * Ep + (int)(v & 0xFFu)] = (int8_t)(v >> 8);
            }
        }
        // P2: re-check estimates at the start of the batch, and each candidate's conflicts with the
        // swaps accepted in earlier batches and with the earlier candidates of this batch.
        for (int j = warp; j < nb; j += nwarps) {
            const int r = r0 + j, cnt = w.nlist[r];
            float acc = 0.f, err = 0.f;
            for (int x = lane; x < cnt; x += 32) {
                const uint32_t v = w.list[r * MP + x];
                const int e = (int)(v & 0xFFu);
                const float xf = (float)(int)(int8_t)(v >> 8), ax = fabsf(xf);
                acc = fmaf(xf, fmaf(m.fa[e], xf, m.fb[e]), acc);
                err = fmaf(ax, fmaf(c.rel * fabsf(m.fa[e]), ax, fmaf(c.rel, fabsf(m.fb[e]), m.beta[e])), err);
            }
            const bool prior = (lane <= (r >> 5)) && ((w.conf[r * nw + lane] & sh.taken[lane]) != 0u);
            const uint32_t any_prior = __ballot_sync(0xFFFFFFFFu, prior);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                err += __shfl_xor_sync(0xFFFFFFFFu, err, o);
            }
            if (lane == 0) {
                w.bD[j] = acc;
                w.bE[j] = fmaf(err, 1.0f + 64.0f * kTwoUlp, kAbsBound);
                w.bPrior[j] = any_prior != 0u ? 1u : 0u;
                w.bMask[j] = w.conf[r * nw + (r0 >> 5)] & ((1u << j) - 1u);
            }
        }
        __syncthreads();
        // P3: cross terms of the batch, X(i, j) = sum_e a_e dN_i dN_j for i < j, from the dense rows
        // four entries at a time, with bounds (E + 4) 2^-23 sum |a dN_i dN_j|.
        for (int x = tid; x < 32 * 32; x += T) {
            const int i = x >> 5, j = x & 31;
            if (i >= j || j >= nb) continue;
            const uint32_t* di = reinterpret_cast<const uint32_t*>(w.dense + i * Ep);
            const uint32_t* dj = reinterpret_cast<const uint32_t*>(w.dense + j * Ep);
            float X = 0.f, mag = 0.f;
            for (int q4 = 0; q4 < Ep / 4; ++q4) {
                const uint32_t u = di[q4], v = dj[q4];
                if (u == 0u || v == 0u) continue;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int p = (int)(int8_t)(u >> (8 * b)) * (int)(int8_t)(v >> (8 * b));
                    if (p == 0) continue;
                    const float fa = m.fa[4 * q4 + b], pf = (float)p;
                    X = fmaf(fa, pf, X);
                    mag = fmaf(fabsf(fa), fabsf(pf), mag);
                }
            }
            w.X[i * 32 + j] = X;
            w.Xe[i * 32 + j] = fmaf(mag, c.rel, kAbsBound);
        }
        __syncthreads();
        // P4: decisions, in order, by warp 0; lane j holds candidate j's estimate, bound and conflict
        // information.  Speculation: every undecided lane evaluates its candidate assuming that all
        // earlier undecided candidates not blocked by earlier batches are accepted; the first lane
        // whose decision contradicts that assumption ends the round: the lanes before it are
        // committed (their assumptions held), it is decided under the committed state, and the next
        // round starts after it.  Rounds = rejections + 1.
        if (warp == 0) {
            float D0 = 0.f, E0 = 0.f;
            uint32_t prior = 1u, mask = 0u;
            if (lane < nb) {
                D0 = w.bD[lane];
                E0 = w.bE[lane];
                prior = w.bPrior[lane];
                mask = w.bMask[lane];
            }
            const uint32_t open = __ballot_sync(0xFFFFFFFFu, lane < nb && prior == 0u);
            float cc = 0.f, ce = 0.f, ca = 0.f;   // corrections from committed accepted candidates
            uint32_t accm = 0u;                  // committed accepted candidates of the batch
            int n_acc = acc_before, nbacc = 0, p = 0;
            bool done = false;
            while (p < nb && !done) {
                const uint32_t below_p = (p >= 32) ? 0xFFFFFFFFu : ((1u << p) - 1u);
                const uint32_t guess = open & ~below_p;
                int dec = 0;
                if (lane >= p && lane < nb) {
                    const uint32_t gl = guess & ((1u << lane) - 1u);
                    float s = cc, e = ce, a = ca;
                    for (uint32_t bits = gl; bits; bits &= bits - 1u) {
                        const int i = __ffs(bits) - 1;
                        const float x = w.X[i * 32 + lane];
                        s += x;
                        e += w.Xe[i * 32 + lane];
                        a += fabsf(x);
                    }
                    const bool blocked = prior != 0u || (mask & (accm | gl)) != 0u;
                    if (!blocked) {
                        if (acc_before == 0 && (accm | gl) == 0u) {
                            dec = 1;   // the step-start state: the candidate is eligible
                        } else {
                            const float v = fmaf(2.0f, s, D0);
                            const float er = fmaf(fmaf(2.0f, e, E0), 1.0f + 2.0f * 64.0f * kTwoUlp,
                                                  fmaf(40.0f * kTwoUlp, fabsf(D0) + 2.0f * a, kAbsBound));
                            dec = eligible_interval(__fadd_rd(v, -er), __fadd_ru(v, er), c.pos_thr, c.thr_lo,
                                                    c.thr_hi);
                        }
                    }
                }
                const uint32_t bad =
                    __ballot_sync(0xFFFFFFFFu, lane >= p && lane < nb && prior == 0u && dec != 1);
                const int js = bad ? (__ffs(bad) - 1) : nb;
                // Commit the accepted candidates of [p, js), at most max_accept in total.
                uint32_t commit = guess & ((js >= 32) ? 0xFFFFFFFFu : ((1u << js) - 1u));
                if (d.max_accept > 0) {
                    const int room = d.max_accept - n_acc;
                    while (__popc(commit) > room) commit &= ~(1u << (31 - __clz(commit)));
                    if (__popc(guess & ((js >= 32) ? 0xFFFFFFFFu : ((1u << js) - 1u))) > room) done = true;
                }
                for (uint32_t bits = commit; bits; bits &= bits - 1u) {
                    const int i = __ffs(bits) - 1;
                    if (lane == 0) sh.red_q[nbacc] = i;
                    if (lane > i && lane < nb) {
                        const float x = w.X[i * 32 + lane];
                        cc += x;
                        ce += w.Xe[i * 32 + lane];
                        ca += fabsf(x);
                    }
                    ++nbacc;
                }
                accm |= commit;
                n_acc += __popc(commit);
                if (done || js >= nb) break;
                if (d.max_accept > 0 && n_acc >= d.max_accept) {
                    done = true;
                    break;
                }
                // Decide candidate js under the committed state.
                int dj = __shfl_sync(0xFFFFFFFFu, dec, js);
                if (dj < 0) {
                    const int r = r0 + js;
                    double Dp = 0.0;
                    if (lane == 0) {
                        const uint32_t q = m.order[r];
                        Dp = exact_key_pending(M, S, m.cnt, m.Q, m.tgt, m.ca, d.w, w.spec[2 * r], w.spec[2 * r + 1],
                                               m.qg + q * M, w.dense, Ep, sh.red_q, nbacc);
                    }
                    Dp = __shfl_sync(0xFFFFFFFFu, Dp, 0);
                    dj = eligible(Dp, false, c.thr) ? 1 : 0;
                }
                if (dj == 1) {
                    if (lane == 0) sh.red_q[nbacc] = js;
                    if (lane > js && lane < nb) {
                        const float x = w.X[js * 32 + lane];
                        cc += x;
                        ce += w.Xe[js * 32 + lane];
                        ca += fabsf(x);
                    }
                    ++nbacc;
                    ++n_acc;
                    accm |= 1u << js;
                    if (d.max_accept > 0 && n_acc >= d.max_accept) done = true;
                }
                p = js + 1;
            }
            if (lane == 0) {
                sh.batch_n = nbacc;
                sh.n_acc = n_acc;
                if (done) sh.walk_done = 1;
            }
        }
        __syncthreads();
        // P5: apply the batch's accepted swaps.
        const int nba = sh.batch_n;
        for (int x = tid; x < nba * MP; x += T) {
            const int r = r0 + sh.red_q[x / MP], f = x % MP;
            if (f >= w.nlist[r]) continue;
            const uint32_t v = w.list[r * MP + f];
            const int e = (int)(v & 0xFFu), dl = (int)(int8_t)(v >> 8);
            atomicAdd(&m.cnt[e], dl);
            atomicAdd(&m.dn[e], dl);
        }
        for (int x = tid; x < nba; x += T) {
            const int r = r0 + sh.red_q[x];
            store_species_atomic<BITS>(m.types, w.site[2 * r], w.spec[2 * r + 1]);
            store_species_atomic<BITS>(m.types, w.site[2 * r + 1], w.spec[2 * r]);
            m.acc[acc_before + x] = m.order[r];
            atomicOr(&sh.taken[r >> 5], 1u << (r & 31));
        }
        __syncthreads();
        // P6: running FP32 coefficients of every entry (an entry whose change returned to 0 needs
        // its coefficient back too).
        if (nba > 0)
            for (int e = tid; e < E; e += T) running_coefficient(e, m.dn[e], m.fw[e], m.fQ, m.fe0, m.tiny, m.fb, m.beta);
        __syncthreads();
    }
}

// Multi-accept walk over the ranked list m.order[0, ne).
template <int KIND, int BITS>
__device__ void walk(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c, int ne) {
    if (ne <= d.pair_cap)
        walk_pairs<KIND, BITS>(d, m, sh, c, ne);
    else
        walk_bitmap<KIND, BITS>(d, m, sh, c, ne);
}

// After a walk: refresh the binary64 coefficients (and their FP32 roundings used by the next
// step's estimates) from the updated counts.
template <int KIND>
__device__ void after_walk(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c) {
    const int na = sh.n_acc;
    if (na > 0) {
        const int S = c.S;
        for (int e = threadIdx.x; e < c.E; e += blockDim.x) {
            const int k = e / (S * S);
            const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)m.cnt[e], m.Q[e])), m.tgt[e]);
            const double b = __dmul_rn(-2.0, __dmul_rn(d.w[k], __dmul_rn(m.Q[e], err)));
            m.cb[e] = b;
            m.fb[e] = (float)b;
            m.fe0[e] = (float)err;
            m.dn[e] = 0;
            m.beta[e] = fmaf(kTwoUlp, fabsf(m.fb[e]), m.tiny[e]);
        }
    }
    __syncthreads();
}

// Depth counter, step budget, depth limit, time budget (Sec. 4.6.4).
__device__ __forceinline__ void bookkeeping(const ChainDesc& d, ChainShared& sh, bool timed_out) {
    if (threadIdx.x == 0) {
        const int na = sh.n_acc;
        sh.accepted += na;
        sh.depth = (na > 0) ? 0 : sh.depth + 1;
        sh.steps += 1;
        bool stop = sh.steps >= d.max_steps;
        if (d.depth_limit > 0 && sh.depth >= d.depth_limit) stop = true;
        if (timed_out) {
            if (!stop) sh.status = HEA_ETIMEOUT;
            stop = true;
        }
        sh.stop = stop ? 1 : 0;
    }
    __syncthreads();
}

template <int BITS>
__device__ void write_back(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c) {
    const uint32_t N = c.N;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) d.types[i] = (uint8_t)load_species<BITS>(m.types, i);
    for (int e = threadIdx.x; e < c.E; e += blockDim.x) d.counts[e] = m.cnt[e];
    if (threadIdx.x == 0) {
        const int S = c.S;
        double f2 = 0.0;
        for (int e = 0; e < c.E; ++e) {
            const int k = e / (S * S);
            const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)m.cnt[e], m.Q[e])), m.tgt[e]);
            f2 = __dadd_rn(f2, __dmul_rn(d.w[k], __dmul_rn(err, err)));
        }
        d.result->steps = sh.steps;
        d.result->trials = sh.steps * (int64_t)c.K;
        d.result->accepted = sh.accepted;
        d.result->depth = sh.depth;
        d.result->status = sh.status;
        d.result->f2 = f2;
        d.result->f = __dsqrt_rn(f2);
    }
}

__device__ __forceinline__ void report_invalid(const ChainDesc& d) {
    if (threadIdx.x == 0) {
        d.result->steps = 0;
        d.result->trials = 0;
        d.result->accepted = 0;
        d.result->depth = d.depth0;
        d.result->status = HEA_EINVAL;
        d.result->f2 = CUDART_NAN;
        d.result->f = CUDART_NAN;
    }
}

// ------------------------------------------------------------------------------------------------
// One chain, run to completion by the calling CTA.
// ------------------------------------------------------------------------------------------------
template <int KIND, int BITS>
__device__ void run_chain(const ChainDesc& d, uint8_t* smem, ChainShared& sh) {
    const ChainLayout L = chain_layout(d.N, d.M, d.S, d.qcap, BITS, d.accept_mode, d.pair_cap);
    ChainSmem m(smem, L);
    ChainCtx c;
    chain_setup<KIND, BITS>(d, m, sh, c);
    if (sh.bad) {
        report_invalid(d);
        return;
    }
    while (!sh.stop) {
        const uint32_t step = d.step0 + (uint32_t)sh.steps;
        if (threadIdx.x == 0) {
            sh.qn = 0;
            sh.n_acc = 0;
            sh.win_q = -1;
        }
        __syncthreads();
        const float my_umin = score_range<KIND, BITS>(d, m, sh, c, step, 0u, (uint32_t)c.K);
        if (d.accept_mode == 0) {
            const float umin = block_min(my_umin, sh);
            best_of_queue<BITS>(m, sh, c, umin, false);
            const int q = sh.win_q;
            if (q >= 0) {
                const uint32_t a = m.qa[q], b = m.qb[q];
                const bool null_move = (a == b) || load_species<BITS>(m.types, a) == load_species<BITS>(m.types, b);
                const bool ok = sh.win_elig >= 0 ? (sh.win_elig == 1 && !null_move) : eligible(m.qD[q], null_move, c.thr);
                if (ok) apply_slot<BITS>(d, m, sh, c, q);
            }
        } else {
            __syncthreads();
            rank_eligible<BITS>(m, sh, c, sh.qn, d.group_size, d.group_top,
                                d.group_top == 0 || d.group_size == 0 || d.group_size >= c.K);
            walk<KIND, BITS>(d, m, sh, c, sh.n_elig);
            after_walk<KIND>(d, m, sh, c);
        }
        __syncthreads();
        const bool timed_out = d.timeout_ns > 0 && (int64_t)(globaltimer_ns() - sh.t0) >= d.timeout_ns;
        bookkeeping(d, sh, timed_out);
    }
    write_back<BITS>(d, m, sh, c);
}

}  // namespace hea
