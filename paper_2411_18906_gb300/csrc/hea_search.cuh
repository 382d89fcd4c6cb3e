// hea_search.cuh -- swap scoring (Sec. 4.5, Sec. 4.6.2) and the persistent parallel Monte Carlo
// search (Alg. parallel_mc; Sec. 4.6.3 selection; Sec. 4.6.4 convergence) for sm_103a.
//
// One CTA runs one chain.  The cell's species live in shared memory (8 or 4 bits per site), the
// counts and the per-entry objective coefficients next to them.  A step:
//   1. every thread draws candidates (Philox), builds the per-shell neighbour histograms of both
//      sites (neighbours computed from coordinates), and evaluates an FP32 estimate of the swap
//      key with a rigorous error bound;
//   2. only candidates whose bound admits acceptance get the exact FP64 key (the same FMA chain
//      as the reference definition), so every decision is taken on the exact key;
//   3. best-of-K: block argmin over (D, k); multi-accept: eligible candidates are ranked by (D, k)
//      and walked by one warp with a neighbourhood bitmap and an exact re-check against the
//      running counts;
//   4. the accepted swap(s) update species, counts and coefficients in place.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "hea_device.cuh"
#include "hea_internal.h"

namespace hea {

static __constant__ ShellTable c_shells[2] = {build_shell_table(kFCC), build_shell_table(kBCC)};

// Error factor of the FP32 key estimate (see the bound in score_float) and its absolute floor.
constexpr float kRelBound = 1.220703125e-4f;   // 2^-13
constexpr float kAbsBound = 7.52316385e-37f;   // 2^-120

struct ChainShared {
    int qn;          // queue length (candidates that need the exact key)
    int n_elig;      // multi-accept: eligible candidates
    int n_acc;       // swaps accepted this step
    int stop;
    int bad;
    int use_filter;
    int depth;
    int status;
    float umin;      // best-of-K: min over candidates of the upper bound on D
    int win_q;       // best-of-K: queue slot of the winner (-1 none)
    double win_D;
    int64_t steps;
    int64_t accepted;
    uint64_t t0;
    float red_f[32];
    double red_d[32];
    uint32_t red_k[32];
    int red_q[32];
};

// Delta of entry (k,i,j) for a swap of species A (site a) and B (site b) with per-shell
// histograms ha, hb (Sec. 4.5): g = h_b - h_a,
//   dN_ij = [i==A] g_j - [i==B] g_j + [j==A] g_i - [j==B] g_i.
__device__ __forceinline__ int entry_delta(uint64_t ha, uint64_t hb, int A, int B, int i, int j) {
    int d = 0;
    if (i == A || i == B) {
        const int gj = hist_field(hb, j) - hist_field(ha, j);
        d += (i == A) ? gj : -gj;
    }
    if (j == A || j == B) {
        const int gi = hist_field(hb, i) - hist_field(ha, i);
        d += (j == A) ? gi : -gi;
    }
    return d;
}

// Exact key: change of F^2, D <- fma(dN, fma(a, dN, b), D) over (k,i,j) row-major; entries with
// dN = 0 leave D unchanged bit for bit and are skipped.
static __device__ double exact_key(int M, int S, const double* __restrict__ ca, const double* __restrict__ cb, int A,
                            int B, const uint64_t* ha, const uint64_t* hb) {
    double D = 0.0;
    for (int k = 0; k < M; ++k) {
        const uint64_t a_h = ha[k], b_h = hb[k];
        for (int i = 0; i < S; ++i) {
            const bool row = (i == A || i == B);
            for (int j = 0; j < S; ++j) {
                if (!row && j != A && j != B) continue;
                const int d = entry_delta(a_h, b_h, A, B, i, j);
                if (d == 0) continue;
                const int e = (k * S + i) * S + j;
                const double x = (double)d;
                D = __fma_rn(x, __fma_rn(ca[e], x, cb[e]), D);
            }
        }
    }
    return D;
}

// FP32 estimate of the key and a bound on its distance to the exact FP64 key.  Both evaluate
// sum_e d_e (a_e d_e + b_e) from the same binary64 coefficients; the FP32 one from their float
// roundings.  With n <= 320 nonzero entries the float evaluation is within
// (n + 2) 2^-24 sum |d| (|a| |d| + |b|) (+ subnormal floor) of the real value and the FP64 chain
// within (n + 1) 2^-53 of the same sum, so |D32 - D64| < 2^-13 sum |d|(|a||d| + |b|) + 2^-120.
__device__ __forceinline__ void score_float(int M, int S, const float* __restrict__ fa, const float* __restrict__ fb,
                                            int A, int B, const uint64_t* ha, const uint64_t* hb, float& D,
                                            float& err) {
    float acc = 0.f, mag = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxShells; ++k) {
        if (k >= M) break;
        const uint64_t a_h = ha[k], b_h = hb[k];
        const int base = k * S * S;
        const int gA = hist_field(b_h, A) - hist_field(a_h, A);
        const int gB = hist_field(b_h, B) - hist_field(a_h, B);
        for (int y = 0; y < S; ++y) {
            const int gy = hist_field(b_h, y) - hist_field(a_h, y);
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
    err = fmaf(mag, kRelBound, kAbsBound);
}

__device__ __forceinline__ bool eligible(double D, bool null_move, double threshold) {
    if (null_move) return false;
    if (D < 0.0) return true;
    return threshold > 0.0 && D <= threshold;
}

// Updates entry e after its count changed by d: e = (1 - n Q) - t; b = -2 (w (Q e)).
__device__ __forceinline__ void refresh_entry(int e, int d, double w, int32_t* cnt, const double* Q,
                                              const double* tgt, double* cb, float* fb) {
    const int n = cnt[e] + d;
    cnt[e] = n;
    if (d == 0) return;
    const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)n, Q[e])), tgt[e]);
    const double b = __dmul_rn(-2.0, __dmul_rn(w, __dmul_rn(Q[e], err)));
    cb[e] = b;
    fb[e] = (float)b;
}

// Site index of site + shell vector v (runtime v), for the bitmap of the multi-accept walk.
template <int KIND>
__device__ __forceinline__ uint32_t neighbour_of(const Geo& g, uint32_t site, int v) {
    int X, Y, Z;
    site_coords<KIND>(g, site, X, Y, Z);
    const ShellTable& T = c_shells[KIND];
    int x = X + T.v[v][0], y = Y + T.v[v][1], z = Z + T.v[v][2];
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

__device__ __forceinline__ bool better(double D1, uint32_t k1, double D2, uint32_t k2) {
    return D1 < D2 || (D1 == D2 && k1 < k2);
}

// ------------------------------------------------------------------------------------------------
// One chain, run to completion by the calling CTA.
// ------------------------------------------------------------------------------------------------
template <int KIND, int BITS>
__device__ void run_chain(const ChainDesc& d, uint8_t* smem, ChainShared& sh) {
    constexpr int MX = kMaxShells;
    const int M = d.M, S = d.S, E = M * S * S, K = d.K;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
    const ChainLayout L = chain_layout(d.N, M, S, K, BITS, d.accept_mode);
    uint8_t* s_types = smem + L.types;
    int32_t* s_cnt = reinterpret_cast<int32_t*>(smem + L.cnt);
    double* s_Q = reinterpret_cast<double*>(smem + L.Q);
    double* s_t = reinterpret_cast<double*>(smem + L.tgt);
    double* s_ca = reinterpret_cast<double*>(smem + L.ca);
    double* s_cb = reinterpret_cast<double*>(smem + L.cb);
    float* s_fa = reinterpret_cast<float*>(smem + L.fa);
    float* s_fb = reinterpret_cast<float*>(smem + L.fb);
    uint32_t* s_qk = reinterpret_cast<uint32_t*>(smem + L.qk);
    uint32_t* s_qa = reinterpret_cast<uint32_t*>(smem + L.qa);
    uint32_t* s_qb = reinterpret_cast<uint32_t*>(smem + L.qb);
    float* s_qlo = reinterpret_cast<float*>(smem + L.qlo);
    double* s_qD = reinterpret_cast<double*>(smem + L.qD);
    uint64_t* s_qha = reinterpret_cast<uint64_t*>(smem + L.qha);
    uint64_t* s_qhb = reinterpret_cast<uint64_t*>(smem + L.qhb);
    uint32_t* s_order = reinterpret_cast<uint32_t*>(smem + L.order);
    uint32_t* s_acc = reinterpret_cast<uint32_t*>(smem + L.acc);
    uint32_t* s_bitmap = reinterpret_cast<uint32_t*>(smem + L.bitmap);

    Geo g;
    g.Lx = d.Lx;
    g.Ly = d.Ly;
    g.Lz = d.Lz;
    g.V = d.Lx * d.Ly * d.Lz;
    g.LxLy = d.Lx * d.Ly;
    g.N = d.N;
    const uint32_t N = (uint32_t)d.N;
    const double thr = d.threshold;
    const uint32_t seed_lo = (uint32_t)(d.seed & 0xFFFFFFFFu), seed_hi = (uint32_t)(d.seed >> 32);
    const ShellTable& TAB = c_shells[KIND];
    const int ztot = TAB.first[M];

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

    // ---- load species (validated against S) and counts; objective coefficients ----
    if (BITS == 8) {
        for (uint32_t i = tid; i < N; i += T) {
            const uint8_t v = d.types[i];
            if (v >= S) sh.bad = 1;
            s_types[i] = v;
        }
    } else {
        for (uint32_t i = tid; i < (N + 1) / 2; i += T) {
            const uint8_t v0 = d.types[2 * i];
            const uint8_t v1 = (2 * i + 1 < N) ? d.types[2 * i + 1] : 0;
            if (v0 >= S || v1 >= S) sh.bad = 1;
            s_types[i] = (uint8_t)((v0 & 0xF) | ((v1 & 0xF) << 4));
        }
    }
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
        s_cnt[e] = n;
        s_Q[e] = Q;
        s_t[e] = t;
        s_ca[e] = a;
        s_cb[e] = b;
        s_fa[e] = (float)a;
        s_fb[e] = (float)b;
        // The FP32 estimate needs every |a| dN^2 and |b| dN to stay far inside the float range;
        // |e| <= 1 + N / N_j + |t| bounds b over the whole search.
        const double zz = 2.0 * TAB.z[k];
        const double bmax = 2.0 * w * Q * (1.0 + (double)d.N / (double)d.n_per[j] + fabs(t));
        if (!(a * zz * zz < 1e30) || !(bmax * zz < 1e30)) sh.use_filter = 0;
    }
    if (d.accept_mode == 1)
        for (uint32_t i = tid; i < (N + 31) / 32; i += T) s_bitmap[i] = 0;
    __syncthreads();
    if (sh.bad) {
        if (tid == 0) {
            d.result->steps = 0;
            d.result->trials = 0;
            d.result->accepted = 0;
            d.result->depth = d.depth0;
            d.result->status = HEA_EINVAL;
            d.result->f2 = CUDART_NAN;
            d.result->f = CUDART_NAN;
        }
        return;
    }
    const bool use_filter = sh.use_filter != 0;

    auto onehot = [&](uint32_t n) -> uint64_t { return 1ull << (8 * load_species<BITS>(s_types, n)); };

    // ---- step loop ----
    while (!sh.stop) {
        const uint32_t step = d.step0 + (uint32_t)sh.steps;
        if (tid == 0) {
            sh.qn = 0;
            sh.n_elig = 0;
            sh.n_acc = 0;
            sh.win_q = -1;
        }
        __syncthreads();

        // 1. Score every candidate with the FP32 estimate; queue those that may be accepted.
        float my_umin = CUDART_INF_F;
        for (int kk = tid; kk < K; kk += T) {
            const Rand4 r = philox((uint32_t)kk, step, d.chain, 1u, seed_lo, seed_hi);
            const uint32_t a = __umulhi(r.r0, N), b = __umulhi(r.r1, N);
            const int A = load_species<BITS>(s_types, a), B = load_species<BITS>(s_types, b);
            if (a == b || A == B) {
                my_umin = fminf(my_umin, 0.f);
                if (thr > 0.0) {
                    const int slot = atomicAdd(&sh.qn, 1);
                    s_qk[slot] = (uint32_t)kk;
                    s_qa[slot] = a;
                    s_qb[slot] = b;
                    s_qlo[slot] = 0.f;
                }
                continue;
            }
            uint64_t ha[MX], hb[MX];
            neighbour_histogram_upto<KIND, MX>(g, a, b, onehot, ha, M);
            neighbour_histogram_upto<KIND, MX>(g, b, a, onehot, hb, M);
            float lo = -CUDART_INF_F;
            if (use_filter) {
                float Dt, err;
                score_float(M, S, s_fa, s_fb, A, B, ha, hb, Dt, err);
                my_umin = fminf(my_umin, __fadd_ru(Dt, err));
                lo = __fadd_rd(Dt, -err);
                if ((double)lo > thr) continue;
            }
            const int slot = atomicAdd(&sh.qn, 1);
            s_qk[slot] = (uint32_t)kk;
            s_qa[slot] = a;
            s_qb[slot] = b;
            s_qlo[slot] = lo;
#pragma unroll
            for (int k = 0; k < MX; ++k) {
                if (k < M) {
                    s_qha[slot * M + k] = ha[k];
                    s_qhb[slot * M + k] = hb[k];
                }
            }
        }

        if (d.accept_mode == 0) {
            // 2a. Block minimum of the upper bounds.
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) my_umin = fminf(my_umin, __shfl_xor_sync(0xFFFFFFFFu, my_umin, o));
            if (lane == 0) sh.red_f[warp] = my_umin;
            __syncthreads();
            if (tid == 0) {
                float u = CUDART_INF_F;
                for (int w = 0; w < nwarps; ++w) u = fminf(u, sh.red_f[w]);
                sh.umin = u;
            }
            __syncthreads();
            // 3a. Exact keys for candidates that can still be the accepted argmin.
            const double tau = use_filter ? fmin((double)sh.umin, thr) : CUDART_INF;
            double bD = CUDART_INF;
            uint32_t bk = 0xFFFFFFFFu;
            int bq = -1;
            const int qn = sh.qn;
            for (int q = tid; q < qn; q += T) {
                if (use_filter && (double)s_qlo[q] > tau) continue;
                const uint32_t a = s_qa[q], b = s_qb[q];
                const int A = load_species<BITS>(s_types, a), B = load_species<BITS>(s_types, b);
                const double D = (a == b || A == B) ? 0.0 : exact_key(M, S, s_ca, s_cb, A, B, s_qha + q * M, s_qhb + q * M);
                if (better(D, s_qk[q], bD, bk)) {
                    bD = D;
                    bk = s_qk[q];
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
            if (tid == 0) {
                double D = CUDART_INF;
                uint32_t k = 0xFFFFFFFFu;
                int q = -1;
                for (int w = 0; w < nwarps; ++w)
                    if (better(sh.red_d[w], sh.red_k[w], D, k)) {
                        D = sh.red_d[w];
                        k = sh.red_k[w];
                        q = sh.red_q[w];
                    }
                bool take = false;
                if (q >= 0) {
                    const uint32_t a = s_qa[q], b = s_qb[q];
                    const bool null_move = (a == b) || load_species<BITS>(s_types, a) == load_species<BITS>(s_types, b);
                    take = eligible(D, null_move, thr);
                }
                sh.win_q = take ? q : -1;
                sh.win_D = D;
            }
            __syncthreads();
            // 4a. Apply the winner.
            const int q = sh.win_q;
            if (q >= 0) {
                const uint32_t a = s_qa[q], b = s_qb[q];
                const int A = load_species<BITS>(s_types, a), B = load_species<BITS>(s_types, b);
                for (int e = tid; e < E; e += T) {
                    const int k = e / (S * S), i = (e / S) % S, j = e % S;
                    const int dl = entry_delta(s_qha[q * M + k], s_qhb[q * M + k], A, B, i, j);
                    refresh_entry(e, dl, d.w[k], s_cnt, s_Q, s_t, s_cb, s_fb);
                }
                __syncthreads();
                if (tid == 0) {
                    store_species<BITS>(s_types, a, B);
                    store_species<BITS>(s_types, b, A);
                    sh.n_acc = 1;
                }
            }
        } else {
            __syncthreads();
            // 2b. Exact keys of all queued candidates; collect the eligible ones.
            const int qn = sh.qn;
            for (int q = tid; q < qn; q += T) {
                const uint32_t a = s_qa[q], b = s_qb[q];
                const int A = load_species<BITS>(s_types, a), B = load_species<BITS>(s_types, b);
                const bool null_move = (a == b || A == B);
                const double D = null_move ? 0.0 : exact_key(M, S, s_ca, s_cb, A, B, s_qha + q * M, s_qhb + q * M);
                s_qD[q] = D;
                if (eligible(D, null_move, thr)) {
                    const int slot = atomicAdd(&sh.n_elig, 1);
                    s_acc[slot] = (uint32_t)q;
                }
            }
            __syncthreads();
            // 3b. Rank the eligible candidates by (D, k).
            const int ne = sh.n_elig;
            for (int s = tid; s < ne; s += T) {
                const uint32_t q = s_acc[s];
                const double D = s_qD[q];
                const uint32_t k = s_qk[q];
                int rank = 0;
                for (int o = 0; o < ne; ++o) {
                    const uint32_t q2 = s_acc[o];
                    rank += better(s_qD[q2], s_qk[q2], D, k) ? 1 : 0;
                }
                s_order[rank] = q;
            }
            __syncthreads();
            // 4b. One warp walks the ranked list (sequential by definition).
            if (warp == 0) {
                int n_acc = 0;
                for (int r = 0; r < ne; ++r) {
                    if (d.max_accept > 0 && n_acc >= d.max_accept) break;
                    const uint32_t q = s_order[r];
                    const uint32_t a = s_qa[q], b = s_qb[q];
                    const bool blocked = ((s_bitmap[a >> 5] >> (a & 31)) & 1u) | ((s_bitmap[b >> 5] >> (b & 31)) & 1u);
                    if (blocked) continue;
                    const int A = load_species<BITS>(s_types, a), B = load_species<BITS>(s_types, b);
                    double Dp = 0.0;
                    if (lane == 0)
                        Dp = (r == 0) ? s_qD[q] : exact_key(M, S, s_ca, s_cb, A, B, s_qha + q * M, s_qhb + q * M);
                    Dp = __shfl_sync(0xFFFFFFFFu, Dp, 0);
                    if (!eligible(Dp, false, thr)) continue;
                    for (int e = lane; e < E; e += 32) {
                        const int k = e / (S * S), i = (e / S) % S, j = e % S;
                        const int dl = entry_delta(s_qha[q * M + k], s_qhb[q * M + k], A, B, i, j);
                        refresh_entry(e, dl, d.w[k], s_cnt, s_Q, s_t, s_cb, s_fb);
                    }
                    for (int v = lane; v < 2 * (ztot + 1); v += 32) {
                        const uint32_t c = (v <= ztot) ? a : b;
                        const int vv = (v <= ztot) ? v : v - (ztot + 1);
                        const uint32_t site = (vv == 0) ? c : neighbour_of<KIND>(g, c, vv - 1);
                        atomicOr(&s_bitmap[site >> 5], 1u << (site & 31));
                    }
                    if (lane == 0) {
                        store_species<BITS>(s_types, a, B);
                        store_species<BITS>(s_types, b, A);
                        s_acc[n_acc] = q;
                    }
                    ++n_acc;
                    __syncwarp();
                }
                if (lane == 0) sh.n_acc = n_acc;
            }
            __syncthreads();
            // 5b. Clear the bitmap around the swapped sites.
            const int na = sh.n_acc;
            const int per = 2 * (ztot + 1);
            for (int x = tid; x < na * per; x += T) {
                const uint32_t q = s_acc[x / per];
                const int v = x % per;
                const uint32_t c = (v <= ztot) ? s_qa[q] : s_qb[q];
                const int vv = (v <= ztot) ? v : v - (ztot + 1);
                const uint32_t site = (vv == 0) ? c : neighbour_of<KIND>(g, c, vv - 1);
                atomicAnd(&s_bitmap[site >> 5], ~(1u << (site & 31)));
            }
        }
        __syncthreads();
        // Bookkeeping: depth counter, step budget, depth limit, time budget (Sec. 4.6.4).
        if (tid == 0) {
            const int na = sh.n_acc;
            sh.accepted += na;
            sh.depth = (na > 0) ? 0 : sh.depth + 1;
            sh.steps += 1;
            bool stop = sh.steps >= d.max_steps;
            if (d.depth_limit > 0 && sh.depth >= d.depth_limit) stop = true;
            if (d.timeout_ns > 0 && (int64_t)(globaltimer_ns() - sh.t0) >= d.timeout_ns) {
                if (!stop) sh.status = HEA_ETIMEOUT;
                stop = true;
            }
            sh.stop = stop ? 1 : 0;
        }
        __syncthreads();
    }

    // ---- write back ----
    if (BITS == 8) {
        for (uint32_t i = tid; i < N; i += T) d.types[i] = s_types[i];
    } else {
        for (uint32_t i = tid; i < N; i += T) d.types[i] = (uint8_t)load_species<4>(s_types, i);
    }
    for (int e = tid; e < E; e += T) d.counts[e] = s_cnt[e];
    if (tid == 0) {
        double f2 = 0.0;
        for (int e = 0; e < E; ++e) {
            const int k = e / (S * S);
            const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)s_cnt[e], s_Q[e])), s_t[e]);
            f2 = __dadd_rn(f2, __dmul_rn(d.w[k], __dmul_rn(err, err)));
        }
        d.result->steps = sh.steps;
        d.result->trials = sh.steps * (int64_t)K;
        d.result->accepted = sh.accepted;
        d.result->depth = sh.depth;
        d.result->status = sh.status;
        d.result->f2 = f2;
        d.result->f = __dsqrt_rn(f2);
    }
}


}  // namespace hea
