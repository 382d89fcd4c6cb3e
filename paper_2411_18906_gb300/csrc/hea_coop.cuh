// hea_coop.cuh -- one search chain run by a grid of co-resident CTAs (Alg. parallel_mc; Sec. 4.6.2
// scoring, Sec. 4.6.3 selection, Sec. 4.6.4 depth counter), with the non-overlapping multi-accept
// step, for sm_103a.
//
// A step of CTA r (one CTA per SM, each with its own copy of the cell in shared memory):
//   1. score candidates [r Kc, (r + 1) Kc) (FP32 screen with rigorous bounds, score_range);
//   2. multi-accept: select its `top` best eligible candidates by (D, k); best-of-K: its argmin on
//      binary64 keys;
//   3. publish them as records in the exchange area, then its tag word (release);
//   4. read every CTA's tag (acquire, bounded wait) and records;
//   5. best-of-K: global argmin; multi-accept: rank all records by (D, k) and walk them in rank
//      order, 32 at a time, with cross terms; apply the accepted swaps.
// Every CTA runs step 5 on the same records, so all copies of the cell stay identical without a
// second exchange.  Only CTA 0 decides the time budget; its decision travels in its tag, so every
// CTA stops after the same step.
//
// Decisions and orders are those of the binary64 keys (the reference definition), taken in three
// tiers: the FP32 interval of each key (score_range's bound) settles almost all of them; where it
// cannot, an exact fixed-point evaluation with a bound of about 2^-30 of the key's terms does; the
// rest (exact ties between different swaps, keys within that bound of zero) use binary64 keys.
//
// Fixed-point keys.  A swap's key is D = sum_e dN_e (a_e dN_e + b_e) over the entries e = (k,i,j)
// it changes (Sec. 4.5: only pairs that touch the two swapped sites change).  With integer copies
// A_e = round(a_e 2^Fa) and B_e = round(b_e 2^F) of the binary64 coefficients (F <= Fa, every |A_e|
// < 2^32 and |B_e| < 2^38) the integer fix = sum B_e dN_e + floor(sum A_e dN_e^2 / 2^(Fa - F)) is
// exact arithmetic, within
//     R = floor(sum dN^2 / 2^(Fa - F + 1)) + 2 + ceil(sum |dN| / 2)
// of 2^F times the real-arithmetic key of the binary64 coefficients; the reference key (binary64
// FMA chain over at most 140 nonzero terms) is within (n + 2) 2^-53 sum |dN| (|a| |dN| + |b|) <=
// 2^-45 Mag of that, Mag being the same magnitude in fixed point with a unit of slack per term.  So
// eps = R + (Mag >> 45) + 1 bounds |fix - 2^F D|.
//
// The walk.  Accepting swap i changes every b_e by 2 a_e dN_i,e (exact algebra), so the key of a
// later swap j against the running counts is D_j + 2 sum_{accepted i} X(i, j) with
// X(i, j) = sum_e a_e dN_i,e dN_j,e.  Per batch of 32 ranked candidates the walk evaluates their keys
// against the running FP32 coefficients (with the bound of running_coefficient) and their cross
// terms in FP32 with bounds; warp 0 then decides in order with scalar corrections.
#pragma once
#include <climits>

#include "hea_search.cuh"

namespace hea {

constexpr int kFixBitsA = 32;   // |A_e| < 2^32
constexpr int kFixBitsB = 38;   // |B_e| < 2^38 at the step start
constexpr int kFastEdges = 64;  // the walk's fast path handles at most this many conflicting record pairs

// Largest F with maxabs 2^F < 2^bits (maxabs finite, >= 0); a large value when maxabs is 0.
__device__ __forceinline__ int fix_scale(double maxabs, int bits) {
    if (!(maxabs > 0.0)) return 1100;
    const int ex = (int)((__double_as_longlong(maxabs) >> 52) & 0x7FF);   // maxabs < 2^(max(ex,1) - 1022)
    return bits + 1022 - (ex ? ex : 1);
}

// x 2^F rounded to nearest (mode 0), down (mode -1) or up (mode 1), saturated to +-2^62.  Integer
// operations on the binary64 encoding only.
__device__ __forceinline__ long long fix_round(double x, int F, int mode) {
    constexpr long long kSat = 1ll << 62;
    const long long bits = __double_as_longlong(x);
    const bool neg = bits < 0;
    const int ex = (int)((bits >> 52) & 0x7FF);
    const unsigned long long frac = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
    if (ex == 0 && frac == 0) return 0;
    if (ex == 0x7FF) return neg ? -kSat : kSat;
    const unsigned long long m = ex ? (frac | (1ull << 52)) : frac;   // |x| = m 2^((ex ? ex : 1) - 1075)
    const int s = (ex ? ex : 1) - 1075 + F;                           // |x| 2^F = m 2^s
    // rounding of the magnitude: 1 up, -1 down, 0 nearest
    const int mm = (mode == 0) ? 0 : (((mode < 0) == neg) ? 1 : -1);
    unsigned long long v;
    if (s >= 0) {
        if (s > 9) return neg ? -kSat : kSat;
        v = m << s;
    } else if (s <= -64) {
        v = (mm > 0) ? 1ull : 0ull;   // 0 < magnitude < 2^-11
    } else {
        const int k = -s;
        const unsigned long long q = m >> k, rem = m & ((1ull << k) - 1ull);
        if (mm > 0) v = q + (rem != 0ull ? 1ull : 0ull);
        else if (mm < 0) v = q;
        else v = q + ((rem >> (k - 1)) & 1ull);
    }
    return neg ? -(long long)v : (long long)v;
}

// floor(v / 2^sh) for sh >= 0.
__device__ __forceinline__ long long shift_floor(long long v, int sh) { return sh >= 63 ? (v < 0 ? -1 : 0) : (v >> sh); }

// Threshold at a scale: floor and ceil of thr 2^F.
struct FixThr {
    long long lo, hi;
    bool pos;
};

__device__ __forceinline__ FixThr fix_threshold(const ChainCtx& c, int F) {
    FixThr t;
    t.pos = c.pos_thr;
    t.lo = c.pos_thr ? fix_round(c.thr, F, -1) : 0;
    t.hi = c.pos_thr ? fix_round(c.thr, F, 1) : 0;
    return t;
}

// Eligibility from a fixed-point interval: 1 eligible, 0 not, -1 open.
__device__ __forceinline__ int fix_eligible(long long fix, long long eps, const FixThr& t) {
    if (t.pos) return (fix + eps <= t.lo) ? 1 : ((fix - eps > t.hi) ? 0 : -1);
    return (fix + eps < 0) ? 1 : ((fix - eps >= 0) ? 0 : -1);
}

// Order of two keys from their intervals: 1 when p's key is smaller, 0 when q's is, -1 open.
__device__ __forceinline__ int fix_order(long long fp, long long ep, long long fq, long long eq) {
    if (fp + ep < fq - eq) return 1;
    if (fq + eq < fp - ep) return 0;
    return -1;
}

// Fixed-point key of a swap of species A and B with per-shell swap vectors gb (Sec. 4.5): A
// coefficients fA at scale F + sh, B coefficients fB at scale F.  `tin` (or null) adds a
// per-entry error term (walk: the distance of the running coefficient to the reference one); without
// it the B coefficients are the roundings of the reference ones (half a unit each).
__device__ __forceinline__ void fix_key(int M, int S, const long long* __restrict__ fA,
                                        const long long* __restrict__ fB, const long long* __restrict__ tin, int A,
                                        int B, const uint64_t* gb, int sh, long long& fix, long long& eps) {
    long long SA = 0, SB = 0, MB = 0, TT = 0;
    int q1 = 0, q2 = 0;
    auto term = [&](int e, int d) {
        const long long dd = d;
        const int ad = d < 0 ? -d : d;
        SA += fA[e] * (dd * dd);
        SB += fB[e] * dd;
        MB += (fB[e] < 0 ? -fB[e] : fB[e]) * ad;
        if (tin) TT += tin[e] * ad;
        q1 += ad;
        q2 += d * d;
    };
    for (int k = 0; k < M; ++k) {
        const uint64_t g_k = gb[k];
        const int base = k * S * S;
        const int gA = g_of(g_k, A), gB = g_of(g_k, B);
        for (int y = 0; y < S; ++y) {
            const int gy = g_of(g_k, y);
            // Row A: dN_Ay = g_y + [y==A] g_A - [y==B] g_A; row B: dN_By = -g_y + [y==A] g_B - [y==B] g_B;
            // columns A and B of every other row y: dN_yA = g_y, dN_yB = -g_y.
            const int dA = gy + (y == A ? gA : 0) - (y == B ? gA : 0);
            const int dB = -gy + (y == A ? gB : 0) - (y == B ? gB : 0);
            if (dA != 0) term(base + A * S + y, dA);
            if (dB != 0) term(base + B * S + y, dB);
            if (y != A && y != B && gy != 0) {
                term(base + y * S + A, gy);
                term(base + y * S + B, -gy);
            }
        }
    }
    const long long sa = shift_floor(SA, sh);
    fix = SB + sa;
    const long long mag = MB + sa + q1 + shift_floor((long long)q2, sh) + 2;
    eps = shift_floor((long long)q2, sh + 1) + 2 + (tin ? TT : (long long)((q1 + 1) >> 1)) + (mag >> 45) + 1;
}

// ---- fixed-point tables -------------------------------------------------------------------------
// A_e at scale Fa (once per chain: the a coefficients do not change) and B_e at the step's scale F.
static __device__ void coop_fix_tables(ChainSmem& m, ChainShared& sh, const ChainCtx& c, bool with_a) {
    const int tid = threadIdx.x, T = blockDim.x;
    if (with_a) {
        if (tid == 0) sh.maxb = 0ull;
        __syncthreads();
        for (int e = tid; e < c.E; e += T) atomicMax(&sh.maxb, (unsigned long long)__double_as_longlong(fabs(m.ca[e])));
        __syncthreads();
        const int Fa = min(fix_scale(__longlong_as_double((long long)sh.maxb), kFixBitsA), 1100);
        for (int e = tid; e < c.E; e += T) m.fA[e] = fix_round(m.ca[e], Fa, 0);
        __syncthreads();
        if (tid == 0) {
            sh.fixFa = Fa;
            sh.maxb = 0ull;
        }
        __syncthreads();
        for (int e = tid; e < c.E; e += T) atomicMax(&sh.maxb, (unsigned long long)__double_as_longlong(fabs(m.cb[e])));
        __syncthreads();
    }
    // precondition here: sh.maxb holds max |b_e| of the final coefficients of the step
    const int F = min(sh.fixFa, fix_scale(__longlong_as_double((long long)sh.maxb), kFixBitsB));
    for (int e = tid; e < c.E; e += T) m.fB[e] = fix_round(m.cb[e], F, 0);
    __syncthreads();
    if (tid == 0) {
        sh.fixF = F;
        sh.maxb = 0ull;
    }
    __syncthreads();
}

// ---- key order at the best precision both slots have ---------------------------------------------
// qflag bits: 1 binary64 key in qD; 2 eligible; 4 selected; 8, 32 scratch marks; 16 fixed-point key
// in qfix / qeps.  Every slot has its FP32 interval [qlo, qhi].
template <int BITS>
__device__ __forceinline__ void slot_fixed(ChainSmem& m, const ChainCtx& c, int q, int shA) {
    if (m.qflag[q] & 16u) return;
    const int A = load_species<BITS>(m.types, m.qa[q]), B = load_species<BITS>(m.types, m.qb[q]);
    long long fix, eps;
    fix_key(c.M, c.S, m.fA, m.fB, nullptr, A, B, m.qg + q * c.M, shA, fix, eps);
    m.qfix[q] = fix;
    m.qeps[q] = eps;
    atomicOr(&m.qflag[q], 16u);   // several threads may settle the same slot (same values)
}

template <int BITS>
__device__ __forceinline__ void slot_exact(ChainSmem& m, const ChainCtx& c, int q) {
    if (m.qflag[q] & 1u) return;
    const int A = load_species<BITS>(m.types, m.qa[q]), B = load_species<BITS>(m.types, m.qb[q]);
    m.qD[q] = exact_key(c.M, c.S, m.ca, m.cb, A, B, m.qg + q * c.M);
    atomicOr(&m.qflag[q], 1u);
}

// 1 when slot p's key comes first in (D, k) order, 0 when q's does, -1 when the precision both
// slots have leaves it open.  Two swaps of the same species pair with the same per-shell swap
// vectors have the same key bit for bit (the key is a function of exactly these), so k orders them.
template <int BITS>
__device__ __forceinline__ int slot_order(const ChainSmem& m, const ChainCtx& c, int p, int q) {
    const uint32_t fp = m.qflag[p], fq = m.qflag[q];
    if (fp & fq & 1u) return better(m.qD[p], m.qk[p], m.qD[q], m.qk[q]) ? 1 : 0;
    if (fp & fq & 16u) {
        const int o = fix_order(m.qfix[p], m.qeps[p], m.qfix[q], m.qeps[q]);
        if (o >= 0) return o;
    }
    if (m.qhi[p] < m.qlo[q]) return 1;
    if (m.qhi[q] < m.qlo[p]) return 0;
    if (load_species<BITS>(m.types, m.qa[p]) == load_species<BITS>(m.types, m.qa[q]) &&
        load_species<BITS>(m.types, m.qb[p]) == load_species<BITS>(m.types, m.qb[q])) {
        bool same = true;
        for (int k = 0; k < c.M; ++k) same = same && m.qg[p * c.M + k] == m.qg[q * c.M + k];
        if (same) return m.qk[p] < m.qk[q] ? 1 : 0;
    }
    return -1;
}

// The first slot in (D, k) order among the slots marked with `bit` (thread 0 only): argmin of the
// lower bounds, then the slots that may still come first get fixed-point and, if needed, binary64
// keys.  Clears the marks.
template <int BITS>
__device__ int first_of_marked(ChainSmem& m, const ChainCtx& c, int n, uint32_t bit, int shA) {
    int w = -1;
    for (int q = 0; q < n; ++q)
        if ((m.qflag[q] & bit) && (w < 0 || m.qlo[q] < m.qlo[w] || (m.qlo[q] == m.qlo[w] && m.qk[q] < m.qk[w]))) w = q;
    for (int tier = 0; tier < 2 && w >= 0; ++tier) {
        // the marked slots whose order against w is open at the current precision
        bool open = false;
        for (int q = 0; q < n; ++q)
            if (q != w && (m.qflag[q] & bit) && slot_order<BITS>(m, c, q, w) < 0) open = true;
        if (!open) break;
        for (int q = 0; q < n; ++q)
            if (m.qflag[q] & bit) {
                if (tier == 0) slot_fixed<BITS>(m, c, q, shA);
                else slot_exact<BITS>(m, c, q);
            }
        for (int q = 0; q < n; ++q)
            if (q != w && (m.qflag[q] & bit) && slot_order<BITS>(m, c, q, w) == 1) w = q;
        // with every marked slot at the new precision the argmin above is exact unless a pair stays
        // open, which the next tier (binary64) settles
    }
    for (int q = 0; q < n; ++q) m.qflag[q] &= ~bit;
    return w;
}

// ---- 2. local selection (multi-accept): the `top` best eligible queued candidates by (D, k) -----
// Eligibility from the FP32 interval, else the fixed-point key, else the binary64 key.  Then `top`
// rounds of: argmin by (lower bound, k) over the eligible; if the FP32 intervals of other eligible
// candidates reach the winner's upper bound, the first among them in (D, k) order is found at a
// higher precision (first_of_marked).
// Slots [0, n_keep) hold candidates carried from the previous chunk (eligible, flags kept).
template <int BITS>
__device__ int coop_select(ChainSmem& m, ChainShared& sh, const ChainCtx& c, int top, int n_keep) {
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const int qn = sh.qn, shA = sh.fixFa - sh.fixF;
    const FixThr thr = fix_threshold(c, sh.fixF);
    for (int q = tid + n_keep; q < qn; q += T) {
        const uint32_t a = m.qa[q], b = m.qb[q];
        const int A = load_species<BITS>(m.types, a), B = load_species<BITS>(m.types, b);
        m.qflag[q] = 0u;
        if (a == b || A == B) continue;   // null moves are never accepted
        int v = eligible_interval(m.qlo[q], m.qhi[q], c.pos_thr, c.thr_lo, c.thr_hi);
        if (v < 0) {
            slot_fixed<BITS>(m, c, q, shA);
            v = fix_eligible(m.qfix[q], m.qeps[q], thr);
        }
        if (v < 0) {
            slot_exact<BITS>(m, c, q);
            v = eligible(m.qD[q], false, c.thr) ? 1 : 0;
        }
        if (v == 1) m.qflag[q] |= 2u;
    }
    __syncthreads();
    int n_sel = 0;
    for (int t = 0; t < top; ++t) {
        float blo = CUDART_INF_F;
        uint32_t bk = 0xFFFFFFFFu;
        int bq = -1;
        for (int q = tid; q < qn; q += T) {
            if ((m.qflag[q] & 6u) != 2u) continue;
            const float lo = m.qlo[q];
            const uint32_t k = m.qk[q];
            if (bq < 0 || lo < blo || (lo == blo && k < bk)) {
                blo = lo;
                bk = k;
                bq = q;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float olo = __shfl_xor_sync(0xFFFFFFFFu, blo, o);
            const uint32_t ok = __shfl_xor_sync(0xFFFFFFFFu, bk, o);
            const int oq = __shfl_xor_sync(0xFFFFFFFFu, bq, o);
            if (oq >= 0 && (bq < 0 || olo < blo || (olo == blo && ok < bk))) {
                blo = olo;
                bk = ok;
                bq = oq;
            }
        }
        if (lane == 0) {
            sh.red_f[warp] = blo;
            sh.red_k[warp] = bk;
            sh.red_q[warp] = bq;
        }
        __syncthreads();
        if (tid == 0) {
            int q = -1;
            for (int x = 0; x < nw; ++x)
                if (sh.red_q[x] >= 0 &&
                    (q < 0 || sh.red_f[x] < m.qlo[q] || (sh.red_f[x] == m.qlo[q] && sh.red_k[x] < m.qk[q])))
                    q = sh.red_q[x];
            sh.win_q = q;
            sh.n_amb = 0;
        }
        __syncthreads();
        const int w = sh.win_q;
        if (w < 0) break;
        const float whi = m.qhi[w];
        for (int q = tid; q < qn; q += T)
            if (q != w && (m.qflag[q] & 6u) == 2u && m.qlo[q] <= whi) {
                m.qflag[q] |= 8u;
                sh.n_amb = 1;
            }
        __syncthreads();
        if (tid == 0) {
            int win = w;
            if (sh.n_amb) {
                m.qflag[w] |= 8u;
                win = first_of_marked<BITS>(m, c, qn, 8u, shA);
            }
            m.qflag[win] |= 4u;
            m.order[n_sel] = (uint32_t)win;
        }
        ++n_sel;
        __syncthreads();
    }
    return n_sel;
}

// Moves the selected slots order[0, n) to slots [0, n) (keeping their keys and flags, clearing the
// selection marks) so that the next chunk's candidates can be queued after them.
static __device__ void carry_winners(ChainSmem& m, const ChainCtx& c, int n) {
    const int tid = threadIdx.x;
    uint32_t k = 0, a = 0, b = 0, fl = 0;
    float lo = 0.f, hi = 0.f;
    double D = 0.0;
    long long fx = 0, ep = 0;
    uint64_t g[kMaxShells] = {};
    if (tid < n) {
        const uint32_t q = m.order[tid];
        k = m.qk[q];
        a = m.qa[q];
        b = m.qb[q];
        lo = m.qlo[q];
        hi = m.qhi[q];
        D = m.qD[q];
        fx = m.qfix[q];
        ep = m.qeps[q];
        fl = m.qflag[q] & 19u;   // binary64 key, eligible, fixed-point key
        for (int s = 0; s < c.M; ++s) g[s] = m.qg[q * c.M + s];
    }
    __syncthreads();
    if (tid < n) {
        m.qk[tid] = k;
        m.qa[tid] = a;
        m.qb[tid] = b;
        m.qlo[tid] = lo;
        m.qhi[tid] = hi;
        m.qD[tid] = D;
        m.qfix[tid] = fx;
        m.qeps[tid] = ep;
        m.qflag[tid] = fl;
        for (int s = 0; s < c.M; ++s) m.qg[tid * c.M + s] = g[s];
        m.order[tid] = (uint32_t)tid;
    }
    __syncthreads();
}

// ---- 3./4. exchange -----------------------------------------------------------------------------
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t load_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Waits (bounded by d.wait_ns) until every CTA has published local step ls, then merges their
// records into slots [0, sh.qn).  One thread polls the step parity's arrival counter (acquire,
// with a short sleep between polls so that the grid's pollers leave L2 to the publishers); after
// the barrier every thread reads one CTA's tag and records from L2 in a single round.  Returns
// false (in every thread) when the wait ran out.
static __device__ bool coop_gather(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c,
                                   const CoopHeader* hdr, const unsigned long long* tags, const CoopRecord* recs,
                                   int par, uint32_t ls, int top) {
    const int tid = threadIdx.x, T = blockDim.x, G = gridDim.x;
    if (tid == 0) {
        sh.qn = 0;
        sh.sync_fail = 0;
        const uint32_t target = (uint32_t)G * (ls / 2u + 1u);
        if (load_acquire_u32(&hdr->arrive[par]) < target) {
            const uint64_t t0 = globaltimer_ns();
            uint32_t it = 0;
            while (load_acquire_u32(&hdr->arrive[par]) < target) {
                __nanosleep(64);
                if ((++it & 15u) == 0u && (int64_t)(globaltimer_ns() - t0) > d.wait_ns) {
                    sh.sync_fail = 1;
                    break;
                }
            }
        }
        // the acquire load orders the reads below (through the barrier) after every release it saw
    }
    __syncthreads();
    if (sh.sync_fail) return false;
    for (int x = tid; x < G * top; x += T) {
        const int r = x / top, i = x - r * top;
        const unsigned long long t = __ldcg(tags + (size_t)par * G + r);
        const CoopRecord* R = &recs[((size_t)par * G + r) * kCoopMaxTop + i];
        // the record's fields are loaded before the tag is checked, so that both take one round trip
        const double D = __ldcg(&R->D);
        const float lo = __ldcg(&R->lo), hi = __ldcg(&R->hi);
        const uint32_t fl = __ldcg(&R->flags), k = __ldcg(&R->k), a = __ldcg(&R->a), b = __ldcg(&R->b);
        uint64_t g[kMaxShells];
#pragma unroll
        for (int s = 0; s < kMaxShells; ++s)
            if (s < c.M) g[s] = __ldcg(&R->g[s]);
        if (i == 0 && r == 0) sh.pub_stop = (int)((t >> 16) & 1u);
        if ((uint32_t)(t >> 32) != ls + 1u) sh.sync_fail = 1;   // cannot happen once the counter is complete
        if (i >= (int)(t & 0xFFu)) continue;
        const int slot = atomicAdd(&sh.qn, 1);
        m.qD[slot] = D;
        m.qlo[slot] = lo;
        m.qhi[slot] = hi;
        m.qflag[slot] = fl;
        m.qk[slot] = k;
        m.qa[slot] = a;
        m.qb[slot] = b;
#pragma unroll
        for (int s = 0; s < kMaxShells; ++s)
            if (s < c.M) m.qg[slot * c.M + s] = g[s];
    }
    __syncthreads();
    return !sh.sync_fail;
}

// ---- rank of a list of slots among themselves by (D, k) ------------------------------------------
// rank(list[x]) = number of list members before it, taken on FP32 intervals, then (for the pairs
// the intervals leave open) on fixed-point keys, then binary64 keys.  Writes m.acc[slot] = rank and
// sorted[rank] = slot.
template <int BITS>
__device__ void rank_list(ChainSmem& m, ChainShared& sh, const ChainCtx& c, const uint16_t* list, int n,
                          uint16_t* sorted) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int shA = sh.fixFa - sh.fixF;
    for (int tier = 0; tier < 3; ++tier) {
        if (tid == 0) sh.n_amb = 0;
        __syncthreads();
        for (int x = tid; x < n; x += T) {
            const int q = list[x];
            uint32_t cnt = 0u;
            bool open = false;
            for (int y = 0; y < n; ++y) {
                const int p = list[y];
                if (p == q) continue;
                const int o = slot_order<BITS>(m, c, p, q);
                if (o < 0)
                    open = true;
                else
                    cnt += (uint32_t)o;
            }
            m.acc[q] = cnt;
            if (open) {
                m.qflag[q] |= 8u;
                sh.n_amb = 1;
            }
        }
        __syncthreads();
        if (!sh.n_amb) break;
        for (int x = tid; x < n; x += T) {
            const int q = list[x];
            if (m.qflag[q] & 8u) {
                if (tier == 0) slot_fixed<BITS>(m, c, q, shA);
                else slot_exact<BITS>(m, c, q);
                m.qflag[q] &= ~8u;
            }
        }
        __syncthreads();
    }
    for (int x = tid; x < n; x += T) sorted[m.acc[list[x]]] = list[x];
    __syncthreads();
}

// ---- 5a. global rank of the merged records by (D, k) --------------------------------------------
// rank(q) = number of records before q.  First counted on the FP32 intervals; records whose interval
// overlaps another's are flagged and, for them only, the open pairs are settled with fixed-point
// keys, then (if still open) binary64 keys.  Writes m.order[rank] = slot.
template <int BITS>
__device__ void coop_rank(ChainSmem& m, ChainShared& sh, const ChainCtx& c, int ne) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int parts = max(1, min(8, T / max(ne, 1)));
    const int shA = sh.fixFa - sh.fixF;
    for (int q = tid; q < ne; q += T) m.acc[q] = 0u;
    if (tid == 0) sh.n_amb = 0;
    __syncthreads();
    for (int x = tid; x < ne * parts; x += T) {
        const int q = x % ne, part = x / ne;
        const int p0 = part * ne / parts, p1 = (part + 1) * ne / parts;
        const float loq = m.qlo[q], hiq = m.qhi[q];
        uint32_t cnt = 0u, amb = 0u;
        for (int p = p0; p < p1; ++p) {
            const float lop = m.qlo[p], hip = m.qhi[p];
            const uint32_t before = hip < loq ? 1u : 0u;
            cnt += before;
            amb |= (p != q && !before && !(hiq < lop)) ? 1u : 0u;
        }
        if (cnt) atomicAdd(&m.acc[q], cnt);
        if (amb) {
            atomicOr(&m.qflag[q], 8u);
            sh.n_amb = 1;
        }
    }
    __syncthreads();
    if (sh.n_amb) {
        // Flagged records: add the records their FP32 interval overlaps and that come first at a
        // higher precision (every flagged record gets a fixed-point key, then the still open ones a
        // binary64 key; an overlap is symmetric, so both records of an open pair are flagged).
        for (int tier = 0; tier < 2; ++tier) {
            for (int q = tid; q < ne; q += T)
                if (m.qflag[q] & 8u) {
                    if (tier == 0) slot_fixed<BITS>(m, c, q, shA);
                    else if (m.qflag[q] & 32u) slot_exact<BITS>(m, c, q);
                }
            if (tid == 0) sh.n_amb = 0;
            __syncthreads();
            // one warp per flagged record, its lanes over the other records
            const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
            for (int q = warp; q < ne; q += nw) {
                const uint32_t fq = m.qflag[q];
                if (!(fq & 8u)) continue;
                if (tier == 1 && !(fq & 32u)) continue;
                const float loq = m.qlo[q], hiq = m.qhi[q];
                uint32_t extra = 0u;
                bool open = false;
                for (int p = lane; p < ne; p += 32) {
                    if (p == q || m.qhi[p] < loq || hiq < m.qlo[p]) continue;
                    const int o = slot_order<BITS>(m, c, p, q);
                    if (o < 0)
                        open = true;
                    else
                        extra += (uint32_t)o;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) extra += __shfl_xor_sync(0xFFFFFFFFu, extra, o);
                open = __any_sync(0xFFFFFFFFu, open);
                if (lane == 0) {
                    if (!open) {
                        m.acc[q] += extra;
                        m.qflag[q] = fq & ~40u;
                    } else {
                        m.qflag[q] = fq | 32u;
                        sh.n_amb = 1;
                    }
                }
            }
            __syncthreads();
            if (!sh.n_amb) break;
        }
    }
    for (int q = tid; q < ne; q += T) m.order[m.acc[q]] = (uint32_t)q;
    __syncthreads();
}

// ---- 5b. the walk ---------------------------------------------------------------------------------
// Shared memory of the walk (offsets in coop_walk_arrays, sizes in coop_walk_bytes).
struct CoopWalk {
    int8_t* dense;     // [nrec][Ep] count changes of the ranked candidates
    uint32_t* site;    // [nrec][2]
    uint8_t* spec;     // [nrec][2] species of a and b at the step start
    int16_t* pos;      // [nrec][6] half-unit positions of a and b
    // (dense, site, spec, pos and conf are indexed by slot; the walk reaches them through m.order)
    uint32_t* conf;    // [nrec][nw] bit q' of row q: merged records q and q' conflict (slot space)
    int32_t* Ptot;     // [Ep] sums over the records of the positive | negative dN_e (low | high 16 bits)
    uint32_t* accb;    // [2 nw] fast path: accepted records, then scratch (slot space)
    uint32_t* edge;    // [2 nrec] conflicting record pairs (slot << 16 | slot)
    uint32_t* cellA;   // occupancy of hashed conventional cells (one bit per hash value)
    uint32_t* cellB;   // cells occupied more than once
    uint16_t* susp;    // sites (2 r + 0 / 1) near another candidate's site
    float* W;          // [32][Ws] batch rows fa_e dN_e (row stride Ws = 4 mod 8 floats: no bank conflicts)
    float* R;          // [32][Ws] batch rows dN_e
    float *XT, *XeT;   // [32][33] cross terms X(i, j) of the batch and their bounds, at [j][i]
    float *PX, *PE, *PA;   // [32][33] at [j][k]: sums over the open i < min(k, j) of X(i, j), its bound, |X(i, j)|
    float *bD, *bE;    // [32] running keys of the batch's candidates and their bounds
    uint32_t *bMask, *bPrior;   // [32] conflicts inside the batch / with swaps accepted before it
};

__host__ __device__ inline uint32_t coop_row_stride(int E) {
    const uint32_t Ep = ((uint32_t)E + 3u) & ~3u;
    return (Ep % 8u == 4u) ? Ep : Ep + 4u;
}

__device__ __forceinline__ CoopWalk coop_walk_arrays(uint8_t* p, int nrec, int E) {
    const uint32_t n = (uint32_t)nrec, Ep = ((uint32_t)E + 3u) & ~3u, Ws = coop_row_stride(E);
    const uint32_t nw = (n + 31u) / 32u;
    CoopWalk w;
    w.dense = reinterpret_cast<int8_t*>(p);
    p += align_up(n * Ep, 16);
    w.site = reinterpret_cast<uint32_t*>(p);
    p += align_up(8 * n, 16);
    w.spec = p;
    p += align_up(2 * n, 16);
    w.pos = reinterpret_cast<int16_t*>(p);
    p += align_up(12 * n, 16);
    w.conf = reinterpret_cast<uint32_t*>(p);
    p += align_up(4 * n * nw, 16);
    w.Ptot = reinterpret_cast<int32_t*>(p);
    p += align_up(4 * Ep, 16);
    w.accb = reinterpret_cast<uint32_t*>(p);
    p += align_up(8 * nw, 16);
    w.edge = reinterpret_cast<uint32_t*>(p);
    p += align_up(8 * n, 16);
    w.cellA = reinterpret_cast<uint32_t*>(p);
    p += kCoopCellWords * 4;
    w.cellB = reinterpret_cast<uint32_t*>(p);
    p += kCoopCellWords * 4;
    w.susp = reinterpret_cast<uint16_t*>(p);
    p += align_up(4 * n, 16);
    w.W = reinterpret_cast<float*>(p);
    p += 4 * 32 * Ws;
    w.R = reinterpret_cast<float*>(p);
    p += 4 * 32 * Ws;
    float* f = reinterpret_cast<float*>(p);
    w.XT = f;
    w.XeT = f + 32 * 33;
    w.PX = f + 2 * 32 * 33;
    w.PE = f + 3 * 32 * 33;
    w.PA = f + 4 * 32 * 33;
    w.bD = f + 5 * 32 * 33;
    w.bE = w.bD + 32;
    w.bMask = reinterpret_cast<uint32_t*>(w.bE + 32);
    w.bPrior = w.bMask + 32;
    return w;
}

// Bits [lo, hi) of a 32-bit mask (0 <= lo <= hi <= 32).
__device__ __forceinline__ uint32_t gl_span(int lo, int hi) {
    const uint32_t below_hi = hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u);
    return below_hi & ~((1u << lo) - 1u);
}

// FP32 rows of the batch starting at ranked candidate r0: R = dN, W = fa dN.
__device__ __forceinline__ void batch_rows(const CoopWalk& w, const ChainSmem& m, int r0, int nb, int E, int Ep,
                                           int Ws) {
    for (int x = threadIdx.x; x < nb * Ep; x += blockDim.x) {
        const int j = x / Ep, e = x - j * Ep;
        const float v = (float)w.dense[m.order[r0 + j] * Ep + e];
        w.R[j * Ws + e] = v;
        w.W[j * Ws + e] = (e < E) ? m.fa[e] * v : 0.0f;
    }
}

// Hash of a conventional cell (cx, cy, cz) into the occupancy bitmaps.
__device__ __forceinline__ uint32_t cell_hash(const Geo& g, int cx, int cy, int cz) {
    const uint32_t cell = ((uint32_t)cz * (uint32_t)g.Ly + (uint32_t)cy) * (uint32_t)g.Lx + (uint32_t)cx;
    if ((uint32_t)g.V <= (1u << kCoopCellBits)) return cell;   // one bit per cell
    return (cell * 0x9E3779B1u) >> (32 - kCoopCellBits);
}

__device__ __forceinline__ int wrap_cell(int x, int L) { return x < 0 ? x + L : (x >= L ? x - L : x); }

template <int KIND, int BITS>
__device__ void coop_walk(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c, int ne) {
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int S = c.S, M = c.M, SS = S * S, E = c.E, Ep = (E + 3) & ~3, Ws = (int)coop_row_stride(E);
    const int nw = (ne + 31) / 32;
    CoopWalk w = coop_walk_arrays(m.walk, d.nrec, E);
    const int reach = c_shells[KIND].reach[M - 1];
    const int rc = (reach + 1) / 2;   // sites within shell M lie in cells at most rc apart per axis
    // P0: sites, step-start species and positions of the merged records (slot space); occupancy of
    // their conventional cells.
    for (int q = tid; q < ne; q += T) {
        const uint32_t a = m.qa[q], b = m.qb[q];
        w.site[2 * q] = a;
        w.site[2 * q + 1] = b;
        w.spec[2 * q] = (uint8_t)load_species<BITS>(m.types, a);
        w.spec[2 * q + 1] = (uint8_t)load_species<BITS>(m.types, b);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int X, Y, Z;
            site_coords<KIND>(c.g, h ? b : a, X, Y, Z);
            w.pos[6 * q + 3 * h + 0] = (int16_t)X;
            w.pos[6 * q + 3 * h + 1] = (int16_t)Y;
            w.pos[6 * q + 3 * h + 2] = (int16_t)Z;
            const uint32_t hc = cell_hash(c.g, X >> 1, Y >> 1, Z >> 1);
            const uint32_t bit = 1u << (hc & 31);
            if (atomicOr(&w.cellA[hc >> 5], bit) & bit) atomicOr(&w.cellB[hc >> 5], bit);
        }
    }
    for (int x = tid; x < ne * nw; x += T) w.conf[x] = 0u;
    for (int x = tid; x < nw; x += T) sh.taken[x] = 0u;
    for (int e = tid; e < Ep; e += T) w.Ptot[e] = 0;
    if (tid == 0) {
        sh.n_acc = 0;
        sh.walk_done = 0;
        sh.n_pairs = 0;
        sh.n_amb = 0;
        sh.n_edges = 0;
    }
    __syncthreads();
    // P1: dense count changes, one (record, shell) block each, and their per-entry totals; suspects:
    // sites whose own cell holds another record's site or whose neighbouring cells hold any.
    for (int x = tid; x < ne * M; x += T) {
        const int q = x / M, k = x - q * M;
        const int A = w.spec[2 * q], B = w.spec[2 * q + 1];
        const uint64_t g_k = m.qg[q * M + k];
        int8_t* row = w.dense + q * Ep + k * SS;
        for (int idx = 0, i = 0, j = 0; idx < SS; ++idx) {
            row[idx] = (int8_t)entry_delta(g_k, A, B, i, j);
            if (++j == S) {
                j = 0;
                ++i;
            }
        }
        if (k == M - 1)
            for (int e = E; e < Ep; ++e) w.dense[q * Ep + e] = 0;
    }
    for (int s2 = tid; s2 < 2 * ne; s2 += T) {
        const int16_t* P3 = w.pos + 3 * s2;
        const int cx = P3[0] >> 1, cy = P3[1] >> 1, cz = P3[2] >> 1;
        bool near = false;
        if (rc == 1) {
            // the 27 cells at once (independent loads)
            int wx[3], wy[3], wz[3];
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                wx[o] = wrap_cell(cx + o - 1, c.g.Lx);
                wy[o] = wrap_cell(cy + o - 1, c.g.Ly);
                wz[o] = wrap_cell(cz + o - 1, c.g.Lz);
            }
            uint32_t hit = 0u;
#pragma unroll
            for (int oz = 0; oz < 3; ++oz)
#pragma unroll
                for (int oy = 0; oy < 3; ++oy)
#pragma unroll
                    for (int ox = 0; ox < 3; ++ox) {
                        const uint32_t hc = cell_hash(c.g, wx[ox], wy[oy], wz[oz]);
                        const uint32_t* map = (ox == 1 && oy == 1 && oz == 1) ? w.cellB : w.cellA;
                        hit |= (map[hc >> 5] >> (hc & 31)) & 1u;
                    }
            near = hit != 0u;
        } else {
            for (int dz = -rc; dz <= rc && !near; ++dz)
                for (int dy = -rc; dy <= rc && !near; ++dy)
                    for (int dx = -rc; dx <= rc; ++dx) {
                        const uint32_t hc = cell_hash(c.g, wrap_cell(cx + dx, c.g.Lx), wrap_cell(cy + dy, c.g.Ly),
                                                      wrap_cell(cz + dz, c.g.Lz));
                        const uint32_t* map = (dx == 0 && dy == 0 && dz == 0) ? w.cellB : w.cellA;
                        if ((map[hc >> 5] >> (hc & 31)) & 1u) {
                            near = true;
                            break;
                        }
                    }
        }
        if (near) w.susp[atomicAdd(&sh.n_pairs, 1)] = (uint16_t)s2;
    }
    __syncthreads();
    // P2: exact conflicts among the suspects (minimum-image distance within shell M, the same relation
    // as closed shell neighbourhoods for cells of at least two conventional cells per axis); the
    // occupancy bits are cleared for the next step.  Sure records: accepting any set of the other
    // records shifts a record's key by 2 sum_i X(i, j) <= U = 2 sum_e a_e |dN_j,e| P_e, P_e the sum over
    // the records of the changes of dN_j,e's sign;
    // a record whose step-start interval stays eligible under that shift (plus the roundings of the
    // binary64 coefficients at the running counts) is accepted unless a conflicting record before it
    // is.
    {
        const int ns = sh.n_pairs;
        const int r2max = c_shells[KIND].radius2[M - 1];
        const int PX = 2 * c.g.Lx, PY = 2 * c.g.Ly, PZ = 2 * c.g.Lz;
        // pairs u < v of the suspects: row u of the strict upper triangle holds ns - 1 - u pairs
        for (int x = tid; x < ns * (ns - 1) / 2; x += T) {
            // invert x = u (2 ns - u - 1) / 2 + (v - u - 1): the largest u with start(u) <= x
            int u = (int)((2.0f * ns - 1.0f - sqrtf((2.0f * ns - 1.0f) * (2.0f * ns - 1.0f) - 8.0f * x)) * 0.5f);
            u = max(0, min(u, ns - 2));
            while (u > 0 && u * (2 * ns - u - 1) / 2 > x) --u;
            while (u + 1 <= ns - 2 && (u + 1) * (2 * ns - u - 2) / 2 <= x) ++u;
            const int v = x - u * (2 * ns - u - 1) / 2 + u + 1;
            const int s0 = w.susp[u], t0 = w.susp[v];
            const int qs = s0 >> 1, qt = t0 >> 1;
            if (qs == qt) continue;
            const int16_t* P = w.pos + 3 * s0;
            const int16_t* Q = w.pos + 3 * t0;
            const int dx = wrap_min_image(P[0] - Q[0], PX), dy = wrap_min_image(P[1] - Q[1], PY),
                      dz = wrap_min_image(P[2] - Q[2], PZ);
            if (dx * dx + dy * dy + dz * dz <= r2max) {
                const uint32_t old_bit = atomicOr(&w.conf[qs * nw + (qt >> 5)], 1u << (qt & 31));
                atomicOr(&w.conf[qt * nw + (qs >> 5)], 1u << (qs & 31));
                if (!((old_bit >> (qt & 31)) & 1u)) {   // a new edge (several site pairs may find it)
                    const int x = atomicAdd(&sh.n_edges, 1);
                    if (x < 2 * d.nrec) w.edge[x] = ((uint32_t)qs << 16) | (uint32_t)qt;
                }
            }
        }
        for (int s2 = tid; s2 < 2 * ne; s2 += T) {
            const int16_t* P3 = w.pos + 3 * s2;
            const uint32_t hc = cell_hash(c.g, P3[0] >> 1, P3[1] >> 1, P3[2] >> 1);
            atomicAnd(&w.cellA[hc >> 5], ~(1u << (hc & 31)));
            atomicAnd(&w.cellB[hc >> 5], ~(1u << (hc & 31)));
        }
        // per-entry totals over the records of the positive and the negative count changes (low and
        // high 16 bits: each is at most 640 x 48), in parts of the record list
        {
            const int parts = max(1, T / Ep);
            for (int x = tid; x < Ep * parts; x += T) {
                const int e = x % Ep, part = x / Ep;
                int sum = 0;
                for (int q = part; q < ne; q += parts) {
                    const int v = w.dense[q * Ep + e];
                    sum += v > 0 ? v : (-v << 16);
                }
                if (sum) atomicAdd(&w.Ptot[e], sum);
            }
        }
        __syncthreads();
        // eight lanes per record, each summing every eighth entry (an entry with dN = 0 adds an exact
        // 0), then a three-level tree: at most 9 roundings per sum, inside the 32 u allowed below
        for (int q0 = 0; q0 < ne; q0 += T / 8) {
            const int q = q0 + (tid >> 3), l8 = tid & 7;
            float U = 0.f, tin = 0.f;
            if (q < ne) {
                const int8_t* row = w.dense + q * Ep;
                for (int e = l8; e < E; e += 8) {
                    // the accepted records' changes sum to S_e in [-Pneg_e, Ppos_e], so a_e dN S_e is at
                    // most a_e dN Ppos_e (dN > 0) or a_e |dN| Pneg_e (dN < 0)
                    const int dl = row[e];
                    const float ad = (float)(dl < 0 ? -dl : dl);
                    const int P = w.Ptot[e];
                    const float side = (float)(dl > 0 ? (P & 0xFFFF) : (P >> 16));
                    U = fmaf(fabsf(m.fa[e]) * ad, side, U);
                    tin = fmaf(ad, 2.0f * m.tiny[e], tin);
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                U += __shfl_xor_sync(0xFFFFFFFFu, U, o);
                tin += __shfl_xor_sync(0xFFFFFFFFu, tin, o);
            }
            if (q < ne && l8 == 0) {
                U = 2.0f * U * (1.0f + 16.0f * kTwoUlp);
                const float hi = m.qhi[q], lo = m.qlo[q];
                const float slack = fmaf(kTwoPow20, (hi - lo) + U, tin + kAbsBound);
                const float top = __fadd_ru(__fadd_ru(hi, U), slack);
                const bool sure = c.pos_thr ? (top <= c.thr_lo) : (top < 0.f);
                if (sure)
                    m.qflag[q] |= 64u;
                else
                    sh.n_amb = 1;
            }
        }
    }
    __syncthreads();
    // The edge list holds 2 nrec pairs; with more conflicting pairs the full path (conflict matrix) runs.
    if (!sh.n_amb && d.max_accept == 0 && sh.n_edges <= kFastEdges && sh.n_edges <= 2 * d.nrec) {
        // Fast path: every record is accepted unless it conflicts with an accepted record before it
        // in (D, k) order.  Only the conflicting pairs need an order: one thread per edge orients it
        // (at the precision that settles it), then the greedy choice is the fixed point of
        // "accepted unless an accepted neighbour comes first", reached from all-accepted in at most
        // (longest chain of edges + 1) sweeps.
        const int ned = sh.n_edges;
        const int shA = sh.fixFa - sh.fixF;
        for (int x = tid; x < nw; x += T) w.accb[x] = (x == nw - 1 && (ne & 31)) ? ((1u << (ne & 31)) - 1u) : 0xFFFFFFFFu;
        for (int x = tid; x < ned; x += T) {
            const int u = (int)(w.edge[x] >> 16), v = (int)(w.edge[x] & 0xFFFFu);
            int o = slot_order<BITS>(m, c, u, v);
            if (o < 0) {
                slot_fixed<BITS>(m, c, u, shA);
                slot_fixed<BITS>(m, c, v, shA);
                o = slot_order<BITS>(m, c, u, v);
            }
            if (o < 0) {
                slot_exact<BITS>(m, c, u);
                slot_exact<BITS>(m, c, v);
                o = slot_order<BITS>(m, c, u, v);
            }
            // stored as (first << 16) | second
            w.edge[x] = o == 1 ? (((uint32_t)u << 16) | (uint32_t)v) : (((uint32_t)v << 16) | (uint32_t)u);
        }
        __syncthreads();
        if (warp == 0) {
            // accepted = all records except those with an accepted record before them in a conflict,
            // iterated from all-accepted to the fixed point; one lane per edge (ned <= 64), one per word
            uint32_t* pred = w.accb + nw;
            uint32_t e0 = 0u, e1 = 0u;
            const bool h0 = lane < ned, h1 = lane + 32 < ned;
            if (h0) e0 = w.edge[lane];
            if (h1) e1 = w.edge[lane + 32];
            for (int sweep = 0; sweep <= ned; ++sweep) {
                if (lane < nw) pred[lane] = 0u;
                __syncwarp();
                if (h0 && ((w.accb[e0 >> 21] >> ((e0 >> 16) & 31)) & 1u))
                    atomicOr(&pred[(e0 & 0xFFFFu) >> 5], 1u << (e0 & 31));
                if (h1 && ((w.accb[e1 >> 21] >> ((e1 >> 16) & 31)) & 1u))
                    atomicOr(&pred[(e1 & 0xFFFFu) >> 5], 1u << (e1 & 31));
                __syncwarp();
                bool changed = false;
                if (lane < nw) {
                    const uint32_t all = (lane == nw - 1 && (ne & 31)) ? ((1u << (ne & 31)) - 1u) : 0xFFFFFFFFu;
                    const uint32_t nv = all & ~pred[lane];
                    changed = nv != w.accb[lane];
                    w.accb[lane] = nv;
                }
                __syncwarp();
                if (!__any_sync(0xFFFFFFFFu, changed)) break;
            }
        }
        __syncthreads();
        // apply every accepted swap: counts, species
        {
            const int parts = max(1, T / max(E, 1));
            for (int x = tid; x < E * parts; x += T) {
                const int e = x % E, part = x / E;
                int dl = 0;
                for (int q = part; q < ne; q += parts)
                    if ((w.accb[q >> 5] >> (q & 31)) & 1u) dl += w.dense[q * Ep + e];
                if (dl) atomicAdd(&m.cnt[e], dl);
            }
            for (int q = tid; q < ne; q += T)
                if ((w.accb[q >> 5] >> (q & 31)) & 1u) {
                    store_species_atomic<BITS>(m.types, w.site[2 * q], w.spec[2 * q + 1]);
                    store_species_atomic<BITS>(m.types, w.site[2 * q + 1], w.spec[2 * q]);
                }
            if (warp == 0) {   // accepted records: the bits of the mask
                int n = 0;
                for (int y = lane; y < nw; y += 32) n += __popc(w.accb[y]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
                if (lane == 0) sh.n_acc = n;
            }
        }
        __syncthreads();
        return;
    }
    // Full path: rank the records by (D, k) (m.order: rank -> slot, m.acc: slot -> rank), then walk.
    coop_rank<BITS>(m, sh, c, ne);
    if (tid == 0) sh.n_pairs = 0;   // bit b: batch b holds a candidate that is not sure
    __syncthreads();
    batch_rows(w, m, 0, min(32, ne), E, Ep, Ws);
    for (int r = tid; r < ne; r += T)
        if (!(m.qflag[m.order[r]] & 64u)) atomicOr(reinterpret_cast<unsigned int*>(&sh.n_pairs), 1u << (r >> 5));
    __syncthreads();
    // The walk in batches of 32 ranked candidates.  For each batch, in parallel: its rows, its
    // candidates' keys against the running state at the start of the batch (FP32 estimates of the
    // running counts' binary64 keys with rigorous bounds), their cross terms X(i, j) and conflicts.
    // Accepting candidate i changes every coefficient b_e by 2 a_e dN_i,e, so the key of a later
    // candidate j moves by exactly 2 X(i, j): warp 0 then decides the batch in order with scalar
    // corrections (the binary64 key against the running counts where the bound cannot decide).
    const float rel = c.rel;
    for (int r0 = 0; r0 < ne; r0 += 32) {
        if (sh.walk_done) break;
        const int nb = min(32, ne - r0);
        const int acc_before = sh.n_acc;
        const bool batch_sure = !((sh.n_pairs >> (r0 >> 5)) & 1);
        // W1: running keys (16 threads per candidate) and cross terms (one warp per column) of the batch,
        // whose rows were built in the previous phase; not needed when every candidate is sure.
        // warp-uniform loop: every lane of a warp takes part in the shuffles
        if (!batch_sure) {
        for (int x0 = tid - lane; x0 < 16 * nb; x0 += T) {
            const int x = x0 + lane;
            const bool act = x < 16 * nb;
            const int j = x >> 4, l16 = x & 15;
            float acc = 0.f, err = 0.f;
            if (act) {
                const float* Rj = w.R + j * Ws;
                for (int e = l16; e < E; e += 16) {
                    const float xv = Rj[e];
                    if (xv == 0.f) continue;
                    const float ax = fabsf(xv);
                    acc = fmaf(xv, fmaf(m.fa[e], xv, m.fb[e]), acc);
                    err = fmaf(ax, fmaf(rel * fabsf(m.fa[e]), ax, fmaf(rel, fabsf(m.fb[e]), m.beta[e])), err);
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                err += __shfl_xor_sync(0xFFFFFFFFu, err, o);
            }
            if (act && l16 == 0) {
                w.bD[j] = acc;
                // A few extra relative ulps cover the rounding of the partial sums.
                w.bE[j] = fmaf(err, 1.0f + 64.0f * kTwoUlp, kAbsBound);
            }
        }
        // Cross terms: one warp per column j, lane i; inclusive scans over i give the prefix sums.
        for (int x = tid; x < 32 * 32; x += T) {
            const int j = x >> 5, i = x & 31;   // warp-uniform j (T is a multiple of 32)
            const bool valid = j < nb && i < j;
            float X = 0.f, Xa = 0.f;
            if (valid) {
                const float4* Wi = reinterpret_cast<const float4*>(w.W + i * Ws);
                const float4* Rj = reinterpret_cast<const float4*>(w.R + j * Ws);
                for (int q4 = 0; q4 < Ep / 4; ++q4) {
                    const float4 u = Wi[q4], v = Rj[q4];
                    X = fmaf(u.x, v.x, X);
                    X = fmaf(u.y, v.y, X);
                    X = fmaf(u.z, v.z, X);
                    X = fmaf(u.w, v.w, X);
                    Xa = fmaf(fabsf(u.x), fabsf(v.x), Xa);
                    Xa = fmaf(fabsf(u.y), fabsf(v.y), Xa);
                    Xa = fmaf(fabsf(u.z), fabsf(v.z), Xa);
                    Xa = fmaf(fabsf(u.w), fabsf(v.w), Xa);
                }
            }
            const float Xe = valid ? fmaf(Xa, rel, kAbsBound) : 0.f;
            float sx = X, se = Xe, sa = fabsf(X);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float tx = __shfl_up_sync(0xFFFFFFFFu, sx, o);
                const float te = __shfl_up_sync(0xFFFFFFFFu, se, o);
                const float ta = __shfl_up_sync(0xFFFFFFFFu, sa, o);
                if (i >= o) {
                    sx += tx;
                    se += te;
                    sa += ta;
                }
            }
            if (j < nb) {
                w.XT[j * 33 + i] = X;
                w.XeT[j * 33 + i] = Xe;
                w.PX[j * 33 + i + 1] = sx;
                w.PE[j * 33 + i + 1] = se;
                w.PA[j * 33 + i + 1] = sa;
                if (i == 0) {
                    w.PX[j * 33] = 0.f;
                    w.PE[j * 33] = 0.f;
                    w.PA[j * 33] = 0.f;
                }
            }
        }
        __syncthreads();
        }
        // W2: decisions, in order, by warp 0; lane j holds candidate j of the batch.  Speculation:
        // every undecided lane evaluates its candidate assuming that all earlier undecided candidates
        // not blocked by earlier batches are accepted; the first lane whose decision contradicts that
        // ends the round, the lanes before it are committed (their assumption held), its own decision
        // was taken under the committed state, and the next round starts after it.  The sums over the
        // assumed candidates [p, j) are differences of the prefix sums, so a round is O(1) per lane.
        if (warp == 0) {
            float D0 = 0.f, E0 = 0.f, pxj = 0.f, pej = 0.f, paj = 0.f;
            uint32_t prior = 1u, mask = 0u;
            const float *PXl = w.PX + lane * 33, *PEl = w.PE + lane * 33, *PAl = w.PA + lane * 33;
            const float* XTl = w.XT + lane * 33;
            bool sure = true;
            if (lane < nb) {
                const int q = m.order[r0 + lane];
                sure = (m.qflag[q] & 64u) != 0u;
                if (!batch_sure) {
                    D0 = w.bD[lane];
                    E0 = w.bE[lane];
                    pxj = PXl[lane];
                    pej = PEl[lane];
                    paj = PAl[lane];
                }
                // conflicts with the swaps accepted in earlier batches, and with earlier candidates here
                prior = 0u;
                for (int y = 0; y < nw; ++y)
                    for (uint32_t bits = w.conf[q * nw + y]; bits; bits &= bits - 1u) {
                        const int rq = (int)m.acc[32 * y + __ffs(bits) - 1];   // rank of the other record
                        if (rq < r0) {
                            if ((sh.taken[rq >> 5] >> (rq & 31)) & 1u) prior = 1u;
                        } else if (rq < r0 + lane) {
                            mask |= 1u << (rq - r0);
                        }
                    }
            }
            // candidates blocked by earlier batches are never accepted; the cross terms of candidates
            // that are not (assumed) accepted, included in the prefix sums, are taken out again
            // wherever a sum spans them
            const uint32_t open = __ballot_sync(0xFFFFFFFFu, lane < nb && prior == 0u);
            float cc = 0.f, ce = 0.f;            // corrections from committed accepted candidates
            uint32_t accm = 0u;                  // committed accepted candidates of the batch
            int n_acc = acc_before, nbacc = 0, p = 0;
            bool done = false;
            while (p < nb && !done) {
                // The guess: the greedy choice among the open candidates from p on if every one of them
                // were eligible -- accepted unless it conflicts with a committed or an earlier guessed
                // candidate.  Each lane depends only on earlier lanes, so iterating the rule from
                // "all open" reaches its unique fixed point (one ballot per link of the longest chain).
                // Candidates that no choice among the undecided ones before them can make eligible:
                // their key at its lowest (committed cross terms plus every negative cross term from
                // p on; sum min(0, X) = (sum X - sum |X|) / 2) is not eligible.  They are rejected
                // without ending a round.
                bool srej = false;
                if (lane >= p && lane < nb && ((open >> lane) & 1u) && !sure && !batch_sure) {
                    const float se = ce + (pej - PEl[p]);
                    const float er = fmaf(fmaf(2.0f, se, E0), 1.0f + 256.0f * kTwoUlp,
                                          fmaf(256.0f * kTwoUlp, fabsf(D0) + 2.0f * (paj + pej), kAbsBound));
                    const float low = cc + 0.5f * ((pxj - PXl[p]) - (paj - PAl[p]));
                    const float vmin = fmaf(2.0f, low, D0);
                    srej = eligible_interval(__fadd_rd(vmin, -2.0f * er), CUDART_INF_F, c.pos_thr, c.thr_lo,
                                             c.thr_hi) == 0;
                }
                const uint32_t cand = open & ~((1u << p) - 1u) & ~__ballot_sync(0xFFFFFFFFu, srej);
                uint32_t guess = cand;
                for (int it = 0; it <= 32; ++it) {
                    const bool in = ((cand >> lane) & 1u) && (mask & (accm | guess)) == 0u;
                    const uint32_t ng = __ballot_sync(0xFFFFFFFFu, in);
                    if (ng == guess) break;
                    guess = ng;
                }
                // A guessed candidate is decided against the committed ones and the guessed ones before
                // it; a candidate left out of the guess is rejected by the guessed one it conflicts with.
                // The round ends at the first guessed candidate that is not eligible (or open).
                int dec = 0;
                if (lane >= p && lane < nb && ((guess >> lane) & 1u)) {
                    const uint32_t gl = guess & ((1u << lane) - 1u);
                    {
                        if (sure || (acc_before == 0 && (accm | gl) == 0u)) {
                            dec = 1;   // sure, or the step-start state: the candidate is eligible
                        } else {
                            float sx = cc + (pxj - PXl[p]);
                            for (uint32_t bb = ~guess & gl_span(p, lane); bb; bb &= bb - 1u) sx -= XTl[__ffs(bb) - 1];
                            const float se = ce + (pej - PEl[p]);
                            const float v = fmaf(2.0f, sx, D0);
                            // Rounding: every prefix sum (5 additions), difference and fold (at most 32
                            // per lane) is within 11 u of the column's total |X| (or total bound), so all
                            // sums taken are within 400 u of them (u = 2^-24); 512 u is allowed.
                            const float er = fmaf(fmaf(2.0f, se, E0), 1.0f + 256.0f * kTwoUlp,
                                                  fmaf(256.0f * kTwoUlp, fabsf(D0) + 2.0f * (paj + pej), kAbsBound));
                            dec = eligible_interval(__fadd_rd(v, -er), __fadd_ru(v, er), c.pos_thr, c.thr_lo, c.thr_hi);
                        }
                    }
                }
                const uint32_t bad = __ballot_sync(0xFFFFFFFFu, lane >= p && lane < nb && ((guess >> lane) & 1u) && dec != 1);
                const int js = bad ? (__ffs(bad) - 1) : nb;
                uint32_t commit = guess & ((js >= 32) ? 0xFFFFFFFFu : ((1u << js) - 1u));
                if (d.max_accept > 0) {
                    const int room = d.max_accept - n_acc;
                    const uint32_t all = commit;
                    while (__popc(commit) > room) commit &= ~(1u << (31 - __clz(commit)));
                    if (__popc(all) > room) done = true;
                }
                if (commit) {
                    // commit is the guessed candidates of [p, end): fold their cross terms in
                    const int end = 32 - __clz(commit);   // one past the last committed candidate
                    if (lane >= end && lane < nb) {
                        cc += PXl[end] - PXl[p];
                        ce += PEl[end] - PEl[p];
                        for (uint32_t bb = ~commit & gl_span(p, end); bb; bb &= bb - 1u) cc -= XTl[__ffs(bb) - 1];
                    }
                }
                if (lane == 0)
                    for (uint32_t bits = commit; bits; bits &= bits - 1u) sh.red_q[nbacc++] = __ffs(bits) - 1;
                nbacc = __shfl_sync(0xFFFFFFFFu, nbacc, 0);
                accm |= commit;
                n_acc += __popc(commit);
                if (done || js >= nb) break;
                if (d.max_accept > 0 && n_acc >= d.max_accept) {
                    done = true;
                    break;
                }
                int dj = __shfl_sync(0xFFFFFFFFu, dec, js);
                if (dj < 0) {
                    // The bound leaves it open: the reference key against the running counts.
                    const int qj = m.order[r0 + js];
                    double Dp = 0.0;
                    if (lane == 0) {
                        int pend[32];
                        for (int x = 0; x < nbacc; ++x) pend[x] = (int)m.order[r0 + sh.red_q[x]];
                        Dp = exact_key_pending(M, S, m.cnt, m.Q, m.tgt, m.ca, d.w, w.spec[2 * qj], w.spec[2 * qj + 1],
                                               m.qg + qj * M, w.dense, Ep, pend, nbacc);
                    }
                    Dp = __shfl_sync(0xFFFFFFFFu, Dp, 0);
                    dj = eligible(Dp, false, c.thr) ? 1 : 0;
                }
                if (dj == 1) {
                    if (lane == 0) sh.red_q[nbacc] = js;
                    if (lane > js && lane < nb) {
                        cc += XTl[js];
                        ce += w.XeT[lane * 33 + js];
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
        // W3: apply the batch's accepted swaps: counts, count changes, running FP32 coefficients,
        // species.
        const int nba = sh.batch_n;
        if (r0 + 32 < ne && !sh.walk_done) batch_rows(w, m, r0 + 32, min(32, ne - r0 - 32), E, Ep, Ws);
        if (nba > 0) {
            for (int e = tid; e < E; e += T) {
                int dl = 0;
                for (int x = 0; x < nba; ++x) dl += w.dense[m.order[r0 + sh.red_q[x]] * Ep + e];
                if (dl == 0) continue;
                m.cnt[e] += dl;
                const int dn = m.dn[e] + dl;
                m.dn[e] = dn;
                running_coefficient(e, dn, m.fw[e], m.fQ, m.fe0, m.tiny, m.fb, m.beta);
            }
            for (int x = tid; x < nba; x += T) {
                const int r = r0 + sh.red_q[x], q = m.order[r];
                store_species_atomic<BITS>(m.types, w.site[2 * q], w.spec[2 * q + 1]);
                store_species_atomic<BITS>(m.types, w.site[2 * q + 1], w.spec[2 * q]);
                atomicOr(&sh.taken[r >> 5], 1u << (r & 31));
            }
        }
        __syncthreads();
    }
}

// After a walk that accepted swaps: binary64 coefficients of every entry from the counts, their
// binary32 roundings for the next step's screen, then the next step's fixed-point B table.
static __device__ void coop_after_walk(const ChainDesc& d, ChainSmem& m, ChainShared& sh, const ChainCtx& c) {
    const int S = c.S;
    const bool changed = sh.n_acc > 0;
    for (int e = threadIdx.x; e < c.E; e += blockDim.x) {
        if (changed) {
            const int k = e / (S * S);
            const double err = __dsub_rn(__dsub_rn(1.0, __dmul_rn((double)m.cnt[e], m.Q[e])), m.tgt[e]);
            const double b = __dmul_rn(-2.0, __dmul_rn(d.w[k], __dmul_rn(m.Q[e], err)));
            m.cb[e] = b;
            m.fb[e] = (float)b;
            m.fe0[e] = (float)err;
            m.dn[e] = 0;
            m.beta[e] = fmaf(kTwoUlp, fabsf(m.fb[e]), m.tiny[e]);
        }
        atomicMax(&sh.maxb, (unsigned long long)__double_as_longlong(fabs(m.cb[e])));
    }
    __syncthreads();
    coop_fix_tables(m, sh, c, false);
}

// ------------------------------------------------------------------------------------------------
// The cooperative chain: gridDim.x co-resident CTAs, CTA r scores candidates [r Kc, (r+1) Kc).
// ------------------------------------------------------------------------------------------------
template <int KIND, int BITS>
__device__ void run_coop_chain(const ChainDesc& d, uint8_t* smem, ChainShared& sh) {
    const ChainLayout L = coop_layout(d.N, d.M, d.S, d.qcap, BITS, d.accept_mode, d.nrec);
    if (L.total > d.smem_bytes) {   // the host placed a different layout: touch nothing
        if (blockIdx.x == 0) report_invalid(d);
        return;
    }
    ChainSmem m(smem, L);
    ChainCtx c;
    chain_setup<KIND, BITS>(d, m, sh, c, false);
    const int G = gridDim.x, rank = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const int top = (d.accept_mode == 0) ? 1 : d.group_top;
    const uint32_t Kc = (uint32_t)(c.K / G);
    uint8_t* ws = static_cast<uint8_t*>(d.workspace);
    CoopHeader* hdr = reinterpret_cast<CoopHeader*>(ws);
    unsigned long long* tags = reinterpret_cast<unsigned long long*>(ws + coop_tags_offset());
    CoopRecord* recs = reinterpret_cast<CoopRecord*>(ws + coop_records_offset(G));
    if (sh.bad) {   // identical in every CTA: the cell is the same
        if (rank == 0) report_invalid(d);
        return;
    }
    if (d.accept_mode == 1) {
        CoopWalk w = coop_walk_arrays(m.walk, d.nrec, c.E);   // occupancy bitmaps start empty
        for (uint32_t x = tid; x < kCoopCellWords; x += T) {
            w.cellA[x] = 0u;
            w.cellB[x] = 0u;
        }
        coop_fix_tables(m, sh, c, true);
    }
    while (!sh.stop) {
        const uint32_t ls = (uint32_t)sh.steps;          // step of this launch
        const uint32_t step = d.step0 + ls;              // Philox step counter
        const int par = (int)(ls & 1u);
        if (tid == 0) {
            sh.qn = 0;
            sh.n_acc = 0;
            sh.win_q = -1;
        }
        __syncthreads();
        const uint32_t k_lo = rank * Kc, k_hi = (rank + 1) * Kc;
        const uint32_t first_end = (d.accept_mode == 1) ? min(k_hi, k_lo + (uint32_t)d.chunk) : k_hi;
        const float my_umin = score_range<KIND, BITS>(d, m, sh, c, step, k_lo, first_end);
        int n_pub = 0;
        if (d.accept_mode == 0) {
            const float umin = block_min(my_umin, sh);
            best_of_queue<BITS>(m, sh, c, umin);
            if (sh.win_q >= 0) {
                if (tid == 0) m.order[0] = (uint32_t)sh.win_q;
                n_pub = 1;
            }
            __syncthreads();
        } else {
            // The slice in chunks: the best `top` so far are carried into the next chunk's slots.
            // (nothing queued beyond the carried winners: they stay the selection, in order)
            __syncthreads();
            n_pub = (sh.qn > 0) ? coop_select<BITS>(m, sh, c, top, 0) : 0;
            for (uint32_t c0 = first_end; c0 < k_hi; c0 += (uint32_t)d.chunk) {
                carry_winners(m, c, n_pub);
                if (tid == 0) sh.qn = n_pub;
                __syncthreads();
                score_range<KIND, BITS>(d, m, sh, c, step, c0, min(k_hi, c0 + (uint32_t)d.chunk));
                __syncthreads();
                if (sh.qn > n_pub) n_pub = coop_select<BITS>(m, sh, c, top, n_pub);
            }
        }
        // Publish this CTA's records for the step (double-buffered by step parity), then the tag.
        for (int x = tid; x < n_pub; x += T) {
            const uint32_t q = m.order[x];
            CoopRecord* R = &recs[((size_t)par * G + rank) * kCoopMaxTop + x];
            R->D = m.qD[q];
            R->lo = m.qlo[q];
            R->hi = m.qhi[q];
            R->flags = (d.accept_mode == 1) ? (m.qflag[q] & 1u) : 1u;
            R->k = m.qk[q];
            R->a = m.qa[q];
            R->b = m.qb[q];
            for (int k = 0; k < c.M; ++k) R->g[k] = m.qg[q * c.M + k];
        }
        __syncthreads();
        if (tid == 0 && d.withhold != rank + 1) {
            const unsigned long long stop =
                (rank == 0 && d.timeout_ns > 0 && (int64_t)(globaltimer_ns() - sh.t0) >= d.timeout_ns) ? 1ull : 0ull;
            __stcg(&tags[(size_t)par * G + rank], ((unsigned long long)(ls + 1u) << 32) | (stop << 16) |
                                                      (unsigned long long)n_pub);
            // release: the records and the tag (written before the barrier above, or by this thread)
            // are visible to every CTA that acquires the counter value this add produces
            red_release_add(&hdr->arrive[par], 1u);
        }
        if (!coop_gather(d, m, sh, c, hdr, tags, recs, par, ls, top)) {
            if (tid == 0) {
                sh.status = HEA_ESYNC;
                atomicExch(&hdr->error, 1);
            }
            __syncthreads();
            break;
        }
        if (d.accept_mode == 0) {
            // Every CTA published its exact argmin: the global argmin over (D, k).
            if (tid == 0) {
                int best = -1;
                for (int q = 0; q < sh.qn; ++q)
                    if (best < 0 || better(m.qD[q], m.qk[q], m.qD[best], m.qk[best])) best = q;
                sh.win_q = best;
            }
            __syncthreads();
            const int q = sh.win_q;
            if (q >= 0) {
                const uint32_t a = m.qa[q], b = m.qb[q];
                const bool null_move = (a == b) || load_species<BITS>(m.types, a) == load_species<BITS>(m.types, b);
                if (eligible(m.qD[q], null_move, c.thr)) apply_slot<BITS>(d, m, sh, c, q);
            }
        } else {
            // No records: nothing to walk; no accepted swap: the coefficients and the fixed-point
            // table of this step stay those of the next one.
            const int ne = sh.qn;
            if (ne > 0) coop_walk<KIND, BITS>(d, m, sh, c, ne);
            __syncthreads();
            if (sh.n_acc > 0) coop_after_walk(d, m, sh, c);
        }
        __syncthreads();
        bookkeeping(d, sh, sh.pub_stop != 0);
    }
    if (rank == 0) write_back<BITS>(d, m, sh, c);
}

}  // namespace hea
