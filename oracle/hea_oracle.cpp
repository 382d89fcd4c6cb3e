// hea_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, serial CPU reference for the short-range-order (SRO) targeted swap search of
// Niu & Liu, "Short-Range Order Based Ultra Fast Large-Scale Modeling of High-Entropy Alloys"
// (arXiv 2411.18906).  Only the test suite, the smoke check and the benchmark's CPU-baseline leg
// may load this library; the product path (the CUDA library) never links, loads or calls it, and
// the two share no code, header, table or constant generator.
//
// What it computes, with the passage each part follows:
//   * Warren-Cowley SRO  alpha_ij^(k) = 1 - P_ij^(k) / c_j                      (Sec. 4.3, Eq. sro)
//     with P_ij^(k) = N_ij^(k) / (N_i Z_k) and c_j = N_j / N, so
//     alpha_ij^(k) = 1 - N_ij^(k) * N / (Z_k N_i N_j).
//   * Fitness F = sqrt( sum_k w_k sum_i sum_j (alpha_ij^(k) - alpha_ij^(k),target)^2 )
//                                                                    (Sec. 4.4, Eq. fitness_function)
//   * Incremental change of the counts for one swap: only pairs that touch the two swapped
//     sites change                                                   (Sec. 4.5, Eq. for Delta alpha)
//   * Parallel Monte Carlo: K tasks each propose one random two-atom swap, the best change is
//     taken, a depth counter counts non-improving rounds             (Sec. 4.2, Alg. parallel_mc)
//   * Depth / step-budget termination                                (Sec. 4.2, Sec. 4.6.4)
//   * An external structure mapped onto the lattice (nearest site)   (Sec. 2.3, application workflow)
//   * Global search: a ranked pool of solutions, fresh random ones each iteration, the best
//     refined by the parallel Monte Carlo search, the worst fraction discarded
//                                                                    (Sec. 4.1, Alg. global_search)
//   * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written here from
//     that paper's definition.
//
// Readings where the paper is silent (each one is listed in the design notes):
//   * Geometry: half-lattice-unit integer coordinates; shells are the distinct lattice-vector
//     lengths in ascending order; vectors inside a shell sorted lexicographically.
//   * Site index = ((b * Lz + cz) * Ly + cy) * Lx + cx, b the basis (sublattice) index.
//     FCC basis (0,0,0),(0,1,1),(1,0,1),(1,1,0); BCC basis (0,0,0),(1,1,1) in half units.
//   * Counts are taken per (site, shell vector) with multiplicity; cells need L >= 2 per axis.
//   * Objective arithmetic (fixed so both implementations agree bit for bit; no implicit FMA):
//       Q_kij = N / ((Z_k * N_i) * N_j),  e_kij = (1 - n_kij * Q_kij) - t_kij,
//       term_kij = w_k * (e_kij * e_kij),  F^2 = sum of terms in (k,i,j) row-major order.
//   * Swap key D = change of F^2, written per entry as dN (a dN + b) with a = w (Q Q) and
//     b = -2 (w (Q e)), summed over (k,i,j) row-major as D <- fma(dN, fma(a, dN, b), D).
//     A swap is accepted only if it strictly lowers the objective (D < 0); a positive threshold
//     additionally accepts non-null moves with D <= threshold.
//   * Best-of-K: argmin over (D, k) with the smaller k on ties.
//   * Multi-accept: candidates with an eligible D walked in ascending (D, k); a candidate is taken
//     if none of its two sites lies in the closed shell neighbourhood of a site already taken this
//     step and its key recomputed against the running counts is still eligible.
//   * Candidate draw: Philox key (lo32(seed), hi32(seed)), counter (k, step, chain, 1);
//     a = floor(r0 * N / 2^32), b = floor(r1 * N / 2^32).
//   * Initial configuration: sites ordered by the 64-bit key (r0 << 32 | i), r0 from Philox counter
//     (i, 0, 0, 0); the site of rank r receives species s with cum[s] <= r < cum[s+1].
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -shared -fPIC: no implicit FMA contraction; the only
// fused operations are the explicit std::fma calls of the swap key.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// Status codes returned by every entry point.
enum { OR_OK = 0, OR_EINVAL = 1, OR_EMISMATCH = 2 };

// ----------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the Philox S-P network on a 128-bit counter
// (c0, c1, c2, c3) with a 64-bit key (k0, k1).  One round:
//   (c0, c1, c2, c3) <- (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
// and the key is bumped by the Weyl constants (k0 += W0, k1 += W1) between rounds.
// ----------------------------------------------------------------------------------------------
void philox_raw(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

void philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    philox_raw(ctr, key, out);
}

// ----------------------------------------------------------------------------------------------
// Lattice geometry (Table 1 caption: supercell S = A * L^3, A = 2 for bcc and 4 for fcc), in
// integer half-lattice-unit coordinates.
// ----------------------------------------------------------------------------------------------
struct Geom {
    int kind;         // 0 = FCC, 1 = BCC
    int L[3];         // conventional cells along x, y, z
    int B;            // basis sites per conventional cell
    int basis[4][3];  // basis offsets in half units
    int64_t V;        // number of conventional cells
    int64_t N;        // number of sites
};

bool make_geom(int kind, int Lx, int Ly, int Lz, Geom* g) {
    if (kind != 0 && kind != 1) return false;
    if (Lx < 2 || Ly < 2 || Lz < 2) return false;
    static const int fcc[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
    static const int bcc[2][3] = {{0, 0, 0}, {1, 1, 1}};
    g->kind = kind;
    g->L[0] = Lx;
    g->L[1] = Ly;
    g->L[2] = Lz;
    g->B = (kind == 0) ? 4 : 2;
    for (int b = 0; b < g->B; ++b)
        for (int a = 0; a < 3; ++a) g->basis[b][a] = (kind == 0) ? fcc[b][a] : bcc[b][a];
    g->V = (int64_t)Lx * Ly * Lz;
    g->N = g->V * g->B;
    return true;
}

// Site index -> half-unit position.
void site_position(const Geom& g, int64_t idx, int P[3]) {
    int64_t cx = idx % g.L[0];
    int64_t rest = idx / g.L[0];
    int64_t cy = rest % g.L[1];
    rest /= g.L[1];
    int64_t cz = rest % g.L[2];
    int64_t b = rest / g.L[2];
    P[0] = (int)(2 * cx) + g.basis[b][0];
    P[1] = (int)(2 * cy) + g.basis[b][1];
    P[2] = (int)(2 * cz) + g.basis[b][2];
}

int wrap(int x, int period) {
    int r = x % period;
    return r < 0 ? r + period : r;
}

// Half-unit position (any integers, taken modulo the period 2L) -> site index, or -1 if the
// point is not a lattice site.
int64_t site_index(const Geom& g, const int Pin[3]) {
    int P[3];
    for (int a = 0; a < 3; ++a) P[a] = wrap(Pin[a], 2 * g.L[a]);
    for (int b = 0; b < g.B; ++b) {
        bool match = true;
        for (int a = 0; a < 3; ++a)
            if ((P[a] & 1) != g.basis[b][a]) match = false;
        if (!match) continue;
        int64_t cx = P[0] >> 1, cy = P[1] >> 1, cz = P[2] >> 1;
        return (((int64_t)b * g.L[2] + cz) * g.L[1] + cy) * g.L[0] + cx;
    }
    return -1;
}

// Coordination shells by brute force: every lattice vector d (origin + d is a lattice site) with
// 0 < |d|^2 <= 16 half units^2, grouped by |d|^2 in ascending order.  Inside a shell the vectors
// are kept in lexicographic (dx, dy, dz) order.
struct Shells {
    int M;
    std::vector<int> Z;                    // coordination number per shell
    std::vector<int> r2;                   // squared length per shell, half units^2
    std::vector<std::vector<int>> vec;     // per shell: dx,dy,dz triples, flattened
};

bool make_shells(const Geom& g, int M, Shells* sh) {
    if (M < 1 || M > 5) return false;
    int origin[3] = {0, 0, 0};
    std::vector<int> lengths;
    std::vector<std::vector<int>> all;  // (r2, dx, dy, dz)
    for (int dx = -4; dx <= 4; ++dx)
        for (int dy = -4; dy <= 4; ++dy)
            for (int dz = -4; dz <= 4; ++dz) {
                int r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0 || r2 > 16) continue;
                // Is origin + d a lattice site?  Test the parity pattern against the basis.
                int P[3] = {origin[0] + dx, origin[1] + dy, origin[2] + dz};
                bool is_site = false;
                for (int b = 0; b < g.B; ++b) {
                    bool m = true;
                    for (int a = 0; a < 3; ++a)
                        if (((P[a] % 2 + 2) % 2) != g.basis[b][a]) m = false;
                    if (m) is_site = true;
                }
                if (!is_site) continue;
                all.push_back({r2, dx, dy, dz});
                lengths.push_back(r2);
            }
    std::sort(lengths.begin(), lengths.end());
    lengths.erase(std::unique(lengths.begin(), lengths.end()), lengths.end());
    if ((int)lengths.size() < M) return false;
    std::sort(all.begin(), all.end());  // by r2, then dx, dy, dz
    sh->M = M;
    sh->Z.assign(M, 0);
    sh->r2.assign(M, 0);
    sh->vec.assign(M, std::vector<int>());
    for (int k = 0; k < M; ++k) {
        sh->r2[k] = lengths[k];
        for (const auto& v : all)
            if (v[0] == lengths[k]) {
                sh->vec[k].push_back(v[1]);
                sh->vec[k].push_back(v[2]);
                sh->vec[k].push_back(v[3]);
                sh->Z[k] += 1;
            }
    }
    return true;
}

int64_t neighbour(const Geom& g, int64_t site, int dx, int dy, int dz) {
    int P[3];
    site_position(g, site, P);
    int Q[3] = {P[0] + dx, P[1] + dy, P[2] + dz};
    return site_index(g, Q);
}

// ----------------------------------------------------------------------------------------------
// Pair counts N_ij^(k) (Sec. 4.3): the number of ordered (site s, vector d in shell k) with
// type(s) = i and type(s + d) = j.  Row i therefore sums to N_i * Z_k.
// ----------------------------------------------------------------------------------------------
void full_counts(const Geom& g, const Shells& sh, int S, const uint8_t* types, int32_t* counts) {
    const int M = sh.M;
    std::memset(counts, 0, sizeof(int32_t) * M * S * S);
    for (int64_t s = 0; s < g.N; ++s) {
        int i = types[s];
        for (int k = 0; k < M; ++k)
            for (int v = 0; v < sh.Z[k]; ++v) {
                int64_t t = neighbour(g, s, sh.vec[k][3 * v], sh.vec[k][3 * v + 1], sh.vec[k][3 * v + 2]);
                int j = types[t];
                counts[(k * S + i) * S + j] += 1;
            }
    }
}

// ----------------------------------------------------------------------------------------------
// Objective (Sec. 4.4, Eq. fitness_function) with Eq. sro for alpha.
// ----------------------------------------------------------------------------------------------
struct Objective {
    int S, M;
    int64_t N;
    std::vector<double> Q;  // [M][S][S]  N / ((Z_k N_i) N_j)
    std::vector<double> t;  // [M][S][S]  target alpha
    std::vector<double> w;  // [M]
};

bool make_objective(const Geom& g, const Shells& sh, int S, const int64_t* n_per, const double* w,
                    const double* target, Objective* ob) {
    if (S < 2 || S > 8) return false;
    int64_t total = 0;
    for (int i = 0; i < S; ++i) {
        if (n_per[i] < 1) return false;  // alpha is undefined for an absent species
        total += n_per[i];
    }
    if (total != g.N) return false;
    ob->S = S;
    ob->M = sh.M;
    ob->N = g.N;
    ob->Q.assign(sh.M * S * S, 0.0);
    ob->t.assign(sh.M * S * S, 0.0);
    ob->w.assign(sh.M, 0.0);
    for (int k = 0; k < sh.M; ++k) {
        if (!std::isfinite(w[k]) || std::signbit(w[k])) return false;  // w_k >= +0
        ob->w[k] = w[k];
        for (int i = 0; i < S; ++i)
            for (int j = 0; j < S; ++j) {
                int e = (k * S + i) * S + j;
                if (!std::isfinite(target[e])) return false;
                ob->t[e] = target[e];
                double denom = ((double)sh.Z[k] * (double)n_per[i]) * (double)n_per[j];
                ob->Q[e] = (double)g.N / denom;
            }
    }
    return true;
}

// Error of one (k,i,j) entry for count n: e = (1 - n Q) - t.
double entry_error(const Objective& ob, int e, int64_t n) {
    double alpha = 1.0 - (double)n * ob.Q[e];
    return alpha - ob.t[e];
}

double entry_term(const Objective& ob, int e, int64_t n) {
    double err = entry_error(ob, e, n);
    int k = e / (ob.S * ob.S);
    return ob.w[k] * (err * err);
}

double objective_f2(const Objective& ob, const int32_t* counts) {
    double f2 = 0.0;
    for (int e = 0; e < ob.M * ob.S * ob.S; ++e) f2 = f2 + entry_term(ob, e, counts[e]);
    return f2;
}

// ----------------------------------------------------------------------------------------------
// Count change of one swap (Sec. 4.5).  For each shell k:
//   h_a[y] = #{ d in shell k : a + d != b and type(a + d) = y },  h_b likewise with a and b swapped,
//   g = h_b - h_a, and with A = type(a), B = type(b):
//   dN[i][j] = [i==A] g[j] - [i==B] g[j] + [j==A] g[i] - [j==B] g[i].
// Bonds between a and b keep the unordered pair {A, B} and so contribute nothing.
// Returns false for a null move (a == b or A == B), with dN all zero.
// ----------------------------------------------------------------------------------------------
bool swap_delta(const Geom& g, const Shells& sh, int S, const uint8_t* types, int64_t a, int64_t b,
                int32_t* dN) {
    const int M = sh.M;
    std::memset(dN, 0, sizeof(int32_t) * M * S * S);
    if (a == b) return false;
    int A = types[a], B = types[b];
    if (A == B) return false;
    std::vector<int> ha(S), hb(S), gv(S);
    for (int k = 0; k < M; ++k) {
        std::fill(ha.begin(), ha.end(), 0);
        std::fill(hb.begin(), hb.end(), 0);
        for (int v = 0; v < sh.Z[k]; ++v) {
            int dx = sh.vec[k][3 * v], dy = sh.vec[k][3 * v + 1], dz = sh.vec[k][3 * v + 2];
            int64_t na = neighbour(g, a, dx, dy, dz);
            if (na != b) ha[types[na]] += 1;
            int64_t nb = neighbour(g, b, dx, dy, dz);
            if (nb != a) hb[types[nb]] += 1;
        }
        for (int y = 0; y < S; ++y) gv[y] = hb[y] - ha[y];
        for (int i = 0; i < S; ++i)
            for (int j = 0; j < S; ++j) {
                int d = 0;
                if (i == A) d += gv[j];
                if (i == B) d -= gv[j];
                if (j == A) d += gv[i];
                if (j == B) d -= gv[i];
                dN[(k * S + i) * S + j] = d;
            }
    }
    return true;
}

// Swap key: the change of F^2 (Eq. fitness_function) caused by dN.  Per entry, with e' = e - dN Q,
//   w (e')^2 - w e^2 = dN (a dN + b),   a = w (Q Q),   b = -2 (w (Q e))      (exact algebra),
// summed over (k,i,j) in row-major order as a chain of fused multiply-adds:
//   D <- fma(dN, fma(a, dN, b), D).
// Entries with dN = 0 leave D unchanged bit for bit, so only rows and columns of the two swapped
// species contribute.
double swap_key(const Objective& ob, const int32_t* counts, const int32_t* dN) {
    double D = 0.0;
    for (int e = 0; e < ob.M * ob.S * ob.S; ++e) {
        int k = e / (ob.S * ob.S);
        double w = ob.w[k], Q = ob.Q[e];
        double err = entry_error(ob, e, counts[e]);
        double a = w * (Q * Q);
        double b = -2.0 * (w * (Q * err));
        double d = (double)dN[e];
        D = std::fma(d, std::fma(a, d, b), D);
    }
    return D;
}

bool eligible(double D, bool null_move, double threshold) {
    if (null_move) return false;
    if (D < 0.0) return true;
    return threshold > 0.0 && D <= threshold;
}

// Candidate pair of task k at step `step` (Alg. parallel_mc: each task swaps two random atoms).
void draw_pair(uint64_t seed, uint32_t chain, uint32_t step, uint32_t k, int64_t N, int64_t* a,
               int64_t* b) {
    uint32_t r[4];
    philox(seed, k, step, chain, 1u, r);
    *a = (int64_t)(((uint64_t)r[0] * (uint64_t)N) >> 32);
    *b = (int64_t)(((uint64_t)r[1] * (uint64_t)N) >> 32);
}

// Closed neighbourhood test: is v equal to u or a shell-1..M neighbour of u?
bool in_closed_neighbourhood(const Geom& g, const Shells& sh, int64_t u, int64_t v) {
    if (u == v) return true;
    for (int k = 0; k < sh.M; ++k)
        for (int n = 0; n < sh.Z[k]; ++n)
            if (neighbour(g, u, sh.vec[k][3 * n], sh.vec[k][3 * n + 1], sh.vec[k][3 * n + 2]) == v)
                return true;
    return false;
}

}  // namespace

// ================================================================================================
// C entry points (loaded with ctypes by the tests, the smoke check and the CPU baseline).
// ================================================================================================
extern "C" {

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    philox_raw(ctr, key, out);
}

// Shell table: Z[M], r2[M], vecs[sum Z][3] (int32).  Returns the total number of vectors, or -1.
int or_shells(int kind, int M, int32_t* Z, int32_t* r2, int32_t* vecs) {
    Geom g;
    Shells sh;
    if (!make_geom(kind, 2, 2, 2, &g) || !make_shells(g, M, &sh)) return -1;
    int total = 0;
    for (int k = 0; k < M; ++k) {
        Z[k] = sh.Z[k];
        r2[k] = sh.r2[k];
        for (int v = 0; v < sh.Z[k]; ++v) {
            vecs[3 * total + 0] = sh.vec[k][3 * v + 0];
            vecs[3 * total + 1] = sh.vec[k][3 * v + 1];
            vecs[3 * total + 2] = sh.vec[k][3 * v + 2];
            ++total;
        }
    }
    return total;
}

int64_t or_num_sites(int kind, int Lx, int Ly, int Lz) {
    Geom g;
    if (!make_geom(kind, Lx, Ly, Lz, &g)) return -1;
    return g.N;
}

// Positions of all sites in half units: pos[N][3].
int or_positions(int kind, int Lx, int Ly, int Lz, int32_t* pos) {
    Geom g;
    if (!make_geom(kind, Lx, Ly, Lz, &g)) return OR_EINVAL;
    for (int64_t s = 0; s < g.N; ++s) {
        int P[3];
        site_position(g, s, P);
        pos[3 * s] = P[0];
        pos[3 * s + 1] = P[1];
        pos[3 * s + 2] = P[2];
    }
    return OR_OK;
}

// Neighbour table nbr[N][sum Z] (site index of s + d for every shell vector, shell-major).
int or_neighbours(int kind, int Lx, int Ly, int Lz, int M, int64_t* nbr) {
    Geom g;
    Shells sh;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !make_shells(g, M, &sh)) return OR_EINVAL;
    int zt = 0;
    for (int k = 0; k < M; ++k) zt += sh.Z[k];
    for (int64_t s = 0; s < g.N; ++s) {
        int c = 0;
        for (int k = 0; k < M; ++k)
            for (int v = 0; v < sh.Z[k]; ++v)
                nbr[s * zt + (c++)] = neighbour(g, s, sh.vec[k][3 * v], sh.vec[k][3 * v + 1], sh.vec[k][3 * v + 2]);
    }
    return OR_OK;
}

// Initial configuration with exact composition (see the header for the ordering rule).
int or_init_config(int64_t N, int S, const int64_t* n_per, uint64_t seed, uint8_t* types) {
    if (N < 1 || S < 1 || S > 255) return OR_EINVAL;
    int64_t total = 0;
    for (int s = 0; s < S; ++s) {
        if (n_per[s] < 0) return OR_EINVAL;
        total += n_per[s];
    }
    if (total != N || N > (int64_t)0xFFFFFFFF) return OR_EINVAL;
    std::vector<std::pair<uint64_t, int64_t>> keyed((size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        uint32_t r[4];
        philox(seed, (uint32_t)i, 0u, 0u, 0u, r);
        keyed[(size_t)i] = {((uint64_t)r[0] << 32) | (uint64_t)i, i};
    }
    std::sort(keyed.begin(), keyed.end());
    int64_t rank = 0;
    for (int s = 0; s < S; ++s)
        for (int64_t c = 0; c < n_per[s]; ++c, ++rank) types[keyed[(size_t)rank].second] = (uint8_t)s;
    return OR_OK;
}

int or_counts(int kind, int Lx, int Ly, int Lz, int M, int S, const uint8_t* types, int32_t* counts) {
    Geom g;
    Shells sh;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !make_shells(g, M, &sh) || S < 1 || S > 255) return OR_EINVAL;
    for (int64_t s = 0; s < g.N; ++s)
        if (types[s] >= S) return OR_EINVAL;
    full_counts(g, sh, S, types, counts);
    return OR_OK;
}

// alpha[M][S][S] from counts (Eq. sro) and F^2 (Eq. fitness_function, squared).
int or_alpha_f2(int kind, int Lx, int Ly, int Lz, int M, int S, const int64_t* n_per, const double* w,
                const double* target, const int32_t* counts, double* alpha, double* f2) {
    Geom g;
    Shells sh;
    Objective ob;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !make_shells(g, M, &sh) ||
        !make_objective(g, sh, S, n_per, w, target, &ob))
        return OR_EINVAL;
    for (int e = 0; e < M * S * S; ++e) alpha[e] = 1.0 - (double)counts[e] * ob.Q[e];
    *f2 = objective_f2(ob, counts);
    return OR_OK;
}

// Delta of the counts and the key for a list of candidate pairs, all against the same state.
// pairs[K][2]; key[K]; dN[K][M][S][S] (may be null); null_out[K] (may be null).
int or_delta_swap(int kind, int Lx, int Ly, int Lz, int M, int S, const int64_t* n_per, const double* w,
                  const double* target, const uint8_t* types, const int32_t* counts, const int64_t* pairs,
                  int64_t K, double* key, int32_t* dN_out, uint8_t* null_out) {
    Geom g;
    Shells sh;
    Objective ob;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !make_shells(g, M, &sh) ||
        !make_objective(g, sh, S, n_per, w, target, &ob))
        return OR_EINVAL;
    std::vector<int32_t> dN(M * S * S);
    for (int64_t c = 0; c < K; ++c) {
        int64_t a = pairs[2 * c], b = pairs[2 * c + 1];
        if (a < 0 || a >= g.N || b < 0 || b >= g.N) return OR_EINVAL;
        bool moved = swap_delta(g, sh, S, types, a, b, dN.data());
        key[c] = moved ? swap_key(ob, counts, dN.data()) : 0.0;
        if (dN_out) std::memcpy(dN_out + c * M * S * S, dN.data(), sizeof(int32_t) * M * S * S);
        if (null_out) null_out[c] = moved ? 0 : 1;
    }
    return OR_OK;
}

// Candidate pairs drawn for steps [step0, step0 + n_steps) (K per step): pairs[n_steps*K][2].
int or_draw_pairs(int64_t N, uint64_t seed, uint32_t chain, uint32_t step0, int64_t n_steps, int K,
                  int64_t* pairs) {
    for (int64_t s = 0; s < n_steps; ++s)
        for (int k = 0; k < K; ++k) {
            int64_t a, b;
            draw_pair(seed, chain, (uint32_t)(step0 + s), (uint32_t)k, N, &a, &b);
            pairs[2 * (s * K + k)] = a;
            pairs[2 * (s * K + k) + 1] = b;
        }
    return OR_OK;
}

// Search parameters and result (Alg. parallel_mc, Sec. 4.6.4).
struct or_search_params {
    int32_t K;             // candidate swaps (tasks) per step
    int32_t accept_mode;   // 0 = best-of-K, 1 = non-overlapping multi-accept
    int64_t max_steps;     // step budget
    int32_t depth_limit;   // stop when the non-improving-step counter reaches this (0 = off)
    int32_t max_accept;    // multi-accept: at most this many swaps per step (0 = unlimited)
    double threshold;      // 0 = strict improvement only
    uint64_t seed;
    uint32_t chain;
    uint32_t step0;        // first step counter (resume)
    int32_t depth0;        // depth counter at entry (resume)
    int32_t group_size;    // multi-accept: candidate k belongs to group k / group_size (0 = one group)
    int32_t group_top;     // multi-accept: only the group_top best eligible of each group are walked (0 = all)
    int32_t check;         // 1 = full recount after every step, compared with the running counts
};

struct or_search_result {
    int64_t steps;     // steps executed
    int64_t trials;    // candidates scored = steps * K
    int64_t accepted;  // swaps applied
    int32_t depth;     // depth counter at exit
    int32_t status;    // 0 ok, 2 incremental counts disagreed with a full recount
    double f2;         // F^2 of the final state, canonical order
    double f;          // sqrt(F^2)
};

int or_search(int kind, int Lx, int Ly, int Lz, int M, int S, const int64_t* n_per, const double* w,
              const double* target, const or_search_params* p, uint8_t* types, int32_t* counts,
              or_search_result* res, int64_t* accepted_log /* [max 2*K*max_steps] or null */) {
    Geom g;
    Shells sh;
    Objective ob;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !make_shells(g, M, &sh) ||
        !make_objective(g, sh, S, n_per, w, target, &ob))
        return OR_EINVAL;
    if (p->K < 1 || p->max_steps < 0 || p->depth_limit < 0 || p->max_accept < 0 || p->group_size < 0 ||
        p->group_top < 0 ||
        (p->accept_mode != 0 && p->accept_mode != 1) || !(p->threshold >= 0.0))
        return OR_EINVAL;
    const int E = M * S * S;
    const int K = p->K;
    std::vector<int64_t> ca(K), cb(K);
    std::vector<double> D(K);
    std::vector<uint8_t> is_null(K);
    std::vector<int32_t> dN((size_t)K * E), dtmp(E), check_counts(E);
    int64_t steps = 0, accepted = 0, n_log = 0;
    int32_t depth = p->depth0;
    int32_t status = OR_OK;
    for (int64_t s = 0; s < p->max_steps; ++s) {
        uint32_t step = (uint32_t)(p->step0 + s);
        // Every task proposes one swap and scores it against the step-start state.
        for (int k = 0; k < K; ++k) {
            draw_pair(p->seed, p->chain, step, (uint32_t)k, g.N, &ca[k], &cb[k]);
            bool moved = swap_delta(g, sh, S, types, ca[k], cb[k], &dN[(size_t)k * E]);
            is_null[k] = moved ? 0 : 1;
            D[k] = moved ? swap_key(ob, counts, &dN[(size_t)k * E]) : 0.0;
        }
        int n_acc = 0;
        if (p->accept_mode == 0) {
            // Best of K: smallest D, smaller task index on ties.
            int best = 0;
            for (int k = 1; k < K; ++k)
                if (D[k] < D[best]) best = k;
            if (eligible(D[best], is_null[best], p->threshold)) {
                std::swap(types[ca[best]], types[cb[best]]);
                for (int e = 0; e < E; ++e) counts[e] += dN[(size_t)best * E + e];
                if (accepted_log) {
                    accepted_log[2 * n_log] = ca[best];
                    accepted_log[2 * n_log + 1] = cb[best];
                    ++n_log;
                }
                n_acc = 1;
            }
        } else {
            // Non-overlapping multi-accept in ascending (D, k).
            auto before = [&](int x, int y) {
                if (D[x] != D[y]) return D[x] < D[y];
                return x < y;
            };
            std::vector<int> order;
            for (int k = 0; k < K; ++k)
                if (eligible(D[k], is_null[k], p->threshold)) order.push_back(k);
            if (p->group_top > 0) {
                // Keep only the group_top best eligible candidates of each group.
                const int G = p->group_size > 0 ? p->group_size : K;
                std::vector<int> kept;
                for (int c : order) {
                    int better = 0;
                    for (int o : order)
                        if (o / G == c / G && before(o, c)) ++better;
                    if (better < p->group_top) kept.push_back(c);
                }
                order.swap(kept);
            }
            std::sort(order.begin(), order.end(), before);
            std::vector<int64_t> taken;  // sites swapped this step
            for (int c : order) {
                if (p->max_accept > 0 && n_acc >= p->max_accept) break;
                bool conflict = false;
                for (int64_t u : taken) {
                    if (in_closed_neighbourhood(g, sh, u, ca[c]) || in_closed_neighbourhood(g, sh, u, cb[c])) {
                        conflict = true;
                        break;
                    }
                }
                if (conflict) continue;
                // With no taken site near a or b, the step-start delta is still exact.
                swap_delta(g, sh, S, types, ca[c], cb[c], dtmp.data());
                for (int e = 0; e < E; ++e)
                    if (dtmp[e] != dN[(size_t)c * E + e]) status = OR_EMISMATCH;
                double Dc = swap_key(ob, counts, dtmp.data());
                if (!eligible(Dc, false, p->threshold)) continue;
                std::swap(types[ca[c]], types[cb[c]]);
                for (int e = 0; e < E; ++e) counts[e] += dtmp[e];
                taken.push_back(ca[c]);
                taken.push_back(cb[c]);
                if (accepted_log) {
                    accepted_log[2 * n_log] = ca[c];
                    accepted_log[2 * n_log + 1] = cb[c];
                    ++n_log;
                }
                ++n_acc;
            }
        }
        accepted += n_acc;
        depth = (n_acc > 0) ? 0 : depth + 1;
        ++steps;
        if (p->check) {
            full_counts(g, sh, S, types, check_counts.data());
            for (int e = 0; e < E; ++e)
                if (check_counts[e] != counts[e]) status = OR_EMISMATCH;
        }
        if (status != OR_OK) break;
        if (p->depth_limit > 0 && depth >= p->depth_limit) break;
    }
    res->steps = steps;
    res->trials = steps * (int64_t)K;
    res->accepted = accepted;
    res->depth = depth;
    res->status = status;
    res->f2 = objective_f2(ob, counts);
    res->f = std::sqrt(res->f2);
    return status;
}

// ------------------------------------------------------------------------------------------------
// External structure onto the lattice (Sec. 2.3, application workflow: a structure simulated by
// an external tool is analysed to give the target SRO).  Atom i at Cartesian position xyz[i]
// (cubic lattice constant a, the cell's origin at origin[]) goes to the lattice site nearest to
// it under periodic boundaries, found by comparing its minimum-image distance to every site.
// Reading: an atom farther than tol * a / 2 from its nearest site is off-lattice; a site taken by
// two atoms or by none, and a species outside 0..S-1, are errors.  report[4] = off-lattice atoms,
// sites taken more than once, empty sites, bad species; types[site] receives the species of the
// (last) atom at that site.
// ------------------------------------------------------------------------------------------------
int or_map_structure(int kind, int Lx, int Ly, int Lz, int S, int64_t n, const double* xyz, const uint8_t* species,
                     double a, const double* origin, double tol, uint8_t* types, int64_t* report) {
    Geom g;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !(a > 0.0) || !(tol >= 0.0) || n < 0) return OR_EINVAL;
    std::vector<int> taken((size_t)g.N, 0);
    for (int r = 0; r < 4; ++r) report[r] = 0;
    for (int64_t s = 0; s < g.N; ++s) types[s] = 0;
    const double half = 0.5 * a;
    for (int64_t i = 0; i < n; ++i) {
        int64_t best = -1;
        double best_d2 = 0.0;
        for (int64_t s = 0; s < g.N; ++s) {
            int P[3];
            site_position(g, s, P);
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double period = 2.0 * g.L[c];
                double d = (xyz[3 * i + c] - origin[c]) / half - (double)P[c];
                d -= period * std::floor(d / period + 0.5);  // minimum image
                d2 += d * d;
            }
            if (best < 0 || d2 < best_d2) {
                best = s;
                best_d2 = d2;
            }
        }
        if (best_d2 > tol * tol) {
            report[0] += 1;
            continue;
        }
        if (species[i] >= S) report[3] += 1;
        taken[(size_t)best] += 1;
        types[best] = species[i];
    }
    for (int64_t s = 0; s < g.N; ++s) {
        if (taken[(size_t)s] > 1) report[1] += 1;
        if (taken[(size_t)s] == 0) report[2] += 1;
    }
    return OR_OK;
}

// ------------------------------------------------------------------------------------------------
// Global search (Sec. 4.1, Alg. global_search).  Readings where the paper leaves a choice open:
//   * Each iteration ranks P solutions: the R solutions kept from the previous iteration (none in
//     the first) and P - R new ones, each a fresh random configuration ("random perturbation": the
//     paper generates new solutions at random in every iteration, the first one entirely so).
//   * Fitness of every solution = F^2 from a full recount; ranking = ascending (F^2, pool index),
//     the kept solutions occupying pool indices 0..R-1 in their rank order, fresh one j index R + j.
//   * The best P_ls solutions of the ranking ("top solutions") are each refined by the parallel
//     Monte Carlo search (Alg. parallel_mc) with T tasks, depth limit d and a step cap; refined
//     slot r of iteration g runs chain g * 65536 + r from step 0 and depth 0.
//   * The refined solutions are ranked by (F^2, slot); the worst fraction p_a = 1 - R / P_ls is
//     discarded and the best R are kept (R <= P_ls / 2: at most half of the refined set).
//   * Fresh solution j of iteration g starts from the initial configuration with the 64-bit seed
//     (r1 << 32) | r0 of Philox counter (j, g, 0, 4) under the search's key.
// The result is the last iteration's refined set, ranked best first.
// ------------------------------------------------------------------------------------------------
struct or_global_params {
    int32_t n_solutions;   // P: solutions ranked per iteration
    int32_t n_refine;      // P_ls: best-ranked solutions refined per iteration (<= P)
    int32_t n_keep;        // R: refined solutions kept for the next iteration (<= P_ls / 2)
    int32_t iterations;    // G
    int32_t tasks;         // T: candidate swaps per Monte Carlo step
    int32_t depth_limit;   // d: a refinement ends after d consecutive steps without an accepted swap
    int64_t max_steps;     // step cap of one refinement
    uint64_t seed;
    int32_t accept_mode;   // 0 best-of-T, 1 multi-accept
    int32_t check;         // 1 = full recount after every Monte Carlo step
};

// One record per (iteration, refined slot).
struct or_global_log {
    int32_t origin;     // pool index the slot was selected from (< R: kept solution of that rank)
    int32_t pad;
    double f2_in;       // F^2 before the refinement
    double f2_out;      // F^2 after it
    int64_t steps;      // Monte Carlo steps of the refinement
    int64_t accepted;   // swaps it accepted
};

// Seed of fresh solution j of iteration g.
uint64_t or_fresh_seed(uint64_t seed, uint32_t g, uint32_t j) {
    uint32_t r[4];
    philox(seed, j, g, 0u, 4u, r);
    return ((uint64_t)r[1] << 32) | (uint64_t)r[0];
}

// types_out[P_ls][N], counts_out[P_ls][M][S][S], f2_out[P_ls]: the final refined set, best first.
// log[G][P_ls] (may be null).  totals[3] = Monte Carlo steps, trials and accepted swaps summed over
// every refinement (may be null).
int or_global_search(int kind, int Lx, int Ly, int Lz, int M, int S, const int64_t* n_per, const double* w,
                     const double* target, const or_global_params* gp, uint8_t* types_out, int32_t* counts_out,
                     double* f2_out, or_global_log* log, int64_t* totals) {
    Geom geo;
    Shells sh;
    Objective ob;
    if (!make_geom(kind, Lx, Ly, Lz, &geo) || !make_shells(geo, M, &sh) ||
        !make_objective(geo, sh, S, n_per, w, target, &ob))
        return OR_EINVAL;
    const int P = gp->n_solutions, PL = gp->n_refine, R = gp->n_keep, G = gp->iterations;
    if (P < 1 || PL < 1 || PL > P || R < 0 || 2 * R > PL || G < 1 || G > 65536 || PL > 65536 ||
        gp->tasks < 1 || gp->depth_limit < 1 || gp->max_steps < 1)
        return OR_EINVAL;
    const int64_t N = geo.N;
    const int E = M * S * S;
    struct Solution {
        std::vector<uint8_t> types;
        std::vector<int32_t> counts;
        double f2;
    };
    std::vector<Solution> kept;  // the R best refined solutions of the previous iteration, best first
    std::vector<Solution> refined;
    int64_t steps = 0, trials = 0, accepted = 0;
    for (int it = 0; it < G; ++it) {
        // New solutions: fresh random configurations after the kept ones.
        std::vector<Solution> pool = kept;
        const int n_kept = (int)kept.size();
        for (int j = 0; j < P - n_kept; ++j) {
            Solution x;
            x.types.resize((size_t)N);
            int rc = or_init_config(N, S, n_per, or_fresh_seed(gp->seed, (uint32_t)it, (uint32_t)j), x.types.data());
            if (rc != OR_OK) return rc;
            pool.push_back(std::move(x));
        }
        // Fitness of every solution from a full recount.
        for (int i = n_kept; i < P; ++i) {
            pool[i].counts.assign(E, 0);
            full_counts(geo, sh, S, pool[i].types.data(), pool[i].counts.data());
            pool[i].f2 = objective_f2(ob, pool[i].counts.data());
        }
        // Top solutions: the P_ls best by (F^2, pool index).
        std::vector<int> order(P);
        for (int i = 0; i < P; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pool[a].f2 < pool[b].f2; });
        refined.clear();
        for (int r = 0; r < PL; ++r) refined.push_back(pool[order[r]]);
        // Local search on each top solution.
        for (int r = 0; r < PL; ++r) {
            or_search_params sp{};
            sp.K = gp->tasks;
            sp.accept_mode = gp->accept_mode;
            sp.max_steps = gp->max_steps;
            sp.depth_limit = gp->depth_limit;
            sp.seed = gp->seed;
            sp.chain = (uint32_t)it * 65536u + (uint32_t)r;
            sp.check = gp->check;
            or_search_result res{};
            const double f2_in = refined[r].f2;
            int rc = or_search(kind, Lx, Ly, Lz, M, S, n_per, w, target, &sp, refined[r].types.data(),
                               refined[r].counts.data(), &res, nullptr);
            if (rc != OR_OK) return rc;
            refined[r].f2 = res.f2;
            steps += res.steps;
            trials += res.trials;
            accepted += res.accepted;
            if (log) {
                or_global_log& L = log[(size_t)it * PL + r];
                L.origin = order[r];
                L.pad = 0;
                L.f2_in = f2_in;
                L.f2_out = res.f2;
                L.steps = res.steps;
                L.accepted = res.accepted;
            }
        }
        // Rank the refined solutions; discard the worst fraction, keep the best R.
        std::vector<int> rank(PL);
        for (int r = 0; r < PL; ++r) rank[r] = r;
        std::stable_sort(rank.begin(), rank.end(), [&](int a, int b) { return refined[a].f2 < refined[b].f2; });
        std::vector<Solution> ranked;
        for (int r = 0; r < PL; ++r) ranked.push_back(refined[rank[r]]);
        refined.swap(ranked);
        kept.assign(refined.begin(), refined.begin() + R);
    }
    for (int r = 0; r < PL; ++r) {
        std::memcpy(types_out + (size_t)r * N, refined[r].types.data(), (size_t)N);
        std::memcpy(counts_out + (size_t)r * E, refined[r].counts.data(), sizeof(int32_t) * E);
        f2_out[r] = refined[r].f2;
    }
    if (totals) {
        totals[0] = steps;
        totals[1] = trials;
        totals[2] = accepted;
    }
    return OR_OK;
}

// ------------------------------------------------------------------------------------------------
// Annealed target recipe (an input generator, not part of the searched method): Metropolis swaps
// on a cell with symmetric shell-1 pair energies eps_ij ~ U[-0.05, 0.05] eV (rounded to 2^-30 eV so
// that every energy change below is exact in doubles), temperature T, `sweeps` x N attempts.
// Energy E = sum over unordered shell-1 bonds of eps = 1/2 sum_ij N_ij^(1) eps_ij.  A move is taken
// if dE <= 0 or u < exp(-dE / (k_B T)).  Writes the final configuration, eps[S][S] and
// alpha[M_out][S][S] of the final configuration.
// ------------------------------------------------------------------------------------------------
int or_anneal(int kind, int Lx, int Ly, int Lz, int S, const int64_t* n_per, uint64_t seed, double T,
              int sweeps, int M_out, uint8_t* types, double* eps, double* alpha_out, int64_t* n_taken) {
    Geom g;
    Shells sh1, shm;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !make_shells(g, 1, &sh1) || !make_shells(g, M_out, &shm))
        return OR_EINVAL;
    if (S < 2 || S > 8 || sweeps < 0 || !(T > 0.0)) return OR_EINVAL;
    int rc = or_init_config(g.N, S, n_per, seed, types);
    if (rc != OR_OK) return rc;
    for (int i = 0; i < S; ++i)
        for (int j = i; j < S; ++j) {
            uint32_t r[4];
            philox(seed, (uint32_t)(i * S + j), 0u, 0u, 2u, r);
            double u = (double)r[0] / 4294967296.0;
            double v = -0.05 + 0.1 * u;
            v = std::nearbyint(v * 1073741824.0) / 1073741824.0;  // multiple of 2^-30 eV
            eps[i * S + j] = v;
            eps[j * S + i] = v;
        }
    const double kB = 8.617333262e-5;  // eV / K
    std::vector<int32_t> dN(S * S);
    int64_t taken = 0;
    const int64_t attempts = (int64_t)sweeps * g.N;
    for (int64_t t = 0; t < attempts; ++t) {
        uint32_t r[4];
        philox(seed, (uint32_t)(t & 0xFFFFFFFFu), (uint32_t)(t >> 32), 0u, 3u, r);
        int64_t a = (int64_t)(((uint64_t)r[0] * (uint64_t)g.N) >> 32);
        int64_t b = (int64_t)(((uint64_t)r[1] * (uint64_t)g.N) >> 32);
        if (!swap_delta(g, sh1, S, types, a, b, dN.data())) continue;
        double dE = 0.0;
        for (int i = 0; i < S; ++i)
            for (int j = 0; j < S; ++j) dE += 0.5 * (double)dN[i * S + j] * eps[i * S + j];
        double u = (double)r[2] / 4294967296.0;
        if (dE <= 0.0 || u < std::exp(-dE / (kB * T))) {
            std::swap(types[a], types[b]);
            ++taken;
        }
    }
    if (n_taken) *n_taken = taken;
    std::vector<int32_t> counts(M_out * S * S);
    full_counts(g, shm, S, types, counts.data());
    for (int k = 0; k < M_out; ++k)
        for (int i = 0; i < S; ++i)
            for (int j = 0; j < S; ++j) {
                int e = (k * S + i) * S + j;
                double denom = ((double)shm.Z[k] * (double)n_per[i]) * (double)n_per[j];
                alpha_out[e] = 1.0 - (double)counts[e] * ((double)g.N / denom);
            }
    return OR_OK;
}

// Total shell-1 energy 1/2 sum_ij N_ij eps_ij from a full recount (used to pin the annealer).
double or_energy(int kind, int Lx, int Ly, int Lz, int S, const uint8_t* types, const double* eps) {
    Geom g;
    Shells sh;
    if (!make_geom(kind, Lx, Ly, Lz, &g) || !make_shells(g, 1, &sh)) return NAN;
    std::vector<int32_t> counts(S * S);
    full_counts(g, sh, S, types, counts.data());
    double E = 0.0;
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) E += 0.5 * (double)counts[i * S + j] * eps[i * S + j];
    return E;
}

}  // extern "C"
