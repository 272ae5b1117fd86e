// Decoupled aggregation on the device (Alg. 4, "ParallelAggregation"): the
// rows of a level split into consecutive tiles; one warp per tile runs the
// sequential Algorithm 1 (with Algorithms 2 and 3, the singleton merge and the
// phase for isolated vertices, Sec. 2.1) on the tile's induced submatrix, with
// the strength of connection of Eq. (symmetric_strong1/2) computed on that
// submatrix.  The algorithm's steps stay sequential; the 32 lanes share the
// work inside each step (rows of the tile, entries of a row, the candidates
// in N(a)), and every choice the sequential algorithm makes by scanning --
// the best candidate of Algorithm 2, the lowest-index vertex of Algorithm 3,
// the seed of minimal N_na with the lowest index -- is a minimum under a
// total order, so a warp reduction picks the same vertex.  The map equals the
// host's aggregate_tiled (the readings of the paper's open points are
// documented in host_setup.cpp):
//   * N(a) is collected member by member in the same order as on the host;
//   * set membership uses stamp arrays, distances inside the growing
//     aggregate an all-pairs table updated per added vertex, as on the host;
//   * the global minimum of N_na is a warp-wide scan of the tile instead of
//     bucket queues.
// All state lives in global scratch indexed by the global row (each tile
// touches only its own rows), so tiles need no synchronisation.

#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "device.h"

namespace amg {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct TileScratch {
    // per row (global index)
    double* diag;
    double* eta;
    int32_t* deg;
    uint8_t* isolated;
    uint8_t* dirichlet;
    uint8_t* inU;
    int32_t* nna;
    int32_t* agg;          // -1 unaggregated, -2 in the isolated aggregate being built, else local id
    uint32_t* in_a;
    uint32_t* in_na;
    uint32_t* adj;         // indexed by t0 + local aggregate id
    int32_t* pos;
    int32_t* size_of;      // indexed by t0 + local aggregate id
    // per entry (global index)
    uint8_t* strong;
    int32_t* tpos;
    // per tile
    int32_t* tile_mem;     // stride per tile: see tile_ints()
    int32_t maxa, maxna;
    // results per tile
    int32_t* n_agg;
    int32_t* max_size;
    int32_t* n_isolated;
    int32_t* n_dirichlet;
};

struct TileParams {
    double delta, beta;
    int32_t s_min, s_max, d_max;
};

__host__ __device__ inline size_t tile_ints(int32_t maxa, int32_t maxna) {
    // a, dist, then per entry of N(a): the vertex, cons_2, cons_1 and its
    // distances to the members
    return (size_t)maxa + (size_t)maxa * maxa + 3 * (size_t)maxna + (size_t)maxna * maxa;
}

__device__ inline double edge_w(double a) { return a < 0.0 ? -a : 0.0; }

__device__ inline unsigned long long warp_min_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(kFull, v, o);
        v = u < v ? u : v;
    }
    return v;
}

__device__ inline unsigned long long key2(int32_t hi, int32_t lo) {
    return ((unsigned long long)(uint32_t)hi << 32) | (uint32_t)lo;
}

// Candidate of Algorithm 2 with the keys it is ranked by.
struct Cand {
    int32_t key1, conn, deg, nb, w, q;   // q < 0: none
};

// true when A ranks before B: key1 desc, connect(v,a)/|N(v)| desc (exact
// cross-multiplication), neighbors(v,a) desc, index asc
__device__ inline bool ranks_before(const Cand& A, const Cand& B) {
    if (B.q < 0) return A.q >= 0;
    if (A.q < 0) return false;
    if (A.key1 != B.key1) return A.key1 > B.key1;
    const long long l = (long long)A.conn * B.deg, r = (long long)B.conn * A.deg;
    if (l != r) return l > r;
    if (A.nb != B.nb) return A.nb > B.nb;
    return A.w < B.w;
}

// One tile's aggregation, run by all 32 lanes of a warp.  Counters such as
// |a|, |N(a)|, |U| and the stamps are warp-uniform (every lane holds the same
// value); writes to shared state are followed by __syncwarp before any lane
// reads them.
class TileAgg {
public:
    __device__ TileAgg(const int32_t* rp, const int32_t* ci, const double* va, int32_t t0,
                       int32_t t1, const TileScratch& S, const TileParams& P, int32_t tile)
        : rp_(rp), ci_(ci), va_(va), t0_(t0), t1_(t1), S_(S), P_(P),
          lane_((int32_t)(threadIdx.x & 31)) {
        int32_t* m = S.tile_mem + (size_t)tile * tile_ints(S.maxa, S.maxna);
        maxa_ = S.maxa;
        a_ = m;
        m += maxa_;
        dist_ = m;
        m += (size_t)maxa_ * maxa_;
        na_ = m;
        m += S.maxna;
        cc2_ = m;
        m += S.maxna;
        cc1_ = m;
        m += S.maxna;
        dws_ = m;
    }

    // diagonal, intra-tile degree, then the couplings, eta_max and the strong
    // flags (the same expressions as the host), rows spread over the lanes
    __device__ void strength() {
        for (int32_t i = t0_ + lane_; i < t1_; i += 32) {
            int32_t d = 0;
            for (int32_t k = rp_[i]; k < rp_[i + 1]; ++k) {
                const int32_t j = ci_[k];
                if (!in_tile(j)) continue;
                if (j == i) S_.diag[i] = va_[k];
                else ++d;
            }
            S_.deg[i] = d;
        }
        __syncwarp();
        for (int32_t i = t0_ + lane_; i < t1_; i += 32) {
            double m = 0.0;
            bool nonzero = false;
            for (int32_t k = rp_[i]; k < rp_[i + 1]; ++k) {
                const int32_t j = ci_[k];
                if (j == i || !in_tile(j)) continue;
                if (va_[k] != 0.0) nonzero = true;
                // position of (j, i)
                int32_t lo = rp_[j], hi = rp_[j + 1];
                while (lo < hi) {
                    const int32_t mid = (lo + hi) >> 1;
                    if (ci_[mid] < i) lo = mid + 1;
                    else hi = mid;
                }
                const int32_t t = (lo < rp_[j + 1] && ci_[lo] == i) ? lo : -1;
                S_.tpos[k] = t;
                const double c = coupling(i, j, k);
                m = c > m ? c : m;
            }
            S_.eta[i] = m;
            S_.isolated[i] = m < P_.beta;
            S_.dirichlet[i] = !nonzero;
        }
        __syncwarp();
        for (int32_t i = t0_ + lane_; i < t1_; i += 32)
            for (int32_t k = rp_[i]; k < rp_[i + 1]; ++k) {
                const int32_t j = ci_[k];
                if (j == i || !in_tile(j)) continue;
                const double c = coupling(i, j, k);
                const double e = fmin(S_.eta[i], S_.eta[j]);
                S_.strong[k] = (c > 0.0 && c > P_.delta * e) ? 1 : 0;
            }
        __syncwarp();
    }

    __device__ void run(int32_t tile) {
        int32_t n_iso = 0, n_dir = 0;
        for (int32_t v = t0_ + lane_; v < t1_; v += 32) {
            S_.agg[v] = -1;
            S_.in_a[v] = 0;
            S_.in_na[v] = 0;
            S_.adj[v] = 0;
            S_.pos[v] = 0;
            S_.inU[v] = (!S_.isolated[v] && !S_.dirichlet[v]) ? 1 : 0;
            n_iso += S_.isolated[v] && !S_.dirichlet[v];
            n_dir += S_.dirichlet[v];
        }
        __syncwarp();
        int32_t cnt = 0;
        for (int32_t v = t0_ + lane_; v < t1_; v += 32) {
            if (!S_.inU[v]) continue;
            int32_t c = 0;
            for (int32_t k = rp_[v]; k < rp_[v + 1]; ++k) {
                const int32_t j = ci_[k];
                if (j != v && in_tile(j) && S_.inU[j]) ++c;
            }
            S_.nna[v] = c;
            ++cnt;
        }
        __syncwarp();
        remaining_ = __reduce_add_sync(kFull, (unsigned)cnt);
        next_id_ = 0;
        if (remaining_ > 0) {
            int32_t v = global_min();
            while (v >= 0) {   // |U| > 0 guarantees a vertex
                start_aggregate(v);
                remove_from_U(v);
                grow();
                round_aggregate();
                if (a_size_ == 1) {
                    merge_singleton(v);
                } else {
                    for (int32_t q = lane_; q < a_size_; q += 32) S_.agg[a_[q]] = next_id_;
                    if (lane_ == 0) S_.size_of[t0_ + next_id_] = a_size_;
                    ++next_id_;
                    __syncwarp();
                }
                if (remaining_ == 0) break;
                build_na();
                unsigned long long best = ~0ull;
                for (int32_t q = lane_; q < na_size_; q += 32) {
                    const int32_t y = na_[q];
                    if (S_.inU[y]) {
                        const unsigned long long k = key2(S_.nna[y], y);
                        best = k < best ? k : best;
                    }
                }
                best = warp_min_u64(best);
                v = best != ~0ull ? (int32_t)(uint32_t)best : global_min();
            }
        }
        const int32_t n_phase1 = next_id_;
        int32_t from = t0_;
        while (true) {
            const int32_t v = next_isolated(from);
            if (v < 0) break;
            start_aggregate(v);
            if (lane_ == 0) S_.agg[v] = -2;
            __syncwarp();
            grow_iso(n_phase1);
            for (int32_t q = lane_; q < a_size_; q += 32) S_.agg[a_[q]] = next_id_;
            if (lane_ == 0) S_.size_of[t0_ + next_id_] = a_size_;
            ++next_id_;
            __syncwarp();
            from = v + 1;
        }
        int32_t ms = 0;
        for (int32_t q = lane_; q < next_id_; q += 32) ms = max(ms, S_.size_of[t0_ + q]);
        ms = (int32_t)__reduce_max_sync(kFull, (unsigned)ms);
        n_iso = (int32_t)__reduce_add_sync(kFull, (unsigned)n_iso);
        n_dir = (int32_t)__reduce_add_sync(kFull, (unsigned)n_dir);
        if (lane_ == 0) {
            S_.n_agg[tile] = next_id_;
            S_.max_size[tile] = ms;
            S_.n_isolated[tile] = n_iso;
            S_.n_dirichlet[tile] = n_dir;
        }
    }

private:
    const int32_t* rp_;
    const int32_t* ci_;
    const double* va_;
    const int32_t t0_, t1_;
    const TileScratch& S_;
    const TileParams& P_;
    const int32_t lane_;
    int32_t maxa_;
    int32_t *a_, *dist_, *na_, *cc2_, *cc1_, *dws_;
    int32_t a_size_ = 0, na_size_ = 0, next_id_ = 0;
    int32_t remaining_ = 0;
    uint32_t stamp_a_ = 0, stamp_na_ = 0, stamp_adj_ = 0;

    __device__ bool in_tile(int32_t j) const { return j >= t0_ && j < t1_; }
    __device__ bool in_a(int32_t v) const { return S_.in_a[v] == stamp_a_; }

    // the coupling of Eq. (symmetric_strong1) for entry k = (i, j)
    __device__ double coupling(int32_t i, int32_t j, int32_t k) const {
        const int32_t t = S_.tpos[k];
        const double wji = t >= 0 ? edge_w(va_[t]) : 0.0;
        return (edge_w(va_[k]) * wji) / (S_.diag[i] * S_.diag[j]);
    }

    __device__ void remove_from_U(int32_t v) {
        if (lane_ == 0) S_.inU[v] = 0;
        --remaining_;
        __syncwarp();
        for (int32_t k = rp_[v] + lane_; k < rp_[v + 1]; k += 32) {
            const int32_t j = ci_[k];
            if (j == v || !in_tile(j) || !S_.inU[j]) continue;
            --S_.nna[j];
        }
        __syncwarp();
    }

    // the vertex of U with minimal N_na, lowest index among ties
    __device__ int32_t global_min() const {
        unsigned long long best = ~0ull;
        for (int32_t v = t0_ + lane_; v < t1_; v += 32)
            if (S_.inU[v]) {
                const unsigned long long k = key2(S_.nna[v], v);
                best = k < best ? k : best;
            }
        best = warp_min_u64(best);
        return best != ~0ull ? (int32_t)(uint32_t)best : -1;
    }

    // first isolated, non-Dirichlet, unaggregated vertex at or after from
    __device__ int32_t next_isolated(int32_t from) const {
        for (int32_t base = from; base < t1_; base += 32) {
            const int32_t v = base + lane_;
            const bool ok = v < t1_ && S_.isolated[v] && !S_.dirichlet[v] && S_.agg[v] == -1;
            const unsigned m = __ballot_sync(kFull, ok);
            if (m) return base + __ffs(m) - 1;
        }
        return -1;
    }

    __device__ void start_aggregate(int32_t v) {
        ++stamp_a_;
        a_size_ = 0;
        if (lane_ == 0) dist_[0] = 0;
        add_member_plain(v);
    }
    __device__ void add_member_plain(int32_t v) {
        if (lane_ == 0) {
            S_.in_a[v] = stamp_a_;
            S_.pos[v] = a_size_;
            a_[a_size_] = v;
        }
        ++a_size_;
        __syncwarp();
    }

    // distances from w (not in a) to every member through edges into a;
    // false if some member is unreachable or farther than d_max (one lane)
    __device__ bool ecc_within(int32_t w, int32_t* dw) const {
        const int32_t m = a_size_;
        for (int32_t t = 0; t < m; ++t) dw[t] = INT_MAX / 2;
        for (int32_t k = rp_[w]; k < rp_[w + 1]; ++k) {
            const int32_t u = ci_[k];
            if (u == w || !in_tile(u) || !in_a(u)) continue;
            const int32_t* row = &dist_[(size_t)S_.pos[u] * maxa_];
            for (int32_t t = 0; t < m; ++t) dw[t] = min(dw[t], row[t] + 1);
        }
        for (int32_t t = 0; t < m; ++t)
            if (dw[t] > P_.d_max) return false;
        return true;
    }

    // append w whose distances to the members are dw; update all pairs
    __device__ void add_member_dist(int32_t w, const int32_t* dw) {
        const int32_t m = a_size_;
        for (int32_t idx = lane_; idx < m * m; idx += 32) {
            const int32_t x = idx / m, y = idx - x * m;
            const int32_t via = dw[x] + dw[y];
            int32_t& d = dist_[(size_t)x * maxa_ + y];
            if (via < d) d = via;
        }
        for (int32_t t = lane_; t < m; t += 32) {
            dist_[(size_t)m * maxa_ + t] = dw[t];
            dist_[(size_t)t * maxa_ + m] = dw[t];
        }
        if (lane_ == 0) dist_[(size_t)m * maxa_ + m] = 0;
        __syncwarp();
        add_member_plain(w);
    }

    // N(a) in the host's order: member by member, entries in column order
    __device__ void build_na() {
        ++stamp_na_;
        na_size_ = 0;
        for (int32_t q = 0; q < a_size_; ++q) {
            const int32_t x = a_[q];
            const int32_t e = rp_[x + 1];
            for (int32_t kb = rp_[x]; kb < e; kb += 32) {
                const int32_t k = kb + lane_;
                int32_t j = -1;
                bool take = false;
                if (k < e) {
                    j = ci_[k];
                    take = j != x && in_tile(j) && !in_a(j) && S_.in_na[j] != stamp_na_;
                }
                const unsigned m = __ballot_sync(kFull, take);
                if (take) {
                    S_.in_na[j] = stamp_na_;
                    na_[na_size_ + __popc(m & ((1u << lane_) - 1u))] = j;
                }
                na_size_ += __popc(m);
                __syncwarp();
            }
        }
    }

    __device__ void cons(int32_t w, int32_t& c2, int32_t& c1) const {
        c2 = 0;
        c1 = 0;
        for (int32_t k = rp_[w]; k < rp_[w + 1]; ++k) {
            const int32_t u = ci_[k];
            if (u == w || !in_tile(u) || !in_a(u)) continue;
            const bool s1 = S_.strong[k] != 0;
            const int32_t t = S_.tpos[k];
            const bool s2 = t >= 0 && S_.strong[t] != 0;
            if (s1 && s2) ++c2;
            else if (s1 != s2) ++c1;
        }
    }

    // mark the aggregates (ids below limit) adjacent to a through N(a)
    __device__ void mark_adjacent(int32_t limit) {
        ++stamp_adj_;
        for (int32_t q = lane_; q < na_size_; q += 32) {
            const int32_t g = S_.agg[na_[q]];
            if (g >= 0 && g < limit) S_.adj[t0_ + g] = stamp_adj_;
        }
        __syncwarp();
    }

    // Algorithm 2
    __device__ void grow() {
        while (a_size_ < P_.s_min) {
            build_na();
            mark_adjacent(INT_MAX);
            int32_t max_c2 = 0;
            bool any = false;
            for (int32_t q = lane_; q < na_size_; q += 32) {
                const int32_t w = na_[q];
                int32_t c2 = -1, c1 = 0;
                if (S_.inU[w]) {
                    cons(w, c2, c1);
                    if (c2 + c1 <= 0 || !ecc_within(w, &dws_[(size_t)q * maxa_])) c2 = -1;
                }
                cc2_[q] = c2;
                cc1_[q] = c1;
                if (c2 >= 0) {
                    any = true;
                    max_c2 = max(max_c2, c2);
                }
            }
            if (!__any_sync(kFull, any)) break;
            max_c2 = (int32_t)__reduce_max_sync(kFull, (unsigned)max_c2);
            Cand best{0, 0, 1, 0, 0, -1};
            for (int32_t q = lane_; q < na_size_; q += 32) {
                if (cc2_[q] < 0) continue;
                Cand c;
                c.key1 = max_c2 > 0 ? cc2_[q] : cc1_[q];
                if (best.q >= 0 && c.key1 < best.key1) continue;
                c.w = na_[q];
                c.q = q;
                c.deg = S_.deg[c.w];
                c.conn = 0;
                c.nb = 0;
                for (int32_t k = rp_[c.w]; k < rp_[c.w + 1]; ++k) {
                    const int32_t u = ci_[k];
                    if (u == c.w || !in_tile(u) || in_a(u)) continue;
                    const int32_t g = S_.agg[u];
                    c.conn += (g >= 0 && S_.adj[t0_ + g] == stamp_adj_) ? 2 : 1;
                    if (S_.inU[u] && S_.in_na[u] != stamp_na_) ++c.nb;
                }
                if (ranks_before(c, best)) best = c;
            }
            for (int o = 16; o > 0; o >>= 1) {
                Cand o_;
                o_.key1 = __shfl_xor_sync(kFull, best.key1, o);
                o_.conn = __shfl_xor_sync(kFull, best.conn, o);
                o_.deg = __shfl_xor_sync(kFull, best.deg, o);
                o_.nb = __shfl_xor_sync(kFull, best.nb, o);
                o_.w = __shfl_xor_sync(kFull, best.w, o);
                o_.q = __shfl_xor_sync(kFull, best.q, o);
                if (ranks_before(o_, best)) best = o_;
            }
            __syncwarp();
            add_member_dist(best.w, &dws_[(size_t)best.q * maxa_]);
            remove_from_U(best.w);
        }
    }

    // Algorithm 3
    __device__ void round_aggregate() {
        while (a_size_ < P_.s_max) {
            build_na();
            int32_t chosen = INT_MAX;
            for (int32_t q = lane_; q < na_size_; q += 32) {
                const int32_t w = na_[q];
                if (!S_.inU[w] || w >= chosen) continue;
                int32_t c2, c1;
                cons(w, c2, c1);
                if (c2 + c1 <= 0) continue;
                int32_t to_a = 0, to_u = 0;
                for (int32_t k = rp_[w]; k < rp_[w + 1]; ++k) {
                    const int32_t u = ci_[k];
                    if (u == w || !in_tile(u) || !S_.strong[k]) continue;
                    if (in_a(u)) ++to_a;
                    else if (S_.inU[u]) ++to_u;
                }
                if (to_a > to_u) chosen = w;
            }
            chosen = (int32_t)__reduce_min_sync(kFull, (unsigned)chosen);
            if (chosen == INT_MAX) break;
            add_member_plain(chosen);
            remove_from_U(chosen);
        }
    }

    // a one-vertex aggregate joins the aggregate of its strongest strong
    // neighbour (lowest aggregate index among ties), else stays alone
    __device__ void merge_singleton(int32_t v) {
        int32_t target = -1;
        double best_s = -1.0;
        for (int32_t k = rp_[v] + lane_; k < rp_[v + 1]; k += 32) {
            const int32_t u = ci_[k];
            if (u == v || !in_tile(u) || !S_.strong[k] || S_.agg[u] < 0) continue;
            const double s = coupling(v, u, k);
            if (s > best_s || (s == best_s && S_.agg[u] < target)) {
                best_s = s;
                target = S_.agg[u];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double os = __shfl_xor_sync(kFull, best_s, o);
            const int32_t ot = __shfl_xor_sync(kFull, target, o);
            if (ot >= 0 && (target < 0 || os > best_s || (os == best_s && ot < target))) {
                best_s = os;
                target = ot;
            }
        }
        if (target >= 0) {
            if (lane_ == 0) {
                S_.agg[v] = target;
                ++S_.size_of[t0_ + target];
            }
        } else {
            if (lane_ == 0) {
                S_.agg[v] = next_id_;
                S_.size_of[t0_ + next_id_] = 1;
            }
            ++next_id_;
        }
        __syncwarp();
    }

    // growth of an aggregate of isolated vertices (lowest index first)
    __device__ void grow_iso(int32_t n_phase1) {
        while (a_size_ < P_.s_min) {
            build_na();
            mark_adjacent(n_phase1);
            unsigned long long best = ~0ull;
            for (int32_t q = lane_; q < na_size_; q += 32) {
                const int32_t w = na_[q];
                if ((unsigned long long)(uint32_t)w << 32 >= best) continue;
                if (!S_.isolated[w] || S_.dirichlet[w] || S_.agg[w] != -1) continue;
                if (!ecc_within(w, &dws_[(size_t)q * maxa_])) continue;
                bool shares = false;
                for (int32_t k = rp_[w]; k < rp_[w + 1] && !shares; ++k) {
                    const int32_t y = ci_[k];
                    if (y == w || !in_tile(y)) continue;
                    const int32_t g = S_.agg[y];
                    if (g >= 0 && g < n_phase1 && S_.adj[t0_ + g] == stamp_adj_) shares = true;
                }
                if (!shares) continue;
                best = key2(w, q);
            }
            best = warp_min_u64(best);
            if (best == ~0ull) break;
            __syncwarp();
            const int32_t w = (int32_t)(best >> 32), q = (int32_t)(uint32_t)best;
            add_member_dist(w, &dws_[(size_t)q * maxa_]);
            if (lane_ == 0) S_.agg[w] = -2;
            __syncwarp();
        }
    }
};

__global__ void k_aggregate_tiles(int32_t n, int32_t tile, int32_t ntiles, const int32_t* __restrict__ rp,
                                  const int32_t* __restrict__ ci, const double* __restrict__ va,
                                  TileScratch S, TileParams P) {
    const int32_t t = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= ntiles) return;   // whole warps leave together
    const int32_t t0 = t * tile, t1 = min(n, t0 + tile);
    TileAgg G(rp, ci, va, t0, t1, S, P, t);
    G.strength();
    G.run(t);
}

}  // namespace

AggResult aggregate_tiles_device(const DevCsr& A, const amg_params& p, cudaStream_t s) {
    const int32_t n = A.n;
    const int32_t tile = p.aggregation_tile;
    const int32_t ntiles = (n + tile - 1) / tile;
    // longest row bounds |N(a)|
    std::vector<int32_t> rp(n + 1);
    AMG_CUDA_TRY(cudaMemcpyAsync(rp.data(), A.rp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t maxdeg = 0;
    for (int32_t i = 0; i < n; ++i) maxdeg = std::max(maxdeg, rp[i + 1] - rp[i]);
    DevArena mem(s);
    TileScratch S{};
    // an aggregate holds at most max(s_min, s_max) rows, and never more than a tile
    S.maxa = std::min(std::max(p.s_max, p.s_min), tile) + 2;
    // N(a) lies inside the tile and within the neighbourhoods of the members
    S.maxna = (int32_t)std::min<int64_t>((int64_t)S.maxa * std::max(1, maxdeg), tile);
    S.diag = mem.alloc<double>(n);
    S.deg = mem.alloc<int32_t>(n);
    S.isolated = mem.alloc<uint8_t>(n);
    S.dirichlet = mem.alloc<uint8_t>(n);
    S.inU = mem.alloc<uint8_t>(n);
    S.nna = mem.alloc<int32_t>(n);
    S.agg = mem.alloc<int32_t>(n);
    S.in_a = mem.alloc<uint32_t>(n);
    S.in_na = mem.alloc<uint32_t>(n);
    S.adj = mem.alloc<uint32_t>(n);
    S.pos = mem.alloc<int32_t>(n);
    S.eta = mem.alloc<double>(n);
    S.size_of = mem.alloc<int32_t>(n);
    S.strong = mem.alloc<uint8_t>(A.nnz);
    S.tpos = mem.alloc<int32_t>(A.nnz);
    S.tile_mem = mem.alloc<int32_t>(tile_ints(S.maxa, S.maxna) * ntiles);
    S.n_agg = mem.alloc<int32_t>(ntiles);
    S.max_size = mem.alloc<int32_t>(ntiles);
    S.n_isolated = mem.alloc<int32_t>(ntiles);
    S.n_dirichlet = mem.alloc<int32_t>(ntiles);
    TileParams P{p.delta, p.beta, p.s_min, p.s_max, p.d_max};
    // one warp per tile; one warp per block spreads a few hundred tiles over
    // all SMs, four per block when there are more tiles than resident blocks
    int dev = 0, sms = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int32_t wpb = ntiles > 32 * sms ? 4 : 1;
    const int32_t blocks = (ntiles + wpb - 1) / wpb;
    k_aggregate_tiles<<<blocks, 32 * wpb, 0, s>>>(n, tile, ntiles, A.rp, A.ci, A.va, S, P);
    AMG_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> agg(n), nagg(ntiles), mx(ntiles), niso(ntiles), ndir(ntiles);
    AMG_CUDA_TRY(cudaMemcpyAsync(agg.data(), S.agg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(nagg.data(), S.n_agg, sizeof(int32_t) * ntiles, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(mx.data(), S.max_size, sizeof(int32_t) * ntiles, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(niso.data(), S.n_isolated, sizeof(int32_t) * ntiles, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(ndir.data(), S.n_dirichlet, sizeof(int32_t) * ntiles, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    AggResult R;
    R.agg.assign(n, -1);
    for (int32_t t = 0; t < ntiles; ++t) {
        const int32_t t0 = t * tile, t1 = std::min(n, t0 + tile);
        for (int32_t i = t0; i < t1; ++i) R.agg[i] = agg[i] >= 0 ? R.nc + agg[i] : -1;
        R.nc += nagg[t];
        R.max_size = std::max(R.max_size, mx[t]);
        R.n_isolated += niso[t];
        R.n_dirichlet += ndir[t];
    }
    return R;
}

}  // namespace amg
