// Decoupled aggregation on the device (Alg. 4, "ParallelAggregation"): the
// rows of a level split into consecutive tiles; one GPU thread per tile runs
// the sequential Algorithm 1 (with Algorithms 2 and 3, the singleton merge
// and the phase for isolated vertices, Sec. 2.1) on the tile's induced
// submatrix, with the strength of connection of Eq. (symmetric_strong1/2)
// computed on that submatrix.  It reproduces, step for step and tie for tie,
// the host implementation in host_setup.cpp applied to each tile (the readings
// of the paper's open points are documented there), so the map equals
// aggregate_tiled's:
//   * the global minimum of N_na (lowest index among ties) is found by a scan
//     of the tile instead of bucket queues;
//   * set membership uses stamp arrays, distances inside the growing
//     aggregate an all-pairs table updated per added vertex, as on the host.
// All state lives in global scratch indexed by the global row (each tile
// touches only its own rows), so tiles need no synchronisation.

#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "device.h"

namespace amg {

namespace {

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
    // a, dist, na, cand (w, c2, c1), dws, dw, best_dw
    return (size_t)maxa + (size_t)maxa * maxa + maxna + 3 * (size_t)maxna + (size_t)maxna * maxa +
           2 * (size_t)maxa;
}

__device__ inline double edge_w(double a) { return a < 0.0 ? -a : 0.0; }

// One tile's aggregation; the member functions follow the host Aggregation
// class line for line.
class TileAgg {
public:
    __device__ TileAgg(const int32_t* rp, const int32_t* ci, const double* va, int32_t t0,
                       int32_t t1, const TileScratch& S, const TileParams& P, int32_t tile)
        : rp_(rp), ci_(ci), va_(va), t0_(t0), t1_(t1), S_(S), P_(P) {
        int32_t* m = S.tile_mem + (size_t)tile * tile_ints(S.maxa, S.maxna);
        maxa_ = S.maxa;
        maxna_ = S.maxna;
        a_ = m;
        m += maxa_;
        dist_ = m;
        m += (size_t)maxa_ * maxa_;
        na_ = m;
        m += maxna_;
        cw_ = m;
        m += maxna_;
        cc2_ = m;
        m += maxna_;
        cc1_ = m;
        m += maxna_;
        dws_ = m;
        m += (size_t)maxna_ * maxa_;
        dw_ = m;
        m += maxa_;
        best_dw_ = m;
    }

    __device__ void strength() {
        // diagonal, intra-tile degree, then the couplings, eta_max and the
        // strong flags (the same expressions as the host)
        for (int32_t i = t0_; i < t1_; ++i) {
            int32_t d = 0;
            for (int32_t k = rp_[i]; k < rp_[i + 1]; ++k) {
                const int32_t j = ci_[k];
                if (!in_tile(j)) continue;
                if (j == i) S_.diag[i] = va_[k];
                else ++d;
            }
            S_.deg[i] = d;
        }
        for (int32_t i = t0_; i < t1_; ++i) {
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
                const double wji = t >= 0 ? edge_w(va_[t]) : 0.0;
                const double c = (edge_w(va_[k]) * wji) / (S_.diag[i] * S_.diag[j]);
                m = c > m ? c : m;
            }
            S_.eta[i] = m;
            S_.isolated[i] = m < P_.beta;
            S_.dirichlet[i] = !nonzero;
        }
        for (int32_t i = t0_; i < t1_; ++i)
            for (int32_t k = rp_[i]; k < rp_[i + 1]; ++k) {
                const int32_t j = ci_[k];
                if (j == i || !in_tile(j)) continue;
                const int32_t t = S_.tpos[k];
                const double wji = t >= 0 ? edge_w(va_[t]) : 0.0;
                const double c = (edge_w(va_[k]) * wji) / (S_.diag[i] * S_.diag[j]);
                const double e = fmin(S_.eta[i], S_.eta[j]);
                S_.strong[k] = (c > 0.0 && c > P_.delta * e) ? 1 : 0;
            }
    }

    __device__ void run(int32_t tile) {
        const int32_t n = t1_ - t0_;
        int32_t n_iso = 0, n_dir = 0;
        for (int32_t v = t0_; v < t1_; ++v) {
            S_.agg[v] = -1;
            S_.in_a[v] = 0;
            S_.in_na[v] = 0;
            S_.adj[v] = 0;
            S_.pos[v] = 0;
            S_.inU[v] = (!S_.isolated[v] && !S_.dirichlet[v]) ? 1 : 0;
            n_iso += S_.isolated[v] && !S_.dirichlet[v];
            n_dir += S_.dirichlet[v];
        }
        remaining_ = 0;
        for (int32_t v = t0_; v < t1_; ++v) {
            if (!S_.inU[v]) continue;
            int32_t c = 0;
            for (int32_t k = rp_[v]; k < rp_[v + 1]; ++k) {
                const int32_t j = ci_[k];
                if (j != v && in_tile(j) && S_.inU[j]) ++c;
            }
            S_.nna[v] = c;
            ++remaining_;
        }
        next_id_ = 0;
        if (remaining_ > 0) {
            int32_t v = global_min();
            while (true) {
                start_aggregate(v);
                remove_from_U(v);
                grow();
                round_aggregate();
                if (a_size_ == 1) {
                    int32_t target = -1;
                    double best_s = -1.0;
                    for (int32_t k = rp_[v]; k < rp_[v + 1]; ++k) {
                        const int32_t u = ci_[k];
                        if (u == v || !in_tile(u) || !S_.strong[k] || S_.agg[u] < 0) continue;
                        const int32_t t = S_.tpos[k];
                        const double wuv = t >= 0 ? edge_w(va_[t]) : 0.0;
                        const double s = (edge_w(va_[k]) * wuv) / (S_.diag[v] * S_.diag[u]);
                        if (s > best_s || (s == best_s && S_.agg[u] < target)) {
                            best_s = s;
                            target = S_.agg[u];
                        }
                    }
                    if (target >= 0) {
                        S_.agg[v] = target;
                        ++S_.size_of[t0_ + target];
                    } else {
                        S_.agg[v] = next_id_;
                        S_.size_of[t0_ + next_id_] = 1;
                        ++next_id_;
                    }
                } else {
                    for (int32_t q = 0; q < a_size_; ++q) S_.agg[a_[q]] = next_id_;
                    S_.size_of[t0_ + next_id_] = a_size_;
                    ++next_id_;
                }
                if (remaining_ == 0) break;
                build_na();
                int32_t seed = -1;
                for (int32_t q = 0; q < na_size_; ++q) {
                    const int32_t y = na_[q];
                    if (S_.inU[y] &&
                        (seed < 0 || S_.nna[y] < S_.nna[seed] || (S_.nna[y] == S_.nna[seed] && y < seed)))
                        seed = y;
                }
                v = seed >= 0 ? seed : global_min();
            }
        }
        const int32_t n_phase1 = next_id_;
        for (int32_t v = t0_; v < t1_; ++v) {
            if (!S_.isolated[v] || S_.dirichlet[v] || S_.agg[v] >= 0) continue;
            start_aggregate(v);
            S_.agg[v] = -2;
            grow_iso(n_phase1);
            for (int32_t q = 0; q < a_size_; ++q) S_.agg[a_[q]] = next_id_;
            S_.size_of[t0_ + next_id_] = a_size_;
            ++next_id_;
        }
        int32_t ms = 0;
        for (int32_t q = 0; q < next_id_; ++q) ms = max(ms, S_.size_of[t0_ + q]);
        S_.n_agg[tile] = next_id_;
        S_.max_size[tile] = ms;
        S_.n_isolated[tile] = n_iso;
        S_.n_dirichlet[tile] = n_dir;
        (void)n;
    }

private:
    const int32_t* rp_;
    const int32_t* ci_;
    const double* va_;
    const int32_t t0_, t1_;
    const TileScratch& S_;
    const TileParams& P_;
    int32_t maxa_, maxna_;
    int32_t *a_, *dist_, *na_, *cw_, *cc2_, *cc1_, *dws_, *dw_, *best_dw_;
    int32_t a_size_ = 0, na_size_ = 0, next_id_ = 0;
    int64_t remaining_ = 0;
    uint32_t stamp_a_ = 0, stamp_na_ = 0, stamp_adj_ = 0;

    __device__ bool in_tile(int32_t j) const { return j >= t0_ && j < t1_; }

    __device__ void remove_from_U(int32_t v) {
        S_.inU[v] = 0;
        --remaining_;
        for (int32_t k = rp_[v]; k < rp_[v + 1]; ++k) {
            const int32_t j = ci_[k];
            if (j == v || !in_tile(j) || !S_.inU[j]) continue;
            --S_.nna[j];
        }
    }

    // the vertex of U with minimal N_na, lowest index among ties
    __device__ int32_t global_min() const {
        int32_t best = -1;
        for (int32_t v = t0_; v < t1_; ++v)
            if (S_.inU[v] && (best < 0 || S_.nna[v] < S_.nna[best])) best = v;
        return best;
    }

    __device__ bool in_a(int32_t v) const { return S_.in_a[v] == stamp_a_; }

    __device__ void start_aggregate(int32_t v) {
        ++stamp_a_;
        a_size_ = 0;
        add_member_plain(v);
        dist_[0] = 0;
    }
    __device__ void add_member_plain(int32_t v) {
        S_.in_a[v] = stamp_a_;
        S_.pos[v] = a_size_;
        a_[a_size_++] = v;
    }

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

    __device__ void add_member_dist(int32_t w, const int32_t* dw) {
        const int32_t m = a_size_;
        for (int32_t x = 0; x < m; ++x)
            for (int32_t y = 0; y < m; ++y) {
                const int32_t via = dw[x] + dw[y];
                int32_t& d = dist_[(size_t)x * maxa_ + y];
                if (via < d) d = via;
            }
        for (int32_t t = 0; t < m; ++t) {
            dist_[(size_t)m * maxa_ + t] = dw[t];
            dist_[(size_t)t * maxa_ + m] = dw[t];
        }
        dist_[(size_t)m * maxa_ + m] = 0;
        add_member_plain(w);
    }

    __device__ void build_na() {
        ++stamp_na_;
        na_size_ = 0;
        for (int32_t q = 0; q < a_size_; ++q) {
            const int32_t x = a_[q];
            for (int32_t k = rp_[x]; k < rp_[x + 1]; ++k) {
                const int32_t j = ci_[k];
                if (j == x || !in_tile(j) || in_a(j) || S_.in_na[j] == stamp_na_) continue;
                S_.in_na[j] = stamp_na_;
                na_[na_size_++] = j;
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

    __device__ void grow() {
        while (a_size_ < P_.s_min) {
            build_na();
            ++stamp_adj_;
            for (int32_t q = 0; q < na_size_; ++q) {
                const int32_t y = na_[q];
                if (S_.agg[y] >= 0) S_.adj[t0_ + S_.agg[y]] = stamp_adj_;
            }
            int32_t nc = 0;
            const int32_t m = a_size_;
            int32_t max_c2 = 0;
            for (int32_t q = 0; q < na_size_; ++q) {
                const int32_t w = na_[q];
                if (!S_.inU[w]) continue;
                int32_t c2, c1;
                cons(w, c2, c1);
                if (c2 + c1 <= 0) continue;
                if (!ecc_within(w, dw_)) continue;
                cw_[nc] = w;
                cc2_[nc] = c2;
                cc1_[nc] = c1;
                for (int32_t t = 0; t < m; ++t) dws_[(size_t)nc * maxa_ + t] = dw_[t];
                ++nc;
                max_c2 = max(max_c2, c2);
            }
            if (nc == 0) break;
            int32_t best = -1;
            int64_t b_key1 = 0, b_conn = 0, b_deg = 1, b_nb = 0;
            for (int32_t q = 0; q < nc; ++q) {
                const int64_t key1 = max_c2 > 0 ? cc2_[q] : cc1_[q];
                if (best >= 0 && key1 < b_key1) continue;
                int64_t conn = 0, nb = 0;
                const int32_t w = cw_[q];
                for (int32_t k = rp_[w]; k < rp_[w + 1]; ++k) {
                    const int32_t u = ci_[k];
                    if (u == w || !in_tile(u) || in_a(u)) continue;
                    const int32_t g = S_.agg[u];
                    conn += (g >= 0 && S_.adj[t0_ + g] == stamp_adj_) ? 2 : 1;
                    if (S_.inU[u] && S_.in_na[u] != stamp_na_) ++nb;
                }
                const int64_t deg = S_.deg[w];
                bool better;
                if (best < 0 || key1 > b_key1) better = true;
                else if (conn * b_deg != b_conn * deg) better = conn * b_deg > b_conn * deg;
                else if (nb != b_nb) better = nb > b_nb;
                else better = w < cw_[best];
                if (better) {
                    best = q;
                    b_key1 = key1;
                    b_conn = conn;
                    b_deg = deg;
                    b_nb = nb;
                }
            }
            const int32_t c = cw_[best];
            add_member_dist(c, &dws_[(size_t)best * maxa_]);
            remove_from_U(c);
        }
    }

    __device__ void round_aggregate() {
        while (a_size_ < P_.s_max) {
            build_na();
            int32_t chosen = INT_MAX;
            for (int32_t q = 0; q < na_size_; ++q) {
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
            if (chosen == INT_MAX) break;
            add_member_plain(chosen);
            remove_from_U(chosen);
        }
    }

    __device__ void grow_iso(int32_t n_phase1) {
        while (a_size_ < P_.s_min) {
            build_na();
            ++stamp_adj_;
            for (int32_t q = 0; q < na_size_; ++q) {
                const int32_t y = na_[q];
                const int32_t g = S_.agg[y];
                if (g >= 0 && g < n_phase1) S_.adj[t0_ + g] = stamp_adj_;
            }
            int32_t chosen = INT_MAX;
            const int32_t m = a_size_;
            for (int32_t q = 0; q < na_size_; ++q) {
                const int32_t w = na_[q];
                if (w >= chosen) continue;
                if (!S_.isolated[w] || S_.dirichlet[w] || S_.agg[w] != -1) continue;
                if (!ecc_within(w, dw_)) continue;
                bool shares = false;
                for (int32_t k = rp_[w]; k < rp_[w + 1] && !shares; ++k) {
                    const int32_t y = ci_[k];
                    if (y == w || !in_tile(y)) continue;
                    const int32_t g = S_.agg[y];
                    if (g >= 0 && g < n_phase1 && S_.adj[t0_ + g] == stamp_adj_) shares = true;
                }
                if (!shares) continue;
                chosen = w;
                for (int32_t t = 0; t < m; ++t) best_dw_[t] = dw_[t];
            }
            if (chosen == INT_MAX) break;
            add_member_dist(chosen, best_dw_);
            S_.agg[chosen] = -2;
        }
    }
};

constexpr int kTileWarps = 4;   // tiles per block: lane 0 of each warp runs one

__global__ void __launch_bounds__(32 * kTileWarps)
k_aggregate_tiles(int32_t n, int32_t tile, int32_t ntiles, const int32_t* __restrict__ rp,
                  const int32_t* __restrict__ ci, const double* __restrict__ va, TileScratch S,
                  TileParams P) {
    const int32_t t = blockIdx.x * kTileWarps + (int32_t)(threadIdx.x >> 5);
    if ((threadIdx.x & 31) != 0 || t >= ntiles) return;
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
    S.maxa = std::max(p.s_max, p.s_min) + 2;
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
    const int32_t blocks = (ntiles + kTileWarps - 1) / kTileWarps;
    k_aggregate_tiles<<<blocks, 32 * kTileWarps, 0, s>>>(n, tile, ntiles, A.rp, A.ci, A.va, S, P);
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
