// Host setup of the hierarchy: strength of connection, greedy aggregation and
// multicolouring of one level (Sec. 2.1 of Blatt, Ippisch & Bastian,
// arXiv:1209.0960).
//
// The aggregation follows Algorithms 1-3 with these readings of the points the
// paper leaves open:
//   * w_E((i,j)) = max(0, -A_ij) (the printed 1/2 (A_ij - |A_ij|) has the wrong
//     sign; the text asks for the absolute value of negative entries);
//     w_V(i) = A_ii; the coupling of Eq. (symmetric_strong1) is
//     w_E(i,j) w_E(j,i) / (A_ii A_jj); a zero coupling is never strong.
//   * A Dirichlet vertex is a row without a non-zero off-diagonal; it is left
//     out of every aggregate.
//   * N_na(u) counts neighbours of u still in U (non-isolated, non-Dirichlet,
//     unaggregated).  Seeds: minimal N_na, lowest index; after an aggregate the
//     next seed comes from its unaggregated neighbours, else from all of U.
//   * Algorithm 2 grows while |a| < s_min over candidates in N(a) ∩ U that keep
//     the induced-subgraph diameter <= d_max and have a strong link to a; it
//     ranks them by cons_2 (cons_1 when no candidate has a two-way link), then
//     connect(v,a)/|N(v)| (exact rational comparison), then neighbors(v,a),
//     then the lowest index.
//   * Algorithm 3 rounds while |a| < s_max with the lowest-index neighbour in U
//     that has more strong links into a than to other vertices of U, and stops
//     when there is none.
//   * A one-vertex aggregate joins the earlier aggregate holding its strongest
//     strong neighbour (ties: lowest aggregate index) when there is one.
//   * Isolated vertices are visited in index order; each seeds an aggregate
//     that grows (lowest index first, up to s_min, diameter <= d_max) by
//     adjacent isolated vertices sharing a neighbouring aggregate of
//     non-isolated vertices with it.
//   * Coarse indices are numbered in the order the aggregates are completed.
//
// This implementation keeps incremental state so that it runs in near-linear
// time: bucket queues for the global N_na minimum, stamp arrays for set
// membership, all-pairs distances inside the growing aggregate for the
// diameter test, and N(a), the aggregates adjacent to it, cons_1 / cons_2 and
// the strong-link counts of Algorithm 3, all updated as members join.
//
// The smoother's colouring is the ascending-order greedy colouring, replaced
// by DSATUR when that needs fewer colours (smoother_colouring).

#include "host_setup.h"

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>
#include <functional>
#include <queue>
#include <atomic>
#include <thread>

namespace amg {

namespace {

// Matrices of at least this many rows run the per-row passes of validation
// and strength on several host threads.  Each row writes only its own results
// and errors are reported for the lowest failing row, so the outcome does not
// depend on the thread count.  (Smaller matrices, like the serving requests
// set up several at a time, stay on the calling thread.)
constexpr int32_t kParallelRows = 1 << 20;

// fn(lo, hi, chunk) over consecutive chunks of [0, n)
template <typename F>
int for_row_chunks(int32_t n, F fn) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int threads = n >= kParallelRows ? (int)std::min(16u, hw) : 1;
    const int32_t chunk = (int32_t)(((int64_t)n + threads - 1) / threads);
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) {
        const int32_t lo = (int32_t)std::min<int64_t>(n, (int64_t)t * chunk);
        const int32_t hi = (int32_t)std::min<int64_t>(n, (int64_t)lo + chunk);
        pool.emplace_back(fn, lo, hi, t);
    }
    fn(0, std::min(n, chunk), 0);
    for (auto& th : pool) th.join();
    return threads;
}

// the first failing row of each chunk and its message
struct RowError {
    int32_t row = INT32_MAX;
    std::string msg;
};
bool first_error(const std::vector<RowError>& e, std::string& err) {
    const RowError* best = nullptr;
    for (const RowError& x : e)
        if (x.row != INT32_MAX && (!best || x.row < best->row)) best = &x;
    if (!best) return false;
    err = best->msg;
    return true;
}

}  // namespace

bool validate_csr(const HostCsr& A, std::string& err) {
    const int32_t n = A.n;
    if (n <= 0) { err = "matrix has no rows"; return false; }
    if ((int64_t)A.rp.size() != (int64_t)n + 1 || A.rp[0] != 0) { err = "bad row_ptr"; return false; }
    for (int32_t i = 0; i < n; ++i)
        if (A.rp[i + 1] < A.rp[i]) { err = "row_ptr not monotone"; return false; }
    if ((int64_t)A.ci.size() != A.nnz() || (int64_t)A.va.size() != A.nnz()) {
        err = "col/val length differs from row_ptr[n]";
        return false;
    }
    std::vector<RowError> errs(16);
    for_row_chunks(n, [&](int32_t lo, int32_t hi, int t) {
        for (int32_t i = lo; i < hi; ++i) {
            bool has_diag = false;
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                int32_t j = A.ci[k];
                if (j < 0 || j >= n) {
                    errs[t] = {i, "column index out of range in row " + std::to_string(i)};
                    return;
                }
                if (k > A.rp[i] && A.ci[k - 1] >= j) {
                    errs[t] = {i, "columns not sorted/unique in row " + std::to_string(i)};
                    return;
                }
                if (j == i) {
                    has_diag = true;
                    if (!(A.va[k] > 0.0)) {
                        errs[t] = {i, "non-positive diagonal in row " + std::to_string(i)};
                        return;
                    }
                }
            }
            if (!has_diag) {
                errs[t] = {i, "missing diagonal in row " + std::to_string(i)};
                return;
            }
        }
    });
    if (first_error(errs, err)) return false;
    // symmetric pattern: every (i,j) has a stored (j,i)
    for_row_chunks(n, [&](int32_t lo, int32_t hi, int t) {
        for (int32_t i = lo; i < hi; ++i)
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                int32_t j = A.ci[k];
                const int32_t* b = A.ci.data() + A.rp[j];
                const int32_t* e = A.ci.data() + A.rp[j + 1];
                if (!std::binary_search(b, e, i)) {
                    errs[t] = {i, "pattern not symmetric at (" + std::to_string(i) + "," + std::to_string(j) +
                                      ")"};
                    return;
                }
            }
    });
    return !first_error(errs, err);
}

bool check_values_symmetric(const HostCsr& A, std::string& err) {
    const char* env = std::getenv("AMG_CHECK");
    if (!env || !*env || std::string(env) == "0") return true;
    for (int32_t i = 0; i < A.n; ++i)
        for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            const int32_t j = A.ci[k];
            if (j <= i) continue;
            const int32_t* b = A.ci.data() + A.rp[j];
            const int32_t* e = A.ci.data() + A.rp[j + 1];
            const int32_t t = (int32_t)(std::lower_bound(b, e, i) - A.ci.data());
            if (!(A.va[t] == A.va[k])) {
                err = "matrix values not symmetric at (" + std::to_string(i) + "," +
                      std::to_string(j) + ")";
                return false;
            }
        }
    return true;
}

namespace {

inline double edge_w(double a) { return a < 0.0 ? -a : 0.0; }

struct Strength {
    std::vector<double> diag, eta;
    std::vector<int32_t> tpos;       // position of (j,i) for entry (i,j)
    std::vector<uint8_t> strong;     // per entry
    std::vector<uint8_t> isolated, dirichlet;
    std::vector<int32_t> deg;        // |N(i)|
};

void compute_strength(const HostCsr& A, const amg_params& p, Strength& S) {
    const int32_t n = A.n;
    const int64_t nnz = A.nnz();
    S.diag.assign(n, 0.0);
    S.eta.assign(n, 0.0);
    S.tpos.assign(nnz, -1);
    S.strong.assign(nnz, 0);
    S.isolated.assign(n, 0);
    S.dirichlet.assign(n, 0);
    S.deg.assign(n, 0);
    // three per-row passes (each reads the previous pass's results of other
    // rows), on host threads for large matrices
    for_row_chunks(n, [&](int32_t lo, int32_t hi, int) {
        for (int32_t i = lo; i < hi; ++i)
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
                if (A.ci[k] == i) S.diag[i] = A.va[k];
                else ++S.deg[i];
    });
    std::vector<double> s(nnz, 0.0);
    for_row_chunks(n, [&](int32_t lo, int32_t hi, int) {
        for (int32_t i = lo; i < hi; ++i) {
            double m = 0.0;
            bool nonzero = false;
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                int32_t j = A.ci[k];
                if (j == i) continue;
                if (A.va[k] != 0.0) nonzero = true;
                const int32_t* b = A.ci.data() + A.rp[j];
                const int32_t* e = A.ci.data() + A.rp[j + 1];
                const int32_t* f = std::lower_bound(b, e, i);
                int32_t t = (f != e && *f == i) ? (int32_t)(f - A.ci.data()) : -1;
                S.tpos[k] = t;
                double wji = t >= 0 ? edge_w(A.va[t]) : 0.0;
                double c = (edge_w(A.va[k]) * wji) / (S.diag[i] * S.diag[j]);
                s[k] = c;
                m = std::max(m, c);
            }
            S.eta[i] = m;
            S.isolated[i] = m < p.beta;
            S.dirichlet[i] = !nonzero;
        }
    });
    for_row_chunks(n, [&](int32_t lo, int32_t hi, int) {
        for (int32_t i = lo; i < hi; ++i)
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                int32_t j = A.ci[k];
                if (j == i) continue;
                S.strong[k] = (s[k] > 0.0 && s[k] > p.delta * std::min(S.eta[i], S.eta[j])) ? 1 : 0;
            }
    });
}

class Aggregation {
public:
    Aggregation(const HostCsr& A, const Strength& S, const amg_params& p)
        : A_(A), S_(S), p_(p), n_(A.n) {}

    AggResult run();

private:
    const HostCsr& A_;
    const Strength& S_;
    const amg_params& p_;
    const int32_t n_;

    std::vector<int32_t> agg_;
    std::vector<uint8_t> inU_;
    std::vector<int32_t> nna_;
    int64_t remaining_ = 0;

    // bucket queues keyed by N_na with lazy deletion
    std::vector<std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>>> buckets_;
    int32_t min_bucket_ = 0;

    // set membership by stamps
    std::vector<uint32_t> in_a_, in_na_, adj_mark_;
    uint32_t stamp_a_ = 0, stamp_na_ = 0;
    // aggregates (ids below adj_limit_) holding a vertex of N(a) carry
    // adj_mark_ == stamp_na_; the isolated phase counts only the aggregates of
    // non-isolated vertices
    int32_t adj_limit_ = INT_MAX;
    std::vector<int32_t> pos_in_a_;

    std::vector<int32_t> a_;          // members of the aggregate being built
    std::vector<int32_t> na_;         // N(a)
    // links into the aggregate being built, kept up to date as members join
    // (valid where lstamp_ == stamp_a_): cons_2, cons_1 and the strong links
    // from the row into a; and the strong links from each row of U into U
    std::vector<uint32_t> lstamp_;
    std::vector<int32_t> lc2_, lc1_, lsa_, su_;
    int32_t maxa_ = 0;
    std::vector<int32_t> dist_;       // all-pairs distances inside a, maxa_ x maxa_

    int32_t next_id_ = 0;

    // v leaves U: its neighbours in U lose one N_na.  Their bucket entries
    // are refreshed once per aggregate (requeue_neighbours): every such
    // neighbour is in N(a), and the global minimum is only asked for between
    // aggregates.
    void remove_from_U(int32_t v) {
        inU_[v] = 0;
        --remaining_;
        for (int32_t k = A_.rp[v]; k < A_.rp[v + 1]; ++k) {
            int32_t j = A_.ci[k];
            if (j == v || !inU_[j]) continue;
            --nna_[j];
            const int32_t t = S_.tpos[k];
            if (t >= 0 && S_.strong[t]) --su_[j];
        }
    }
    void requeue_neighbours() {
        for (int32_t y : na_) {
            if (!inU_[y]) continue;
            const int32_t c = nna_[y];
            buckets_[c].push(y);
            if (c < min_bucket_) min_bucket_ = c;
        }
    }

    int32_t global_min() {
        for (int32_t c = min_bucket_; c < (int32_t)buckets_.size(); ++c) {
            auto& h = buckets_[c];
            while (!h.empty()) {
                int32_t v = h.top();
                if (inU_[v] && nna_[v] == c) { min_bucket_ = c; return v; }
                h.pop();
            }
        }
        return -1;
    }

    bool in_a(int32_t v) const { return in_a_[v] == stamp_a_; }

    void start_aggregate(int32_t v) {
        ++stamp_a_;
        a_.clear();
        ++stamp_na_;
        na_.clear();
        add_member_plain(v);
        dist_[0] = 0;
    }
    // v joins a.  N(a) grows by v's neighbours outside a; v itself stays in
    // the list (every reader skips members: they are not in U, and not
    // unaggregated isolated vertices), so the list is N(a) plus former
    // members, in the order they were reached.
    void add_member_plain(int32_t v) {
        in_a_[v] = stamp_a_;
        pos_in_a_[v] = (int32_t)a_.size();
        a_.push_back(v);
        for (int32_t k = A_.rp[v]; k < A_.rp[v + 1]; ++k) {
            const int32_t j = A_.ci[k];
            if (j == v || in_a(j) || in_na_[j] == stamp_na_) continue;
            in_na_[j] = stamp_na_;
            na_.push_back(j);
            const int32_t g = agg_[j];
            if (g >= 0 && g < adj_limit_) adj_mark_[g] = stamp_na_;
        }
        // the new member's links as its neighbours see them: s1 = (w, v)
        // strong, s2 = (v, w) strong, counted only where w's row stores v
        for (int32_t k = A_.rp[v]; k < A_.rp[v + 1]; ++k) {
            const int32_t w = A_.ci[k];
            const int32_t t = S_.tpos[k];
            if (w == v || t < 0) continue;
            if (lstamp_[w] != stamp_a_) {
                lstamp_[w] = stamp_a_;
                lc2_[w] = lc1_[w] = lsa_[w] = 0;
            }
            const bool s1 = S_.strong[t] != 0, s2 = S_.strong[k] != 0;
            if (s1 && s2) ++lc2_[w];
            else if (s1 != s2) ++lc1_[w];
            lsa_[w] += s1;
        }
    }

    // distances from w (not in a) to every member through edges into a
    // (shortest paths never return through w); false if some member is
    // unreachable or farther than d_max.
    bool ecc_within(int32_t w, int32_t* dw) const {
        const int32_t m = (int32_t)a_.size();
        for (int32_t t = 0; t < m; ++t) dw[t] = INT_MAX / 2;
        for (int32_t k = A_.rp[w]; k < A_.rp[w + 1]; ++k) {
            int32_t u = A_.ci[k];
            if (u == w || !in_a(u)) continue;
            const int32_t* row = &dist_[(size_t)pos_in_a_[u] * maxa_];
            for (int32_t t = 0; t < m; ++t) dw[t] = std::min(dw[t], row[t] + 1);
        }
        for (int32_t t = 0; t < m; ++t)
            if (dw[t] > p_.d_max) return false;
        return true;
    }

    // append w whose distances to the members are dw; update all pairs
    void add_member_dist(int32_t w, const int32_t* dw) {
        const int32_t m = (int32_t)a_.size();
        for (int32_t x = 0; x < m; ++x)
            for (int32_t y = 0; y < m; ++y) {
                int32_t via = dw[x] + dw[y];
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

    // cons_2 / cons_1 of w with respect to a: links (w, u), u in a, strong both
    // ways / one way (kept up to date by add_member_plain)
    void cons(int32_t w, int32_t& c2, int32_t& c1) const {
        const bool live = lstamp_[w] == stamp_a_;
        c2 = live ? lc2_[w] : 0;
        c1 = live ? lc1_[w] : 0;
    }
    int32_t strong_into_a(int32_t w) const { return lstamp_[w] == stamp_a_ ? lsa_[w] : 0; }

    void grow();
    void round_aggregate();
    void grow_iso(int32_t n_phase1);
};

void Aggregation::grow() {
    struct Cand { int32_t w, c2, c1; };
    std::vector<Cand> cands;
    std::vector<int32_t> dws;      // distance rows of the candidates
    std::vector<int32_t> dw(maxa_);
    while ((int32_t)a_.size() < p_.s_min) {
        cands.clear();
        dws.clear();
        const int32_t m = (int32_t)a_.size();
        int32_t max_c2 = 0;
        for (int32_t w : na_) {
            if (!inU_[w]) continue;
            int32_t c2, c1;
            cons(w, c2, c1);
            if (c2 + c1 <= 0) continue;
            if (!ecc_within(w, dw.data())) continue;
            cands.push_back({w, c2, c1});
            dws.insert(dws.end(), dw.begin(), dw.begin() + m);
            max_c2 = std::max(max_c2, c2);
        }
        if (cands.empty()) break;
        // lexicographic best: key1 desc, connect ratio desc, neighbors desc, index asc
        int best = -1;
        int64_t b_key1 = 0, b_conn = 0, b_deg = 1, b_nb = 0;
        for (size_t q = 0; q < cands.size(); ++q) {
            const Cand& c = cands[q];
            int64_t key1 = max_c2 > 0 ? c.c2 : c.c1;
            if (best >= 0 && key1 < b_key1) continue;
            int64_t conn = 0, nb = 0;
            const int32_t w = c.w;
            for (int32_t k = A_.rp[w]; k < A_.rp[w + 1]; ++k) {
                int32_t u = A_.ci[k];
                if (u == w || in_a(u)) continue;
                conn += (agg_[u] >= 0 && adj_mark_[agg_[u]] == stamp_na_) ? 2 : 1;
                if (inU_[u] && in_na_[u] != stamp_na_) ++nb;
            }
            int64_t deg = S_.deg[w];
            bool better;
            if (best < 0 || key1 > b_key1) better = true;
            else if (conn * b_deg != b_conn * deg) better = conn * b_deg > b_conn * deg;
            else if (nb != b_nb) better = nb > b_nb;
            else better = w < cands[best].w;
            if (better) {
                best = (int)q;
                b_key1 = key1;
                b_conn = conn;
                b_deg = deg;
                b_nb = nb;
            }
        }
        const int32_t c = cands[best].w;
        add_member_dist(c, &dws[(size_t)best * m]);
        remove_from_U(c);
    }
}

void Aggregation::round_aggregate() {
    while ((int32_t)a_.size() < p_.s_max) {
        int32_t chosen = INT_MAX;
        for (int32_t w : na_) {
            if (!inU_[w] || w >= chosen) continue;
            int32_t c2, c1;
            cons(w, c2, c1);
            if (c2 + c1 <= 0) continue;
            // strong links from w into a and into U (members of a have left U)
            if (strong_into_a(w) > su_[w]) chosen = w;
        }
        if (chosen == INT_MAX) break;
        add_member_plain(chosen);   // distances are not needed after Algorithm 2
        remove_from_U(chosen);
    }
}

void Aggregation::grow_iso(int32_t n_phase1) {
    std::vector<int32_t> dw(maxa_), best_dw(maxa_);
    while ((int32_t)a_.size() < p_.s_min) {
        int32_t chosen = INT_MAX;
        const int32_t m = (int32_t)a_.size();
        for (int32_t w : na_) {
            if (w >= chosen) continue;
            if (!S_.isolated[w] || S_.dirichlet[w] || agg_[w] != -1) continue;
            if (!ecc_within(w, dw.data())) continue;
            bool shares = false;
            for (int32_t k = A_.rp[w]; k < A_.rp[w + 1] && !shares; ++k) {
                int32_t y = A_.ci[k];
                if (y == w) continue;
                int32_t g = agg_[y];
                if (g >= 0 && g < n_phase1 && adj_mark_[g] == stamp_na_) shares = true;
            }
            if (!shares) continue;
            chosen = w;
            std::copy(dw.begin(), dw.begin() + m, best_dw.begin());
        }
        if (chosen == INT_MAX) break;
        add_member_dist(chosen, best_dw.data());
        agg_[chosen] = -2;
    }
}

AggResult Aggregation::run() {
    agg_.assign(n_, -1);
    inU_.assign(n_, 0);
    nna_.assign(n_, 0);
    in_a_.assign(n_, 0);
    in_na_.assign(n_, 0);
    adj_mark_.assign(n_, 0);
    pos_in_a_.assign(n_, 0);
    lstamp_.assign(n_, 0);
    lc2_.assign(n_, 0);
    lc1_.assign(n_, 0);
    lsa_.assign(n_, 0);
    su_.assign(n_, 0);
    maxa_ = std::max(p_.s_max, p_.s_min) + 2;
    dist_.assign((size_t)maxa_ * maxa_, 0);

    AggResult R;
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n_; ++v) {
        maxdeg = std::max(maxdeg, S_.deg[v]);
        inU_[v] = (!S_.isolated[v] && !S_.dirichlet[v]) ? 1 : 0;
        R.n_isolated += S_.isolated[v] && !S_.dirichlet[v];
        R.n_dirichlet += S_.dirichlet[v];
    }
    buckets_.assign(maxdeg + 1, {});
    for (int32_t v = 0; v < n_; ++v) {
        if (!inU_[v]) continue;
        int32_t c = 0, su = 0;
        for (int32_t k = A_.rp[v]; k < A_.rp[v + 1]; ++k) {
            int32_t j = A_.ci[k];
            if (j != v && inU_[j]) {
                ++c;
                su += S_.strong[k] != 0;
            }
        }
        su_[v] = su;
        nna_[v] = c;
        buckets_[c].push(v);
        ++remaining_;
    }
    min_bucket_ = 0;

    std::vector<int32_t> size_of;   // aggregate sizes, for the report
    if (remaining_ > 0) {
        int32_t v = global_min();
        while (true) {
            start_aggregate(v);
            remove_from_U(v);
            grow();
            round_aggregate();
            if (a_.size() == 1) {
                int32_t target = -1;
                double best_s = -1.0;
                for (int32_t k = A_.rp[v]; k < A_.rp[v + 1]; ++k) {
                    int32_t u = A_.ci[k];
                    if (u == v || !S_.strong[k] || agg_[u] < 0) continue;
                    int32_t t = S_.tpos[k];
                    double wuv = t >= 0 ? edge_w(A_.va[t]) : 0.0;
                    double s = (edge_w(A_.va[k]) * wuv) / (S_.diag[v] * S_.diag[u]);
                    if (s > best_s || (s == best_s && agg_[u] < target)) {
                        best_s = s;
                        target = agg_[u];
                    }
                }
                if (target >= 0) {
                    agg_[v] = target;
                    ++size_of[target];
                } else {
                    agg_[v] = next_id_++;
                    size_of.push_back(1);
                }
            } else {
                for (int32_t x : a_) agg_[x] = next_id_;
                size_of.push_back((int32_t)a_.size());
                ++next_id_;
            }
            if (remaining_ == 0) break;
            requeue_neighbours();
            int32_t seed = -1;
            for (int32_t y : na_)
                if (inU_[y] && (seed < 0 || nna_[y] < nna_[seed] || (nna_[y] == nna_[seed] && y < seed)))
                    seed = y;
            v = seed >= 0 ? seed : global_min();
        }
    }
    const int32_t n_phase1 = next_id_;
    adj_limit_ = n_phase1;
    for (int32_t v = 0; v < n_; ++v) {
        if (!S_.isolated[v] || S_.dirichlet[v] || agg_[v] >= 0) continue;
        start_aggregate(v);
        agg_[v] = -2;
        grow_iso(n_phase1);
        for (int32_t x : a_) agg_[x] = next_id_;
        size_of.push_back((int32_t)a_.size());
        ++next_id_;
    }
    R.agg.swap(agg_);
    R.nc = next_id_;
    for (int32_t s : size_of) R.max_size = std::max(R.max_size, s);
    return R;
}

}  // namespace

AggResult aggregate(const HostCsr& A, const amg_params& p) {
    Strength S;
    compute_strength(A, p, S);
    Aggregation G(A, S, p);
    return G.run();
}

AggResult aggregate_tiled(const HostCsr& A, const amg_params& p, int32_t tile, int threads) {
    const int32_t n = A.n;
    const int32_t ntiles = (n + tile - 1) / tile;
    std::vector<AggResult> parts(ntiles);
    auto work = [&](int32_t t) {
        const int32_t t0 = t * tile, t1 = std::min(n, t0 + tile);
        HostCsr sub;
        sub.n = t1 - t0;
        sub.rp.assign(sub.n + 1, 0);
        for (int32_t i = t0; i < t1; ++i) {
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                const int32_t j = A.ci[k];
                if (j < t0 || j >= t1) continue;
                sub.ci.push_back(j - t0);
                sub.va.push_back(A.va[k]);
            }
            sub.rp[i - t0 + 1] = (int32_t)sub.ci.size();
        }
        parts[t] = aggregate(sub, p);
    };
    std::atomic<int32_t> next{0};
    auto worker = [&] {
        for (int32_t t = next++; t < ntiles; t = next++) work(t);
    };
    const int nth = std::max(1, std::min<int>(threads, ntiles));
    std::vector<std::thread> pool;
    for (int i = 1; i < nth; ++i) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    AggResult R;
    R.agg.assign(n, -1);
    for (int32_t t = 0; t < ntiles; ++t) {
        const AggResult& P = parts[t];
        const int32_t t0 = t * tile;
        for (size_t i = 0; i < P.agg.size(); ++i)
            R.agg[t0 + i] = P.agg[i] >= 0 ? R.nc + P.agg[i] : -1;
        R.nc += P.nc;
        R.max_size = std::max(R.max_size, P.max_size);
        R.n_isolated += P.n_isolated;
        R.n_dirichlet += P.n_dirichlet;
    }
    return R;
}

int32_t greedy_colouring(const HostCsr& A, std::vector<int32_t>& colour) {
    const int32_t n = A.n;
    colour.assign(n, -1);
    std::vector<int32_t> seen;
    int32_t nc = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            int32_t j = A.ci[k];
            if (j < i) {
                int32_t c = colour[j];
                if (c >= (int32_t)seen.size()) seen.resize(c + 1, -1);
                seen[c] = i;
            }
        }
        int32_t c = 0;
        while (c < (int32_t)seen.size() && seen[c] == i) ++c;
        colour[i] = c;
        nc = std::max(nc, c + 1);
    }
    return nc;
}



int32_t dsatur_colouring(const HostCsr& A, std::vector<int32_t>& colour) {
    const int32_t n = A.n;
    // per-row state in one record, so that a neighbour update touches one
    // cache line; colours >= 64 seen by a row go to an overflow list
    struct Row {
        uint64_t low = 0;        // colours < 64 among the coloured neighbours
        uint32_t stamp = 0;      // when the saturation last changed
        int32_t sat = 0;
        int32_t deg = 0;
        int32_t colour = -1;
    };
    std::vector<Row> R(n);
    std::vector<std::vector<int32_t>> high;   // sorted colours >= 64, by overflow slot
    std::vector<int32_t> high_slot;           // row -> overflow slot (-1: none)
    auto has = [&](int32_t j, int32_t c) {
        if (c < 64) return ((R[j].low >> c) & 1u) != 0;
        if (high_slot.empty() || high_slot[j] < 0) return false;
        const auto& h = high[high_slot[j]];
        return std::binary_search(h.begin(), h.end(), c);
    };
    auto add = [&](int32_t j, int32_t c) {
        if (c < 64) {
            R[j].low |= uint64_t(1) << c;
            return;
        }
        if (high_slot.empty()) high_slot.assign(n, -1);
        if (high_slot[j] < 0) {
            high_slot[j] = (int32_t)high.size();
            high.emplace_back();
        }
        auto& h = high[high_slot[j]];
        h.insert(std::lower_bound(h.begin(), h.end(), c), c);
    };
    auto smallest_free = [&](int32_t v) {
        if (~R[v].low) return (int32_t)__builtin_ctzll(~R[v].low);
        int32_t c = 64;
        if (!high_slot.empty() && high_slot[v] >= 0)
            for (int32_t h : high[high_slot[v]]) {
                if (h != c) break;
                ++c;
            }
        return c;
    };
    int32_t maxdeg = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t d = 0;
        for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) d += A.ci[k] != i;
        R[i].deg = d;
        R[i].stamp = (uint32_t)i;
        maxdeg = std::max(maxdeg, d);
    }
    // FIFO buckets by (saturation, degree) with lazy deletion: an entry is
    // live while its row is uncoloured and its stamp is the row's latest, so a
    // bucket's first live entry is the row that reached it first
    struct Bucket {
        std::vector<std::pair<int32_t, uint32_t>> q;   // (row, stamp)
        size_t head = 0;
        int64_t live = 0;
    };
    const int32_t D = maxdeg + 1;
    std::vector<std::vector<Bucket>> buckets(1, std::vector<Bucket>(D));
    std::vector<int32_t> dtop(1, -1);   // highest degree with live entries, per saturation
    for (int32_t i = 0; i < n; ++i) {
        Bucket& b = buckets[0][R[i].deg];
        b.q.emplace_back(i, (uint32_t)i);
        ++b.live;
        dtop[0] = std::max(dtop[0], R[i].deg);
    }
    uint32_t clock = (uint32_t)n;
    int32_t top = 0, nc = 0;
    for (int32_t done = 0; done < n; ++done) {
        int32_t v = -1;
        while (v < 0) {
            int32_t& d = dtop[top];
            while (d >= 0 && buckets[top][d].live == 0) --d;
            if (d < 0) {
                --top;
                continue;
            }
            Bucket& b = buckets[top][d];
            while (true) {
                const auto e = b.q[b.head++];
                if (R[e.first].colour < 0 && R[e.first].stamp == e.second) {
                    v = e.first;
                    break;
                }
            }
            --b.live;
        }
        const int32_t c = smallest_free(v);
        R[v].colour = c;
        nc = std::max(nc, c + 1);
        for (int32_t k = A.rp[v]; k < A.rp[v + 1]; ++k) {
            const int32_t j = A.ci[k];
            if (j == v || R[j].colour >= 0 || has(j, c)) continue;
            add(j, c);
            --buckets[R[j].sat][R[j].deg].live;
            const int32_t s = ++R[j].sat;
            if (s >= (int32_t)buckets.size()) {
                buckets.emplace_back(D);
                dtop.push_back(-1);
            }
            R[j].stamp = clock++;
            Bucket& b = buckets[s][R[j].deg];
            b.q.emplace_back(j, R[j].stamp);
            ++b.live;
            dtop[s] = std::max(dtop[s], R[j].deg);
            top = std::max(top, s);
        }
    }
    colour.resize(n);
    for (int32_t i = 0; i < n; ++i) colour[i] = R[i].colour;
    return nc;
}

int32_t smoother_colouring(const HostCsr& A, std::vector<int32_t>& colour) {
    const int32_t nc = greedy_colouring(A, colour);
    if (nc <= 2) return nc;   // DSATUR cannot use fewer colours than two here
    std::vector<int32_t> alt;
    const int32_t na = dsatur_colouring(A, alt);
    if (na < nc) {
        colour.swap(alt);
        return na;
    }
    return nc;
}

}  // namespace amg
