// Oracle for the aggregation AMG-preconditioned CG of Blatt, Ippisch & Bastian,
// "A Massively Parallel Algebraic Multigrid Preconditioner based on Aggregation
// for Elliptic Problems with Heterogeneous Coefficients" (arXiv:1209.0960).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
// FP64 CPU restatement of the method, used by the tests and by the benchmark's
// CPU baseline to check and time the CUDA library.  It shares no code, header
// or constant with the library and must never be linked into it.
//
// Every step follows the paper's order and notation.  Where the paper is silent,
// garbled or ambiguous, the documented reading is used; the readings are listed
// at each step below.  Compile with -ffp-contract=off so no FMA is introduced.
//
// The same source also builds with -fopenmp, for the CPU baseline on all host
// cores only: the SpMV, the rows of one colour in a Gauss-Seidel sweep, the
// residual, the prolongation and the CG vector updates then run in parallel
// (each row or element is computed exactly as in the serial build); the
// restriction, the dot products and the coarsest triangular solves stay
// sequential.  The serial build ignores the pragmas.
//
// Parity status: strength, aggregation, colouring, Galerkin product, V-cycle
// and PCG are pinned by tests against closed forms, hand-derived maps, dense
// direct solves and invariants.  The aggregation's ranking and tie-breaking
// are pinned on large graphs by hand-derived closed forms (long chains and
// 2 x m ladders); irregular graphs rest on those rules and the invariants.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <queue>
#include <set>
#include <tuple>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Sparse matrix (Sec. 4.2: scalar CSR, columns sorted within each row)
// ---------------------------------------------------------------------------
struct Csr {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<double> va;

    // position of entry (i, j) in row i, or -1 when it is not stored
    int find(int i, int j) const {
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == j) return k;
        return -1;
    }
    double entry(int i, int j) const {
        int k = find(i, j);
        return k < 0 ? 0.0 : va[k];
    }
    // N(i): adjacent vertices in the matrix graph (stored off-diagonals)
    std::vector<int> neighbours(int i) const {
        std::vector<int> out;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] != i) out.push_back(ci[k]);
        return out;
    }
};

struct Params {
    double delta;          // strong-edge threshold, Eq. (symmetric_strong2)
    double beta;           // isolated-vertex threshold, Sec. 2.1 (b)
    double omega;          // over-correction, end of Sec. 2.1
    int s_min, s_max, d_max;   // Alg. 1 arguments
    int coarsen_target;    // stop when a level has at most this many rows
    int max_levels;
    int dense_cap;         // largest coarsest level solved densely
    double min_rate;       // stop when n_l / n_{l+1} falls below this
    int agg_tile = 0;      // > 0: decoupled aggregation in tiles of this many
                           // consecutive rows (Alg. 4), else one sequential pass
    int smoother = 0;      // 0: multicolour symmetric GS (the GPU's order);
                           // 1: sequential symmetric GS in index order (the
                           //    paper's hybrid smoother on a single process)
};

// ---------------------------------------------------------------------------
// Strength of connection (Sec. 2.1, Eq. symmetric_strong1 / symmetric_strong2)
// ---------------------------------------------------------------------------
// w_E((i,j)): 0 for positive off-diagonals, the magnitude of negative ones.
// (The printed formula 1/2 (A_ij - |A_ij|) is non-positive; the text says
// "the absolute value otherwise", which this reading follows.  The product
// w_E(i,j) w_E(j,i) is the same under either sign.)
double edge_weight(double aij) { return aij < 0.0 ? -aij : 0.0; }

struct Strength {
    std::vector<double> eta;         // eta_max(i)
    std::vector<char> isolated;      // eta_max(i) < beta
    std::vector<char> dirichlet;     // row without a non-zero off-diagonal
    std::vector<char> strong;        // per stored entry k = (i, j): edge strong
};

// The normalised coupling of Eq. (symmetric_strong1):
//   w_E(i,j) w_E(j,i) / (w_V(i) w_V(j)),   w_V(i) = A_ii.
double coupling(const Csr& A, int i, int j) {
    double num = edge_weight(A.entry(i, j)) * edge_weight(A.entry(j, i));
    double den = A.entry(i, i) * A.entry(j, j);
    return num / den;
}

Strength compute_strength(const Csr& A, const Params& p) {
    Strength S;
    int n = A.n;
    S.eta.assign(n, 0.0);
    S.isolated.assign(n, 0);
    S.dirichlet.assign(n, 0);
    S.strong.assign(A.ci.size(), 0);
    // eta_max(i) = max over k in N(i) of the coupling (0 without neighbours)
    for (int i = 0; i < n; ++i) {
        double m = 0.0;
        for (int j : A.neighbours(i)) m = std::max(m, coupling(A, i, j));
        S.eta[i] = m;
        S.isolated[i] = (m < p.beta) ? 1 : 0;          // Sec. 2.1 (b)
        bool any_nonzero = false;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (A.ci[k] != i && A.va[k] != 0.0) any_nonzero = true;
        S.dirichlet[i] = any_nonzero ? 0 : 1;
    }
    // (a) edge strong iff coupling > delta min(eta_max(i), eta_max(j)); a zero
    // coupling is never strong.
    for (int i = 0; i < n; ++i)
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            int j = A.ci[k];
            if (j == i) continue;
            double s = coupling(A, i, j);
            S.strong[k] = (s > 0.0 && s > p.delta * std::min(S.eta[i], S.eta[j])) ? 1 : 0;
        }
    return S;
}

bool is_strong(const Csr& A, const Strength& S, int i, int j) {
    int k = A.find(i, j);
    return k >= 0 && S.strong[k];
}

// ---------------------------------------------------------------------------
// Aggregation (Sec. 2.1, Algorithms 1-3 and GrowIsoAggregate)
// ---------------------------------------------------------------------------
struct Aggregator {
    const Csr& A;
    const Strength& S;
    const Params& p;
    std::vector<int> agg;          // coarse index of each vertex, -1 = none
    std::vector<char> inU;         // U: still-unaggregated candidates
    std::set<std::pair<int, int>> by_count;   // (N_na(u), u) for u in U
    std::vector<int> nna;          // N_na(u) = |N(u) ∩ U|
    std::vector<std::vector<int>> nbrs;   // N(i) of every vertex
    int next_id = 0;

    Aggregator(const Csr& A_, const Strength& S_, const Params& p_)
        : A(A_), S(S_), p(p_), agg(A_.n, -1), inU(A_.n, 0), nna(A_.n, 0) {
        nbrs.resize(A.n);
        for (int i = 0; i < A.n; ++i) nbrs[i] = A.neighbours(i);
    }

    // N(a) = vertices outside a adjacent to some vertex of a
    std::set<int> nbr_of_set(const std::set<int>& a) const {
        std::set<int> out;
        for (int x : a)
            for (int j : nbrs[x])
                if (!a.count(j)) out.insert(j);
        return out;
    }

    // diam(a, v): diameter of the subgraph induced by a ∪ {v} (matrix-graph
    // edges), by breadth-first search from every vertex.  Disconnected -> INT_MAX.
    int diameter(const std::set<int>& vset) const {
        std::vector<int> verts(vset.begin(), vset.end());
        const int m = (int)verts.size();
        auto index_of = [&](int v) {
            for (int t = 0; t < m; ++t)
                if (verts[t] == v) return t;
            return -1;
        };
        int diam = 0;
        for (int s = 0; s < m; ++s) {
            std::vector<int> dist(m, -1);
            std::vector<int> queue = {s};
            dist[s] = 0;
            for (size_t h = 0; h < queue.size(); ++h) {
                int u = queue[h];
                for (int w : nbrs[verts[u]]) {
                    int t = index_of(w);
                    if (t >= 0 && dist[t] < 0) {
                        dist[t] = dist[u] + 1;
                        queue.push_back(t);
                    }
                }
            }
            for (int t = 0; t < m; ++t) {
                if (dist[t] < 0) return std::numeric_limits<int>::max();
                diam = std::max(diam, dist[t]);
            }
        }
        return diam;
    }

    // cons_2(v, a): two-way strong connections between v and a;
    // cons_1(v, a): one-way strong connections (Sec. 2.1, after Alg. 2)
    int cons2(int v, const std::set<int>& a) const {
        int c = 0;
        for (int u : a)
            if (is_strong(A, S, v, u) && is_strong(A, S, u, v)) ++c;
        return c;
    }
    int cons1(int v, const std::set<int>& a) const {
        int c = 0;
        for (int u : a)
            if (is_strong(A, S, v, u) != is_strong(A, S, u, v)) ++c;
        return c;
    }

    // connect(v, a): neighbours of v outside a count twice when they belong to
    // an aggregate already adjacent to a, once otherwise (unaggregated, or in an
    // aggregate not yet adjacent to a).
    int connect(int v, const std::set<int>& a, const std::set<int>& adj_aggs) const {
        int c = 0;
        for (int u : nbrs[v]) {
            if (a.count(u)) continue;
            if (agg[u] >= 0 && adj_aggs.count(agg[u])) c += 2;
            else c += 1;
        }
        return c;
    }

    // neighbors(v, a): unaggregated neighbours of v that are not yet
    // neighbours of a (Sec. 2.1, last tie-break of Alg. 2)
    int neighbors_score(int v, const std::set<int>& a, const std::set<int>& Na) const {
        int c = 0;
        for (int u : nbrs[v])
            if (inU[u] && !a.count(u) && !Na.count(u)) ++c;
        return c;
    }

    void remove_from_U(int v) {
        if (!inU[v]) return;
        by_count.erase({nna[v], v});
        inU[v] = 0;
        for (int j : nbrs[v])
            if (inU[j]) {
                by_count.erase({nna[j], j});
                --nna[j];
                by_count.insert({nna[j], j});
            }
    }

    // Algorithm 2: grow a until |a| = s_min (the comment's reading of the loop
    // test), adding the best candidate within the diameter limit.
    void grow(std::set<int>& a) {
        while ((int)a.size() < p.s_min) {
            std::set<int> Na = nbr_of_set(a);
            std::set<int> adj_aggs;
            for (int y : Na)
                if (agg[y] >= 0) adj_aggs.insert(agg[y]);
            // C_0: unaggregated neighbours of a within the diameter limit that
            // have a strong connection to a
            std::vector<int> C0;
            for (int w : Na) {
                if (!inU[w]) continue;
                std::set<int> aw = a;
                aw.insert(w);
                if (diameter(aw) > p.d_max) continue;
                if (cons2(w, a) + cons1(w, a) <= 0) continue;
                C0.push_back(w);
            }
            if (C0.empty()) break;
            // C_1: maximal cons_2 (two-way connections preferred), else cons_1
            int m2 = 0;
            for (int w : C0) m2 = std::max(m2, cons2(w, a));
            std::vector<int> C1;
            if (m2 > 0) {
                for (int w : C0)
                    if (cons2(w, a) == m2) C1.push_back(w);
            } else {
                int m1 = 0;
                for (int w : C0) m1 = std::max(m1, cons1(w, a));
                for (int w : C0)
                    if (cons1(w, a) == m1) C1.push_back(w);
            }
            // maximal connect(v, a) / |N(v)|, compared exactly as integers
            if (C1.size() > 1) {
                long long bc = -1, bn = 1;
                for (int w : C1) {
                    long long c = connect(w, a, adj_aggs);
                    long long nw = (long long)nbrs[w].size();
                    if (bc < 0 || c * bn > bc * nw) { bc = c; bn = nw; }
                }
                std::vector<int> keep;
                for (int w : C1) {
                    long long c = connect(w, a, adj_aggs);
                    long long nw = (long long)nbrs[w].size();
                    if (c * bn == bc * nw) keep.push_back(w);
                }
                C1 = keep;
            }
            // maximal neighbors(v, a)
            if (C1.size() > 1) {
                int best = -1;
                for (int w : C1) best = std::max(best, neighbors_score(w, a, Na));
                std::vector<int> keep;
                for (int w : C1)
                    if (neighbors_score(w, a, Na) == best) keep.push_back(w);
                C1 = keep;
            }
            // remaining ties: lowest index (C0 was built in ascending order)
            int c = C1.front();
            a.insert(c);
            remove_from_U(c);
        }
    }

    // Algorithm 3: round a while |a| < s_max by adding neighbours with more
    // strong connections to a than to other unaggregated vertices.  (The
    // printed condition compares a quantity with itself; the text after the
    // algorithm gives its meaning.  The loop stops when no candidate is left.)
    void round(std::set<int>& a) {
        while ((int)a.size() < p.s_max) {
            std::set<int> Na = nbr_of_set(a);
            int chosen = -1;
            for (int w : Na) {          // ascending: the first hit is the lowest index
                if (!inU[w]) continue;
                if (cons2(w, a) + cons1(w, a) <= 0) continue;     // D
                int to_a = 0, to_u = 0;
                for (int u : nbrs[w]) {
                    if (!is_strong(A, S, w, u)) continue;          // N_delta(w)
                    if (a.count(u)) ++to_a;
                    else if (inU[u] && u != w) ++to_u;
                }
                if (to_a > to_u) { chosen = w; break; }          // C
            }
            if (chosen < 0) break;
            a.insert(chosen);
            remove_from_U(chosen);
        }
    }

    int select_seed(const std::set<int>& S_cand) const {
        // minimal N_na, then lowest index
        int best = -1;
        for (int u : S_cand)
            if (best < 0 || nna[u] < nna[best]) best = u;
        return best;
    }

    // GrowIsoAggregate (not printed in the paper).  Reading: grow by the
    // lowest-index adjacent isolated, unaggregated, non-Dirichlet vertex that
    // keeps the diameter limit and shares an adjacent aggregate of non-isolated
    // vertices with a, until |a| = s_min or no such vertex exists.
    void grow_iso(std::set<int>& a, int n_phase1) {
        while ((int)a.size() < p.s_min) {
            std::set<int> Na = nbr_of_set(a);
            std::set<int> adj_a;
            for (int y : Na)
                if (agg[y] >= 0 && agg[y] < n_phase1) adj_a.insert(agg[y]);
            int chosen = -1;
            for (int w : Na) {
                if (!S.isolated[w] || S.dirichlet[w] || agg[w] >= 0) continue;
                std::set<int> aw = a;
                aw.insert(w);
                if (diameter(aw) > p.d_max) continue;
                bool shares = false;
                for (int y : nbrs[w])
                    if (agg[y] >= 0 && agg[y] < n_phase1 && adj_a.count(agg[y])) shares = true;
                if (!shares) continue;
                chosen = w;
                break;
            }
            if (chosen < 0) break;
            a.insert(chosen);
            agg[chosen] = -2;      // taken by the aggregate being built
        }
    }

    // Algorithm 1
    int run() {
        int n = A.n;
        for (int v = 0; v < n; ++v)
            inU[v] = (!S.isolated[v] && !S.dirichlet[v]) ? 1 : 0;
        for (int v = 0; v < n; ++v) {
            if (!inU[v]) continue;
            int c = 0;
            for (int j : nbrs[v])
                if (inU[j]) ++c;
            nna[v] = c;
            by_count.insert({c, v});
        }
        int remaining = 0;
        for (int v = 0; v < n; ++v) remaining += inU[v];
        if (remaining > 0) {
            int v = by_count.begin()->second;    // global minimum of N_na, lowest index
            while (true) {
                std::set<int> a = {v};
                remove_from_U(v);
                grow(a);
                round(a);
                if (a.size() == 1) {
                    // merge a one-vertex aggregate into the aggregate holding its
                    // strongest strong neighbour (ties: lowest aggregate index)
                    int target = -1;
                    double best_s = -1.0;
                    for (int u : nbrs[v]) {
                        if (!is_strong(A, S, v, u) || agg[u] < 0) continue;
                        double s = coupling(A, v, u);
                        if (s > best_s || (s == best_s && agg[u] < target)) {
                            best_s = s;
                            target = agg[u];
                        }
                    }
                    if (target >= 0) agg[v] = target;
                    else agg[v] = next_id++;
                } else {
                    for (int x : a) agg[x] = next_id;
                    ++next_id;
                }
                if (by_count.empty()) break;
                // next seed: among unaggregated neighbours of a_v, else globally
                std::set<int> Sc;
                for (int y : nbr_of_set(a))
                    if (inU[y]) Sc.insert(y);
                if (!Sc.empty()) v = select_seed(Sc);
                else v = by_count.begin()->second;
            }
        }
        // isolated, non-Dirichlet vertices
        int n_phase1 = next_id;
        for (int v = 0; v < n; ++v) {
            if (!S.isolated[v] || S.dirichlet[v] || agg[v] >= 0) continue;
            std::set<int> a = {v};
            agg[v] = -2;
            grow_iso(a, n_phase1);
            for (int x : a) agg[x] = next_id;
            ++next_id;
        }
        return next_id;
    }
};

// ---------------------------------------------------------------------------
// Multicolour ordering for the Gauss-Seidel smoother.  The paper smooths each
// process's rows in their natural order (Sec. 3.2); the GPU needs rows that
// can be updated at once, so both sides use the same colouring.  Two greedy
// colourings are formed and the one with fewer colours is kept (ties: the
// first), because every colour costs the GPU one dependent pass per sweep.
// ---------------------------------------------------------------------------

// Greedy in ascending row order: each row takes the smallest colour no
// already coloured neighbour has (red-black on the structured grids).
int greedy_colour(const Csr& A, std::vector<int>& colour) {
    colour.assign(A.n, -1);
    int nc = 0;
    for (int i = 0; i < A.n; ++i) {
        std::set<int> used;
        for (int j : A.neighbours(i))
            if (j < i) used.insert(colour[j]);
        int c = 0;
        while (used.count(c)) ++c;
        colour[i] = c;
        nc = std::max(nc, c + 1);
    }
    return nc;
}

// DSATUR (Brelaz, 1979): repeatedly colour the uncoloured row whose
// neighbours already show the most distinct colours (its saturation); ties go
// to the row with more neighbours, then to the row whose saturation reached
// its value first (initially: the lower index; a colouring step raises its
// neighbours' saturations in column order).  The row takes the smallest
// colour none of its neighbours has.
int dsatur_colour(const Csr& A, std::vector<int>& colour) {
    const int n = A.n;
    colour.assign(n, -1);
    std::vector<std::set<int>> seen(n);   // colours among the coloured neighbours
    std::vector<int> deg(n), stamp(n);
    std::set<std::tuple<int, int, int>> order;   // (-saturation, -degree, stamp)
    std::map<int, int> row_of;                   // stamp -> row
    for (int i = 0; i < n; ++i) {
        deg[i] = (int)A.neighbours(i).size();
        stamp[i] = i;
        row_of[i] = i;
        order.insert(std::make_tuple(0, -deg[i], i));
    }
    int clock = n, nc = 0;
    while (!order.empty()) {
        const int v = row_of[std::get<2>(*order.begin())];
        order.erase(order.begin());
        int c = 0;
        while (seen[v].count(c)) ++c;
        colour[v] = c;
        nc = std::max(nc, c + 1);
        for (int j : A.neighbours(v)) {
            if (colour[j] >= 0 || seen[j].count(c)) continue;
            order.erase(std::make_tuple(-(int)seen[j].size(), -deg[j], stamp[j]));
            seen[j].insert(c);
            stamp[j] = clock++;
            row_of[stamp[j]] = j;
            order.insert(std::make_tuple(-(int)seen[j].size(), -deg[j], stamp[j]));
        }
    }
    return nc;
}

// The smoother's colouring: DSATUR when it needs fewer colours than the
// ascending-order greedy, else the greedy one.
int smoother_colour(const Csr& A, std::vector<int>& colour) {
    const int nc = greedy_colour(A, colour);
    std::vector<int> alt;
    const int na = dsatur_colour(A, alt);
    if (na < nc) {
        colour.swap(alt);
        return na;
    }
    return nc;
}

// ---------------------------------------------------------------------------
// Galerkin product (Eq. prolongation and the coarse operator after it).
// P(i, I) = 1 iff i in a_I.  G = P^T A P: G_IJ = sum of A_ij over i in a_I,
// j in a_J, summed left to right in fine CSR order (i ascending, then row
// position).  The 1/omega factor is applied at prolongation instead.
// ---------------------------------------------------------------------------
Csr galerkin(const Csr& A, const std::vector<int>& agg, int nc) {
    std::vector<std::map<int, double>> rows(nc);
    for (int i = 0; i < A.n; ++i) {
        int I = agg[i];
        if (I < 0) continue;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            int J = agg[A.ci[k]];
            if (J < 0) continue;
            auto it = rows[I].find(J);
            if (it == rows[I].end()) rows[I][J] = A.va[k];
            else it->second = it->second + A.va[k];
        }
    }
    Csr G;
    G.n = nc;
    G.rp.assign(nc + 1, 0);
    for (int I = 0; I < nc; ++I) {
        for (auto& kv : rows[I]) {
            G.ci.push_back(kv.first);
            G.va.push_back(kv.second);
        }
        G.rp[I + 1] = (int)G.ci.size();
    }
    return G;
}

// ---------------------------------------------------------------------------
// Dense Cholesky for the coarsest level (the paper factors it once with a
// sparse direct solver; a dense factor gives the same exact solve).
// Uses the lower triangle (row i, columns j <= i).
// ---------------------------------------------------------------------------
bool cholesky(const Csr& A, std::vector<double>& L) {
    int n = A.n;
    std::vector<double> M((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            M[(size_t)i * n + A.ci[k]] = A.va[k];
    L.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = M[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        double ljj = std::sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = M[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = s / ljj;
        }
    }
    return true;
}

void cholesky_solve(const std::vector<double>& L, int n, const double* b, double* x) {
    std::vector<double> y(n);
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
        y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
}

// ---------------------------------------------------------------------------
// Hierarchy and V-cycle (Sec. 2: smooth, restrict the residual, correct from
// the coarser level, smooth again; direct solve on the coarsest level)
// ---------------------------------------------------------------------------
struct Level {
    Csr A;
    std::vector<int> agg;       // to level l+1 (empty on the coarsest level)
    int nc = 0;
    std::vector<int> colour;
    int ncolours = 0;
    std::vector<char> isolated, dirichlet;
};

struct Hierarchy {
    Params p;
    std::vector<Level> levels;
    std::vector<double> L;      // Cholesky factor of the coarsest matrix
    int status = 0;
};

void spmv(const Csr& A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.va[k] * x[A.ci[k]];
        y[i] = s;
    }
}

// One Gauss-Seidel update of every row of colour c:
//   x_i = (b_i - sum_{j != i} A_ij x_j) / A_ii
void gs_colour(const Level& lv, int c, const double* b, double* x) {
    const Csr& A = lv.A;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A.n; ++i) {
        if (lv.colour[i] != c) continue;
        double t = b[i];
        double d = 0.0;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            if (A.ci[k] == i) d = A.va[k];
            else t -= A.va[k] * x[A.ci[k]];
        }
        x[i] = t / d;
    }
}

// One symmetric Gauss-Seidel step in the multicolour ordering: colours
// 0..C-1 forward, then C-2..0 backward (repeating colour C-1 would change
// nothing, since its rows depend only on other colours).
void sgs(const Level& lv, const double* b, double* x) {
    for (int c = 0; c < lv.ncolours; ++c) gs_colour(lv, c, b, x);
    for (int c = lv.ncolours - 2; c >= 0; --c) gs_colour(lv, c, b, x);
}

// One symmetric Gauss-Seidel step in index order (Sec. 3.2: inside each
// process the hybrid smoother is a sequential GS sweep; on one process it is
// exactly this): rows 0..n-1 forward, then n-1..0 backward, each using the
// newest values of its neighbours.
void gs_row(const Csr& A, int i, const double* b, double* x) {
    double t = b[i];
    double d = 0.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        if (A.ci[k] == i) d = A.va[k];
        else t -= A.va[k] * x[A.ci[k]];
    }
    x[i] = t / d;
}

void sgs_sequential(const Level& lv, const double* b, double* x) {
    for (int i = 0; i < lv.A.n; ++i) gs_row(lv.A, i, b, x);
    for (int i = lv.A.n - 1; i >= 0; --i) gs_row(lv.A, i, b, x);
}

void smooth(const Hierarchy& H, const Level& lv, const double* b, double* x) {
    if (H.p.smoother == 1) sgs_sequential(lv, b, x);
    else sgs(lv, b, x);
}

void vcycle(const Hierarchy& H, int l, const double* b, double* x) {
    const Level& lv = H.levels[l];
    int n = lv.A.n;
    if (l == (int)H.levels.size() - 1) {
        cholesky_solve(H.L, n, b, x);
        return;
    }
    std::fill(x, x + n, 0.0);
    smooth(H, lv, b, x);                             // pre-smoothing, one step
    std::vector<double> r(n);
    spmv(lv.A, x, r.data());
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];  // residual
    std::vector<double> rc(lv.nc, 0.0), ec(lv.nc, 0.0);
    std::vector<char> started(lv.nc, 0);
    for (int i = 0; i < n; ++i) {                    // P^T r, ascending i
        int I = lv.agg[i];
        if (I < 0) continue;
        if (!started[I]) { rc[I] = r[i]; started[I] = 1; }
        else rc[I] = rc[I] + r[i];
    }
    vcycle(H, l + 1, rc.data(), ec.data());
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {                    // x += omega P e
        int I = lv.agg[i];
        if (I >= 0) x[i] = x[i] + H.p.omega * ec[I];
    }
    smooth(H, lv, b, x);                             // post-smoothing, one step
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

Csr make_csr(int n, const int* rp, const int* ci, const double* va) {
    Csr A;
    A.n = n;
    A.rp.assign(rp, rp + n + 1);
    A.ci.assign(ci, ci + rp[n]);
    A.va.assign(va, va + rp[n]);
    return A;
}

Params make_params(const double* q) {
    Params p;
    p.delta = q[0];
    p.beta = q[1];
    p.omega = q[2];
    p.s_min = (int)q[3];
    p.s_max = (int)q[4];
    p.d_max = (int)q[5];
    p.coarsen_target = (int)q[6];
    p.max_levels = (int)q[7];
    p.dense_cap = (int)q[8];
    p.min_rate = q[9];
    p.smoother = (int)q[10];
    p.agg_tile = (int)q[11];
    return p;
}

// Decoupled aggregation (Alg. 4, "ParallelAggregation"): the rows split into
// consecutive tiles of `tile` rows, each aggregated by the sequential
// Algorithm 1 on the tile's induced submatrix (edges that leave the tile
// dropped, strength recomputed on the submatrix); aggregates are numbered tile
// by tile and, inside a tile, in completion order.  isolated / dirichlet
// report the per-tile classification.
int aggregate_tiled(const Csr& A, const Params& p, int tile, std::vector<int>& agg,
                    std::vector<char>& isolated, std::vector<char>& dirichlet) {
    const int n = A.n;
    agg.assign(n, -1);
    isolated.assign(n, 0);
    dirichlet.assign(n, 0);
    int nc = 0;
    for (int t0 = 0; t0 < n; t0 += tile) {
        const int t1 = std::min(n, t0 + tile);
        Csr sub;
        sub.n = t1 - t0;
        sub.rp.assign(sub.n + 1, 0);
        for (int i = t0; i < t1; ++i) {
            for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                const int j = A.ci[k];
                if (j < t0 || j >= t1) continue;
                sub.ci.push_back(j - t0);
                sub.va.push_back(A.va[k]);
            }
            sub.rp[i - t0 + 1] = (int)sub.ci.size();
        }
        Strength S = compute_strength(sub, p);
        Aggregator G(sub, S, p);
        const int k = G.run();
        for (int i = 0; i < sub.n; ++i) {
            agg[t0 + i] = G.agg[i] >= 0 ? nc + G.agg[i] : -1;
            isolated[t0 + i] = S.isolated[i];
            dirichlet[t0 + i] = S.dirichlet[i];
        }
        nc += k;
    }
    return nc;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (called through ctypes by the tests and the benchmark)
// params: [delta, beta, omega, s_min, s_max, d_max, coarsen_target,
//          max_levels, dense_cap, min_rate, smoother, agg_tile]
// ---------------------------------------------------------------------------
extern "C" {

void oracle_strength(int n, const int* rp, const int* ci, const double* va,
                     const double* params, double* eta, char* isolated,
                     char* dirichlet, char* strong) {
    Csr A = make_csr(n, rp, ci, va);
    Params p = make_params(params);
    Strength S = compute_strength(A, p);
    for (int i = 0; i < n; ++i) {
        eta[i] = S.eta[i];
        isolated[i] = S.isolated[i];
        dirichlet[i] = S.dirichlet[i];
    }
    for (int k = 0; k < rp[n]; ++k) strong[k] = S.strong[k];
}

int oracle_aggregate(int n, const int* rp, const int* ci, const double* va,
                     const double* params, int* agg) {
    Csr A = make_csr(n, rp, ci, va);
    Params p = make_params(params);
    if (p.agg_tile > 0) {
        std::vector<int> a;
        std::vector<char> iso, dir;
        const int nc = aggregate_tiled(A, p, p.agg_tile, a, iso, dir);
        for (int i = 0; i < n; ++i) agg[i] = a[i];
        return nc;
    }
    Strength S = compute_strength(A, p);
    Aggregator G(A, S, p);
    int nc = G.run();
    for (int i = 0; i < n; ++i) agg[i] = G.agg[i];
    return nc;
}

// method: 0 = the smoother's colouring, 1 = ascending-order greedy, 2 = DSATUR
int oracle_colour(int n, const int* rp, const int* ci, int* colour, int method) {
    Csr A;
    A.n = n;
    A.rp.assign(rp, rp + n + 1);
    A.ci.assign(ci, ci + rp[n]);
    A.va.assign(rp[n], 0.0);
    std::vector<int> c;
    const int nc = method == 1 ? greedy_colour(A, c) : method == 2 ? dsatur_colour(A, c)
                                                                    : smoother_colour(A, c);
    for (int i = 0; i < n; ++i) colour[i] = c[i];
    return nc;
}

// Galerkin product; returns nnz of G, fills the outputs when they are non-null
// (call once with null outputs to size them).
int oracle_galerkin(int n, const int* rp, const int* ci, const double* va,
                    const int* agg, int nc, int* grp, int* gci, double* gva) {
    Csr A = make_csr(n, rp, ci, va);
    std::vector<int> a(agg, agg + n);
    Csr G = galerkin(A, a, nc);
    if (grp) {
        for (int I = 0; I <= nc; ++I) grp[I] = G.rp[I];
        for (size_t k = 0; k < G.ci.size(); ++k) {
            gci[k] = G.ci[k];
            gva[k] = G.va[k];
        }
    }
    return (int)G.ci.size();
}

void oracle_spmv(int n, const int* rp, const int* ci, const double* va,
                 const double* x, double* y) {
    Csr A = make_csr(n, rp, ci, va);
    spmv(A, x, y);
}

// Build the hierarchy.  *status: 0 ok, -1 coarsest level too large for the
// dense solve, -2 coarsest matrix not positive definite.
void* oracle_setup(int n, const int* rp, const int* ci, const double* va,
                   const double* params, int* status) {
    Hierarchy* H = new Hierarchy;
    H->p = make_params(params);
    Level l0;
    l0.A = make_csr(n, rp, ci, va);
    H->levels.push_back(l0);
    while (true) {
        Level& cur = H->levels.back();
        int lidx = (int)H->levels.size() - 1;
        if (cur.A.n <= H->p.coarsen_target) break;
        if (lidx >= H->p.max_levels - 1) break;
        std::vector<int> agg;
        std::vector<char> iso, dir;
        int nc;
        if (H->p.agg_tile > 0) {
            nc = aggregate_tiled(cur.A, H->p, H->p.agg_tile, agg, iso, dir);
        } else {
            Strength S = compute_strength(cur.A, H->p);
            Aggregator G(cur.A, S, H->p);
            nc = G.run();
            agg = G.agg;
            iso = S.isolated;
            dir = S.dirichlet;
        }
        if (nc == 0 || (double)cur.A.n / (double)nc < H->p.min_rate) break;
        cur.agg = agg;
        cur.nc = nc;
        cur.isolated = iso;
        cur.dirichlet = dir;
        cur.ncolours = smoother_colour(cur.A, cur.colour);
        Level next;
        next.A = galerkin(cur.A, cur.agg, nc);
        H->levels.push_back(next);
    }
    const Csr& Ac = H->levels.back().A;
    H->status = 0;
    if (Ac.n > H->p.dense_cap) H->status = -1;
    else if (!cholesky(Ac, H->L)) H->status = -2;
    *status = H->status;
    return H;
}

int oracle_num_levels(void* h) { return (int)((Hierarchy*)h)->levels.size(); }

void oracle_level_info(void* h, int l, int* info) {
    const Level& lv = ((Hierarchy*)h)->levels[l];
    info[0] = lv.A.n;
    info[1] = (int)lv.A.ci.size();
    info[2] = lv.nc;
    info[3] = lv.ncolours;
}

// rp/ci/va sized by oracle_level_info; agg/colour (n entries) are written
// only for levels that have them.
void oracle_level_export(void* h, int l, int* rp, int* ci, double* va,
                         int* agg, int* colour) {
    const Level& lv = ((Hierarchy*)h)->levels[l];
    std::copy(lv.A.rp.begin(), lv.A.rp.end(), rp);
    std::copy(lv.A.ci.begin(), lv.A.ci.end(), ci);
    std::copy(lv.A.va.begin(), lv.A.va.end(), va);
    if (agg && !lv.agg.empty()) std::copy(lv.agg.begin(), lv.agg.end(), agg);
    if (colour && !lv.colour.empty()) std::copy(lv.colour.begin(), lv.colour.end(), colour);
}

// z = B r: one V(1,1)-cycle with zero initial guess
void oracle_vcycle(void* h, const double* r, double* z) {
    Hierarchy* H = (Hierarchy*)h;
    vcycle(*H, 0, r, z);
}

// Preconditioned CG (the paper uses BiCGSTAB; CG is the method used here for
// the SPD case) until ||r_k|| <= tol ||r_0||.  x holds x_0 on entry.
// flexible != 0 uses beta = r_{k+1}.(z_{k+1} - z_k) / rho_k.
// out[0] = recursive relative residual, out[1] = true relative residual
// ||b - A x|| / ||b - A x_0||.  Returns the iteration count, -1 when
// p.Ap <= 0, -2 when maxit is reached.
int oracle_pcg(void* h, const double* b, double* x, double tol, int maxit,
               int flexible, double* out) {
    Hierarchy* H = (Hierarchy*)h;
    const Csr& A = H->levels[0].A;
    int n = A.n;
    std::vector<double> xv(x, x + n), r(n), z(n), zold(n), p(n), q(n);
    spmv(A, xv.data(), q.data());
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double r0 = std::sqrt(dot(r, r));
    int it = 0;
    int status = 0;
    double rel = 1.0;
    if (r0 == 0.0) {
        rel = 0.0;
    } else {
        vcycle(*H, 0, r.data(), z.data());
        p = z;
        double rho = dot(r, z);
        while (true) {
            if (it >= maxit) { status = -2; break; }
            spmv(A, p.data(), q.data());
            double pq = dot(p, q);
            if (!(pq > 0.0)) { status = -1; break; }
            double alpha = rho / pq;
#pragma omp parallel for schedule(static)
            for (int i = 0; i < n; ++i) {
                xv[i] = xv[i] + alpha * p[i];
                r[i] = r[i] - alpha * q[i];
            }
            ++it;
            rel = std::sqrt(dot(r, r)) / r0;
            if (rel <= tol) break;
            zold = z;
            vcycle(*H, 0, r.data(), z.data());
            double rho_new = dot(r, z);
            double beta;
            if (flexible) {
                double s = 0.0;
                for (int i = 0; i < n; ++i) s += r[i] * (z[i] - zold[i]);
                beta = s / rho;
            } else {
                beta = rho_new / rho;
            }
#pragma omp parallel for schedule(static)
            for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
            rho = rho_new;
        }
    }
    spmv(A, xv.data(), q.data());
    std::vector<double> rt(n);
    for (int i = 0; i < n; ++i) rt[i] = b[i] - q[i];
    out[0] = rel;
    out[1] = r0 > 0.0 ? std::sqrt(dot(rt, rt)) / r0 : 0.0;
    for (int i = 0; i < n; ++i) x[i] = xv[i];
    return status < 0 ? status : it;
}

// Preconditioned BiCGSTAB (van der Vorst 1992; the preconditioned form of
// the Templates book), the Krylov method of the paper's experiments (Sec. 5),
// with the V-cycle as the preconditioner B: two V-cycles per iteration.
//   r = b - A x, rt = r; per iteration i:
//     rho = rt.r; p = r (i = 1) or p = r + (rho/rho_prev)(alpha/w)(p - w v);
//     y = B p; v = A y; alpha = rho / rt.v; s = r - alpha v;
//     if ||s|| <= tol ||r_0||: x += alpha y, stop (the half iteration counts);
//     z = B s; t = A z; w = t.s / t.t; x += alpha y + w z; r = s - w t;
//     stop when ||r|| <= tol ||r_0||.
// out[0] = recursive relative residual, out[1] = true relative residual,
// out[2] = V-cycles applied.  Returns the iteration count, -1 on a breakdown
// (rho, rt.v or t.t zero), -2 when maxit is reached.
int oracle_bicgstab(void* h, const double* b, double* x, double tol, int maxit, double* out) {
    Hierarchy* H = (Hierarchy*)h;
    const Csr& A = H->levels[0].A;
    int n = A.n;
    std::vector<double> xv(x, x + n), r(n), rt(n), p(n, 0.0), v(n, 0.0), y(n), s(n), z(n), t(n);
    spmv(A, xv.data(), t.data());
    for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
    rt = r;
    const double r0 = std::sqrt(dot(r, r));
    int it = 0, status = 0, vcycles = 0;
    double rel = r0 > 0.0 ? 1.0 : 0.0;
    double rho_prev = 1.0, alpha = 1.0, w = 1.0;
    while (rel > tol) {
        if (it >= maxit) { status = -2; break; }
        const double rho = dot(rt, r);
        if (rho == 0.0) { status = -1; break; }
        if (it == 0) {
            p = r;
        } else {
            const double beta = (rho / rho_prev) * (alpha / w);
            for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - w * v[i]);
        }
        vcycle(*H, 0, p.data(), y.data());
        ++vcycles;
        spmv(A, y.data(), v.data());
        const double rtv = dot(rt, v);
        if (rtv == 0.0) { status = -1; break; }
        alpha = rho / rtv;
        for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        ++it;
        const double srel = std::sqrt(dot(s, s)) / r0;
        if (srel <= tol) {
            for (int i = 0; i < n; ++i) xv[i] = xv[i] + alpha * y[i];
            rel = srel;
            break;
        }
        vcycle(*H, 0, s.data(), z.data());
        ++vcycles;
        spmv(A, z.data(), t.data());
        const double tt = dot(t, t);
        if (tt == 0.0) { status = -1; break; }
        w = dot(t, s) / tt;
        for (int i = 0; i < n; ++i) {
            xv[i] = xv[i] + alpha * y[i] + w * z[i];
            r[i] = s[i] - w * t[i];
        }
        rel = std::sqrt(dot(r, r)) / r0;
        rho_prev = rho;
    }
    std::vector<double> q(n);
    spmv(A, xv.data(), q.data());
    for (int i = 0; i < n; ++i) q[i] = b[i] - q[i];
    out[0] = rel;
    out[1] = r0 > 0.0 ? std::sqrt(dot(q, q)) / r0 : 0.0;
    out[2] = vcycles;
    for (int i = 0; i < n; ++i) x[i] = xv[i];
    return status < 0 ? status : it;
}

void oracle_free(void* h) { delete (Hierarchy*)h; }

// threads the OpenMP build uses (returns the count in effect; 1 in the serial
// build)
int oracle_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

}  // extern "C"
