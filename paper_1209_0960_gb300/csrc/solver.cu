// Hierarchy construction, V-cycle, preconditioned CG and the C ABI of libamg
// (Blatt, Ippisch & Bastian, arXiv:1209.0960: Sec. 2 multigrid cycle,
// Sec. 2.1 coarsening, Sec. 5 solver configuration).

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>
#include <tuple>
#include <type_traits>

#include "device.h"

namespace amg {

thread_local std::string t_last_error;

void set_last_error(const std::string& msg) { t_last_error = msg; }

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

void check_params(const amg_params& p) {
    if (!(p.delta > 0.0 && p.delta < 1.0)) throw Error{AMG_EINVAL, "delta must lie in (0, 1)"};
    if (!(p.beta > 0.0 && p.beta < 1.0)) throw Error{AMG_EINVAL, "beta must lie in (0, 1)"};
    if (!(p.omega > 0.0)) throw Error{AMG_EINVAL, "omega must be positive"};
    if (p.s_min < 1 || p.s_max < p.s_min || p.s_max > 64)
        throw Error{AMG_EINVAL, "need 1 <= s_min <= s_max <= 64"};
    if (p.d_max < 1) throw Error{AMG_EINVAL, "d_max must be >= 1"};
    if (p.max_levels < 1 || p.max_levels > 64) throw Error{AMG_EINVAL, "max_levels must be in 1..64"};
    if (p.dense_cap < 1 || p.dense_cap > 16384) throw Error{AMG_EINVAL, "dense_cap must be in 1..16384"};
    if (!(p.min_coarsen_rate >= 1.0)) throw Error{AMG_EINVAL, "min_coarsen_rate must be >= 1"};
    if (p.precision != AMG_FP64 && p.precision != AMG_FP32_IN_FP64)
        throw Error{AMG_EINVAL, "precision must be AMG_FP64 or AMG_FP32_IN_FP64"};
    if (p.launch_overlap != 0 && p.launch_overlap != 1)
        throw Error{AMG_EINVAL, "launch_overlap must be 0 or 1"};
    if (p.aggregation_tile < 0) throw Error{AMG_EINVAL, "aggregation_tile must be >= 0"};
    if (p.aggregation_device != 0 && p.aggregation_device != 1)
        throw Error{AMG_EINVAL, "aggregation_device must be 0 or 1"};
    if (p.autotune != 0 && p.autotune != 1) throw Error{AMG_EINVAL, "autotune must be 0 or 1"};
    if (p.coarsest_fp32 != 0 && p.coarsest_fp32 != 1)
        throw Error{AMG_EINVAL, "coarsest_fp32 must be 0 or 1"};
    if (p.device_loop != 0 && p.device_loop != 1) throw Error{AMG_EINVAL, "device_loop must be 0 or 1"};
    if (p.host_threads < 0 || p.host_threads > 256)
        throw Error{AMG_EINVAL, "host_threads must be in [0, 256]"};
}

// aggregation of one level under the parameters (Algorithm 1, or Alg. 4 in
// tiles on host threads or on the device)
AggResult aggregate_level(const HostCsr& A, const DevCsr* Ad, const amg_params& p, cudaStream_t s) {
    if (p.aggregation_tile <= 0) return aggregate(A, p);
    if (p.aggregation_device && Ad) return aggregate_tiles_device(*Ad, p, s);
    const unsigned hw = std::thread::hardware_concurrency();
    const int threads = p.host_threads > 0 ? p.host_threads : (int)std::max(1u, std::min(hw, 64u));
    return aggregate_tiled(A, p, p.aggregation_tile, threads);
}

template <typename T>
void upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
    if (!src.empty())
        AMG_CUDA_TRY(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
}

// Smoothing order of level l: rows sorted by (colour, coarse aggregate index,
// original index).  Aggregates are numbered in the order the greedy front built
// them, so consecutive rows stay spatially close (x gathers hit in cache) and
// the members of one aggregate are contiguous inside each colour.  Rows outside
// every aggregate come last inside their colour.  (Ordering the rows of each
// 256-row window by length, to cut the padding of the sliced layout, was
// measured slower on the 512^3 anisotropic workload: the coarse levels lost
// more to the scattered restriction and gathers than the staging saved.)
// Two stable counting sorts (by aggregate, then by colour) give that order in
// O(n + aggregates + colours); a comparison sort of the 134M rows of a 512^3
// level took about 20 s of setup.
std::vector<int32_t> smoothing_order(const HostLevel& h) {
    const int32_t n = h.A.n;
    const int32_t nc = h.agg.nc, ncol = h.ncolours;
    const std::vector<int32_t>& agg = h.agg.agg;
    const std::vector<int32_t>& colour = h.colour;
    auto slot = [&](int32_t i) { return agg[i] >= 0 ? agg[i] : nc; };   // unaggregated last
    std::vector<int32_t> by_agg(n), cnt((size_t)std::max(nc, ncol) + 2, 0);
    for (int32_t i = 0; i < n; ++i) ++cnt[slot(i) + 1];
    for (int32_t q = 0; q <= nc; ++q) cnt[q + 1] += cnt[q];
    for (int32_t i = 0; i < n; ++i) by_agg[cnt[slot(i)]++] = i;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int32_t i = 0; i < n; ++i) ++cnt[colour[i] + 1];
    for (int32_t q = 0; q < ncol; ++q) cnt[q + 1] += cnt[q];
    std::vector<int32_t> perm(n);
    for (int32_t i : by_agg) perm[i] = cnt[colour[i]]++;
    return perm;
}

// Modelled (algorithmic) DRAM bytes of the V-cycle passes: every stored entry
// and vector element a pass needs is counted once; neighbour values gathered
// several times are counted once (they are served from cache).  v = bytes of a
// value, 4 per index, 2 per row length.

// colour pass over the m rows of colour col (z entries) reading neighbour
// values at positions < jmax: entries, lengths, b, 1/A_ii, x written, and the
// neighbour values once
double pass_bytes(const DevLevel& L, int col, int jmax, int vb) {
    const double m = L.cptr[col + 1] - L.cptr[col];
    const double z = (double)L.cnnz[col];
    const double nb = std::min(z, (double)jmax - (jmax > L.cptr[col] ? m : 0.0));
    return z * (vb + 4) + m * (2 + 3.0 * vb) + std::max(0.0, nb) * vb;
}
// fused first two forward passes: colour 0 reads b and 1/A_ii and writes x;
// colour 1 reads its entries, b, 1/A_ii, writes x (colour-0 b and 1/A_ii are
// already counted); the next level's right-hand side is zeroed when the
// restriction is fused
double first_bytes(const DevLevel& L, int vb) {
    const double c1 = L.cptr[1];
    const double m1 = L.ncolours > 1 ? L.cptr[2] - L.cptr[1] : 0.0;
    const double z1 = L.ncolours > 1 ? (double)L.cnnz[1] : 0.0;
    return c1 * 3.0 * vb + z1 * (vb + 4) + m1 * (2 + 3.0 * vb) +
           (L.fused_restrict ? (double)L.n_coarse * vb : 0.0);
}
// residual of the rows of colour >= 1 and restriction: entries, lengths, A_ii,
// b, own x, colour-0 neighbour values once, then either the coarse index (and
// weight) and one atomic add per aggregate (fused) or the written r, the
// restriction lists, r again and the coarse right-hand side
double residual_restrict_bytes(const DevLevel& L, int vb, bool scaled) {
    const double m = L.n - L.cptr[1];
    const double z = (double)(L.nnz_off - L.cnnz[0]);
    const double core = z * (vb + 4) + m * (2 + 3.0 * vb) + std::min(z, (double)L.cptr[1]) * vb;
    if (L.fused_restrict) return core + m * (4 + (scaled ? 4 : 0)) + (double)L.n_coarse * 2 * vb;
    return core + m * vb + m * (4 + vb + (scaled ? 4 : 0)) + 4.0 * (L.n_coarse + 1) +
           (double)L.n_coarse * vb;
}
double prolong_bytes(const DevLevel& L, int vb, bool scaled) {
    const double m = L.n - L.cptr[1];
    return m * (4 + 2.0 * vb + (scaled ? 4 : 0)) + (double)L.n_coarse * vb;
}

// modelled bytes of one V-cycle on a level, following the pass sequence of
// vcycle64/vcycle32; the coarsest level reads its dense inverse once
// mb: bytes per entry of the coarsest inverse as applied (8, or 4 for its
// float32 copy in the float32 V-cycle)
double level_vcycle_bytes(const DevLevel& L, bool coarsest, int vb, int mb = 8) {
    if (coarsest) return (double)L.n * L.n * mb + 2.0 * L.n * vb;
    const bool scaled = vb == 4;
    const int C = L.ncolours;
    double t = first_bytes(L, vb);
    for (int col = 2; col < C; ++col) t += pass_bytes(L, col, L.cptr[col], vb);
    for (int col = C - 2; col >= 0; --col) t += pass_bytes(L, col, L.n, vb);
    t += residual_restrict_bytes(L, vb, scaled);
    t += prolong_bytes(L, vb, scaled);
    for (int col = 0; col < C; ++col) t += pass_bytes(L, col, L.n, vb);
    for (int col = C - 2; col >= 0; --col) t += pass_bytes(L, col, L.n, vb);
    return t;
}

void fill_info(amg_ctx* c) {
    const int L = (int)c->dl.size();
    c->linfo.assign(L, amg_level_info{});
    double b64 = 0, b32 = 0, nnz0 = 0, nnzs = 0;
    for (int l = 0; l < L; ++l) {
        const auto& h = c->hl[l];
        const auto& d = c->dl[l];
        amg_level_info& li = c->linfo[l];
        li.n = h.A.n;
        li.nnz = (int32_t)h.A.nnz();
        const bool last = l == L - 1;
        li.n_coarse = last ? 0 : h.agg.nc;
        li.ncolours = last ? 0 : h.ncolours;
        li.max_agg_size = last ? 0 : h.agg.max_size;
        li.n_isolated = last ? 0 : h.agg.n_isolated;
        li.n_dirichlet = last ? 0 : h.agg.n_dirichlet;
        li.vcycle_bytes_fp64 = level_vcycle_bytes(d, last, 8);
        li.vcycle_bytes_fp32 = level_vcycle_bytes(d, last, 4, c->p.coarsest_fp32 ? 4 : 8);
        li.lanes_per_row = last ? 0 : d.lpr;
        li.threads_per_block = last ? 0 : d.block;
        li.sweep = (!last && d.sweep) ? 1 : 0;
        li.carveout = last ? -1 : d.carve;
        li.compact = d.soff ? 1 : 0;
        li.staged_entries = d.soff ? d.stage_entries : d.padded;
        b64 += li.vcycle_bytes_fp64;
        b32 += li.vcycle_bytes_fp32;
        if (l == 0) nnz0 = li.nnz;
        nnzs += li.nnz;
    }
    c->summary.num_levels = L;
    c->summary.coarsest_n = c->nL;
    c->summary.operator_complexity = nnzs / nnz0;
    c->summary.vcycle_bytes_fp64 = b64;
    c->summary.vcycle_bytes_fp32 = b32;
    // CG outside the V-cycle, float64 level-0 vectors: SpMV q = A p (matrix,
    // read p, write q), update x, r (read x, p, r, q; write x, r), r.z (read
    // r, z), p = z + beta p (read z, p; write p)
    const DevLevel& d0 = c->dl[0];
    const double n = d0.n;
    const double M64 = d0.nnz_off * 12.0 + 2.0 * n + 8.0 * n;
    const double cg = (M64 + 16.0 * n) + 48.0 * n + 16.0 * n + 24.0 * n;
    c->summary.pcg_iter_bytes_fp64 = cg + b64;
    c->summary.pcg_iter_bytes_fp32 = cg + b32 + 8.0 * n * 3;  // conversions in and out
}

// ---------------------------------------------------------------------------
// launch profiler: CUDA events around launches, grouped by kernel class, with
// the modelled algorithmic DRAM bytes of each launch
// ---------------------------------------------------------------------------
const char* kKindNames[kKGraphFrom] = {
    "gs_level0", "gs_coarse", "residual_level0", "residual_coarse", "restrict", "prolong",
    "coarse_solve", "first_level0", "gs_prolong_level0", "cg_spmv_dot", "cg_update_dot", "cg_dot", "cg_p_update", "convert",
    "zero", "permute", "graph_cg_part", "graph_vcycle_part"};

struct ProfScope {
    amg_ctx* c;
    int idx = -1;
    ProfScope(amg_ctx* c_, int kind, double bytes, bool graph_level = false) : c(c_) {
        Profiler& P = c->prof;
        const bool rec = graph_level ? P.graphs : P.on;
        if (!rec) return;
        if (P.next + 2 > (int)P.events.size() && !grow(P)) return;
        idx = P.next;
        P.next += 2;
        cudaEventRecord(P.events[idx], c->stream);
        P.recs.push_back({kind, bytes, idx});
    }
    ~ProfScope() {
        if (idx >= 0) cudaEventRecord(c->prof.events[idx + 1], c->stream);
    }
    // a long solve outgrows the event pool: double it (up to 2^21 events),
    // never while the stream is being captured
    bool grow(Profiler& P) {
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return false;
        }
        const size_t old = P.events.size();
        if (old >= (size_t(1) << 21)) return false;
        P.events.resize(std::max<size_t>(2 * old, 1024), nullptr);
        for (size_t k = old; k < P.events.size(); ++k)
            if (cudaEventCreate(&P.events[k]) != cudaSuccess) {
                cudaGetLastError();
                P.events.resize(k & ~size_t(1));
                return P.next + 2 <= (int)P.events.size();
            }
        return true;
    }
};

// ---------------------------------------------------------------------------
// V-cycle (Sec. 2): pre-smooth, restrict the residual, recurse, prolongate
// with omega, post-smooth; dense solve on the coarsest level
// ---------------------------------------------------------------------------
// One V-cycle on level l in precision T (double: FP64 path; float: the scaled
// float32 levels).  Pass sequence on a level with C colours:
//   pre   first (colours 0 and 1 from zero), colours 2..C-1 forward reading
//         only earlier colours, colours C-2..0 backward;
//   restrict the residual of colours >= 1 (colour 0 was smoothed last);
//   recurse; then x += omega P e on colours >= 1 (colour 0 is recomputed
//         by the next pass without reading its old values), then colours
//         0..C-1, C-2..0.
template <typename T>
struct Prec;
template <>
struct Prec<double> {
    static double* x(DevLevel& L) { return L.x; }
    static double* b(DevLevel& L) { return L.b; }
    static double* r(DevLevel& L) { return L.r; }
    static constexpr int vb = 8;
};
template <>
struct Prec<float> {
    static float* x(DevLevel& L) { return L.x32; }
    static float* b(DevLevel& L) { return L.b32; }
    static float* r(DevLevel& L) { return L.r32; }
    static constexpr int vb = 4;
};

inline void k_first(const DevLevel& L, const double* b, double* x, double* bc, int nc, cudaStream_t s) { launch_first(L, b, x, bc, nc, s); }
inline void k_first(const DevLevel& L, const float* b, float* x, float* bc, int nc, cudaStream_t s) { launch_first32(L, b, x, bc, nc, s); }
inline void k_pass(const DevLevel& L, int col, int jmax, const double* b, double* x, cudaStream_t s) { launch_pass(L, col, jmax, b, x, s); }
inline void k_pass(const DevLevel& L, int col, int jmax, const float* b, float* x, cudaStream_t s) { launch_pass32(L, col, jmax, b, x, s); }
inline void k_resres(const DevLevel& L, const double* b, const double* x, double* r, double* bc, cudaStream_t s) { launch_residual_restrict(L, b, x, r, bc, s); }
inline void k_resres(const DevLevel& L, const float* b, const float* x, float* r, float* bc, cudaStream_t s) { launch_residual_restrict32(L, b, x, r, bc, s); }
inline void k_prolong(const DevLevel& L, const double* e, double* x, double w, cudaStream_t s) { launch_prolong(L, e, x, w, s); }
inline void k_prolong(const DevLevel& L, const float* e, float* x, double w, cudaStream_t s) { launch_prolong32(L, e, x, w, s); }
inline void k_sweep(const DevLevel& L, const SweepPlan& P, const double* b, double* x, cudaStream_t s) { launch_sweep(L, P, b, x, s); }
inline void k_sweep(const DevLevel& L, const SweepPlan& P, const float* b, float* x, cudaStream_t s) { launch_sweep32(L, P, b, x, s); }
inline void k_coarsest(amg_ctx* c, const double* b, double* x) { launch_dense_gemv(c->nL, c->Ainv, b, x, c->stream); }
inline void k_coarsest(amg_ctx* c, const float* b, float* x) {
    if (c->Ainv_s32) launch_dense_gemv_f32(c->nL, c->ld32, c->Ainv_s32, b, x, c->stream);
    else launch_dense_gemv32(c->nL, c->Ainv_s, b, x, c->stream);
}

// Position of the next V-cycle launches, for merging the recorded V-cycles
// of several contexts step by step (see VRec): descent of level l (0, l,
// step), ascent (1, 64 - l, step); within a level the first passes take steps
// 0-1, forward colour c step 2 + c, backward colour c step 100 + (C - 2 - c),
// residual and restriction 200-201, prolongation 0 of the ascent.
inline void vkey(int phase, int level, int step) { t_vkey = VKey{phase, level, step}; }

template <typename T>
void vcycle(amg_ctx* c, int l, const T* b, T* x) {
    using P = Prec<T>;
    constexpr int vb = P::vb;
    constexpr bool scaled = vb == 4;
    const int nlev = (int)c->dl.size();
    DevLevel& L = c->dl[l];
    cudaStream_t s = c->stream;
    if (l == nlev - 1) {
        const double mb = (vb == 4 && c->Ainv_s32) ? 4.0 : 8.0;
        ProfScope ps(c, kKCoarseSolve, (double)c->nL * c->nL * mb + 2.0 * vb * c->nL);
        vkey(0, l, 0);
        k_coarsest(c, b, x);
        return;
    }
    DevLevel& N = c->dl[l + 1];
    const int C = L.ncolours;
    const int kind = l == 0 ? kKGsL0 : kKGsCoarse;
    if (L.sweep) {
        // the whole pre-smoother as one dependency-driven kernel
        double bytes = first_bytes(L, vb);
        for (int col = 2; col < C; ++col) bytes += pass_bytes(L, col, L.cptr[col], vb);
        for (int col = C - 2; col >= 0; --col) bytes += pass_bytes(L, col, L.n, vb);
        ProfScope ps(c, kind, bytes);
        k_sweep(L, *L.plan_pre, b, x, s);
    } else {
        {
            ProfScope ps(c, l == 0 ? kKFirstL0 : kKGsCoarse, first_bytes(L, vb));
            vkey(0, l, 0);
            k_first(L, b, x, L.fused_restrict ? P::b(N) : (T*)nullptr, N.n, s);
        }
        for (int col = 2; col < C; ++col) {
            ProfScope ps(c, kind, pass_bytes(L, col, L.cptr[col], vb));
            vkey(0, l, 2 + col);
            k_pass(L, col, L.cptr[col], b, x, s);
        }
        for (int col = C - 2; col >= 0; --col) {
            ProfScope ps(c, kind, pass_bytes(L, col, L.n, vb));
            vkey(0, l, 100 + (C - 2 - col));
            k_pass(L, col, L.n, b, x, s);
        }
    }
    {
        ProfScope ps(c, l == 0 ? kKResidualL0 : kKResidualCoarse, residual_restrict_bytes(L, vb, scaled));
        vkey(0, l, 200);
        k_resres(L, b, x, P::r(L), P::b(N), s);
    }
    vcycle<T>(c, l + 1, P::b(N), P::x(N));
    {
        ProfScope ps(c, kKProlong, prolong_bytes(L, vb, scaled));
        vkey(1, 64 - l, 0);
        k_prolong(L, P::x(N), x, c->p.omega, s);
    }
    if (L.sweep) {
        // the whole post-smoother as one dependency-driven kernel
        double bytes = 0.0;
        for (int col = 0; col < C; ++col) bytes += pass_bytes(L, col, L.n, vb);
        for (int col = C - 2; col >= 0; --col) bytes += pass_bytes(L, col, L.n, vb);
        ProfScope ps(c, kind, bytes);
        k_sweep(L, *L.plan_post, b, x, s);
        return;
    }
    for (int col = 0; col < C; ++col) {
        ProfScope ps(c, kind, pass_bytes(L, col, L.n, vb));
        vkey(1, 64 - l, 2 + col);
        k_pass(L, col, L.n, b, x, s);
    }
    for (int col = C - 2; col >= 0; --col) {
        ProfScope ps(c, kind, pass_bytes(L, col, L.n, vb));
        vkey(1, 64 - l, 100 + (C - 2 - col));
        k_pass(L, col, L.n, b, x, s);
    }
}

void vcycle64(amg_ctx* c, int l, const double* b, double* x) { vcycle<double>(c, l, b, x); }
void vcycle32(amg_ctx* c, int l, const float* b, float* x) { vcycle<float>(c, l, b, x); }

// The float32 V-cycle with its float64 entry and exit folded into the
// fine-level passes: the first pass forms b = r / s itself, and the last
// pass over each colour writes z = x / s (same values as separate conversion
// kernels, two launches and a vector round trip fewer).
void vcycle32_fused(amg_ctx* c, const double* r, double* z) {
    DevLevel& L = c->dl[0];
    DevLevel& N = c->dl[1];
    cudaStream_t s = c->stream;
    const int C = L.ncolours;
    const double* isq = c->isq0;
    float* b = L.b32;
    float* x = L.x32;
    {
        ProfScope ps(c, kKFirstL0, first_bytes(L, 4) + 12.0 * L.n);
        vkey(0, 0, 0);
        launch_first32_from64(L, r, isq, b, x, L.fused_restrict ? N.b32 : nullptr, N.n, s);
    }
    for (int col = 2; col < C; ++col) {
        ProfScope ps(c, kKGsL0, pass_bytes(L, col, L.cptr[col], 4));
        vkey(0, 0, 2 + col);
        launch_pass32(L, col, L.cptr[col], b, x, s);
    }
    for (int col = C - 2; col >= 0; --col) {
        ProfScope ps(c, kKGsL0, pass_bytes(L, col, L.n, 4));
        vkey(0, 0, 100 + (C - 2 - col));
        launch_pass32(L, col, L.n, b, x, s);
    }
    {
        ProfScope ps(c, kKResidualL0, residual_restrict_bytes(L, 4, true));
        vkey(0, 0, 200);
        launch_residual_restrict32(L, b, x, L.r32, N.b32, s);
    }
    vcycle32(c, 1, N.b32, N.x32);
    {
        ProfScope ps(c, kKProlong, prolong_bytes(L, 4, true));
        vkey(1, 64, 0);
        launch_prolong32(L, N.x32, x, c->p.omega, s);
    }
    // the last pass over each colour also writes z
    for (int col = 0; col < C; ++col) {
        const bool last = col == C - 1;
        ProfScope ps(c, kKGsL0, pass_bytes(L, col, L.n, 4) + (last ? 16.0 * (L.cptr[col + 1] - L.cptr[col]) : 0.0));
        vkey(1, 64, 2 + col);
        if (last) launch_pass32_to64(L, col, L.n, b, x, z, isq, s);
        else launch_pass32(L, col, L.n, b, x, s);
    }
    for (int col = C - 2; col >= 0; --col) {
        ProfScope ps(c, kKGsL0, pass_bytes(L, col, L.n, 4) + 16.0 * (L.cptr[col + 1] - L.cptr[col]));
        vkey(1, 64, 100 + (C - 2 - col));
        launch_pass32_to64(L, col, L.n, b, x, z, isq, s);
    }
}

// z = B r on level 0 (smoothing order) in the context's precision
void precondition(amg_ctx* c, const double* r, double* z) {
    if (c->precision == AMG_FP64) {
        vcycle64(c, 0, r, z);
    } else if (c->dl.size() > 1 && c->dl[0].lpr == 0 && c->dl[0].ncolours == 2) {
        // (two colours: the first pass covers every row, so it can form all of b)
        vcycle32_fused(c, r, z);
    } else {
        DevLevel& L0 = c->dl[0];
        {
            ProfScope ps(c, kKConvert, 20.0 * L0.n);
            vkey(-1, 0, 0);
            launch_to_scaled32(L0.n, r, c->isq0, L0.b32, c->stream);
        }
        vcycle32(c, 0, L0.b32, L0.x32);
        {
            ProfScope ps(c, kKConvert, 20.0 * L0.n);
            vkey(2, 0, 0);
            launch_from_scaled32(L0.n, L0.x32, c->isq0, z, c->stream);
        }
    }
    AMG_CUDA_TRY(cudaGetLastError());
}

void ensure_fp32(amg_ctx* c) {
    if (c->fp32_ready) return;
    const int nlev = (int)c->dl.size();
    for (int l = 0; l < nlev; ++l) {
        DevLevel& L = c->dl[l];
        const double* cdiag = (l + 1 < nlev) ? c->dl[l + 1].diag : nullptr;
        build_level_fp32(L, cdiag, c->mem, c->stream);
    }
    c->Ainv_s = c->mem.alloc<double>((size_t)c->nL * c->nL);
    scale_inverse_device(c->nL, c->dl[nlev - 1].diag, c->Ainv, c->Ainv_s, c->stream);
    if (c->p.coarsest_fp32) {
        c->ld32 = (c->nL + 3) & ~3;
        c->Ainv_s32 = c->mem.alloc<float>((size_t)c->nL * c->ld32);
        to_float_padded_device(c->nL, c->ld32, c->Ainv_s, c->Ainv_s32, c->stream);
    }
    AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->fp32_ready = true;
}

// Order the context stream after the caller's stream (enter) and the
// caller's stream after the context stream (leave).
void enter(amg_ctx* c) {
    t_launch_overlap = c->p.launch_overlap != 0;
    AMG_CUDA_TRY(cudaEventRecord(c->ev_in, c->user_stream));
    AMG_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
}
void leave(amg_ctx* c) {
    AMG_CUDA_TRY(cudaEventRecord(c->ev_out, c->stream));
    AMG_CUDA_TRY(cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
}

// Capture the launches issued by f on the context stream into an executable
// graph.
template <typename F>
cudaGraphExec_t capture_graph(amg_ctx* c, F&& f) {
    AMG_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t g = nullptr;
    try {
        f();
    } catch (...) {
        cudaStreamEndCapture(c->stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    AMG_CUDA_TRY(cudaStreamEndCapture(c->stream, &g));
    cudaGraphExec_t e = nullptr;
    cudaError_t err = cudaGraphInstantiate(&e, g, 0);
    cudaGraphDestroy(g);
    AMG_CUDA_TRY(err);
    return e;
}

// ---------------------------------------------------------------------------
// launch shapes: fixed rules at setup, optional autotuning
// ---------------------------------------------------------------------------

void drop_graphs(amg_ctx* c) {
    for (int a = 0; a < 2; ++a) {
        for (int b = 0; b < 2; ++b) {
            if (c->graph_a[a][b]) cudaGraphExecDestroy(c->graph_a[a][b]);
            if (c->graph_b[a][b]) cudaGraphExecDestroy(c->graph_b[a][b]);
            if (c->graph_solve[a][b]) cudaGraphExecDestroy(c->graph_solve[a][b]);
            c->graph_a[a][b] = c->graph_b[a][b] = c->graph_solve[a][b] = nullptr;
            c->solve_graph_state[a][b] = 0;
        }
        c->vrec_ok[a] = false;
        if (c->graph_bi[a]) cudaGraphExecDestroy(c->graph_bi[a]);
        c->graph_bi[a] = nullptr;
        c->bi_graph_state[a] = 0;
        for (cudaGraphExec_t& g : c->graph_from[a]) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    }
}

constexpr int kStaged = 0;   // DevLevel::lpr of the staged one-row-per-thread kernels

// A launch shape as one code: lanes per row (0 = staged kernels, 1, 2, 4 or
// 8) plus kHalfBlock for blocks of 128 instead of 256 threads (row kernels
// only), plus kSweep for smoothing sweeps run as one dependency-driven kernel
// each (lane shapes only), plus (staged kernels only) the preferred
// shared-memory carveout + 1 in the bits from kCarveShift (0: the driver's).
constexpr int kHalfBlock = 16;
constexpr int kSweep = 32;
constexpr int kCarveShift = 8;
constexpr int kCarveMask = 0x7f << kCarveShift;
// sweeps are planned on the host from the level's graph (adjacency of every
// item): kept to levels where a pass is short
constexpr int32_t kSweepMaxRows = 1 << 20;
inline int shape_lanes(int code) { return code & (kHalfBlock - 1); }
inline int shape_block(int code) { return (code & kHalfBlock) ? 128 : 256; }
inline int shape_carve(int code) { return ((code & kCarveMask) >> kCarveShift) - 1; }
inline int with_carve(int code, int carve) { return (code & ~kCarveMask) | ((carve + 1) << kCarveShift); }

bool shape_allowed(const DevLevel& L, int code) {
    const int lanes = shape_lanes(code);
    if (code & ~(kSweep | kHalfBlock | (kHalfBlock - 1) | kCarveMask)) return false;
    if (shape_carve(code) > 100) return false;
    if (lanes == kStaged) return (code & ~kCarveMask) == kStaged && staged_fits(L);
    if (code & kCarveMask) return false;
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) return false;
    if (code & kSweep)
        return !L.fused_ok && L.ncolours >= 2 && 2 * L.ncolours - 1 <= kSweepMaxPasses &&
               L.n <= kSweepMaxRows;
    return true;
}

int shape_of(const DevLevel& L) {
    const int code = L.lpr | (L.block == 128 ? kHalfBlock : 0) | (L.sweep ? kSweep : 0);
    return L.lpr == kStaged && L.carve >= 0 ? with_carve(code, L.carve) : code;
}

// The dependency plan of one sweep of level l (see SweepPlan) for items of
// `rows` rows: pre = the pre-smoother (colour 0 from zero, colours 1..C-1
// forward reading only earlier colours, C-2..0 backward), else the
// post-smoother (0..C-1, C-2..0).  Uploaded into the context's memory.
void plan_sweep(amg_ctx* c, int l, int rows, bool pre, SweepPlan& P) {
    const HostLevel& h = c->hl[l];
    const DevLevel& L = c->dl[l];
    const int32_t n = L.n;
    const int C = L.ncolours;
    std::vector<int32_t> colr(n), tiles(C), tile0(C + 1, 0);
    for (int col = 0; col < C; ++col) {
        for (int32_t r = L.cptr[col]; r < L.cptr[col + 1]; ++r) colr[r] = col;
        const int32_t base = L.cptr[col] & ~31;
        tiles[col] = L.cptr[col + 1] > L.cptr[col] ? (L.cptr[col + 1] - base + rows - 1) / rows : 0;
        tile0[col + 1] = tile0[col] + tiles[col];
    }
    auto gtile = [&](int32_t r) {
        const int col = colr[r];
        return tile0[col] + (r - (L.cptr[col] & ~31)) / rows;
    };
    // tiles holding neighbours of each tile's rows
    std::vector<int32_t> inv(n);
    for (int32_t i = 0; i < n; ++i) inv[h.perm[i]] = i;
    std::vector<std::vector<int32_t>> adj(tile0[C]);
    for (int32_t r = 0; r < n; ++r) {
        const int32_t i = inv[r];
        std::vector<int32_t>& a = adj[gtile(r)];
        for (int32_t k = h.A.rp[i]; k < h.A.rp[i + 1]; ++k)
            if (h.A.ci[k] != i) a.push_back(gtile(h.perm[h.A.ci[k]]));
    }
    for (auto& a : adj) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    // the passes, and the colour of each
    std::vector<SweepPass> pass;
    std::vector<int> pcol;
    auto add = [&](int col, int32_t jmax, int first) {
        if (tiles[col] == 0) return;
        SweepPass q;
        q.r0 = L.cptr[col];
        q.r1 = L.cptr[col + 1];
        q.jmax = jmax;
        q.first = first;
        q.tiles = tiles[col];
        q.item0 = pass.empty() ? 0 : pass.back().item0 + pass.back().tiles;
        pass.push_back(q);
        pcol.push_back(col);
    };
    for (int col = 0; col < C; ++col) {
        if (pre) add(col, col == 0 ? 0 : L.cptr[col], col == 0 ? 1 : 0);
        else add(col, n, 0);
    }
    for (int col = C - 2; col >= 0; --col) add(col, n, 0);
    const int np = (int)pass.size();
    if (np > kSweepMaxPasses) throw Error{AMG_EINVAL, "too many colour passes for a sweep kernel"};
    const int32_t items = np ? pass.back().item0 + pass.back().tiles : 0;
    // dependencies of every item, in item order
    std::vector<int32_t> dep_ptr(1, 0), dep;
    for (int p = 0; p < np; ++p) {
        const int col = pcol[p];
        int prev = -1;
        for (int q = p - 1; q >= 0; --q)
            if (pcol[q] == col) {
                prev = q;
                break;
            }
        for (int32_t t = 0; t < pass[p].tiles; ++t) {
            if (prev >= 0) dep.push_back(pass[prev].item0 + t);
            for (int q = prev + 1; q < p; ++q) {
                if (q < p - 1) {
                    dep.push_back(-(q + 1));
                    continue;
                }
                const int qc = pcol[q];
                for (int32_t g : adj[tile0[col] + t])
                    if (g >= tile0[qc] && g < tile0[qc + 1])
                        dep.push_back(pass[q].item0 + (g - tile0[qc]));
            }
            dep_ptr.push_back((int32_t)dep.size());
        }
    }
    cudaStream_t s = c->stream;
    P.rows = rows;
    P.npass = np;
    P.items = items;
    P.mean_deps = items ? (double)dep.size() / items : 0.0;
    P.pass = c->mem.alloc<SweepPass>(std::max(np, 1));
    P.dep_ptr = c->mem.alloc<int32_t>(dep_ptr.size());
    P.dep = c->mem.alloc<int32_t>(std::max<size_t>(dep.size(), 1));
    P.flag = c->mem.alloc<uint32_t>(std::max(items, 1));
    P.done = c->mem.alloc<unsigned long long>(std::max(np, 1));
    P.arrive = c->mem.alloc<unsigned long long>(1);
    P.grid = std::min(items, sweep_grid(L.lpr, L.block));
    P.failed = c->mem.alloc<int32_t>(1);
    upload(P.pass, pass, s);
    upload(P.dep_ptr, dep_ptr, s);
    upload(P.dep, dep, s);
    AMG_CUDA_TRY(cudaMemsetAsync(P.flag, 0, sizeof(uint32_t) * std::max(items, 1), s));
    AMG_CUDA_TRY(cudaMemsetAsync(P.done, 0, sizeof(unsigned long long) * std::max(np, 1), s));
    AMG_CUDA_TRY(cudaMemsetAsync(P.arrive, 0, sizeof(unsigned long long), s));
    AMG_CUDA_TRY(cudaMemsetAsync(P.failed, 0, sizeof(int32_t), s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));   // the host vectors go out of scope
}

void set_shape(amg_ctx* c, int l, int code) {
    DevLevel& L = c->dl[l];
    const int lanes = shape_lanes(code);
    L.lpr = lanes;
    L.lpr_wide = lanes;
    L.block = shape_block(code);
    L.fused_restrict = lanes == kStaged && L.fused_ok;
    L.sweep = (code & kSweep) != 0 && lanes >= 1;
    L.carve = lanes == kStaged ? shape_carve(code) : -1;
    L.plan_pre = L.plan_post = nullptr;
    if (L.sweep) {
        // the plan (items, and the cooperative grid) depends on lanes and block
        const int rows = L.block / lanes;
        auto& pp = c->sweep_plans[std::make_pair(l, lanes + 16 * L.block)];
        if (pp.first.rows == 0) {
            plan_sweep(c, l, rows, true, pp.first);
            plan_sweep(c, l, rows, false, pp.second);
        }
        L.plan_pre = &pp.first;
        L.plan_post = &pp.second;
    }
}

// Level signature for the process-wide cache of tuned shapes: levels that
// agree on it run the same kernels over similar slices.
struct ShapeKey {
    int precision, size_class, width_class, mean, ncolours, fine;
    bool operator<(const ShapeKey& o) const {
        return std::tie(precision, size_class, width_class, mean, ncolours, fine) <
               std::tie(o.precision, o.size_class, o.width_class, o.mean, o.ncolours, o.fine);
    }
};

ShapeKey shape_key(const amg_ctx* c, int l) {
    const DevLevel& L = c->dl[l];
    // octave size classes, slice widths in steps of 4, whole mean row lengths:
    // coarse enough that requests of similar grids share their tuning
    const int size_class = (int)std::floor(std::log2(std::max(1, L.n)));
    const int mean = (int)std::lround((double)L.nnz_off / std::max(1, L.n));
    return {c->precision, size_class, (L.width + 3) / 4, mean, L.ncolours, l == 0 ? 1 : 0};
}

std::mutex g_shape_mu;
std::map<ShapeKey, int> g_shape_cache;

// Device time of one replay of the V-cycle from level l (the whole
// preconditioner for l = 0), as a CUDA graph: the minimum over three batches
// sized to about 0.3 ms each.
double time_vcycle_from(amg_ctx* c, int l) {
    cudaStream_t s = c->stream;
    cudaGraphExec_t g = capture_graph(c, [&] {
        if (l == 0) precondition(c, c->r, c->z);
        else if (c->precision == AMG_FP64) vcycle64(c, l, c->dl[l].b, c->dl[l].x);
        else vcycle32(c, l, c->dl[l].b32, c->dl[l].x32);
    });
    struct GraphGuard {
        cudaGraphExec_t g;
        ~GraphGuard() { cudaGraphExecDestroy(g); }
    } guard{g};
    float ms = 0.f;
    AMG_CUDA_TRY(cudaGraphLaunch(g, s));   // warm-up
    AMG_CUDA_TRY(cudaEventRecord(c->ev0, s));
    AMG_CUDA_TRY(cudaGraphLaunch(g, s));
    AMG_CUDA_TRY(cudaEventRecord(c->ev1, s));
    AMG_CUDA_TRY(cudaEventSynchronize(c->ev1));
    AMG_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    const int reps = std::max(1, std::min(64, (int)std::ceil(0.3 / std::max(1e-3, (double)ms))));
    double best = 1e30;
    for (int batch = 0; batch < 3; ++batch) {
        AMG_CUDA_TRY(cudaEventRecord(c->ev0, s));
        for (int r = 0; r < reps; ++r) AMG_CUDA_TRY(cudaGraphLaunch(g, s));
        AMG_CUDA_TRY(cudaEventRecord(c->ev1, s));
        AMG_CUDA_TRY(cudaEventSynchronize(c->ev1));
        AMG_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        best = std::min(best, (double)ms / reps);
    }
    return best;
}

// Pick each level's shape by timing, coarse levels first, so that the
// V-cycle below the level being tuned already runs its final shapes.  The
// rule's shape is kept unless a candidate is more than 3 % faster, which keeps
// the choice stable against timing noise.  Returns the milliseconds spent.
double autotune_shapes(amg_ctx* c) {
    NvtxRange nvtx("autotune");
    const int nlev = (int)c->dl.size();
    if (nlev < 2) return 0.0;
    const double t0 = now_ms();
    cudaStream_t s = c->stream;
    bool timed = false;
    auto zero_inputs = [&] {
        // zero right-hand sides: the kernels do the same work for any values
        AMG_CUDA_TRY(cudaMemsetAsync(c->r, 0, sizeof(double) * c->dl[0].n, s));
        for (DevLevel& L : c->dl) {
            AMG_CUDA_TRY(cudaMemsetAsync(L.b, 0, sizeof(double) * L.n, s));
            if (L.b32) AMG_CUDA_TRY(cudaMemsetAsync(L.b32, 0, sizeof(float) * L.n, s));
        }
    };
    for (int l = nlev - 2; l >= 0; --l) {
        DevLevel& L = c->dl[l];
        const ShapeKey key = shape_key(c, l);
        {
            std::lock_guard<std::mutex> lk(g_shape_mu);
            auto it = g_shape_cache.find(key);
            if (it != g_shape_cache.end() && shape_allowed(L, it->second)) {
                set_shape(c, l, it->second);
                continue;
            }
        }
        if (!timed) {
            zero_inputs();
            timed = true;
        }
        const int rule = L.lpr;
        double t_rule = 1e30, t_best = 1e30;
        int best = rule;
        // staged kernels also with a smaller shared-memory carveout (percent
        // of the maximum 228 KB: 100, 132 or 164 KB), leaving more L1 for the
        // neighbour gathers
        for (int lanes : {kStaged, with_carve(kStaged, 44), with_carve(kStaged, 58),
                          with_carve(kStaged, 72), 1, 1 | kHalfBlock, 2, 2 | kHalfBlock, 4,
                          4 | kHalfBlock, 8, 8 | kHalfBlock, 2 | kSweep, 2 | kHalfBlock | kSweep,
                          4 | kSweep, 4 | kHalfBlock | kSweep, 8 | kSweep, 8 | kHalfBlock | kSweep}) {
            if (!shape_allowed(L, lanes)) continue;
            set_shape(c, l, lanes);
            const double t = time_vcycle_from(c, l);
            if (lanes == rule) t_rule = t;
            if (t < t_best) {
                t_best = t;
                best = lanes;
            }
        }
        if (t_rule <= 1.03 * t_best) best = rule;
        // a context tuning the same signature concurrently may have stored
        // its choice first: every context then runs the stored one
        std::lock_guard<std::mutex> lk(g_shape_mu);
        const int stored = g_shape_cache.emplace(key, best).first->second;
        set_shape(c, l, shape_allowed(L, stored) ? stored : best);
    }
    for (int l = 0; l + 1 < nlev; ++l) c->shapes[c->precision][l] = shape_of(c->dl[l]);
    c->tuned[c->precision] = true;
    drop_graphs(c);
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return timed ? now_ms() - t0 : 0.0;
}

// Make the levels run the shapes of the context's precision.
void apply_shapes(amg_ctx* c) {
    for (int l = 0; l + 1 < (int)c->dl.size(); ++l) set_shape(c, l, c->shapes[c->precision][l]);
}

// ---------------------------------------------------------------------------
// preconditioned CG on level-0 vectors in smoothing order (c->bb, c->x)
// ---------------------------------------------------------------------------

// One CG iteration is two parts.  A: q = A p, alpha, x/r update, copy of the
// CG scalars to the host.  B: z = B r, beta, p update.
void cg_part_a(amg_ctx* c, bool copy_back = true) {
    DevLevel& L0 = c->dl[0];
    const int n = L0.n;
    cudaStream_t s = c->stream;
    {
        ProfScope ps(c, kKCgSpmv, (double)L0.nnz_off * 12 + 2.0 * n + 24.0 * n);
        launch_cg_spmv_pq(L0, c->pv, c->q, c->work, s);
    }
    {
        ProfScope ps(c, kKCgUpdate, 48.0 * n);
        launch_cg_update(n, c->x, c->r, c->pv, c->q, c->work, s);
    }
    if (copy_back)
        AMG_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->work.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
}

void cg_part_b(amg_ctx* c) {
    const int n = c->dl[0].n;
    cudaStream_t s = c->stream;
    precondition(c, c->r, c->z);
    {
        ProfScope ps(c, kKCgDot, (c->flexible ? 24.0 : 16.0) * n);
        launch_cg_rz(n, c->r, c->z, c->zold, c->pv, c->work, c->flexible ? kRZFlex : kRZ, s);
    }
    {
        ProfScope ps(c, kKCgP, (c->flexible ? 32.0 : 24.0) * n);
        launch_cg_p(n, c->z, c->pv, c->flexible ? c->zold : nullptr, c->work, s);
    }
}

bool cg_graphs(const amg_ctx* c) { return c->use_graphs && !c->prof.on; }

void run_part_a(amg_ctx* c) {
    if (!cg_graphs(c)) return cg_part_a(c);
    cudaGraphExec_t& ga = c->graph_a[c->precision][c->flexible];
    if (!ga) ga = capture_graph(c, [&] { cg_part_a(c); });
    ProfScope ps(c, kKGraphA, 0.0, true);
    AMG_CUDA_TRY(cudaGraphLaunch(ga, c->stream));
}

void run_part_b(amg_ctx* c) {
    if (!cg_graphs(c)) return cg_part_b(c);
    cudaGraphExec_t& gb = c->graph_b[c->precision][c->flexible];
    if (!gb) gb = capture_graph(c, [&] { cg_part_b(c); });
    ProfScope ps(c, kKGraphB, 0.0, true);
    AMG_CUDA_TRY(cudaGraphLaunch(gb, c->stream));
}

// CG start: scalars to the device, r = b - A x, ||r||^2 and the scalars back
void cg_start(amg_ctx* c, double tol, int32_t maxit) {
    cudaStream_t s = c->stream;
    PcgScalars init{};
    init.tol2 = tol * tol;
    init.flexible = c->flexible;
    init.maxit = maxit;
    *c->sc_host = init;
    AMG_CUDA_TRY(cudaMemcpyAsync(c->work.sc, c->sc_host, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
    launch_cg_residual(c->dl[0], c->bb, c->x, c->r, c->work, kRR0, nullptr, s);
    AMG_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->work.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
}

// first preconditioning: z = B r, rho = r.z, p = z
void cg_first_direction(amg_ctx* c) {
    const int n = c->dl[0].n;
    cudaStream_t s = c->stream;
    precondition(c, c->r, c->z);
    launch_cg_rz(n, c->r, c->z, nullptr, c->pv, c->work, kRho0, s);
    if (c->flexible)
        AMG_CUDA_TRY(cudaMemcpyAsync(c->zold, c->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
}

// true residual of the final iterate into c->norm_dev
void cg_true_residual(amg_ctx* c) {
    launch_cg_residual(c->dl[0], c->bb, c->x, nullptr, c->work, kStore, c->norm_dev, c->stream);
}

void cg_fill_info(const amg_ctx* c, int status, double rr_true, amg_solve_info* info) {
    const PcgScalars& h = *c->sc_host;
    info->status = status;
    info->iterations = h.iters;
    info->rel_residual = h.rr0 > 0 ? std::sqrt(h.rr / h.rr0) : 0.0;
    info->true_rel_residual = h.rr0 > 0 ? std::sqrt(rr_true / h.rr0) : 0.0;
    info->device_loop = c->last_device_loop;
}

// A Krylov iteration loop as one graph: `pre` on the context stream, then
// `cond(h, stream)` (a one-thread kernel setting the loop condition h from the
// device scalars), then a WHILE node whose body is `body` followed by `cond`
// again, then `post`.  No iteration waits on the host; the scalars come back
// once, in `post`.  Returns nullptr (and clears the error) when the runtime
// refuses the graph.
template <typename Pre, typename Cond, typename Body, typename Post>
cudaGraphExec_t build_while_graph(amg_ctx* c, Pre&& pre, Cond&& cond, Body&& body, Post&& post) {
    if (!c->stream_body)
        AMG_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream_body, cudaStreamNonBlocking));
    cudaStream_t s = c->stream;
    cudaGraph_t g = nullptr;
    bool body_capturing = false;
    const auto fail = [&](cudaError_t e) {
        if (body_capturing) {
            cudaGraph_t b = nullptr;
            cudaStreamEndCapture(c->stream_body, &b);   // the body belongs to g
        }
        c->stream = s;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return e;
    };
    const auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal))) {
        cudaGetLastError();
        return nullptr;
    }
    try {
        pre();
        cudaStreamCaptureStatus st;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edges = nullptr;
        size_t nd = 0;
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, &edges, &nd);
        if (ok(e)) e = cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault);
        if (!ok(e)) { fail(e); return nullptr; }
        cond(h, s);
        e = cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, &edges, &nd);
        cudaGraphNodeParams prm = {};
        prm.type = cudaGraphNodeTypeConditional;
        prm.conditional.handle = h;
        prm.conditional.type = cudaGraphCondTypeWhile;
        prm.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (ok(e)) e = cudaGraphAddNode(&node, cg, deps, edges, nd, &prm);
        if (ok(e)) e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (ok(e)) e = cudaStreamBeginCaptureToGraph(c->stream_body, prm.conditional.phGraph_out[0], nullptr,
                                                     nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (!ok(e)) { fail(e); return nullptr; }
        body_capturing = true;
        c->stream = c->stream_body;
        body();
        cond(h, c->stream);
        c->stream = s;
        cudaGraph_t bg = nullptr;
        e = cudaStreamEndCapture(c->stream_body, &bg);
        body_capturing = false;
        if (!ok(e)) { fail(e); return nullptr; }
        post();
    } catch (const Error&) {
        fail(cudaSuccess);   // a launch the capture refused: the host-driven loop runs
        return nullptr;
    } catch (...) {
        fail(cudaSuccess);
        throw;
    }
    if (!ok(cudaStreamEndCapture(s, &g))) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return nullptr;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (!ok(e)) {
        cudaGetLastError();
        return nullptr;
    }
    return ex;
}

// The iteration loop of PCG as one graph: the first direction (z = B r,
// rho, p = z) and the first update (q = A p, alpha, x, r, ||r||), then a
// WHILE node whose body is one more iteration (z = B r, beta, p; q = A p,
// alpha, x, r, ||r||).  The loop condition kernel runs after each update.
// The launches are those of the host-driven loop, in the same order.
cudaGraphExec_t build_solve_graph(amg_ctx* c) {
    return build_while_graph(
        c,
        [&] {
            cg_first_direction(c);
            cg_part_a(c, false);
        },
        [&](cudaGraphConditionalHandle h, cudaStream_t st) { launch_cg_continue(h, c->work.sc, st); },
        [&] {
            cg_part_b(c);
            cg_part_a(c, false);
        },
        [&] {
            AMG_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->work.sc, sizeof(PcgScalars),
                                         cudaMemcpyDeviceToHost, c->stream));
        });
}

// The solve graph of the context's precision and CG variant, built on first
// use; nullptr when device loops are off, graph-level profiling times the
// iteration parts, or the runtime refused the graph.  Should the runtime
// refuse programmatic dependent launches inside the loop body, the graph is
// built once more with plain stream order.
cudaGraphExec_t solve_graph(amg_ctx* c) {
    if (!c->p.device_loop || !cg_graphs(c) || c->prof.graphs) return nullptr;
    int& state = c->solve_graph_state[c->precision][c->flexible];
    cudaGraphExec_t& ex = c->graph_solve[c->precision][c->flexible];
    if (state == 0) {
        ex = build_solve_graph(c);
        if (!ex && t_launch_overlap) {
            t_launch_overlap = false;
            ex = build_solve_graph(c);
            t_launch_overlap = true;
            if (ex) c->solve_graph_plain = true;
        }
        state = ex ? 1 : -1;
    }
    return ex;
}

int pcg(amg_ctx* c, double tol, int32_t maxit, amg_solve_info* info) {
    cudaStream_t s = c->stream;
    cg_start(c, tol, maxit);
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    int status = c->sc_host->status != 0 ? c->sc_host->status : AMG_OK;
    c->last_device_loop = 0;
    cudaGraphExec_t loop = (!c->sc_host->done && maxit > 0) ? solve_graph(c) : nullptr;
    if (loop) {
        // the whole loop on the device: one launch, one wait
        AMG_CUDA_TRY(cudaGraphLaunch(loop, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        c->last_device_loop = c->solve_graph_plain ? 2 : 1;
        const PcgScalars& h = *c->sc_host;
        if (h.status != 0) status = h.status;
        else if (h.done) status = AMG_OK;
        else if (h.iters >= maxit) status = AMG_ENOTCONV;
        else throw Error{AMG_ECUDA, "device-side CG loop stopped before its condition"};
    } else if (!c->sc_host->done) {
        cg_first_direction(c);
        while (true) {
            if (c->sc_host->iters >= maxit) { status = AMG_ENOTCONV; break; }
            run_part_a(c);
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
            if (c->sc_host->status != 0) { status = c->sc_host->status; break; }
            if (c->sc_host->done) break;
            if (c->sc_host->iters >= maxit) { status = AMG_ENOTCONV; break; }
            run_part_b(c);
        }
        // graph-level profiling: time the V-cycle from each level l >= 1 alone
        // (diagnostic replays after the solve; they rewrite only coarse-level
        // scratch vectors, which the next V-cycle recomputes)
        if (cg_graphs(c) && c->prof.graphs && c->dl.size() > 1) {
            auto& gv = c->graph_from[c->precision];
            gv.resize(c->dl.size(), nullptr);
            for (int l = 1; l < (int)c->dl.size(); ++l) {
                if (!gv[l])
                    gv[l] = capture_graph(c, [&] {
                        if (c->precision == AMG_FP64) vcycle64(c, l, c->dl[l].b, c->dl[l].x);
                        else vcycle32(c, l, c->dl[l].b32, c->dl[l].x32);
                    });
                for (int rep = 0; rep < 10; ++rep) {
                    ProfScope ps(c, kKGraphFrom + l, 0.0, true);
                    AMG_CUDA_TRY(cudaGraphLaunch(gv[l], s));
                }
            }
        }
    }
    AMG_CUDA_TRY(cudaGetLastError());
    if (info) {
        cg_true_residual(c);
        double rr = 0.0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&rr, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        cg_fill_info(c, status, rr, info);
    }
    return status;
}

// ---------------------------------------------------------------------------
// preconditioned BiCGSTAB (Sec. 5: the Krylov method of the paper's
// experiments), two V-cycles per iteration; vectors in smoothing order
// (c->bb = b, c->x = x0 in, x out).  The scalars live on the device (the
// reductions form alpha, w, rho and the convergence tests), so one iteration
// is a fixed sequence of launches: by default the whole loop runs as one graph
// with a device-side WHILE node; the host-driven loop (profiling, or a
// refused graph) reads the scalars back once per iteration.
// ---------------------------------------------------------------------------
void bi_iteration(amg_ctx* c) {
    DevLevel& L0 = c->dl[0];
    const int n = L0.n;
    cudaStream_t s = c->stream;
    double* x = c->x;
    double* r = c->r;
    double* p = c->pv;
    double* z = c->z;
    launch_bi_direction(n, r, c->bv, p, c->bsc, s);
    precondition(c, p, c->by);
    launch_bi_spmv(L0, c->by, c->bv, c->rt, false, c->work, c->bsc, c->stream);
    launch_bi_half(n, r, c->bv, c->bs, c->work, c->bsc, c->stream);
    // after a converged half step this V-cycle's result is not used
    precondition(c, c->bs, z);
    launch_bi_spmv(L0, z, c->bt, c->bs, true, c->work, c->bsc, c->stream);
    launch_bi_update(n, x, c->by, z, c->bs, c->bt, r, c->rt, c->work, c->bsc, c->stream);
}

cudaGraphExec_t bicgstab_graph(amg_ctx* c) {
    if (!c->p.device_loop || !cg_graphs(c) || c->prof.graphs) return nullptr;
    int& state = c->bi_graph_state[c->precision];
    cudaGraphExec_t& ex = c->graph_bi[c->precision];
    if (state == 0) {
        auto build = [&] {
            return build_while_graph(
                c, [] {},
                [&](cudaGraphConditionalHandle h, cudaStream_t st) { launch_bi_continue(h, c->bsc, st); },
                [&] { bi_iteration(c); },
                [&] {
                    AMG_CUDA_TRY(cudaMemcpyAsync(c->bsc_host, c->bsc, sizeof(BiScalars),
                                                 cudaMemcpyDeviceToHost, c->stream));
                });
        };
        ex = build();
        if (!ex && t_launch_overlap) {
            t_launch_overlap = false;
            ex = build();
            t_launch_overlap = true;
        }
        state = ex ? 1 : -1;
    }
    return ex;
}

int bicgstab(amg_ctx* c, double tol, int32_t maxit, amg_solve_info* info, std::string& why) {
    DevLevel& L0 = c->dl[0];
    const int n = L0.n;
    cudaStream_t s = c->stream;
    if (!c->rt) {
        c->rt = c->mem.alloc<double>(n);
        c->bv = c->mem.alloc<double>(n);
        c->by = c->mem.alloc<double>(n);
        c->bs = c->mem.alloc<double>(n);
        c->bt = c->mem.alloc<double>(n);
        c->bsc = c->mem.alloc<BiScalars>(1);
        c->bsc_host = static_cast<BiScalars*>(pinned_alloc(sizeof(BiScalars)));
    }
    BiScalars& h = *c->bsc_host;
    std::memset(&h, 0, sizeof(BiScalars));
    h.tol = tol;
    h.maxit = maxit;
    AMG_CUDA_TRY(cudaMemcpyAsync(c->bsc, c->bsc_host, sizeof(BiScalars), cudaMemcpyHostToDevice, s));
    // r = b - A x, rt = r, rho = r.r, and the start of the loop
    launch_bi_start(L0, c->bb, c->x, c->r, c->rt, c->work, c->bsc, s);
    AMG_CUDA_TRY(cudaMemcpyAsync(c->bsc_host, c->bsc, sizeof(BiScalars), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    c->last_device_loop = 0;
    if (!h.done) {
        if (cudaGraphExec_t loop = bicgstab_graph(c)) {
            AMG_CUDA_TRY(cudaGraphLaunch(loop, s));
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
            c->last_device_loop = 1;
            if (!h.done && !h.status)
                throw Error{AMG_ECUDA, "device-side BiCGSTAB loop stopped before its condition"};
        } else {
            while (bi_continue(h)) {
                bi_iteration(c);
                AMG_CUDA_TRY(cudaMemcpyAsync(c->bsc_host, c->bsc, sizeof(BiScalars),
                                             cudaMemcpyDeviceToHost, s));
                AMG_CUDA_TRY(cudaStreamSynchronize(s));
            }
        }
    }
    AMG_CUDA_TRY(cudaGetLastError());
    const int status = h.status ? h.status : AMG_OK;
    if (status != AMG_OK) {
        static const char* kWhy[] = {"maximum iterations reached", "BiCGSTAB breakdown: rt.r = 0",
                                     "BiCGSTAB breakdown: rt.v = 0", "BiCGSTAB breakdown: t.t = 0",
                                     "a dot product of the iteration is not finite"};
        why = status == AMG_ERANGE ? "a kernel met an index outside its range (checked build)"
                                   : kWhy[std::min(std::max(h.why, 0), 4)];
    }
    if (info) {
        cg_true_residual(c);
        double rr = 0.0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&rr, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        info->status = status;
        info->iterations = h.iters;
        info->rel_residual = h.rel;
        info->true_rel_residual = h.r0 > 0.0 ? std::sqrt(rr) / h.r0 : 0.0;
        info->device_loop = c->last_device_loop;
    }
    return status;
}

}  // namespace

// ---------------------------------------------------------------------------
// the same CG, one step at a time, for the server: every step issues work on
// the context's stream and records an event; the next step runs once that
// event has completed, so the host never blocks and many contexts iterate
// concurrently on the device.  The issued launches, and so the results, are
// exactly those of pcg().
// ---------------------------------------------------------------------------
void pcg_async_begin(amg_ctx* c, double tol, int32_t maxit) {
    AsyncCg& a = c->acg;
    if (!a.ev) AMG_CUDA_TRY(cudaEventCreateWithFlags(&a.ev, cudaEventDisableTiming));
    if (!a.rr_host) a.rr_host = static_cast<double*>(pinned_alloc(sizeof(double)));
    a.tol = tol;
    a.maxit = maxit;
    a.status = AMG_OK;
    t_launch_overlap = c->p.launch_overlap != 0;
    cg_start(c, tol, maxit);
    AMG_CUDA_TRY(cudaEventRecord(a.ev, c->stream));
    a.state = AsyncCg::kStarted;
}

// issues the true-residual computation and its copy to the host
static void async_finish(amg_ctx* c, int status) {
    AsyncCg& a = c->acg;
    a.status = status;
    cg_true_residual(c);
    AMG_CUDA_TRY(cudaMemcpyAsync(a.rr_host, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
    AMG_CUDA_TRY(cudaEventRecord(a.ev, c->stream));
    a.state = AsyncCg::kFinishing;
}

int pcg_async_step(amg_ctx* c) {
    AsyncCg& a = c->acg;
    if (a.state == AsyncCg::kDone) return 2;
    if (a.state == AsyncCg::kIdle) throw Error{AMG_EINVAL, "no solve in progress"};
    const cudaError_t q = cudaEventQuery(a.ev);
    if (q == cudaErrorNotReady) return 0;
    AMG_CUDA_TRY(q);
    t_launch_overlap = c->p.launch_overlap != 0;
    const PcgScalars& h = *c->sc_host;
    switch (a.state) {
        case AsyncCg::kStarted:
            if (h.status != 0) { async_finish(c, h.status); break; }
            if (h.done) { async_finish(c, AMG_OK); break; }
            if (cudaGraphExec_t loop = a.maxit > 0 ? solve_graph(c) : nullptr) {
                // the whole iteration loop on the device; one more wait for this solve
                AMG_CUDA_TRY(cudaGraphLaunch(loop, c->stream));
                AMG_CUDA_TRY(cudaEventRecord(a.ev, c->stream));
                c->last_device_loop = c->solve_graph_plain ? 2 : 1;
                a.state = AsyncCg::kLooping;
                break;
            }
            c->last_device_loop = 0;
            cg_first_direction(c);
            if (h.iters >= a.maxit) { async_finish(c, AMG_ENOTCONV); break; }
            run_part_a(c);
            AMG_CUDA_TRY(cudaEventRecord(a.ev, c->stream));
            a.state = AsyncCg::kIterating;
            break;
        case AsyncCg::kIterating:
            if (h.status != 0) { async_finish(c, h.status); break; }
            if (h.done) { async_finish(c, AMG_OK); break; }
            if (h.iters >= a.maxit) { async_finish(c, AMG_ENOTCONV); break; }
            run_part_b(c);
            run_part_a(c);
            AMG_CUDA_TRY(cudaEventRecord(a.ev, c->stream));
            break;
        case AsyncCg::kLooping:
            if (h.status != 0) async_finish(c, h.status);
            else if (h.done) async_finish(c, AMG_OK);
            else if (h.iters >= a.maxit) async_finish(c, AMG_ENOTCONV);
            else throw Error{AMG_ECUDA, "device-side CG loop stopped before its condition"};
            break;
        case AsyncCg::kFinishing:
            cg_fill_info(c, a.status, *a.rr_host, &a.info);
            a.state = AsyncCg::kDone;
            return 2;
        default:
            break;
    }
    AMG_CUDA_TRY(cudaGetLastError());
    return 1;
}

// ---------------------------------------------------------------------------
// the V-cycles of several contexts, batched step by step
// ---------------------------------------------------------------------------

// The V-cycle of the context's precision on its level-0 vectors (z = B r for
// c->r, c->z) as launch records, recorded once per precision and launch
// shapes.  nullptr when a level runs its sweeps as dependency-driven kernels
// (cooperative launches, which do not batch).
const std::vector<VRec>* vcycle_records(amg_ctx* c) {
    const int pr = c->precision;
    if (!c->vrec_ok[pr]) {
        for (const DevLevel& L : c->dl)
            if (L.sweep) return nullptr;
        std::vector<VRec>& rec = c->vrec[pr];
        rec.clear();
        const bool prof = c->prof.on;
        c->prof.on = false;
        t_vrecord = &rec;
        try {
            precondition(c, c->r, c->z);
        } catch (...) {
            t_vrecord = nullptr;
            c->prof.on = prof;
            throw;
        }
        t_vrecord = nullptr;
        c->prof.on = prof;
        c->vrec_ok[pr] = true;
    }
    return &c->vrec[pr];
}

void precondition_context(amg_ctx* c) { precondition(c, c->r, c->z); }

void batched_precondition(amg_ctx* const* cs, int n, cudaStream_t s) {
    NvtxRange nvtx("batched V-cycle");
    std::vector<const VRec*> all;
    for (int k = 0; k < n; ++k) {
        const std::vector<VRec>* r = vcycle_records(cs[k]);
        if (!r) throw Error{AMG_EINVAL, "a context with sweep kernels cannot join a batched V-cycle"};
        for (const VRec& v : *r) all.push_back(&v);
    }
    // each context's keys increase along its V-cycle, so a stable merge by key
    // keeps every context's order; equal keys are independent steps of
    // different contexts
    auto key = [](const VRec* a) { return std::make_tuple(a->phase, a->level, a->step); };
    std::stable_sort(all.begin(), all.end(), [&](const VRec* a, const VRec* b) { return key(a) < key(b); });
    auto body = [](const VRec* a) { return std::make_pair(reinterpret_cast<uintptr_t>(a->launch), a->block); };
    size_t i = 0;
    while (i < all.size()) {
        size_t j = i;
        while (j < all.size() && key(all[j]) == key(all[i])) ++j;
        std::stable_sort(all.begin() + (long)i, all.begin() + (long)j,
                         [&](const VRec* a, const VRec* b) { return body(a) < body(b); });
        for (size_t k = i; k < j;) {
            size_t m = k;
            while (m < j && body(all[m]) == body(all[k])) ++m;
            launch_vrecords(&all[k], (int)(m - k), s);
            k = m;
        }
        i = j;
    }
    AMG_CUDA_TRY(cudaGetLastError());
}

// The same stepping split around the preconditioner, for a scheduler that
// applies it to several contexts at once: poll returns 0 (busy), 1 (issued
// the end of the solve), 2 (finished) or 3 when the next step needs
// z = B r on c->r (first: the first direction); the caller issues it after
// the context stream's work and then calls resume, which issues the rest of
// the iteration exactly as pcg_async_step does.
int pcg_async_poll(amg_ctx* c, bool* first) {
    AsyncCg& a = c->acg;
    if (a.state == AsyncCg::kDone) return 2;
    if (a.state == AsyncCg::kIdle) throw Error{AMG_EINVAL, "no solve in progress"};
    const cudaError_t q = cudaEventQuery(a.ev);
    if (q == cudaErrorNotReady) return 0;
    AMG_CUDA_TRY(q);
    t_launch_overlap = c->p.launch_overlap != 0;
    const PcgScalars& h = *c->sc_host;
    switch (a.state) {
        case AsyncCg::kStarted:
            c->last_device_loop = 0;
            if (h.status != 0) { async_finish(c, h.status); return 1; }
            if (h.done) { async_finish(c, AMG_OK); return 1; }
            if (h.iters >= a.maxit) { async_finish(c, AMG_ENOTCONV); return 1; }
            *first = true;
            return 3;
        case AsyncCg::kIterating:
            if (h.status != 0) { async_finish(c, h.status); return 1; }
            if (h.done) { async_finish(c, AMG_OK); return 1; }
            if (h.iters >= a.maxit) { async_finish(c, AMG_ENOTCONV); return 1; }
            *first = false;
            return 3;
        case AsyncCg::kFinishing:
            cg_fill_info(c, a.status, *a.rr_host, &a.info);
            a.state = AsyncCg::kDone;
            return 2;
        default:
            throw Error{AMG_EINVAL, "the device-side loop does not step"};
    }
}

void pcg_async_resume(amg_ctx* c, bool first) {
    AsyncCg& a = c->acg;
    t_launch_overlap = c->p.launch_overlap != 0;
    const int n = c->dl[0].n;
    cudaStream_t s = c->stream;
    if (first) {
        launch_cg_rz(n, c->r, c->z, nullptr, c->pv, c->work, kRho0, s);
        if (c->flexible)
            AMG_CUDA_TRY(cudaMemcpyAsync(c->zold, c->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
        launch_cg_rz(n, c->r, c->z, c->zold, c->pv, c->work, c->flexible ? kRZFlex : kRZ, s);
        launch_cg_p(n, c->z, c->pv, c->flexible ? c->zold : nullptr, c->work, s);
    }
    run_part_a(c);
    AMG_CUDA_TRY(cudaEventRecord(a.ev, s));
    a.state = AsyncCg::kIterating;
    AMG_CUDA_TRY(cudaGetLastError());
}

namespace {

struct Guard {
    template <typename F>
    static int run(F&& f) {
        try {
            f();
            t_last_error.clear();
            return AMG_OK;
        } catch (const Error& e) {
            t_last_error = e.msg;
            return e.code;
        } catch (const std::bad_alloc&) {
            t_last_error = "host allocation failed";
            return AMG_ENOMEM;
        } catch (const std::exception& e) {
            t_last_error = e.what();
            return AMG_EINVAL;
        }
    }
};

std::mutex g_pinned_mu;
std::map<size_t, std::vector<void*>> g_pinned_free;   // size class -> free blocks
std::map<void*, size_t> g_pinned_class;                // block -> size class

}  // namespace

void* pinned_alloc(size_t bytes) {
    size_t cls = 256;
    while (cls < bytes) cls <<= 1;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto& fl = g_pinned_free[cls];
    if (!fl.empty()) {
        void* p = fl.back();
        fl.pop_back();
        return p;
    }
    void* p = nullptr;
    const cudaError_t e = cudaMallocHost(&p, cls);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{AMG_ENOMEM, "pinned host allocation of " + std::to_string(cls) + " bytes failed"};
    }
    g_pinned_class[p] = cls;
    return p;
}

void pinned_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned_class.find(p);
    if (it != g_pinned_class.end()) g_pinned_free[it->second].push_back(p);
}

namespace {

// Stream-ordered allocations come from the device's default memory pool; keep
// freed blocks in the pool (no release at synchronisation points), so
// contexts that come and go reuse them.  The setting lasts for this process.
void init_device_pool(int device) {
    static std::once_flag once[64];
    if (device < 0 || device >= 64) return;
    std::call_once(once[device], [device] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
}

void setup_impl(const amg_csr* A, const amg_params* prm, amg_ctx** out) {
    NvtxRange nvtx("amg_setup");
    if (!A || !prm || !out) throw Error{AMG_EINVAL, "null argument"};
    *out = nullptr;
    check_params(*prm);
    if (A->n <= 0 || A->nnz <= 0 || !A->row_ptr || !A->col || !A->val)
        throw Error{AMG_EINVAL, "empty or null matrix"};
    const double t_start = now_ms();
    auto c = std::make_unique<amg_ctx>();
    c->p = *prm;
    c->user_stream = static_cast<cudaStream_t>(prm->cuda_stream);
    AMG_CUDA_TRY(cudaGetDevice(&c->device));
    AMG_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    init_device_pool(c->device);
    c->mem.set_stream(c->stream);
    AMG_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    AMG_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    enter(c.get());
    int sms = 0;
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    // launch shapes from the SM count, set once per process (contexts are set
    // up concurrently by the server's threads while others launch)
    static std::once_flag shapes_once;
    std::call_once(shapes_once, [sms] {
        g_reduction_blocks = std::max(1, sms) * 8;
        g_overlap_max_blocks = std::max(1, sms) * 2;
    });
    cudaStream_t s = c->stream;

    // level 0 on the host (original numbering)
    c->hl.emplace_back();
    HostCsr& A0 = c->hl[0].A;
    A0.n = A->n;
    A0.rp.resize((size_t)A->n + 1);
    const cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    AMG_CUDA_TRY(cudaMemcpy(A0.rp.data(), A->row_ptr, sizeof(int32_t) * (A->n + 1), kind));
    if (A0.rp[A->n] != A->nnz) throw Error{AMG_EINVAL, "row_ptr[n] != nnz"};
    A0.ci.resize(A->nnz);
    A0.va.resize(A->nnz);
    AMG_CUDA_TRY(cudaMemcpy(A0.ci.data(), A->col, sizeof(int32_t) * A->nnz, kind));
    AMG_CUDA_TRY(cudaMemcpy(A0.va.data(), A->val, sizeof(double) * A->nnz, kind));
    std::string err;
    if (!validate_csr(A0, err) || !check_values_symmetric(A0, err)) throw Error{AMG_EINVAL, err};

    DevArena setup_mem(s);   // original-order level matrices, freed at the end
    std::vector<DevCsr> dA(1);
    dA[0].n = A0.n;
    dA[0].nnz = A0.nnz();
    dA[0].rp = setup_mem.alloc<int32_t>(A0.n + 1);
    dA[0].ci = setup_mem.alloc<int32_t>(A0.nnz());
    dA[0].va = setup_mem.alloc<double>(A0.nnz());
    upload(dA[0].rp, A0.rp, s);
    upload(dA[0].ci, A0.ci, s);
    upload(dA[0].va, A0.va, s);

    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        ~EventPair() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    AMG_CUDA_TRY(cudaEventCreate(&ev.a));
    AMG_CUDA_TRY(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    double host_ms = 0.0, galerkin_ms = 0.0, agg_ms = 0.0;
    while (true) {
        const int l = (int)c->hl.size() - 1;
        HostLevel& cur = c->hl[l];
        if (cur.A.n <= prm->coarsen_target || l >= prm->max_levels - 1) break;
        double t0 = now_ms();
        NvtxRange nvtx_level("setup level: aggregation, colouring, Galerkin");
        AggResult R = aggregate_level(cur.A, &dA[l], *prm, s);
        agg_ms += now_ms() - t0;
        host_ms += now_ms() - t0;
        if (R.nc == 0 || (double)cur.A.n / (double)R.nc < prm->min_coarsen_rate) break;
        t0 = now_ms();
        cur.ncolours = smoother_colouring(cur.A, cur.colour);
        host_ms += now_ms() - t0;
        cur.agg = std::move(R);
        HostCsr G;
        DevCsr Gd;
        AMG_CUDA_TRY(cudaEventRecord(e0, s));
        galerkin_device(dA[l], cur.A, cur.agg, setup_mem, Gd, G, s);
        AMG_CUDA_TRY(cudaEventRecord(e1, s));
        AMG_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        AMG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        galerkin_ms += ms;
        c->hl.emplace_back();
        c->hl.back().A = std::move(G);
        dA.push_back(Gd);
    }
    const int nlev = (int)c->hl.size();
    c->nL = c->hl.back().A.n;
    if (c->nL > prm->dense_cap)
        throw Error{AMG_EINVAL, "coarsest level has " + std::to_string(c->nL) +
                                    " rows, more than dense_cap = " + std::to_string(prm->dense_cap)};

    // smoothing orders, bottom-up
    const double t_dev0 = now_ms();
    {
        std::vector<int32_t>& pl = c->hl[nlev - 1].perm;
        pl.resize(c->nL);
        std::iota(pl.begin(), pl.end(), 0);
        for (int l = nlev - 2; l >= 0; --l) c->hl[l].perm = smoothing_order(c->hl[l]);
    }
    c->dl.resize(nlev);
    for (int l = 0; l < nlev; ++l) {
        HostLevel& h = c->hl[l];
        DevLevel& L = c->dl[l];
        build_level_device(dA[l], h.A, h.perm, c->mem, L, s);
        L.x = c->mem.alloc<double>(L.n);
        L.b = c->mem.alloc<double>(L.n);
        L.r = c->mem.alloc<double>(L.n);
        if (l == nlev - 1) {
            L.cptr = {0, L.n};
            L.ncolours = 0;
            continue;
        }
        L.ncolours = h.ncolours;
        L.cptr.assign(h.ncolours + 1, 0);
        L.cnnz.assign(h.ncolours, 0);
        for (int32_t i = 0; i < L.n; ++i) {
            ++L.cptr[h.colour[i] + 1];
            L.cnnz[h.colour[i]] += h.A.rp[i + 1] - h.A.rp[i] - 1;
        }
        for (int col = 0; col < h.ncolours; ++col) L.cptr[col + 1] += L.cptr[col];
        const std::vector<int32_t>& pn = c->hl[l + 1].perm;
        const int32_t nc = h.agg.nc;
        L.n_coarse = nc;
        // restriction lists: the rows of colour >= 1 of each aggregate (colour 0
        // is smoothed last and has a zero residual), ascending positions
        std::vector<int32_t> aggp(L.n, -1), rptr(nc + 1, 0), ridx;
        for (int32_t i = 0; i < L.n; ++i) {
            const int32_t a = h.agg.agg[i];
            if (a < 0) continue;
            aggp[h.perm[i]] = pn[a];
            if (h.colour[i] > 0) ++rptr[pn[a] + 1];
        }
        for (int32_t J = 0; J < nc; ++J) rptr[J + 1] += rptr[J];
        ridx.resize(rptr[nc]);
        {
            std::vector<int32_t> fill(rptr.begin(), rptr.end() - 1);
            for (int32_t r = L.cptr[1]; r < L.n; ++r)
                if (aggp[r] >= 0) ridx[fill[aggp[r]]++] = r;
        }
        {
            int32_t most = 0;
            for (int32_t J = 0; J < nc; ++J) most = std::max(most, rptr[J + 1] - rptr[J]);
            // the fused kernel needs the rows of colour >= 1 to be one block
            // sorted by coarse index (two colours) and runs shorter than a warp
            L.fused_ok = L.ncolours == 2 && most <= 32;
            L.fused_restrict = L.lpr == 0 && L.fused_ok;
        }
        L.agg = c->mem.alloc<int32_t>(L.n);
        L.rptr = c->mem.alloc<int32_t>(nc + 1);
        L.ridx = c->mem.alloc<int32_t>(ridx.size());
        upload(L.agg, aggp, s);
        upload(L.rptr, rptr, s);
        upload(L.ridx, ridx, s);
    }
    // coarsest level: dense inverse
    c->Ainv = c->mem.alloc<double>((size_t)c->nL * c->nL);
    const double t_inv0 = now_ms();
    NvtxRange nvtx_inv("coarsest inverse");
    if (!dense_inverse_device(dA[nlev - 1], c->Ainv, s))
        throw Error{AMG_ENOTSPD, "coarsest matrix is not positive definite"};
    const double inverse_ms = now_ms() - t_inv0;

    // level-0 CG state (c->hl has grown: take the level-0 matrix afresh)
    const HostCsr& A0f = c->hl[0].A;
    const int32_t n = A0f.n;
    c->x = c->mem.alloc<double>(n);
    c->r = c->mem.alloc<double>(n);
    c->z = c->mem.alloc<double>(n);
    c->zold = c->mem.alloc<double>(n);
    c->pv = c->mem.alloc<double>(n);
    c->q = c->mem.alloc<double>(n);
    c->bb = c->mem.alloc<double>(n);
    c->perm0 = c->mem.alloc<int32_t>(n);
    upload(c->perm0, c->hl[0].perm, s);
    {
        std::vector<double> isq(n);
        std::vector<int32_t> inv(n);
        for (int32_t i = 0; i < n; ++i) inv[c->hl[0].perm[i]] = i;
        std::vector<double> diag(n, 0.0);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = A0f.rp[i]; k < A0f.rp[i + 1]; ++k)
                if (A0f.ci[k] == i) diag[i] = A0f.va[k];
        for (int32_t r = 0; r < n; ++r) isq[r] = 1.0 / std::sqrt(diag[inv[r]]);
        c->isq0 = c->mem.alloc<double>(n);
        upload(c->isq0, isq, s);
    }
    c->work.partials = c->mem.alloc<double>(g_reduction_blocks);
    c->work.partials2 = c->mem.alloc<double>(g_reduction_blocks);
    c->work.counters = c->mem.alloc<unsigned int>(16);
    AMG_CUDA_TRY(cudaMemsetAsync(c->work.counters, 0, sizeof(unsigned int) * 16, s));
    c->work.sc = c->mem.alloc<PcgScalars>(1);
    AMG_CUDA_TRY(cudaMemsetAsync(c->work.sc, 0, sizeof(PcgScalars), s));
    // kernel-side errors (a bounded wait that ran out) land in the CG status
    // word, which the iteration loop reads back every iteration
    for (DevLevel& L : c->dl)
        L.err = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(c->work.sc) +
                                           offsetof(PcgScalars, status));
    c->norm_dev = c->mem.alloc<double>(1);
    c->sc_host = static_cast<PcgScalars*>(pinned_alloc(sizeof(PcgScalars)));
    AMG_CUDA_TRY(cudaEventCreate(&c->ev0));
    AMG_CUDA_TRY(cudaEventCreate(&c->ev1));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));

    c->flexible = prm->flexible_cg > 0 ? 1 : 0;
    c->precision = prm->precision;
    if (c->precision == AMG_FP32_IN_FP64) ensure_fp32(c.get());
    for (int pr = 0; pr < 2; ++pr) {
        c->shapes[pr].assign(nlev - 1, 0);
        for (int l = 0; l + 1 < nlev; ++l) c->shapes[pr][l] = shape_of(c->dl[l]);
    }
    const double tune_ms = prm->autotune ? autotune_shapes(c.get()) : 0.0;
    fill_info(c.get());
    c->summary.autotune_ms = tune_ms;
    c->summary.coarsest_inverse_ms = inverse_ms;
    c->summary.host_setup_ms = host_ms;
    c->summary.aggregation_ms = agg_ms;
    c->summary.gpu_galerkin_ms = galerkin_ms;
    c->summary.gpu_other_ms = now_ms() - t_dev0;
    c->summary.total_setup_ms = now_ms() - t_start;
    leave(c.get());
    *out = c.release();
}

}  // namespace
}  // namespace amg

using namespace amg;

extern "C" {

int amg_params_default(amg_params* p, int32_t dim) {
    if (!p || dim < 1 || dim > 3) {
        t_last_error = "amg_params_default: null pointer or dim outside 1..3";
        return AMG_EINVAL;
    }
    std::memset(p, 0, sizeof(*p));
    p->delta = 1.0 / 3.0;
    p->beta = 1e-5;
    p->omega = 1.6;
    p->s_min = 1 << dim;
    p->s_max = 3 * (1 << (dim - 1));
    p->d_max = dim;
    p->coarsen_target = 5000;
    p->max_levels = 20;
    p->dense_cap = 8192;
    p->min_coarsen_rate = 1.2;
    p->precision = AMG_FP64;
    p->flexible_cg = -1;
    p->cuda_stream = nullptr;
    p->launch_overlap = 1;
    p->aggregation_tile = 0;
    p->aggregation_device = 0;
    p->autotune = 0;
    p->coarsest_fp32 = 0;
    p->device_loop = 1;
    p->host_threads = 0;
    return AMG_OK;
}

int amg_setup(const amg_csr* A, const amg_params* p, amg_ctx** out) {
    if (out) *out = nullptr;
    return Guard::run([&] { setup_impl(A, p, out); });
}

int amg_set_precision(amg_ctx* c, int32_t precision, int32_t flexible_cg) {
    return Guard::run([&] {
        if (!c) throw Error{AMG_EINVAL, "null context"};
        if (precision != AMG_FP64 && precision != AMG_FP32_IN_FP64)
            throw Error{AMG_EINVAL, "precision must be AMG_FP64 or AMG_FP32_IN_FP64"};
        enter(c);
        if (precision == AMG_FP32_IN_FP64) ensure_fp32(c);
        c->precision = precision;
        c->flexible = flexible_cg > 0 ? 1 : 0;
        AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));   // no graph of this context in flight
        if (c->p.autotune && !c->tuned[precision]) {
            apply_shapes(c);
            c->summary.autotune_ms += autotune_shapes(c);
        }
        apply_shapes(c);
        for (int l = 0; l + 1 < (int)c->dl.size(); ++l) {
            c->linfo[l].lanes_per_row = c->dl[l].lpr;
            c->linfo[l].threads_per_block = c->dl[l].block;
            c->linfo[l].sweep = c->dl[l].sweep ? 1 : 0;
            c->linfo[l].carveout = c->dl[l].carve;
        }
        leave(c);
    });
}

int amg_vcycle(amg_ctx* c, const double* r_dev, double* z_dev) {
    return Guard::run([&] {
        if (!c || !r_dev || !z_dev) throw Error{AMG_EINVAL, "null argument"};
        const int n = c->dl[0].n;
        enter(c);
            launch_scatter(n, c->perm0, r_dev, c->r, c->stream);
        precondition(c, c->r, c->z);
        launch_gather(n, c->perm0, c->z, z_dev, c->stream);
        AMG_CUDA_TRY(cudaGetLastError());
        leave(c);
    });
}

static int solve_common(amg_ctx* c, const double* b, double* x, double tol, int32_t maxit,
                        amg_solve_info* info, bool host, bool use_bicgstab = false,
                        bool zero_guess = false) {
    int status = AMG_OK;
    std::string why;
    int rc = Guard::run([&] {
        if (!c || !b || !x) throw Error{AMG_EINVAL, "null argument"};
        if (!(tol >= 0.0) || maxit < 0) throw Error{AMG_EINVAL, "tol must be >= 0 and maxit >= 0"};
        const int n = c->dl[0].n;
        cudaStream_t s = c->stream;
        enter(c);
        AMG_CUDA_TRY(cudaEventRecord(c->ev0, s));
        const double* bd = b;
        double* xd = x;
        if (host) {
            // stage through the level-0 scratch vectors q (b) and z (x0)
            AMG_CUDA_TRY(cudaMemcpyAsync(c->q, b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
            if (!zero_guess)
                AMG_CUDA_TRY(cudaMemcpyAsync(c->z, x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
            bd = c->q;
            xd = c->z;
        }
        launch_scatter(n, c->perm0, bd, c->bb, s);
        if (zero_guess) AMG_CUDA_TRY(cudaMemsetAsync(c->x, 0, sizeof(double) * n, s));
        else launch_scatter(n, c->perm0, xd, c->x, s);
        amg_solve_info local{};
        {
            NvtxRange nvtx(use_bicgstab ? "bicgstab" : "pcg");
            status = use_bicgstab ? bicgstab(c, tol, maxit, &local, why) : pcg(c, tol, maxit, &local);
        }
        if (host) {
            launch_gather(n, c->perm0, c->x, c->z, s);
            AMG_CUDA_TRY(cudaMemcpyAsync(x, c->z, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        } else {
            launch_gather(n, c->perm0, c->x, x, s);
        }
        AMG_CUDA_TRY(cudaEventRecord(c->ev1, s));
        AMG_CUDA_TRY(cudaEventSynchronize(c->ev1));
        float ms = 0.f;
        AMG_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        local.solve_ms = ms;
        leave(c);
        if (info) *info = local;
        if (status != AMG_OK && why.empty())
            why = status == AMG_ENOTCONV ? "maximum iterations reached"
                  : status == AMG_ENONFINITE ? "a dot product of the iteration is not finite"
                  : status == AMG_ERANGE ? "a kernel met an index outside its range (checked build)"
                  : status == AMG_ETIMEOUT ? "a bounded device-side wait gave up: free the context"
                                           : "p.Ap <= 0: operator or preconditioner not SPD";
    });
    if (rc != AMG_OK) return rc;
    if (status != AMG_OK) t_last_error = why;   // after the guard, which clears it on success
    return status;
}

int amg_pcg_solve(amg_ctx* c, const double* b_dev, double* x_dev, double tol, int32_t maxit,
                  amg_solve_info* info) {
    return solve_common(c, b_dev, x_dev, tol, maxit, info, false);
}

int amg_bicgstab_solve(amg_ctx* c, const double* b_dev, double* x_dev, double tol,
                       int32_t maxit, amg_solve_info* info) {
    return solve_common(c, b_dev, x_dev, tol, maxit, info, false, true);
}

int amg_pcg_solve_host(amg_ctx* c, const double* b_host, double* x_host, double tol,
                       int32_t maxit, amg_solve_info* info) {
    return solve_common(c, b_host, x_host, tol, maxit, info, true);
}

int amg_pcg_solve_host_zero_guess(amg_ctx* c, const double* b_host, double* x_host, double tol,
                                  int32_t maxit, amg_solve_info* info) {
    return solve_common(c, b_host, x_host, tol, maxit, info, true, false, true);
}

int amg_residual_norm(amg_ctx* c, const double* b_dev, const double* x_dev, double* out_norm) {
    return Guard::run([&] {
        if (!c || !b_dev || !x_dev || !out_norm) throw Error{AMG_EINVAL, "null argument"};
        const int n = c->dl[0].n;
        cudaStream_t s = c->stream;
        enter(c);
        launch_scatter(n, c->perm0, b_dev, c->q, s);
        launch_scatter(n, c->perm0, x_dev, c->pv, s);
        launch_cg_residual(c->dl[0], c->q, c->pv, nullptr, c->work, kStore, c->norm_dev, s);
        double rr = 0.0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&rr, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        leave(c);
        *out_norm = std::sqrt(rr);
    });
}

int amg_hierarchy_info(const amg_ctx* c, amg_summary* summary, amg_level_info* levels, int32_t cap) {
    if (!c || cap < 0 || (cap > 0 && !levels)) {
        t_last_error = "amg_hierarchy_info: bad arguments";
        return AMG_EINVAL;
    }
    if (summary) *summary = c->summary;
    for (int32_t l = 0; l < cap && l < (int32_t)c->linfo.size(); ++l) levels[l] = c->linfo[l];
    return (int)c->linfo.size();
}

int amg_export_level(const amg_ctx* c, int32_t l, int32_t* row_ptr, int32_t* col, double* val,
                     int32_t* agg, int32_t* colour) {
    if (!c || l < 0 || l >= (int32_t)c->hl.size()) {
        t_last_error = "amg_export_level: level out of range";
        return AMG_EINVAL;
    }
    const HostLevel& h = c->hl[l];
    const bool last = l == (int32_t)c->hl.size() - 1;
    if (last && (agg || colour)) {
        t_last_error = "amg_export_level: the coarsest level has no aggregates or colours";
        return AMG_EINVAL;
    }
    if (row_ptr) std::memcpy(row_ptr, h.A.rp.data(), sizeof(int32_t) * h.A.rp.size());
    if (col) std::memcpy(col, h.A.ci.data(), sizeof(int32_t) * h.A.ci.size());
    if (val) std::memcpy(val, h.A.va.data(), sizeof(double) * h.A.va.size());
    if (agg) std::memcpy(agg, h.agg.agg.data(), sizeof(int32_t) * h.A.n);
    if (colour) std::memcpy(colour, h.colour.data(), sizeof(int32_t) * h.A.n);
    return AMG_OK;
}

static HostCsr host_copy(const amg_csr* A) {
    if (!A || A->n <= 0 || A->nnz <= 0 || !A->row_ptr || !A->col || !A->val)
        throw Error{AMG_EINVAL, "empty or null matrix"};
    if (A->on_device) throw Error{AMG_EINVAL, "this entry point takes a host matrix"};
    HostCsr H;
    H.n = A->n;
    H.rp.assign(A->row_ptr, A->row_ptr + A->n + 1);
    if (H.rp[A->n] != A->nnz) throw Error{AMG_EINVAL, "row_ptr[n] != nnz"};
    H.ci.assign(A->col, A->col + A->nnz);
    H.va.assign(A->val, A->val + A->nnz);
    std::string err;
    if (!validate_csr(H, err) || !check_values_symmetric(H, err)) throw Error{AMG_EINVAL, err};
    return H;
}

int amg_selftest_bounded_wait(int64_t polls, void* cuda_stream, int32_t* status,
                              double* elapsed_ms) {
    return Guard::run([&] {
        if (!status || !elapsed_ms || polls < 0) throw Error{AMG_EINVAL, "null output or polls < 0"};
        wait_selftest((long long)polls, static_cast<cudaStream_t>(cuda_stream), status, elapsed_ms);
    });
}

int amg_set_level_shape(amg_ctx* c, int32_t l, int32_t lanes_per_row, int32_t threads_per_block) {
    return Guard::run([&] {
        if (!c) throw Error{AMG_EINVAL, "null context"};
        if (l < 0 || l >= (int32_t)c->dl.size() - 1)
            throw Error{AMG_EINVAL, "level out of range (the coarsest level has no shape)"};
        if (threads_per_block != 0 && threads_per_block != 256 && threads_per_block != 128)
            throw Error{AMG_EINVAL, "threads_per_block must be 0, 256 or 128"};
        const bool sweep = (lanes_per_row & AMG_SHAPE_SWEEP) != 0;
        const int lanes = lanes_per_row & ~AMG_SHAPE_SWEEP;
        const int code = lanes | (threads_per_block == 128 ? kHalfBlock : 0) | (sweep ? kSweep : 0);
        if (lanes < 0 || lanes > 8 || !shape_allowed(c->dl[l], code))
            throw Error{AMG_EINVAL, "lanes_per_row must be 1, 2, 4 or 8 (optionally with "
                                    "AMG_SHAPE_SWEEP on a level of at most 2^20 rows that is not "
                                    "two-colour fused), or 0 (256 threads) on a level whose staged "
                                    "tile fits in 96 KB"};
        enter(c);
        AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));   // no graph of this context in flight
        drop_graphs(c);
        set_shape(c, l, code);
        c->shapes[c->precision][l] = code;
        c->linfo[l].lanes_per_row = c->dl[l].lpr;
        c->linfo[l].threads_per_block = c->dl[l].block;
        c->linfo[l].sweep = c->dl[l].sweep ? 1 : 0;
        c->linfo[l].carveout = c->dl[l].carve;
        leave(c);
    });
}

int amg_set_level_carveout(amg_ctx* c, int32_t l, int32_t percent) {
    return Guard::run([&] {
        if (!c) throw Error{AMG_EINVAL, "null context"};
        if (l < 0 || l >= (int32_t)c->dl.size() - 1)
            throw Error{AMG_EINVAL, "level out of range (the coarsest level has no shape)"};
        if (percent < -1 || percent > 100) throw Error{AMG_EINVAL, "percent must be -1 .. 100"};
        if (c->dl[l].lpr != kStaged)
            throw Error{AMG_EINVAL, "the carveout applies to the staged kernels (lanes_per_row 0)"};
        enter(c);
        AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));   // no graph of this context in flight
        drop_graphs(c);
        const int code = with_carve(shape_of(c->dl[l]), percent);
        set_shape(c, l, code);
        c->shapes[c->precision][l] = code;
        c->linfo[l].carveout = c->dl[l].carve;
        leave(c);
    });
}

int amg_aggregate(const amg_csr* A, const amg_params* p, int32_t* agg, int32_t* n_coarse) {
    return Guard::run([&] {
        if (!p || !agg || !n_coarse) throw Error{AMG_EINVAL, "null argument"};
        check_params(*p);
        HostCsr H = host_copy(A);
        AggResult R;
        if (p->aggregation_tile > 0 && p->aggregation_device) {
            cudaStream_t s = static_cast<cudaStream_t>(p->cuda_stream);
            DevArena mem(s);
            DevCsr D;
            D.n = H.n;
            D.nnz = H.nnz();
            D.rp = mem.alloc<int32_t>(H.n + 1);
            D.ci = mem.alloc<int32_t>(H.nnz());
            D.va = mem.alloc<double>(H.nnz());
            upload(D.rp, H.rp, s);
            upload(D.ci, H.ci, s);
            upload(D.va, H.va, s);
            R = aggregate_level(H, &D, *p, s);
        } else {
            R = aggregate_level(H, nullptr, *p, nullptr);
        }
        std::memcpy(agg, R.agg.data(), sizeof(int32_t) * H.n);
        *n_coarse = R.nc;
    });
}

int amg_colour(const amg_csr* A, int32_t* colour, int32_t* ncolours) {
    return Guard::run([&] {
        if (!colour || !ncolours) throw Error{AMG_EINVAL, "null argument"};
        HostCsr H = host_copy(A);
        std::vector<int32_t> c;
        *ncolours = smoother_colouring(H, c);
        std::memcpy(colour, c.data(), sizeof(int32_t) * H.n);
    });
}

int amg_profile_enable(amg_ctx* c, int32_t enable) {
    return Guard::run([&] {
        if (!c) throw Error{AMG_EINVAL, "null context"};
        Profiler& P = c->prof;
        if (enable) {
            if (P.events.empty()) {
                P.events.resize(1 << 16);
                for (auto& e : P.events) AMG_CUDA_TRY(cudaEventCreate(&e));
            }
            AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
            P.recs.clear();
            P.next = 0;
        }
        if (enable < 0 || enable > 2) throw Error{AMG_EINVAL, "enable must be 0, 1 or 2"};
        P.on = enable == 1;
        P.graphs = enable == 2;
    });
}

int amg_profile_read(amg_ctx* c, amg_kernel_stat* stats, int32_t cap) {
    int count = 0;
    int rc = Guard::run([&] {
        if (!c || cap < 0 || (cap > 0 && !stats)) throw Error{AMG_EINVAL, "bad arguments"};
        AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
        const int nk = kKGraphFrom + 64;
        std::vector<amg_kernel_stat> acc(nk);
        for (int k = 0; k < nk; ++k) {
            std::memset(&acc[k], 0, sizeof(amg_kernel_stat));
            if (k < kKGraphFrom)
                std::strncpy(acc[k].name, kKindNames[k], sizeof(acc[k].name) - 1);
            else
                std::snprintf(acc[k].name, sizeof(acc[k].name), "graph_from_level_%d", k - kKGraphFrom);
        }
        for (const auto& r : c->prof.recs) {
            float ms = 0.f;
            AMG_CUDA_TRY(cudaEventElapsedTime(&ms, c->prof.events[r.ev], c->prof.events[r.ev + 1]));
            acc[r.kind].launches += 1;
            acc[r.kind].total_ms += ms;
            acc[r.kind].bytes += r.bytes;
        }
        for (int k = 0; k < nk; ++k)
            if (acc[k].launches > 0) {
                if (count < cap) stats[count] = acc[k];
                ++count;
            }
    });
    return rc == AMG_OK ? count : rc;
}

int amg_free(amg_ctx* c) {
    if (!c) return AMG_OK;
    delete c;   // the destructor drains the context stream first
    return AMG_OK;
}

const char* amg_last_error(void) { return t_last_error.c_str(); }

int amg_device_checks(void) {
#ifdef AMG_DEVICE_CHECKS
    return 1;
#else
    return 0;
#endif
}

int amg_debug_set_column(amg_ctx* c, int32_t l, int32_t row, int32_t k, int32_t col) {
    return Guard::run([&] {
#ifndef AMG_DEVICE_CHECKS
        (void)c, (void)l, (void)row, (void)k, (void)col;
        throw Error{AMG_EINVAL, "amg_debug_set_column exists in the checked build only"};
#else
        if (!c || l < 1 || l >= (int32_t)c->dl.size() - 1)
            throw Error{AMG_EINVAL, "level out of range (levels 1 .. L-2 have stored rows)"};
        const DevLevel& L = c->dl[l];
        if (row < 0 || row >= L.n) throw Error{AMG_EINVAL, "row out of range"};
        // a column at or beyond the level's rows: skipped by every pass bound,
        // so no kernel can dereference it
        if (col < L.n) throw Error{AMG_EINVAL, "col must be >= the level's rows"};
        const int32_t r = c->hl[l].perm[row];
        uint16_t rl = 0;
        AMG_CUDA_TRY(cudaMemcpy(&rl, L.rlen + r, sizeof(uint16_t), cudaMemcpyDeviceToHost));
        const int32_t len = rl;
        if (k < 0 || k >= len) throw Error{AMG_EINVAL, "k out of range of the row's entries"};
        const int64_t e = (int64_t)(r >> 5) * L.sw + 32 * (int64_t)k + (r & 31);
        AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
        AMG_CUDA_TRY(cudaMemcpy(L.scol + e, &col, sizeof(int32_t), cudaMemcpyHostToDevice));
        if (L.soff) {
            // the same entry in the copy with per-slice widths
            int64_t pos = 0;
            AMG_CUDA_TRY(cudaMemcpy(&pos, L.soff + (r >> 5), sizeof(int64_t), cudaMemcpyDeviceToHost));
            pos += 32 * (int64_t)k + (r & 31);
            AMG_CUDA_TRY(cudaMemcpy(L.ccol + pos, &col, sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        drop_graphs(c);
#endif
    });
}

}  // extern "C"
