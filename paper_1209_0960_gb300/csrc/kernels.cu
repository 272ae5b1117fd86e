// Solve-phase kernels: multicolour Gauss-Seidel, residual, restriction,
// prolongation, dense coarsest solve, and the CG vector operations
// (Sec. 2 V-cycle; Sec. 3.2 smoother applied in a fixed multicolour order;
// Sec. 5 Krylov iteration).
//
// Layout: every level stores its rows in the smoothing order (colour blocks,
// then coarse aggregate, then original index), the off-diagonal part in the
// sliced layout described in device.h (32-row slices of a common width, so
// the address of an entry is arithmetic: no pointer load precedes it) and the
// diagonal separately.  Row
// kernels give one thread to a row: for each k the 32 threads of a warp read
// entry k of their 32 rows from 32 consecutive addresses, and the row sum is a
// chain of fused multiply-adds with no cross-lane reduction (GB300 executes
// float64 at 1/64 of the float32 rate, so the float64 path keeps the
// arithmetic at one FMA per stored entry).  All reductions are deterministic:
// per-block partial sums in a fixed grid, combined in a fixed order by the
// last block to finish.

#include <algorithm>
#include <type_traits>

#include <map>
#include <mutex>

#include "device.h"

namespace amg {

namespace {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <int W, typename T>
__device__ __forceinline__ T group_sum(T s) {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off, W);
    return s;
}

__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The checked build (compiled with AMG_DEVICE_CHECKS): every gathered index,
// restriction-list row and aggregate index is tested against its range
// before use; one outside it is recorded as AMG_ERANGE in the solve's status
// word and contributes zero instead of being read.  In the regular build the
// test is the constant true and costs nothing.
#ifdef AMG_DEVICE_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif
__device__ __forceinline__ bool index_ok(int j, int n, int32_t* err) {
    if (!kChecks) return true;
    if ((unsigned)j < (unsigned)n) return true;
    if (err) atomicCAS(err, 0, AMG_ERANGE);
    return false;
}

// programmatic dependent launch: let the next kernel of the stream start, and
// wait for every predecessor to finish (both are no-ops without the launch
// attribute)
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// load of setup-time per-row data (length, diagonal): evict-first on the
// streamed fine level
template <bool STREAM, typename T>
__device__ __forceinline__ T ldm(const T* p) {
    return STREAM ? __ldcs(p) : *p;
}

// acc + sgn * sum_k A_row,k x_col(k) over the stored off-diagonal entries of a
// SELL-32 row (base = slice start + row mod 32)
template <bool NEG, typename T, typename X>
__device__ __forceinline__ T sell_row(int64_t base, int len, const int32_t* __restrict__ scol,
                                      const T* __restrict__ sval, const X* x, T acc, int n,
                                      int32_t* err) {
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
        const int64_t e = base + 32 * (int64_t)k;
        const T a = __ldcs(sval + e);
        const int j = __ldcs(scol + e);
        acc = fmad(NEG ? -a : a, index_ok(j, n, err) ? T(x[j]) : T(0), acc);
    }
    return acc;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; ++w) t += sh[w];
    }
    __syncthreads();
    return t;   // valid in thread 0
}


// Called by every block after it has a block sum (in thread 0).  The last
// block to arrive combines all partial sums in index order and applies the
// CG scalar update of `mode`.
__device__ void finish_reduction(double v0, double v1, double* partials, double* partials2,
                                 unsigned int* counter, PcgScalars* sc, double* out, int mode,
                                 double* sh);
__device__ __forceinline__ bool finite_dot(double a) { return isfinite(a); }

__device__ void finish_reduction(double v0, double v1, double* partials, double* partials2,
                                 unsigned int* counter, PcgScalars* sc, double* out, int mode,
                                 double* sh) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v0;
        if (mode == kRZFlex) partials2[blockIdx.x] = v1;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a += __ldcg(partials + i);
        if (mode == kRZFlex) b += __ldcg(partials2 + i);
    }
    a = block_sum(a, sh);
    if (mode == kRZFlex) b = block_sum(b, sh);
    if (threadIdx.x != 0) return;
    *counter = 0u;
    // a NaN or infinity in a dot product of the iteration ends the solve
    if (mode != kStore && (!finite_dot(a) || (mode == kRZFlex && !finite_dot(b)))) {
        if (mode == kRR0) {
            sc->rr0 = a;
            sc->rr = a;
            sc->iters = 0;
        }
        sc->status = AMG_ENONFINITE;
        sc->done = 1;
        sc->alpha = 0.0;
        return;
    }
    switch (mode) {
        case kRR0:
            sc->rr0 = a;
            sc->rr = a;
            sc->done = (a == 0.0) ? 1 : 0;
            sc->iters = 0;
            sc->status = 0;
            break;
        case kPQ:
            sc->pq = a;
            if (!(a > 0.0)) {
                sc->status = AMG_ENOTSPD;
                sc->done = 1;
                sc->alpha = 0.0;
            } else {
                sc->alpha = sc->rho / a;
            }
            break;
        case kRR:
            sc->rr = a;
            sc->iters += 1;
            if (a <= sc->tol2 * sc->rr0) sc->done = 1;
            break;
        case kRZ:
            sc->beta = a / sc->rho;
            sc->rho = a;
            break;
        case kRZFlex:
            sc->beta = b / sc->rho;
            sc->rho = a;
            break;
        case kRho0:
            sc->rho = a;
            break;
        default:
            out[0] = a;
            break;
    }
}

// Condition of the device-side PCG loop, evaluated after each x/r update:
// continue while ||r|| > tol ||r_0||, p.Ap > 0 and fewer than maxit
// iterations.  The evaluation count is a second, independent bound.
__global__ void k_cg_continue(cudaGraphConditionalHandle h, PcgScalars* sc) {
    const int32_t loops = ++sc->loops;
    const bool go = sc->done == 0 && sc->status == 0 && sc->iters < sc->maxit && loops < sc->maxit;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// V-cycle kernels
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// V-cycle passes
//
// Row updates gather their neighbour values in unrolled batches: a lane first
// loads the column indices and values of up to kUnroll of its entries, then
// all the neighbour values, then does the FMAs.  On the coarse levels, where a
// pass is a few thousand rows, the kernel time is the length of its chain of
// dependent loads, and batching cuts that chain to three round trips.
//
// Neighbour values come in three forms:
//   kNbrX        x_j for positions j < jmax; positions >= jmax hold rows of
//                later colours, which are still zero during the forward sweep
//                of pre-smoothing, and are skipped;
//   kNbrFirst    b_j / A_jj for j < jmax: the colour-0 values of the first
//                pass from a zero guess, recomputed instead of read back.
// (Prolongating the other colour's values on the fly inside the first
// post-smoothing pass of a two-colour level was measured slower than a
// separate prolongation kernel: six gathers of agg, t and e per row.)
// ---------------------------------------------------------------------------
enum NbrMode : int { kNbrX = 0, kNbrFirst = 1 };

constexpr int kUnroll = 8;

template <int MODE, typename T>
__device__ __forceinline__ T nbr_value(int j, const T* x, const T* b, const T* __restrict__ dinv) {
    if (MODE == kNbrFirst) return b[j] * dinv[j];
    return x[j];
}

// The row sum starts from acc(), which reads vectors of the solve: it and all
// neighbour values are read after pdl_wait().  With several lanes per row the
// first batch of column indices and values (setup-time data) is loaded before
// it, so those loads overlap the predecessor kernel.
// LPR = lanes per row (1, 2, 4 or 8).  The fine level has kernels of its own
// (below), with the matrix staged in shared memory.
constexpr int kFine = 0;
template <int LPR>
__host__ __device__ constexpr int lanes_of() { return LPR == kFine ? 1 : LPR; }
// entries per lane gathered in one batch: with fewer lanes per row a lane
// takes more of the row, still in one batch for the usual coarse widths
template <int LPR>
__host__ __device__ constexpr int unroll_of() { return LPR == 1 ? 24 : LPR == 2 ? 12 : kUnroll; }

struct PdlWait {
    __device__ void operator()() const { pdl_wait(); }
};

// Wait: what the row does between loading its first batch of setup-time
// entries and reading the first vector value (the predecessor's completion,
// or a dependency wait).
template <int LPR, int MODE, typename T, typename AccF, typename Wait = PdlWait>
__device__ __forceinline__ T row_update(int64_t base, int len, int width, int lane, int jmax,
                                        const int32_t* __restrict__ scol,
                                        const T* __restrict__ sval, const T* x,
                                        const T* b, const T* __restrict__ dinv, int nrows,
                                        int32_t* err, AccF acc, Wait wait = Wait()) {
    static_assert(LPR != kFine, "the fine level uses the staged kernels");
    // every lane of the warp runs the same number of batches (the slice width
    // bounds every row length), so the warp-wide votes below see all 32 lanes
    constexpr int G = lanes_of<LPR>();
    constexpr int U = unroll_of<LPR>();
    constexpr int per = G * U;
    const int batches = (width + per - 1) / per;
    int j[U];
    T a[U];
    auto load_batch = [&](int it) {
        const int k0 = lane + it * per;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * G;
            const bool in = k < len;
            const int64_t ee = base + 32 * (int64_t)(in ? k : 0);
            j[u] = in ? scol[ee] : jmax;
            a[u] = in ? sval[ee] : T(0);
            // checked build: a stored index out of range is skipped (and recorded)
            if (kChecks && in && !index_ok(j[u], nrows, err)) j[u] = jmax;
        }
    };
    load_batch(0);
    wait();
    // two partial sums halve the chain of dependent float64 FMAs
    T s = lane == 0 ? acc() : T(0), s1 = T(0);
    for (int it = 0; it < batches; ++it) {
        if (it > 0) load_batch(it);
        // slots past the longest row of the warp are skipped by a warp-uniform
        // branch: a predicated-off float64 FMA would still occupy the pipe
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = T(0);
            if (__any_sync(0xffffffffu, j[u] < jmax) && j[u] < jmax)
                v[u] = nbr_value<MODE, T>(j[u], x, b, dinv);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (__any_sync(0xffffffffu, j[u] < jmax) && j[u] < jmax) {
                if (u & 1) s1 = fmad(-a[u], v[u], s1);
                else s = fmad(-a[u], v[u], s);
            }
    }
    return group_sum<G>(s + s1);
}

// Rows handled by a launch: LPR lanes per row, rows from r0 rounded down to a
// slice boundary so that warps read whole slices.
template <int LPR>
struct RowOf {
    int row, lane;
    bool valid;
    __device__ RowOf(int r0, int r1, int bid) {
        constexpr int G = lanes_of<LPR>();
        const int64_t tt = bid * (int64_t)blockDim.x + threadIdx.x;
        row = (r0 & ~31) + (int)(tt / G);
        lane = (int)(tt % G);
        valid = row >= r0 && row < r1;
    }
};

// Fused first two forward passes of the pre-smoother from a zero initial
// guess: rows of colour 0 ([0, c1)) have only zero neighbours, so
// x_i = b_i / A_ii; rows of colour 1 ([c1, c2)) see colour-0 neighbours (their
// new values b_j / A_jj) and zeros.  Arguments: c1 = jmax, c2 = r1, dv = 1/A_ii.
template <int LPR, typename T>
struct FirstBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int c1 = a.jmax, c2 = a.r1;
        const int64_t sw = a.sw;
        const uint16_t* __restrict__ rlen = a.rlen;
        const int32_t* __restrict__ scol = a.scol;
        const T* __restrict__ sval = static_cast<const T*>(a.sval);
        const T* __restrict__ dinv = static_cast<const T*>(a.dv);
        const T* b = static_cast<const T*>(a.b);
        T* x = static_cast<T*>(a.x);
        pdl_launch_dependents();
        const RowOf<LPR> R(0, c2, bid);
        const int rr = R.valid ? R.row : 0;
        // colour-0 rows take no neighbour term (length 0: s = b_i exactly); every
        // lane of the warp still reaches the shuffles of the group sum
        const int len = (R.valid && rr >= c1) ? (int)rlen[rr] : 0;
        const int64_t base = (int64_t)(rr >> 5) * sw + (rr & 31);
        const T di = R.valid ? dinv[rr] : T(0);
        const T s = row_update<LPR, kNbrFirst, T>(base, len, (int)(sw >> 5), R.lane, c1, scol, sval, x,
                                                   b, dinv, a.n, a.err,
                                                   [&] { return R.valid ? b[rr] : T(0); });
        if (R.valid && R.lane == 0) x[rr] = s * di;
    }
};

// One Gauss-Seidel update of the rows [r0, r1) of one colour:
//   x_i = (b_i - sum_{j != i, j < jmax} A_ij x_j) / A_ii.
// Rows of one colour are not coupled, so they update in parallel.
// Arguments: r0, r1, jmax, dv = 1/A_ii.
template <int LPR, typename T>
struct PassBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int r0 = a.r0, r1 = a.r1, jmax = a.jmax;
        const int64_t sw = a.sw;
        const uint16_t* __restrict__ rlen = a.rlen;
        const int32_t* __restrict__ scol = a.scol;
        const T* __restrict__ sval = static_cast<const T*>(a.sval);
        const T* __restrict__ dinv = static_cast<const T*>(a.dv);
        const T* b = static_cast<const T*>(a.b);
        T* x = static_cast<T*>(a.x);
        pdl_launch_dependents();
        const RowOf<LPR> R(r0, r1, bid);
        const int rr = R.valid ? R.row : r0;
        const int64_t base = (int64_t)(rr >> 5) * sw + (rr & 31);
        const T di = R.valid ? dinv[rr] : T(0);
        const T s = row_update<LPR, kNbrX, T>(base, R.valid ? (int)rlen[rr] : 0, (int)(sw >> 5),
                                              R.lane, jmax, scol, sval, x, b, dinv, a.n, a.err,
                                              [&] { return R.valid ? b[rr] : T(0); });
        if (R.valid && R.lane == 0) x[rr] = s * di;
    }
};

// r = b - A x for rows [r0, n).  Arguments: r0, r1 = n, dv = A_ii, out = r.
template <int LPR, typename T>
struct ResidualBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int r0 = a.r0, n = a.r1;
        const int64_t sw = a.sw;
        const uint16_t* __restrict__ rlen = a.rlen;
        const int32_t* __restrict__ scol = a.scol;
        const T* __restrict__ sval = static_cast<const T*>(a.sval);
        const T* __restrict__ diag = static_cast<const T*>(a.dv);
        const T* b = static_cast<const T*>(a.b);
        const T* x = static_cast<const T*>(a.x);
        T* r = static_cast<T*>(a.out);
        pdl_launch_dependents();
        const RowOf<LPR> R(r0, n, bid);
        const int rr = R.valid ? R.row : r0;
        const int64_t base = (int64_t)(rr >> 5) * sw + (rr & 31);
        const T dg = R.valid ? diag[rr] : T(0);
        const T v = row_update<LPR, kNbrX, T>(
            base, R.valid ? (int)rlen[rr] : 0, (int)(sw >> 5), R.lane, n, scol, sval, x,
            (const T*)nullptr, (const T*)nullptr, a.n, a.err,
            [&] { return R.valid ? fmad(-dg, x[rr], b[rr]) : T(0); });
        if (R.valid && R.lane == 0) r[rr] = v;
    }
};

// ---------------------------------------------------------------------------
// Dependency-driven sweep (see SweepPlan in device.h): every colour pass of a
// symmetric Gauss-Seidel sweep in one launch, one block per item of rows.
// The rows of an item are updated exactly as PassBody (and, for the first
// pass from a zero guess, FirstBody) updates them, so the results are those of
// the pass-per-launch kernels; only the waits between passes differ.
// ---------------------------------------------------------------------------
constexpr long long kDepSpinLimit = 1LL << 20;   // polls per dependency (over a second)

// polls are relaxed loads; once a warp has seen everything it waits for,
// one acquire fence (after the warp barrier) orders the block's later reads
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A persistent grid of G co-resident blocks (a cooperative launch guarantees
// co-residency); block g takes items g, g + G, g + 2G, ... in order.  An item
// depends only on smaller items, and every block takes its items in
// increasing order, so the block holding the smallest unfinished item always
// has what it waits for: the sweep cannot deadlock.  The launch's epoch comes
// from a counter of block arrivals (G per launch).
template <int LPR, typename T>
__global__ void __launch_bounds__(kBlock) k_sweep(int npass, const SweepPass* __restrict__ passes,
                                                  int items, const int32_t* __restrict__ dep_ptr,
                                                  const int32_t* __restrict__ dep, uint32_t* flag,
                                                  unsigned long long* done,
                                                  unsigned long long* arrive, int32_t* failed,
                                                  int64_t sw, const uint16_t* __restrict__ rlen,
                                                  const int32_t* __restrict__ scol,
                                                  const T* __restrict__ sval,
                                                  const T* __restrict__ dinv, const T* b, T* x,
                                                  int32_t* err, int nrows) {
    __shared__ SweepPass sp[kSweepMaxPasses];
    __shared__ uint32_t s_epoch;
    __shared__ int s_ok;
    for (int i = threadIdx.x; i < npass; i += blockDim.x) sp[i] = passes[i];
    if (threadIdx.x == 0) {
        s_epoch = (uint32_t)(atomicAdd(arrive, 1ull) / gridDim.x) + 1u;
        s_ok = 1;
    }
    __syncthreads();
    const uint32_t epoch = s_epoch;
    constexpr int G = lanes_of<LPR>();
    const int rows_per = (int)blockDim.x / G;
    const int lane = (int)threadIdx.x % G;
    int p = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        while (p + 1 < npass && sp[p + 1].item0 <= item) ++p;
        const SweepPass P = sp[p];
        const int row = (P.r0 & ~31) + (item - P.item0) * rows_per + (int)threadIdx.x / G;
        const bool valid = row >= P.r0 && row < P.r1;
        const int rr = valid ? row : P.r0;
        const int64_t base = (int64_t)(rr >> 5) * sw + (rr & 31);
        const T di = valid ? dinv[rr] : T(0);
        const int len = (valid && !P.first) ? (int)rlen[rr] : 0;
        // warp 0 polls the item's dependencies (a lane per dependency, bounded);
        // the block then reads x
        auto wait = [&] {
            if (threadIdx.x < 32) {
                bool ok = true;
                const int k1 = dep_ptr[item + 1];
                for (int k = dep_ptr[item] + (int)threadIdx.x; k < k1 && ok; k += 32) {
                    const int d = dep[k];
                    for (long long it = 0;; ++it) {
                        bool sat;
                        if (d >= 0) {
                            sat = ld_relaxed_u32(flag + d) == epoch;
                        } else {
                            const int q = -d - 1;
                            sat = ld_relaxed_u64(done + q) >=
                                  (unsigned long long)epoch * (unsigned long long)sp[q].tiles;
                        }
                        if (sat) break;
                        if (it >= kDepSpinLimit || *(volatile int32_t*)failed != 0) {
                            ok = false;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                ok = __all_sync(0xffffffffu, ok);
                __syncwarp();   // orders every lane's polls before lane 0's acquire fence
                if (threadIdx.x == 0) {
                    fence_acq_rel_gpu();
                    if (!ok) {
                        s_ok = 0;
                        atomicExch(failed, 1);
                        atomicExch(err, AMG_ETIMEOUT);
                    }
                }
            }
            __syncthreads();
        };
        const T v = row_update<LPR, kNbrX, T>(base, len, (int)(sw >> 5), lane, P.jmax, scol, sval, x,
                                              b, dinv, nrows, err,
                                              [&] { return valid ? b[rr] : T(0); }, wait);
        if (!s_ok) return;
        if (valid && lane == 0) x[rr] = v * di;
        __syncthreads();
        if (threadIdx.x == 0) {   // release: the block's writes (ordered by the barrier) first
            st_release_u32(flag + item, epoch);
            red_release_add_u64(done + p, 1ull);
        }
    }
}

// ---------------------------------------------------------------------------
// Fine-level kernels: the matrix staged in shared memory by the bulk-copy
// engine.
//
// A block of kBlock threads owns kBlock / 32 consecutive slices, one row per
// thread.  Those slices are contiguous in scol and sval, so one thread starts
// two cp.async.bulk copies of them into shared memory, completing on an
// mbarrier, before the block waits for its predecessor kernel.  The matrix
// stream (about two thirds of the bytes of a fine-level pass) is then in
// flight without holding registers, in one request per array and block
// instead of one per warp and entry.  The copies carry an evict-first L2
// policy: the fine matrix is read once per pass and is larger than L2, and
// keeping it out of L2 leaves the coarse levels resident there from one
// V-cycle to the next.  Row lengths and diagonals are loaded evict-first too.
// The same kernels run on the coarse levels, from a copy whose slices are
// padded only to their own longest row where that saves more than a tenth
// (the block's start and its warps' slices then come from the slice offsets),
// with a per-level preferred L1/shared-memory split for their gathers.
// ---------------------------------------------------------------------------
constexpr int kFineBlock = 256;                    // rows (threads) per fine-level block
constexpr int kSlicesPerBlock = kFineBlock / 32;
constexpr long long kStageSpinLimit = 1LL << 18;   // about 1 s of polls on GB300

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Every thread of the block: wait (bounded) for the copies on `bar`.  Returns
// false, with AMG_ETIMEOUT recorded in *err, if they have not completed within
// the spin limit; the decision is one for the whole block, so that no thread
// waits at a later barrier for threads that gave up.
__device__ bool stage_wait(uint64_t* bar, int32_t* err, long long limit = kStageSpinLimit) {
    const uint32_t ub = smem_u32(bar);
    uint32_t done = 0;
    for (long long it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(ub) : "memory");
    const int all = __syncthreads_and((int)done);
    if (!all && threadIdx.x == 0) atomicExch(err, AMG_ETIMEOUT);
    return all != 0;
}

// Stage the block's `nsl` slices, starting at slice `slice0` (common width W),
// into shared memory as they are: the block's slices are contiguous, so
// thread 0 issues one copy per array against one mbarrier.  Every thread of
// the block calls this and gets the position of its row's entry 0 (entry k at
// loc + 32 k).  Returns false, with AMG_ETIMEOUT recorded in *err, if the
// copies have not completed within the spin limit.
template <typename T>
__device__ bool stage_slices(int64_t slice0, int nsl, int width, const int32_t* scol, const T* sval,
                             int32_t* s_col, T* s_val, uint64_t* bar, int32_t* err, int& loc) {
    const int w = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    loc = w * 32 * width + lane;
    if (width == 0) return true;   // no off-diagonal entries: nothing to stage
    if (threadIdx.x == 0) {
        const uint32_t ub = smem_u32(bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ub) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t ent = (uint32_t)nsl * 32u * (uint32_t)width;
        const int64_t e0 = slice0 * 32 * width;
        uint64_t state, pol;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                     : "=l"(state) : "r"(ub), "r"(ent * (4u + (uint32_t)sizeof(T))) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
            " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(s_col)), "l"(scol + e0), "r"(ent * 4u),
            "r"(ub), "l"(pol) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
            " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(s_val)), "l"(sval + e0),
            "r"(ent * (uint32_t)sizeof(T)), "r"(ub), "l"(pol) : "memory");
    }
    __syncthreads();
    return stage_wait(bar, err);
}

// Stage the block's `nsl` slices from the layout with per-slice widths: slice
// s is padded only to its own longest row K_s and starts at soff[s] (entry k
// of lane i at soff[s] + 32 k + i).  The block's slices are contiguous, so
// thread 0 issues one copy per array against one mbarrier, and the tile is
// laid out like the global arrays.  Every thread calls this and gets the
// position of its row's entry 0 in the tile.  Returns false, with
// AMG_ETIMEOUT recorded in *err, if the copies have not completed within the
// spin limit.
// Slice offsets are read with an evict-last L2 policy: every block's copy
// waits for them, and the level's gathers would otherwise push them out of L2.
__device__ __forceinline__ int64_t ld_offset(const int64_t* p) {
    uint64_t pol;
    int64_t v;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("ld.global.nc.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
}

template <typename T>
__device__ bool stage_own_width(int64_t slice0, int nsl, const int64_t* soff, const int32_t* ccol,
                                const T* cval, int32_t* s_col, T* s_val, uint64_t* bar, int32_t* err,
                                int& loc) {
    const int w = (int)(threadIdx.x >> 5);
    const int64_t e0 = ld_offset(soff + slice0);
    loc = (int)(ld_offset(soff + slice0 + min(w, nsl)) - e0) + (int)(threadIdx.x & 31);
    if (threadIdx.x == 0) {
        const uint32_t ub = smem_u32(bar);
        const uint32_t ent = (uint32_t)(ld_offset(soff + slice0 + nsl) - e0);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ub) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        uint64_t state;
        if (ent == 0) {
            asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(ub) : "memory");
        } else {
            uint64_t pol;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                         : "=l"(state) : "r"(ub), "r"(ent * (4u + (uint32_t)sizeof(T))) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(s_col)), "l"(ccol + e0), "r"(ent * 4u),
                "r"(ub), "l"(pol) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(s_val)), "l"(cval + e0),
                "r"(ent * (uint32_t)sizeof(T)), "r"(ub), "l"(pol) : "memory");
        }
    }
    __syncthreads();
    return stage_wait(bar, err);
}

// Self-test of the bounded wait: an mbarrier that expects 16 bytes of copies
// that are never issued, so the wait runs out after `limit` polls and records
// AMG_ETIMEOUT.  No copy is in flight when the block exits.
__global__ void k_wait_selftest(int32_t* err, long long limit) {
    __shared__ uint64_t bar;
    const uint32_t ub = smem_u32(&bar);
    if (threadIdx.x == 0) {
        uint64_t state;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ub) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                     : "=l"(state) : "r"(ub), "r"(16u) : "memory");
    }
    __syncthreads();
    stage_wait(&bar, err, limit > 0 ? limit : kStageSpinLimit);
}

// The block's slices, its shared-memory tiles and this thread's row.  The
// tiles hold up to `cap` entries (the level's stage capacity): column indices
// first, then values.
template <typename T>
struct FineTile {
    int64_t slice0;
    int nsl;
    int row;
    int loc;          // offset of this row's entry 0 in the tiles (entry k at loc + 32 k),
                      // set by the staging (stage_tile)
    int32_t* s_col;
    T* s_val;
    __device__ FineTile(int r0, int64_t nslices, int64_t cap, unsigned char* smem, int bid) {
        slice0 = (int64_t)(r0 >> 5) + (int64_t)bid * kSlicesPerBlock;
        nsl = (int)min((int64_t)kSlicesPerBlock, nslices - slice0);
        row = (int)(slice0 * 32) + (int)threadIdx.x;
        loc = (int)(threadIdx.x & 31);
        s_col = reinterpret_cast<int32_t*>(smem);
        s_val = reinterpret_cast<T*>(smem + (size_t)cap * sizeof(int32_t));
    }
};

// acc - sum over the staged entries of this thread's row with j < jmax of
// A_ij nbr(j).  (Batching the gathers eight at a time was measured slower in
// float64 on the 512^3 anisotropic workload: 3.07 s against 2.88 s a solve.)
template <typename T, typename Nbr>
__device__ __forceinline__ T fine_row(const FineTile<T>& F, int len, int jmax, Nbr nbr, T acc,
                                      int nrows, int32_t* err) {
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
        const int j = F.s_col[F.loc + 32 * k];
        const T a = F.s_val[F.loc + 32 * k];
        if (index_ok(j, nrows, err) && j < jmax) acc = fmad(-a, nbr(j), acc);
    }
    return acc;
}

// Stage the block's slices (per-slice widths when soff is set, else the
// common width) and return whether the copies completed.
template <typename T>
__device__ __forceinline__ bool stage_tile(FineTile<T>& F, const VArgs& a, uint64_t* bar) {
    const T* sval = static_cast<const T*>(a.sval);
    if (a.soff)
        return stage_own_width(F.slice0, F.nsl, a.soff, a.scol, sval, F.s_col, F.s_val, bar, a.err,
                               F.loc);
    return stage_slices(F.slice0, F.nsl, a.width, a.scol, sval, F.s_col, F.s_val, bar, a.err, F.loc);
}

// First forward pass from a zero guess on a level with the staged kernels,
// colour 0 (rows [0, c1)): x_i = b_i / A_ii; the colour-1 rows follow as an
// ordinary staged pass whose later-colour neighbours (positions >= c1) are
// still zero.  With r_in set (float32 V-cycle inside float64 CG) this kernel
// first forms the scaled right-hand side b_i = r_i / s_i (isq = 1/s) of every
// row.  It also zeroes the next level's right-hand side for the fused
// residual-restriction kernel.  Arguments: r1 = c1, n = rows of b, dv = 1/A_ii,
// out = the vector to zero (nc entries), rin, isq.
template <typename T>
struct FineFirst0Body {
    static __device__ __forceinline__ void run(int bid, int gdim, const VArgs& a) {
        const int c1 = a.r1, nb = a.n, nc = a.nc;
        const T* __restrict__ dinv = static_cast<const T*>(a.dv);
        T* b = const_cast<T*>(static_cast<const T*>(a.b));
        T* x = static_cast<T*>(a.x);
        T* bc_zero = static_cast<T*>(a.out);
        const double* r_in = a.rin;
        const double* __restrict__ isq = a.isq;
        pdl_launch_dependents();
        pdl_wait();
        const int stride = gdim * blockDim.x;
        for (int i = bid * blockDim.x + threadIdx.x; i < nb; i += stride) {
            T bi;
            if (r_in) {
                bi = (T)(r_in[i] * isq[i]);
                b[i] = bi;
            } else {
                bi = b[i];
            }
            if (i < c1) x[i] = bi * dinv[i];
        }
        if (bc_zero)
            for (int i = bid * blockDim.x + threadIdx.x; i < nc; i += stride) bc_zero[i] = T(0);
    }
};

// The staged pass of the rows [r0, r1) of one colour.  With z set (the last
// pass over these rows in a float32 V-cycle) the new value also goes out
// unscaled in float64: z_i = x_i / s_i (isq = 1/s).  Arguments: r0, r1, jmax,
// width, nslices, cap, soff, dv = 1/A_ii, z, isq, err.
template <typename T>
struct FinePassBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int r0 = a.r0, r1 = a.r1, jmax = a.jmax;
        const int64_t nslices = a.nslices, cap = a.cap;
        const uint16_t* __restrict__ rlen = a.rlen;
        const T* __restrict__ dinv = static_cast<const T*>(a.dv);
        const T* b = static_cast<const T*>(a.b);
        T* x = static_cast<T*>(a.x);
        double* z_out = a.z;
        const double* __restrict__ isq = a.isq;
        extern __shared__ __align__(128) unsigned char smem[];
        __shared__ uint64_t bar;
        pdl_launch_dependents();
        FineTile<T> F(r0, nslices, cap, smem, bid);
        const bool valid = F.row >= r0 && F.row < r1;
        const int len = valid ? (int)__ldcs(rlen + F.row) : 0;
        const T di = valid ? __ldcs(dinv + F.row) : T(0);
        if (!stage_tile(F, a, &bar)) return;
        pdl_wait();
        if (!valid) return;
        const T xi = fine_row<T>(F, len, jmax, [&](int j) { return x[j]; }, b[F.row], a.n, a.err) * di;
        x[F.row] = xi;
        if (z_out) z_out[F.row] = (double)xi * isq[F.row];
    }
};

// The staged residual r = b - A x of the rows [r0, n).  Arguments: r0,
// r1 = n, width, nslices, cap, soff, dv = A_ii, out = r, err.
template <typename T>
struct FineResidualBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int r0 = a.r0, n = a.r1;
        const int64_t nslices = a.nslices, cap = a.cap;
        const uint16_t* __restrict__ rlen = a.rlen;
        const T* __restrict__ diag = static_cast<const T*>(a.dv);
        const T* b = static_cast<const T*>(a.b);
        const T* x = static_cast<const T*>(a.x);
        T* r = static_cast<T*>(a.out);
        extern __shared__ __align__(128) unsigned char smem[];
        __shared__ uint64_t bar;
        pdl_launch_dependents();
        FineTile<T> F(r0, nslices, cap, smem, bid);
        const bool valid = F.row >= r0 && F.row < n;
        const int len = valid ? (int)__ldcs(rlen + F.row) : 0;
        const T dg = valid ? __ldcs(diag + F.row) : T(0);
        if (!stage_tile(F, a, &bar)) return;
        pdl_wait();
        if (!valid) return;
        r[F.row] = fine_row<T>(F, len, n, [&](int j) { return x[j]; }, fmad(-dg, x[F.row], b[F.row]),
                               a.n, a.err);
    }
};

// Residual and restriction in one pass on a two-colour fine level: the rows
// of colour 1 ([c1, n)) are sorted by coarse index, so the rows of one
// aggregate are consecutive (with more colours an aggregate would recur in
// every colour block).  Each thread stores (t_i) r_i in shared memory; the
// first row of every run of equal coarse index inside the block sums the run
// in order and adds it to bc (zeroed by the first pass).  A run is shorter
// than a block, so a coarse entry receives at most two additions onto zero (a
// run cut by a block boundary), whose result does not depend on their order:
// the sum stays deterministic.  Arguments: r0 = c1, r1 = n, width, nslices,
// cap, soff, dv = A_ii, idx = aggregate map, t, out = bc, err.
template <typename T, bool SCALED>
struct FineResRestrictBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int c1 = a.r0, n = a.r1;
        const int64_t nslices = a.nslices, cap = a.cap;
        const uint16_t* __restrict__ rlen = a.rlen;
        const T* __restrict__ diag = static_cast<const T*>(a.dv);
        const T* b = static_cast<const T*>(a.b);
        const T* x = static_cast<const T*>(a.x);
        const int32_t* __restrict__ agg = a.idx;
        const T* __restrict__ t = static_cast<const T*>(a.t);
        T* bc = static_cast<T*>(a.out);
        extern __shared__ __align__(128) unsigned char smem[];
        __shared__ uint64_t bar;
        __shared__ T sv[kFineBlock];
        __shared__ int sk[kFineBlock];
        pdl_launch_dependents();
        FineTile<T> F(c1, nslices, cap, smem, bid);
        const bool valid = F.row >= c1 && F.row < n;
        const int len = valid ? (int)__ldcs(rlen + F.row) : 0;
        const T dg = valid ? __ldcs(diag + F.row) : T(0);
        const int key = valid ? __ldcs(agg + F.row) : -1;
        const T ti = (SCALED && valid) ? __ldcs(t + F.row) : T(1);
        if (!stage_tile(F, a, &bar)) return;
        pdl_wait();
        T v = T(0);
        if (valid) {
            const T ri = fine_row<T>(F, len, n, [&](int j) { return x[j]; },
                                     fmad(-dg, x[F.row], b[F.row]), a.n, a.err);
            v = SCALED ? ti * ri : ri;
        }
        const int tid = threadIdx.x;
        sv[tid] = v;
        sk[tid] = key;
        __syncthreads();
        if (key < 0 || (tid > 0 && sk[tid - 1] == key)) return;
        T sum = v;
        for (int u = tid + 1; u < kFineBlock && sk[u] == key; ++u) sum += sv[u];
        atomicAdd(bc + key, sum);
    }
};

// coarse right-hand side: bc_J = sum over the fine rows i of aggregate J of
// (t_i) r_i, in the stored order (Eq. prolongation: R = P^T).  The lists hold
// the rows of colour >= 1 only: the pre-smoother's last pass updates colour 0,
// whose residual is therefore zero.  Arguments: nc, idx = list pointers,
// idx2 = list rows, t, b = r, out = bc.
template <typename T, bool SCALED>
struct RestrictBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int nc = a.nc;
        const int32_t* __restrict__ rptr = a.idx;
        const int32_t* __restrict__ ridx = a.idx2;
        const T* __restrict__ t = static_cast<const T*>(a.t);
        const T* r = static_cast<const T*>(a.b);
        T* bc = static_cast<T*>(a.out);
        pdl_launch_dependents();
        const int J = bid * blockDim.x + threadIdx.x;
        if (J >= nc) return;
        const int kb = rptr[J], k1 = rptr[J + 1];
        int i[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) i[u] = (kb + u < k1) ? ridx[kb + u] : -1;
        pdl_wait();
        T s = T(0);
        for (int k0 = kb; k0 < k1; k0 += kUnroll) {
            if (k0 > kb) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) i[u] = (k0 + u < k1) ? ridx[k0 + u] : -1;
            }
            T v[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (i[u] >= 0 && !index_ok(i[u], a.n, a.err)) i[u] = -1;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                v[u] = i[u] >= 0 ? (SCALED ? t[i[u]] * r[i[u]] : r[i[u]]) : T(0);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (i[u] >= 0) s += v[u];
        }
        bc[J] = s;
    }
};

// x_i += omega (t_i) e_{agg(i)} on rows [r0, n): piecewise-constant
// prolongation with the over-correction factor omega.  Callers pass r0 = the
// first row of colour 1: the post-smoother's first pass recomputes colour 0
// without reading its old values.  Arguments: r0, r1 = n, idx = aggregate
// map, t, b = e, x, omega.
template <typename T, bool SCALED>
struct ProlongBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int r0 = a.r0, n = a.r1;
        const int32_t* __restrict__ agg = a.idx;
        const T* __restrict__ t = static_cast<const T*>(a.t);
        const T* e = static_cast<const T*>(a.b);
        T* x = static_cast<T*>(a.x);
        const T omega = (T)a.omega;
        pdl_launch_dependents();
        const int i = r0 + (int)(bid * blockDim.x + threadIdx.x);
        if (i >= n) return;
        const int g = agg[i];
        if (g < 0 || !index_ok(g, a.nc, a.err)) return;
        const T w = SCALED ? omega * t[i] : omega;
        pdl_wait();
        x[i] = fmad(w, e[g], x[i]);
    }
};

// x = M b, M dense row-major (coarsest-level solve with the inverse formed at
// setup); one warp per row, float64 arithmetic.  A float32 b is first copied,
// converted to float64, into shared memory by the block: every row reads all
// of b, and reading it as float32 would cost a conversion per matrix entry on
// the float64 pipe.  A float64 b is read directly (L1 serves the rows of the
// block).  Arguments: n, dv = M (float64), b, x.
template <typename TB>
struct GemvBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        constexpr int kPre = 4;   // row entries per lane loaded before the wait
        constexpr bool kStage = !std::is_same<TB, double>::value;
        const int n = a.n;
        const double* __restrict__ M = static_cast<const double*>(a.dv);
        const TB* b = static_cast<const TB*>(a.b);
        TB* x = static_cast<TB*>(a.x);
        extern __shared__ double sbuf[];
        pdl_launch_dependents();
        const int lane = threadIdx.x & 31;
        const int row = (int)((bid * (int64_t)blockDim.x + threadIdx.x) >> 5);
        const double* m = M + (size_t)min(row, n - 1) * n;
        double m0[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) m0[u] = (lane + 32 * u < n) ? m[lane + 32 * u] : 0.0;
        pdl_wait();
        const double* sb;
        if (kStage) {
            for (int k = threadIdx.x; k < n; k += blockDim.x) sbuf[k] = (double)b[k];
            __syncthreads();
            sb = sbuf;
        } else {
            sb = reinterpret_cast<const double*>(b);
        }
        if (row >= n) return;
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < kPre; ++u)
            if (lane + 32 * u < n) s += m0[u] * sb[lane + 32 * u];
        for (int k = lane + 32 * kPre; k < n; k += 32) s += m[k] * sb[k];
        s = group_sum<32>(s);
        if (lane == 0) x[row] = (TB)s;
    }
};

// Coarsest solve of the float32 V-cycle with the float32 copy of the inverse
// (coarsest_fp32): rows of ld = n rounded up to 4 floats, zero beyond n, read
// as float4 beside the matching float4 of b (16-byte aligned; its last
// partial group read by scalars); one warp per row, float32 products and sums.
__device__ __forceinline__ float4 b_group(const float* __restrict__ b, int n, int q) {
    if (4 * q + 3 < n) return reinterpret_cast<const float4*>(b)[q];
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (4 * q < n) {
        c.x = b[4 * q];
        if (4 * q + 1 < n) c.y = b[4 * q + 1];
        if (4 * q + 2 < n) c.z = b[4 * q + 2];
    }
    return c;
}

// Arguments: n, ld, dv = M (float32), b, x.
struct GemvF32Body {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        constexpr int kU = 4;   // float4 groups of the row per lane in flight
        const int n = a.n, ld = a.ld;
        const float* __restrict__ M = static_cast<const float*>(a.dv);
        const float* __restrict__ b = static_cast<const float*>(a.b);
        float* x = static_cast<float*>(a.x);
        pdl_launch_dependents();
        const int lane = threadIdx.x & 31;
        const int row = (int)((bid * (int64_t)blockDim.x + threadIdx.x) >> 5);
        const int q4 = ld >> 2;
        const float4* m = reinterpret_cast<const float4*>(M + (size_t)min(row, n - 1) * ld);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) v[u] = lane + 32 * u < q4 ? m[lane + 32 * u] : zero;
        pdl_wait();
        if (row >= n) return;
        float acc[kU] = {};
        for (int q = lane;; q += 32 * kU) {
            float4 c[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) c[u] = q + 32 * u < q4 ? b_group(b, n, q + 32 * u) : zero;
            const int qn = q + 32 * kU;
            float4 w[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) w[u] = qn + 32 * u < q4 ? m[qn + 32 * u] : zero;
#pragma unroll
            for (int u = 0; u < kU; ++u)
                acc[u] = fmaf(v[u].x, c[u].x, fmaf(v[u].y, c[u].y, fmaf(v[u].z, c[u].z,
                         fmaf(v[u].w, c[u].w, acc[u]))));
            if (qn >= q4) break;
#pragma unroll
            for (int u = 0; u < kU; ++u) v[u] = w[u];
        }
        float t = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) x[row] = t;
    }
};

__global__ void k_gather(int n, const int32_t* __restrict__ idx, const double* x, double* y) {
    pdl_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = idx[i];
    pdl_wait();
    y[i] = x[j];
}

__global__ void k_scatter(int n, const int32_t* __restrict__ idx, const double* x, double* y) {
    pdl_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = idx[i];
    pdl_wait();
    y[j] = x[i];
}

// float64 -> scaled float32 at V-cycle entry: rhat = r / s, s = sqrt(A_ii).
// Arguments: n, rin = r, isq, x = rhat.
struct ToScaledBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int n = a.n;
        const double* r = a.rin;
        const double* __restrict__ isq = a.isq;
        float* rhat = static_cast<float*>(a.x);
        pdl_launch_dependents();
        const int i = bid * blockDim.x + threadIdx.x;
        if (i >= n) return;
        const double w = isq[i];
        pdl_wait();
        rhat[i] = (float)(r[i] * w);
    }
};

// scaled float32 -> float64 at V-cycle exit: z = zhat / s.
// Arguments: n, b = zhat, isq, z.
struct FromScaledBody {
    static __device__ __forceinline__ void run(int bid, int, const VArgs& a) {
        const int n = a.n;
        const float* zhat = static_cast<const float*>(a.b);
        const double* __restrict__ isq = a.isq;
        double* z = a.z;
        pdl_launch_dependents();
        const int i = bid * blockDim.x + threadIdx.x;
        if (i >= n) return;
        const double w = isq[i];
        pdl_wait();
        z[i] = (double)zhat[i] * w;
    }
};

// ---------------------------------------------------------------------------
// V-cycle launches: a body as its own launch (k_single), or several records
// of one body as one launch (k_batched).  In a batched launch the records'
// grids follow one another; each block finds its record by the running sums
// of the grids (kernel parameters, read through the constant cache) and runs
// the body with the block index inside that record's grid.
// ---------------------------------------------------------------------------
struct VBatch {
    int nrec;
    int bstart[kMaxVBatch + 1];
    int grid[kMaxVBatch];
    VArgs a[kMaxVBatch];
};

template <typename Body>
__global__ void __launch_bounds__(kBlock) k_single(const VArgs a) {
    Body::run((int)blockIdx.x, (int)gridDim.x, a);
}

template <typename Body>
__global__ void __launch_bounds__(kBlock) k_batched(const VBatch p) {
    int r = 0;
    while (r + 1 < p.nrec && p.bstart[r + 1] <= (int)blockIdx.x) ++r;
    Body::run((int)blockIdx.x - p.bstart[r], p.grid[r], p.a[r]);
}

// ---------------------------------------------------------------------------
// CG kernels (level 0, float64, smoothing order)
// ---------------------------------------------------------------------------

// r = b - A x and ||r||^2 (grid-stride over rows)
__global__ void __launch_bounds__(kBlock) k_cg_residual(int n, int64_t sw,
                                                        const uint16_t* __restrict__ rlen,
                                                        const int32_t* __restrict__ scol,
                                                        const double* __restrict__ sval,
                                                        const double* __restrict__ diag,
                                                        const double* __restrict__ b,
                                                        const double* __restrict__ x,
                                                        double* __restrict__ r, double* partials,
                                                        unsigned int* counter, PcgScalars* sc,
                                                        double* out, int mode) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    double acc = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int64_t base = (int64_t)(row >> 5) * sw + (row & 31);
        const double s0 = fmad(-__ldcs(diag + row), x[row], b[row]);
        const double v = sell_row<true>(base, __ldcs(rlen + row), scol, sval, x, s0, n, &sc->status);
        if (r) r[row] = v;
        acc = fmad(v, v, acc);
    }
    const double t = block_sum(acc, sh);
    finish_reduction(t, 0.0, partials, nullptr, counter, sc, out, mode, sh);
}

// q = A p and p.q -> alpha
__global__ void __launch_bounds__(kBlock) k_cg_spmv_pq(int n, int64_t sw,
                                                       const uint16_t* __restrict__ rlen,
                                                       const int32_t* __restrict__ scol,
                                                       const double* __restrict__ sval,
                                                       const double* __restrict__ diag,
                                                       const double* __restrict__ p,
                                                       double* __restrict__ q, double* partials,
                                                       unsigned int* counter, PcgScalars* sc) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    double acc = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int64_t base = (int64_t)(row >> 5) * sw + (row & 31);
        const double pi = p[row];
        const double v = sell_row<false>(base, __ldcs(rlen + row), scol, sval, p,
                                         __ldcs(diag + row) * pi, n, &sc->status);
        q[row] = v;
        acc = fmad(pi, v, acc);
    }
    const double t = block_sum(acc, sh);
    finish_reduction(t, 0.0, partials, nullptr, counter, sc, nullptr, kPQ, sh);
}

// x += alpha p, r -= alpha q, ||r||^2 -> convergence test
__global__ void __launch_bounds__(kBlock) k_cg_update(int n, double* __restrict__ x,
                                                      double* __restrict__ r,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ q,
                                                      double* partials, unsigned int* counter,
                                                      PcgScalars* sc) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    const double alpha = sc->alpha;
    double acc = 0.0;
    // pairs of elements through 128-bit accesses (the vectors are 256-byte
    // aligned allocations), the odd last element by the first thread
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    double2* x2 = reinterpret_cast<double2*>(x);
    double2* r2 = reinterpret_cast<double2*>(r);
    const double2* p2 = reinterpret_cast<const double2*>(p);
    const double2* q2 = reinterpret_cast<const double2*>(q);
#pragma unroll 2
    for (int i = tid; i < (n >> 1); i += stride) {
        const double2 xv = x2[i], pv = p2[i], rv = r2[i], qv = q2[i];
        x2[i] = make_double2(xv.x + alpha * pv.x, xv.y + alpha * pv.y);
        const double2 v = make_double2(rv.x - alpha * qv.x, rv.y - alpha * qv.y);
        r2[i] = v;
        acc = fmad(v.x, v.x, acc);
        acc = fmad(v.y, v.y, acc);
    }
    if ((n & 1) && tid == 0) {
        const int i = n - 1;
        x[i] += alpha * p[i];
        const double v = r[i] - alpha * q[i];
        r[i] = v;
        acc = fmad(v, v, acc);
    }
    const double t = block_sum(acc, sh);
    finish_reduction(t, 0.0, partials, nullptr, counter, sc, nullptr, kRR, sh);
}

// rho = r.z (and, flexible, r.(z - z_old)) -> beta; mode kRho0 sets p = z too
__global__ void __launch_bounds__(kBlock) k_cg_rz(int n, const double* __restrict__ r,
                                                  const double* __restrict__ z,
                                                  const double* __restrict__ zold,
                                                  double* __restrict__ p, double* partials,
                                                  double* partials2, unsigned int* counter,
                                                  PcgScalars* sc, int mode) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    double a = 0.0, b = 0.0;
    // pairs of elements through 128-bit accesses, the odd last element by the
    // first thread
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    const double2* r2 = reinterpret_cast<const double2*>(r);
    const double2* z2 = reinterpret_cast<const double2*>(z);
    const double2* o2 = reinterpret_cast<const double2*>(zold);
#pragma unroll 2
    for (int i = tid; i < (n >> 1); i += stride) {
        const double2 rv = r2[i], zv = z2[i];
        a += rv.x * zv.x;
        a += rv.y * zv.y;
        if (mode == kRZFlex) {
            const double2 ov = o2[i];
            b += rv.x * (zv.x - ov.x);
            b += rv.y * (zv.y - ov.y);
        }
        if (mode == kRho0) reinterpret_cast<double2*>(p)[i] = zv;
    }
    if ((n & 1) && tid == 0) {
        const int i = n - 1;
        const double ri = r[i], zi = z[i];
        a += ri * zi;
        if (mode == kRZFlex) b += ri * (zi - zold[i]);
        if (mode == kRho0) p[i] = zi;
    }
    const double ta = block_sum(a, sh);
    double tb = 0.0;
    if (mode == kRZFlex) tb = block_sum(b, sh);
    finish_reduction(ta, tb, partials, partials2, counter, sc, nullptr, mode, sh);
}

// p = z + beta p (and z_old = z for the flexible variant)
__global__ void __launch_bounds__(kBlock) k_cg_p(int n, const double* __restrict__ z,
                                                 double* __restrict__ p, double* __restrict__ zold,
                                                 const PcgScalars* sc) {
    pdl_launch_dependents();
    pdl_wait();
    const double beta = sc->beta;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    const double2* z2 = reinterpret_cast<const double2*>(z);
    double2* p2 = reinterpret_cast<double2*>(p);
#pragma unroll 2
    for (int i = tid; i < (n >> 1); i += stride) {
        const double2 zv = z2[i], pv = p2[i];
        p2[i] = make_double2(zv.x + beta * pv.x, zv.y + beta * pv.y);
        if (zold) reinterpret_cast<double2*>(zold)[i] = zv;
    }
    if ((n & 1) && tid == 0) {
        const int i = n - 1;
        const double zi = z[i];
        p[i] = zi + beta * p[i];
        if (zold) zold[i] = zi;
    }
}

// ---------------------------------------------------------------------------
// BiCGSTAB (level 0, float64, smoothing order) with its scalars on the device.
// Each kernel that ends in dot products combines them with the deterministic
// last-block reduction and applies the scalar step of the iteration there, so
// the iteration needs no host round trip: the host-driven loop reads the
// scalars once per iteration, the graph loop never.  A kernel whose work the
// iteration no longer needs (after a breakdown, or after the first half step
// met the tolerance) returns before touching anything; the decision reads
// scalars written by an earlier kernel, so it is the same for every block.
// ---------------------------------------------------------------------------
enum BiMode : int { kBiStart = 0, kBiRtv = 1, kBiHalf = 2, kBiW = 3, kBiUpdate = 4 };

__device__ void finish_bi(double v0, double v1, double* partials, double* partials2,
                          unsigned int* counter, BiScalars* bs, int mode, double* sh) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v0;
        partials2[blockIdx.x] = v1;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a += __ldcg(partials + i);
        b += __ldcg(partials2 + i);
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x != 0) return;
    *counter = 0u;
    // a NaN or infinity in a dot product of the iteration ends the solve
    if (!finite_dot(a) || !finite_dot(b)) {
        if (mode == kBiStart) {
            bs->r0 = sqrt(a);
            bs->iters = 0;
            bs->rel = 0.0;
        }
        bs->status = AMG_ENONFINITE;
        bs->why = 4;
        return;
    }
    switch (mode) {
        case kBiStart:   // a = r.r
            bs->r0 = sqrt(a);
            bs->rho = a;
            bs->rho_prev = 1.0;
            bs->alpha = 1.0;
            bs->w = 1.0;
            bs->rel = bs->r0 > 0.0 ? 1.0 : 0.0;
            bs->done = !(bs->rel > bs->tol);
            bs->iters = 0;
            bs->status = 0;
            bs->half = 0;
            bs->why = 0;
            bs->loops = 0;
            break;
        case kBiRtv:     // a = rt.v
            bs->rtv = a;
            if (a == 0.0) {
                bs->status = AMG_ENOTCONV;
                bs->why = 2;
            } else {
                bs->alpha = bs->rho / a;
            }
            break;
        case kBiHalf: {  // a = s.s
            bs->iters += 1;
            const double srel = sqrt(a) / bs->r0;
            if (srel <= bs->tol) {
                bs->half = 1;
                bs->done = 1;
                bs->rel = srel;
            }
            break;
        }
        case kBiW:       // a = t.s, b = t.t
            bs->ts = a;
            bs->tt = b;
            if (b == 0.0) {
                bs->status = AMG_ENOTCONV;
                bs->why = 3;
            } else {
                bs->w = a / b;
            }
            break;
        default:         // kBiUpdate: a = r.r, b = rt.r
            bs->rel = sqrt(a) / bs->r0;
            bs->rho_prev = bs->rho;
            bs->rho = b;
            bs->done = !(bs->rel > bs->tol);
            break;
    }
}

// r = b - A x, rt = r, and the start scalars from r.r
__global__ void __launch_bounds__(kBlock) k_bi_start(int n, int64_t sw,
                                                     const uint16_t* __restrict__ rlen,
                                                     const int32_t* __restrict__ scol,
                                                     const double* __restrict__ sval,
                                                     const double* __restrict__ diag,
                                                     const double* b, const double* x, double* r,
                                                     double* rt, double* partials, double* partials2,
                                                     unsigned int* counter, BiScalars* bs) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    double a = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int64_t base = (int64_t)(row >> 5) * sw + (row & 31);
        const double s0 = fmad(-__ldcs(diag + row), x[row], b[row]);
        const double v = sell_row<true>(base, __ldcs(rlen + row), scol, sval, x, s0, n, &bs->status);
        r[row] = v;
        rt[row] = v;
        a = fmad(v, v, a);
    }
    const double ta = block_sum(a, sh);
    finish_bi(ta, 0.0, partials, partials2, counter, bs, kBiStart, sh);
}

// search direction: p = r on the first iteration, else
// p = r + beta (p - w v) with beta = (rho / rho_prev) (alpha / w)
__global__ void __launch_bounds__(kBlock) k_bi_direction(int n, const double* r, const double* v,
                                                         double* p, const BiScalars* bs) {
    pdl_launch_dependents();
    pdl_wait();
    if (bs->done || bs->status) return;
    const bool first = bs->iters == 0;
    const double w = bs->w;
    const double beta = (bs->rho / bs->rho_prev) * (bs->alpha / w);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = first ? r[i] : r[i] + beta * (p[i] - w * v[i]);
}

// y = A x with the dot products of the mode: kBiRtv: rt.y; kBiW: s.y and y.y
// (skipped once the iteration has stopped)
__global__ void __launch_bounds__(kBlock) k_bi_spmv(int n, int64_t sw,
                                                    const uint16_t* __restrict__ rlen,
                                                    const int32_t* __restrict__ scol,
                                                    const double* __restrict__ sval,
                                                    const double* __restrict__ diag,
                                                    const double* x, double* y, const double* w,
                                                    double* partials, double* partials2,
                                                    unsigned int* counter, BiScalars* bs, int mode) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    if (bs->status || (mode == kBiW && bs->half)) return;
    double a = 0.0, b = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int64_t base = (int64_t)(row >> 5) * sw + (row & 31);
        const double v = sell_row<false>(base, __ldcs(rlen + row), scol, sval, x,
                                         __ldcs(diag + row) * x[row], n, &bs->status);
        y[row] = v;
        a = fmad(w[row], v, a);
        if (mode == kBiW) b = fmad(v, v, b);
    }
    const double ta = block_sum(a, sh);
    const double tb = block_sum(b, sh);
    finish_bi(ta, tb, partials, partials2, counter, bs, mode, sh);
}

// s = r - alpha v and s.s (the half-step test)
__global__ void __launch_bounds__(kBlock) k_bi_half(int n, const double* r, const double* v,
                                                    double* sv, double* partials,
                                                    double* partials2, unsigned int* counter,
                                                    BiScalars* bs) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    if (bs->status) return;
    const double c = -bs->alpha;
    double a = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double o = fmad(c, v[i], r[i]);
        sv[i] = o;
        a = fmad(o, o, a);
    }
    const double ta = block_sum(a, sh);
    finish_bi(ta, 0.0, partials, partials2, counter, bs, kBiHalf, sh);
}

// x += alpha y + w z, r = s - w t, r.r and rt.r; after a converged half step
// only x += alpha y
__global__ void __launch_bounds__(kBlock) k_bi_update(int n, double* x, const double* y,
                                                      const double* z, const double* s,
                                                      const double* t, double* r, const double* rt,
                                                      double* partials, double* partials2,
                                                      unsigned int* counter, BiScalars* bs) {
    __shared__ double sh[kBlock / 32];
    pdl_launch_dependents();
    pdl_wait();
    if (bs->status) return;
    const double alpha = bs->alpha;
    const int stride = gridDim.x * blockDim.x;
    if (bs->half) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
            x[i] = fmad(alpha, y[i], x[i]);
        return;
    }
    const double w = bs->w;
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        x[i] = x[i] + alpha * y[i] + w * z[i];
        const double ri = s[i] - w * t[i];
        r[i] = ri;
        a = fmad(ri, ri, a);
        b = fmad(rt[i], ri, b);
    }
    const double ta = block_sum(a, sh);
    const double tb = block_sum(b, sh);
    finish_bi(ta, tb, partials, partials2, counter, bs, kBiUpdate, sh);
}

// Condition of the BiCGSTAB loop (a WHILE graph node), evaluated before every
// iteration: stop once converged or broken down, at maxit, or when
// rho = rt.r is zero (a breakdown); the evaluation count is a second bound.
__global__ void k_bi_continue(cudaGraphConditionalHandle h, BiScalars* bs) {
    const int32_t loops = ++bs->loops;
    const int go = bi_continue(*bs) && loops <= bs->maxit + 1;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

inline int blocks_for(int64_t threads) { return (int)((threads + kBlock - 1) / kBlock); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void raise_dyn_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;   // (device, function) -> bytes
    int dev = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return;
    AMG_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
}

thread_local bool t_launch_overlap = false;
int g_overlap_max_blocks = 304;
int g_reduction_blocks = 1216;

int reduction_blocks(int64_t work_threads) {
    int64_t b = (work_threads + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, g_reduction_blocks);
}

inline int row_blocks(int r0, int r1, int lpr, int block = kBlock) {
    const int64_t threads = (int64_t)(r1 - (r0 & ~31)) * std::max(lpr, 1);
    return (int)((threads + block - 1) / block);
}

// lanes per row of a launch over `rows` rows: passes over many rows are
// bound by float64 instruction throughput, which fewer lanes per row use
// better (no cross-lane sums, no idle slots); short passes are bound by
// latency, which more lanes per row shorten
inline int launch_lpr(const DevLevel& L, int rows) {
    return rows >= L.wide_rows ? L.lpr_wide : L.lpr;
}

#define AMG_LPR_DISPATCH(lpr, CALL)                          \
    switch (lpr) {                                           \
        case 1: { constexpr int LPR = 1; CALL; } break;      \
        case 2: { constexpr int LPR = 2; CALL; } break;      \
        case 4: { constexpr int LPR = 4; CALL; } break;      \
        default: { constexpr int LPR = 8; CALL; } break;     \
    }

template <typename T>
struct LevelArrays;
template <>
struct LevelArrays<double> {
    const double *sval, *cval, *dinv, *diag, *t;
    explicit LevelArrays(const DevLevel& L)
        : sval(L.sval), cval(L.cval), dinv(L.dinv), diag(L.diag), t(nullptr) {}
};
template <>
struct LevelArrays<float> {
    const float *sval, *cval, *dinv, *diag, *t;
    explicit LevelArrays(const DevLevel& L)
        : sval(L.sval32), cval(L.cval32), dinv(L.dinv32), diag(L.diag32), t(L.t32) {}
};

// dynamic shared memory a kernel gets without opting in, with room for its
// static shared memory inside the 48 KB default
constexpr size_t kDefaultDynSmem = 40 * 1024;

// fine-level launches: one block per kFineBlock / 32 slices, the slices staged
// in dynamic shared memory (column indices, then values)
inline int fine_blocks(int r0, int r1) {
    return (int)(((int64_t)r1 - (r0 & ~31) + kFineBlock - 1) / kFineBlock);
}
inline int64_t fine_nslices(const DevLevel& L) { return ((int64_t)L.n + 31) / 32; }
inline size_t fine_smem(const DevLevel& L, size_t value_bytes) { return (size_t)stage_bytes(L, value_bytes); }

// Launches records of one body as one grid (at most kMaxVBatch records).
template <typename Body>
void vbatch_launch(const VRec* const* recs, int n, cudaStream_t s) {
    VBatch p;
    p.nrec = n;
    p.bstart[0] = 0;
    size_t smem = 0;
    int carve = recs[0]->carve;
    for (int k = 0; k < n; ++k) {
        p.grid[k] = recs[k]->grid;
        p.a[k] = recs[k]->a;
        p.bstart[k + 1] = p.bstart[k] + recs[k]->grid;
        smem = std::max(smem, recs[k]->smem);
        if (recs[k]->carve != carve) carve = -1;
    }
    // the 48 KB default covers static and dynamic shared memory together
    if (smem > kDefaultDynSmem) raise_dyn_smem(k_batched<Body>, smem);
    launch_kernel_carve(k_batched<Body>, p.bstart[n], recs[0]->block, smem, carve, s, p);
}

thread_local std::vector<VRec>* t_vrecord = nullptr;
thread_local VKey t_vkey;

// One V-cycle launch of `Body`: issued as its own kernel, or, while a V-cycle
// is being recorded, appended to the record list at the current key.
template <typename Body>
void vlaunch(int grid, int block, size_t smem, cudaStream_t s, const VArgs& a, int carve = -1) {
    if (grid <= 0) return;
    if (t_vrecord) {
        VRec r;
        r.launch = &vbatch_launch<Body>;
        r.grid = grid;
        r.block = block;
        r.smem = smem;
        r.carve = carve;
        r.phase = t_vkey.phase;
        r.level = t_vkey.level;
        r.step = t_vkey.step++;
        r.a = a;
        t_vrecord->push_back(r);
        return;
    }
    if (smem > kDefaultDynSmem) raise_dyn_smem(k_single<Body>, smem);
    launch_kernel_carve(k_single<Body>, grid, block, smem, carve, s, a);
}

// arguments shared by the row kernels of a level
template <typename T>
VArgs level_args(const DevLevel& L, const LevelArrays<T>& A) {
    VArgs a;
    a.n = L.n;
    a.sw = L.sw;
    a.width = L.width;
    a.nslices = fine_nslices(L);
    a.cap = L.stage_cap;
    a.rlen = L.rlen;
    a.scol = L.scol;
    a.sval = A.sval;
    a.err = L.err;
    return a;
}

// the staged kernels read the compact layout where the level has one
template <typename T>
void use_compact(const DevLevel& L, const LevelArrays<T>& A, VArgs& a) {
    if (!L.soff) return;
    a.soff = L.soff;
    a.scol = L.ccol;
    a.sval = A.cval;
}

// r_in / isq (fine level only): form b = r * isq in the first pass (the
// float32 V-cycle's entry); b is then written, not read
template <typename T>
void first_impl(const DevLevel& L, const T* b, T* x, T* bc_zero, int nc, cudaStream_t s,
                const double* r_in = nullptr, const double* isq = nullptr) {
    const LevelArrays<T> A(L);
    const int c1 = L.cptr[1], c2 = L.cptr[std::min(2, L.ncolours)];
    if (L.lpr == kFine) {
        const int nb = r_in ? L.n : c1;
        VArgs f;
        f.r1 = c1;
        f.n = nb;
        f.nc = nc;
        f.dv = A.dinv;
        f.b = b;
        f.x = x;
        f.out = bc_zero;
        f.rin = r_in;
        f.isq = isq;
        vlaunch<FineFirst0Body<T>>(std::max(1, blocks_for(std::max(nb, nc))), kBlock, 0, s, f);
        if (c2 > c1) {
            VArgs a = level_args<T>(L, A);
            a.r0 = c1;
            a.r1 = c2;
            a.jmax = c1;
            a.dv = A.dinv;
            a.b = b;
            a.x = x;
            use_compact(L, A, a);
            vlaunch<FinePassBody<T>>(fine_blocks(c1, c2), kFineBlock, fine_smem(L, sizeof(T)), s, a,
                                     L.carve);
        }
        return;
    }
    if (r_in) throw Error{AMG_EINVAL, "the fused float32 entry needs the fine-level kernels"};
    VArgs a = level_args<T>(L, A);
    a.r1 = c2;
    a.jmax = c1;
    a.dv = A.dinv;
    a.b = b;
    a.x = x;
    AMG_LPR_DISPATCH(launch_lpr(L, c2),
                     (vlaunch<FirstBody<LPR, T>>(std::max(1, row_blocks(0, c2, LPR, L.block)), L.block,
                                                 0, s, a)));
}

// z_out / isq (fine level only): also write z = x * isq in float64 for the
// rows of this pass (the float32 V-cycle's exit)
template <typename T>
void pass_impl(const DevLevel& L, int col, int jmax, const T* b, T* x, cudaStream_t s,
               double* z_out = nullptr, const double* isq = nullptr) {
    const LevelArrays<T> A(L);
    const int r0 = L.cptr[col], r1 = L.cptr[col + 1];
    if (r1 <= r0) return;
    VArgs a = level_args<T>(L, A);
    a.r0 = r0;
    a.r1 = r1;
    a.jmax = jmax;
    a.dv = A.dinv;
    a.b = b;
    a.x = x;
    if (L.lpr == kFine) {
        a.z = z_out;
        a.isq = isq;
        use_compact(L, A, a);
        vlaunch<FinePassBody<T>>(fine_blocks(r0, r1), kFineBlock, fine_smem(L, sizeof(T)), s, a,
                                 L.carve);
        return;
    }
    if (z_out) throw Error{AMG_EINVAL, "the fused float32 exit needs the fine-level kernels"};
    AMG_LPR_DISPATCH(launch_lpr(L, r1 - r0),
                     (vlaunch<PassBody<LPR, T>>(row_blocks(r0, r1, LPR, L.block), L.block, 0, s, a)));
}

template <typename T>
void residual_restrict_impl(const DevLevel& L, const T* b, const T* x, T* r, T* bc,
                            cudaStream_t s) {
    const LevelArrays<T> A(L);
    const int c1 = L.cptr[1];
    constexpr bool SC = std::is_same<T, float>::value;
    VArgs a = level_args<T>(L, A);
    a.r0 = c1;
    a.r1 = L.n;
    a.dv = A.diag;
    a.b = b;
    a.x = const_cast<T*>(x);
    if (L.fused_restrict) {
        if (L.n > c1) {
            a.idx = L.agg;
            a.t = A.t;
            a.out = bc;
            use_compact(L, A, a);
            vlaunch<FineResRestrictBody<T, SC>>(fine_blocks(c1, L.n), kFineBlock,
                                                fine_smem(L, sizeof(T)), s, a, L.carve);
        }
        return;
    }
    if (L.n > c1) {
        a.out = r;
        if (L.lpr == kFine) {
            use_compact(L, A, a);
            vlaunch<FineResidualBody<T>>(fine_blocks(c1, L.n), kFineBlock, fine_smem(L, sizeof(T)), s, a,
                                         L.carve);
        } else {
            AMG_LPR_DISPATCH(launch_lpr(L, L.n - c1),
                             (vlaunch<ResidualBody<LPR, T>>(row_blocks(c1, L.n, LPR, L.block), L.block,
                                                            0, s, a)));
        }
    }
    VArgs q;
    q.n = L.n;
    q.err = L.err;
    q.nc = L.n_coarse;
    q.idx = L.rptr;
    q.idx2 = L.ridx;
    q.t = A.t;
    q.b = r;
    q.out = bc;
    vlaunch<RestrictBody<T, SC>>(blocks_for(L.n_coarse), kBlock, 0, s, q);
}

template <typename T>
void prolong_impl(const DevLevel& L, const T* e, T* x, double omega, cudaStream_t s) {
    const LevelArrays<T> A(L);
    const int r0 = L.cptr[1];
    if (L.n <= r0) return;
    constexpr bool SC = std::is_same<T, float>::value;
    VArgs a;
    a.r0 = r0;
    a.r1 = L.n;
    a.nc = L.n_coarse;
    a.err = L.err;
    a.idx = L.agg;
    a.t = A.t;
    a.b = e;
    a.x = x;
    a.omega = (double)(T)omega;
    vlaunch<ProlongBody<T, SC>>(blocks_for(L.n - r0), kBlock, 0, s, a);
}

template <int LPR, typename T>
void sweep_launch(const DevLevel& L, const SweepPlan& P, const T* sval, const T* dinv, const T* b,
                  T* x, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P.grid);
    cfg.blockDim = dim3((unsigned)L.block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        cudaLaunchKernelEx(&cfg, k_sweep<LPR, T>, P.npass, (const SweepPass*)P.pass, P.items,
                           (const int32_t*)P.dep_ptr, (const int32_t*)P.dep, P.flag, P.done,
                           P.arrive, P.failed, L.sw, (const uint16_t*)L.rlen,
                           (const int32_t*)L.scol, sval, dinv, b, x, L.err, L.n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{AMG_ECUDA, std::string("sweep launch (grid ") + std::to_string(P.grid) +
                                   ") failed: " + cudaGetErrorString(e)};
    }
}

template <typename T>
void sweep_impl(const DevLevel& L, const SweepPlan& P, const T* b, T* x, cudaStream_t s) {
    const LevelArrays<T> A(L);
    if (P.items <= 0) return;
    if (L.lpr < 1 || P.rows * L.lpr != L.block || P.npass > kSweepMaxPasses || P.grid < 1)
        throw Error{AMG_EINVAL, "sweep plan does not match the level's launch shape"};
    AMG_LPR_DISPATCH(L.lpr, (sweep_launch<LPR, T>(L, P, A.sval, A.dinv, b, x, s)));
}

template <int LPR>
int sweep_blocks_per_sm(int block) {
    int a = 0, b = 0;
    AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_sweep<LPR, double>, block, 0));
    AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep<LPR, float>, block, 0));
    return std::min(a, b);
}

// co-resident blocks of the sweep kernel with `lanes` lanes per row and
// `block` threads, in both precisions: the grid of its cooperative launch
int sweep_grid(int lanes, int block) {
    int dev = 0, sms = 0, per_sm = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AMG_LPR_DISPATCH(lanes, (per_sm = sweep_blocks_per_sm<LPR>(block)));
    return std::max(1, per_sm) * sms;
}

void launch_sweep(const DevLevel& L, const SweepPlan& P, const double* b, double* x, cudaStream_t s) {
    sweep_impl<double>(L, P, b, x, s);
}
void launch_sweep32(const DevLevel& L, const SweepPlan& P, const float* b, float* x, cudaStream_t s) {
    sweep_impl<float>(L, P, b, x, s);
}

void launch_first(const DevLevel& L, const double* b, double* x, double* bc_zero, int nc,
                  cudaStream_t s) {
    first_impl<double>(L, b, x, bc_zero, nc, s);
}
void launch_first32(const DevLevel& L, const float* b, float* x, float* bc_zero, int nc,
                    cudaStream_t s) {
    first_impl<float>(L, b, x, bc_zero, nc, s);
}
void launch_pass(const DevLevel& L, int col, int jmax, const double* b, double* x, cudaStream_t s) {
    pass_impl<double>(L, col, jmax, b, x, s);
}
void launch_pass32(const DevLevel& L, int col, int jmax, const float* b, float* x, cudaStream_t s) {
    pass_impl<float>(L, col, jmax, b, x, s);
}
void launch_first32_from64(const DevLevel& L, const double* r, const double* isq, float* b,
                           float* x, float* bc_zero, int nc, cudaStream_t s) {
    first_impl<float>(L, b, x, bc_zero, nc, s, r, isq);
}
void launch_pass32_to64(const DevLevel& L, int col, int jmax, const float* b, float* x,
                        double* z, const double* isq, cudaStream_t s) {
    pass_impl<float>(L, col, jmax, b, x, s, z, isq);
}
void launch_residual_restrict(const DevLevel& L, const double* b, const double* x, double* r,
                              double* bc, cudaStream_t s) {
    residual_restrict_impl<double>(L, b, x, r, bc, s);
}
void launch_residual_restrict32(const DevLevel& L, const float* b, const float* x, float* r,
                                float* bc, cudaStream_t s) {
    residual_restrict_impl<float>(L, b, x, r, bc, s);
}
void launch_prolong(const DevLevel& L, const double* e, double* x, double omega, cudaStream_t s) {
    prolong_impl<double>(L, e, x, omega, s);
}
void launch_prolong32(const DevLevel& L, const float* e, float* x, double omega, cudaStream_t s) {
    prolong_impl<float>(L, e, x, omega, s);
}

template <typename TB>
void dense_gemv_impl(int n, const double* M, const TB* b, TB* x, cudaStream_t s) {
    const size_t smem = std::is_same<TB, double>::value ? 0 : sizeof(double) * (size_t)n;
    VArgs a;
    a.n = n;
    a.dv = M;
    a.b = b;
    a.x = x;
    vlaunch<GemvBody<TB>>(blocks_for((int64_t)n * 32), kBlock, smem, s, a);
}

void launch_dense_gemv(int n, const double* M, const double* b, double* x, cudaStream_t s) {
    dense_gemv_impl<double>(n, M, b, x, s);
}

void launch_dense_gemv32(int n, const double* M, const float* b, float* x, cudaStream_t s) {
    dense_gemv_impl<float>(n, M, b, x, s);
}

void launch_vrecords(const VRec* const* recs, int n, cudaStream_t s) {
    for (int k0 = 0; k0 < n; k0 += kMaxVBatch) {
        const int m = std::min(kMaxVBatch, n - k0);
        recs[k0]->launch(recs + k0, m, s);
    }
}

void launch_cg_continue(cudaGraphConditionalHandle h, PcgScalars* sc, cudaStream_t s) {
    k_cg_continue<<<1, 1, 0, s>>>(h, sc);
    AMG_CUDA_TRY(cudaGetLastError());
}

void launch_dense_gemv_f32(int n, int ld, const float* M, const float* b, float* x, cudaStream_t s) {
    if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(M)) & 15 || ld % 4 || ld < n)
        throw Error{AMG_EINVAL, "float32 coarsest solve: operands must be 16-byte aligned"};
    VArgs a;
    a.n = n;
    a.ld = ld;
    a.dv = M;
    a.b = b;
    a.x = x;
    vlaunch<GemvF32Body>(blocks_for((int64_t)n * 32), kBlock, 0, s, a);
}

void launch_gather(int n, const int32_t* idx, const double* x, double* y, cudaStream_t s) {
    launch_kernel(k_gather, blocks_for(n), kBlock, 0, s, n, idx, x, y);
}

void launch_scatter(int n, const int32_t* idx, const double* x, double* y, cudaStream_t s) {
    launch_kernel(k_scatter, blocks_for(n), kBlock, 0, s, n, idx, x, y);
}

void launch_to_scaled32(int n, const double* r, const double* isq, float* rhat, cudaStream_t s) {
    VArgs a;
    a.n = n;
    a.rin = r;
    a.isq = isq;
    a.x = rhat;
    vlaunch<ToScaledBody>(blocks_for(n), kBlock, 0, s, a);
}

void launch_from_scaled32(int n, const float* zhat, const double* isq, double* z, cudaStream_t s) {
    VArgs a;
    a.n = n;
    a.b = zhat;
    a.isq = isq;
    a.z = z;
    vlaunch<FromScaledBody>(blocks_for(n), kBlock, 0, s, a);
}

void launch_cg_residual(const DevLevel& L, const double* b, const double* x, double* r,
                        CgWork& w, int mode, double* out, cudaStream_t s) {
    launch_kernel(k_cg_residual, reduction_blocks(L.n), kBlock, 0, s, L.n, L.sw, L.rlen, L.scol, L.sval,
                                                           L.diag, b, x, r, w.partials,
                                                           w.counters, w.sc, out, mode);
}

void launch_cg_spmv_pq(const DevLevel& L, const double* p, double* q, CgWork& w, cudaStream_t s) {
    launch_kernel(k_cg_spmv_pq, reduction_blocks(L.n), kBlock, 0, s, L.n, L.sw, L.rlen, L.scol, L.sval,
                                                          L.diag, p, q, w.partials,
                                                          w.counters + 1, w.sc);
}

void wait_selftest(long long limit, cudaStream_t s, int32_t* status, double* elapsed_ms) {
    DevArena mem(s);
    int32_t* err = mem.alloc<int32_t>(1);
    AMG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    AMG_CUDA_TRY(cudaEventCreate(&e0));
    AMG_CUDA_TRY(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } guard{e0, e1};
    AMG_CUDA_TRY(cudaEventRecord(e0, s));
    k_wait_selftest<<<1, kBlock, 0, s>>>(err, limit);
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(cudaEventRecord(e1, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(status, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    AMG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *elapsed_ms = ms;
}

void launch_cg_update(int n, double* x, double* r, const double* p, const double* q, CgWork& w,
                      cudaStream_t s) {
    launch_kernel(k_cg_update, reduction_blocks(n), kBlock, 0, s, n, x, r, p, q, w.partials, w.counters + 2,
                                                       w.sc);
}

void launch_cg_rz(int n, const double* r, const double* z, const double* zold, double* p,
                  CgWork& w, int mode, cudaStream_t s) {
    launch_kernel(k_cg_rz, reduction_blocks(n), kBlock, 0, s, n, r, z, zold, p, w.partials, w.partials2,
                                                   w.counters + 3, w.sc, mode);
}

void launch_cg_p(int n, const double* z, double* p, double* zold, const CgWork& w,
                 cudaStream_t s) {
    launch_kernel(k_cg_p, reduction_blocks(n), kBlock, 0, s, n, z, p, zold, w.sc);
}

void launch_bi_start(const DevLevel& L, const double* b, const double* x, double* r, double* rt,
                     CgWork& wk, BiScalars* bs, cudaStream_t s) {
    launch_kernel(k_bi_start, reduction_blocks(L.n), kBlock, 0, s, L.n, L.sw, L.rlen, L.scol,
                  L.sval, L.diag, b, x, r, rt, wk.partials, wk.partials2, wk.counters + 4, bs);
}

void launch_bi_direction(int n, const double* r, const double* v, double* p, const BiScalars* bs,
                         cudaStream_t s) {
    launch_kernel(k_bi_direction, reduction_blocks(n), kBlock, 0, s, n, r, v, p, bs);
}

void launch_bi_spmv(const DevLevel& L, const double* x, double* y, const double* w, bool second,
                    CgWork& wk, BiScalars* bs, cudaStream_t s) {
    launch_kernel(k_bi_spmv, reduction_blocks(L.n), kBlock, 0, s, L.n, L.sw, L.rlen, L.scol,
                  L.sval, L.diag, x, y, w, wk.partials, wk.partials2, wk.counters + (second ? 6 : 5),
                  bs, second ? (int)kBiW : (int)kBiRtv);
}

void launch_bi_half(int n, const double* r, const double* v, double* sv, CgWork& wk,
                    BiScalars* bs, cudaStream_t s) {
    launch_kernel(k_bi_half, reduction_blocks(n), kBlock, 0, s, n, r, v, sv, wk.partials,
                  wk.partials2, wk.counters + 7, bs);
}

void launch_bi_update(int n, double* x, const double* y, const double* z, const double* sv,
                      const double* t, double* r, const double* rt, CgWork& wk, BiScalars* bs,
                      cudaStream_t s) {
    launch_kernel(k_bi_update, reduction_blocks(n), kBlock, 0, s, n, x, y, z, sv, t, r, rt,
                  wk.partials, wk.partials2, wk.counters + 8, bs);
}

void launch_bi_continue(cudaGraphConditionalHandle h, BiScalars* bs, cudaStream_t s) {
    k_bi_continue<<<1, 1, 0, s>>>(h, bs);
    AMG_CUDA_TRY(cudaGetLastError());
}

}  // namespace amg
