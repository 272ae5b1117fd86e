// Solve-phase kernels: multicolour Gauss-Seidel, residual, restriction,
// prolongation, dense coarsest solve, and the CG vector operations
// (Sec. 2 V-cycle; Sec. 3.2 smoother applied in a fixed multicolour order;
// Sec. 5 Krylov iteration).
//
// Layout: every level stores its rows in the smoothing order (colour blocks,
// then coarse aggregate, then original index), the off-diagonal part in the
// SELL-32 layout described in device.h and the diagonal separately.  Row
// kernels give one thread to a row: for each k the 32 threads of a warp read
// entry k of their 32 rows from 32 consecutive addresses, and the row sum is a
// chain of fused multiply-adds with no cross-lane reduction (GB300 executes
// float64 at 1/64 of the float32 rate, so the float64 path keeps the
// arithmetic at one FMA per stored entry).  All reductions are deterministic:
// per-block partial sums in a fixed grid, combined in a fixed order by the
// last block to finish.

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

// acc + sgn * sum_k A_row,k x_col(k) over the stored off-diagonal entries of a
// SELL-32 row (base = slice start + row mod 32)
template <bool NEG, typename T, typename X>
__device__ __forceinline__ T sell_row(int64_t base, int len, const int32_t* __restrict__ scol,
                                      const T* __restrict__ sval, const X* x, T acc) {
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
        const int64_t e = base + 32 * (int64_t)k;
        const T a = sval[e];
        acc = fmad(NEG ? -a : a, T(x[scol[e]]), acc);
    }
    return acc;
}

// Same sum split over the LPR lanes of a group (lane-strided entries, then a
// shuffle reduction); acc is added once.  Every lane returns the full sum.
template <int LPR, bool NEG, typename T, typename X>
__device__ __forceinline__ T sell_row_group(int64_t base, int len, int lane,
                                            const int32_t* __restrict__ scol,
                                            const T* __restrict__ sval, const X* x, T acc) {
    if (LPR == 1) return sell_row<NEG>(base, len, scol, sval, x, acc);
    T s = lane == 0 ? acc : T(0);
#pragma unroll 2
    for (int k = lane; k < len; k += LPR) {
        const int64_t e = base + 32 * (int64_t)k;
        const T a = sval[e];
        s = fmad(NEG ? -a : a, T(x[scol[e]]), s);
    }
    return group_sum<LPR>(s);
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

// ---------------------------------------------------------------------------
// V-cycle kernels
// ---------------------------------------------------------------------------

// One Gauss-Seidel update of rows [r0, r1) of one colour:
//   x_i = (b_i - sum_{j != i} A_ij x_j) / A_ii.
// Rows of one colour are not coupled, so they update in parallel.  LPR lanes
// share a row (LPR = 1 on the fine level, where float64 arithmetic is the
// scarce resource; 4 or 8 on the denser coarse levels, where the latency of
// the gathers dominates).  Threads start at the slice boundary below r0 so
// warps read whole slices.
template <int LPR, typename T>
__global__ void __launch_bounds__(kBlock) k_gs(int r0, int r1, const int64_t* __restrict__ sptr,
                                               const uint16_t* __restrict__ rlen,
                                               const int32_t* __restrict__ scol,
                                               const T* __restrict__ sval,
                                               const T* __restrict__ dinv,
                                               const T* __restrict__ b, T* x) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int row = (r0 & ~31) + (int)(t / LPR);
    const int lane = (int)(t % LPR);
    const bool valid = row >= r0 && row < r1;
    if (LPR == 1 && !valid) return;
    const int rr = valid ? row : r0;
    const int64_t base = sptr[rr >> 5] + (rr & 31);
    const T s = sell_row_group<LPR, true>(base, valid ? (int)rlen[rr] : 0, lane, scol, sval, x,
                                          valid ? b[rr] : T(0));
    if (valid && lane == 0) x[row] = s * dinv[row];
}

// First Gauss-Seidel pass from a zero initial guess: the rows of colour 0
// [0, c1) have only zero neighbours, so x_i = b_i / A_ii there, and every other
// row starts at 0 (no matrix entries are read).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_first(int c1, int n, const T* __restrict__ dinv,
                                                     const T* __restrict__ b, T* __restrict__ x) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    x[row] = row < c1 ? b[row] * dinv[row] : T(0);
}

// r = b - A x for rows [r0, n)
template <int LPR, typename T>
__global__ void __launch_bounds__(kBlock) k_residual(int r0, int n, const int64_t* __restrict__ sptr,
                                                     const uint16_t* __restrict__ rlen,
                                                     const int32_t* __restrict__ scol,
                                                     const T* __restrict__ sval,
                                                     const T* __restrict__ diag,
                                                     const T* __restrict__ b,
                                                     const T* __restrict__ x, T* __restrict__ r) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int row = (r0 & ~31) + (int)(t / LPR);
    const int lane = (int)(t % LPR);
    const bool valid = row >= r0 && row < n;
    if (LPR == 1 && !valid) return;
    const int rr = valid ? row : r0;
    const int64_t base = sptr[rr >> 5] + (rr & 31);
    const T s0 = valid ? fmad(-diag[rr], x[rr], b[rr]) : T(0);
    const T v = sell_row_group<LPR, true>(base, valid ? (int)rlen[rr] : 0, lane, scol, sval, x, s0);
    if (valid && lane == 0) r[row] = v;
}

// coarse right-hand side: bc_J = sum over the fine rows i of aggregate J of
// (t_i) r_i, summed in the stored order (Eq. prolongation: R = P^T).  The lists
// hold the rows of colour >= 1 only: the pre-smoother's last pass updates
// colour 0, whose residual is therefore zero.
template <typename T, bool SCALED>
__global__ void __launch_bounds__(kBlock) k_restrict(int nc, const int32_t* __restrict__ rptr,
                                                     const int32_t* __restrict__ ridx,
                                                     const T* __restrict__ t,
                                                     const T* __restrict__ r, T* __restrict__ bc) {
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nc) return;
    T s = T(0);
    for (int k = rptr[J]; k < rptr[J + 1]; ++k) {
        const int i = ridx[k];
        s = SCALED ? fmad(t[i], r[i], s) : s + r[i];
    }
    bc[J] = s;
}

// x_i += omega (t_i) e_{agg(i)}: piecewise-constant prolongation with the
// over-correction factor omega, on rows [r0, n).  The caller passes r0 = the
// first row of colour 1: the post-smoother's first pass recomputes colour 0
// without reading its old values.
template <typename T, bool SCALED>
__global__ void __launch_bounds__(kBlock) k_prolong(int r0, int n, const int32_t* __restrict__ agg,
                                                    const T* __restrict__ t,
                                                    const T* __restrict__ e, T* __restrict__ x,
                                                    T omega) {
    const int i = r0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const int a = agg[i];
    if (a < 0) return;
    const T c = SCALED ? omega * t[i] : omega;
    x[i] += c * e[a];
}

// x = M b, M dense row-major (coarsest-level solve with the inverse formed at
// setup); one warp per row, float64 arithmetic.
template <typename TB>
__global__ void __launch_bounds__(kBlock) k_dense_gemv(int n, const double* __restrict__ M,
                                                       const TB* __restrict__ b, TB* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (row >= n) return;
    const double* m = M + (size_t)row * n;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s += m[k] * (double)b[k];
    s = group_sum<32>(s);
    if (lane == 0) x[row] = (TB)s;
}

__global__ void k_gather(int n, const int32_t* __restrict__ idx, const double* __restrict__ x,
                         double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[idx[i]];
}

__global__ void k_scatter(int n, const int32_t* __restrict__ idx, const double* __restrict__ x,
                          double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[idx[i]] = x[i];
}

// float64 -> scaled float32 at V-cycle entry: rhat = r / s, s = sqrt(A_ii)
__global__ void k_to_scaled32(int n, const double* __restrict__ r, const double* __restrict__ isq,
                              float* __restrict__ rhat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rhat[i] = (float)(r[i] * isq[i]);
}

// scaled float32 -> float64 at V-cycle exit: z = zhat / s
__global__ void k_from_scaled32(int n, const float* __restrict__ zhat, const double* __restrict__ isq,
                                double* __restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = (double)zhat[i] * isq[i];
}

// ---------------------------------------------------------------------------
// CG kernels (level 0, float64, smoothing order)
// ---------------------------------------------------------------------------

// r = b - A x and ||r||^2 (grid-stride over rows)
__global__ void __launch_bounds__(kBlock) k_cg_residual(int n, const int64_t* __restrict__ sptr,
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
    double acc = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int64_t base = sptr[row >> 5] + (row & 31);
        const double s0 = fmad(-diag[row], x[row], b[row]);
        const double v = sell_row<true>(base, rlen[row], scol, sval, x, s0);
        if (r) r[row] = v;
        acc = fmad(v, v, acc);
    }
    const double t = block_sum(acc, sh);
    finish_reduction(t, 0.0, partials, nullptr, counter, sc, out, mode, sh);
}

// q = A p and p.q -> alpha
__global__ void __launch_bounds__(kBlock) k_cg_spmv_pq(int n, const int64_t* __restrict__ sptr,
                                                       const uint16_t* __restrict__ rlen,
                                                       const int32_t* __restrict__ scol,
                                                       const double* __restrict__ sval,
                                                       const double* __restrict__ diag,
                                                       const double* __restrict__ p,
                                                       double* __restrict__ q, double* partials,
                                                       unsigned int* counter, PcgScalars* sc) {
    __shared__ double sh[kBlock / 32];
    double acc = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int64_t base = sptr[row >> 5] + (row & 31);
        const double pi = p[row];
        const double v = sell_row<false>(base, rlen[row], scol, sval, p, diag[row] * pi);
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
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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
    const double beta = sc->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double zi = z[i];
        p[i] = zi + beta * p[i];
        if (zold) zold[i] = zi;
    }
}

inline int blocks_for(int64_t threads) { return (int)((threads + kBlock - 1) / kBlock); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int g_reduction_blocks = 1216;

int reduction_blocks(int64_t work_threads) {
    int64_t b = (work_threads + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, g_reduction_blocks);
}

inline int row_blocks(int r0, int r1, int lpr) { return blocks_for((int64_t)(r1 - (r0 & ~31)) * lpr); }

#define AMG_LPR_DISPATCH(lpr, CALL)                          \
    switch (lpr) {                                           \
        case 1: { constexpr int LPR = 1; CALL; } break;      \
        case 4: { constexpr int LPR = 4; CALL; } break;      \
        default: { constexpr int LPR = 8; CALL; } break;     \
    }

void launch_gs(const DevLevel& L, int r0, int r1, const double* b, double* x, cudaStream_t s) {
    if (r1 <= r0) return;
    AMG_LPR_DISPATCH(L.lpr, (k_gs<LPR, double><<<row_blocks(r0, r1, LPR), kBlock, 0, s>>>(
                                r0, r1, L.sptr, L.rlen, L.scol, L.sval, L.dinv, b, x)));
}

void launch_gs32(const DevLevel& L, int r0, int r1, const float* b, float* x, cudaStream_t s) {
    if (r1 <= r0) return;
    AMG_LPR_DISPATCH(L.lpr, (k_gs<LPR, float><<<row_blocks(r0, r1, LPR), kBlock, 0, s>>>(
                                r0, r1, L.sptr, L.rlen, L.scol, L.sval32, L.dinv32, b, x)));
}

void launch_residual(const DevLevel& L, int r0, const double* b, const double* x, double* r,
                     cudaStream_t s) {
    if (L.n <= r0) return;
    AMG_LPR_DISPATCH(L.lpr, (k_residual<LPR, double><<<row_blocks(r0, L.n, LPR), kBlock, 0, s>>>(
                                r0, L.n, L.sptr, L.rlen, L.scol, L.sval, L.diag, b, x, r)));
}

void launch_residual32(const DevLevel& L, int r0, const float* b, const float* x, float* r,
                       cudaStream_t s) {
    if (L.n <= r0) return;
    AMG_LPR_DISPATCH(L.lpr, (k_residual<LPR, float><<<row_blocks(r0, L.n, LPR), kBlock, 0, s>>>(
                                r0, L.n, L.sptr, L.rlen, L.scol, L.sval32, L.diag32, b, x, r)));
}

void launch_restrict(const DevLevel& L, const double* r, double* bc, cudaStream_t s) {
    k_restrict<double, false><<<blocks_for(L.n_coarse), kBlock, 0, s>>>(L.n_coarse, L.rptr, L.ridx,
                                                                        nullptr, r, bc);
}

void launch_restrict32(const DevLevel& L, const float* r, float* bc, cudaStream_t s) {
    k_restrict<float, true><<<blocks_for(L.n_coarse), kBlock, 0, s>>>(L.n_coarse, L.rptr, L.ridx,
                                                                      L.t32, r, bc);
}

void launch_prolong(const DevLevel& L, const double* e, double* x, double omega, cudaStream_t s) {
    const int r0 = L.cptr[1];
    if (L.n <= r0) return;
    k_prolong<double, false><<<blocks_for(L.n - r0), kBlock, 0, s>>>(r0, L.n, L.agg, nullptr, e, x,
                                                                     omega);
}

void launch_prolong32(const DevLevel& L, const float* e, float* x, float omega, cudaStream_t s) {
    const int r0 = L.cptr[1];
    if (L.n <= r0) return;
    k_prolong<float, true><<<blocks_for(L.n - r0), kBlock, 0, s>>>(r0, L.n, L.agg, L.t32, e, x,
                                                                   omega);
}

void launch_gs_first(const DevLevel& L, const double* b, double* x, cudaStream_t s) {
    k_gs_first<double><<<blocks_for(L.n), kBlock, 0, s>>>(L.cptr[1], L.n, L.dinv, b, x);
}

void launch_gs_first32(const DevLevel& L, const float* b, float* x, cudaStream_t s) {
    k_gs_first<float><<<blocks_for(L.n), kBlock, 0, s>>>(L.cptr[1], L.n, L.dinv32, b, x);
}

void launch_dense_gemv(int n, const double* M, const double* b, double* x, cudaStream_t s) {
    k_dense_gemv<double><<<blocks_for((int64_t)n * 32), kBlock, 0, s>>>(n, M, b, x);
}

void launch_dense_gemv32(int n, const double* M, const float* b, float* x, cudaStream_t s) {
    k_dense_gemv<float><<<blocks_for((int64_t)n * 32), kBlock, 0, s>>>(n, M, b, x);
}

void launch_gather(int n, const int32_t* idx, const double* x, double* y, cudaStream_t s) {
    k_gather<<<blocks_for(n), kBlock, 0, s>>>(n, idx, x, y);
}

void launch_scatter(int n, const int32_t* idx, const double* x, double* y, cudaStream_t s) {
    k_scatter<<<blocks_for(n), kBlock, 0, s>>>(n, idx, x, y);
}

void launch_to_scaled32(int n, const double* r, const double* isq, float* rhat, cudaStream_t s) {
    k_to_scaled32<<<blocks_for(n), kBlock, 0, s>>>(n, r, isq, rhat);
}

void launch_from_scaled32(int n, const float* zhat, const double* isq, double* z, cudaStream_t s) {
    k_from_scaled32<<<blocks_for(n), kBlock, 0, s>>>(n, zhat, isq, z);
}

void launch_cg_residual(const DevLevel& L, const double* b, const double* x, double* r,
                        CgWork& w, int mode, double* out, cudaStream_t s) {
    k_cg_residual<<<reduction_blocks(L.n), kBlock, 0, s>>>(L.n, L.sptr, L.rlen, L.scol, L.sval,
                                                           L.diag, b, x, r, w.partials,
                                                           w.counters, w.sc, out, mode);
}

void launch_cg_spmv_pq(const DevLevel& L, const double* p, double* q, CgWork& w, cudaStream_t s) {
    k_cg_spmv_pq<<<reduction_blocks(L.n), kBlock, 0, s>>>(L.n, L.sptr, L.rlen, L.scol, L.sval,
                                                          L.diag, p, q, w.partials,
                                                          w.counters + 1, w.sc);
}

void launch_cg_update(int n, double* x, double* r, const double* p, const double* q, CgWork& w,
                      cudaStream_t s) {
    k_cg_update<<<reduction_blocks(n), kBlock, 0, s>>>(n, x, r, p, q, w.partials, w.counters + 2,
                                                       w.sc);
}

void launch_cg_rz(int n, const double* r, const double* z, const double* zold, double* p,
                  CgWork& w, int mode, cudaStream_t s) {
    k_cg_rz<<<reduction_blocks(n), kBlock, 0, s>>>(n, r, z, zold, p, w.partials, w.partials2,
                                                   w.counters + 3, w.sc, mode);
}

void launch_cg_p(int n, const double* z, double* p, double* zold, const CgWork& w,
                 cudaStream_t s) {
    k_cg_p<<<reduction_blocks(n), kBlock, 0, s>>>(n, z, p, zold, w.sc);
}

}  // namespace amg
