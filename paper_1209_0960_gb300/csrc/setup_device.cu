// Device part of the hierarchy setup: Galerkin coarse operator, reordering of
// each level into its smoothing order, dense inverse of the coarsest matrix
// and the scaled float32 level copies.

#include <algorithm>
#include <numeric>

#include "device.h"

namespace amg {

namespace {

inline int blocks_for(int64_t threads, int block = kBlock) {
    return (int)((threads + block - 1) / block);
}

// ---------------------------------------------------------------------------
// Galerkin product G = P^T A P (Eq. prolongation and the coarse operator that
// follows it).  One warp builds coarse row I: it stages the (J = agg(j), A_ij)
// pairs of the rows i of aggregate I -- members in ascending order, entries
// in row order -- in shared memory, marks the first occurrence of each J,
// and for each distinct J sums its entries left to right in that staged
// order, which is the fine CSR order.  The result is therefore independent
// of the launch configuration and bit-identical to a sequential sum.
// Pass 1 (FILL = false) counts the distinct J of every row; pass 2 writes
// the sorted columns and the sums at the row offsets.
// ---------------------------------------------------------------------------
template <bool FILL>
__global__ void k_galerkin(int nc, const int32_t* __restrict__ mptr, const int32_t* __restrict__ mem,
                           const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ va, const int32_t* __restrict__ agg, int cap,
                           int32_t* __restrict__ cnt, const int32_t* __restrict__ grp,
                           int32_t* __restrict__ gci, double* __restrict__ gva) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* sV = reinterpret_cast<double*>(smem) + (size_t)warp * cap;
    int32_t* sJ = reinterpret_cast<int32_t*>(reinterpret_cast<double*>(smem) + (size_t)wpb * cap) +
                  (size_t)warp * cap;
    uint8_t* sF = reinterpret_cast<uint8_t*>(reinterpret_cast<int32_t*>(
                      reinterpret_cast<double*>(smem) + (size_t)wpb * cap) + (size_t)wpb * cap) +
                  (size_t)warp * cap;
    const int I = blockIdx.x * wpb + warp;
    if (I >= nc) return;
    int m = 0;
    for (int t = mptr[I]; t < mptr[I + 1]; ++t) {
        const int i = mem[t];
        const int k0 = rp[i], len = rp[i + 1] - k0;
        for (int q = lane; q < len; q += 32) {
            sJ[m + q] = agg[ci[k0 + q]];
            if (FILL) sV[m + q] = va[k0 + q];
        }
        m += len;
    }
    __syncwarp();
    for (int e = lane; e < m; e += 32) {
        const int J = sJ[e];
        bool first = J >= 0;
        for (int f = 0; f < e && first; ++f)
            if (sJ[f] == J) first = false;
        sF[e] = first ? 1 : 0;
    }
    __syncwarp();
    if (!FILL) {
        int c = 0;
        for (int e = lane; e < m; e += 32) c += sF[e];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        if (lane == 0) cnt[I] = c;
        return;
    }
    const int base = grp[I];
    for (int e = lane; e < m; e += 32) {
        if (!sF[e]) continue;
        const int J = sJ[e];
        int rank = 0;
        for (int f = 0; f < m; ++f) rank += (sF[f] && sJ[f] < J) ? 1 : 0;
        double s = sV[e];
        for (int f = e + 1; f < m; ++f)
            if (sJ[f] == J) s = s + sV[f];
        gci[base + rank] = J;
        gva[base + rank] = s;
    }
}

// Copy row inv[r] of A into row r of the smoothing-order level: off-diagonal
// entries (in their stored order, columns renumbered by perm) and diagonal.
__global__ void k_reorder_rows(int n, const int32_t* __restrict__ inv, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ va, const int32_t* __restrict__ nrp,
                               int32_t* __restrict__ nci, double* __restrict__ nva,
                               double* __restrict__ diag, double* __restrict__ dinv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int i = inv[r];
    int out = nrp[r];
    double d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        if (j == i) {
            d = va[k];
        } else {
            nci[out] = perm[j];
            nva[out] = va[k];
            ++out;
        }
    }
    diag[r] = d;
    dinv[r] = 1.0 / d;
}

// Scatter the off-diagonal CSR rows into the SELL-32 arrays; padding entries
// point at the row itself with value 0.
__global__ void k_csr_to_sell(int n, const int32_t* __restrict__ nrp, const int32_t* __restrict__ nci,
                              const double* __restrict__ nva, int width,
                              int32_t* __restrict__ scol, double* __restrict__ sval) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t base = (int64_t)(r >> 5) * 32 * width + (r & 31);
    const int k0 = nrp[r], len = nrp[r + 1] - k0;
    for (int k = 0; k < width; ++k) {
        const int64_t e = base + 32 * (int64_t)k;
        if (k < len) {
            scol[e] = nci[k0 + k];
            sval[e] = nva[k0 + k];
        } else {
            scol[e] = r;
            sval[e] = 0.0;
        }
    }
}

// Copy the sliced arrays (common width W) into the layout with per-slice
// widths: slice s starts at soff[s] and keeps K_s = (soff[s+1] - soff[s]) / 32
// entries a row, entry k of lane i at soff[s] + 32 k + i (padding entries as
// in the common layout: the row itself with value 0).  One thread per row.
template <typename T>
__global__ void k_sell_own_width(int n, int width, const int64_t* __restrict__ soff,
                                 const int32_t* __restrict__ scol, const T* __restrict__ sval,
                                 int32_t* __restrict__ ccol, T* __restrict__ cval) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t src = (int64_t)(r >> 5) * 32 * width + (r & 31);
    const int64_t dst = soff[r >> 5] + (r & 31);
    const int ks = (int)((soff[(r >> 5) + 1] - soff[r >> 5]) >> 5);
    for (int k = 0; k < ks; ++k) {
        if (ccol) ccol[dst + 32 * (int64_t)k] = scol[src + 32 * (int64_t)k];
        cval[dst + 32 * (int64_t)k] = sval[src + 32 * (int64_t)k];
    }
}

// ---------------------------------------------------------------------------
// coarsest level: dense Cholesky factor (lower triangle, row-major, in place)
// and the inverse through two triangular solves per unit vector
// ---------------------------------------------------------------------------
__global__ void k_dense_from_csr(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ va, double* __restrict__ M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k) M[(size_t)i * n + ci[k]] = va[k];
}

// ---------------------------------------------------------------------------
// Dense inverse of the coarsest matrix M (n x n, row-major), float64:
// blocked Cholesky M = L L^T in 32-column panels, then Y = L^-1 by blocked
// forward substitution and M^-1 = Y^T Y.  Work is n^3/6 fused multiply-adds
// per phase, almost all of it in 64 x 64 (or 32 x 32) output tiles staged in
// shared memory.  Only the lower triangle of the working matrix W is read.
// ---------------------------------------------------------------------------
constexpr int kPanel = 32;

// Factor the diagonal block W[k0.., k0..] (m <= 32 rows) in shared memory,
// one thread per entry (32 x 32 threads); write L_kk back (upper part zero)
// and D = L_kk^-1 to Dk (32 x 32, row-major).  A pivot <= 0 sets *err and
// continues with 1.
__global__ void __launch_bounds__(kPanel * kPanel) k_potrf_block(int n, int k0, double* __restrict__ W,
                                                                 double* __restrict__ Dk,
                                                                 int* __restrict__ err) {
    __shared__ double T[kPanel][kPanel + 1];
    __shared__ double Y[kPanel][kPanel + 1];
    const int r = threadIdx.x / kPanel, c = threadIdx.x % kPanel;
    const int m = min(kPanel, n - k0);
    T[r][c] = (r < m && c <= r) ? W[(size_t)(k0 + r) * n + k0 + c] : 0.0;
    Y[r][c] = (r == c && r < m) ? 1.0 : 0.0;
    __syncthreads();
    // right-looking Cholesky: column j, then the rank-1 update of the rest
    for (int j = 0; j < m; ++j) {
        if (r == j && c == j) {
            double d = T[j][j];
            if (!(d > 0.0)) {
                *err = 1;
                d = 1.0;
            }
            T[j][j] = sqrt(d);
        }
        __syncthreads();
        if (c == j && r > j && r < m) T[r][j] /= T[j][j];
        __syncthreads();
        if (r > j && r < m && c > j && c <= r) T[r][c] -= T[r][j] * T[c][j];
        __syncthreads();
    }
    // D = L_kk^-1 by forward elimination on the identity, row j at a time
    for (int j = 0; j < m; ++j) {
        if (r == j && c <= j) Y[j][c] /= T[j][j];
        __syncthreads();
        if (r > j && r < m && c <= j) Y[r][c] -= T[r][j] * Y[j][c];
        __syncthreads();
    }
    if (r < m && c < m) W[(size_t)(k0 + r) * n + k0 + c] = T[r][c];
    Dk[r * kPanel + c] = Y[r][c];
}

// Panel below the diagonal block: W[i, k0:k0+m] <- W[i, k0:k0+m] D^T for
// i >= k0 + m (solves x L_kk^T = a), one warp per row, lane = column.
__global__ void __launch_bounds__(kBlock) k_panel(int n, int k0, int m, double* __restrict__ W,
                                                  const double* __restrict__ Dk) {
    __shared__ double D[kPanel][kPanel + 1];
    const int lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < kPanel * kPanel; t += blockDim.x)
        D[t / kPanel][t % kPanel] = Dk[t];
    __syncthreads();
    const int i = k0 + m + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= n) return;
    double* row = W + (size_t)i * n + k0;
    const double a = lane < m ? row[lane] : 0.0;
    double out = 0.0;
    for (int t = 0; t < m; ++t) {
        const double at = __shfl_sync(0xffffffffu, a, t);
        if (t <= lane) out = fma(at, D[lane][t], out);
    }
    if (lane < m) row[lane] = out;
}

// Tile index of the lower-triangle tile pair number b: (I, J), I >= J.
__device__ __forceinline__ void tri_pair(int b, int& I, int& J) {
    I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= b) ++I;
    while (I * (I + 1) / 2 > b) --I;
    J = b - I * (I + 1) / 2;
}

// Trailing update W[i][j] -= sum_t P[i][t] P[j][t] over the lower tiles of
// rows/columns >= r0 (P = the panel W[:, k0:k0+m]); 64 x 64 tiles, 256
// threads, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) k_syrk(int n, int r0, int k0, int m, double* __restrict__ W) {
    __shared__ double Pa[64][kPanel + 1];
    __shared__ double Pb[64][kPanel + 1];
    int I, J;
    tri_pair((int)blockIdx.x, I, J);
    const int i0 = r0 + 64 * I, j0 = r0 + 64 * J;
    for (int t = threadIdx.x; t < 64 * kPanel; t += blockDim.x) {
        const int r = t / kPanel, q = t % kPanel;
        Pa[r][q] = (i0 + r < n && q < m) ? W[(size_t)(i0 + r) * n + k0 + q] : 0.0;
        Pb[r][q] = (j0 + r < n && q < m) ? W[(size_t)(j0 + r) * n + k0 + q] : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double acc[4][4] = {};
    for (int q = 0; q < m; ++q) {
        double av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            av[u] = Pa[ty * 4 + u][q];
            bv[u] = Pb[tx * 4 + u][q];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
            if (i < n && j < n && j <= i) W[(size_t)i * n + j] -= acc[u][v];
        }
}

// Y = L^-1, right-looking by 32-row block rows.  Row block j of Y holds
// the running sums S_jc = sum_{c <= t < i} L_jt Y_tc until its turn; then
// Y_jc = -D_j S_jc for c < j and Y_jj = D_j.
//
// Finalise block row i0 (m rows): column tile c = blockIdx.x (c0 <= i0).
// 32 x 32 threads, one output each.
__global__ void __launch_bounds__(kPanel * kPanel) k_trinv_final(int n, int i0, int m,
                                                                 double* __restrict__ Y,
                                                                 const double* __restrict__ Di) {
    __shared__ double D[kPanel][kPanel + 1];
    __shared__ double S[kPanel][kPanel + 1];
    const int r = threadIdx.x / kPanel, c = threadIdx.x % kPanel;
    const int c0 = kPanel * (int)blockIdx.x;
    D[r][c] = Di[r * kPanel + c];
    if (c0 == i0) {
        if (r < m && c0 + c < n) Y[(size_t)(i0 + r) * n + c0 + c] = D[r][c];
        return;
    }
    S[r][c] = (r < m) ? Y[(size_t)(i0 + r) * n + c0 + c] : 0.0;
    __syncthreads();
    if (r >= m) return;
    double out = 0.0;
    for (int q = 0; q <= r; ++q) out = fma(D[r][q], S[q][c], out);
    Y[(size_t)(i0 + r) * n + c0 + c] = -out;
}

// Update after block row i0 is final: S_jc += L_j,i Y_i,c for the block rows
// j > i0 and column tiles c <= i0, 64 x 64 output tiles of (rows >= i0 + m,
// columns < i0 + m), K = m; 256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) k_trinv_update(int n, int i0, int m, const double* __restrict__ L,
                                                      double* __restrict__ Y) {
    __shared__ double Pa[64][kPanel + 1];   // L[j rows, i0 .. i0+m)
    __shared__ double Pb[kPanel][64 + 1];   // Y[i0 .. i0+m, c columns]
    const int r0 = i0 + m, ncol = i0 + m;
    const int tiles_c = (ncol + 63) / 64;
    const int J = (int)blockIdx.x / tiles_c, C = (int)blockIdx.x % tiles_c;
    const int j0 = r0 + 64 * J, c0 = 64 * C;
    for (int t = threadIdx.x; t < 64 * kPanel; t += blockDim.x) {
        const int rr = t / kPanel, q = t % kPanel;
        Pa[rr][q] = (j0 + rr < n && q < m) ? L[(size_t)(j0 + rr) * n + i0 + q] : 0.0;
        const int qq = t / 64, cc = t % 64;
        Pb[qq][cc] = (qq < m && c0 + cc < ncol) ? Y[(size_t)(i0 + qq) * n + c0 + cc] : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double acc[4][4] = {};
    for (int q = 0; q < m; ++q) {
        double av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            av[u] = Pa[ty * 4 + u][q];
            bv[u] = Pb[q][tx * 4 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = j0 + ty * 4 + u, cc = c0 + tx * 4 + v;
            if (j < n && cc < ncol) Y[(size_t)j * n + cc] += acc[u][v];
        }
}

// X = Y^T Y for the lower tiles (I >= J) of 64 x 64, mirrored to the upper
// part: X[i][j] = sum_{k >= 64 I} Y[k][i] Y[k][j] (Y is lower triangular).
__global__ void __launch_bounds__(256) k_yty(int n, const double* __restrict__ Y, double* __restrict__ X) {
    __shared__ double Ya[kPanel][64 + 1];
    __shared__ double Yb[kPanel][64 + 1];
    int I, J;
    tri_pair((int)blockIdx.x, I, J);
    const int i0 = 64 * I, j0 = 64 * J;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double acc[4][4] = {};
    for (int k0 = i0; k0 < n; k0 += kPanel) {
        for (int t = threadIdx.x; t < kPanel * 64; t += blockDim.x) {
            const int kk = t / 64, c = t % 64;
            const bool ok = k0 + kk < n;
            Ya[kk][c] = (ok && i0 + c < n) ? Y[(size_t)(k0 + kk) * n + i0 + c] : 0.0;
            Yb[kk][c] = (ok && j0 + c < n) ? Y[(size_t)(k0 + kk) * n + j0 + c] : 0.0;
        }
        __syncthreads();
        for (int q = 0; q < kPanel; ++q) {
            double av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                av[u] = Ya[q][ty * 4 + u];
                bv[u] = Yb[q][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
            if (i < n && j < n && j <= i) {
                X[(size_t)i * n + j] = acc[u][v];
                X[(size_t)j * n + i] = acc[u][v];
            }
        }
}

// Minv_s = S Minv S with S = diag(sqrt(A_ii)): the inverse of S^-1 A S^-1
__global__ void k_scale_inverse(int n, const double* __restrict__ diag, const double* __restrict__ X,
                                double* __restrict__ Xs) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    Xs[t] = sqrt(diag[i]) * X[t] * sqrt(diag[j]);
}

// float32 level: A^ = S^-1 A S^-1 (off-diagonal, diagonal and its inverse),
// and the transfer weights t_i = s_i / s_coarse(agg(i)).
__global__ void k_level_fp32(int n, int width, const int32_t* __restrict__ scol,
                             const double* __restrict__ sval, const double* __restrict__ diag,
                             const int32_t* __restrict__ agg, const double* __restrict__ cdiag,
                             float* __restrict__ sval32, float* __restrict__ diag32,
                             float* __restrict__ dinv32, float* __restrict__ t32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double si = sqrt(diag[i]);
    const int64_t base = (int64_t)(i >> 5) * 32 * width + (i & 31);
    for (int k = 0; k < width; ++k) {
        const int64_t e = base + 32 * (int64_t)k;
        sval32[e] = (float)(sval[e] / (si * sqrt(diag[scol[e]])));
    }
    const double dh = diag[i] / (si * si);
    diag32[i] = (float)dh;
    dinv32[i] = (float)(1.0 / dh);
    if (t32) {
        const int a = agg[i];
        t32[i] = a >= 0 ? (float)(si / sqrt(cdiag[a])) : 0.0f;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host-side drivers
// ---------------------------------------------------------------------------

void galerkin_device(const DevCsr& A, const HostCsr& Ah, const AggResult& R, DevArena& arena,
                     DevCsr& Gd, HostCsr& Gh, cudaStream_t s) {
    const int32_t n = Ah.n, nc = R.nc;
    // members of each aggregate in ascending order (counting sort)
    std::vector<int32_t> mptr(nc + 1, 0), mem;
    for (int32_t i = 0; i < n; ++i)
        if (R.agg[i] >= 0) ++mptr[R.agg[i] + 1];
    for (int32_t I = 0; I < nc; ++I) mptr[I + 1] += mptr[I];
    mem.resize(mptr[nc]);
    {
        std::vector<int32_t> fill(mptr.begin(), mptr.end() - 1);
        for (int32_t i = 0; i < n; ++i)
            if (R.agg[i] >= 0) mem[fill[R.agg[i]]++] = i;
    }
    // staging capacity: largest number of fine entries feeding one coarse row
    int64_t cap = 1;
    for (int32_t I = 0; I < nc; ++I) {
        int64_t m = 0;
        for (int32_t t = mptr[I]; t < mptr[I + 1]; ++t) m += Ah.rp[mem[t] + 1] - Ah.rp[mem[t]];
        cap = std::max(cap, m);
    }
    cap = (cap + 15) / 16 * 16;
    const size_t per_warp = (size_t)cap * (sizeof(double) + sizeof(int32_t) + 1);
    const size_t smem_limit = 200 * 1024;
    if (per_warp > smem_limit)
        throw Error{AMG_EINVAL, "Galerkin product: a coarse row gathers " + std::to_string(cap) +
                                    " fine entries, more than the shared-memory staging holds"};
    int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, smem_limit / per_warp));
    const size_t smem = per_warp * wpb;
    if (smem > 40 * 1024) {   // the 48 KB default also holds static shared memory
        raise_dyn_smem(k_galerkin<false>, smem);
        raise_dyn_smem(k_galerkin<true>, smem);
    }
    DevArena tmp(s);
    int32_t* d_agg = tmp.alloc<int32_t>(n);
    int32_t* d_mptr = tmp.alloc<int32_t>(nc + 1);
    int32_t* d_mem = tmp.alloc<int32_t>(mem.size());
    int32_t* d_cnt = tmp.alloc<int32_t>(nc);
    AMG_CUDA_TRY(cudaMemcpyAsync(d_agg, R.agg.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(d_mptr, mptr.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(d_mem, mem.data(), sizeof(int32_t) * mem.size(), cudaMemcpyHostToDevice, s));
    const int grid = (nc + wpb - 1) / wpb;
    k_galerkin<false><<<grid, 32 * wpb, smem, s>>>(nc, d_mptr, d_mem, A.rp, A.ci, A.va, d_agg, (int)cap,
                                                   d_cnt, nullptr, nullptr, nullptr);
    AMG_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> cnt(nc);
    AMG_CUDA_TRY(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    Gh.n = nc;
    Gh.rp.assign(nc + 1, 0);
    for (int32_t I = 0; I < nc; ++I) {
        if ((int64_t)Gh.rp[I] + cnt[I] >= INT32_MAX)
            throw Error{AMG_EINVAL, "coarse matrix exceeds int32 entries"};
        Gh.rp[I + 1] = Gh.rp[I] + cnt[I];
    }
    const int64_t gnnz = Gh.rp[nc];
    Gd.n = nc;
    Gd.nnz = gnnz;
    Gd.rp = arena.alloc<int32_t>(nc + 1);
    Gd.ci = arena.alloc<int32_t>(gnnz);
    Gd.va = arena.alloc<double>(gnnz);
    AMG_CUDA_TRY(cudaMemcpyAsync(Gd.rp, Gh.rp.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s));
    k_galerkin<true><<<grid, 32 * wpb, smem, s>>>(nc, d_mptr, d_mem, A.rp, A.ci, A.va, d_agg, (int)cap,
                                                  nullptr, Gd.rp, Gd.ci, Gd.va);
    AMG_CUDA_TRY(cudaGetLastError());
    Gh.ci.resize(gnnz);
    Gh.va.resize(gnnz);
    AMG_CUDA_TRY(cudaMemcpyAsync(Gh.ci.data(), Gd.ci, sizeof(int32_t) * gnnz, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(Gh.va.data(), Gd.va, sizeof(double) * gnnz, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
}

void build_level_device(const DevCsr& A, const HostCsr& Ah, const std::vector<int32_t>& perm,
                        DevArena& arena, DevLevel& L, cudaStream_t s) {
    const int32_t n = Ah.n;
    std::vector<int32_t> inv(n), nrp(n + 1, 0);
    std::vector<uint16_t> rlen(n);
    for (int32_t i = 0; i < n; ++i) inv[perm[i]] = i;
    for (int32_t r = 0; r < n; ++r) {
        const int32_t i = inv[r];
        const int32_t len = Ah.rp[i + 1] - Ah.rp[i] - 1;
        if (len > 65535) throw Error{AMG_EINVAL, "a matrix row has more than 65535 off-diagonal entries"};
        rlen[r] = (uint16_t)len;
        nrp[r + 1] = nrp[r] + len;
    }
    const int32_t nslices = (n + 31) / 32;
    int width = 0;
    for (int32_t r = 0; r < n; ++r) width = std::max<int>(width, rlen[r]);
    L.n = n;
    L.nnz_off = nrp[n];
    L.width = width;
    L.sw = 32 * (int64_t)width;
    L.padded = (int64_t)nslices * L.sw;
    // staged blocks cover 8 consecutive slices (256 rows) starting at any
    // slice (colours start anywhere): their tile bounds are maxima over every
    // window of 8 slices
    constexpr int kSlicesPerStage = 8;
    auto window_max = [&](const std::vector<int64_t>& per_slice) {
        int64_t run = 0, best = 0;
        for (int32_t sl = 0; sl < nslices; ++sl) {
            run += per_slice[sl];
            if (sl >= kSlicesPerStage) run -= per_slice[sl - kSlicesPerStage];
            best = std::max(best, run);
        }
        return best;
    };
    // per-slice widths: each slice padded only to its own longest row
    std::vector<int64_t> kmax(nslices, 0), soff(nslices + 1, 0);
    for (int32_t r = 0; r < n; ++r) kmax[r >> 5] = std::max<int64_t>(kmax[r >> 5], rlen[r]);
    for (int32_t sl = 0; sl < nslices; ++sl) soff[sl + 1] = soff[sl] + 32 * kmax[sl];
    // kept where the common width pads more than a tenth over that (the
    // coarse levels; the fine level's rows are nearly all W long)
    const bool compact = width > 0 && 10 * L.padded > 11 * soff[nslices];
    L.stage_cap = compact ? 32 * window_max(kmax) : 256 * (int64_t)width;
    L.rlen = arena.alloc<uint16_t>(n);
    L.scol = arena.alloc<int32_t>(L.padded);
    L.sval = arena.alloc<double>(L.padded);
    L.diag = arena.alloc<double>(n);
    L.dinv = arena.alloc<double>(n);
    DevArena tmp(s);
    int32_t* d_inv = tmp.alloc<int32_t>(n);
    int32_t* d_perm = tmp.alloc<int32_t>(n);
    int32_t* d_nrp = tmp.alloc<int32_t>(n + 1);
    int32_t* d_nci = tmp.alloc<int32_t>(L.nnz_off);
    double* d_nva = tmp.alloc<double>(L.nnz_off);
    AMG_CUDA_TRY(cudaMemcpyAsync(d_inv, inv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(d_nrp, nrp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(L.rlen, rlen.data(), sizeof(uint16_t) * n, cudaMemcpyHostToDevice, s));
    k_reorder_rows<<<blocks_for(n), kBlock, 0, s>>>(n, d_inv, d_perm, A.rp, A.ci, A.va, d_nrp, d_nci,
                                                    d_nva, L.diag, L.dinv);
    k_csr_to_sell<<<blocks_for(n), kBlock, 0, s>>>(n, d_nrp, d_nci, d_nva, width, L.scol, L.sval);
    AMG_CUDA_TRY(cudaGetLastError());
    if (compact) {
        const int64_t ce = soff[nslices];
        L.stage_entries = ce;
        L.soff = arena.alloc<int64_t>(nslices + 1);
        L.ccol = arena.alloc<int32_t>(ce);
        L.cval = arena.alloc<double>(ce);
        AMG_CUDA_TRY(cudaMemcpyAsync(L.soff, soff.data(), sizeof(int64_t) * (nslices + 1),
                                     cudaMemcpyHostToDevice, s));
        // rows past n in the last slice: padding entries of no row
        AMG_CUDA_TRY(cudaMemsetAsync(L.ccol, 0, sizeof(int32_t) * ce, s));
        AMG_CUDA_TRY(cudaMemsetAsync(L.cval, 0, sizeof(double) * ce, s));
        k_sell_own_width<double><<<blocks_for(n), kBlock, 0, s>>>(n, width, L.soff, L.scol, L.sval,
                                                                   L.ccol, L.cval);
        AMG_CUDA_TRY(cudaGetLastError());
    }
    // lanes per row: the staged one-row-per-thread kernels on sparse rows
    // (bandwidth bound), several lanes on the denser coarse rows (gather
    // latency bound)
    const double avg = n > 0 ? (double)L.nnz_off / n : 0.0;
    L.lpr = (avg <= 7.0 && staged_fits(L)) ? 0 : avg <= 16.0 ? 4 : 8;
    L.lpr_wide = L.lpr;
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
}

bool dense_inverse_device(const DevCsr& A, double* Minv, cudaStream_t s) {
    const int n = A.n;
    const int np = (n + kPanel - 1) / kPanel;
    DevArena tmp(s);
    double* W = tmp.alloc<double>((size_t)n * n);
    double* Y = tmp.alloc<double>((size_t)n * n);
    double* D = tmp.alloc<double>((size_t)np * kPanel * kPanel);
    int* err = tmp.alloc<int>(1);
    AMG_CUDA_TRY(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)n * n, s));
    AMG_CUDA_TRY(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)n * n, s));
    AMG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_dense_from_csr<<<blocks_for(n), kBlock, 0, s>>>(n, A.rp, A.ci, A.va, W);
    // Cholesky, right-looking by 32-column panels
    for (int p = 0; p < np; ++p) {
        const int k0 = p * kPanel, m = std::min(kPanel, n - k0), r0 = k0 + m;
        k_potrf_block<<<1, kPanel * kPanel, 0, s>>>(n, k0, W, D + (size_t)p * kPanel * kPanel, err);
        if (r0 < n) {
            k_panel<<<blocks_for((int64_t)(n - r0) * 32), kBlock, 0, s>>>(n, k0, m, W,
                                                                           D + (size_t)p * kPanel * kPanel);
            const int t = (n - r0 + 63) / 64;
            k_syrk<<<t * (t + 1) / 2, 256, 0, s>>>(n, r0, k0, m, W);
        }
    }
    // Y = L^-1 (Y starts at zero: the running sums), then M^-1 = Y^T Y
    for (int p = 0; p < np; ++p) {
        const int i0 = p * kPanel, m = std::min(kPanel, n - i0), r0 = i0 + m;
        k_trinv_final<<<p + 1, kPanel * kPanel, 0, s>>>(n, i0, m, Y, D + (size_t)p * kPanel * kPanel);
        if (r0 < n) {
            const int tiles = ((n - r0 + 63) / 64) * ((r0 + 63) / 64);
            k_trinv_update<<<tiles, 256, 0, s>>>(n, i0, m, W, Y);
        }
    }
    const int t = (n + 63) / 64;
    k_yty<<<t * (t + 1) / 2, 256, 0, s>>>(n, Y, Minv);
    AMG_CUDA_TRY(cudaGetLastError());
    int herr = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return herr == 0;
}

__global__ void k_to_float_padded(int n, int ld, const double* __restrict__ in, float* __restrict__ out) {
    const size_t count = (size_t)n * ld;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = t / ld, j = t % ld;
        out[t] = j < (size_t)n ? (float)in[i * n + j] : 0.f;
    }
}

void to_float_padded_device(int n, int ld, const double* in, float* out, cudaStream_t s) {
    const int64_t count = (int64_t)n * ld;
    k_to_float_padded<<<std::max(1, (int)std::min<int64_t>(blocks_for(count), 1216 * 4)), kBlock, 0, s>>>(
        n, ld, in, out);
    AMG_CUDA_TRY(cudaGetLastError());
}

void scale_inverse_device(int n, const double* diag, const double* Minv, double* Minv_s,
                          cudaStream_t s) {
    k_scale_inverse<<<blocks_for((int64_t)n * n), kBlock, 0, s>>>(n, diag, Minv, Minv_s);
    AMG_CUDA_TRY(cudaGetLastError());
}

void build_level_fp32(DevLevel& L, const double* coarse_diag, DevArena& arena, cudaStream_t s) {
    const int n = L.n;
    L.sval32 = arena.alloc<float>(L.padded);
    L.diag32 = arena.alloc<float>(n);
    L.dinv32 = arena.alloc<float>(n);
    L.t32 = coarse_diag ? arena.alloc<float>(n) : nullptr;
    L.x32 = arena.alloc<float>(n);
    L.b32 = arena.alloc<float>(n);
    L.r32 = arena.alloc<float>(n);
    k_level_fp32<<<blocks_for(n), kBlock, 0, s>>>(n, L.width, L.scol, L.sval, L.diag, L.agg, coarse_diag,
                                                  L.sval32, L.diag32, L.dinv32, L.t32);
    AMG_CUDA_TRY(cudaGetLastError());
    if (L.soff) {
        const int64_t ce = L.stage_entries;
        L.cval32 = arena.alloc<float>(ce);
        AMG_CUDA_TRY(cudaMemsetAsync(L.cval32, 0, sizeof(float) * ce, s));
        k_sell_own_width<float><<<blocks_for(n), kBlock, 0, s>>>(n, L.width, L.soff, nullptr,
                                                                  L.sval32, nullptr, L.cval32);
        AMG_CUDA_TRY(cudaGetLastError());
    }
}

}  // namespace amg
