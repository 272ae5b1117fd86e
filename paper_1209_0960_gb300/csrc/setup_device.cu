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

// L_jj = sqrt(M_jj - sum_{k<j} L_jk^2); one warp
__global__ void k_chol_diag(int n, int j, double* __restrict__ L, int* __restrict__ err) {
    const int lane = threadIdx.x;
    const double* row = L + (size_t)j * n;
    double s = 0.0;
    for (int k = lane; k < j; k += 32) s += row[k] * row[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        const double d = row[j] - s;
        if (!(d > 0.0)) {
            *err = 1;
            L[(size_t)j * n + j] = 1.0;
        } else {
            L[(size_t)j * n + j] = sqrt(d);
        }
    }
}

// L_ij = (M_ij - sum_{k<j} L_ik L_jk) / L_jj for i > j; one warp per row i
__global__ void k_chol_col(int n, int j, double* __restrict__ L) {
    const int lane = threadIdx.x & 31;
    const int i = j + 1 + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= n) return;
    const double* ri = L + (size_t)i * n;
    const double* rj = L + (size_t)j * n;
    double s = 0.0;
    for (int k = lane; k < j; k += 32) s += ri[k] * rj[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) L[(size_t)i * n + j] = (ri[j] - s) / rj[j];
}

// U = L^T (row access to the columns of L in the backward substitution)
__global__ void k_transpose(int n, const double* __restrict__ L, double* __restrict__ U) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    U[(size_t)j * n + i] = L[t];
}

// Column c of the inverse, one warp per column: forward L y = e_c (y_k = 0
// for k < c), then backward L^T x = y, with the column held in shared memory;
// the lanes split each inner product.
__global__ void k_chol_inverse(int n, const double* __restrict__ L, const double* __restrict__ U,
                               double* __restrict__ X) {
    extern __shared__ double y[];
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    for (int k = lane; k < n; k += 32) y[k] = 0.0;
    __syncwarp();
    for (int i = c; i < n; ++i) {
        const double* li = L + (size_t)i * n;
        double s = 0.0;
        for (int k = c + lane; k < i; k += 32) s = __fma_rn(li[k], y[k], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) y[i] = ((i == c) ? 1.0 - s : -s) / li[i];
        __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
        const double* ui = U + (size_t)i * n;
        double s = 0.0;
        for (int k = i + 1 + lane; k < n; k += 32) s = __fma_rn(ui[k], y[k], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) y[i] = (y[i] - s) / ui[i];
        __syncwarp();
    }
    for (int k = lane; k < n; k += 32) X[(size_t)k * n + c] = y[k];
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
    // lanes per row: the staged one-row-per-thread kernels on sparse rows
    // (bandwidth bound), several lanes on the denser coarse rows (gather
    // latency bound)
    const double avg = n > 0 ? (double)L.nnz_off / n : 0.0;
    L.lpr = (avg <= 7.0 && width <= kFineMaxWidth) ? 0 : avg <= 16.0 ? 4 : 8;
    L.lpr_wide = L.lpr;
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
}

bool dense_inverse_device(const DevCsr& A, double* Minv, cudaStream_t s) {
    const int n = A.n;
    DevArena tmp(s);
    double* L = tmp.alloc<double>((size_t)n * n);
    int* err = tmp.alloc<int>(1);
    AMG_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(double) * (size_t)n * n, s));
    AMG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_dense_from_csr<<<blocks_for(n), kBlock, 0, s>>>(n, A.rp, A.ci, A.va, L);
    for (int j = 0; j < n; ++j) {
        k_chol_diag<<<1, 32, 0, s>>>(n, j, L, err);
        if (j + 1 < n) k_chol_col<<<blocks_for((int64_t)(n - j - 1) * 32), kBlock, 0, s>>>(n, j, L);
    }
    AMG_CUDA_TRY(cudaGetLastError());
    double* U = tmp.alloc<double>((size_t)n * n);
    k_transpose<<<blocks_for((int64_t)n * n), kBlock, 0, s>>>(n, L, U);
    const size_t smem = sizeof(double) * (size_t)n;
    if (smem > 40 * 1024)   // the 48 KB default also holds static shared memory
        raise_dyn_smem(k_chol_inverse, smem);
    k_chol_inverse<<<n, 32, smem, s>>>(n, L, U, Minv);
    AMG_CUDA_TRY(cudaGetLastError());
    int herr = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return herr == 0;
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
}

}  // namespace amg
