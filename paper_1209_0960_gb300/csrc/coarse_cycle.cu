// Persistent kernel for the coarse part of the V-cycle (Sec. 2): every level
// from the first "small" level down to the coarsest and back up runs inside one
// cooperative launch, with grid-wide barriers between the dependent phases
// instead of one kernel launch per colour pass.  On the coarse levels the
// work per phase is a few microseconds or less, so launch latency, not DRAM
// traffic, would otherwise bound the cycle.
//
// Phases per level (C colours, rows stored colour block by colour block):
//   pre-smoothing   colour 0 with zero initial guess (x = b / A_ii on colour 0,
//                   x = 0 elsewhere), then colours 1..C-1, then C-2..0;
//   restriction     one thread per coarse row: residuals of its fine rows,
//                   summed (the rows of colour 0 were updated last and have a
//                   zero residual, so their lists leave them out);
//   (coarser levels; dense solve with the precomputed inverse on the coarsest)
//   prolongation    x_i += omega t_i e_agg(i) on rows of colour >= 1 (colour 0
//                   is recomputed by the first post-smoothing pass, which does
//                   not read its old value);
//   post-smoothing  colours 0..C-1, then C-2..0.
//
// The grid barrier spins with a time limit: if a block waits longer than about
// one second the kernel records AMG_ETIMEOUT in the CG status word and every
// block returns, so the host gets an error instead of a hung context.

#include "device.h"

namespace amg {

namespace {

constexpr long long kBarrierTimeoutCycles = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Sense-counting grid barrier with a bounded wait.  Returns false when the
// barrier (in this or an earlier phase) timed out.
__device__ __forceinline__ bool grid_sync(GridBarrier* gb, unsigned int nblocks, PcgScalars* sc) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &gb->gen;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&gb->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (*(volatile int*)&gb->err) break;
                if (clock64() - t0 > kBarrierTimeoutCycles) {
                    atomicExch(&gb->err, 1);
                    sc->status = AMG_ETIMEOUT;
                    sc->done = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)&gb->err == 0;
}

template <typename T>
__device__ __forceinline__ T ld(const T* p) { return __ldcg(p); }

// b_i - sum_j A_ij x_j over the off-diagonal entries of row i (x read through
// L2: other blocks wrote it in earlier phases)
template <typename T>
__device__ __forceinline__ T offdiag_update(const CoarseLevel<T>& L, int row, T s) {
    const int64_t base = L.sptr[row >> 5] + (row & 31);
    const int len = L.rlen[row];
    for (int k = 0; k < len; ++k) {
        const int64_t e = base + 32 * (int64_t)k;
        s = fmad(-L.sval[e], ld(L.x + L.scol[e]), s);
    }
    return s;
}

template <typename T>
__device__ __forceinline__ void gs_pass(const CoarseLevel<T>& L, int c) {
    const int r0 = L.cptr[c], r1 = L.cptr[c + 1];
    const int stride = gridDim.x * blockDim.x;
    for (int row = r0 + blockIdx.x * blockDim.x + threadIdx.x; row < r1; row += stride)
        L.x[row] = offdiag_update(L, row, ld(L.b + row)) * L.dinv[row];
}

template <typename T, bool SCALED>
__global__ void __launch_bounds__(kBlock) k_coarse_cycle(const CoarseLevel<T>* __restrict__ levels,
                                                         int lf, int lc, int nL,
                                                         const double* __restrict__ Minv, T omega,
                                                         GridBarrier* gb, PcgScalars* sc) {
    const unsigned int nb = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    // ---- down: pre-smoothing and restriction ----
    for (int l = lf; l < lc; ++l) {
        const CoarseLevel<T> L = levels[l];
        const CoarseLevel<T>& N = levels[l + 1];
        const int c1 = L.cptr[1];
        for (int row = tid; row < L.n; row += stride)
            L.x[row] = row < c1 ? ld(L.b + row) * L.dinv[row] : T(0);
        if (!grid_sync(gb, nb, sc)) return;
        for (int c = 1; c < L.ncolours; ++c) {
            gs_pass(L, c);
            if (!grid_sync(gb, nb, sc)) return;
        }
        for (int c = L.ncolours - 2; c >= 0; --c) {
            gs_pass(L, c);
            if (!grid_sync(gb, nb, sc)) return;
        }
        for (int J = tid; J < L.n_coarse; J += stride) {
            T acc = T(0);
            for (int k = L.rptr[J]; k < L.rptr[J + 1]; ++k) {
                const int i = L.ridx[k];
                const T ri = offdiag_update(L, i, fmad(-L.diag[i], ld(L.x + i), ld(L.b + i)));
                acc = SCALED ? fmad(L.t[i], ri, acc) : acc + ri;
            }
            N.b[J] = acc;
        }
        if (!grid_sync(gb, nb, sc)) return;
    }
    // ---- coarsest level: x = M b, one warp per row, float64 ----
    {
        const CoarseLevel<T>& C = levels[lc];
        const int lane = threadIdx.x & 31;
        const int warps = stride >> 5;
        for (int row = tid >> 5; row < nL; row += warps) {
            const double* m = Minv + (size_t)row * nL;
            double s = 0.0;
            for (int k = lane; k < nL; k += 32) s = fmad(m[k], (double)ld(C.b + k), s);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) C.x[row] = (T)s;
        }
        if (!grid_sync(gb, nb, sc)) return;
    }
    // ---- up: prolongation and post-smoothing ----
    for (int l = lc - 1; l >= lf; --l) {
        const CoarseLevel<T> L = levels[l];
        const T* e = levels[l + 1].x;
        for (int row = L.cptr[1] + tid; row < L.n; row += stride) {
            const int a = L.agg[row];
            if (a >= 0) L.x[row] = fmad(SCALED ? omega * L.t[row] : omega, ld(e + a), ld(L.x + row));
        }
        if (!grid_sync(gb, nb, sc)) return;
        for (int c = 0; c < L.ncolours; ++c) {
            gs_pass(L, c);
            if (!grid_sync(gb, nb, sc)) return;
        }
        for (int c = L.ncolours - 2; c >= 0; --c) {
            gs_pass(L, c);
            if (c > 0 || l > lf) {
                if (!grid_sync(gb, nb, sc)) return;
            }
        }
    }
}

template <typename T, bool SCALED>
void launch_impl(const CoarseCycle& cc, const CoarseLevel<T>* levels, const double* Minv,
                 double omega, PcgScalars* sc, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cc.blocks);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_coarse_cycle<T, SCALED>, levels, cc.lf, cc.lc, cc.nL,
                                    Minv, (T)omega, cc.barrier, sc));
}

}  // namespace

int coarse_cycle_blocks(int sms) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_coarse_cycle<double, false>, kBlock, 0);
    int per_sm32 = 0;
    cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm32, k_coarse_cycle<float, true>, kBlock, 0);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    per_sm = std::min(std::min(per_sm, per_sm32), 2);
    return per_sm * sms;
}

void launch_coarse_cycle64(const CoarseCycle& cc, const double* Minv, double omega, PcgScalars* sc,
                           cudaStream_t s) {
    launch_impl<double, false>(cc, cc.lv64, Minv, omega, sc, s);
}

void launch_coarse_cycle32(const CoarseCycle& cc, const double* Minv, double omega, PcgScalars* sc,
                           cudaStream_t s) {
    launch_impl<float, true>(cc, cc.lv32, Minv, omega, sc, s);
}

}  // namespace amg
