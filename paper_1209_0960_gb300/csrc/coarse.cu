// Persistent kernels for the coarse part of the V-cycle (Sec. 2).
//
// On the coarse levels a colour pass touches a few thousand rows; launched one
// kernel per pass, the V-cycle would be about 140 dependent launches whose cost
// is launch and memory latency, not bandwidth.  Here:
//   * the medium levels (up to ~600k rows) run their pre-smoothing and
//     restriction in one cooperative launch and their prolongation and
//     post-smoothing in another, with a grid-wide barrier between dependent
//     phases;
//   * the small levels (up to ~50k rows) and the coarsest dense solve run as a
//     whole V-cycle inside one thread-block cluster, with the hardware cluster
//     barrier between phases.
// The phases are the same passes as the one-kernel-per-pass path (kernels.cu),
// built from the row operations in row_ops.cuh, with every vector that other
// blocks write inside the kernel read through L2.
//
// The grid barrier waits with a time limit (about one second): on expiry it
// records AMG_ETIMEOUT in the CG status word and every block returns.

#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "device.h"
#include "row_ops.cuh"

namespace amg {

namespace {

using namespace rowops;
namespace cgr = cooperative_groups;

constexpr long long kBarrierTimeoutCycles = 2000000000LL;   // about 1 s

// Grid-wide barrier: block 0 adds 2^31 - (blocks - 1), every other block adds
// 1, so the top bit of the counter flips exactly when all blocks have arrived;
// each block waits for the flip of the value it saw on arrival.
__device__ __forceinline__ bool grid_barrier(GridBarrier* gb, PcgScalars* sc) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int inc = blockIdx.x == 0 ? (0x80000000u - (gridDim.x - 1)) : 1u;
        __threadfence();
        const unsigned int old = atomicAdd(&gb->arrive, inc);
        volatile unsigned int* va = &gb->arrive;
        volatile int* ve = &gb->err;
        const long long t0 = clock64();
        unsigned int spins = 0;
        while (((old ^ *va) & 0x80000000u) == 0u) {
            if ((++spins & 255u) == 0u) {
                if (*ve) break;
                if (clock64() - t0 > kBarrierTimeoutCycles) {
                    atomicExch(&gb->err, 1);
                    sc->status = AMG_ETIMEOUT;
                    sc->done = 1;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = *ve == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool cluster_barrier() {
    cgr::this_cluster().sync();
    return true;
}

// Rows [r0, r1) in groups of LPR lanes, looped so that all 32 lanes of a warp
// run the same iterations (the row operations vote across the warp).
template <int LPR, typename F>
__device__ __forceinline__ void for_rows(int r0, int r1, int gtid, int gthreads, F&& f) {
    constexpr int rpw = 32 / LPR;
    const int warp = gtid >> 5, nwarps = gthreads >> 5;
    const int l32 = gtid & 31;
    const int sub = l32 / LPR, lane = l32 % LPR;
    for (int base = (r0 & ~31) + warp * rpw; base < r1; base += nwarps * rpw) {
        const int row = base + sub;
        f(row, lane, row >= r0 && row < r1);
    }
}

template <int LPR, typename T>
__device__ void ph_first(const LevelView<T>& L, int gtid, int gth) {
    const int c1 = L.cptr[1];
    const int c2 = L.cptr[L.ncolours > 1 ? 2 : 1];
    for_rows<LPR>(0, c2, gtid, gth, [&](int row, int lane, bool valid) {
        const int rr = valid ? row : 0;
        const int len = (valid && rr >= c1) ? (int)L.rlen[rr] : 0;
        const int64_t base = L.sptr[rr >> 5] + (rr & 31);
        const T s = row_update<LPR, kNbrFirst, false, T, true>(
            base, len, lane, c1, L.scol, L.sval, L.x, L.b, L.dinv, nullptr, nullptr, nullptr, T(0),
            valid ? __ldcg(L.b + rr) : T(0));
        if (valid && lane == 0) L.x[rr] = s * L.dinv[rr];
    });
}

template <int LPR, int MODE, bool SCALED, typename T>
__device__ void ph_pass(const LevelView<T>& L, int col, int jmax, const T* e, T omega, int gtid,
                        int gth) {
    const int r0 = L.cptr[col], r1 = L.cptr[col + 1];
    for_rows<LPR>(r0, r1, gtid, gth, [&](int row, int lane, bool valid) {
        const int rr = valid ? row : r0;
        const int64_t base = L.sptr[rr >> 5] + (rr & 31);
        const T s = row_update<LPR, MODE, SCALED, T, true>(
            base, valid ? (int)L.rlen[rr] : 0, lane, jmax, L.scol, L.sval, L.x, nullptr, L.dinv, L.agg,
            L.t, e, omega, valid ? __ldcg(L.b + rr) : T(0));
        if (valid && lane == 0) L.x[rr] = s * L.dinv[rr];
    });
}

template <int LPR, typename T>
__device__ void ph_residual(const LevelView<T>& L, int gtid, int gth) {
    const int c1 = L.cptr[1];
    for_rows<LPR>(c1, L.n, gtid, gth, [&](int row, int lane, bool valid) {
        const int rr = valid ? row : c1;
        const int64_t base = L.sptr[rr >> 5] + (rr & 31);
        const T s0 = valid ? fmad(-L.diag[rr], __ldcg(L.x + rr), __ldcg(L.b + rr)) : T(0);
        const T v = row_update<LPR, kNbrX, false, T, true>(
            base, valid ? (int)L.rlen[rr] : 0, lane, L.n, L.scol, L.sval, L.x, nullptr, nullptr,
            nullptr, nullptr, nullptr, T(0), s0);
        if (valid && lane == 0) L.r[rr] = v;
    });
}

template <bool SCALED, typename T>
__device__ void ph_restrict(const LevelView<T>& L, T* bc, int gtid, int gth) {
    for (int J = gtid; J < L.n_coarse; J += gth) {
        const int k1 = L.rptr[J + 1];
        T s = T(0);
        for (int k0 = L.rptr[J]; k0 < k1; k0 += kUnroll) {
            int i[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) i[u] = (k0 + u < k1) ? L.ridx[k0 + u] : -1;
            T v[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                v[u] = i[u] >= 0 ? (SCALED ? L.t[i[u]] * __ldcg(L.r + i[u]) : __ldcg(L.r + i[u])) : T(0);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (i[u] >= 0) s += v[u];
        }
        bc[J] = s;
    }
}

template <bool SCALED, typename T>
__device__ void ph_prolong(const LevelView<T>& L, const T* e, T omega, int gtid, int gth) {
    for (int i = L.cptr[1] + gtid; i < L.n; i += gth) {
        const int a = L.agg[i];
        if (a >= 0) L.x[i] = fmad(SCALED ? omega * L.t[i] : omega, __ldcg(e + a), __ldcg(L.x + i));
    }
}

// x = M b on the coarsest level, one warp per row, float64
template <typename T>
__device__ void ph_dense(const LevelView<T>& C, const double* __restrict__ M, int gtid, int gth) {
    const int lane = gtid & 31;
    const int n = C.n;
    for (int row = gtid >> 5; row < n; row += gth >> 5) {
        const double* m = M + (size_t)row * n;
        double s = 0.0;
        for (int k = lane; k < n; k += 32) s = fmad(m[k], (double)__ldcg(C.b + k), s);
        s = group_sum<32>(s);
        if (lane == 0) C.x[row] = (T)s;
    }
}

#define AMG_DEV_LPR(lpr, CALL)                               \
    switch (lpr) {                                           \
        case 1: { constexpr int LPR = 1; CALL; } break;      \
        case 4: { constexpr int LPR = 4; CALL; } break;      \
        default: { constexpr int LPR = 8; CALL; } break;     \
    }

// Pre-smoothing and restriction of one level; `sync` separates dependent
// phases.  Returns false when a barrier failed.
template <bool SCALED, typename T, typename Sync>
__device__ bool level_down(const LevelView<T>& L, T* bc, int gtid, int gth, Sync&& sync) {
    const int C = L.ncolours;
    AMG_DEV_LPR(L.lpr, (ph_first<LPR, T>(L, gtid, gth)));
    if (!sync()) return false;
    for (int col = 2; col < C; ++col) {
        AMG_DEV_LPR(L.lpr, (ph_pass<LPR, kNbrX, SCALED, T>(L, col, L.cptr[col], nullptr, T(0), gtid, gth)));
        if (!sync()) return false;
    }
    for (int col = C - 2; col >= 0; --col) {
        AMG_DEV_LPR(L.lpr, (ph_pass<LPR, kNbrX, SCALED, T>(L, col, L.n, nullptr, T(0), gtid, gth)));
        if (!sync()) return false;
    }
    AMG_DEV_LPR(L.lpr, (ph_residual<LPR, T>(L, gtid, gth)));
    if (!sync()) return false;
    ph_restrict<SCALED>(L, bc, gtid, gth);
    return sync();
}

// Prolongation and post-smoothing of one level; the final phase is followed by
// a barrier only when `sync_last`.
template <bool SCALED, typename T, typename Sync>
__device__ bool level_up(const LevelView<T>& L, const T* e, T omega, bool sync_last, int gtid,
                         int gth, Sync&& sync) {
    const int C = L.ncolours;
    if (C == 2) {
        AMG_DEV_LPR(L.lpr, (ph_pass<LPR, kNbrProlong, SCALED, T>(L, 0, L.n, e, omega, gtid, gth)));
        if (!sync()) return false;
        AMG_DEV_LPR(L.lpr, (ph_pass<LPR, kNbrX, SCALED, T>(L, 1, L.n, nullptr, T(0), gtid, gth)));
        if (!sync()) return false;
        AMG_DEV_LPR(L.lpr, (ph_pass<LPR, kNbrX, SCALED, T>(L, 0, L.n, nullptr, T(0), gtid, gth)));
        return sync_last ? sync() : true;
    }
    ph_prolong<SCALED>(L, e, omega, gtid, gth);
    if (!sync()) return false;
    for (int col = 0; col < C; ++col) {
        AMG_DEV_LPR(L.lpr, (ph_pass<LPR, kNbrX, SCALED, T>(L, col, L.n, nullptr, T(0), gtid, gth)));
        if (!sync()) return false;
    }
    for (int col = C - 2; col >= 0; --col) {
        AMG_DEV_LPR(L.lpr, (ph_pass<LPR, kNbrX, SCALED, T>(L, col, L.n, nullptr, T(0), gtid, gth)));
        if (col > 0 || sync_last) {
            if (!sync()) return false;
        }
    }
    return true;
}

// Cooperative grid: down (up == 0) runs levels l0..l1-1 from fine to coarse;
// up (up == 1) runs levels l1-1..l0 from coarse to fine.
template <typename T, bool SCALED>
__global__ void __launch_bounds__(kBlock) k_medium(const LevelView<T>* __restrict__ lv, int l0, int l1,
                                                   int up, T omega, GridBarrier* gb, PcgScalars* sc) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gth = gridDim.x * blockDim.x;
    auto sync = [&] { return grid_barrier(gb, sc); };
    if (!up) {
        for (int l = l0; l < l1; ++l) {
            const LevelView<T> L = lv[l];
            if (!level_down<SCALED>(L, lv[l + 1].b, gtid, gth, sync)) return;
        }
    } else {
        for (int l = l1 - 1; l >= l0; --l) {
            const LevelView<T> L = lv[l];
            if (!level_up<SCALED>(L, lv[l + 1].x, omega, l > l0, gtid, gth, sync)) return;
        }
    }
}

// One thread-block cluster: full V-cycle of levels ls..lc (lc = coarsest).
template <typename T, bool SCALED>
__global__ void __launch_bounds__(kSmallBlock) k_small(const LevelView<T>* __restrict__ lv, int ls,
                                                       int lc, const double* __restrict__ M, T omega) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gth = gridDim.x * blockDim.x;
    auto sync = [] { return cluster_barrier(); };
    for (int l = ls; l < lc; ++l) {
        const LevelView<T> L = lv[l];
        level_down<SCALED>(L, lv[l + 1].b, gtid, gth, sync);
    }
    ph_dense(lv[lc], M, gtid, gth);
    if (lc > ls) cluster_barrier();
    for (int l = lc - 1; l >= ls; --l) {
        const LevelView<T> L = lv[l];
        level_up<SCALED>(L, lv[l + 1].x, omega, l > ls, gtid, gth, sync);
    }
}

template <typename T, bool SCALED>
void launch_medium_impl(const Persistent& P, const LevelView<T>* lv, int up, double omega,
                        PcgScalars* sc, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.coop_blocks);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_medium<T, SCALED>, lv, P.lm0, P.ls, up, (T)omega,
                                    P.barrier, sc));
}

template <typename T, bool SCALED>
void launch_small_impl(const Persistent& P, const LevelView<T>* lv, const double* M, double omega,
                       cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.cluster);
    cfg.blockDim = dim3(kSmallBlock);
    cfg.dynamicSmemBytes = kSmallSmem;   // one CTA per SM
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_small<T, SCALED>, lv, P.ls, P.lc, M, (T)omega));
}

template <typename K>
int cluster_size_for(K kernel) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSmem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int cs : {16, 8}) {
        if (cs > 8 &&
            cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kSmallBlock);
        cfg.dynamicSmemBytes = kSmallSmem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) == cudaSuccess && nclusters > 0)
            return cs;
        cudaGetLastError();
    }
    return 0;
}

}  // namespace

bool persistent_config(int sms, int& coop_blocks, int& cluster) {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_medium<double, false>, kBlock, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_medium<float, true>, kBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    coop_blocks = std::min(std::min(a, b), 2) * sms;
    const int c64 = cluster_size_for(k_small<double, false>);
    const int c32 = cluster_size_for(k_small<float, true>);
    cluster = std::min(c64, c32);
    return coop_blocks > 0 && cluster > 0;
}

void launch_medium64(const Persistent& P, int up, double omega, PcgScalars* sc, cudaStream_t s) {
    launch_medium_impl<double, false>(P, P.lv64, up, omega, sc, s);
}
void launch_medium32(const Persistent& P, int up, double omega, PcgScalars* sc, cudaStream_t s) {
    launch_medium_impl<float, true>(P, P.lv32, up, omega, sc, s);
}
void launch_small64(const Persistent& P, const double* M, double omega, cudaStream_t s) {
    launch_small_impl<double, false>(P, P.lv64, M, omega, s);
}
void launch_small32(const Persistent& P, const double* M, double omega, cudaStream_t s) {
    launch_small_impl<float, true>(P, P.lv32, M, omega, s);
}

}  // namespace amg
