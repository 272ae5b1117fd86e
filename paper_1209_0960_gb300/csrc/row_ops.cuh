// Device-side row operations shared by the solve kernels (kernels.cu) and the
// persistent coarse-level kernels (coarse.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace amg {
namespace rowops {

template <int W, typename T>
__device__ __forceinline__ T group_sum(T s) {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off, W);
    return s;
}

__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }

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
//                pass from a zero guess, recomputed instead of read back;
//   kNbrProlong  x_j + omega t_j e_agg(j): the post-smoothing of a two-colour
//                level reads the prolongated values of the other colour
//                without writing them (the next pass overwrites that colour).
// ---------------------------------------------------------------------------
enum NbrMode : int { kNbrX = 0, kNbrFirst = 1, kNbrProlong = 2 };

constexpr int kUnroll = 8;

// Load of a vector that other blocks may have written earlier in the same
// kernel (persistent kernels): through L2, bypassing the non-coherent L1.
template <bool COH, typename T>
__device__ __forceinline__ T ldv(const T* p) {
    if (COH) return __ldcg(p);
    return *p;
}

template <int MODE, bool SCALED, bool COH, typename T>
__device__ __forceinline__ T nbr_value(int j, const T* x, const T* b, const T* __restrict__ dinv,
                                       const int32_t* __restrict__ agg, const T* __restrict__ t,
                                       const T* e, T omega) {
    if (MODE == kNbrFirst) return ldv<COH>(b + j) * dinv[j];
    T v = ldv<COH>(x + j);
    if (MODE == kNbrProlong) {
        const int ag = agg[j];
        if (ag >= 0) v = fmad(SCALED ? omega * t[j] : omega, ldv<COH>(e + ag), v);
    }
    return v;
}

template <int LPR, int MODE, bool SCALED, typename T, bool COH = false>
__device__ __forceinline__ T row_update(int64_t base, int len, int lane, int jmax,
                                        const int32_t* __restrict__ scol,
                                        const T* __restrict__ sval, const T* x, const T* b,
                                        const T* __restrict__ dinv,
                                        const int32_t* __restrict__ agg, const T* __restrict__ t,
                                        const T* e, T omega, T acc) {
    if (LPR == 1) {
        // one thread per row (the fine level): a plain loop keeps the register
        // count low, so enough warps stay resident to saturate DRAM
        T s = acc;
#pragma unroll 4
        for (int k = 0; k < len; ++k) {
            const int64_t ee = base + 32 * (int64_t)k;
            const int j = scol[ee];
            const T a = sval[ee];
            if (j < jmax) s = fmad(-a, nbr_value<MODE, SCALED, COH>(j, x, b, dinv, agg, t, e, omega), s);
        }
        return s;
    }
    T s = lane == 0 ? acc : T(0);
    // every lane of the warp runs the same number of batches (the warp's
    // longest row decides), so the warp-wide votes below see all 32 lanes
    constexpr int per = LPR * kUnroll;
    const int mine = len > lane ? (len - lane + per - 1) / per : 0;
    const int batches = __reduce_max_sync(0xffffffffu, mine);
    for (int it = 0; it < batches; ++it) {
        const int k0 = lane + it * per;
        int j[kUnroll];
        T a[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int k = k0 + u * LPR;
            const bool in = k < len;
            const int64_t ee = base + 32 * (int64_t)(in ? k : 0);
            j[u] = in ? scol[ee] : jmax;
            a[u] = in ? sval[ee] : T(0);
        }
        // slots past the longest row of the warp are skipped by a warp-uniform
        // branch: a predicated-off float64 FMA would still occupy the pipe
        T v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            v[u] = T(0);
            if (__any_sync(0xffffffffu, j[u] < jmax) && j[u] < jmax)
                v[u] = nbr_value<MODE, SCALED, COH>(j[u], x, b, dinv, agg, t, e, omega);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (__any_sync(0xffffffffu, j[u] < jmax) && j[u] < jmax) s = fmad(-a[u], v[u], s);
    }
    return group_sum<LPR>(s);
}

// Rows handled by a launch: LPR lanes per row, rows from r0 rounded down to a
// slice boundary so that warps read whole slices.
template <int LPR>
struct RowOf {
    int row, lane;
    bool valid;
    __device__ RowOf(int r0, int r1) {
        const int64_t tt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        row = (r0 & ~31) + (int)(tt / LPR);
        lane = (int)(tt % LPR);
        valid = row >= r0 && row < r1;
    }
};

}  // namespace rowops
}  // namespace amg
