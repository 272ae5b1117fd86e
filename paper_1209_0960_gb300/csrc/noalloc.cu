// amg_residual_norm_noalloc: ||b - A x||_2 for a CSR matrix in device memory,
// computed without allocating any memory.
//
// Why: some callers cannot call cudaMalloc at the point where they need a
// residual check.  cudaMalloc and cudaFree may synchronise the whole device,
// which a latency-bound loop sharing the GPU with other streams cannot afford;
// an allocator hook or callback must not re-enter the allocator; and a
// process that has handed all device memory to a pool it does not control has
// nothing left to allocate from.  This entry point needs no context and no
// allocation: the per-block partial sums of its deterministic two-stage
// reduction live in a fixed file-scope device array.
//
// The array holds kMaxBlocks partial sums, one per 256-row block, so matrices
// of up to kMaxBlocks * 256 = 16,777,216 rows are accepted; larger ones are
// rejected with AMG_EINVAL.  Every GPU that loads the library holds the array
// (512 KiB plus a counter) until the process exits.  All calls share it and it
// keeps the last call's contents; each call clears the arrival counter before
// its kernel runs.  Calls that overlap on the GPU (concurrent streams, or
// several host threads) race on the array and must be serialised by the
// caller.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current, and caches it for
// the life of the process (a device reset invalidates it).
//
// Every pointer argument is checked with cudaPointerGetAttributes (a query,
// not an allocation): it must be device or managed memory of the current
// device, else the call returns AMG_EINVAL before anything is launched.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "device.h"

namespace amg {

namespace {

constexpr int kNaBlock = 256;
constexpr int kMaxBlocks = 65536;
constexpr int64_t kMaxRows = (int64_t)kMaxBlocks * kNaBlock;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    double partial[kMaxBlocks];   // one partial sum per block
    unsigned int counter;         // blocks finished; reset by the last one and before each call
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_scratch_mu;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the symbol's host-side name is not a device address).
NoAllocScratch* scratch_for_current_device() {
    int dev = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw Error{AMG_EINVAL, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            throw Error{AMG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    return g_scratch_ptr[dev];
}

// Reject anything but device or managed memory: a host pointer handed to the
// kernel would fault or read the wrong memory.  Returns the device that owns
// device memory, -1 for managed memory (reachable from every device).
int device_of_pointer(const void* p, const char* name) {
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{AMG_EINVAL, std::string(name) + ": cannot query the pointer (" +
                                    cudaGetErrorString(e) + ")"};
    }
    if (at.type == cudaMemoryTypeManaged) return -1;
    if (at.type != cudaMemoryTypeDevice) throw Error{AMG_EINVAL, std::string(name) + " is not device memory"};
    return at.device;
}

// One thread per row: r_i = b_i - sum_k A_ik x_k, then r_i^2 summed per block
// in a fixed order; the last block to finish adds the block sums in index
// order and writes the square root.
__global__ void __launch_bounds__(kNaBlock) k_csr_residual_norm(
    int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const double* __restrict__ va, const double* __restrict__ b, const double* __restrict__ x,
    NoAllocScratch* __restrict__ scratch, double* __restrict__ out) {
    __shared__ double sh[kNaBlock / 32];
    __shared__ bool last;
    const int row = blockIdx.x * kNaBlock + threadIdx.x;
    double v = 0.0;
    if (row < n) {
        double t = b[row];
        for (int k = rp[row]; k < rp[row + 1]; ++k) t = __fma_rn(-va[k], x[ci[k]], t);
        v = t * t;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNaBlock / 32; ++w) s += sh[w];
        scratch->partial[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&scratch->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    double a = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kNaBlock) a += __ldcg(scratch->partial + i);
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    __syncthreads();
    if (lane == 0) sh[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNaBlock / 32; ++w) s += sh[w];
        *out = sqrt(s);
        scratch->counter = 0u;
    }
}

}  // namespace
}  // namespace amg

using namespace amg;

extern "C" int amg_residual_norm_noalloc(const amg_csr* A, const double* b_dev,
                                         const double* x_dev, double* norm_dev,
                                         void* cuda_stream) {
    try {
        if (!A || !b_dev || !x_dev || !norm_dev) throw Error{AMG_EINVAL, "null argument"};
        if (!A->on_device) throw Error{AMG_EINVAL, "the matrix must be in device memory (on_device = 1)"};
        if (A->n <= 0 || !A->row_ptr || !A->col || !A->val) throw Error{AMG_EINVAL, "empty or null matrix"};
        if ((int64_t)A->n > kMaxRows)
            throw Error{AMG_EINVAL, "n = " + std::to_string(A->n) +
                                        " exceeds the fixed scratch of this entry point (at most " +
                                        std::to_string(kMaxRows) + " rows)"};
        const void* ptrs[] = {A->row_ptr, A->col, A->val, b_dev, x_dev, norm_dev};
        const char* names[] = {"A->row_ptr", "A->col", "A->val", "b_dev", "x_dev", "norm_dev"};
        int owner[6];
        for (int k = 0; k < 6; ++k) owner[k] = device_of_pointer(ptrs[k], names[k]);
        int dev = 0;
        AMG_CUDA_TRY(cudaGetDevice(&dev));
        for (int k = 0; k < 6; ++k)
            if (owner[k] >= 0 && owner[k] != dev)
                throw Error{AMG_EINVAL, std::string(names[k]) + " belongs to device " +
                                            std::to_string(owner[k]) + ", not the current device " +
                                            std::to_string(dev)};
        NoAllocScratch* scratch = scratch_for_current_device();
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        AMG_CUDA_TRY(cudaMemsetAsync(&scratch->counter, 0, sizeof(unsigned int), s));
        const int grid = (A->n + kNaBlock - 1) / kNaBlock;
        k_csr_residual_norm<<<grid, kNaBlock, 0, s>>>(A->n, A->row_ptr, A->col, A->val, b_dev, x_dev,
                                                      scratch, norm_dev);
        AMG_CUDA_TRY(cudaGetLastError());
        set_last_error("");
        return AMG_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    }
}
