// Internal declarations shared by the CUDA translation units of libamg.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "amg.h"
#include "host_setup.h"

namespace amg {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

void set_last_error(const std::string& msg);

// An NVTX range for the length of a scope: the setup phases, the solves and
// the server's batches show up named in a profiler's timeline (no cost when
// no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
    ~NvtxRange() { nvtxRangePop(); }
};

#define AMG_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess)                                                      \
            throw ::amg::Error{AMG_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// ---------------------------------------------------------------------------
// device memory owned by a context
//
// Allocations are stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// owner's stream): freeing a context or a setup temporary does not wait for
// the whole device, so contexts that set up or retire while others solve (the
// server) do not stall them.  Without a stream the arena falls back to
// cudaMalloc / cudaFree.
// ---------------------------------------------------------------------------
class DevArena {
public:
    DevArena() = default;
    explicit DevArena(cudaStream_t s) : stream_(s), async_(true) {}
    DevArena(const DevArena&) = delete;
    DevArena& operator=(const DevArena&) = delete;
    ~DevArena() { release(); }
    void set_stream(cudaStream_t s) {
        stream_ = s;
        async_ = true;
    }
    template <typename T>
    T* alloc(size_t count) {
        if (count == 0) count = 1;
        void* p = nullptr;
        const size_t bytes = count * sizeof(T);
        cudaError_t e = async_ ? cudaMallocAsync(&p, bytes, stream_) : cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{AMG_ENOMEM, "device allocation of " + std::to_string(bytes) +
                                        " bytes failed: " + cudaGetErrorString(e)};
        }
        ptrs_.push_back(p);
        bytes_ += bytes;
        return static_cast<T*>(p);
    }
    void release() {
        for (void* p : ptrs_)
            if (p) async_ ? cudaFreeAsync(p, stream_) : cudaFree(p);
        ptrs_.clear();
        bytes_ = 0;
    }
    size_t bytes() const { return bytes_; }

private:
    std::vector<void*> ptrs_;
    size_t bytes_ = 0;
    cudaStream_t stream_ = nullptr;
    bool async_ = false;
};

// Pinned host memory from a process-wide pool: blocks are rounded up to a
// power of two, reused after pinned_free and never returned to the driver
// (freeing pinned memory can wait for the whole device, which would stall
// other contexts' solves).  Thread-safe.
void* pinned_alloc(size_t bytes);
void pinned_free(void* p);

// Scalars of the CG recurrence, resident on the device.
struct PcgScalars {
    double rr0;       // ||r_0||^2
    double rr;        // ||r_k||^2
    double rho;       // r_k . z_k
    double pq;        // p . A p
    double alpha, beta;
    double tol2;      // tol^2
    int32_t done;     // 1 once ||r_k|| <= tol ||r_0||
    int32_t iters;
    int32_t status;   // 0, or AMG_ENOTSPD
    int32_t flexible;
    int32_t maxit;
    int32_t loops;    // device-side loop: conditions evaluated (a bound of its own)
};

// Scalars of the BiCGSTAB recurrence, resident on the device.
struct BiScalars {
    double r0;        // ||r_0||
    double rho;       // rt . r of the current iteration
    double rho_prev;
    double alpha, w;
    double rtv;       // rt . v
    double ts, tt;    // t . s, t . t
    double rel;       // ||r|| / ||r_0|| (||s|| / ||r_0|| after a converged half step)
    double tol;
    int32_t iters;    // iterations begun (a converged half step counts as one)
    int32_t maxit;
    int32_t status;   // 0, or AMG_ENOTCONV on breakdown / maxit
    int32_t done;     // 1 once rel <= tol
    int32_t half;     // 1: the first half step met the tolerance (x += alpha y only)
    int32_t why;      // breakdown: 1 rt.r = 0, 2 rt.v = 0, 3 t.t = 0; 0 maxit
    int32_t loops;    // loop conditions evaluated (device-side loop bound)
    int32_t pad;
};

// Whether another BiCGSTAB iteration runs; on maxit or a zero rho it records
// the stop in the scalars.  Shared by the device-side loop condition and the
// host-driven loop, so both stop at the same point.
__host__ __device__ inline bool bi_continue(BiScalars& b) {
    if (b.done || b.status) return false;
    if (b.iters >= b.maxit) {
        b.status = AMG_ENOTCONV;
        b.why = 0;
        return false;
    }
    if (b.rho == 0.0) {
        b.status = AMG_ENOTCONV;
        b.why = 1;
        return false;
    }
    return true;
}

// A symmetric Gauss-Seidel sweep of one level as a single kernel.  Each
// colour pass of the sweep is cut into items of `rows` consecutive rows.  A
// persistent grid of co-resident blocks (a cooperative launch) takes the
// items in pass order, block g the items g, g + grid, g + 2 grid, ...; before
// reading x an item waits (bounded) for what it depends on, computed at setup
// from the level's graph:
//   - the item of the same rows in the previous pass over its colour (its
//     values are overwritten);
//   - in the pass just before it, the items holding neighbours of its rows
//     (their new values are read);
//   - every earlier pass since its colour's previous update, complete (their
//     reads of the old values, and the latest values of the other colours).
// Every dependency is a smaller item and every block takes its items in
// increasing order, so the sweep cannot deadlock.  Flags and counters are
// never reset: a launch's epoch is its count of arriving blocks divided by
// the grid, a flag holds the epoch of the launch that finished the item, and
// the pass counters count finished items over all launches.
struct SweepPass {
    int32_t r0, r1;   // rows of the pass's colour (smoothing order)
    int32_t jmax;     // neighbours at positions >= jmax are taken as zero
    int32_t first;    // 1: colour 0 from a zero guess, x = b / A_ii
    int32_t tiles;    // items of the pass
    int32_t item0;    // index of its first item
};

constexpr int kSweepMaxPasses = 64;

struct SweepPlan {
    int32_t rows = 0;                        // rows per item
    int32_t npass = 0;
    int32_t items = 0;
    double mean_deps = 0.0;
    SweepPass* pass = nullptr;               // [npass] (device)
    int32_t* dep_ptr = nullptr;              // [items + 1]
    int32_t* dep = nullptr;                  // >= 0: an item; < 0: -(q + 1), all of pass q
    uint32_t* flag = nullptr;                // [items] epoch of the last launch that finished it
    unsigned long long* done = nullptr;      // [npass] items finished, all launches
    unsigned long long* arrive = nullptr;    // blocks started, all launches (grid per launch)
    int32_t grid = 0;                        // co-resident blocks of the cooperative launch
    int32_t* failed = nullptr;               // set once a wait of this plan gave up
};

// One level of the hierarchy on the device.  Rows are stored in the level's
// smoothing order: grouped by colour, inside a colour by coarse aggregate,
// then by original index.  The off-diagonal part is kept in a sliced layout
// with 32-row slices of one common width W (the level's longest row): the k-th
// off-diagonal entry of row r sits at (r / 32) * 32 W + 32 k + (r mod 32), so
// a warp reading entry k of its 32 rows reads 32 consecutive values and the
// address needs no pointer load.  Padding entries point at the row itself with
// value 0; rlen holds the true row lengths so the padding costs no arithmetic.
// The diagonal is separate.
struct DevLevel {
    int32_t n = 0;
    int64_t nnz_off = 0;              // true off-diagonal entries
    int64_t padded = 0;               // entries of the padded sliced arrays
    int32_t width = 0;                // common slice width W (longest row)
    int64_t sw = 0;                   // slice stride 32 W
    int64_t stage_cap = 0;            // entries a staged block (8 consecutive slices) needs at
                                      // most: 256 W, or with per-slice widths 32 x max over
                                      // 8-slice windows of the sum of the slices' longest rows
    int32_t ncolours = 0;
    int32_t n_coarse = 0;
    std::vector<int32_t> cptr;        // host copy: first row of each colour, [ncolours+1]
    std::vector<int64_t> cnnz;        // host copy: off-diagonal entries of each colour block
    int32_t lpr = 0;                  // lanes per row of the row kernels: 0 = the fine
                                      // level's kernels (one row per thread, slices staged
                                      // in shared memory, tiles within kMaxStageBytes), else
                                      // 1, 2, 4 or 8 lanes with batched gathers
    int32_t block = 256;              // threads per block of the row kernels (lpr >= 1): 256 or 128
    int32_t lpr_wide = 0;             // lanes per row of launches over >= wide_rows rows
    int32_t wide_rows = 0x7fffffff;
    bool fused_restrict = false;      // residual and restriction in one kernel (lpr == 0)
    bool fused_ok = false;            // the level allows the fused kernel (two colours,
                                      // aggregates of at most 32 rows of colour 1)
    int32_t* err = nullptr;           // device status word for kernel-side errors (timeouts)
    uint16_t* rlen = nullptr;         // [n] off-diagonal entries per row
    int32_t* scol = nullptr;          // [padded] permuted column indices
    double* sval = nullptr;           // [padded]
    // sliced layout with per-slice widths, for the staged kernels on levels
    // whose rows vary in length (null elsewhere): slice s padded only to its
    // longest row K_s, at soff[s] = 32 (K_0 + ... + K_{s-1}), entry k of lane
    // i at soff[s] + 32 k + i
    int64_t* soff = nullptr;          // [nslices + 1]
    int64_t stage_entries = 0;        // soff[nslices]
    int32_t carve = -1;               // preferred shared-memory carveout of the staged kernels
                                      // (percent of the SM's maximum; the rest is L1 for the
                                      // neighbour gathers), -1: the driver's choice
    int32_t* ccol = nullptr;
    double* cval = nullptr;
    float* cval32 = nullptr;
    double* diag = nullptr;           // [n]
    double* dinv = nullptr;           // [n] 1 / A_ii
    int32_t* agg = nullptr;           // [n] permuted coarse index or -1
    int32_t* rptr = nullptr;          // [n_coarse+1] restriction lists
    int32_t* ridx = nullptr;          // fine rows of colour >= 1 of each coarse row
    double* x = nullptr;              // level correction
    double* b = nullptr;              // level right-hand side
    double* r = nullptr;              // level residual
    // float32 copies, symmetric diagonal scaling S^-1 A S^-1 with S = diag(sqrt(A_ii))
    float* sval32 = nullptr;
    float* dinv32 = nullptr;
    float* diag32 = nullptr;
    float* t32 = nullptr;             // s_fine[i] / s_coarse[agg[i]] for the transfers
    float* x32 = nullptr;
    float* b32 = nullptr;
    float* r32 = nullptr;
    // smoothing sweeps as dependency-driven kernels (lane shapes only): the
    // pre-smoother (first two colours from zero, forward, backward) and the
    // post-smoother (forward, backward), planned for rows = block / lpr
    bool sweep = false;
    const SweepPlan* plan_pre = nullptr;
    const SweepPlan* plan_post = nullptr;
};

// largest tile of the staged kernels (index and value of the entries of 8
// consecutive slices): two blocks still fit on an SM.  With the common width
// that is a longest row of at most 32 off-diagonals.
constexpr int64_t kMaxStageBytes = 96 * 1024;
// shared memory of a staged block's tile
inline int64_t stage_bytes(const DevLevel& L, size_t value_bytes) {
    return L.stage_cap * (int64_t)(sizeof(int32_t) + value_bytes);
}
inline bool staged_fits(const DevLevel& L) { return stage_bytes(L, sizeof(double)) <= kMaxStageBytes; }

// Launch profiler: events around launches, grouped by kernel class.
struct Profiler {
    bool on = false;        // events around every launch (graphs off)
    bool graphs = false;    // events around graph launches only (graphs on)
    struct Rec { int kind; double bytes; int ev; };
    std::vector<cudaEvent_t> events;   // pool, pairs (start, end)
    std::vector<Rec> recs;
    int next = 0;
};

enum KernelKind : int {
    kKGsL0 = 0, kKGsCoarse, kKResidualL0, kKResidualCoarse, kKRestrict, kKProlong, kKCoarseSolve,
    kKFirstL0, kKPassProlongL0,
    kKCgSpmv, kKCgUpdate, kKCgDot, kKCgP, kKConvert, kKZero, kKPermute, kKGraphA, kKGraphB,
    kKGraphFrom   // kKGraphFrom + l: V-cycle replayed from level l (graph profiling)
};

struct HostLevel {
    HostCsr A;                        // original numbering of this level
    AggResult agg;                    // aggregation of this level (not on the coarsest)
    std::vector<int32_t> colour;
    int32_t ncolours = 0;
    std::vector<int32_t> perm;        // original index -> position in smoothing order
};

}  // namespace amg

namespace amg {

// ---------------------------------------------------------------------------
// kernel launchers (kernels.cu)
// ---------------------------------------------------------------------------
constexpr int kBlock = 256;

// modes of the deterministic "last block" reduction
enum FinalMode : int {
    kRR0 = 0,       // initial residual norm
    kPQ = 1,        // p.Ap -> alpha
    kRR = 2,        // updated residual norm -> convergence test
    kRZ = 3,        // r.z -> beta (standard CG)
    kRZFlex = 4,    // r.z and r.(z - z_old) -> beta (flexible CG)
    kRho0 = 5,      // initial r.z, p = z
    kStore = 6,     // raw sum into out[0]
};

// device work areas of the CG reductions
struct CgWork {
    double* partials = nullptr;       // [max blocks]
    double* partials2 = nullptr;
    unsigned int* counters = nullptr; // one per reduction kernel, self-resetting
    PcgScalars* sc = nullptr;
};

// Solve-phase launches.  With programmatic dependent launch (PDL) a kernel
// may begin while its stream predecessor is still running: every solve kernel
// signals its dependents as soon as it starts and, before it reads anything a
// solve kernel writes (vectors, CG scalars, counters) or writes anything,
// waits (griddepcontrol.wait) until all its predecessors have finished and
// their writes are visible.  What it does before the wait reads only
// matrices and index lists fixed at setup, so the overlap hides launch
// latency and the first dependent loads of each kernel.  Set per calling
// thread from the context at API entry.
// Sets the condition of the device-side CG loop (a WHILE graph node) to
// "not converged, no breakdown, fewer than maxit iterations" from the device
// scalars; it also counts its own evaluations and stops at maxit.
void launch_cg_continue(cudaGraphConditionalHandle h, PcgScalars* sc, cudaStream_t s);
extern thread_local bool t_launch_overlap;
// grids above this many blocks launch without the overlap: a wide grid that
// starts early only occupies the SMs its predecessor is still using
extern int g_overlap_max_blocks;

// Dynamic shared memory above the default needs a per-function attribute,
// which is process-wide state: contexts set up and solved on several threads
// at once must never lower it under another thread's launch.  This raises
// the function's limit to at least `bytes` (never lowers it), once per size.
void raise_dyn_smem(const void* func, size_t bytes);
template <typename... KArgs>
void raise_dyn_smem(void (*kernel)(KArgs...), size_t bytes) {
    raise_dyn_smem(reinterpret_cast<const void*>(kernel), bytes);
}

// carve >= 0: the launch's preferred shared-memory carveout, in percent of
// the SM's maximum shared memory (the rest of the unified L1/shared array is
// L1 cache); -1: the driver's choice
template <typename... KArgs, typename... Args>
void launch_kernel_carve(void (*kernel)(KArgs...), int grid, int block, size_t smem, int carve,
                         cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    unsigned n = 0;
    if (t_launch_overlap && grid <= g_overlap_max_blocks) {
        attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    if (carve >= 0) {
        attr[n].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
        attr[n].val.sharedMemCarveout = (unsigned)carve;
        ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{AMG_ECUDA, std::string("kernel launch (grid ") + std::to_string(grid) +
                                   ", block " + std::to_string(block) + ", shared " +
                                   std::to_string(smem) + " B) failed: " + cudaGetErrorString(e)};
    }
}

template <typename... KArgs, typename... Args>
void launch_kernel(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                   Args&&... args) {
    launch_kernel_carve(kernel, grid, block, smem, -1, s, std::forward<Args>(args)...);
}

// Runs the staged kernels' bounded wait against an mbarrier that no copy
// completes (at most `limit` polls; 0: the kernels' own limit) and returns the
// status the kernel recorded and the kernel's time (kernels.cu).
void wait_selftest(long long limit, cudaStream_t s, int32_t* status, double* elapsed_ms);

extern int g_reduction_blocks;        // grid of the reduction kernels (SMs x 8)
int reduction_blocks(int64_t work_threads);

// ---------------------------------------------------------------------------
// V-cycle launches as records
//
// Every V-cycle kernel is a body run(bid, gdim, VArgs) over one block: as its
// own launch (the block and grid of the launch) or as one segment of a
// launch that covers the same step of several contexts' V-cycles (each block
// finds its segment and runs the body with that segment's block index and
// arguments).  A segment's rows are computed exactly as in its own launch, so
// a batched V-cycle gives each context the bits of its own V-cycle.
// ---------------------------------------------------------------------------
struct VArgs {
    int32_t r0 = 0, r1 = 0, jmax = 0, n = 0, nc = 0, width = 0, ld = 0;
    int64_t sw = 0, nslices = 0, cap = 0;
    const uint16_t* rlen = nullptr;
    const int32_t* scol = nullptr;
    const int32_t* idx = nullptr;     // aggregate map, or restriction list pointers
    const int32_t* idx2 = nullptr;    // restriction list rows
    const void* sval = nullptr;
    const int64_t* soff = nullptr;    // staged kernels: slice offsets of the layout with
                                      // per-slice widths (scol / sval then point at it)
    const void* dv = nullptr;         // 1/A_ii, A_ii, or the dense coarsest inverse
    const void* t = nullptr;          // transfer weights of the scaled levels
    const void* b = nullptr;          // right-hand side / residual / coarse correction
    void* x = nullptr;
    void* out = nullptr;              // residual, coarse right-hand side, or zeroed vector
    const double* rin = nullptr;      // float64 residual entering the float32 V-cycle
    const double* isq = nullptr;      // 1 / sqrt(A_ii) of level 0
    double* z = nullptr;              // float64 output of the float32 V-cycle
    int32_t* err = nullptr;
    double omega = 0.0;
};

struct VRec;
// launches up to kMaxVBatch records of one body and block size as one grid
using VBatchLauncher = void (*)(const VRec* const* recs, int n, cudaStream_t s);
constexpr int kMaxVBatch = 32;

// A recorded V-cycle launch and its place in the V-cycle: phase (-1 entry
// conversion, 0 descent and coarsest solve, 1 ascent, 2 exit conversion),
// level key (the level on the descent, 64 - level on the ascent, so that
// deeper levels come first) and step within the level.  Merging the records
// of several contexts by (phase, level key, step) keeps each context's order.
struct VRec {
    VBatchLauncher launch = nullptr;
    int grid = 0, block = 0;
    size_t smem = 0;
    int carve = -1;   // preferred shared-memory carveout (percent), -1: the driver's
    int phase = 0, level = 0, step = 0;
    VArgs a;
};

// When set, the V-cycle launchers append records here instead of launching;
// t_vkey is the position the next record gets (set by the V-cycle driver).
struct VKey {
    int phase = 0, level = 0, step = 0;
};
extern thread_local std::vector<VRec>* t_vrecord;
extern thread_local VKey t_vkey;

// Launch records that share body and block size as one grid per kMaxVBatch
// records (records of one step of different contexts: independent).
void launch_vrecords(const VRec* const* recs, int n, cudaStream_t s);

// V-cycle passes (see kernels.cu).  first: the first two forward colour passes
// from a zero guess (optionally zeroing the next level's right-hand side);
// pass: one colour, neighbours at positions >= jmax taken as zero;
// residual_restrict: coarse right-hand side from the
// residual of the rows of colour >= 1; prolong: x += omega P e on colour >= 1.
void launch_first(const DevLevel& L, const double* b, double* x, double* bc_zero, int nc,
                  cudaStream_t s);
void launch_first32(const DevLevel& L, const float* b, float* x, float* bc_zero, int nc,
                    cudaStream_t s);
void launch_pass(const DevLevel& L, int col, int jmax, const double* b, double* x, cudaStream_t s);
void launch_pass32(const DevLevel& L, int col, int jmax, const float* b, float* x, cudaStream_t s);
// fine level of the float32 V-cycle: the first pass forms b = r / s from the
// float64 residual (isq = 1/s), and the last pass over each colour also
// writes z = x / s in float64 (the V-cycle's output)
void launch_first32_from64(const DevLevel& L, const double* r, const double* isq, float* b,
                           float* x, float* bc_zero, int nc, cudaStream_t s);
void launch_pass32_to64(const DevLevel& L, int col, int jmax, const float* b, float* x,
                        double* z, const double* isq, cudaStream_t s);
void launch_residual_restrict(const DevLevel& L, const double* b, const double* x, double* r,
                              double* bc, cudaStream_t s);
void launch_residual_restrict32(const DevLevel& L, const float* b, const float* x, float* r,
                                float* bc, cudaStream_t s);
void launch_prolong(const DevLevel& L, const double* e, double* x, double omega, cudaStream_t s);
// blocks of a sweep launch: those that fit on the device at once
int sweep_grid(int lanes, int block);
// one smoothing sweep of plan P as one kernel (lane shapes, L.lpr lanes per row)
void launch_sweep(const DevLevel& L, const SweepPlan& P, const double* b, double* x, cudaStream_t s);
void launch_sweep32(const DevLevel& L, const SweepPlan& P, const float* b, float* x, cudaStream_t s);
void launch_prolong32(const DevLevel& L, const float* e, float* x, double omega, cudaStream_t s);
void launch_dense_gemv(int n, const double* M, const double* b, double* x, cudaStream_t s);
void launch_dense_gemv32(int n, const double* M, const float* b, float* x, cudaStream_t s);
// x = M b with a float32 matrix of row stride ld (a multiple of 4, zero
// beyond column n) and float32 sums (one warp per row)
void launch_dense_gemv_f32(int n, int ld, const float* M, const float* b, float* x, cudaStream_t s);
// out[i*ld + j] = (float) in[i*n + j] for j < n, 0 for n <= j < ld (setup_device.cu)
void to_float_padded_device(int n, int ld, const double* in, float* out, cudaStream_t s);
void launch_gather(int n, const int32_t* idx, const double* x, double* y, cudaStream_t s);
void launch_scatter(int n, const int32_t* idx, const double* x, double* y, cudaStream_t s);
void launch_to_scaled32(int n, const double* r, const double* isq, float* rhat, cudaStream_t s);
void launch_from_scaled32(int n, const float* zhat, const double* isq, double* z, cudaStream_t s);

void launch_cg_residual(const DevLevel& L, const double* b, const double* x, double* r,
                        CgWork& w, int mode, double* out, cudaStream_t s);
void launch_cg_spmv_pq(const DevLevel& L, const double* p, double* q, CgWork& w, cudaStream_t s);
void launch_cg_update(int n, double* x, double* r, const double* p, const double* q, CgWork& w,
                      cudaStream_t s);
void launch_cg_rz(int n, const double* r, const double* z, const double* zold, double* p,
                  CgWork& w, int mode, cudaStream_t s);
void launch_cg_p(int n, const double* z, double* p, double* zold, const CgWork& w,
                 cudaStream_t s);

// BiCGSTAB (level 0, float64, smoothing order), scalars in *bs (device):
// bi_start: r = b - A x, rt = r, start scalars; bi_direction: p = r (first
// iteration) or r + beta (p - w v); bi_spmv: y = A x with rt.y -> alpha
// (second = false) or s.y, y.y -> w (second = true); bi_half: s = r - alpha v,
// s.s -> half-step test; bi_update: x += alpha y + w z, r = s - w t, r.r, rt.r
// (x += alpha y only after a converged half step); bi_continue: the loop
// condition of a WHILE graph node.
void launch_bi_start(const DevLevel& L, const double* b, const double* x, double* r, double* rt,
                     CgWork& wk, BiScalars* bs, cudaStream_t s);
void launch_bi_direction(int n, const double* r, const double* v, double* p, const BiScalars* bs,
                         cudaStream_t s);
void launch_bi_spmv(const DevLevel& L, const double* x, double* y, const double* w, bool second,
                    CgWork& wk, BiScalars* bs, cudaStream_t s);
void launch_bi_half(int n, const double* r, const double* v, double* sv, CgWork& wk,
                    BiScalars* bs, cudaStream_t s);
void launch_bi_update(int n, double* x, const double* y, const double* z, const double* sv,
                      const double* t, double* r, const double* rt, CgWork& wk, BiScalars* bs,
                      cudaStream_t s);
void launch_bi_continue(cudaGraphConditionalHandle h, BiScalars* bs, cudaStream_t s);

// ---------------------------------------------------------------------------
// setup on the device (setup_device.cu)
// ---------------------------------------------------------------------------
struct DevCsr {
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t* rp = nullptr;
    int32_t* ci = nullptr;
    double* va = nullptr;
};

// G = P^T A P for the aggregation agg (device, original numbering).  The host
// receives G (rows sorted, sums in fine CSR order) in Gh; the device copy in
// Gd is allocated from arena.
void galerkin_device(const DevCsr& A, const HostCsr& Ah, const AggResult& agg, DevArena& arena,
                     DevCsr& Gd, HostCsr& Gh, cudaStream_t s);

// Build the smoothing-order device level from the original-order device
// matrix A and the permutation perm (original -> new position).
void build_level_device(const DevCsr& A, const HostCsr& Ah, const std::vector<int32_t>& perm,
                        DevArena& arena, DevLevel& L, cudaStream_t s);

// Decoupled aggregation (Alg. 4) on the device: the rows of A (original
// order) split into consecutive tiles of p.aggregation_tile rows, one warp per
// tile running Algorithm 1 (with the strength of connection) on the tile's
// induced submatrix; the same result as aggregate_tiled on the host.  Returns
// the map on the host.
AggResult aggregate_tiles_device(const DevCsr& A, const amg_params& p, cudaStream_t s);

// Dense inverse of the (original-order) coarsest matrix through a Cholesky
// factorisation of its lower triangle; returns false when a pivot is not
// positive.
bool dense_inverse_device(const DevCsr& A, double* Minv, cudaStream_t s);

// Minv_s = S Minv S, S = diag(sqrt(diag)): the inverse of S^-1 A S^-1.
void scale_inverse_device(int n, const double* diag, const double* Minv, double* Minv_s,
                          cudaStream_t s);

// float32 copies of a level scaled by S = diag(sqrt(A_ii)) (fine) and its
// coarse neighbour (for t32); coarse_diag is null on the coarsest level.
void build_level_fp32(DevLevel& L, const double* coarse_diag, DevArena& arena, cudaStream_t s);

}  // namespace amg

// State of a CG solve driven one step at a time (pcg_async_*).
struct AsyncCg {
    enum State { kIdle, kStarted, kIterating, kLooping, kFinishing, kDone };
    State state = kIdle;
    double tol = 0.0;
    int32_t maxit = 0;
    int status = 0;
    amg_solve_info info{};
    cudaEvent_t ev = nullptr;       // completes when the work of the current step is done
    double* rr_host = nullptr;      // pinned: ||b - A x||^2 of the final iterate
};

struct amg_ctx {
    amg_params p;
    int device = 0;
    cudaStream_t stream = nullptr;        // the context's own stream (all library work)
    cudaStream_t user_stream = nullptr;   // params.cuda_stream, ordered against `stream`
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // CUDA graphs of one CG iteration, [precision][flexible]: A = q = A p,
    // alpha, x/r update, status copy; B = z = B r, beta, p update
    cudaGraphExec_t graph_a[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t graph_b[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    std::vector<cudaGraphExec_t> graph_from[2];   // V-cycle from level l (profiling), per precision
    // the whole iteration loop as one graph with a device-side WHILE node,
    // [precision][flexible]; solve_graph_state 0 = not built yet, 1 = built,
    // -1 = the runtime refused it (the host-driven loop runs instead)
    cudaGraphExec_t graph_solve[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int solve_graph_state[2][2] = {{0, 0}, {0, 0}};
    cudaStream_t stream_body = nullptr;   // capture stream of the loop body
    bool solve_graph_plain = false;       // the loop graphs were built without launch overlap
    int32_t last_device_loop = 0;         // the last PCG solve ran its loop on the device
    bool use_graphs = true;
    amg::DevArena mem;
    std::vector<amg::HostLevel> hl;
    std::vector<amg::DevLevel> dl;
    int32_t nL = 0;                   // coarsest size
    double* Ainv = nullptr;           // [nL x nL] inverse of the coarsest matrix
    double* Ainv_s = nullptr;         // [nL x nL] inverse of the scaled coarsest matrix
    float* Ainv_s32 = nullptr;        // its float32 copy, rows of ld32 floats (coarsest_fp32 only)
    int ld32 = 0;                     // nL rounded up to a multiple of 4
    double* isq0 = nullptr;           // [n] 1 / sqrt(A_ii) of level 0 (FP32 entry/exit)
    int32_t* perm0 = nullptr;         // [n] device copy of the level-0 order: caller index -> position
    // level-0 CG vectors, smoothing order
    double *x = nullptr, *r = nullptr, *z = nullptr, *zold = nullptr, *pv = nullptr,
           *q = nullptr, *bb = nullptr;
    amg::CgWork work;
    amg::PcgScalars* sc_host = nullptr;   // pinned mirror of *work.sc
    double* norm_dev = nullptr;
    int precision = AMG_FP64;
    int flexible = 0;
    bool fp32_ready = false;
    // launch shape (DevLevel::lpr) of every level but the coarsest, per
    // precision, and whether the autotuner has chosen them
    std::vector<int32_t> shapes[2];
    bool tuned[2] = {false, false};
    amg_summary summary{};
    std::vector<amg_level_info> linfo;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    amg::Profiler prof;
    AsyncCg acg;
    // BiCGSTAB vectors (level 0, smoothing order), allocated on first use
    double *rt = nullptr, *bv = nullptr, *by = nullptr, *bs = nullptr, *bt = nullptr;
    // sweep plans by (level, lanes + 16 x block): the pre- and post-smoother
    std::map<std::pair<int, int>, std::pair<amg::SweepPlan, amg::SweepPlan>> sweep_plans;
    // the V-cycle of each precision as launch records (batched serving)
    std::vector<amg::VRec> vrec[2];
    bool vrec_ok[2] = {false, false};
    amg::BiScalars* bsc = nullptr;        // BiCGSTAB scalars (device)
    amg::BiScalars* bsc_host = nullptr;   // pinned mirror
    cudaGraphExec_t graph_bi[2] = {nullptr, nullptr};      // BiCGSTAB loop, per precision
    int bi_graph_state[2] = {0, 0};       // 0 not built, 1 built, -1 refused

    amg_ctx() = default;
    amg_ctx(const amg_ctx&) = delete;
    amg_ctx& operator=(const amg_ctx&) = delete;
    ~amg_ctx() {
        if (sc_host) amg::pinned_free(sc_host);
        if (acg.rr_host) amg::pinned_free(acg.rr_host);
        if (bsc_host) amg::pinned_free(bsc_host);
        for (cudaGraphExec_t g : graph_bi)
            if (g) cudaGraphExecDestroy(g);
        if (acg.ev) cudaEventDestroy(acg.ev);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (cudaEvent_t e : prof.events) cudaEventDestroy(e);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                if (graph_a[a][b]) cudaGraphExecDestroy(graph_a[a][b]);
                if (graph_b[a][b]) cudaGraphExecDestroy(graph_b[a][b]);
                if (graph_solve[a][b]) cudaGraphExecDestroy(graph_solve[a][b]);
            }
        for (int a = 0; a < 2; ++a)
            for (cudaGraphExec_t g : graph_from[a])
                if (g) cudaGraphExecDestroy(g);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        mem.release();   // stream-ordered frees, before the stream goes away
        if (stream) {
            cudaStreamSynchronize(stream);
            cudaStreamDestroy(stream);
        }
        if (stream_body) cudaStreamDestroy(stream_body);
    }
};

namespace amg {
// CG driven one step at a time on a context's own stream (solver.cu); the
// launches, and so the results, are those of amg_pcg_solve.  begin expects the
// right-hand side in c->bb and the initial guess in c->x (smoothing order).
// step never blocks: 0 = the previous step's work is still running, 1 = the
// next step was issued, 2 = the solve has finished and c->acg.info is final.
void pcg_async_begin(amg_ctx* c, double tol, int32_t maxit);
int pcg_async_step(amg_ctx* c);
// The stepping split around the preconditioner (batched serving): poll
// returns 0 busy, 1 issued the end of the solve, 2 finished, 3 needs
// z = B r on c->r (first: the first direction); resume issues the rest of
// the iteration after the caller has ordered z = B r before it.
int pcg_async_poll(amg_ctx* c, bool* first);
void pcg_async_resume(amg_ctx* c, bool first);
// z = B r on the context's level-0 vectors (c->r -> c->z) on its own stream
void precondition_context(amg_ctx* c);
// z = B r for the contexts cs[0..n), their V-cycles merged step by step into
// shared launches on stream s (records are built on first use)
void batched_precondition(amg_ctx* const* cs, int n, cudaStream_t s);
}  // namespace amg
