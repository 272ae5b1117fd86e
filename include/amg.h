/*
 * amg.h -- C ABI of libamg: aggregation-based algebraic multigrid as a
 * preconditioner for conjugate gradients on one NVIDIA GB300 (sm_103a).
 *
 * Method: Blatt, Ippisch & Bastian, "A Massively Parallel Algebraic
 * Multigrid Preconditioner based on Aggregation for Elliptic Problems with
 * Heterogeneous Coefficients" (arXiv:1209.0960).
 *   - problem statement A x = b, A symmetric positive definite, from the
 *     discretisation of div(K grad u) = f: Sec. 2, Eq. (model), Eq. (ls);
 *   - strength of connection: Sec. 2.1, Eq. (symmetric_strong1/2);
 *   - greedy aggregation: Sec. 2.1, Algorithms 1-3;
 *   - piecewise-constant prolongation and Galerkin coarse operator with the
 *     over-correction factor omega: Sec. 2.1, Eq. (prolongation) and the
 *     coarse-matrix formula after it;
 *   - V-cycle with one symmetric Gauss-Seidel step pre and post and a direct
 *     coarsest solve: Sec. 2 and Sec. 5; stopping on a relative residual
 *     reduction: Sec. 5.
 *
 * Conventions for every entry point:
 *   - Return value: AMG_OK (0) on success, a negative AMG_E* code on error
 *     (AMG_PENDING > 0 only from amg_poll).  amg_last_error() returns a
 *     thread-local message for the last failure on the calling thread.
 *     No C++ exception ever crosses this interface.
 *   - Matrices are CSR with int32 row pointers and column indices and
 *     float64 values, square, columns sorted and unique within each row,
 *     diagonal stored and positive, symmetric pattern and values.  The
 *     pattern is always checked; with the environment variable AMG_CHECK
 *     set (to anything but 0) amg_setup and amg_aggregate also require
 *     A_ij == A_ji exactly and return AMG_EINVAL naming the first entry that
 *     differs.
 *   - Inputs are borrowed for the duration of the call; the library copies
 *     what it keeps.  Outputs are allocated by the caller.
 *   - "device" pointers are CUDA device (or managed) memory on the device
 *     that was current when the context was created; "host" pointers are
 *     ordinary or pinned host memory.
 *   - All GPU work of a context is ordered on params.cuda_stream.  Calls
 *     that return results to the host synchronise that stream; amg_vcycle
 *     does not (its output is ready when the stream reaches that point).
 *   - Vectors passed to the library use the caller's row numbering.
 *   - Threads: different contexts may be used from different threads at the
 *     same time (the server does so); one context must not be used by two
 *     threads at once.  Setup, aggregation and colouring calls are
 *     reentrant.  The process-wide state (the tuned-shape cache, kernel
 *     attributes) is guarded internally.
 */
#ifndef AMG_H
#define AMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMG_OK 0
#define AMG_PENDING 1        /* amg_poll: request not finished yet */
#define AMG_EINVAL (-1)      /* malformed input or parameters */
#define AMG_ENOMEM (-2)      /* device or host allocation failed / refused */
#define AMG_ENOTSPD (-3)     /* coarsest pivot <= 0 or p.Ap <= 0 in CG */
#define AMG_ENOTCONV (-4)    /* maxit reached before the tolerance */
#define AMG_ETIMEOUT (-5)    /* a bounded device-side wait gave up; the context must then be
                                freed (copies may have been in flight, dependency counters
                                are behind) and the system set up again */
#define AMG_ECUDA (-6)       /* a CUDA runtime call failed */
#define AMG_ENOTFOUND (-7)   /* unknown ticket */
#define AMG_ERANGE (-8)      /* checked build: a kernel met an index outside its range (the
                                access was skipped); the hierarchy is corrupt */
#define AMG_ENONFINITE (-9)  /* a NaN or infinity in a dot product of the Krylov iteration */

#define AMG_FP64 0           /* every step in float64 */
#define AMG_FP32_IN_FP64 1   /* float32 V-cycle inside float64 CG */

/* or'ed into amg_set_level_shape's lanes_per_row (1, 2, 4 or 8): run each
 * smoothing sweep of the level (the pre- and the post-smoother) as one
 * dependency-driven kernel instead of one launch per colour pass */
#define AMG_SHAPE_SWEEP 0x100

typedef struct amg_ctx amg_ctx;

typedef struct {
    int32_t n;                /* rows = columns */
    int32_t nnz;              /* stored entries, = row_ptr[n] */
    const int32_t *row_ptr;   /* [n+1] */
    const int32_t *col;       /* [nnz], sorted within each row */
    const double *val;        /* [nnz] */
    int32_t on_device;        /* 1: the three arrays are device pointers */
} amg_csr;

/* Setup and solve parameters.  amg_params_default fills the documented
 * reading of the paper's unspecified constants. */
typedef struct {
    double delta;             /* strong-edge threshold, Eq. (symmetric_strong2); default 1/3 */
    double beta;              /* isolated-vertex threshold, Sec. 2.1 (b); default 1e-5 */
    double omega;             /* over-correction of the coarse correction, Sec. 2.1; default 1.6 */
    int32_t s_min;            /* Algorithm 1 minimum aggregate size; default 2^dim */
    int32_t s_max;            /* Algorithm 1 maximum aggregate size; default 3*2^(dim-1) */
    int32_t d_max;            /* Algorithm 2 diameter limit; default dim */
    int32_t coarsen_target;   /* stop coarsening at <= this many rows; default 5000 */
    int32_t max_levels;       /* default 20 */
    int32_t dense_cap;        /* largest coarsest level solved densely; default 8192 */
    double min_coarsen_rate;  /* stop when n_l / n_{l+1} < this; default 1.2 */
    int32_t precision;        /* AMG_FP64 or AMG_FP32_IN_FP64 */
    int32_t flexible_cg;      /* 1: flexible beta = r.(z - z_old) / rho; 0 or -1 (default):
                                 standard beta in both precisions (the float32
                                 V-cycle is symmetric up to rounding; measured on four
                                 workloads, flexible beta saved no iteration) */
    void *cuda_stream;        /* cudaStream_t for all work; NULL = default stream */
    int32_t launch_overlap;   /* 1 (default): consecutive solve kernels use programmatic
                                 dependent launch (a kernel starts while its predecessor
                                 drains and reads only setup-time data until the
                                 predecessor has finished); 0: plain stream order.
                                 Results are identical either way. */
    int32_t aggregation_tile; /* 0 (default): Algorithm 1 over the whole level on one host
                                 thread.  > 0: decoupled aggregation (Alg. 4): the rows of a
                                 level split into consecutive tiles of this many rows, each
                                 aggregated by Algorithm 1 on its own induced submatrix
                                 (edges leaving the tile dropped), aggregates numbered tile
                                 by tile.  A different hierarchy, built in parallel. */
    int32_t aggregation_device; /* with aggregation_tile > 0: 1 = the tiles run on the GPU
                                 (one warp per tile), 0 = on the host threads.  Same
                                 result either way. */
    int32_t host_threads;     /* host threads of the tiled aggregation (aggregation_tile > 0,
                                 aggregation_device = 0); 0 (default): one per host core,
                                 at most 64.  The map does not depend on it. */
    int32_t coarsest_fp32;    /* with AMG_FP32_IN_FP64: 1 applies the coarsest-level inverse
                                 (computed in float64 from the float64 Cholesky factor) as
                                 a float32 matrix with float32 sums, like the rest of the
                                 float32 V-cycle; 0 (default): the float64 matrix. */
    int32_t device_loop;      /* 1 (default): amg_pcg_solve (and a server's solves) run the
                                 iteration loop as one CUDA graph with a device-side WHILE
                                 node (the loop condition is set on the device after each
                                 update; no iteration waits for the host).  0: the host
                                 launches each iteration and reads the residual back.  Same
                                 launches in the same order, so results are identical. */
    int32_t autotune;         /* 0 (default): launch shapes of the smoother and residual
                                 kernels from fixed rules on the level's row lengths.
                                 1: amg_setup times each candidate shape per level (the
                                 V-cycle from that level, replayed as a CUDA graph in the
                                 context's precision) and keeps the fastest; choices are
                                 cached per process by level signature (precision, size
                                 class, slice width, mean row length, colours), so later
                                 setups of similar levels reuse them.  Shapes change the
                                 order of floating-point sums only. */
} amg_params;

typedef struct {
    int32_t status;           /* AMG_OK, AMG_ENOTCONV or AMG_ENOTSPD */
    int32_t iterations;       /* CG iterations performed */
    double rel_residual;      /* recursively updated ||r_k|| / ||r_0|| */
    double true_rel_residual; /* ||b - A x|| / ||b - A x_0||, recomputed at the end */
    double solve_ms;          /* device time of the whole solve (CUDA events) */
    int32_t device_loop;      /* 0: the host drove the iterations; 1: they ran as a
                                 device-side graph loop; 2: the same in plain stream
                                 order (the runtime refused launch overlap there) */
} amg_solve_info;

typedef struct {
    int32_t n;                /* rows of this level */
    int32_t nnz;              /* stored entries including the diagonal */
    int32_t n_coarse;         /* rows of the next level (0 on the coarsest) */
    int32_t ncolours;         /* colours of the smoother ordering (0 on the coarsest) */
    int32_t max_agg_size;     /* largest aggregate built on this level */
    int32_t n_isolated;       /* isolated vertices, Sec. 2.1 (b) */
    int32_t n_dirichlet;      /* rows without a non-zero off-diagonal */
    double vcycle_bytes_fp64; /* modelled DRAM bytes of this level per FP64 V-cycle */
    double vcycle_bytes_fp32; /* same for the FP32 V-cycle (coarsest inverse at 4 bytes
                                 an entry with coarsest_fp32) */
    int32_t lanes_per_row;    /* launch shape of the level's smoother and residual kernels:
                                 0 = one row per thread with the matrix slices staged in
                                 shared memory, else 1, 2, 4 or 8 lanes per row */
    int32_t threads_per_block; /* threads per block of those kernels with lanes_per_row >= 1
                                 (256, or 128 when the autotuner chose it) */
    int32_t sweep;            /* 1: each smoothing sweep of the level runs as one
                                 dependency-driven kernel (AMG_SHAPE_SWEEP): the colour
                                 passes are cut into items of threads_per_block /
                                 lanes_per_row rows, and an item starts as soon as the items
                                 of earlier passes it reads or overwrites have finished;
                                 same arithmetic as one launch per pass */
    int32_t compact;          /* 1: the staged kernels (lanes_per_row 0) read a copy of the
                                 level's off-diagonal entries in 32-row slices padded only
                                 to each slice's longest row; chosen at setup where the
                                 common width (the level's longest row) pads more than a
                                 tenth over that.  0: they read the common-width slices */
    int64_t staged_entries;   /* entries (index + value) that layout holds, padding
                                 included: one pass over every row stages this many */
    int32_t carveout;         /* preferred shared-memory carveout of the staged kernels, in
                                 percent of the SM's maximum shared memory (the rest of the
                                 unified L1/shared array caches the neighbour gathers);
                                 -1: the driver's choice */
} amg_level_info;

typedef struct {
    int32_t num_levels;
    int32_t coarsest_n;
    double operator_complexity;   /* sum_l nnz_l / nnz_0 */
    double host_setup_ms;         /* strength, aggregation, colouring, all levels (the
                                     aggregation on the device when aggregation_device = 1) */
    double gpu_galerkin_ms;       /* Galerkin products (device, all levels) */
    double gpu_other_ms;          /* reordering, coarsest factorisation, FP32 copies */
    double total_setup_ms;        /* wall time of amg_setup */
    double vcycle_bytes_fp64;     /* sum of the per-level figures */
    double vcycle_bytes_fp32;
    double pcg_iter_bytes_fp64;   /* modelled DRAM bytes per CG iteration incl. V-cycle */
    double pcg_iter_bytes_fp32;
    double aggregation_ms;        /* strength and aggregation alone, all levels (part of
                                     host_setup_ms) */
    double autotune_ms;           /* launch-shape tuning (part of gpu_other_ms; 0 when
                                     autotune = 0 or every level came from the cache) */
    double coarsest_inverse_ms;   /* Cholesky factorisation and explicit inverse of the
                                     coarsest level (part of gpu_other_ms) */
} amg_summary;

/* Per-kernel-class record of the profiler (amg_profile_*). */
typedef struct {
    char name[32];            /* kernel class, e.g. "gs_level0" */
    int32_t launches;         /* launches recorded since the profiler was enabled */
    double total_ms;          /* sum of their CUDA-event durations */
    double bytes;             /* sum of their modelled (algorithmic) DRAM bytes */
} amg_kernel_stat;

/* Fill *p with the defaults for a problem of spatial dimension dim (1-3).
 * Returns AMG_EINVAL for p == NULL or dim outside 1..3. */
int amg_params_default(amg_params *p, int32_t dim);

/* Build the hierarchy (Sec. 2.1; Algorithm 1 per level, then the Galerkin
 * product per level on the GPU, then the dense factorisation of the coarsest
 * level).  Strength, aggregation and colouring run on the host; the level
 * matrices, the reordering for the smoother and the coarsest inverse are
 * computed on the GPU.  *out receives a context owning all device memory.
 * Errors: AMG_EINVAL (bad CSR: unsorted/duplicate columns, missing or
 * non-positive diagonal, asymmetric pattern, asymmetric values under
 * AMG_CHECK; bad params; coarsest level
 * larger than dense_cap), AMG_ENOTSPD (coarsest pivot <= 0), AMG_ENOMEM,
 * AMG_ECUDA.  On error *out is set to NULL and nothing leaks. */
int amg_setup(const amg_csr *A, const amg_params *p, amg_ctx **out);

/* Select the arithmetic of later solves: AMG_FP64 or AMG_FP32_IN_FP64, and
 * the CG variant (flexible_cg as in amg_params).  The first switch to
 * AMG_FP32_IN_FP64 builds the scaled float32 level copies (S^-1 A S^-1,
 * S = diag(sqrt(A_ii)), per level).  Errors: AMG_EINVAL, AMG_ENOMEM. */
int amg_set_precision(amg_ctx *c, int32_t precision, int32_t flexible_cg);

/* z = B r for one V(1,1)-cycle B of the hierarchy, zero initial guess
 * (Sec. 2; one symmetric Gauss-Seidel step pre and post in the multicolour
 * ordering, residual restriction by aggregate sums, coarse correction
 * prolongated with factor omega, dense solve on the coarsest level).
 * r_dev, z_dev: device float64 [n] in the caller's numbering; they may not
 * alias.  Uses the context's current precision.  Asynchronous on the
 * context stream.  Errors: AMG_EINVAL (NULL), AMG_ECUDA. */
int amg_vcycle(amg_ctx *c, const double *r_dev, double *z_dev);

/* Preconditioned CG with one V-cycle per iteration until
 * ||b - A x_k|| <= tol ||b - A x_0|| (Sec. 5 stopping rule) or maxit
 * iterations.  b_dev: device float64 [n]; x_dev: device float64 [n], the
 * initial guess on entry and the solution on exit.  info may be NULL.
 * Returns AMG_OK on convergence, AMG_ENOTCONV at maxit (x holds the last
 * iterate), AMG_ENOTSPD when p.Ap <= 0, AMG_EINVAL, AMG_ECUDA.
 * Synchronises the context stream. */
int amg_pcg_solve(amg_ctx *c, const double *b_dev, double *x_dev, double tol,
                  int32_t maxit, amg_solve_info *info);

/* Preconditioned BiCGSTAB (the Krylov method of the paper's experiments,
 * Sec. 5) with the same V-cycle, two V-cycles per iteration; arguments,
 * stopping rule and errors as amg_pcg_solve (a half iteration that meets the
 * tolerance counts as an iteration).  A breakdown (rt.r, rt.v or t.t zero)
 * returns AMG_ENOTCONV with the reason in amg_last_error(). */
int amg_bicgstab_solve(amg_ctx *c, const double *b_dev, double *x_dev, double tol,
                       int32_t maxit, amg_solve_info *info);

/* As amg_pcg_solve with host buffers: copies b and x_0 to the device,
 * solves, copies x back (all on the context stream; pinned buffers make the
 * copies asynchronous DMA).  info->solve_ms includes the copies. */
int amg_pcg_solve_host(amg_ctx *c, const double *b_host, double *x_host, double tol,
                       int32_t maxit, amg_solve_info *info);

/* As amg_pcg_solve_host from the initial guess x_0 = 0: x_host is only
 * written (no x_0 is read or copied to the device), so one vector fewer
 * crosses to the device.  Results are those of amg_pcg_solve_host with
 * x_host zeroed.  Errors as amg_pcg_solve. */
int amg_pcg_solve_host_zero_guess(amg_ctx *c, const double *b_host, double *x_host, double tol,
                                  int32_t maxit, amg_solve_info *info);

/* ||b - A x||_2 for the level-0 matrix of the context, reduced in a fixed
 * order (deterministic).  b_dev, x_dev: device float64 [n] in the caller's
 * numbering.  *out_norm is written on the host (synchronises the stream).
 * Uses device scratch owned by the context.  Errors: AMG_EINVAL, AMG_ECUDA. */
int amg_residual_norm(amg_ctx *c, const double *b_dev, const double *x_dev, double *out_norm);

/* Self-test of the library's failure detection.  The staged fine-level
 * kernels wait for their shared-memory copies on an mbarrier with a bounded
 * number of polls; when the limit runs out they record AMG_ETIMEOUT in the CG
 * status word and return instead of hanging.  This call runs that same wait
 * in a one-block kernel against an mbarrier whose copies are never issued,
 * with at most `polls` polls (0: the kernels' own limit, 2^18, about one second
 * on GB300), on
 * cuda_stream (NULL: the legacy default stream).  *status receives what the
 * kernel recorded (AMG_ETIMEOUT when the wait ran out) and *elapsed_ms the
 * kernel's time.  Nothing faults or hangs and the device stays usable.
 * Errors: AMG_EINVAL (null outputs, polls < 0), AMG_ECUDA. */
int amg_selftest_bounded_wait(int64_t polls, void *cuda_stream, int32_t *status,
                              double *elapsed_ms);

/* ||b - A x||_2 for a CSR matrix A held in device memory (A->on_device = 1),
 * with b_dev, x_dev device float64 [n]; the result is written to the device
 * double *norm_dev, asynchronously on cuda_stream (NULL = default stream).
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory where they need a residual check -- a loop that
 * shares the GPU with other streams and cannot afford the device-wide
 * synchronisation cudaMalloc / cudaFree may cause, an allocator hook or
 * callback that must not re-enter the allocator, or a program whose device
 * memory is entirely owned by a pool it does not control.  It needs no
 * context and calls no allocator: the partial sums of its deterministic
 * reduction live in a fixed device array of 512 KiB that every GPU loading
 * the library keeps until exit, which limits n to 16,777,216 rows (larger n:
 * AMG_EINVAL).  The first call on each device looks up that array's address
 * and caches it for the life of the process (a device reset invalidates the
 * cache).  All calls share
 * the array and it keeps the last call's contents (each call clears its
 * counter first): calls that overlap on the GPU race and must be serialised
 * by the caller.  Every pointer is checked with cudaPointerGetAttributes: host
 * memory, or device memory of another device, is AMG_EINVAL before anything
 * is launched.
 * Errors: AMG_EINVAL (null, host or other-device pointers, n out of range),
 * AMG_ECUDA. */
int amg_residual_norm_noalloc(const amg_csr *A, const double *b_dev, const double *x_dev,
                              double *norm_dev, void *cuda_stream);

/* Hierarchy description: *summary (may be NULL) and up to cap level records
 * (levels may be NULL when cap == 0).  Returns the number of levels
 * (>= 1) or a negative error. */
int amg_hierarchy_info(const amg_ctx *c, amg_summary *summary, amg_level_info *levels,
                       int32_t cap);

/* Host copies of level l in the caller's (level-0) or aggregate-id (l >= 1)
 * numbering, for parity checks: row_ptr [n+1], col [nnz], val [nnz] of the
 * level matrix (the Galerkin product for l >= 1, bit-identical to what the
 * GPU computed); agg [n] (coarse index of every row, -1 for rows left out)
 * and colour [n] for every level but the coarsest.  Any output may be NULL.
 * Errors: AMG_EINVAL (l out of range, or agg/colour requested on the
 * coarsest level). */
int amg_export_level(const amg_ctx *c, int32_t l, int32_t *row_ptr, int32_t *col,
                     double *val, int32_t *agg, int32_t *colour);

/* Launch shape of level l's smoother and residual kernels (0 <= l < number of
 * levels - 1; the coarsest level is the dense solve).  lanes_per_row: 0 = one
 * row per thread with the slices staged in shared memory (levels where the
 * entries of any 8 consecutive 32-row slices, in the layout those kernels read,
 * take at most 96 KB as index and value: with the padded slices, a longest row
 * of at most 32 off-diagonals), or 1, 2, 4, 8 lanes per row, optionally
 * or'ed with AMG_SHAPE_SWEEP (levels of at most 2^20 rows that are not
 * two-colour levels with the fused residual): each smoothing sweep then runs
 * as one kernel whose blocks wait, with bounded polls, only for the earlier
 * colour-pass blocks they depend on (planned on the host from the level's
 * graph at the first use of a block size).  threads_per_block: 256 or 128 for
 * lanes_per_row >= 1 (0 means 256; the staged kernels always use 256).
 * Results differ only in the order of floating-point sums (a sweep gives the
 * same values as the pass-per-launch kernels of its lanes and block size).
 * The CUDA graphs of the context are rebuilt on the next solve.  Errors:
 * AMG_EINVAL (l, lanes_per_row or threads_per_block out of range, 0 lanes on a
 * level whose tile does not fit, a sweep where it is not allowed). */
int amg_set_level_shape(amg_ctx *c, int32_t l, int32_t lanes_per_row, int32_t threads_per_block);

/* Preferred shared-memory carveout of level l's staged kernels (the level's
 * shape must have lanes_per_row 0): percent (0 .. 100) of the SM's maximum
 * shared memory to configure for those launches, the rest of the unified
 * L1/shared array serving as L1 cache for the neighbour gathers; -1 restores
 * the driver's choice.  A hint: the driver still configures at least what one
 * block needs.  Fewer resident blocks and a larger L1 can be faster on levels
 * whose passes gather many neighbour values; results are identical for every
 * value.  The autotuner chooses it per level among a few values.  The CUDA
 * graphs of the context are rebuilt on the next solve.  Errors: AMG_EINVAL (l
 * or percent out of range, a level without the staged kernels). */
int amg_set_level_carveout(amg_ctx *c, int32_t l, int32_t percent);

/* Aggregation of one level, exactly as amg_setup runs it (Sec. 2.1): strength
 * of connection (Eq. symmetric_strong1/2) and Algorithm 1 with Algorithms 2
 * and 3, the singleton merge and the isolated-vertex phase, on the matrix
 * graph of A -- or, with p->aggregation_tile > 0, on each tile's induced
 * submatrix (Alg. 4).  A must be a host matrix (on_device = 0).  agg: host
 * int32 [n], receives the coarse index of every row in completion order (-1
 * for rows left out: no non-zero off-diagonal inside the graph aggregated);
 * *n_coarse receives the number of aggregates.  Runs on the host and needs no
 * GPU, except with aggregation_tile > 0 and aggregation_device = 1, where the
 * tiles run on the GPU on p->cuda_stream (the map is the same).  Errors:
 * AMG_EINVAL (bad CSR or parameters), AMG_ECUDA / AMG_ENOMEM (device path). */
int amg_aggregate(const amg_csr *A, const amg_params *p, int32_t *agg, int32_t *n_coarse);

/* Multicolour ordering of the smoother (the GPU form of the Gauss-Seidel
 * smoother of Sec. 3.2), as amg_setup forms it on every level: the greedy
 * colouring of the matrix graph of A (host matrix) in ascending row order
 * (smallest colour not used by an already coloured neighbour), replaced by the
 * DSATUR colouring (next row: most distinct colours among its neighbours, then
 * more neighbours, then the lower index) when that needs fewer colours.
 * colour: host int32 [n]; *ncolours receives the number of colours.  Needs no
 * GPU.  Errors: AMG_EINVAL. */
int amg_colour(const amg_csr *A, int32_t *colour, int32_t *ncolours);

/* Profiler.  enable == 1 clears the records and brackets every later kernel
 * launch of the context with CUDA events on the context stream (the solve
 * then launches kernels one by one instead of through CUDA graphs, and each
 * launch costs a few microseconds more).  enable == 2 keeps the graphs and
 * brackets each graph launch instead ("graph_cg_part": SpMV and updates,
 * "graph_vcycle_part": V-cycle and direction update), and after every solve
 * replays the V-cycle from each level l >= 1 ten times ("graph_from_level_l").
 * enable == 0 stops recording.  Errors: AMG_EINVAL. */
int amg_profile_enable(amg_ctx *c, int32_t enable);

/* Synchronises the context stream and fills up to cap records, one per kernel
 * class that launched; returns the number of classes (>= 0) or an error. */
int amg_profile_read(amg_ctx *c, amg_kernel_stat *stats, int32_t cap);

/* Release every resource of the context (NULL is allowed). */
int amg_free(amg_ctx *c);

/* ---------------------------------------------------------------------------
 * Serving: many independent solves A_k x_k = b_k with continuous batching.
 *
 * A server owns a scheduling thread and a pool of setup threads.  Submitted
 * requests wait in FIFO order until a slot and enough device memory are free
 * (admission by HBM: each request reserves an estimate of its hierarchy and
 * Krylov state, replaced by the actual size after setup).  An admitted
 * request is set up on a setup thread (host aggregation, then the GPU
 * Galerkin products on the request's own stream) and then joins the running
 * set; the scheduling thread advances every running solve one CG iteration
 * at a time (CUDA graphs per request, on per-request streams, never blocking
 * on any of them), so the iterations and V-cycles of all in-flight solves
 * overlap on the device, new requests are admitted as soon as a finished one
 * frees its slot, and a result is exactly the one amg_setup + amg_pcg_solve
 * give for the same request alone.  The method per request is the one of the
 * rest of this interface (Sec. 2, Sec. 5).
 * ------------------------------------------------------------------------- */
typedef struct amg_server amg_server;

typedef struct {
    amg_params params;        /* setup and solve parameters of every request
                                 (cuda_stream is ignored: each request gets its
                                 own stream) */
    int32_t max_slots;        /* most requests admitted at once; default 32 */
    int32_t setup_threads;    /* host threads running request setup; default 4 */
    int32_t maxit;            /* CG iteration cap per request; default 500 */
    double hbm_budget_bytes;  /* device memory the admitted requests may reserve;
                                 <= 0: 80 % of the free device memory at creation */
    int32_t batch_vcycles;    /* 1 (with params.device_loop = 0): every scheduler tick runs
                                 the V-cycles of all requests whose next CG step needs one
                                 as shared launches, level by level (one launch per colour
                                 pass, residual, restriction, prolongation and coarsest
                                 solve over all of them); each request's rows are computed
                                 exactly as in its own V-cycle.  0 (default, measured
                                 faster on the serving stream): every request issues its
                                 own launches on its own stream. */
} amg_server_params;

/* Timings of one request (host steady clock, milliseconds). */
typedef struct {
    double queue_ms;          /* submit -> admitted */
    double setup_ms;          /* admitted -> hierarchy ready */
    double solve_ms;          /* ready -> solution on the host */
    double total_ms;          /* submit -> solution on the host */
    double hbm_bytes;         /* device memory the request held */
} amg_request_times;

/* Server totals since creation. */
typedef struct {
    int64_t submitted, completed, failed;
    int32_t queued, running, peak_running;
    double hbm_reserved_bytes, hbm_budget_bytes;
    int64_t batched_vcycles;      /* batched V-cycle launch sequences issued */
    int64_t batched_requests;     /* request V-cycles they covered */
} amg_server_stats;

/* Defaults: batch_vcycles 0; params = amg_params_default(dim) with precision
 * AMG_FP32_IN_FP64 and a coarsening target of 1000 rows (the dense coarsest
 * factorisation is per-request setup work), device_loop 0 (the stepper
 * launches each iteration: measured faster with 32 solves sharing the GPU than
 * capturing a whole-loop graph per request), max_slots 32, setup_threads 4,
 * maxit 500, hbm_budget_bytes 0.  Errors: AMG_EINVAL. */
int amg_server_params_default(amg_server_params *p, int32_t dim);

/* Create a server on the current device and start its threads.
 * Errors: AMG_EINVAL (bad parameters), AMG_ECUDA. */
int amg_server_create(const amg_server_params *p, amg_server **out);

/* Queue the solve of A x = b to relative residual tol (x0 = 0).  A is a host
 * CSR matrix (on_device must be 0), b a host vector of A->n doubles; both are
 * copied before the call returns.  *ticket identifies the request.  Errors:
 * AMG_EINVAL (malformed matrix, tol < 0, server stopping). */
int amg_submit(amg_server *s, const amg_csr *A, const double *b, double tol, uint64_t *ticket);

/* Non-blocking.  AMG_PENDING while the request is queued, being set up or
 * solving.  Once it has finished: copies the solution (A->n doubles, caller
 * numbering) to x_out and the solve record to info and the timings to times
 * (each may be NULL), forgets the ticket and returns the request's status
 * (AMG_OK, AMG_ENOTCONV, AMG_ENOTSPD, AMG_ENOMEM, ...).  Unknown or already
 * collected tickets: AMG_ENOTFOUND. */
int amg_poll(amg_server *s, uint64_t ticket, double *x_out, amg_solve_info *info,
             amg_request_times *times);

/* Snapshot of the server's counters.  Errors: AMG_EINVAL. */
int amg_server_stats_read(amg_server *s, amg_server_stats *out);

/* Stop the threads (running solves finish first; queued requests are
 * dropped), release every resource.  NULL is allowed. */
int amg_server_destroy(amg_server *s);

/* ---------------------------------------------------------------------------
 * The checked build.  libamg_checked.so is the same library compiled with
 * AMG_DEVICE_CHECKS: every kernel of the solve tests each index it gathers
 * with (neighbour columns, restriction-list rows, aggregate indices) against
 * its range before use and records AMG_ERANGE in the solve's status word
 * instead of reading out of range; a solve then returns AMG_ERANGE.  It
 * stands in for a memory sanitizer on a GPU where none can run.  Both builds
 * stop a Krylov solve with AMG_ENONFINITE when a dot product is not finite.
 * ------------------------------------------------------------------------- */

/* 1 in the checked build, 0 in the regular one. */
int amg_device_checks(void);

/* Checked build only (AMG_EINVAL in the regular one): overwrite the column
 * index of the k-th stored off-diagonal entry of row `row` (level-l
 * numbering; l >= 1) with `col` on the device, to test that the checks catch
 * a corrupt hierarchy.  A column >= the level's rows is never dereferenced by
 * any kernel of either build (neighbours at positions beyond the pass bound
 * are skipped), so this cannot make a kernel read out of range.  The context
 * is corrupt afterwards: free it.  Errors: AMG_EINVAL (build, l, row, k, or
 * col < the level's rows). */
int amg_debug_set_column(amg_ctx *c, int32_t l, int32_t row, int32_t k, int32_t col);

/* Thread-local description of the last error on this thread ("" if none). */
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMG_H */
