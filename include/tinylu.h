/*
 * tinylu.h -- C ABI of the GB300 (sm_103a) tiny batched LU library.
 *
 * Solves very large batches of independent general dense systems
 * A_s x_s = b_s of dimension n <= 32 in IEEE binary64 by LU factorization
 * with partial pivoting (LUpp): PA = LU, then Ly = Pb and Ux = y
 * (paper Sec. 2.2).  The same solvers run inside a fused kernel that carries
 * each integration point's own Newton loop (paper Sec. 2.1 Eqs. 1-3 and
 * Algorithm 2).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every data pointer is a DEVICE pointer owned by the caller unless the
 *    call's comment says otherwise.  The library never frees caller memory.
 *  - Calls are asynchronous on `stream` (NULL = legacy default stream).
 *    Argument errors are detected on the host before any launch and return
 *    TL_ERR_INVALID_ARG synchronously; tl_last_bad_arg() then gives the
 *    1-based position of the offending argument, LAPACK style.  Nothing is
 *    thrown across the ABI.  A CUDA launch error returns TL_ERR_CUDA and
 *    tl_last_cuda_error() gives the cudaError_t value.
 *  - A handle is not thread-safe: use one handle per host thread.
 *  - Matrix entry (i,j) of system s (0-based) is stored
 *      TL_LAYOUT_PER_SYSTEM : A[s*n*n + j*n + i]   (column-major per system,
 *                                                    LAPACK convention of the
 *                                                    batched solvers, Sec. 3.1)
 *      TL_LAYOUT_INTERLEAVED: A[(j*n + i)*ld + s]   (batch-minor: consecutive
 *                                                    systems adjacent, the
 *                                                    coalescing layout of
 *                                                    Sec. 2.3)
 *    Vectors (b, x, one right-hand side) are b[s*n + i] or b[i*ld + s];
 *    pivots ipiv[s*n + k] or ipiv[k*ld + s]; info is always info[s].
 *    `ld` (ld_batch) must be >= batch for the interleaved layout and is
 *    ignored for the per-system layout.  All device pointers must be
 *    8-byte aligned (4-byte for int32 arrays).
 *  - Pivots follow LAPACK: ipiv[k] (1-based) is the row interchanged with
 *    row k at elimination step k.  The pivot row is the FIRST row of largest
 *    magnitude in the column (ties go to the smallest current row index).
 *  - Per-system info: 0 success; k+1 if the pivot of step k is exactly zero
 *    (the factorization still completes, no solve is attempted and x is set
 *    to NaN); -1 if an entry of A is NaN or +-Inf (nothing is factored,
 *    ipiv is the identity and x is NaN).
 *  - Arithmetic is binary64 throughout the factorization with one rounding
 *    per operation: multipliers l_ik = a_ik * RN(1/a_kk) (a_ik / a_kk when
 *    |a_kk| < DBL_MIN) and Schur updates fma(-l_ik, u_kj, a_ij), so the LU
 *    factors and the pivots are bit-identical to a sequential textbook
 *    right-looking elimination with those operations.
 */
#ifndef TINYLU_H
#define TINYLU_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TL_MAX_N 32

typedef struct tl_handle tl_handle;

typedef enum {
    TL_OK = 0,
    TL_ERR_INVALID_ARG = -1,   /* see tl_last_bad_arg()                     */
    TL_ERR_CUDA = -2,          /* see tl_last_cuda_error()                  */
    TL_ERR_NO_MEMORY = -3,     /* workspace could not be allocated          */
    TL_ERR_UNSUPPORTED = -4,   /* valid request the library does not support */
    TL_ERR_TIMEOUT = -5        /* a bounded device wait gave up             */
} tl_status;

typedef enum { TL_LAYOUT_PER_SYSTEM = 0, TL_LAYOUT_INTERLEAVED = 1 } tl_layout;

typedef enum { TL_PREC_FP64 = 0, TL_PREC_FP32_IR = 1 } tl_precision;

typedef enum { TL_LAW_NORTON = 0, TL_LAW_TANH = 1 } tl_law_id;

/* Per-point Newton status codes written by tl_newton_integrate. */
enum {
    TL_NEWTON_CONVERGED = 0,
    TL_NEWTON_MAX_ITER = 1,
    TL_NEWTON_SINGULAR = 2,
    TL_NEWTON_NONFINITE = 3
};

/*
 * Constitutive law descriptor for tl_newton_integrate.
 *   TL_LAW_NORTON: n must be 7; params = {E, nu, A, m, dt} (m a positive
 *     integer stored as double).  Implicit Euler of an isotropic-elastic,
 *     J2, Norton-viscoplastic law (the law class of Sec. 4.3); unknowns
 *     x = (de_el[6] in Mandel notation, dp).
 *   TL_LAW_TANH: n in 1..32; F(x) = A x + c .* tanh(x) - b per point;
 *     params unused.
 */
typedef struct {
    int32_t id;
    int32_t n;
    double params[6];
} tl_law;

/* Create a handle on the current CUDA device.  Allocates no device memory. */
tl_status tl_create(tl_handle **h);

/* Destroy a handle and release the workspace it owns (synchronizes it). */
tl_status tl_destroy(tl_handle *h);

/* Static, human-readable name of a status code.  Never NULL. */
const char *tl_status_string(tl_status s);

/* cudaError_t of the last TL_ERR_CUDA on this handle (0 if none). */
tl_status tl_last_cuda_error(tl_handle *h, int *err);

/* 1-based position of the argument rejected by the last TL_ERR_INVALID_ARG
 * on this handle (0 if none). */
int tl_last_bad_arg(tl_handle *h);

/*
 * tl_check_bounds_violations -- the bounds-checked build of the library
 * (libtinylu_checked.so: the C ABI of the fixed-size and ragged solves with
 * the shared-memory solvers compiled with -DTL_CHECK_BOUNDS) checks every
 * shared-memory index of the element-walk elimination and of the loads
 * into shared memory against its system's block; a violation is counted
 * and the access redirected inside the block (no trap, no fault).  This
 * call synchronizes the device and returns in *count (host) the violations
 * counted since the last call, then clears the counters.  The normal
 * library has no checks and returns TL_ERR_UNSUPPORTED.
 */
tl_status tl_check_bounds_violations(unsigned long long *count);

/*
 * tl_getrf_batched -- LUpp factorization in place (Sec. 2.2, PA = LU).
 *   n      1..32
 *   A      in: the batch of matrices; out: L (unit lower, strictly below the
 *          diagonal) and U, LAPACK getrf storage, in the given layout.
 *   ipiv   out: n pivots per system (same layout rules as a vector, int32).
 *   info   out: one int32 per system, see the conventions above.
 *   batch  >= 0 (0 is a no-op).
 */
tl_status tl_getrf_batched(tl_handle *h, int n, double *A, tl_layout layout, int64_t ld_batch,
                           int32_t *ipiv, int32_t *info, int64_t batch, cudaStream_t stream);

/*
 * tl_getrs_batched -- solve with the factors of tl_getrf_batched
 * (Sec. 2.2: Ly = Pb, Ux = y).
 *   nrhs   1..32 right-hand sides per system.
 *   LU, ipiv  as written by tl_getrf_batched (not modified).
 *   B      in: right-hand sides, out: solutions.  Per-system layout:
 *          B[s*n*nrhs + r*n + i] (column-major n x nrhs); interleaved:
 *          B[(r*n + i)*ld + s].
 *   Systems with a zero pivot produce Inf/NaN as the arithmetic gives
 *   (LAPACK getrs does not test for singularity either).
 */
tl_status tl_getrs_batched(tl_handle *h, int n, int nrhs, const double *LU, const int32_t *ipiv,
                           tl_layout layout, int64_t ld_batch, double *B, int64_t batch,
                           cudaStream_t stream);

/*
 * tl_gesv_batched -- fused factor + solve for one right-hand side
 * (Sec. 3.1, the gesv form of the batched solvers; the elimination carries b
 * along as an extra column so that Ly = Pb is formed during the
 * factorization).
 *   A       in, not modified.
 *   LU_out  nullable; if not NULL receives the getrf factors.
 *   b       in, not modified.  x out (may alias b).
 *   ipiv, info  out.
 * The back substitution multiplies by the reciprocals RN(1/u_ii) formed
 * during the factorization instead of dividing by u_ii; x therefore agrees
 * with a dividing substitution to within a few units in the last place per
 * step (well inside the normwise backward-error bound), while LU, ipiv and
 * the forward-substituted y are bit-identical to the sequential algorithm.
 */
tl_status tl_gesv_batched(tl_handle *h, int n, const double *A, double *LU_out, const double *b,
                          double *x, int32_t *ipiv, int32_t *info, tl_layout layout,
                          int64_t ld_batch, int64_t batch, cudaStream_t stream);

/*
 * tl_gesv_batched_tilepiv -- tl_gesv_batched with the tile-local pivoting of
 * the paper's Tiled solvers (Sec. 3.2; threshold 1e-10 in Sec. 4.1): the
 * pivot of step k is the first maximum over the rows of the diagonal tile
 * (rows k .. min(n, (k/tile + 1) tile) - 1), and over all rows k .. n-1
 * only when that maximum is below `threshold` in magnitude.  This is not
 * textbook partial pivoting: pivots, factors and x differ from
 * tl_gesv_batched whenever a step keeps an in-tile pivot that a full-column
 * search would not take (the stability cost the paper quantifies); tile 0
 * or tile >= n is textbook partial pivoting.  Arguments after threshold as
 * tl_gesv_batched (numbered 5..14).  Runs the shared-memory kernels.
 */
tl_status tl_gesv_batched_tilepiv(tl_handle *h, int n, int tile, double threshold, const double *A,
                                  double *LU_out, const double *b, double *x, int32_t *ipiv, int32_t *info,
                                  tl_layout layout, int64_t ld_batch, int64_t batch, cudaStream_t stream);

/*
 * tl_lupp_solve_batched -- ragged batch: system s has its own size n[s]
 * (1..32) and lives anywhere in the A / b / ipiv arrays (per-system
 * column-major storage at the given element offsets).
 *   n       device int32[batch]
 *   a_off   device int64[batch]: A_s starts at A + a_off[s]
 *   b_off   device int64[batch]: b_s at b + b_off[s] and x_s at x + b_off[s]
 *   piv_off device int64[batch]: ipiv_s at ipiv + piv_off[s]
 *   info    device int32[batch]
 *   prec    TL_PREC_FP64: binary64 LUpp of every system.
 *           TL_PREC_FP32_IR: mixed precision (iterative refinement, Langou
 *           et al. 2006; the paper factors in binary64 only): factor a
 *           binary32 copy of A_s, x = solve(b) in binary32, then up to 3
 *           corrections x += solve(r) with the residual r = b - A x formed
 *           in binary64, stopping once max|r_i| <= max|x_i| * ||A32||_inf *
 *           sqrt(n) * 2^-53 (a binary64 backward error).  ipiv then holds
 *           the binary32 pivots and info[s] = 0.  A system whose binary32
 *           copy is out of range, whose binary32 factor meets a pivot
 *           outside [FLT_MIN, Inf), whose solves overflow or whose residual
 *           has not met the test after 3 corrections is solved by the
 *           binary64 LUpp instead (x, ipiv and info exactly as with
 *           TL_PREC_FP64).
 *           Sizes routed to binary64 (tl_ragged_dispatch_set; by default
 *           n <= 20, where refinement measured slower) are solved by the
 *           binary64 LUpp directly.
 *   refine_steps  nullable device int32[batch], TL_PREC_FP32_IR only (not
 *           written with TL_PREC_FP64): corrections applied (0..3), or -1
 *           when the system was solved in binary64 (fallback, size routed
 *           to binary64, or n[s] invalid).
 * info[s] = -2 when n[s] is outside 1..32 (that system is skipped, its x
 * and ipiv are not written); otherwise as for tl_gesv_batched.
 * Systems are bucketed by n on the device in the handle's workspace (grown
 * on demand with cudaMalloc; a call that would need to grow it while the
 * stream is being captured returns TL_ERR_NO_MEMORY; 4 bytes per system,
 * 8 with TL_PREC_FP32_IR, plus 1 KiB) and, in the default mode, the binary64
 * solves of every size run in ONE persistent launch (warps take work items
 * of one size class from a device counter, largest n first; lanes per
 * system per n from the dispatch table's shared-memory ragged variant, see
 * tl_dispatch_set); with TL_PREC_FP32_IR the systems handed back go through
 * that binary64 launch afterwards.  No host synchronization.  batch must be
 * below 2^31.
 */
tl_status tl_lupp_solve_batched(tl_handle *h, int64_t batch, const int32_t *n, const int64_t *a_off,
                                const double *A, const int64_t *b_off, const double *b, double *x,
                                const int64_t *piv_off, int32_t *ipiv, int32_t *info,
                                tl_precision prec, int32_t *refine_steps, cudaStream_t stream);

/*
 * tl_ragged_set_mode -- how tl_lupp_solve_batched (and its no-allocation
 * form) runs the binary64 solves of a ragged batch:
 *   TL_RAGGED_PERSISTENT  one persistent launch over every size class
 *                         (default; Sec. 2.3 batching with the work of all
 *                         sizes fused into one kernel).
 *   TL_RAGGED_PER_SIZE    one launch per size class 1..32 with the per-n
 *                         kernels of tl_gesv_batched (the comparator of the
 *                         single launch).
 * Results are identical in both modes.  Other values: TL_ERR_INVALID_ARG.
 */
typedef enum { TL_RAGGED_PERSISTENT = 0, TL_RAGGED_PER_SIZE = 1 } tl_ragged_mode;
tl_status tl_ragged_set_mode(tl_handle *h, int mode);

/*
 * tl_lupp_solve_batched_noalloc -- the ragged solve of tl_lupp_solve_batched
 * (FP64 only) for callers that must not allocate device memory.  The paper
 * has no counterpart; this entry exists for the library's users.
 *
 * tl_lupp_solve_batched keeps its per-size index lists in a workspace the
 * handle grows with cudaMalloc, which also synchronizes the whole device and
 * frees the old buffer.  Callers that run under a device-memory budget owned
 * by someone else, latency-bound serving loops that must never stall the
 * device, and code that may not synchronize other GPU work cannot accept
 * that.  This call uses instead a fixed scratch array built into the
 * library: it never calls cudaMalloc, cudaFree or any allocating routine.
 *
 *   batch  at most TL_NOALLOC_MAX_BATCH systems; a larger batch returns
 *          TL_ERR_INVALID_ARG with tl_last_bad_arg() == 2 and launches
 *          nothing.  Other arguments and results as tl_lupp_solve_batched.
 *   The scratch array (TL_NOALLOC_MAX_BATCH + 256 int32, about 4 MiB) exists
 *   on every GPU that loads the library, from load until process exit.
 *   The first call with a given device current looks up the array's device
 *   address (cudaGetSymbolAddress) and caches it; make that first call
 *   before any stream capture on that device.  The cached address belongs
 *   to that device's context: after cudaDeviceReset (or anything else that
 *   destroys the primary context) the library must be unloaded and loaded
 *   again before this entry is called on that device.
 *   Every call on a device shares the one array and its counters are
 *   cleared at the start of each call on `stream`: calls that may overlap on
 *   the GPU (different streams, or different host threads) race and must be
 *   serialized by the caller, e.g. by issuing them on one stream.
 */
#define TL_NOALLOC_MAX_BATCH (1 << 20)
tl_status tl_lupp_solve_batched_noalloc(tl_handle *h, int64_t batch, const int32_t *n,
                                        const int64_t *a_off, const double *A,
                                        const int64_t *b_off, const double *b, double *x,
                                        const int64_t *piv_off, int32_t *ipiv, int32_t *info,
                                        cudaStream_t stream);

/*
 * tl_newton_integrate -- one fused kernel runs every point's own Newton loop
 * (Algorithm 2; Eqs. 1-3 of Sec. 2.1): assemble F and J, solve
 * J dx = -F by the in-register LUpp, x += dx, test convergence.
 *   law      law descriptor (host pointer, read during the call).
 *   inputs   per-point law data, field-major with stride npoints
 *            (inputs[f*npoints + p]):
 *              Norton: f = 0..5 sig0 (Mandel), f = 6..11 deps (Mandel);
 *              tanh  : f = 0..n*n-1 A column-major, then c (n), then b (n).
 *   x        out: final unknowns, x[i*npoints + p].  The initial guess is
 *            the law's own (Norton: the elastic predictor (deps, 0);
 *            tanh: 0).
 *   outputs  nullable; Norton: end-of-step stress sig[i*npoints + p].
 *   iterations, status  int32[npoints]: linear solves performed and the
 *            TL_NEWTON_* code.
 *   rtol     stop when ||F(x_k)||_2 <= rtol * ||F(x_0)||_2 (or F(x_0) = 0).
 *   max_iter at most this many linear solves (>= 0).
 */
tl_status tl_newton_integrate(tl_handle *h, const tl_law *law, int64_t npoints,
                              const double *inputs, double *x, double *outputs,
                              int32_t *iterations, int32_t *status, double rtol, int max_iter,
                              cudaStream_t stream);

/*
 * tl_newton_integrate_tangent -- tl_newton_integrate for the Norton law that
 * also returns, for every converged point, the consistent tangent operator
 * dsig/ddeps (Sec. 4.3: one multi-right-hand-side solve after convergence):
 * the converged Jacobian is factored once and solved for the six columns of
 * [I_6; 0]; the strain rows are mapped to stress by the Mandel elasticity.
 *   tangent  device double[36 * npoints]:
 *            tangent[(i + 6 j) * npoints + p] = dsig_i / ddeps_j; NaN for
 *            points that did not converge.
 * Other arguments as tl_newton_integrate (tangent is argument 7; the
 * arguments after it are numbered one higher).  TL_LAW_TANH returns
 * TL_ERR_UNSUPPORTED.
 */
tl_status tl_newton_integrate_tangent(tl_handle *h, const tl_law *law, int64_t npoints,
                                      const double *inputs, double *x, double *outputs, double *tangent,
                                      int32_t *iterations, int32_t *status, double rtol, int max_iter,
                                      cudaStream_t stream);

/*
 * tl_newton_integrate_cpu_driven -- the batched, CPU-driven evaluation of
 * the same Newton problem (Algorithm 1; the comparator of the fused kernel,
 * Sec. 2.4): each iteration launches one kernel that assembles F and J for
 * every point still iterating and tests convergence, copies the count of
 * points still iterating to the host and waits for it, then (if any) calls
 * tl_gesv_batched on all npoints systems -- points that have stopped carry
 * an identity system -- and launches the update x += dx.
 * Arguments, initial guess, stopping test and results are those of
 * tl_newton_integrate; results equal the fused kernel's.  Norton law only
 * (TL_LAW_TANH returns TL_ERR_UNSUPPORTED).  Synchronizes `stream` once per
 * iteration; uses the handle's device workspace (about 520 bytes per point,
 * grown with cudaMalloc on demand) and a pinned host word owned by the
 * handle; must not run during stream capture.
 */
tl_status tl_newton_integrate_cpu_driven(tl_handle *h, const tl_law *law, int64_t npoints,
                                         const double *inputs, double *x, double *outputs,
                                         int32_t *iterations, int32_t *status, double rtol,
                                         int max_iter, cudaStream_t stream);

/*
 * tl_autotune -- time the candidate kernels (thread-to-system mapping and
 * block size) for every n in [n_min, n_max] and the layout on the current
 * device, and keep the fastest per n in the handle's dispatch table (the
 * "best X" size-aware dispatcher, Sec. 4.1) for tl_gesv_batched,
 * tl_getrf_batched and tl_getrs_batched; the ragged solves keep their own
 * table (tl_autotune_ragged).  table_path nullable: if given, the table is
 * also written there as JSON.  Allocates and frees a temporary device batch;
 * must not run during stream capture.
 */
tl_status tl_autotune(tl_handle *h, int n_min, int n_max, tl_layout layout,
                      const char *table_path);

/*
 * tl_measure_fma_peak -- measure the FMA throughput of the current device.
 * The LU kernels are bound by the binary64 FMA pipe (Sec. 2.2: O(n^3) fused
 * multiply-adds against O(n^2) bytes), so the pipe's measured rate is the
 * roofline their throughput is compared with.  Launches 4 blocks of 256
 * threads per SM, each thread running 8 independent FMA chains, three times
 * on `stream` (the first warms up), and synchronizes the stream.
 *   bits                64 (binary64 DFMA) or 32 (binary32 FFMA).
 *   tflops              out (host): 2 x FMAs per second / 1e12 of the
 *                       fastest timed launch (CUDA events).
 *   fma_per_clk_per_sm  out (host, nullable): FMA lanes per SM per SM clock,
 *                       from the SM cycle counter of the same launch.
 *   sm_mhz              out (host, nullable): the SM clock the launch ran at.
 * Allocates nothing; must not run during stream capture
 * (TL_ERR_UNSUPPORTED).
 */
tl_status tl_measure_fma_peak(tl_handle *h, int bits, double *tflops, double *fma_per_clk_per_sm,
                              double *sm_mhz, cudaStream_t stream);

/*
 * tl_autotune_ragged -- tune tl_lupp_solve_batched per size n in
 * [n_min, n_max] on homogeneous batches of the current device (uniform
 * [-1, 1] entries, some 1.6 GFLOP of work per size): the lanes per system
 * of the single persistent binary64 launch (2, 4, 8, 16 or 32; n >= 2) and,
 * for TL_PREC_FP32_IR, the refinement kernel (the register kernel of its
 * lane count or the shared-memory warp kernel, whichever is faster) and
 * whether size n refines a binary32 factorization or goes straight to the
 * binary64 solve (refinement only where it was at least 15% faster on the
 * tuning batch: systems whose conditioning defeats the refinement fall back
 * to binary64 and pay for both, so workloads with many such systems may
 * prefer binary64 for more sizes).
 * The choices stay in the handle; table_path (nullable) receives them as
 * JSON.  Allocates and frees a temporary device batch; synchronizes; must
 * not run during stream capture.
 */
tl_status tl_autotune_ragged(tl_handle *h, int n_min, int n_max, const char *table_path);

/*
 * tl_ragged_dispatch_set / tl_ragged_dispatch_get -- per size n: lanes per
 * system of the persistent ragged launch (0 = default: one thread with the
 * system in registers up to n = 7, then 2 lanes up to n = 10, 4 up to 14, 8 up
 * to 22, 16 above; 1 (n <= 7 only) or 2..32 a power of two) and the
 * mixed-precision route (-1 = default: refine from n = 21 on, binary64
 * below; 0 = refine; 1 = binary64; systems of a size routed to binary64 get
 * refine_steps -1).  get returns the lanes the launch uses (widened when a
 * warp's systems would not fit in shared memory) and whether n refines.
 */
tl_status tl_ragged_dispatch_set(tl_handle *h, int n, int lanes, int mixed_route);
tl_status tl_ragged_dispatch_get(tl_handle *h, int n, int *lanes, int *refines);

/*
 * tl_dispatch_set / tl_dispatch_get -- read or override the per-n dispatch
 * table that tl_autotune fills (the size-aware "best X" dispatcher of
 * Sec. 4.1).
 *   variant  lanes + 100 * storage: lanes per system (1 = one thread per
 *            system, 2, 4, 8, 16, 32), storage 0 = registers (a kernel
 *            compiled for that n; 1..16 lanes), 1 = shared memory (run-time
 *            n, n >= 2; 2..32 lanes; the trailing update of 2..8 lanes on a
 *            lane tile, of 16 and 32 lanes element by element), 2 = shared
 *            memory with the element-by-element trailing update for 2..8
 *            lanes.  0 restores the built-in default.  A
 *            variant not built for n is rejected with TL_ERR_INVALID_ARG
 *            (argument 4).
 *   block    0 (occupancy + wave-fill heuristic) or 32, 64, 128 threads.
 * The choice applies to tl_gesv_batched and tl_getrf_batched for (n,
 * layout); tl_getrs_batched uses the register kernel with the same lane
 * count when one exists; the two parts of tl_lupp_solve_batched take the
 * register or shared-memory ragged kernel of the same id when one exists.
 * Their defaults: binary64, register kernels up to n = 16, shared memory
 * with 16 lanes up to n = 26, 32 lanes above; mixed precision, one thread
 * per system up to n = 10, 4 lanes in registers up to n = 16, one warp per
 * system in shared memory (id 132) above.
 */
tl_status tl_dispatch_set(tl_handle *h, int n, tl_layout layout, int variant, int block);
tl_status tl_dispatch_get(tl_handle *h, int n, tl_layout layout, int *variant, int *block);

/*
 * Request server: continuous batching of Newton-integration and
 * standalone-solve requests on one device.  The paper integrates one batch
 * of points per call (Algorithm 2); the server keeps a request loop on the
 * host (a native thread owned by the server) that admits requests as they
 * arrive against a device memory budget, and batches every admitted request
 * into "ticks": one tick copies its requests' inputs into the server's
 * device arena, launches one fused Newton kernel per law class over the
 * concatenated points of all its requests (a job table: every point keeps
 * its own request's arrays and parameters) and one ragged LUpp over all its
 * solve systems, and copies the results back.  Up to `slots` ticks are in
 * flight on their own streams, so requests that arrive while others run are
 * admitted as soon as a slot and arena room free up, and their work overlaps
 * on the device.  A point's or system's arithmetic does not depend on the
 * other work in its tick: every result equals the one tl_newton_integrate
 * (tl_lupp_solve_batched, TL_PREC_FP64) gives for the request alone.
 */
typedef struct tl_server tl_server;

typedef enum { TL_REQ_NEWTON = 0, TL_REQ_SOLVE = 1 } tl_request_kind;

/*
 * One request.  Every pointer is a HOST pointer (page-locked memory gives
 * asynchronous copies); the caller keeps the arrays valid and unmodified
 * until the request is reported done.
 *   TL_REQ_NEWTON: law, count = points; in = law fields and x, aux (Norton
 *     stress, nullable), i1 = iterations, i2 = status, all as the arguments
 *     of tl_newton_integrate (field-major with stride count), except that
 *     the fields may have a larger stride ld_in (0 = count): field f of
 *     point p at in[f*ld_in + p], so requests can share one input pool.
 *   TL_REQ_SOLVE: n (1..32), count = systems; in = A (per system
 *     column-major, n*n doubles each), rhs = b (n each), x = solutions (n
 *     each), i1 = ipiv (n each), i2 = info (one each), as
 *     tl_lupp_solve_batched with TL_PREC_FP64 and consecutive systems.
 */
typedef struct {
    int32_t kind;
    int32_t n;
    tl_law law;
    int64_t count;
    int64_t ld_in;
    const double *in;
    const double *rhs;
    double *x;
    double *aux;
    int32_t *i1;
    int32_t *i2;
} tl_request;

/*
 * Server configuration.
 *   budget_bytes        device arena holding every admitted request's
 *                       buffers and each tick's tables (one cudaMalloc at
 *                       creation).  A request that could never fit is
 *                       refused at submission with TL_ERR_NO_MEMORY.
 *   slots               ticks in flight at once (1..16), one stream each.
 *   max_points_per_tick admission cap per tick (points + systems; a single
 *                       larger request still forms a tick on its own);
 *                       0 = one request per tick (plain per-request launches
 *                       in arrival order, the comparator of batching).
 *   rtol, max_iter      Newton stopping test of every Newton request.
 */
typedef struct {
    size_t budget_bytes;
    int32_t slots;
    int64_t max_points_per_tick;
    double rtol;
    int32_t max_iter;
} tl_server_config;

typedef struct {
    int64_t submitted;
    int64_t completed;
    int64_t failed;
    int64_t ticks;
    int64_t points;       /* Newton points + solve systems completed */
    size_t arena_high_water;
    double host_enqueue_s;  /* request-loop time spent forming and issuing ticks */
    double kernel_busy_s;   /* time at least one of the server's kernels ran
                               (union of the kernel intervals, CUDA events) */
} tl_server_stats;

/* Create a server on the handle's device (the handle must outlive it).
 * Each tick's bucket workspace for its solve requests comes out of the
 * arena, so a running server allocates no device memory and never
 * synchronizes the device. */
tl_status tl_server_create(tl_handle *h, const tl_server_config *cfg, tl_server **out);
/* Queue a request (the descriptor is copied); *id identifies it.  Invalid
 * descriptors return TL_ERR_INVALID_ARG (tl_last_bad_arg of the server's
 * handle is not set), requests larger than the arena TL_ERR_NO_MEMORY. */
tl_status tl_server_submit(tl_server *s, const tl_request *req, int64_t *id);
/* Non-blocking: *done = 1 once the request's results are in its host
 * arrays; then *req_status is its outcome (TL_OK or the error of its tick)
 * and *latency_s the time from submission to completion.  An id reported
 * done is released (later calls return TL_ERR_INVALID_ARG). */
tl_status tl_server_test(tl_server *s, int64_t id, int32_t *done, int32_t *req_status, double *latency_s);
/* Block until the request is done or timeout_s passes (TL_ERR_TIMEOUT, the
 * request stays queued or running). */
tl_status tl_server_wait(tl_server *s, int64_t id, double timeout_s, int32_t *req_status, double *latency_s);
tl_status tl_server_stats_get(tl_server *s, tl_server_stats *out);
/* Stop (paused != 0) or resume admitting queued requests into ticks.  Ticks
 * already issued run to completion; submissions are still accepted and
 * queued.  tl_server_destroy resumes admission so that every queued request
 * finishes. */
tl_status tl_server_pause(tl_server *s, int paused);
/* Finish every queued request, stop the request loop, free the arena. */
tl_status tl_server_destroy(tl_server *s);

#ifdef __cplusplus
}
#endif

#endif /* TINYLU_H */
