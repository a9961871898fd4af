/*
 * l1ls -- l1-regularised least squares on one GB300: the instance generator, the products
 * A x and A^T y, FISTA and primal-dual Newton-CG, behind a plain C ABI.
 *
 * Problem (Eq. prob1 of Fountoulakis & Gondzio, "Performance of First- and Second-Order
 * Methods for l1-Regularized Least Squares Problems"):
 *
 *     minimise  f_tau(x) = tau ||x||_1 + 1/2 ||A x - b||_2^2,   A in R^{m x n}.
 *
 * Conventions for every entry point
 *  - Status: every function returns an l1ls_status; on anything but L1LS_OK a message for
 *    the calling thread is available from l1ls_last_error().  No entry point aborts, exits
 *    or traps; a CUDA error is reported as L1LS_ECUDA.
 *  - Ownership: a context owns all device memory it allocates (instances, work buffers).
 *    Buffers passed in by the caller stay owned by the caller.
 *  - Pointers: vector arguments may point to device memory (any pointer CUDA reports as
 *    device or managed memory) or to host memory.  Device pointers are used in place and
 *    the work is only enqueued on `stream` (the caller synchronises).  Host pointers are
 *    staged through context buffers and the call returns after the result has been copied
 *    back (it synchronises `stream`).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  It must belong to the device the context was created on.
 *  - Threads: one thread at a time per context, except l1ls_submit / l1ls_poll /
 *    l1ls_cancel, which may be called from any thread.
 *  - Row order: the library stores P1^T A (rows relabelled by the generator's row
 *    permutation, so the two rows mixed by one left rotation are adjacent).  Every entry
 *    point that takes or returns an m-vector (b, y of l1ls_matvec / l1ls_rmatvec, exports)
 *    uses the ORIGINAL row order of A.
 */
#ifndef L1LS_H
#define L1LS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct l1ls_ctx l1ls_ctx;     /* one GPU: streams, work buffers, memory budget      */
typedef struct l1ls_inst l1ls_inst;   /* a generated instance resident in device memory     */
typedef struct l1ls_batch l1ls_batch; /* a ragged batch of instances solved together         */

typedef enum {
    L1LS_OK = 0,
    L1LS_EINVAL = 1,      /* an argument is out of range or inconsistent                    */
    L1LS_ENOMEM = 2,      /* device or host allocation failed, or the budget is exceeded    */
    L1LS_ECUDA = 3,       /* a CUDA call failed; the context may be unusable                */
    L1LS_ETIMEOUT = 4,    /* time limit reached before convergence (result still filled)    */
    L1LS_ENOCONV = 5,     /* iteration limit reached before convergence (result filled)      */
    L1LS_ENUMERIC = 6,    /* a NaN or Inf appeared in the iteration                          */
    L1LS_EBUSY = 7,       /* the request does not fit the memory budget right now            */
    L1LS_ENOTFOUND = 8,   /* unknown ticket                                                   */
    L1LS_ECANCELLED = 9   /* the request was cancelled                                        */
} l1ls_status;

typedef enum { L1LS_F64 = 0, L1LS_F32 = 1, L1LS_BF16 = 2 } l1ls_dtype;

/*
 * Generator parameters: Procedure IGen (Sec. 3.1) for m >= n, IGen2 (Sec. 3.2) for m < n,
 * matrix A = (P1 G~ P2) Sigma G^T of Eq. (bd8) with the Givens stages of Sec. 4.1-4.2 and
 * x* from Procedure OsGen (Sec. 6).
 *   right_stages  w >= 1 stages in the right factor R = T_w ... T_1, T_1 on planes
 *                 (0,1),(2,3),... and T_2 on planes (1,2),(3,4),..., alternating.
 *   left_stages   0 (L = I, the A = Sigma G^T of the experiments of Sec. 8) or 1
 *                 (L = P G~ P of Sec. 4.1; m must then be even).
 *   kappa         kappa(A) = sigma_max / sigma_min >= 1; sigma_i = kappa^(-rank_i/(n-1)).
 *   tau           the tau of IGen; x* is the unique minimiser of f_tau for this tau.
 *   xstar_frac    s = floor(frac * n + 0.5) nonzeros (clamped to [1, min(m, n)]) with
 *                 magnitudes U[xstar_lo, xstar_hi] and random signs.
 *   theta,        rotation angles of the right and left stages (vartheta NaN: = theta).
 *   vartheta
 *   value_dtype   l1ls_dtype in which the nonzeros of A are stored (rounded from FP64).
 *   g_offsupport  0: g_i ~ U(-1,1) off the support of x*; 1: g_i = 0 there.
 *   n_nnz_per_col IGen2 only: nonzeros per column of N.
 *   sigma_mode    0: sigma_i = kappa^(-rank_i/(n-1)) (log-spaced, random assignment);
 *                 1: sigma_i = sigma_odd for odd i and sigma_even for even i (1-based), the
 *                 singular values of the huge-scale instances of Sec. 8.9.
 *   xstar_mode    0: OsGen magnitudes U[xstar_lo, xstar_hi] with random signs; 1: the first
 *                 half of the support (index order) -xstar_hi, the rest +xstar_lo (Sec. 8.9);
 *                 2: Procedure OsGen3 (Sec. 6): x = G gamma (Sigma^T Sigma)^{-1} 1 with its
 *                 s1 = s/2 smallest nonzero and s - s1 largest |x_i| kept (m >= n only).
 *   gamma         OsGen3's gamma (default 100).
 *   matrix_free   1: A is not assembled; products apply its factors (Algorithms MvPA /
 *                 MvPAt of Sec. 4: the stages of R, Sigma, the permutation and the left
 *                 rotations), so the instance holds O(m + n) memory.  IGen (m >= n) with
 *                 FP32 value_dtype only; l1ls_matvec / l1ls_rmatvec, FISTA and pdNCG work
 *                 on it (batches and exports of A do not: EINVAL).
 *   seed          all random draws are SplitMix64 streams of this seed.
 */
typedef struct {
    uint64_t m, n, seed;
    double kappa;
    double tau;
    double xstar_frac, xstar_lo, xstar_hi;
    double theta, vartheta;
    int32_t right_stages;
    int32_t left_stages;
    int32_t value_dtype;
    int32_t g_offsupport;
    int32_t n_nnz_per_col;
    int32_t matrix_free;
    int32_t sigma_mode, xstar_mode;
    double sigma_odd, sigma_even;
    double gamma;
} l1ls_gen_params;

/* Fill p with the defaults: m = 2048, n = 1024, seed 0, kappa 100, tau 1, frac 0.05,
 * magnitudes [1, 10], w = 1, one left stage, theta = vartheta = 2 pi / 10, FP64 values,
 * sigma_mode = xstar_mode = 0 (sigma_odd 0.1, sigma_even 100 for mode 1). */
void l1ls_gen_params_default(l1ls_gen_params* p);

typedef struct {
    uint64_t m, n, nnz, s;
    double f_star;        /* f_tau(x*) at tau = tau_gen                                       */
    double lipschitz;     /* L >= lambda_max(A^T A), the step constant FISTA uses              */
    double lam_max;       /* ||A^T b||_inf: every tau >= lam_max has minimiser 0               */
    double tau_gen;
    int32_t value_dtype, right_stages, left_stages, igen2;
    int32_t matrix_free, reserved;
    uint64_t device_bytes;/* device memory held by the instance                                */
} l1ls_inst_info;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the device memory the
 * context may hold for instances and solver state (0 = 90% of the free memory at creation).
 * The context also holds 512 KiB of pinned host memory (512 slots) into which the solvers
 * read their per-step state back; pinned copies from concurrent threads do not queue behind
 * each other as pageable ones do.  If that allocation fails, or all slots are taken, solvers
 * fall back to pageable memory.  Errors: EINVAL (bad device), ECUDA. */
l1ls_status l1ls_create(int device, size_t hbm_budget_bytes, l1ls_ctx** out);

/* Destroy a context: waits for its serving thread, frees every instance it still owns. */
l1ls_status l1ls_destroy(l1ls_ctx* ctx);

/* Generate an instance on the device (Procedures IGen / IGen2, Eq. bd8, OsGen): random keys
 * and permutations, singular values, x*, g, e and b by the matrix-free route of Sec. 4
 * (two products with the right factor and a diagonal scaling), and CSR(P1^T A) and
 * CSR(A^T P1) with FP64 values rounded once to value_dtype.  The integer structure is
 * fully determined by the parameters.  Enqueued on `stream`; returns after completion.
 * Errors: EINVAL (sizes, stages, kappa < 1, nnz >= 2^31), ENOMEM (budget), ECUDA. */
l1ls_status l1ls_generate(l1ls_ctx* ctx, const l1ls_gen_params* p, void* stream, l1ls_inst** out);

l1ls_status l1ls_inst_free(l1ls_inst* inst);
/* The conditioning of x* of Eq. (bd12): kappa_rho(x*) = ||x*|| / ||P_rho x*||, P_rho the
 * projection on the eigenvectors of A^T A with eigenvalue >= rho (with A^T A = R Sigma^2 R^T:
 * the entries of R^T x* with sigma_i^2 >= rho); +inf when that projection is 0.  IGen (m >= n)
 * instances.  Synchronous (a stream of its own).  Errors: EINVAL (NULL, an IGen2 instance, rho
 * NaN), ENOMEM, ECUDA. */
l1ls_status l1ls_inst_kappa_rho(const l1ls_inst* inst, double rho, double* out);
l1ls_status l1ls_inst_get_info(const l1ls_inst* inst, l1ls_inst_info* info);

/* Copy an instance to host buffers (any may be NULL).  A is returned in CSR with the
 * ORIGINAL row order and ascending column indices within each row; values converted to
 * double from the stored dtype.  row_ptr: m+1, col_idx/vals: nnz, b: m, xstar/sigma: n
 * (sigma: the singular values of the square factor, length min(m, n)), perm: m (the row
 * permutation P, (P v)_i = v_{perm[i]}; identity when left_stages = 0).  Synchronous. */
l1ls_status l1ls_inst_export(const l1ls_inst* inst, int64_t* row_ptr, int32_t* col_idx, double* vals,
                             double* b, double* xstar, double* sigma, int64_t* perm);

/* Copy CSR(A^T) (= CSC of A) to host: col_ptr n+1, row_idx/vals nnz, row indices in the
 * ORIGINAL row order, ascending within each column.  Synchronous. */
l1ls_status l1ls_inst_export_t(const l1ls_inst* inst, int64_t* col_ptr, int32_t* row_idx, double* vals);

/* y = A x (Algorithm MvPA computes the same product matrix-free).  x: n entries, y: m
 * entries, both of type vec_dtype (L1LS_F64 or L1LS_F32).  Accumulation is in FP64 for
 * FP64 values and FP32 otherwise.  Errors: EINVAL, ECUDA. */
l1ls_status l1ls_matvec(const l1ls_inst* inst, const void* x, l1ls_dtype vec_dtype, void* y, void* stream);

/* x = A^T y (Algorithm MvPAt).  y: m entries, x: n entries, as for l1ls_matvec. */
l1ls_status l1ls_rmatvec(const l1ls_inst* inst, const void* y, l1ls_dtype vec_dtype, void* x, void* stream);

/* x = A^T y like l1ls_rmatvec, for callers that cannot allocate device memory: real-time
 * loops that must not stall on the device-wide synchronisation cudaMalloc / cudaFree may
 * imply, and host applications that own all device memory (a fixed budget handed out up
 * front, libraries not allowed to allocate).  (The paper has no counterpart; this is an
 * interface of this library.)
 *   y, x: DEVICE pointers only (m and n entries of vec_dtype, L1LS_F64 or L1LS_F32); a host
 *   pointer is refused with L1LS_EINVAL before anything is enqueued.
 *   The one m-vector of scratch the product needs lives in a fixed array compiled into the
 *   library: 2^20 doubles (8 MiB) held by every GPU that loads the library until the process
 *   exits.  Instances with m > 2^20 are rejected with L1LS_EINVAL.
 *   No cudaMalloc, cudaFree or other allocating call is made.  The first call on a device
 *   looks up the array's device address (cudaGetSymbolAddress) with that device current.
 *   The address is kept for the life of the process, which assumes the device's primary
 *   context is never reset (cudaDeviceReset).
 *   All calls share the array and it keeps the last call's contents (every entry used is
 *   written before it is read, so nothing needs clearing).  Calls whose work overlaps on the
 *   GPU (different streams, or different threads) race on the array: order them.
 *   Enqueued on `stream`; errors as for l1ls_rmatvec. */
l1ls_status l1ls_rmatvec_noalloc(const l1ls_inst* inst, const void* y, l1ls_dtype vec_dtype, void* x, void* stream);

/* Solver options.  Defaults (l1ls_solve_opts_default): tau 1, rel_gap_tol 1e-6,
 * max_iter 100000 (FISTA iterations; Newton steps for pdNCG), no time limit, mu 1e-5,
 * mu_min 1e-14, mu_start 1, pcg_rtol 0.1, pcg_max 1000, ls_max 50, armijo 1e-4,
 * check_every 32, f_target -inf.  pdNCG only: mu (the paper's smoothing parameter, Sec. 8.3) is reached by
 * continuation from mu_start (divided by 10 after each full Newton step); below mu it is
 * divided by 10 again, down to mu_min, when a full step fails to halve the gap. */
typedef struct {
    double tau;
    double rel_gap_tol;
    int64_t max_iter;
    double time_limit_s;      /* <= 0: none */
    double mu, mu_min, mu_start, pcg_rtol, armijo;
    int32_t ls_max, pcg_max;
    int32_t check_every;      /* iterations per graph launch between host checks          */
    int32_t restart;          /* FISTA: 1 = gradient restart of O'Donoghue & Candes (t <- 1 when
                                 (y_k - x_k)^T (x_k - x_{k-1}) > 0); 0 = none, as in the paper  */
    int32_t accum;            /* FISTA, FP32 / BF16 values: 0 = products summed in FP32 (the
                                 default); 1 = products of the float-float iterate and residual
                                 summed in float-float (about 44 bits), for gaps below the FP32
                                 floor at small tau or large kappa.  EINVAL with FP64 values.
                                 Batches always use 1.  pdNCG, FP32 / BF16 values: 1 = the
                                 two products of each Newton step that give the gradient and
                                 the certificate (r = b - A x, A^T r) in float-float, the PCG
                                 products in FP32; ignored with FP64 values.                   */
    double f_target;          /* FISTA, FISTA with backtracking, pdNCG: also stop (status OK) as
                                 soon as the certified objective f(x_k) <= f_target, the rule by
                                 which the paper ends its comparison solvers (Sec. 8.3); -inf
                                 (the default): off.  Batches ignore it.                       */
} l1ls_solve_opts;

void l1ls_solve_opts_default(l1ls_solve_opts* o);

typedef struct {
    int64_t iters;            /* FISTA iterations / Newton steps performed                  */
    int64_t products;         /* products with A or A^T                                      */
    int64_t cg_iters, ls_trials;
    double f;                 /* primal objective f_tau at the returned x                    */
    double dual;              /* dual objective of the certifying dual point                  */
    double gap, rel_gap;      /* f - dual and (f - dual) / f                                  */
    double seconds;           /* wall time of the call                                        */
    double mu;                /* final smoothing parameter (pdNCG)                            */
    int32_t status;           /* l1ls_status of the solve                                     */
    int32_t reserved;
    double queue_s;           /* serving (l1ls_poll): submission to admission, seconds         */
    double latency_s;         /* serving (l1ls_poll): submission to completion, seconds        */
    double L;                 /* l1ls_solve_fista_bt: the final step constant                 */
} l1ls_result;

/* FISTA (Sec. 8.1; Beck & Teboulle) with fixed L = info.lipschitz from x0 (NULL: 0).  Stops
 * when the duality-gap certificate P(x_k) - max_j D(theta(y_j)) is at most rel_gap_tol * P(x_k),
 * where theta(y) = s (b - A y), s = min(1, tau / ||A^T (b - A y)||_inf).  x0 and x_out are
 * n doubles (device or host; x_out may be NULL).  Returns ENOCONV / ETIMEOUT with `res`
 * filled when a limit is hit, ENUMERIC on NaN/Inf.  Blocking. */
l1ls_status l1ls_solve_fista(l1ls_inst* inst, const l1ls_solve_opts* o, const double* x0, double* x_out,
                             l1ls_result* res, void* stream);

/* FISTA with backtracking on L (Beck & Teboulle's FISTA with backtracking; the paper runs
 * FISTA through TFOCS, whose L is dynamic, Sec. 8.1).  Starts from L = L0 (> 0); in every
 * iteration the prox-gradient trial x = S_{tau/L}(y_k + A^T r_k / L) is accepted when
 * ||A (x - y_k)||^2 <= L ||x - y_k||^2 (the sufficient-decrease test of 1/2 ||Ax - b||^2),
 * otherwise L is multiplied by eta (> 1) and the trial repeated, at most o->ls_max times per
 * iteration (then ENUMERIC).  L never decreases.  Each trial costs one product with A, each
 * iteration one with A^T.  The certificate is that of l1ls_solve_fista evaluated at the
 * iteration's own output x_k.  FP64 vectors; assembled matrices only (EINVAL for
 * matrix_free).  res->ls_trials counts the increases of L, res->L is the final L.  Other
 * arguments, statuses and the stopping rule as for l1ls_solve_fista (o->restart and
 * o->accum are ignored).  Blocking. */
l1ls_status l1ls_solve_fista_bt(l1ls_inst* inst, const l1ls_solve_opts* o, double L0, double eta, const double* x0,
                                double* x_out, l1ls_result* res, void* stream);

/* FISTA in steps, for callers that drive the iteration themselves (benchmarks, schedulers):
 *   l1ls_fista_begin  sets up the state of l1ls_solve_fista at x0 (NULL: 0) and enqueues it;
 *   l1ls_fista_step   enqueues `iters` further iterations (two kernels each) without any
 *                     host synchronisation; iterations after the stop test fired are no-ops.
 *                     With kernel_ms != NULL (2 floats) CUDA events on `stream` bracket the
 *                     two kernels of every iteration and their summed durations in ms are
 *                     returned (this synchronises `stream`).
 *   l1ls_fista_end    waits for `stream`, then returns the last certified iterate (x_out may
 *                     be NULL) and its certificate; status ENOCONV if the stop test has not
 *                     fired yet.
 * One FISTA run per instance at a time; l1ls_solve_fista is begin + graph-captured steps + end. */
l1ls_status l1ls_fista_begin(l1ls_inst* inst, const l1ls_solve_opts* o, const double* x0, void* stream);
l1ls_status l1ls_fista_step(l1ls_inst* inst, int64_t iters, float* kernel_ms, void* stream);
l1ls_status l1ls_fista_end(l1ls_inst* inst, double* x_out, l1ls_result* res, void* stream);

/* pdNCG (Sec. 8.1, parameters of Sec. 8.3): primal-dual Newton-CG on the pseudo-Huber
 * smoothing (Eqs. pseudoHuber, prob2, bd4) with diagonal-preconditioned CG stopped at
 * relative residual pcg_rtol (in the preconditioner's norm), a halving Armijo line search of
 * at most ls_max trials, and mu-continuation as described with l1ls_solve_opts.  Certified
 * with the same gap as FISTA at the current iterate.  Arguments as for l1ls_solve_fista.
 * Matrix-free instances: L in A = L Sigma R^T is orthogonal, so the gradient is A^T b (formed
 * once per instance, FP64) - R Sigma^2 R^T x and the CG product A^T A p = R Sigma^2 R^T p:
 * the gradient and the certificate run in an FP64 sweep over the stages of R, the CG product
 * and the line search's ||A d|| in FP32 sweeps; o->accum is ignored.  The first solve on such an
 * instance also forms diag(A^T A) and A^T b (n doubles each, kept with the instance). */
l1ls_status l1ls_solve_pdncg(l1ls_inst* inst, const l1ls_solve_opts* o, const double* x0, double* x_out,
                             l1ls_result* res, void* stream);

/* Ragged batches and tau paths (the regularisation study of Sec. 8.8 as a workload).
 *   l1ls_batch_create   groups `count` instances of one context that have one left stage and
 *                       FP32 or BF16 values (all the same); it allocates their iterates and
 *                       the batch tables (counted in the context budget).  The instances must
 *                       outlive the batch.
 *   l1ls_batch_solve_path  solves every instance i along its path taus[i*ntau .. i*ntau+ntau-1]
 *                       with FISTA (as l1ls_solve_fista: o->rel_gap_tol, o->max_iter per tau,
 *                       o->time_limit_s for the whole call; o->tau is ignored), all instances in
 *                       one persistent cooperative kernel per o->check_every FISTA steps.  The
 *                       first tau starts from 0; each later tau starts from the last iterate of
 *                       the previous one (one prox-gradient step past the certified iterate).
 *                       results: count*ntau entries (instance-major), filled per tau (a tau not
 *                       finished when the call ends early gets the call's status); x_out: NULL
 *                       or count pointers (each NULL, device or host; n doubles) receiving the
 *                       certified solution at the last tau.  An instance's results do not depend
 *                       on the other instances of the batch or on the kernel schedule.  Blocking.
 *   l1ls_batch_get_schedule  schedule chosen by the built-in autotuner (0 before the first
 *                       solve): threads per block and entries per lane of the traversal (0: the
 *                       staged stream, where each lane sums its own row from shared memory),
 *                       and tune_ms (4 doubles, may be NULL): the time of the four probe steps
 *                       of each candidate (256, 0), (128, 0), (256, 8), (128, 8), in ms.
 *   l1ls_batch_get_stats  of the last solve: batch steps run (each one FISTA step of every
 *                       active instance) and the device time of its launches in ms (CUDA
 *                       events on the solve's stream around the launch loop).
 * Errors: EINVAL, ENOMEM, ECUDA (including an expired bounded grid barrier), ETIMEOUT. */
l1ls_status l1ls_batch_create(l1ls_ctx* ctx, int count, l1ls_inst* const* insts, l1ls_batch** out);
l1ls_status l1ls_batch_solve_path(l1ls_batch* batch, const double* taus, int ntau, const l1ls_solve_opts* o,
                                  l1ls_result* results, double* const* x_out, void* stream);
l1ls_status l1ls_batch_get_schedule(const l1ls_batch* batch, int* block, int* entries_per_lane, double* tune_ms);
l1ls_status l1ls_batch_get_stats(const l1ls_batch* batch, int64_t* steps, double* device_ms);
/* Failure-detection self-test of the batched kernel's bounded grid barrier: runs one step in
 * which the barrier expects one block more than the grid holds, so every block's wait runs out
 * after max_polls polls (each with a short sleep), records the expiry and leaves the kernel.
 * Returns L1LS_ECUDA with the message a real expiry gives, the elapsed wall time in *seconds
 * (may be NULL), and leaves the batch and its context usable (the next solve runs normally). */
l1ls_status l1ls_batch_barrier_selftest(l1ls_batch* batch, uint32_t max_polls, double* seconds);
l1ls_status l1ls_batch_free(l1ls_batch* batch);

/* Serving: solve requests admitted by device-memory footprint and run concurrently.
 * A request is (generator parameters, solver options, method): the instance is generated on
 * the device, solved to o->rel_gap_tol at o->tau, and freed; the caller receives x (n
 * doubles) and the certificate.  Each context runs `slots` worker threads, each with its own
 * CUDA stream.  Requests are admitted in submission order: the oldest waiting request starts
 * as soon as a slot is free and its footprint (l1ls_footprint) fits next to the footprints of
 * the running requests within the capacity; later requests never overtake it.  Requests
 * that arrive while others run are admitted as slots and memory free up, and their kernels
 * overlap on the device.  A request's result does not depend on the other requests.
 *   l1ls_serve_config  optional, before the first l1ls_submit: slots (1..256; default 8) and
 *                      the capacity in bytes (0: the context budget not yet used).  EBUSY if
 *                      the loop is already running.  With more than 8 slots, set the
 *                      environment variable CUDA_DEVICE_MAX_CONNECTIONS to the slot count
 *                      (up to 32) before the process initialises CUDA, so that the slots'
 *                      streams do not share hardware work queues.
 *   l1ls_submit        queues a request; returns at once with its ticket.  o->tau < 0 means
 *                      |o->tau| * lambda_max of the generated instance.  EBUSY if its
 *                      footprint exceeds the whole capacity, EINVAL for bad options (bad
 *                      generator parameters are reported by l1ls_poll).
 *   l1ls_poll          waits up to wait_ms (0: no wait) for the request.  Not finished: EBUSY
 *                      (nothing written, the ticket stays valid).  Finished: fills res
 *                      (including queue_s and latency_s) and x_out (n doubles, host, may be
 *                      NULL), releases the ticket, and returns the request's status (OK,
 *                      ENOCONV, ETIMEOUT, ENUMERIC, EINVAL, ENOMEM, ECUDA or ECANCELLED).
 *                      Unknown or released ticket: ENOTFOUND.
 *   l1ls_cancel        a queued request never runs (l1ls_poll then returns ECANCELLED); a
 *                      running one stops at its next host check and returns ECANCELLED.
 *   l1ls_serve_stats   counters of the loop (all zero before the first request).
 * l1ls_destroy cancels every request and joins the workers.  These functions may be called
 * from any thread. */
typedef enum { L1LS_FISTA = 0, L1LS_PDNCG = 1 } l1ls_method;
typedef struct {
    int32_t slots, running, peak_running, reserved0;
    uint64_t completed, queued;
    uint64_t capacity_bytes, reserved_bytes, peak_reserved_bytes;
} l1ls_serve_info;
size_t l1ls_footprint(const l1ls_gen_params* p, int method);
l1ls_status l1ls_serve_config(l1ls_ctx* ctx, int slots, size_t capacity_bytes);
l1ls_status l1ls_submit(l1ls_ctx* ctx, const l1ls_gen_params* p, const l1ls_solve_opts* o, int method,
                        uint64_t* ticket);
l1ls_status l1ls_poll(l1ls_ctx* ctx, uint64_t ticket, int wait_ms, l1ls_result* res, double* x_out);
l1ls_status l1ls_cancel(l1ls_ctx* ctx, uint64_t ticket);
l1ls_status l1ls_serve_stats(l1ls_ctx* ctx, l1ls_serve_info* info);

/* Thread-local message describing the last non-OK status returned on this thread. */
const char* l1ls_last_error(void);

/* Library version string. */
const char* l1ls_version(void);

#ifdef __cplusplus
}
#endif

#endif /* L1LS_H */
