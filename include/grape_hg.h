/*
 * grape_hg.h -- C ABI of the GB300 hard-coded-gradient (HG) GRAPE library.
 *
 * One evaluation returns the composite GRAPE cost and its gradient with respect
 * to every piecewise-constant control amplitude (arXiv:2304.06200, Sec. II and
 * Sec. III).  Propagators exp(-i H_n dt) are never formed: each step applies the
 * scaled truncated-Taylor action (e^{B}_m)^s, B = -i H_n dt / s (Sec. III.B, Eqs.
 * (scaling squaring equation), (eBm equation), (eBmpsi)), with (m, s) chosen per
 * step by the paper's error bound E_A(m, s) <= tau (Eq. (accuracy inequality),
 * App. C Eq. (overallupperbound)).  The gradient follows the forward-backward
 * scheme of Sec. III.C / Fig. 1: a forward sweep to psi_N, then a backward sweep
 * that re-propagates psi and the costate with the adjoint step and accumulates
 * <costate| dU_n/du_kn |psi_{n-1}> (Eqs. (stgradient), (gategradient),
 * (C2stgrad)), the derivative being that of the Taylor approximant at frozen
 * (m, s) (Eq. (auxiliary equation)).  Alternatively (descriptor field `propagator`) each step
 * propagator comes from a Hermitian eigendecomposition and its derivative from the divided
 * differences of exp on the spectrum (App. F), exact up to rounding.
 *
 * Cost (all terms optional through their weights):
 *   C     = w_fid * C1 + w_forbid * C2 + w_amp * C_amp + w_tint * C3
 *   C1    = 1 - |g / n|^2,  g = sum_h <phi_T^h | psi_N^h>     Eq. (C1st) / gate form, Sec. III.A
 *   C2    = 1/(N n) sum_{n'=1..N} sum_h <psi_n'^h|Omega|psi_n'^h>   App. A, Eq. (c2st)
 *   C_amp = 1/N sum_{k,n} u_kn^2                    amplitude penalty named in Sec. II
 *   C3    = 1 - 1/(N n^2) sum_n' |g_n'|^2          time-integrated infidelity, App. A (weight w_tint)
 * with n = n_states columns propagated together as one block.
 *
 * Conventions
 *   - Complex numbers are interleaved (re, im) doubles.
 *   - State blocks (psi0, target) are dim x n_states, column-major: column h is
 *     dim contiguous complex numbers.
 *   - Controls u and gradients are n_controls x n_steps doubles, row-major
 *     (row k = control channel k, column n = time step n).
 *   - Every function returns a grape_status; no C++ exception crosses the ABI.
 *     On failure grape_last_error() returns a thread-local message.
 *   - Host arrays passed to grape_problem_create are deep-copied: the caller
 *     keeps ownership.  The problem object owns all device memory it uses.
 *   - One problem must not be used from two host threads or two streams at once.
 */
#ifndef GRAPE_HG_H
#define GRAPE_HG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRAPE_ABI_VERSION 5

typedef struct grape_problem grape_problem;

typedef enum {
  GRAPE_OK = 0,
  GRAPE_EINVAL = 1,          /* bad argument, shape or pointer                                */
  GRAPE_ENOMEM = 2,          /* a device or host allocation failed                            */
  GRAPE_ECUDA = 3,           /* a CUDA runtime call failed (message in grape_last_error)      */
  GRAPE_ETOL = 4,            /* some step has no (m, s) with E_A(m, s) <= tau (App. C)         */
  GRAPE_ETIMEOUT = 5,        /* a bounded device wait gave up                                 */
  GRAPE_ENOTHERMITIAN = 6,   /* H0 or some H_k is not Hermitian                               */
  GRAPE_ESTATE = 7,          /* call order: grape_grad without a preceding grape_cost         */
  GRAPE_ENONFINITE = 8       /* a control amplitude is NaN or infinite                       */
} grape_status;

typedef enum { GRAPE_CSR = 0, GRAPE_DENSE = 1 } grape_format;

/* Arithmetic of the propagation bulk.  Cost, overlaps, gradient sums and the
 * step norms are FP64 in every mode. */
typedef enum {
  GRAPE_FP64 = 0,        /* complex128 throughout                                        */
  GRAPE_FP32_BULK = 1,   /* compensated FP32 bulk: every Taylor term, product and Horner vector
                            is a pair of complex64 numbers hi + lo, accumulated with error-free
                            FP32 transformations (TwoProduct by FMA, TwoSum), about 2^-48
                            relative per operation; states, costates, W and reductions FP64.
                            Scheduled by the FP64 rule (u = 2^-53); errors are measured.       */
  GRAPE_TC_FP16 = 2,     /* dense operator: every Taylor product is a real-split GEMM on the
                            tensor cores (FP16 hi/lo operands, FP32 accumulation); states,
                            costates and reductions FP64.  Needs dim % 128 == 0, n_states <= 16. */
  GRAPE_TC_BF16 = 3      /* as GRAPE_TC_FP16 with BF16 hi/lo operands (8 + 8 significant bits
                            instead of 11 + 11: wider exponent range, ~2^-16 relative operands) */
} grape_precision;

/* How each step's propagator exp(-i H_n dt) acts.
 *   GRAPE_PROP_TAYLOR: truncated Taylor series with scaling and squaring, (m, s) by the bound
 *                      E_A(m, s) <= tau (Sec. III.B, App. C); sparse operators, any dim.
 *   GRAPE_PROP_EIG:    Hermitian eigendecomposition per step, U_n = V diag(exp(-i lambda dt)) V^+,
 *                      and the propagator derivative from the divided differences of exp on the
 *                      spectrum (App. F).  Exact up to rounding; operators treated as dense;
 *                      needs GRAPE_FP64 and dim <= 96 (the step matrix lives in shared memory);
 *                      tau, m_max, ckpt_every, cluster and backward_mode are ignored.  Memory
 *                      grows with N d^2 (three d x d blocks per step). */
typedef enum { GRAPE_PROP_TAYLOR = 0, GRAPE_PROP_EIG = 1 } grape_propagator;

/* One Hermitian operator (H0 or a control H_k), dim x dim.
 *   fmt == GRAPE_CSR:   rowptr[dim+1] (int64, rowptr[0] == 0), colind[nnz] (int32, 0-based,
 *                       any order within a row, no duplicates), values[2*nnz] complex.
 *   fmt == GRAPE_DENSE: values[2*dim*dim] complex, row-major; rowptr/colind ignored.
 * Zero entries of a dense operator are dropped. */
typedef struct {
  int32_t fmt;
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* values;
} grape_op;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a device pointer aligned to 256 bytes or NULL; free releases it.
 * Both NULL: cudaMalloc / cudaFree. */
typedef void* (*grape_alloc_fn)(size_t bytes, void* ctx);
typedef void (*grape_free_fn)(void* ptr, size_t bytes, void* ctx);

typedef struct {
  int64_t dim;                 /* Hilbert-space dimension d                               */
  int32_t n_controls;          /* K >= 0 (at most 32)                                      */
  int32_t n_steps;             /* N >= 1                                                  */
  int32_t n_states;            /* n, 1 <= n <= dim: columns propagated together           */
  double dt;                   /* step length (> 0), same time unit as 1/H                */
  grape_op H0;                 /* drift H_s                                               */
  const grape_op* Hk;          /* K control operators h_k                                 */
  const double* psi0;          /* dim x n complex, column-major: initial states psi_0^h   */
  const double* target;        /* dim x n complex, column-major: phi_T^h = U_T psi_0^h    */
  const double* omega_diag;    /* dim real: diagonal of the forbidden-state operator, or NULL */
  double w_fid, w_forbid, w_amp;   /* weights alpha_1..alpha_3 of the composite cost      */
  double tau;                  /* tolerance of the (m, s) rule, 0 < tau < 1                */
  int32_t m_max;               /* largest Taylor order considered, 1..60 (0 = 60)          */
  int32_t ckpt_every;          /* M: psi checkpoint every M steps for the backward sweep;
                                  0 = automatic, < 0 = no checkpoints (pure re-propagation) */
  int32_t precision;           /* grape_precision                                         */
  int32_t cluster;             /* CTAs per column team: 0 = automatic, else 1..16 (both sweeps) */
  int32_t device;              /* CUDA device ordinal                                     */
  grape_alloc_fn alloc;        /* optional device allocator (see above)                   */
  grape_free_fn free;
  void* alloc_ctx;
  int32_t backward_mode;       /* 0 = automatic (three-stage when ckpt_every >= 0 and N >= 2,
                                  else 1), 1 = one team per column runs both backward phases
                                  (adjoint re-propagation of psi between checkpoints), 3 =
                                  three-stage: the forward stores every state (ckpt_every 0 or 1;
                                  N * dim * n_states * 16 bytes; automatic up to 8 GiB) or every
                                  M-th one (ckpt_every = M > 1, or automatically M = 50 above
                                  8 GiB; two segments of M states are recomputed from them), one
                                  team per column runs only the costate chain and stores its
                                  Horner vectors in three rotating block buffers, and the gradient
                                  terms of every step of a block are computed independently on
                                  the remaining SMs                                          */
  double bulk_norm_cap;        /* > 0: the (m, s) rule only considers s >= ||A||_1 / cap, i.e.
                                  ||B||_1 <= cap, which bounds the largest Taylor term; 0 = default
                                  (2.0 for the tensor-core modes, no cap for GRAPE_FP64 and
                                  GRAPE_FP32_BULK, i.e. the paper's rule unchanged)             */
  double w_tint;               /* weight alpha_4 of the time-integrated infidelity
                                  C3 = 1 - 1/(N n^2) sum_{n'=1..N} |sum_h <phi_T^h|psi_n'^h>|^2
                                  (App. A, C3st / C3g; 0 = off)                                 */
  int32_t propagator;          /* grape_propagator (0 = Taylor)                               */
  int32_t grad_cluster;        /* three-stage backward: CTAs per (step, column) team of the gradient
                                  kernel, 0 = automatic (the smallest team whose working set fits
                                  shared memory), else 1..16                                   */
  int32_t block_steps;         /* three-stage backward: steps per block (the unit handed from the
                                  costate chain to the gradient kernel), 0 = automatic          */
} grape_desc;

/* Information about a problem (valid after create; schedule fields after an evaluation). */
typedef struct {
  int64_t device_bytes;        /* device memory held by the problem                      */
  int64_t union_nnz;           /* non-zeros of the union pattern of H0 and all H_k        */
  int64_t ctrl_entries;        /* stored control entries (sum of nnz(H_k))                 */
  int32_t sigma;               /* sigma': largest row count of the union pattern (Eq. (sigmapdef)) */
  int32_t m_cap;               /* largest Taylor order the schedule table can return      */
  int32_t s_cap;               /* largest scaling factor the schedule table can return    */
  int32_t cluster;             /* CTAs per column team of the backward sweep               */
  int32_t ckpt_every;          /* checkpoint spacing actually used (0 = none)             */
  int32_t smem_bytes;          /* dynamic shared memory per CTA of the sweep kernels       */
  int64_t total_terms;         /* sum over steps of m_n * s_n for the last evaluation (-1 before) */
  double max_norm;             /* max_n ||A_n||_1 of the last evaluation (-1 before)       */
  int32_t backward_mode;       /* 1 = one team per column, 3 = three-stage (costate chain +
                                  per-step gradient kernels)                                   */
  int32_t cluster_forward;     /* CTAs per column team of the forward sweep                */
  int32_t propagator;          /* grape_propagator of the problem                          */
  int32_t grad_cluster;        /* three-stage backward: CTAs per gradient team (0 = not used)  */
  int32_t block_steps;         /* three-stage backward: steps per block (0 = not used)         */
  int32_t fused_fallback;      /* three-stage backward: 1 if the last evaluation's Horner vectors
                                  did not fit the block buffers and the one-team fused backward
                                  ran instead, 0 if the three stages ran, -1 otherwise          */
} grape_info;

/* Create a problem (Sec. II: H(t) = H_s + sum_k a_k(t) h_k, piecewise constant over N steps
 * of length dt).  Validates shapes, Hermiticity and finiteness, builds the union sparsity
 * pattern, the (m, s) breakpoint table of App. C for the given tau and sigma', and
 * uploads everything to the device.  On failure *out is set to NULL.
 * Basis order and speed: the sparse sweeps give each thread one row and each warp 32 consecutive
 * rows, which pays for its longest row in every loop; they run fastest when consecutive basis
 * states couple alike (e.g. the product basis with its largest factor, a cavity, varying fastest).
 * Results do not depend on the order beyond rounding. */
grape_status grape_problem_create(const grape_desc* desc, grape_problem** out);

/* Release every resource of the problem (NULL is accepted). */
void grape_problem_destroy(grape_problem* prob);

/* One full evaluation: cost (forward sweep, Fig. 1(a)) and gradient (backward sweep,
 * Fig. 1(b)).
 *   u     n_controls x n_steps controls (row-major), host or device per on_device.
 *   cost  1 double (host or device); grad n_controls x n_steps doubles or NULL.
 *   on_device  0: u, cost, grad are host pointers (the call synchronises the stream
 *              and reports device-side errors); 1: device pointers (asynchronous,
 *              call grape_sync_status to collect device-side errors).
 *   stream  cudaStream_t to run on (NULL = legacy default stream). */
grape_status grape_cost_and_grad(grape_problem* prob, const double* u, double* cost, double* grad,
                                 int32_t on_device, void* stream);

/* Forward sweep only (Fig. 1(a)): cost, with the state needed by a later grape_grad
 * (psi_N, checkpoints, g) kept inside the problem. */
grape_status grape_cost(grape_problem* prob, const double* u, double* cost, int32_t on_device, void* stream);

/* Backward sweep only (Fig. 1(b)) for the controls of the preceding grape_cost call.
 * GRAPE_ESTATE if no forward sweep has run. */
grape_status grape_grad(grape_problem* prob, double* grad, int32_t on_device, void* stream);

/* GRAPE by steepest descent (Sec. II, Eq. (4): a^(j+1) = a^(j) - eta grad C(a^(j)), constant
 * learning rate eta): n_iter iterations, each a full evaluation (forward sweep, cost, backward
 * sweep, gradient) followed by the update u - (eta * g) (two roundings), recorded once into a CUDA
 * graph on a problem-owned stream (on the first call, when eta changes and when n_iter exceeds all
 * earlier calls) and launched n_iter times on `stream`.
 *   u         K x N controls, row-major: initial values in, final values out.  Caller-owned; host
 *             memory if on_device == 0, device memory on the problem's device otherwise.
 *   n_iter    >= 1.
 *   eta       finite, > 0.
 *   costs     n_iter doubles (same memory kind as u): costs[j] = C(a^(j)), the cost before update j.
 * Errors: GRAPE_EINVAL for bad arguments or a tensor-core problem (its sweeps are driven from
 * the host); device errors of any iteration (non-finite controls, ETOL, ETIMEOUT) are returned when
 * on_device == 0 (the call then synchronises `stream`), else by grape_sync_status.  A following
 * grape_grad needs a new grape_cost (the stored sweep state belongs to the last iterate). */
grape_status grape_optimize(grape_problem* prob, double* u, int32_t n_iter, double eta, double* costs,
                            int32_t on_device, void* stream);

/* Wait for the problem's pending work on `stream` and return the device error word
 * (GRAPE_OK, GRAPE_ETOL: no feasible (m, s) or an eigenvalue iteration that did not converge,
 * GRAPE_ENONFINITE or GRAPE_ETIMEOUT); the word is then cleared. */
grape_status grape_sync_status(grape_problem* prob, void* stream);

/* Problem information (see grape_info). */
grape_status grape_problem_info(grape_problem* prob, grape_info* info);

/* Kernel tracing (no counterpart in the paper: measurement support).  With tracing enabled, every
 * evaluation records a pair of CUDA events around each launch of the sweep kernels (on the stream
 * the kernel runs on; nothing is recorded while a stream is being captured into a CUDA graph), and
 * grape_kernel_times sums their durations over the evaluations since the last call (which resets
 * the sums; it waits for the problem's pending work).  Index: 0 = k_forward, 1 = k_costate,
 * 2 = k_gradient, 3 = the fused one-team backward kernel, 4 = the forward launches that recompute
 * a segment's states (three-stage backward with checkpoints more than one step apart). */
typedef struct {
  int32_t launches[5];
  double ms[5];
} grape_kernel_times_t;
grape_status grape_set_kernel_tracing(grape_problem* prob, int32_t enable);
grape_status grape_kernel_times(grape_problem* prob, grape_kernel_times_t* out);

/* Measurement support (no counterpart in the paper): the device's FP64 fused multiply-add rate in
 * GFLOP/s (2 flops per FMA), from one launch of independent FMA chains on every SM timed with CUDA
 * events; the sweep kernels are bound by FP64 issue, so this is their roofline's peak.  Allocates
 * and frees a small buffer; synchronises the device; about 0.1 s. */
grape_status grape_fp64_fma_rate(int32_t device, double* gflops);

/* Per-step schedule of the last evaluation, copied to host arrays of n_steps entries
 * each (any may be NULL): Taylor order m_n, scaling factor s_n, and ||A_n||_1. */
grape_status grape_step_schedule(grape_problem* prob, int32_t* m, int32_t* s, double* norm1);

/* The paper's rule on the host (Sec. III.B; App. C Eq. (overallupperbound)): the smallest
 * s, then the smallest m <= m_max, with E_A(m, s) <= tau for ||A||_1 = x and sigma' = sigma,
 * unit roundoff 2^-53 (precision GRAPE_FP64) or 2^-24 (precision 1: the bound for plain FP32
 * terms; GRAPE_FP32_BULK problems themselves are scheduled with 2^-53).
 * GRAPE_ETOL if no pair with s <= s_max qualifies.  Pure host computation. */
grape_status grape_select_ms(double x, double tau, int32_t sigma, int32_t precision, int32_t m_max,
                             int32_t s_max, int32_t* m, int32_t* s);

/* E_A(m, s) itself (App. C Eq. (overallupperbound)); +inf when s R_m(x/s) >= 1. */
double grape_error_bound(double x, int32_t m, int32_t s, int32_t sigma, int32_t precision);

/* ---- Batches: many independent problems evaluated by one CUDA-graph launch.
 * The paper evaluates one instance at a time (Sec. III); a batch evaluates many uneven instances
 * together so that their small column teams fill the GPU.  grape_batch_create records, once, one
 * CUDA graph that evaluates every member (forward sweep, cost, backward sweep, gradient):
 *   - Work queue: members whose column teams are single CTAs in the forward and the fused backward
 *     sweep (grape_info: cluster_forward == 1 and cluster == 1; FP64 or GRAPE_FP32_BULK) become
 *     (member, column) items, ordered longest first by Taylor terms x union entries.  One launch
 *     computes all their (m, s) schedules; then ONE persistent kernel per sweep direction runs
 *     queue_ctas CTAs that take items from an atomic counter until none is left.  The CTA that
 *     completes a member's last column reduces that member's partials (cost after the forward,
 *     gradient after the backward), so no CTA waits for another.  Queued members of the
 *     three-stage kind run their fused backward there.
 *   - Lanes: every other member's own launches (cluster teams, three-stage backward) on n_streams
 *     concurrent graph branches (0 = 8), assigned longest first; the queue shares lane 0.
 * queue_ctas: 0 = automatic (from the members' timed warm evaluations: the count that balances
 * the queue's CTA-time on its CTAs against the lane members' SM-time on the SMs left), > 0 = that
 * many CTAs, < 0 = no queue (every member on the lanes).
 * u_warm: NULL, or per member NULL or HOST controls (K_i x N_i) of the warm evaluation that runs
 * before the recording (zero controls otherwise).  Three-stage members size their block buffers
 * for that evaluation's schedule, with 25% headroom; while a batch exists these buffers are not
 * replaced, and an evaluation whose schedule needs more runs that member's fused backward instead
 * (same result, slower).
 * Members must be distinct problems on one device and not tensor-core problems.  The batch does
 * not own the problems: destroy the batch before them.  The members' own cost and gradient
 * buffers are not updated by batch evaluations of queued members. */
typedef struct grape_batch grape_batch;
typedef struct {
  int32_t members;       /* problems in the batch */
  int32_t queued;        /* problems evaluated by the work-queue kernels */
  int32_t queue_items;   /* (member, column) items */
  int32_t queue_ctas;    /* CTAs of the largest work-queue launch (0: no queue) */
  int32_t lanes;         /* graph branches */
  int32_t lane_members;  /* problems evaluated by their own launches on the lanes */
} grape_batch_info_t;
grape_status grape_batch_create(grape_problem* const* probs, int32_t count, int32_t n_streams, int32_t queue_ctas,
                                const double* const* u_warm, grape_batch** out);
grape_status grape_batch_info(const grape_batch* batch, grape_batch_info_t* out);
void grape_batch_destroy(grape_batch* batch);
/* u[i]: member i's controls (K_i x N_i), costs[count], grads[i] (K_i x N_i, the array may be NULL or
 * hold NULLs).  on_device selects host or device pointers as in grape_cost_and_grad. */
grape_status grape_batch_cost_and_grad(grape_batch* batch, const double* const* u, double* costs,
                                       double* const* grads, int32_t on_device, void* stream);

/* Allocation-free propagation of one step.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory.  Such callers include code that runs
 * while a stream is being captured into a CUDA graph (cudaMalloc is not allowed there), real-time
 * loops that cannot afford cudaMalloc/cudaFree (both can synchronise the whole device), and host
 * programs that hand out all device memory from their own fixed pool.  The call computes
 *     psi_out = (e^{B}_m)^s psi_in,   B = -i dt H / s,   e^{B}_m = sum_{q=0..m} B^q / q!
 * for a dim x n_states block, column-major, and uses no memory besides the caller's buffers and a
 * 16 MiB array built into the library:
 *   - rowptr[dim+1] (int64), colind[nnz] (int32), values[2*nnz] (complex): H in CSR, DEVICE
 *     pointers.  Expected: rowptr[0] = 0, non-decreasing, rowptr[dim] = nnz.  The kernel clamps
 *     every row's entry range to [0, nnz) and skips column indices outside [0, dim), so malformed
 *     arrays give wrong numbers, never reads outside the arrays.
 *   - m in 1..60 and 1 <= s <= 4096 are taken as given (grape_select_ms gives the error-bound
 *     choice); s bounds the call's work, s * m sparse products per column.
 *   - psi_in, psi_out: dim x n_states complex DEVICE arrays (may be the same array).
 *   - Limit: 3 * dim * n_states <= 349525 (16 MiB / 48 bytes); larger requests return GRAPE_EINVAL
 *     before anything is launched.
 *   - It never calls cudaMalloc, cudaFree or any allocating library routine.  The built-in array
 *     is held on every GPU that loads the library until the process exits.
 *   - The first call on a device (make that device current) looks up the array's device address;
 *     make this first call before any stream capture begins.
 *   - Every call on a device shares the one array: calls whose GPU work overlaps (different
 *     streams, or different host threads) race and corrupt each other's results.  Serialise them.
 *     Nothing in the array needs to start at zero; it keeps the last call's contents.
 *   - Asynchronous on `stream` (NULL = legacy default stream); launch errors are returned. */
grape_status grape_taylor_step_noalloc(int64_t dim, int64_t nnz, int32_t n_states, const int64_t* rowptr,
                                       const int32_t* colind, const double* values, double dt, int32_t m, int32_t s,
                                       const double* psi_in, double* psi_out, void* stream);

const char* grape_status_string(grape_status st);
const char* grape_last_error(void);
int32_t grape_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GRAPE_HG_H */
