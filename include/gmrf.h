/*
 * gmrf.h -- C ABI of the GB300 Krylov GMRF sampler and Lanczos log-determinant.
 *
 * The operations follow Simpson, Turner, Strickland and Pettitt, "Scalable
 * iterative methods for sampling from massive Gaussian random vectors":
 *
 *   gmrf_create  -- a precision matrix Q given matrix-free as a lattice
 *                   stencil with a coefficient field (Section 2: Q is never
 *                   formed, only Q v is computed), optionally with the
 *                   constant-coefficient preconditioner M of Section 5.1
 *                   (Theorem 2) used through Proposition 1.
 *   gmrf_sample  -- x_m ~= Q^{-1/2} z by the Lanczos sampler (Section 4,
 *                   Algorithm 1), m chosen adaptively from the a-posteriori
 *                   bound of Theorem 1 (eq. krylov_bound).
 *   gmrf_create_sparse -- a general sparse Q in CSR, optionally with an
 *                   incomplete-Cholesky factor as the preconditioner
 *                   (Section 5.2); gmrf_ichol computes that factor.
 *   gmrf_logdet  -- log det Q by the Hutchinson estimator with Rademacher
 *                   probes and Lanczos (Gauss) quadrature (Section 6), with
 *                   the preconditioned split of Section 6.2
 *                   (log det Q = log det(F^-1 Q F^-T) + log det M).
 *
 * Operator family (unit lattice spacing, graph Laplacian L):
 *   GMRF_OP_SHIFTED_LAPLACIAN  Q = tau (K + L)      5-point 2-D / 7-point 3-D
 *   GMRF_OP_SPDE_SQUARED       Q = tau (K + L)^2    13-point 2-D
 * with K = diag(kappa^2(s)).  Boundary: periodic (torus), cell-centred
 * Neumann (a boundary cell counts only neighbours inside the grid) or
 * Dirichlet (zero outside the grid).  Cell (z, y, x) has index
 * x + nx*(y + ny*z).  Vectors of a batch are stored one after another:
 * element i of vector s is at [s*n + i] ("[nvec][n]" layout).
 *
 * Memory: every pointer argument may be host memory or device memory of the
 * current device (detected with cudaPointerGetAttributes).  The caller keeps
 * ownership of everything it passes; the library copies kappa2 during
 * gmrf_create and owns its own workspaces (Lanczos basis, scalars,
 * transform tables), which gmrf_destroy frees.
 *
 * Streams: all device work of a problem is issued on the stream given to
 * gmrf_create (NULL = the legacy default stream).  Every call returns after
 * its results are complete (it synchronises that stream).
 *
 * Errors: 0 = GMRF_OK, otherwise a negative code below; gmrf_strerror maps a
 * code to a static string.  On GMRF_ERR_NOT_CONVERGED the sample is still
 * written (with the last subspace size) and each info record carries its own
 * status and error estimate.  A problem must not be used from two threads at
 * once; different problems may be used from different host threads
 * concurrently, and their device work then overlaps.
 */
#ifndef GMRF_H
#define GMRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GMRF_OK 0
#define GMRF_ERR_INVALID (-1)       /* bad dimensions, kappa2 < 0 or not finite, tol <= 0, ... */
#define GMRF_ERR_OOM (-2)           /* device memory for one vector's Lanczos state not available */
#define GMRF_ERR_NOT_CONVERGED (-3) /* m_max reached before the stopping rule held */
#define GMRF_ERR_NOT_SPD (-4)       /* a non-positive pivot of T_m: Q (or A) is not SPD */
#define GMRF_ERR_NUMERIC (-5)       /* NaN or Inf during the iteration */
#define GMRF_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define GMRF_ERR_TIMEOUT (-7)       /* a device-side wait ran out of its iteration budget */
#define GMRF_ERR_UNSUPPORTED (-8)   /* a valid combination this library does not implement */

typedef struct gmrf_problem gmrf_problem; /* opaque, library-owned */

typedef enum { GMRF_BC_PERIODIC = 0, GMRF_BC_NEUMANN = 1, GMRF_BC_DIRICHLET = 2 } gmrf_bc;

typedef enum {
  GMRF_OP_SHIFTED_LAPLACIAN = 0, /* tau (K + L) */
  GMRF_OP_SPDE_SQUARED = 1,      /* tau (K + L)^2, 2-D only */
  GMRF_OP_SPDE_PLUS_DIAG = 2     /* tau ((kappa_c^2 I + L)^2 + D), 2-D only: a stationary (block-circulant
                                    on a torus) prior plus a non-negative diagonal, e.g. the Fisher
                                    information of the LGCP sMMALA proposal (Section 3; Section 5.1,
                                    Table 1).  kappa_c^2 = kappa2_const (> 0 unless Dirichlet);
                                    D = diag(kappa2 field), entries >= 0 (NULL: D = 0).
                                    Preconditioned by the prior itself, M = tau (kappa_c^2 + L)^2, so
                                    A = I + M^{-1/2} (tau D) M^{-1/2}; that needs matched boundaries
                                    (PERIODIC with CIRCULANT, NEUMANN with MIRROR) and
                                    kappa2_precond <= 0 or equal to kappa2_const. */
} gmrf_op;

/* Preconditioner M (Proposition 1 with F = M^{1/2}; Section 5.1):
 *   NONE      -- plain Algorithm 1 on Q;
 *   CIRCULANT -- M = the same operator with constant kappa_bar^2 on the
 *                grid's own torus (block circulant, applied by 2-D FFT);
 *   MIRROR    -- M = the same operator with constant kappa_bar^2 on the
 *                mirror-extended torus, i.e. the cell-centred Neumann
 *                operator, applied by 2-D DCT-II (an FFT of the reflected
 *                grid).
 * Preconditioning needs dim == 2 and power-of-two nx, ny in [8, 4096].  FP64
 * problems with 4096-point lines are supported only where the preconditioner
 * matches the boundary (CIRCULANT with periodic, MIRROR with Neumann: no
 * boundary correction terms); otherwise gmrf_create returns
 * GMRF_ERR_UNSUPPORTED. */
typedef enum { GMRF_PREC_NONE = 0, GMRF_PREC_CIRCULANT = 1, GMRF_PREC_MIRROR = 2 } gmrf_precond;

/* Vector arithmetic of the Krylov iteration.  FP32: vectors, stencil and
 * transforms in FP32, dot products in compensated FP32 (pairs of floats)
 * finished in FP64, alpha/beta, T_m and quadrature in FP64.  FP64:
 * everything in FP64. */
typedef enum { GMRF_FP32 = 0, GMRF_FP64 = 1 } gmrf_precision;

typedef struct {
  int32_t dim;       /* 2 or 3 */
  int32_t bc;        /* gmrf_bc */
  int32_t op;        /* gmrf_op */
  int32_t precond;   /* gmrf_precond */
  int64_t nx, ny, nz;  /* grid extents (nz ignored for dim == 2); each >= 2 */
  const float* kappa2; /* [n] coefficient field, host or device; NULL => kappa2_const */
  double kappa2_const; /* used when kappa2 == NULL */
  double tau;          /* precision scale, > 0 */
  double kappa2_precond; /* constant kappa_bar^2 of M; <= 0 => exp(mean log kappa2) */
  int32_t precision;   /* gmrf_precision */
  int32_t reserved;    /* must be 0 */
} gmrf_desc;

/* Storage of the Lanczos basis V_m that the assembly x_m = ||z|| V_m y reads
 * (Algorithm 1, last step).
 *   NATIVE -- the vector precision (FP32 or FP64);
 *   BF16   -- FP32 problems only: v_j is also rounded to bfloat16 into a
 *             basis copy of (m_max + 1) * n * 2 bytes per vector, and the
 *             FP32 basis keeps only v_{j-1} and v_j for the recurrence.  The
 *             iteration (alpha, beta, m, the stopping rule) is bitwise the
 *             same as with NATIVE; x_m carries the bfloat16 rounding of V_m,
 *             about 1e-3 relative, instead of reaching tol.  Halves the
 *             memory of V_m, so more vectors or larger m fit in HBM.  FP64
 *             problems return GMRF_ERR_UNSUPPORTED.  The paper stores V_m
 *             at working precision; this is an option of this library. */
/*   NONE   -- no basis kept: two passes.  The first runs the iteration with
 *             only v_{j-1}, v_j and finds alpha, beta, m and y; the second
 *             runs the same iteration again (bitwise the same, from the same
 *             z) and adds ||z|| y_j v_j to x after every step.  x_m is
 *             bitwise the one NATIVE returns; device memory per vector is
 *             O(n) instead of (m_max + 1) n, for twice the steps.  Not in the
 *             paper; an option of this library. */
typedef enum { GMRF_VSTORE_NATIVE = 0, GMRF_VSTORE_BF16 = 1, GMRF_VSTORE_NONE = 2 } gmrf_vstore;

typedef struct {
  double tol;          /* relative tolerance of the Theorem 1 estimate, > 0 */
  int32_t m_max;       /* largest subspace size, >= 1 */
  int32_t nsamples;    /* number of vectors z (>= 1) */
  uint64_t seed;       /* Philox-4x32-10 key for z when z_in == NULL */
  const void* z_in;    /* optional [nsamples][n] noise, float (FP32) or double (FP64), host or device */
  int32_t check_every; /* steps between host polls of the convergence flags (<= 0: 16) */
  int32_t v_storage;   /* gmrf_vstore: storage of the basis V_m kept for the assembly */
} gmrf_sample_opts;

typedef struct {
  int32_t m_used;  /* subspace size of the returned vector */
  int32_t status;  /* GMRF_OK, GMRF_ERR_NOT_CONVERGED, GMRF_ERR_NOT_SPD or GMRF_ERR_NUMERIC */
  double err_est;  /* relative Theorem 1 estimate at m_used (0 after an exact breakdown) */
} gmrf_result_info;

typedef struct {
  double tol;          /* same stopping rule as gmrf_sample, per probe */
  int32_t m_max;
  int32_t nprobes;     /* N >= 1 (>= 2 for a standard error) */
  uint64_t seed;       /* Philox key of the Rademacher probes when probes_in == NULL */
  const void* probes_in; /* optional probes (float / double by precision): [nprobes * ncolours][n] */
  int32_t check_every;
  int32_t colour_dist;  /* p >= 0: coloured Hutchinson estimator (Section 6.1) over the distance-p
                           lattice colouring colour = coords mod (p + 1), ncolours = (p + 1)^dim;
                           0 = plain Hutchinson (one colour) */
} gmrf_logdet_opts;

/* Section 2 / 5.1: build a problem.  Validates the descriptor, copies kappa2,
 * builds the preconditioner's spectral tables.  stream: a cudaStream_t or
 * NULL.  *out receives the handle. */
int gmrf_create(const gmrf_desc* desc, void* stream, gmrf_problem** out);

/* Number of cells n of a problem. */
int gmrf_size(const gmrf_problem* p, int64_t* n);

/* Section 4, Algorithm 1 (+ Proposition 1 when preconditioned): writes
 * x_out [nsamples][n] (float for FP32, double for FP64; host or device) and
 * info [nsamples] (host, may be NULL).  Returns the worst per-vector status. */
int gmrf_sample(gmrf_problem* p, const gmrf_sample_opts* opts, void* x_out, gmrf_result_info* info);

/* Section 6 (+ Section 6.2 when preconditioned): N = nprobes Rademacher
 * draws v_d.  With colour_dist = p > 0 (Section 6.1) each draw is split over
 * the ncolours colour classes c, v_dc = v_d on c and 0 elsewhere (the
 * device stream of draw d is the one of plain probe d), so the library runs
 * N * ncolours Lanczos quadratures, ordered draw-major.  With
 * Q_d = sum_c q_dc (Q_d = q_d for p = 0):
 * *logdet = mean_d Q_d + log det M + n log tau, *std_err = sd(Q_d)/sqrt(N)
 * (NaN for N == 1), q_out [N * ncolours] (host, may be NULL) = the terms
 * q_dc = ||v_dc||^2 e_1^T log(T_m) e_1 of the (preconditioned) operator,
 * info [N * ncolours] as for gmrf_sample.  logdet and std_err are host
 * pointers.  GMRF_ERR_INVALID for colour_dist < 0 or > 15. */
int gmrf_logdet(gmrf_problem* p, const gmrf_logdet_opts* opts, double* logdet, double* std_err,
                double* q_out, gmrf_result_info* info);

/* Sections 4 and 6 in one Lanczos batch: the nsamples samples of sample_opts
 * (Algorithm 1) and the nprobes * ncolours log-det probes of logdet_opts run
 * as one block of vectors through the same step kernels (many z vectors and
 * Hutchinson probes per launch), samples first.  Every output is bitwise the
 * one of the separate calls gmrf_sample(sample_opts) and
 * gmrf_logdet(logdet_opts) with the same seeds or inputs: the arithmetic of a
 * vector does not depend on the rest of its batch.  Both option sets must
 * have the same tol and m_max, and sample_opts.v_storage must be NATIVE
 * (otherwise GMRF_ERR_INVALID); sample_opts.check_every is used.  Outputs as
 * for the two calls (x_out, sample_info [nsamples]; logdet, std_err host
 * pointers; q_out, probe_info [nprobes * ncolours], may be NULL).  Returns the
 * worst status over all vectors; GMRF_ERR_OOM when one vector does not fit. */
int gmrf_sample_logdet(gmrf_problem* p, const gmrf_sample_opts* sample_opts, const gmrf_logdet_opts* logdet_opts,
                       void* x_out, gmrf_result_info* sample_info, double* logdet, double* std_err, double* q_out,
                       gmrf_result_info* probe_info);

typedef struct {
  double tol;          /* relative residual at which an iteration stops, > 0 (see gmrf_solve) */
  int32_t m_max;       /* largest subspace size (CG steps), 1 .. 8192 */
  int32_t nrhs;        /* number of right-hand sides (>= 1) */
  int32_t check_every; /* steps between host polls of the convergence flags (<= 0: 16) */
  int32_t reserved;    /* must be 0 */
} gmrf_solve_opts;

/* Section 5.1: x = Q^{-1} b, the linear solve of the sMMALA proposal mean
 * (Q + H)^{-1} grad log pi(y | x), run by the same Lanczos iteration and
 * the same preconditioner as the sampler ("one preconditioner ... both
 * problems").  The iteration is the Lanczos form of conjugate gradients:
 * from v_1 = b / ||b|| it builds V_m and T_m exactly as Algorithm 1 and
 * returns x_m = ||b|| V_m T_m^{-1} e_1 (T_m^{-1} in place of T_m^{-1/2}).
 * With a preconditioner M = tau B_bar^p (Proposition 1's factor
 * F = M^{1/2}) it solves A u = M^{-1/2} b with A = M^{-1/2} Q M^{-1/2} and
 * returns x = M^{-1/2} u.
 *
 * Stopping rule: the relative residual of the iterated system,
 * ||r_m|| / ||b~|| = beta_m |e_m^T T_m^{-1} e_1| <= tol, with b~ = b
 * (no preconditioner; r_m = b - Q x_m scaled by 1/tau) or
 * b~ = M^{-1/2} b (r_m the residual of A u = b~), from the LDL^T recurrence
 * of the stopping rule of gmrf_sample.  info[k].err_est is that relative
 * residual; info[k].m_used the number of steps.
 *
 * b and x: [nrhs][n] of the problem's precision (float for FP32, double for
 * FP64), host or device, must not overlap; b is not modified.  info [nrhs]
 * (host, may be NULL).  Returns the worst per-right-hand-side status
 * (GMRF_OK, GMRF_ERR_NOT_CONVERGED with x_m at m_max written,
 * GMRF_ERR_NOT_SPD, GMRF_ERR_NUMERIC); GMRF_ERR_INVALID for a bad option;
 * GMRF_ERR_OOM when one right-hand side does not fit in device memory.
 * A zero right-hand side gives x = 0 with status GMRF_OK and m_used = 0. */
int gmrf_solve(gmrf_problem* p, const gmrf_solve_opts* opts, const void* b, void* x, gmrf_result_info* info);

/* Asynchronous calls.  gmrf_submit_sample / _logdet / _solve queue the call
 * with the same arguments as the synchronous function and return at once with
 * a ticket (> 0); a host worker thread owned by the library (one per problem,
 * started at its first submit, on the device current at that submit) runs the
 * problem's submitted calls in submission order, each exactly as the
 * synchronous call, on the problem's stream.  The option struct is copied at
 * submit; every buffer it or the call names (x_out, info, z_in, probes_in, b,
 * logdet, std_err, q_out) belongs to the caller and must stay valid and
 * untouched until the ticket has completed.  While calls are outstanding the
 * problem must not be used by synchronous calls.  Calls on different problems
 * run concurrently.  gmrf_destroy runs what was submitted, then frees.
 * Submit returns GMRF_ERR_INVALID for NULL p, opts or ticket (other argument
 * errors are the completed call's result).
 *   gmrf_poll: *done = 1 once the call has completed, and then *result (may be
 *   NULL) = its return code; non-blocking.
 *   gmrf_wait: blocks until the call has completed; *result (may be NULL) =
 *   its return code.
 * Both return GMRF_ERR_INVALID for a ticket this problem did not issue.
 * The paper's method has no counterpart: this is the call form a serving layer
 * needs to keep several problems' iterations in flight from one host thread. */
int gmrf_submit_sample(gmrf_problem* p, const gmrf_sample_opts* opts, void* x_out, gmrf_result_info* info,
                       int64_t* ticket);
int gmrf_submit_logdet(gmrf_problem* p, const gmrf_logdet_opts* opts, double* logdet, double* std_err,
                       double* q_out, gmrf_result_info* info, int64_t* ticket);
int gmrf_submit_solve(gmrf_problem* p, const gmrf_solve_opts* opts, const void* b, void* x, gmrf_result_info* info,
                      int64_t* ticket);
int gmrf_poll(gmrf_problem* p, int64_t ticket, int32_t* done, int32_t* result);
int gmrf_wait(gmrf_problem* p, int64_t ticket, int32_t* result);

/* ---- Continuous-batching server --------------------------------------------
 * The samples of Algorithm 1 and the probes of Section 6 are independent
 * Lanczos runs, so the vectors of many requests can share every launch.  A
 * server keeps the Lanczos state of `nslots` vectors of one problem resident
 * on the device (bases V_m, alpha/beta, per-vector state) and runs one CUDA
 * graph of check_every steps over all slots per gmrf_server_step.  Between
 * replays it admits waiting vectors into free slots (requests first come,
 * first served; a request may be admitted a part at a time while other slots
 * are in mid-iteration), and finishes each vector as soon as it stops: a
 * sample gets T_m^{-1/2} e_1, x = ||z|| V_m y (then M^{-1/2}) and the
 * accuracy check of gmrf_sample, a probe its quadrature term.  A request is
 * complete when its last vector is; a log det then gets the reduction of
 * gmrf_logdet over its probes.  The paper's method has no server; this is the
 * serving pattern of this library.
 *
 * Results: every result is bitwise the one the synchronous calls return for
 * the same request: a sample request (kind 0, count vectors, seed, tau) gives
 * the x and info of gmrf_sample(nsamples = count, seed, z_in = NULL,
 * v_storage NATIVE) on a problem whose tau is this problem's tau times the
 * request's tau; a log-det request (kind 1, count probes) gives the logdet,
 * std_err and info of gmrf_logdet(nprobes = count, seed, colour_dist 0) on
 * such a problem.  tol, m_max and check_every are the server's.
 *
 * While a server exists the problem serves it alone: the problem's other
 * calls return GMRF_ERR_INVALID until gmrf_server_destroy (gmrf_destroy
 * destroys an attached server first).  One host thread at a time per server.
 * Device memory: the Lanczos buffers of nslots vectors at m_max, allocated by
 * gmrf_server_create (GMRF_ERR_OOM if they do not fit), plus per-call
 * workspaces of the finishing steps. */
typedef struct gmrf_server gmrf_server; /* opaque, library-owned */
typedef struct {
  int32_t nslots;      /* vectors resident at once, 1 .. 65535 */
  int32_t m_max;       /* largest subspace size per vector, 1 .. 8192 */
  double tol;          /* stopping tolerance of every vector (gmrf_sample's rule), > 0 */
  int32_t check_every; /* steps per gmrf_server_step (<= 0: 16) */
  int32_t reserved;    /* must be 0 */
} gmrf_server_opts;
int gmrf_server_create(gmrf_problem* p, const gmrf_server_opts* opts, gmrf_server** out);
/* Queues a request (no device work for samples; a log det allocates its
 * [count + 2] result array).  kind 0: count samples into x_out, device memory
 * [count][n] of the problem's precision that must stay valid until the request
 * has completed; kind 1: a log det with count Rademacher probes (x_out
 * ignored).  tau > 0 scales the precision (see Results).  *req receives the
 * request id.  GMRF_ERR_INVALID for a bad kind, count < 1, tau <= 0 or a host
 * x_out. */
int gmrf_server_submit(gmrf_server* sv, int32_t kind, int32_t count, uint64_t seed, double tau, void* x_out,
                       int64_t* req);
/* Admits, runs one replay of check_every steps over all slots, finishes what
 * stopped, completes requests.  *active (may be NULL) = vectors running or
 * waiting afterwards (0: idle).  Synchronises the problem's work stream. */
int gmrf_server_step(gmrf_server* sv, int32_t* active);
/* *done = 1 once request req has completed; then *result (may be NULL) = its
 * worst per-vector status, info [count] (host, may be NULL) the per-vector
 * records, *logdet / *std_err (may be NULL) its log-det estimate (kind 1), and
 * the request is forgotten.  GMRF_ERR_INVALID for an unknown id. */
int gmrf_server_poll(gmrf_server* sv, int64_t req, int32_t* done, int32_t* result, gmrf_result_info* info,
                     double* logdet, double* std_err);
void gmrf_server_destroy(gmrf_server* sv);

/* Matrix-free operator applies on nvec vectors of the problem's precision
 * (Section 2's "routine that computes the matrix-vector product"), for
 * testing and for callers composing their own solvers:
 *   which = 0: y = Q v
 *   which = 1: y = A v, A = M^{-1/2} Q M^{-1/2} (Proposition 1; needs a preconditioner)
 *   which = 2: y = M^{-1/2} v                  (needs a preconditioner)
 * v and y are [nvec][n], host or device, must not overlap. */
int gmrf_apply(gmrf_problem* p, int32_t which, int64_t nvec, const void* v, void* y);

/* Device Philox-4x32-10 streams (the z of Algorithm 1 and the probes of
 * Section 6), [nvec][n]:
 *   kind 0 = N(0,1) (float if precision == GMRF_FP32, else double),
 *   kind 1 = Rademacher +-1 (same types),
 *   kind 2 = the raw 32-bit words of the Gaussian stream ([nvec][4*ceil(n/4)] uint32).
 * out: host or device; stream: cudaStream_t or NULL. */
int gmrf_rng(int32_t kind, int32_t precision, int64_t nvec, int64_t n, uint64_t seed, void* out,
             void* stream);

/* Tracing (a build facility, not a step of the paper's method): launch counts
 * and CUDA-event timing of the library's kernels by class, for profiling and
 * the roofline report.  Classes: 0 fused stencil step, 1 preconditioned
 * row-forward, 2 column transform, 3 row-mid, 4 row-last, 5 ||z||, 6 Philox,
 * 7 T_m functions, 8 assembly, 9 plain preconditioner applies, 10 other,
 * 11 sparse (CSR) Lanczos step.
 *   op 0: reset counters and times;  op 1: enable event timing (events are
 *   recorded around every launch on its stream);  op 2: disable timing;
 *   op 3: query class kclass (-1 = all): *total_ms = summed kernel time,
 *   *launches = kernel launches, *timed = launches that were timed.
 * Process-wide and thread-safe (counts and times of all threads are summed);
 * any output pointer may be NULL. */
int gmrf_trace(int32_t op, int32_t kclass, double* total_ms, int64_t* launches, int64_t* timed);

/* Allocation-free y = M^{-1/2} v (the operation of gmrf_apply with which = 2).
 * The paper has no counterpart.  It exists for callers that must not allocate
 * device memory while they call into this library: applications that hand
 * all device memory to their own pool or allocator up front and forbid
 * allocations behind its back (an allocation outside the pool can fail, or
 * push a tight memory budget over its limit), and latency-critical loops that
 * cannot afford the synchronisation and latency of an allocation.
 * gmrf_apply may grow the problem's transform workspace with cudaMalloc on
 * first use; this entry point calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * Its transform scratch is one library-wide static device array of
 * GMRF_NOALLOC_SCRATCH_BYTES (32 MiB), held on every GPU that loads the
 * library until the process exits.  A call needs nvec * ny * (nx + 2) *
 * (4 for FP32, 8 for FP64) bytes of it; larger requests return
 * GMRF_ERR_INVALID (a 1024 x 1024 FP32 grid fits 7 vectors per call).
 * v and y: device pointers, [nvec][n] of the problem's precision; host
 * pointers return GMRF_ERR_INVALID.  The problem needs a preconditioner.
 * The device the problem was created on must be the current device
 * (otherwise GMRF_ERR_INVALID).  The call returns once y is complete.
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents; nothing in it needs to start at zero,
 * because every call overwrites the part it reads.  Calls whose GPU work
 * overlaps -- from different problems, streams or host threads -- race on
 * the array and must be serialised by the caller.  With kernel tracing
 * enabled (gmrf_trace op 1) the library still creates CUDA events, which are
 * not device memory. */
#define GMRF_NOALLOC_SCRATCH_BYTES (32 << 20)
int gmrf_apply_inv_sqrt_noalloc(gmrf_problem* p, int64_t nvec, const void* v, void* y);

/* Tuning of the batched Lanczos launches (a facility of this library, not
 * part of the paper's method).
 *   block_width -- vectors per Lanczos launch (one batch of the SpMM-like
 *                  step); 0 = as many as fit in free HBM;
 *   zchunk      -- 3-D FP32 Dirichlet / zero-Neumann grids without a
 *                  preconditioner: z planes per work item of the TMA-staged
 *                  stencil step; 0 = the default for the grid; ignored
 *                  elsewhere.
 * A zchunk changes how the step's dot products are grouped, so results can
 * change in the last bits; they stay independent of the batch. */
typedef struct {
  int32_t block_width;
  int32_t zchunk;
  double vec_steps_per_s; /* gmrf_autotune: measured rate of the chosen configuration */
  int32_t candidates;     /* gmrf_autotune: configurations timed */
  int32_t host_loop;      /* 0 (default): with launch timing off, the Lanczos
                           * steps of a call run as one graph launch whose
                           * conditional WHILE node repeats a step until no
                           * vector is running (one host wait per call);
                           * 1: the host replays graphs of check_every steps
                           * and reads the vector states between them (the
                           * mode for per-kernel profilers).  Results are
                           * bitwise the same.  gmrf_autotune leaves it as
                           * set; other values are GMRF_ERR_INVALID. */
} gmrf_tuning;

/* Times short Lanczos runs (8 untimed + 8 timed steps on Rademacher vectors,
 * CUDA events on the problem's work stream) over the candidate z chunks
 * (nz, nz/2, ... >= 8 planes) at a block width of min(16, cap), then over
 * the block widths 1, 2, 4, ... and the largest that fits free HBM
 * (<= nvec_max), and keeps the smallest block width within 3% of the best
 * rate.  The choice is stored in the problem (used by later gmrf_sample /
 * gmrf_logdet calls) and returned in *out.  Synchronises the work stream.
 * Errors: GMRF_ERR_INVALID (null pointers, nvec_max < 1), GMRF_ERR_OOM,
 * GMRF_ERR_CUDA. */
int gmrf_autotune(gmrf_problem* p, int32_t nvec_max, gmrf_tuning* out);

/* Sets the tuning explicitly (e.g. one found by gmrf_autotune on another
 * problem with the same grid).  GMRF_ERR_INVALID for negative fields or a
 * host_loop other than 0 or 1. */
int gmrf_set_tuning(gmrf_problem* p, const gmrf_tuning* t);

/* ---- General sparse Q with an incomplete-Cholesky preconditioner ----------
 * Section 5.2 proposes the incomplete Cholesky factor F of a general sparse Q
 * (F lower triangular and sparse, F F^T close to Q) as the preconditioner
 * M = F F^T of Proposition 1, so that
 *     x = tau^{-1/2} F^{-T} A^{-1/2} z,     A = F^{-1} Q F^{-T},
 *     log det(tau Q) = log det A + 2 sum_i log F_ii + n log tau   (Section 6.2),
 * with A^{-1/2} z and the quadrature of log A from Algorithm 1 on A.  Figure 3
 * runs it on (31^2 G)^2, G the 5-point Dirichlet Laplacian of a 30 x 30
 * lattice, for factors with several drop thresholds.
 *
 * gmrf_sparse_desc (all arrays are host memory, copied by gmrf_create_sparse):
 *   n                     dimension, >= 1
 *   rowptr[n+1], colind[nnz], val[nnz]
 *                         Q in CSR with both triangles; rowptr[0] = 0 and
 *                         non-decreasing; columns in [0, n), no duplicates
 *                         within a row, any order; Q must be symmetric
 *                         (value Q_ij == Q_ji exactly) with a positive diagonal
 *   f_rowptr, f_colind, f_val
 *                         F in CSR, or f_rowptr == NULL for no preconditioner
 *                         (Algorithm 1 on Q itself); every entry has column
 *                         <= row, every row has a positive diagonal entry
 *   tau                   precision scale (> 0): the problem is tau Q
 *   precision             gmrf_precision of the vectors and of the copies of
 *                         Q and F the kernels use (FP32 rounds them to float)
 *   reserved              must be 0
 *
 * A sparse problem supports gmrf_sample (v_storage GMRF_VSTORE_NATIVE only,
 * otherwise GMRF_ERR_UNSUPPORTED), gmrf_logdet and gmrf_sample_logdet
 * (colour_dist 0 only: the coloured probes of Section 6.1 need the lattice),
 * gmrf_solve (x = tau^{-1} F^{-T} A^{-1} F^{-1} b), the asynchronous forms,
 * gmrf_size, gmrf_autotune and gmrf_set_tuning, and gmrf_apply with
 *   which = 0: y = tau Q v
 *   which = 1: y = A v = F^{-1} Q F^{-T} v      (needs F)
 *   which = 2: y = tau^{-1/2} F^{-T} v          (needs F; the map from
 *              A^{-1/2} z to the sample, the role M^{-1/2} has on lattices).
 * gmrf_apply_inv_sqrt_noalloc returns GMRF_ERR_UNSUPPORTED.
 *
 * Device design: one thread block per vector keeps that vector's working
 * vectors in shared memory for a whole Lanczos step; the products with Q
 * read Q's CSR arrays from L2, and the triangular solves with F and F^T run
 * level by level (the rows of one level depend only on earlier levels and
 * are solved in parallel).  Hence n is limited by the shared memory of one
 * block: 3 n elements of the precision must fit in the device's opt-in
 * limit less 2 KiB (about n <= 18,000 in FP32, 9,000 in FP64 on a GPU with
 * 227 KiB); larger n returns GMRF_ERR_UNSUPPORTED.
 *
 * Errors: GMRF_ERR_INVALID for NULL desc/out/rowptr/colind/val, n < 1, a
 * malformed or asymmetric Q, a non-positive diagonal, an F entry above the
 * diagonal or a missing / non-positive F diagonal, non-finite values,
 * tau <= 0, reserved != 0; GMRF_ERR_UNSUPPORTED for n above the limit;
 * GMRF_ERR_OOM, GMRF_ERR_CUDA. */
typedef struct {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* val;
  const int64_t* f_rowptr;
  const int32_t* f_colind;
  const double* f_val;
  double tau;
  int32_t precision;
  int32_t reserved;
} gmrf_sparse_desc;
int gmrf_create_sparse(const gmrf_sparse_desc* desc, void* stream, gmrf_problem** out);

/* Threshold incomplete Cholesky factor F of A' = Q + shift diag(Q) (Section
 * 5.2), host code only (no device work, callable without a GPU).  Column j =
 * 0 .. n-1, left-looking:
 *     w = A'[j:, j] - F[j:, :j] F[j, :j]^T,   F_jj = sqrt(w_0),
 *     F_ij = w_i / F_jj (i > j), kept unless
 *       droptol <  0 (IC(0)):  A'_ij == 0      (no fill outside Q's pattern)
 *       droptol >= 0 (ICT):    |w_i| < droptol * sum_{i >= j} |A'_ij|
 * (the paper gives no dropping rule; this one does not depend on the scale
 * of Q); entries that are exactly zero are not stored.  droptol = 0 gives
 * the exact Cholesky factor, a very large droptol the diagonal
 * sqrt(diag A').  Q: CSR as in gmrf_sparse_desc.
 * Output F in CSR: f_rowptr[n+1], and per row its columns ascending with the
 * diagonal last, in f_colind / f_val.
 *   Size query: with f_colind == NULL or f_val == NULL only *f_nnz (and
 *   f_rowptr, if not NULL) are written.  Otherwise cap is the capacity of
 *   f_colind and f_val; a factor with more entries returns GMRF_ERR_INVALID
 *   with *f_nnz set and nothing else written.
 * Errors: GMRF_ERR_INVALID (NULL rowptr/colind/val/f_nnz, malformed or
 * asymmetric Q, non-finite values, shift < 0 or not finite, droptol NaN);
 * GMRF_ERR_NOT_SPD for a pivot w_0 <= 0, with *f_nnz = the column where it
 * occurred (a larger shift usually cures it); GMRF_ERR_OOM for host memory. */
int gmrf_ichol(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double droptol,
               double shift, int64_t cap, int64_t* f_rowptr, int32_t* f_colind, double* f_val, int64_t* f_nnz);

void gmrf_destroy(gmrf_problem* p);
const char* gmrf_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GMRF_H */
