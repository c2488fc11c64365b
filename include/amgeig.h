/*
 * amgeig.h -- C ABI of the GB300 (sm_103a) solve phase of the algebraic
 * multigrid multilevel-correction eigensolver of Zhang, Han, He, Xie and You,
 * "An Algebraic Multigrid Method for Eigenvalue Problems in Some Different
 * Cases" (arXiv:1503.08462).
 *
 * Problem (Sec. 1, Eq. eigenvalue_problem): find the q smallest eigenpairs
 * (lambda_j, u_j) of A u = lambda M u with A sparse SPD and M sparse SPD, and
 * u_j^T M u_k = delta_jk.  The AMG hierarchy of Sec. 2 (levels A_k, M_k and
 * prolongations I_{k+1}^k) is built once on the host and handed over as a
 * serialized blob; this library runs Algorithm 3.2 (AMG Eigenvalue Solver)
 * with Algorithm 3.1 (AMG Correction Step) on the GPU.
 *
 * Conventions for every entry point:
 *   - return value: AMGEIG_OK (0) or a negative AMGEIG_E* code; no call aborts
 *     the process.  amgeig_strerror() names a code; amgeig_last_error() gives a
 *     one-line description of the most recent failure on the calling thread.
 *   - caller buffers are read (or written) only during the call; the library
 *     keeps no pointer to them.
 *   - dense blocks of vectors are row-major N x q: entry (i, j) of vector j is
 *     at index i * q + j.
 *   - level 0 is the paper's finest level 1; level n-1 its coarsest level n.
 */
#ifndef AMGEIG_H
#define AMGEIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define AMGEIG_OK 0
#define AMGEIG_EINVAL (-1)   /* invalid argument (NULL pointer, q out of range, ...) */
#define AMGEIG_ECORRUPT (-2) /* hierarchy blob fails validation (magic, checksum, bounds) */
#define AMGEIG_ENOMEM (-3)   /* device allocation failed or admission refused */
#define AMGEIG_ENOTSPD (-4)  /* a Cholesky factorisation met a non-positive pivot */
#define AMGEIG_ENOCONV (-5)  /* max_corrections reached; outputs are still written */
#define AMGEIG_ENAN (-6)     /* a NaN or Inf appeared in the iterates */
#define AMGEIG_ECUDA (-7)    /* CUDA runtime error (see amgeig_last_error) */
#define AMGEIG_ENOTFOUND (-8) /* unknown request id */

/* ---- precision of the V-cycle ------------------------------------------- */
#define AMGEIG_FP64 0       /* every step in float64 */
#define AMGEIG_MIXED_FP32 1 /* V-cycle (smoothing, transfers, coarse solve) in float32;
                               defect, Rayleigh-Ritz, Gram/cross blocks and the
                               recombination in float-float (48-bit significand) */
#define AMGEIG_MIXED_BF16 2 /* as AMGEIG_MIXED_FP32, with the V-cycle's operators (A_l, R_l,
                               P_l) stored in bfloat16 and applied with float32
                               accumulation; the defect keeps the exact A */

typedef struct amgeig_hierarchy_t* amgeig_hierarchy;

/* Solver options.  Defaults (amgeig_default_options) follow Sec. 4.1 except the
 * smoother: one V-cycle (m = 1) with one pre- and one post-smoothing sweep of
 * point l1-Jacobi (the paper smooths with Gauss-Seidel), n1 = n, p_k = 1 on the
 * intermediate levels and at most 20 corrections on the finest level. */
typedef struct {
  int max_corrections;   /* finest-level corrections at most (p_1 <= 20, Sec. 4.1) */
  int v_cycles;          /* m, V-cycles per AMG call (Eq. inexact_inverse_iter), >= 1 */
  int pre_sweeps;        /* l1-Jacobi sweeps before the coarse correction, >= 0 */
  int post_sweeps;       /* l1-Jacobi sweeps after the coarse correction, >= 0 */
  int q_extra;           /* extra eigenpairs carried along (Sec. 4, Examples 4-6), >= 0 */
  int precision;         /* AMGEIG_FP64, AMGEIG_MIXED_FP32 or AMGEIG_MIXED_BF16 */
  int fixed_corrections; /* > 0: run exactly this many finest-level corrections and
                            ignore tol (iteration-level parity mode) */
  int coarse_modes;      /* 0: the pencil of Algorithm 3.1 step 2 uses all of V_n (the
                            paper's method).  m > 0: only the m lowest eigenvectors of
                            the coarsest pencil (A_n, M_n) span its coarse part (an
                            option of this library: the pencil shrinks from d_n + q to
                            m + q; the fixed point, the exact eigenpairs, is unchanged) */
  int smoother;          /* AMGEIG_SMOOTHER_L1_JACOBI (default) or AMGEIG_SMOOTHER_GAUSS_SEIDEL:
                            the paper's Gauss-Seidel (Sec. 4.1) in a multicolour ordering --
                            rows coloured first-fit in row order, colours ascending before the
                            coarse correction and descending after it (a symmetric V-cycle);
                            the colouring is computed on the first such solve */
  int n1;                /* initial level of Algorithm 3.2 step 1, 0-based (level 0 the finest):
                            -1 (default) = the coarsest level with at least q + q_extra rows (the
                            paper's n1 = n whenever the coarsest level is large enough, Sec. 4.1);
                            otherwise a level with q + q_extra <= N_n1 <= 2048.  The initial
                            eigenproblem (A_n1, M_n1) is solved densely on the GPU; the pencils
                            of every correction still use the coarsest space V_n */
  int refine;            /* 0 (default): the eigenvalues are the last Rayleigh-Ritz step's values.
                            1: after the last correction each vector's Rayleigh quotient
                            u^T A u / u^T M u and relative residual are recomputed in float64 with
                            the exact operator values (for the mixed path, whose Ritz data use A
                            and M rounded to 48 bits); 2: the same with the quotient's sums
                            accumulated in compensated float64 (as if in twice the precision),
                            so that the returned eigenvalues are those of the returned vectors
                            to a few units of float64 rounding, where plain float64 sums lose
                            ~u * lambda_max / lambda_j to cancellation.  With 1 or 2 the values are
                            sorted ascending and the vectors permuted alike */
  int graphs;            /* 1 (default): the nested phase and each finest-level correction are
                            captured as CUDA graphs (per settings and buffer roles) the second time
                            they run, and replayed from then on; 0: every kernel launched directly.
                            Same arithmetic, same bits.  Not used while profiling is enabled or
                            when the caller's stream is capturing */
  int autotune;          /* mixed precisions: 1 (default) = the first solve at each block width times
                            every lane layout of the float32 smoothing and transfer kernels on each
                            level's operators (lanes per row, columns per lane, nonzero streams per
                            row) and keeps the fastest in the hierarchy; layouts with another stream
                            count add a row's terms in another order (float32 rounding in the
                            V-cycle; later solves on the hierarchy repeat bit for bit); the choices
                            are also kept for the process, keyed by each operator's role, size and
                            nonzero count, so a hierarchy of the same problem loaded again reuses
                            them without timing; 0 = no tuning now (layouts tuned by earlier solves
                            stay in use) */
  int batch;             /* amgeig_submit only: 1 (default) = the request may share one solve with
                            other queued requests on the same hierarchy whose options agree but for
                            q, q_extra, tol and max_corrections (the shared solve takes the widest
                            and the tightest of each; every request receives its own leading q
                            pairs and its own residual test); 0 = always solved on its own */
  double shift;          /* sigma of a shifted inner solve (the remark after Algorithm 3.1): 0
                            (default) = the paper's step 1; otherwise step 1 runs its V-cycles on
                            (A_k - sigma M_k) u~ = (lambda_j - sigma) M_k u_j from u_j, on the
                            hierarchy of A_l - sigma M_l (made on the GPU for the last sigma used;
                            the defect is unchanged, lambda M u - A u).  sigma must lie below the
                            lowest eigenvalue of (A_n, M_n) (EINVAL otherwise); with the
                            l1-Jacobi smoother only, not with AMGEIG_MIXED_BF16 */
  int krylov;            /* depth s of the correction space (the remark after Algorithm 3.1, "V_n +
                            Krylov spaces"): 1 (default) = the paper's V_n + span(V); 2 = V_n +
                            span(T U, T^2 U), T the step's inexact inverse iteration (m V-cycles on
                            the defect with the step's Ritz values), the pencil on the block
                            [T U | T^2 U - T U] of 2 (q + q_extra) columns; needs 2 (q + q_extra) <=
                            128, and q + q_extra <= 32 on the mixed paths (EINVAL otherwise) */
} amgeig_options;

#define AMGEIG_SMOOTHER_L1_JACOBI 0
#define AMGEIG_SMOOTHER_GAUSS_SEIDEL 1

/* Per-solve report. */
typedef struct {
  int corrections;   /* finest-level corrections performed */
  int converged;     /* 1 if max_j relres_j <= tol */
  int n1;            /* initial level (0-based) */
  int status;        /* AMGEIG_OK or the error code of the solve */
  double max_relres; /* max_j ||A u_j - lambda_j M u_j||_2 / (|lambda_j| ||M u_j||_2), j < q */
  int dense_fallbacks; /* corrections (all levels) whose small pencil needed the dense eigensolver
                          because the Rayleigh quotient iteration's result failed its check */
} amgeig_info;

/* Fill *opt with the defaults above.  opt must not be NULL. */
void amgeig_default_options(amgeig_options* opt);

/* Load a serialized hierarchy (layout: the writer in the package's
 * inputs/hierarchy.py; magic "AMGEIGH1", u64 checksum trailer) onto CUDA device
 * `device`.  blob: host pointer to `bytes` bytes, read during the call only.
 * The library copies every level (A_k, M_k in one shared-pattern CSR, P_k and
 * its transpose R_k = P_k^T, Sec. 2.3) to the device, derives the l1-Jacobi
 * diagonals and float32 copies, builds the composite prolongations I_n^k, and
 * factors the coarsest level on the GPU (the exact coarse solve of the V-cycle).
 * The M_n-orthonormal eigenbasis of the coarsest pencil (A_n, M_n), used by
 * step 1 of Algorithm 3.2 and by every correction, is computed on the GPU by the
 * first solve that needs it, only its leading modes (all d_n with coarse_modes
 * = 0), and kept for later solves.  On success *out owns all device memory of
 * the hierarchy until amgeig_free_hierarchy.  Errors: EINVAL (NULL argument,
 * bad device), ECORRUPT (validation), ENOMEM, ENOTSPD (A_n or M_n not SPD),
 * ECUDA. */
int amgeig_load_hierarchy(const void* blob, size_t bytes, int device, amgeig_hierarchy* out);

/* As amgeig_load_hierarchy, and also computes the `modes` lowest eigenpairs of
 * the coarsest pencil (A_n, M_n) (Algorithm 3.2 step 1) during the load: the
 * coarsest level is uploaded, factored and decomposed on a second stream while
 * the host validates and converts the finer levels, so a first solve whose
 * pencil needs at most `modes` coarse modes (coarse_modes <= modes and q +
 * q_extra <= modes) starts without computing them.  modes = 0 or modes > d_n:
 * all d_n modes (the paper's pencil, coarse_modes = 0).  The modes are the same
 * bits a first solve would compute on its own with that count.  Errors: as
 * amgeig_load_hierarchy; EINVAL also for modes < 0. */
int amgeig_load_hierarchy_modes(const void* blob, size_t bytes, int device, int modes, amgeig_hierarchy* out);

/* Release every device and host resource of h.  NULL is accepted.  Pending
 * requests on h must have been polled to completion first (EINVAL otherwise). */
int amgeig_free_hierarchy(amgeig_hierarchy h);

/* Level count and per-level sizes: n_levels receives n; sizes (may be NULL)
 * receives min(n, max_sizes) row counts N_0 >= ... >= N_{n-1}. */
int amgeig_hierarchy_info(amgeig_hierarchy h, int* n_levels, int64_t* sizes, int max_sizes);

/* Algorithm 3.2 with Algorithm 3.1 on the GPU.
 *   q         number of wanted eigenpairs, 1 <= q, q + q_extra <= min(128, N_0).
 *             The initial eigenproblem (Algorithm 3.2 step 1) is solved on level
 *             n1 (options.n1; by default the coarsest level with at least
 *             q + q_extra rows), which must hold at most 2048 rows when it is
 *             not the coarsest; EINVAL otherwise.
 *   tol       stopping test max_j relres_j <= tol on the finest level (the paper
 *             stops on the total error against reference eigenvalues, Sec. 4.1,
 *             which a solver cannot know).
 *   opt       options, NULL for defaults.
 *   eigvals   host buffer of q doubles: the q smallest Ritz values, ascending.
 *   eigvecs   buffer of N_0 * q doubles, row-major N_0 x q: M-orthonormal vectors,
 *             each signed so that its largest-magnitude entry (lowest index on
 *             ties) is positive.  Device pointer if eigvecs_on_device != 0, host
 *             pointer otherwise; NULL skips the vectors.
 *   info      report (may be NULL).
 *   stream    cudaStream_t to run on (NULL: the library's own stream).  The call
 *             returns after the results are in the caller's buffers.
 * Errors: EINVAL, ENOMEM, ENOTSPD (the Gram block of the augmented pencil is not
 * SPD), ENAN, ECUDA.  ENOCONV when max_corrections ran out: eigvals, eigvecs and
 * info are still written. */
int amgeig_solve(amgeig_hierarchy h, int q, double tol, const amgeig_options* opt, double* eigvals,
                 double* eigvecs, int eigvecs_on_device, amgeig_info* info, void* stream);

/* Serving: queue a solve on h and return at once with *request_id.  The options
 * are copied.  Four library threads take requests in arrival order, skipping
 * one whose hierarchy is already solving: requests on different hierarchies run
 * at the same time on their hierarchies' streams, and queued requests on the
 * taken request's hierarchy join its solve (options.batch) when their width
 * fits its workspace.  Each hierarchy keeps its
 * iterate workspace resident (sized for the widest q + q_extra it has served).
 * A request whose workspace does not fit in free device memory waits until a
 * running request ends (ENOMEM is reported through amgeig_poll if it cannot fit
 * with nothing else running).  Errors: EINVAL. */
int amgeig_submit(amgeig_hierarchy h, int q, double tol, const amgeig_options* opt, uint64_t* request_id);

/* Poll a request.  *done = 0 while it is queued or running.  Once done, copies
 * the q eigenvalues (host, may be NULL), the N_0 x q eigenvectors (host, may be
 * NULL) and the report (may be NULL), releases the request and returns its
 * status (AMGEIG_OK, ENOCONV, ...).  Errors: ENOTFOUND for an unknown or already
 * released id. */
int amgeig_poll(uint64_t request_id, int* done, double* eigvals, double* eigvecs, amgeig_info* info);

/* Serving: cap the device memory the request service keeps in iterate
 * workspaces (the workspaces of hierarchies it has served stay resident between
 * requests).  bytes = 0 (the default): no cap beyond free device memory.  Under
 * a cap, a request whose workspace does not fit first releases the workspaces
 * of idle hierarchies, least recently used first; if it still does not fit it
 * waits for running requests to end, and a request whose workspace alone
 * exceeds the cap (or that cannot fit with nothing else running) ends with
 * ENOMEM, reported by amgeig_poll.  Takes effect for the next admission
 * decision.  Returns AMGEIG_OK. */
int amgeig_service_set_memory_limit(uint64_t bytes);

/* Serving: the bytes the service's resident workspaces hold now, and how many
 * workspaces it has released to admit other requests so far (either pointer
 * may be NULL, not both).  Errors: EINVAL. */
int amgeig_service_memory(uint64_t* resident_bytes, uint64_t* evictions);

/* ---- AMG setup ------------------------------------------------------------ */

/* Build the AMG hierarchy of Sec. 2 for the pencil (A, M), A and M given as one
 * shared-pattern CSR (host arrays: rp int32[n+1], ci int32[nnz], a and m
 * float64[nnz]), and return it as a hierarchy blob for amgeig_load_hierarchy.
 * Per level: strength theta on the negative couplings (Sec. 2.1; 0.25 in
 * Sec. 4.1) and the classical Ruge-Stueben C/F splitting on the host; direct
 * interpolation (Eqs. Interpolation_Def, Interpolation_Dir) and the Galerkin
 * products A_{k+1} = P^T A_k P, M_{k+1} = P^T M_k P (Eq. Coarse_Matrices) on
 * device `device`; levels until the coarsest has at most coarse_cap rows or
 * max_levels are made.  The same hierarchy as the package's host setup
 * (inputs/hierarchy.py): identical levels, splittings and sparsity patterns,
 * values equal up to the rounding of sums taken in another order.
 *   blob, bytes   receive a library-allocated host buffer (free it with
 *                 amgeig_free_blob) and its size.
 *   seconds       may be NULL; else seconds[0] = the whole setup, seconds[1] =
 *                 its host C/F splitting.
 * Errors: EINVAL (NULL argument, bad CSR, theta outside (0, 1), bad device),
 * ENOMEM (allocation), ECUDA. */
int amgeig_setup_blob(int64_t n, const int32_t* rp, const int32_t* ci, const double* a, const double* m,
                      double theta, int64_t coarse_cap, int max_levels, int device, void** blob, size_t* bytes,
                      double* seconds);

/* Release a blob returned by amgeig_setup_blob (NULL is accepted). */
void amgeig_free_blob(void* blob);

/* ---- building blocks, exposed for verification -------------------------- */

/* The nwant smallest eigenpairs of the symmetric n x n matrix H (host, row-major,
 * float64), computed on device `device` by the solver's own dense eigensolver
 * (the black-box eigensolver of Algorithm 3.1 step 2: Householder
 * tridiagonalisation, Sturm bisection, inverse iteration and a Rayleigh-Ritz
 * clean-up, in float-float arithmetic).  evals: host, nwant doubles ascending;
 * evecs: host, n x nwant row-major, orthonormal columns.  1 <= nwant <= n <= 2048.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int amgeig_sym_eigh(int device, int n, int nwant, const double* H, double* evals, double* evecs);

/* The defect of Algorithm 3.1 step 1 (the right-hand side of the correction
 * equation, Eq. Linear_Equation): r_j = lambda_j M_l u_j - A_l u_j on level
 * `level` of h, with the relative residuals ||A u_j - lambda_j M u_j||_2 /
 * (|lambda_j| ||M u_j||_2) from the same pass.  U (N_l x width, row-major) and
 * lam (width) are host inputs; R (N_l x width) and relres (width, may be NULL)
 * host outputs.  The options' precision selects the float64 kernel or the
 * mixed path's float-float kernel, whose defect is rounded to float32 (the
 * V-cycle's right-hand side).  1 <= width <= 128.  Errors: EINVAL, ENOMEM,
 * ECUDA. */
int amgeig_apply_defect(amgeig_hierarchy h, int level, int width, const amgeig_options* opt, const double* U,
                        const double* lam, double* R, double* relres);

/* One AMG V-cycle for A_l x = b from x = 0 on level `level` of h (Algorithm
 * 3.1 step 1 with the options' pre/post l1-Jacobi sweeps and precision): b and
 * x are host buffers of N_l x width doubles (row-major), 1 <= width <= 128.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int amgeig_apply_vcycle(amgeig_hierarchy h, int level, int width, const amgeig_options* opt, const double* b,
                        double* x);

/* Allocation-free form of amgeig_sym_eigh, for callers that cannot allocate
 * device memory when they need it (work inside a foreign memory pool, code that
 * must not synchronise the device as cudaFree does, hosts whose allocator
 * belongs to another runtime).  The paper has no counterpart: it treats the
 * small eigenproblems as a black box.
 *   n, nwant  1 <= nwant <= n, n <= 128, nwant <= 64 (EINVAL beyond).
 *   H         device pointer, n x n row-major float64, symmetric.
 *   evals     device pointer, nwant doubles (ascending).
 *   evecs     device pointer, n x nwant row-major float64.
 *   stream    cudaStream_t (NULL: the legacy default stream).
 * The call only enqueues work on `stream` (no synchronisation, no cudaMalloc,
 * cudaFree or allocating library call).  Its scratch is one file-scope device
 * array of 512 KiB that every GPU loading the library holds until exit; the
 * first call on a device looks the array's device address up with
 * cudaGetSymbolAddress, so make that first call outside any stream capture.
 * All calls share the array and it keeps the last call's contents (the solver
 * writes every scratch element before reading it); calls that overlap on the
 * GPU race on it and must be serialised by the caller.
 * Errors: EINVAL, ECUDA. */
int amgeig_sym_eigh_noalloc(int n, int nwant, const double* H, double* evals, double* evecs, void* stream);

/* ---- measurement ---------------------------------------------------------- */

/* The launch-shape tuner's choices on h so far, as JSON text: a list of
 * {"level", "kernel" (smooth | restrict | prolong), "w4" (block width in float4
 * columns), "G" (lanes per row), "cpt" (float4 columns per lane), "S" (streams
 * the row's nonzeros are split over: G / S lanes each; set by the rule, kept by
 * the tuner), "us" (its time), "rule_G", "rule_cpt", "rule_us" (the fixed
 * rule's shape and time)}.
 * Errors: EINVAL (NULL argument, buffer too small; the text is truncated). */
int amgeig_tuning_report(amgeig_hierarchy h, char* buf, size_t len);

/* Per kernel class totals recorded while profiling is enabled. */
typedef struct {
  char name[24];    /* kernel class: defect, smooth, transfer, coarse_solve, augment,
                       gram, pencil, recombine, other */
  int64_t launches; /* timed launch scopes */
  int64_t kernels;  /* kernels inside those scopes */
  double total_ms;  /* sum of CUDA-event durations, recorded on the launching stream */
  double bytes;     /* algorithmic HBM bytes of those launches (each operand moved once) */
  double flops;     /* algorithmic floating-point operations of those launches */
} amgeig_prof_entry;

/* Enable (1; clears the table) or disable (0) CUDA-event timing of every launch
 * of this library in this process.  Timing adds two event records per launch.
 * Returns AMGEIG_OK. */
int amgeig_profile_enable(int enable);

/* Synchronise on the recorded events and write up to max_entries per-class
 * totals (classes with no launches are skipped) into out, followed by the
 * classes of the V-cycle per level (names "<class>@<level>", levels 0-based);
 * *n_entries receives the count.  Errors: EINVAL, ECUDA. */
int amgeig_profile_read(amgeig_prof_entry* out, int max_entries, int* n_entries);

/* Cumulative number of kernels this library has launched in this process. */
uint64_t amgeig_kernel_launches(void);

/* Static description of a status code. */
const char* amgeig_strerror(int code);

/* Description of the last failure on the calling thread ("" if none). */
const char* amgeig_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMGEIG_H */
