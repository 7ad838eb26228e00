/*
 * mor_spai.h -- C ABI of the GB300 library for the shifted-solve hot path of
 * projection-based model order reduction with reused SPAI preconditioners
 * (Singh & Ahuja, "Reusing Preconditioners in Projection based Model Order
 * Reduction Algorithms").
 *
 * Problem (Sec. II, first-order form of Algorithms 2 and 3):
 *     E x'(t) = A x(t) + B u(t),   y(t) = C^T x(t),
 * with sparse A, E (n x n), B (n x m), C (n x q).  Every solve of the method
 * is with A(sigma) = sigma E - A or its plain transpose (Algorithm 2 lines 4-5,
 * Algorithm 3 lines 4 and 10; the paper's sequence A_i X_i = F_i of Sec. III.B).
 * Second-order systems M x'' + D x' + K x = F u with D = alpha M + beta K
 * (Eq. linear-non-para, Algorithm 1) are accepted through
 * mor_set_system_2nd: their matrix s^2 M + s D + K is
 * (s^2 + alpha s) M + (1 + beta s) K, applied on the fly.
 *
 * Conventions for every entry point
 *   - Status: every function returns MOR_OK (0) or a mor_status code; on
 *     failure mor_last_error(h) returns a message owned by the library
 *     (valid until the next call on h).  No call aborts the process or traps
 *     the GPU; device-side waits are bounded.
 *   - Pointers: host pointers unless the MOR_DEVICE_PTRS flag is passed, in
 *     which case the array arguments of that call are device pointers on the
 *     handle's device, read/written in stream order on the handle's stream.
 *   - Dense arrays are column-major: an n x k block X has X[i + n*j].
 *   - Complex values are interleaved (re, im) doubles (mor_c64; the same
 *     layout as C99 double complex).
 *   - Ownership: inputs are copied (or converted) into memory the library
 *     owns; the caller may free them as soon as the call returns.  Outputs
 *     are written into caller buffers.  A handle owns all of its device
 *     memory and frees it in mor_destroy.
 *   - Thread safety: one handle must not be used by two host threads at the
 *     same time; different handles are independent.
 */
#ifndef MOR_SPAI_H
#define MOR_SPAI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mor_ctx* mor_t;

/* FP64 complex scalar (shift, eigenvalue, transfer-function value). */
typedef struct { double re, im; } mor_c64;

/* Compressed sparse row matrix, 0-based, int32 indices, FP64 values.
 * Requirements (checked, MOR_EINVAL otherwise): n > 0, rowptr[0] = 0,
 * rowptr non-decreasing, rowptr[n] = nnz, 0 <= col < n, column indices
 * strictly increasing inside each row, finite values.  A missing diagonal
 * entry is inserted as an explicit zero (the SPAI pattern needs j in J_j). */
typedef struct {
    int64_t        n;
    int64_t        nnz;
    const int32_t* rowptr;   /* n + 1 */
    const int32_t* col;      /* nnz   */
    const double*  val;      /* nnz   */
} mor_csr;

enum mor_status {
    MOR_OK = 0,
    MOR_EINVAL = 1,      /* invalid argument or malformed matrix            */
    MOR_ENOMEM = 2,      /* device or host allocation failed                 */
    MOR_ECUDA = 3,       /* a CUDA runtime call failed (message has details) */
    MOR_ENOCONV = 4,     /* a solve hit maxit; outputs hold the best iterate */
    MOR_EBREAKDOWN = 5,  /* Krylov breakdown persisted after restarts        */
    MOR_ESINGULAR = 6,   /* singular least-squares column or reduced pencil  */
    MOR_ETIMEOUT = 7,    /* a bounded device wait ran out                    */
    MOR_ESTATE = 8       /* call order violated (e.g. update before build)   */
};

/* flags */
#define MOR_DEVICE_PTRS 1u   /* array arguments of this call are device pointers */
#define MOR_REAL_VECTORS 2u  /* mor_apply_operator / mor_apply_precond: compute
                                in real arithmetic (FP64, or FP32 for MOR_MIXED)
                                on the real parts of X; Y gets zero imaginary
                                parts.  Needs real shifts (and a real chain). */

/* precision of the Krylov arithmetic */
enum mor_precision {
    MOR_FP64 = 0,   /* FP64 / complex128 throughout                               */
    MOR_MIXED = 1   /* FP32 / complex64 Krylov, matrix and preconditioner values,
                       inside FP64 iterative refinement of b - A(sigma) x          */
};

enum mor_solver {
    MOR_BICGSTAB = 0,  /* right-preconditioned BiCGSTAB (default)                  */
    MOR_GMRES = 1,     /* right-preconditioned restarted GMRES(m), m = restart: the
                          solver of the paper's experiments (Sec. IV); one system
                          only (not mor_batch_solve)                               */
    MOR_BGMRES = 2     /* right-preconditioned restarted block GMRES(m): the
                          columns of a solve that share a shift (and its chain)
                          share one block Krylov space (at most 8 columns per
                          block; columns with different shifts form separate
                          blocks); the MIMO form of the shifted solves of
                          Algorithm 2 lines 4-5.  One system only              */
};

/* sparse storage of the operator and of every preconditioner factor */
enum mor_format {
    MOR_FMT_AUTO = 0,  /* timed choice at mor_set_system (the autotuner); the
                          choice is kept for the process by pattern signature
                          (device, n, nnz, kind of E, hash of the pattern) */
    MOR_FMT_CSR = 1,   /* compressed sparse row, one thread per row      */
    MOR_FMT_SELL = 2,  /* SELL-C-sigma with C = 32, sigma = 1 (slices of 32 rows,
                          column-major inside a slice: coalesced loads)   */
    MOR_FMT_DIA = 3    /* diagonal layout: one value array per distinct
                          offset c - r, column = row + offset (no column
                          indices; values and gathers coalesced).  Only for
                          patterns with at most 32 distinct diagonals and at
                          most 25% padding (structured-grid stencils);
                          MOR_EINVAL otherwise.  The autotuner times it
                          whenever the pattern qualifies. */
};

/* Options of a solve sweep.  mor_default_opts fills the defaults shown. */
typedef struct {
    int    precision;    /* mor_precision, default MOR_MIXED                         */
    int    solver;       /* mor_solver, default MOR_BICGSTAB                         */
    double tol;          /* true relative residual ||b - A(s)x|| / ||b||, FP64, 1e-8 */
    int    maxit;        /* Krylov iterations per column, summed over refinements,
                            default 20000                                            */
    double inner_tol;    /* MOR_MIXED: relative reduction of each inner solve, 1e-4  */
    int    max_refine;   /* MOR_MIXED: FP64 refinement steps, default 10             */
    int    batch;        /* 1: all shifts of a sweep advance in one lock-step batch
                            (one matrix read serves every shift); 0: one shift at a
                            time.  Default 1                                         */
    int    use_graph;    /* 1: Krylov iterations are replayed from a captured CUDA
                            graph; 0: launched one by one.  Default 1                */
    int    graph_chunk;  /* iterations per graph replay between convergence reads,
                            default 16                                               */
    int    precond;      /* 0: reuse schedule of Algorithm 4 (default); 1: a new
                            SPAI for every shift; 2: no preconditioner               */
    int    max_chain;    /* irka_step: rebuild P_1 when the vertical chain would
                            exceed this many factors; 0 = unlimited (default)        */
    int    restart;      /* MOR_GMRES: Krylov basis size m per cycle, 1..64,
                            default 50                                               */
    int    precond_precision; /* precision of the SPAI / reuse factors that
                            mor_irka_step, mor_airga_step and precond = 1 build:
                            -1 (default) = precision; MOR_MIXED = FP32 / complex64
                            factors, which also serve MOR_FP64 solves (widened on
                            load; the preconditioner's precision does not limit
                            the solve's accuracy, and FP64 least squares are slow
                            on GPUs with a narrow FP64 pipe)                        */
    int    fp64_fallback; /* MOR_MIXED: 1 (default) = a column whose mixed-precision
                            solve fails before maxit (FP32 breakdown, an inner solve
                            that stops improving, or a refinement step that cuts
                            the FP64 residual by less than 10%) is
                            solved again from zero with FP64 Krylov iterations and
                            the same preconditioner; 0 = report the failure      */
    int    concurrent_sweeps; /* mor_irka_step(_tangential): 1 (default) = the
                            primal (V) and transposed (W) sweeps run at the same
                            time on two streams, W from a second host thread;
                            0 = one after the other from the calling thread
                            (same kernels; for tools that follow one host thread) */
    int    reuse;        /* reuse variant of the schedule (precond = 0), mor_reuse:
                            MOR_REUSE_CHAIN (default), MOR_REUSE_FIRST or
                            MOR_REUSE_AUTO                                        */
    int    moments;      /* mor_airga_step: moment blocks J per expansion point
                            (Algorithm 1 lines 7-12), 1 (default) = zeroth only  */
} mor_solve_opts;

/* Reuse variants of the preconditioner schedule (Table II, Algorithm 4). */
enum mor_reuse {
    MOR_REUSE_CHAIN = 0,  /* second approach, Algorithm 4: P_i = Q_i P_{i-1} along
                             the shifts of an iteration (horizontal), the first
                             shift's chain extended across iterations (vertical)  */
    MOR_REUSE_FIRST = 1,  /* first approach of Table II along the shifts: P_i =
                             Q_i P_1 with Q_i minimising ||A_1 - A_i Q||_F, so every
                             shift's chain is the vertical chain plus one factor;
                             vertical as MOR_REUSE_CHAIN                          */
    MOR_REUSE_AUTO = 2    /* MOR_REUSE_CHAIN with the reuse decision of the Frobenius
                             ratios of Sec. IV (Tables III / VII): a factor from
                             s_old to s_new is built only when ||A(s_old) - A(s_new)||_F
                             / ||A(s_old)||_F is below 1 and below ||I - A(s_new)||_F
                             / ||I||_F; otherwise a fresh SPAI at s_new starts a new
                             chain (the paper states no thresholds: this reading)  */
};

/* Per-column statistics of a solve. */
typedef struct {
    int    iters;        /* Krylov iterations (sum over refinement steps)  */
    int    refinements;  /* FP64 outer steps taken                          */
    double relres;       /* final true relative residual, FP64              */
    int    status;       /* mor_status of this column                       */
    int    fallback;     /* 1: solved again in FP64 after a failed mixed-
                            precision solve (iters counts both solves,
                            refinements the FP64 one)                      */
} mor_solve_stats;

#define MOR_MAX_R 64
#define MOR_MAX_IO 8

/* Reduced system (caller-allocated, fixed capacity): column-major r x r
 * pencil (A_r, E_r), B_r (r x m), C_r (r x q). */
typedef struct {
    int    r, m, q;
    double Ar[MOR_MAX_R * MOR_MAX_R];
    double Er[MOR_MAX_R * MOR_MAX_R];
    double Br[MOR_MAX_R * MOR_MAX_IO];
    double Cr[MOR_MAX_R * MOR_MAX_IO];
} mor_reduced;

/* Statistics of one IRKA iteration. */
typedef struct {
    int    z;              /* iteration index after this call (1-based)       */
    int    nsolve;         /* shifts solved (one per conjugate pair)           */
    int    builds_spai;    /* full SPAI builds done in this call               */
    int    builds_reuse;   /* reuse factors Q built in this call               */
    int    chain_len;      /* factors in the longest chain applied             */
    int    iters_V;        /* Krylov iterations, all V solves                  */
    int    iters_W;        /* Krylov iterations, all W solves                  */
    double max_relres;     /* worst true relative residual of the sweep        */
    double shift_change;   /* max_i |s_new - s_old| / |s_new|                  */
    double ms_precond, ms_solve, ms_orth, ms_reduce;  /* stage times (CUDA events) */
    int    status;
    int    fallbacks;      /* columns solved again in FP64 (fp64_fallback)     */
} mor_irka_stats;

/* ------------------------------------------------------------------------ */
/* handle                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a handle on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * the library will use for all its work (e.g. torch.cuda.current_stream()),
 * or NULL for a stream the handle creates and owns. */
int mor_create(mor_t* h, int device, void* cuda_stream);

/* Free every device and host resource of h.  h may be NULL. */
int mor_destroy(mor_t h);

/* Message of the last failed call on h (library-owned, NUL-terminated). */
const char* mor_last_error(mor_t h);

/* Fill *o with the defaults documented in mor_solve_opts. */
void mor_default_opts(mor_solve_opts* o);

/* ------------------------------------------------------------------------ */
/* system set-up                                                            */
/* ------------------------------------------------------------------------ */

/* Set the first-order system E x' = A x + B u, y = C^T x (Sec. II).
 *   A       required CSR.
 *   E       CSR of E, or NULL.
 *   E_diag  length-n diagonal of E (used when E == NULL), or NULL for E = I.
 *   B       n x m (column-major), 1 <= m <= MOR_MAX_IO.
 *   C       n x q (column-major), 1 <= q <= MOR_MAX_IO.
 *   format  mor_format of the stored operator and preconditioner factors.
 * The SPAI pattern S is the pattern of sigma E - A for generic sigma
 * (pattern(A) + pattern(E) + diagonal).  Resets every preconditioner chain
 * and the IRKA iteration counter.  Errors: MOR_EINVAL for malformed input,
 * MOR_ENOMEM, MOR_ECUDA. */
int mor_set_system(mor_t h, const mor_csr* A, const mor_csr* E, const double* E_diag,
                   const double* B, int m, const double* C, int q,
                   int format, unsigned flags);

/* Second-order system M x'' + D x' + K x = F u, y = C^T x with Rayleigh
 * damping D = alpha M + beta K (Eq. linear-non-para).  M is given by its
 * diagonal M_diag (length n).  The shifted matrix of a solve at s is
 * s^2 M + s D + K = (s^2 + alpha s) M + (1 + beta s) K.  K plays the role of
 * A's CSR (its pattern is the SPAI pattern).  Same errors as mor_set_system. */
int mor_set_system_2nd(mor_t h, const mor_csr* K, const double* M_diag,
                       double alpha, double beta,
                       const double* F, int m, const double* C, int q,
                       int format, unsigned flags);

/* n, nnz of the stored pattern, chosen format, and 1 if A(sigma)^T = A(sigma). */
int mor_get_info(mor_t h, int64_t* n, int64_t* nnz, int* format, int* symmetric);

/* Number of inputs m (columns of B, or F) and outputs q (columns of C). */
int mor_get_io(mor_t h, int* m, int* q);

/* ------------------------------------------------------------------------ */
/* preconditioner (Sec. III)                                                */
/* ------------------------------------------------------------------------ */

/* SPAI of A(sigma) (transpose = 0) or A(sigma)^T (transpose = 1) on the
 * static pattern S: the n independent column problems
 *     min || e_j - A(sigma) p_j ||_2 ,  p_j supported on J_j
 * of Eq. (gen-precond-par), each solved by Householder QR of the dense
 * |I_j| x |J_j| block (I_j = rows reached by the columns J_j) -- one warp per
 * column on the GPU.  Clears the chain of that operator and makes P the
 * first factor.  precision: MOR_FP64 (complex128 / FP64 values) or
 * MOR_MIXED (complex64 / FP32 values, the precision the inner solves use).
 * Errors: MOR_ESTATE (no system), MOR_ESINGULAR (a rank-deficient column;
 * that column of P is left zero). */
int mor_build_precond(mor_t h, mor_c64 sigma, int transpose, int precision);

/* Reuse update (Table II, second approach; Sec. III.C): with sigma_old the
 * shift of the chain's last factor, build Q minimising
 *     || A(sigma_old) - A(sigma_new) Q ||_F
 * column by column (right-hand side: column j of A(sigma_old) on I_j) and
 * append it to the chain, so that the preconditioner for sigma_new is
 * Q P_old, applied as successive mat-vecs and never formed.
 * Errors: MOR_ESTATE when no P was built for this operator/precision. */
int mor_update_precond(mor_t h, mor_c64 sigma_new, int transpose);

/* Keep only the first `length` factors of the chain (0 clears it): the
 * chain Q_L ... Q_2 P_1 of Sec. III.B cut back to Q_length ... P_1. */
int mor_truncate_precond(mor_t h, int transpose, int length);

/* Number of factors and precision of the chain (Sec. III.B, P_i = Q_i
 * P_{i-1} kept as its factors) of one operator. */
int mor_chain_info(mor_t h, int transpose, int* length, int* precision);

/* Copy factor `index` (0 = P, the SPAI of Eq. gen-precond; later ones the
 * reuse factors Q of Table II) of a chain to the caller: values (complex128,
 * nnz entries in the CSR order of the pattern returned by mor_get_pattern)
 * and the shifts it maps between (sigma_from = sigma_to for a full SPAI). */
int mor_get_factor(mor_t h, int transpose, int index, mor_c64* vals,
                   mor_c64* sigma_from, mor_c64* sigma_to);

/* CSR pattern S (transpose = 0) or S^T (transpose = 1): rowptr (n + 1) and
 * col (nnz) into caller host buffers. */
int mor_get_pattern(mor_t h, int transpose, int32_t* rowptr, int32_t* col);

/* ------------------------------------------------------------------------ */
/* kernels of the solve path, exposed one by one                            */
/* ------------------------------------------------------------------------ */

/* Y(:, c) = A(sigma_c) X(:, c), c = 0..k-1 (or the transposed operator),
 * without forming A(sigma_c): sigma E - A for first-order systems (the
 * shifted matrix of the solves of Algorithm 2, lines 4-5), (s^2 + alpha s) M
 * + (1 + beta s) K for second-order ones (Algorithm 1, line 4, with Rayleigh
 * damping D = alpha M + beta K).  X, Y: n x k complex128, column-major.
 * precision MOR_MIXED computes in FP32/complex64 (inputs rounded), MOR_FP64
 * in FP64 / complex128; with MOR_REAL_VECTORS in flags, real FP32 / FP64 on
 * the real parts of X (real shifts only).  1 <= k <= 16. */
int mor_apply_operator(mor_t h, const mor_c64* sigma, int k, int transpose, int precision,
                       const mor_c64* X, mor_c64* Y, unsigned flags);

/* Y(:, c) = P(sigma_c) X(:, c): the chain prefix that ends at the last
 * factor built for sigma_c (the whole chain when none was), applied factor
 * by factor in the chain's precision (Sec. III.B: Q_i ... Q_2 P_1 is applied
 * as successive mat-vecs, never formed; Algorithm 4).  Shapes and flags as
 * mor_apply_operator (MOR_REAL_VECTORS needs real factors). */
int mor_apply_precond(mor_t h, const mor_c64* sigma, int k, int transpose,
                      const mor_c64* X, mor_c64* Y, unsigned flags);

/* Solve A(sigma_c) X(:, c) = R(:, c) (transpose = 0) or
 * A(sigma_c)^T X(:, c) = R(:, c) (transpose = 1) for c = 0..k-1, right-
 * preconditioned (A P y = r, x = P y; Sec. III.A) with the chain prefix of
 * sigma_c (see mor_apply_precond; opts->precond = 2 solves unpreconditioned,
 * 1 builds a fresh SPAI per shift).  R: n x k complex128 right-hand sides, or
 * NULL for B(:, 0) (transpose = 0) / C(:, 0) (transpose = 1) in every column.
 * X: n x k complex128 out.  stats: k entries (may be NULL).  Returns
 * MOR_ENOCONV / MOR_EBREAKDOWN if any column failed (X holds its best
 * iterate).  1 <= k <= 64; batches of at most 16 columns advance together. */
int mor_solve_shifts(mor_t h, const mor_c64* sigma, int k, int transpose,
                     const mor_solve_opts* opts, const mor_c64* R, mor_c64* X,
                     mor_solve_stats* stats, unsigned flags);

/* Moment blocks with one matrix and one preconditioner per shift: the higher
 * moments [(s_i D - K)^{-1} D]^j (s_i D - K)^{-1} F of QB-IHOMM (Algorithm 3
 * line 4) in the first-order form of this library (D -> E, K -> A, F -> R):
 *     X_0(s_i) = A(s_i)^{-1} R,   X_j(s_i) = A(s_i)^{-1} E X_{j-1}(s_i),
 * j = 0 .. J-1, for the l shifts s_i (transpose = 1: A(s_i)^{-T} and E^T, the
 * left blocks of a two-sided projection).  X_j(s_i) = (-1)^j / j! times the
 * j-th derivative of (sE - A)^{-1} R at s_i, so projecting on the real span
 * of the blocks matches that many derivatives of H at every shift.
 *   R      n x m complex128 (host, or device with MOR_DEVICE_PTRS), or NULL for
 *          B (transpose 0) / C (transpose 1); 1 <= m <= MOR_MAX_IO, l m <= 64.
 *   X      out: n x (l J m) complex128, block (i, j) in columns
 *          (i J + j) m ... (i J + j) m + m - 1.
 *   stats  l J m entries in the same order (may be NULL).
 * The l m columns of a level advance in one lock-step batch; every level of
 * a shift is solved with the same matrix and preconditioner, which
 * opts->precond picks: 0 = the schedule's chain along the shifts (SPAI at
 * s_1, a reuse factor Q from s_{i-1} to s_i for each further shift), 1 = a
 * fresh SPAI per shift, 2 = none.  Single first-order systems only
 * (MOR_EINVAL otherwise); errors as mor_solve_shifts. */
int mor_moment_blocks(mor_t h, const mor_c64* sigma, int l, int J, int transpose,
                      const mor_solve_opts* opts, const mor_c64* R, int m, mor_c64* X,
                      mor_solve_stats* stats, unsigned flags);

/* In-place two-pass classical Gram-Schmidt (Algorithm 2 line 6, orth) of the
 * n x k FP64 block X (column-major), k <= MOR_MAX_R.  MOR_ESINGULAR if a
 * column is numerically dependent (its norm after both passes is below
 * 1e-14 of its original norm). */
int mor_orthonormalize(mor_t h, double* X, int k, unsigned flags);

/* Petrov-Galerkin reduced system of the stored first-order system in pencil
 * form (Algorithm 2 line 7): A_r = W^T A V, E_r = W^T E V, B_r = W^T B,
 * C_r = V^T C.  V, W: n x r FP64 column-major (host or device per flags);
 * rom: host struct. */
int mor_project(mor_t h, const double* V, const double* W, int r, mor_reduced* rom,
                unsigned flags);

/* Eigenvalues lambda of the reduced pencil (A_r, E_r) (r of them, on the GPU
 * in FP64: LU of E_r, Hessenberg reduction, Francis double-shift QR) and the
 * next IRKA shifts sigma_i = |Re lambda_i| - i Im lambda_i (= -lambda_i for
 * stable poles; Algorithm 2 line 3), conjugate pairs exact, sorted by
 * (Re, |Im|, -Im).  Either output may be NULL.  MOR_ESINGULAR if E_r is
 * singular or QR does not converge. */
int mor_reduced_poles(mor_t h, const mor_reduced* rom, mor_c64* lambda, mor_c64* shifts);

/* One IRKA iteration (Algorithm 2 with N_j = 0) with the reuse schedule of
 * Algorithm 4: for the solved shifts (one per conjugate pair, sorted) the
 * primal and transposed chains get, on the first call, a full SPAI at the
 * first shift; on later calls a vertical Q from the previous first shift;
 * and a horizontal Q for every further shift.  Then V and W solves
 * (A(s_i) v_i = B, A(s_i)^T w_i = C, SISO), real bases [Re v, Im v],
 * Gram-Schmidt, projection, reduced poles and new shifts.
 *   shifts  in: r current shifts (closed under conjugation); out: next shifts
 *   rom     out (may be NULL); st out (may be NULL).
 * SISO form: MOR_EINVAL unless m = q = 1 (MIMO: mor_irka_step_tangential).
 * Errors as mor_solve_shifts; MOR_EINVAL if r > MOR_MAX_R or the shift set
 * is not closed under conjugation. */
int mor_irka_step(mor_t h, mor_c64* shifts, int r, const mor_solve_opts* opts,
                  mor_reduced* rom, mor_irka_stats* st);

/* One tangential IRKA iteration for a MIMO system (Algorithm 2 lines 3-7
 * with N_j = 0, the directions of its line 3 read on the pencil) with the
 * reuse schedule of mor_irka_step: v_i = (s_i E - A)^{-1} B b_i and
 * w_i = (s_i E - A)^{-T} C c_i at the solved shifts, real bases, CGS2,
 * projection, then the next shifts and directions: for the pole lambda_i of
 * E_r^{-1} A_r = R Lambda R^{-1}, b_i = row i of R^{-1} E_r^{-1} B_r and
 * c_i = column i of C_r^T R (eigenvectors by inverse iteration on the GPU,
 * FP64).
 *   shifts  in/out as in mor_irka_step.
 *   btil    r x m complex, row-major: row i is b_i of shifts[i] (in/out).
 *   ctil    r x q complex, row-major: row i is c_i (in/out).
 * On return the rows follow the sorted new shifts and the -Im member of a
 * conjugate pair carries the conjugate directions.  The scale of b_i and c_i
 * is that of the eigenvectors; only the products c_i b_i^T are invariant.
 * Errors as mor_irka_step. */
int mor_irka_step_tangential(mor_t h, mor_c64* shifts, mor_c64* btil, mor_c64* ctil, int r,
                             const mor_solve_opts* opts, mor_reduced* rom, mor_irka_stats* st);

/* Reduced second-order system (caller-allocated, fixed capacity): M_r =
 * V^T M V and K_r = V^T K V (r x r, column-major), D_r = alpha M_r + beta K_r,
 * F_r = V^T F (r x m), C_r = V^T C (r x q). */
#define MOR_MAX_R2 32
typedef struct {
    int    r, m, q;
    double alpha, beta;
    double Mr[MOR_MAX_R2 * MOR_MAX_R2];
    double Kr[MOR_MAX_R2 * MOR_MAX_R2];
    double Fr[MOR_MAX_R2 * MOR_MAX_IO];
    double Cr[MOR_MAX_R2 * MOR_MAX_IO];
} mor_reduced2;

/* One iteration of the second-order reduction (AIRGA, Algorithm 1) of a
 * system set by mor_set_system_2nd, with the reuse schedule of mor_irka_step
 * on s^2 M + s D + K: block solves X^(0)(s_i) = (s_i^2 M + s_i D + K)^{-1} F
 * at the points with Im >= 0 (one lock-step column per (point, input)); then,
 * for opts->moments = J > 1, the inner moment loop of lines 7-12 for a fixed
 * J (its H2 stopping test is not taken): V_j = X^(j-1) / ||X^(j-1)||_F per
 * point and X^(j) = -(s_i^2 M + s_i D + K)^{-1} M V_j with the same matrix
 * and the same chain; V = CGS2 of [Re X^(j), Im X^(j)] (per point and block),
 * Galerkin M_r, K_r, D_r, F_r, C_r (Sec. II), and the point update, which
 * the paper leaves unstated (line 11), read as: the mirror images
 * |Re lambda| - i Im lambda of the eigenvalues of the reduced quadratic
 * eigenproblem (companion pencil, FP64 on the GPU) of smallest modulus, as
 * many as before, closed under conjugation (a pair only when two places are
 * left; a last single place with only pairs to come takes the real point
 * |lambda| of the first pair that did not fit).
 *   points  in: l expansion points (closed under conjugation); out: the next
 *           l points, sorted (Re, |Im|, -Im).
 *   r = m J l must not exceed MOR_MAX_R2.  rom, st: out (may be NULL);
 *   st->iters_V sums the block solves' iterations, st->nsolve counts the
 *   solved columns of all J blocks.
 * MOR_EINVAL for a first-order system, a batch, r > MOR_MAX_R2 or
 * precond = 1; otherwise errors as mor_irka_step. */
int mor_airga_step(mor_t h, mor_c64* points, int l, const mor_solve_opts* opts,
                   mor_reduced2* rom, mor_irka_stats* st);

/* H_r(i omega_w) = C_r^T ((i w)^2 M_r + i w D_r + K_r)^{-1} F_r of a reduced
 * second-order system (the reduced system of Sec. II's Galerkin projection)
 * for nw frequencies; layout and flags as mor_eval_tf. */
int mor_eval_tf2(mor_t h, const mor_reduced2* rom, const double* omega, int nw,
                 mor_c64* H, unsigned flags);

/* Restart the reuse schedule (the next mor_irka_step is iteration 1 of
 * Algorithm 4: a full SPAI at the first shift). */
int mor_irka_reset(mor_t h);

/* H_r(i omega_w) = C_r^T (i omega_w E_r - A_r)^{-1} B_r for nw frequencies
 * (the reduced transfer function whose error Sec. IV plots over s = i omega,
 * Fig. 3; on the GPU, one block per frequency, FP64 complex LU with partial
 * pivoting).  H: nw x q x m complex128, H[w + nw*(iq + q*im)].  omega and H are
 * host arrays unless flags has MOR_DEVICE_PTRS. */
int mor_eval_tf(mor_t h, const mor_reduced* rom, const double* omega, int nw,
                mor_c64* H, unsigned flags);

/* ------------------------------------------------------------------------ */
/* batches of independent systems                                           */
/* ------------------------------------------------------------------------ */

/* Set nsys independent SISO first-order systems E_s x' = A_s x + b_s u,
 * y = c_s^T x of uneven sizes n_s as one batch (replacing any system of h).
 * They are stored as one block-diagonal operator whose blocks keep separate
 * Krylov scalars and convergence: every reduction of a solve is per
 * (system, shift) (Eq. gen-precond-par's column independence also keeps
 * every SPAI column inside its own block).  A: nsys CSR matrices (host);
 * E_diag: NULL (all E_s = I) or nsys pointers (each NULL for I, or a
 * length-n_s diagonal); B, C: nsys pointers to length-n_s vectors.  The
 * preconditioner calls (mor_build_precond, mor_update_precond) then act on
 * all systems at once with the same shift.  Host pointers only
 * (MOR_DEVICE_PTRS is rejected).  Errors as mor_set_system. */
int mor_set_batch(mor_t h, int nsys, const mor_csr* A, const double* const* E_diag,
                  const double* const* B, const double* const* C, int format, unsigned flags);

/* Number of systems of the batch (independent problems of the solve
 * sequence of Sec. III.A, one segment each) and its row offsets (nsys + 1 entries;
 * system s owns rows offsets[s] .. offsets[s+1]-1 of the batch). */
int mor_batch_info(mor_t h, int* nsys, int64_t* offsets);

/* Solve A_s(sigma_c) x_{s,c} = b_s (transpose = 0) or A_s(sigma_c)^T
 * x_{s,c} = c_s (transpose = 1) for every system s of the batch and every
 * shift c = 0..k-1 (the right-preconditioned solves of Sec. III.A, each
 * system with its own chain factors of Sec. III.B), all in the same lock-step launches (the shift columns of
 * all systems advance together; each (system, shift) pair converges on its
 * own relative residual).  Preconditioning, precision and options as in
 * mor_solve_shifts.  X: N x k complex128 column-major over the batch rows
 * (N = offsets[nsys]); stats: nsys x k entries, stats[s * k + c] (may be
 * NULL).  1 <= k <= 64. */
int mor_batch_solve(mor_t h, const mor_c64* sigma, int k, int transpose, const mor_solve_opts* opts,
                    mor_c64* X, mor_solve_stats* stats, unsigned flags);

/* ------------------------------------------------------------------------ */
/* measurement                                                              */
/* ------------------------------------------------------------------------ */

/* Number of CUDA kernels this library has executed in the process so far
 * (graph replays count every kernel node they run).  Process-wide. */
int mor_launch_count(int64_t* count);

/* Launches of one SpMV kernel since the process started, by width:
 *   which     0 operator SpMV, 1 preconditioner-factor SpMV;
 *   vec_type  vector type: 0 FP32, 1 FP64, 2 complex64, 3 complex128;
 *   counts    MOR_KMAX_COLS + 1 entries out; counts[k] = launches over k real
 *             (non-padding) shift columns (graph replays count every
 *             recorded launch).  Process-wide. */
#define MOR_KMAX_COLS 16
int mor_kernel_tally(int which, int vec_type, int64_t* counts);

/* Time one hot-loop kernel of the solve exactly as the inner BiCGSTAB
 * iteration launches it, with CUDA events on the handle's stream:
 *   which = 0   operator SpMV  Y = A(sigma_c) X over k columns;
 *   which = 1   one factor SpMV Y = F X over k columns (the chain's last
 *               factor of the vectors' kind: complex values when any sigma_c
 *               is complex, else real ones, else the last factor; requires a
 *               built preconditioner).
 * precision selects FP32/complex64 (MOR_MIXED) or FP64 vectors; complex
 * vectors are used when any sigma_c is complex.  `reps` launches are timed
 * after 3 untimed ones, each after a read of twice the L2 size (no launch
 * finds the previous one's data in L2); launches and flushes run back to
 * back between one pair of events and the time of the flushes alone is
 * subtracted, so *ms, the mean per launch, is the kernel's duration plus one
 * inter-kernel gap.  The input vectors are resident device buffers of n x k
 * entries. */
int mor_time_kernel(mor_t h, int which, const mor_c64* sigma, int k, int precision, int reps,
                    double* ms);

/* ------------------------------------------------------------------------ */
/* allocation-free entry point (no counterpart in the paper)                */
/* ------------------------------------------------------------------------ */

/* The same two-pass Gram-Schmidt as mor_orthonormalize (orth of Algorithm 2,
 * line 6), for callers that
 * cannot let a library allocate device memory: frameworks whose own caching
 * allocator holds the whole device budget, real-time or embedded loops that
 * must keep a fixed memory map, and code that must not pay the implicit
 * device synchronisation of cudaMalloc / cudaFree.  It needs no handle and
 * allocates nothing: its scratch is one fixed array of 313,088 bytes that
 * the library reserves on every GPU that loads it, until the process exits.
 *   X       device pointer, n x k FP64, column-major, orthonormalised in
 *           place on the current CUDA device.
 *   n       1 <= n <= 2^31 - 1;  k: 1 <= k <= 64 (MOR_EINVAL beyond).
 *   stream  cudaStream_t for the work (NULL = the legacy default stream);
 *           the call returns once the work is enqueued.
 * The first call on a device looks up the scratch's device address (keep
 * that first call outside any stream capture).  All calls share the one
 * scratch array, so calls whose work overlaps on the GPU (other streams,
 * other host threads) race: serialise them.  No dependency check is made --
 * a numerically dependent column comes out non-finite; use
 * mor_orthonormalize to have it reported.  Returns MOR_OK, MOR_EINVAL or
 * MOR_ECUDA. */
int mor_orthonormalize_noalloc(double* X, int64_t n, int k, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MOR_SPAI_H */
