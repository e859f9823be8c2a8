/*
 * sfgmres.h -- C ABI of the GB300 sketched-FGMRES solver.
 *
 * The library solves A x = b for a large sparse nonsymmetric A in CSR form (Section 1 of Guettel & Pearson,
 * "Stabilizing randomized GMRES through flexible GMRES") by FGMRES (Algorithm 1) whose variable preconditioner is
 * one cycle of sketched GMRES (Eq. 3; Section 3): a truncated-Arnoldi Krylov basis (Section 4.1), a seeded
 * sparse-sign subspace embedding S (Eq. 1), and the sketched least-squares problem solved through a Gram-Schmidt QR
 * with reorthogonalisation, with the inner length chosen by the stop rules C1-C3 of Section 3 (C3 uses the
 * residual bound of Eq. 5 and the FFOM residual of Eq. 4).
 *
 * Every step of the solve runs in this library's CUDA kernels (sm_103a).  The library uses the CUDA runtime only
 * for memory, streams and events; it has no CPU fallback.
 *
 * Conventions
 *  - Parameter names follow the paper's inner notation through this mapping: `m` = maximum inner sGMRES basis size
 *    (the paper's k_max, rule C1), `k` = Arnoldi truncation depth (the paper's t), `s` = sketch rows (m <= s << n).
 *  - Return values: 0 (SFGMRES_OK) on success, positive values for numerical outcomes that still leave a valid
 *    result, negative values for errors; sfgmres_last_error() then describes the error.
 *  - Pointers: "device" means memory the current CUDA device can address (cudaMalloc, torch CUDA tensors);
 *    "host" means ordinary or pinned host memory.  Where an argument accepts both, the library inspects the
 *    pointer with cudaPointerGetAttributes and stages host data through device buffers it owns.
 *  - A handle is bound to the device that was current at sfgmres_create and to one CUDA stream; calls on one
 *    handle must not overlap in time (the handle owns the workspaces).  Different handles are independent.
 *  - Every call that launches kernels returns only after its work has completed on the handle's stream.
 */
#ifndef SFGMRES_H
#define SFGMRES_H

#include <stdint.h>

#if defined(__GNUC__)
#define SFGMRES_API __attribute__((visibility("default")))
#else
#define SFGMRES_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------------------------ */
#define SFGMRES_OK 0               /* converged: ||b - A x|| <= tol * ||b|| (recomputed, not estimated) */
#define SFGMRES_NOT_CONVERGED 1    /* outer budget exhausted; x holds the last FGMRES iterate (still valid) */
#define SFGMRES_BREAKDOWN 2        /* an inner cycle produced no correction (first sketched column zero);
                                      x holds the last FGMRES iterate */
#define SFGMRES_ERR_INVALID_ARG (-1)
#define SFGMRES_ERR_CUDA (-2)
#define SFGMRES_ERR_OOM (-3)
#define SFGMRES_ERR_NAN (-4)       /* NaN or Inf met in b, x0 or a reduction */

/* ---- sfgmres_create flags ---------------------------------------------------------------------------------- */
#define SFGMRES_CSR_HOST 1         /* row_ptr/col_idx/vals are host pointers (default: device pointers) */

/* ---- option keys for sfgmres_set_option / sfgmres_get_option ---------------------------------------------- */
#define SFGMRES_OPT_PRECISION 1      /* inner-cycle precision: 0 = FP64 (default), 1 = FP32 values/basis/sketch
                                        with FP32 accumulation, 2 = as 1 with the basis stored in BF16.  The outer
                                        FGMRES, the sketched QR and least squares, z = B y and the residual
                                        recomputation are FP64 in every mode. */
#define SFGMRES_OPT_ZETA 2           /* nonzeros per sketch column, 1..16 (default 8; 1 = Clarkson-Woodruff) */
#define SFGMRES_OPT_COND_THRESHOLD 3 /* rule C2 threshold on the condition proxy of S A B_k (default 1e15) */
#define SFGMRES_OPT_C3 4             /* rule C3 (Eq. 5 bound stops the inner cycle): 1 = on (default), 0 = off */
#define SFGMRES_OPT_MAX_OUTER 5      /* outer FGMRES iteration budget (default 50) */
#define SFGMRES_OPT_SKETCH_KIND 6    /* 0 = sparse-sign (default), 1 = identity (requires s == n; tests) */
#define SFGMRES_OPT_PROFILE 7        /* 1 = time the kernels with CUDA events around every launch, 2 = time each
                                        inner cycle's chain of step launches with one pair of events (see
                                        sfgmres_stats), default 0 */
#define SFGMRES_OPT_SPMV_VECTOR 8    /* lanes per CSR row in the SpMV (2,4,8,16,32), or 0 (default) = chosen by the
                                        library: one thread per row when no row has more than 16 entries, else the
                                        length-binned SpMV (each row block's rows ordered by length: short rows one
                                        thread each, 17..64 entries 8 lanes, longer rows a warp).  Reading it
                                        returns the shape in use: 1, 2..32, or 0 for the length-binned SpMV. */
#define SFGMRES_OPT_BLOCK_ROWS 9     /* rows per row block of the fused inner kernels: a multiple of 32 in
                                        [32, 8192], or 0 (default) = chosen by the library (one system: about a
                                        multiple of the SM count of blocks, less 8 SMs with FP64 inner cycles, which
                                        are left to the sketched-QR update running beside the fused kernel; several
                                        systems: 4096).  Reading it returns the size in use. */
#define SFGMRES_OPT_GRAPH 10         /* 1 (default): each outer step (one inner cycle for every problem and the outer
                                        FGMRES update) is captured once into a CUDA graph and replayed; the graphs
                                        are kept while the solve's parameters and workspaces stay the same.  0: the
                                        kernels are launched one by one.  Results are identical either way.
                                        With SFGMRES_OPT_PROFILE = 1 or 2 the timing events are part of the graphs. */
/* (keys 11 and 12 are not used) */
#define SFGMRES_OPT_FUSED_STEP 13    /* 1 (default): where all row blocks of a plan fit on the GPU at once (one system
                                        of up to about 2 x SMs blocks), the truncation window is at most 4 and the
                                        SpMV is not the FP64 length-binned one (measured slower fused), each
                                        inner step runs as one launch: the inner SpMV kernel's work, a grid-wide
                                        arrival of every CTA, then the Arnoldi update of the CTA's own rows (the same
                                        arithmetic in the same order, so results are identical).  The wait is bounded;
                                        if it gives up the solve returns SFGMRES_ERR_CUDA.  With profiling on, the
                                        fused launch is reported as the inner SpMV kernel (t_inner_spmv_ms) and the
                                        update's fields stay 0.  0: two launches per step. */
#define SFGMRES_OPT_STEP_WAIT_EXTRA 14 /* test of the fused step's give-up path: the grid-wide wait also waits for this
                                        many arrivals that never come (default 0).  With a positive value the first
                                        wait of a cycle gives up after its bounded polls (about a second), the later
                                        ones return at once, and the solve returns SFGMRES_ERR_CUDA; the handle stays
                                        usable. */
#define SFGMRES_OPT_OUTER_VARIANT 15  /* 0 (default): FGMRES, the iterate minimises the residual over x0 + span Z
                                        (Algorithm 1).  1: FFOM, the iterate solves the square Hessenberg system
                                        (Galerkin condition), its residual given by Eq. 4; the convergence test and
                                        res_est use that residual, and a step whose square system is singular ends
                                        the solve with SFGMRES_BREAKDOWN keeping the previous iterate. */
#define SFGMRES_OPT_PRECOND 16        /* 0 (default): none.  1: zero-fill incomplete LU (ILU(0)) right preconditioning
                                        (the "-p" runs of Section 4): the rows are ordered colour by colour (a greedy
                                        colouring of the pattern of A + A^T in the natural order: no two coupled rows
                                        share a colour), L U is the ILU(0) factorisation of the permuted matrix
                                        P A P^T and M = P^T L U P; every sGMRES cycle works on A M^{-1} and its
                                        correction is z_j = M^{-1} B_k y_k, so the outer FGMRES still minimises the
                                        residual of A x = b.  Each colour's rows are independent in both triangular
                                        solves (one pass per colour).  Single-system handles, one right-hand side,
                                        FP64 inner cycles, not the transposed solve (other uses return
                                        SFGMRES_ERR_INVALID_ARG); A must store every diagonal entry and no repeated
                                        entries.  The ordering is built at the first solve that uses it, the
                                        factors again after sfgmres_update_values. */
/* ---- sfgmres_solve_batch flags ---------------------------------------------------------------------------- */
#define SFGMRES_SOLVE_TRANSPOSE 1    /* solve A_q^T x = b for every problem (see sfgmres_solve_transpose) */

/* ---- solve statistics ------------------------------------------------------------------------------------- */
/* Filled by sfgmres_solve when a non-NULL pointer is passed.  The array members are caller-owned host arrays of
 * length hist_cap (or NULL); entries beyond outer_iters (or beyond hist_cap) are left untouched. */
typedef struct {
    int32_t status;          /* same as the return value */
    int32_t outer_iters;     /* FGMRES iterations performed */
    int32_t total_inner;     /* sum over cycles of the inner basis size k */
    int32_t hist_cap;        /* capacity of the arrays below (set by the caller) */
    int32_t* inner_k;        /* inner basis size k of each cycle */
    int32_t* inner_reason;   /* rule that ended each cycle: 1 = C1, 2 = C2, 3 = C3, 4 = Arnoldi breakdown,
                                5 = degenerate (no column accepted) */
    double* res_est;         /* ||beta e1 - H_j y_j|| / ||b|| after each outer step (Givens estimate) */
    double* ffom_res;        /* FFOM residual norm (Eq. 4) / ||b|| after each outer step */
    double rel_res_true;     /* recomputed ||b - A x|| / ||b|| of the returned x */
    double rel_res_est;      /* last Givens estimate */
    int64_t kernel_launches; /* kernels this call launched */
    /* with SFGMRES_OPT_PROFILE = 1 (otherwise 0), over the launches of the inner steps that built a basis vector
       (steps i < k_j of each outer step j; the launches after a cycle stopped only read the stop flag): */
    double t_inner_spmv_ms;  /* total device time of the fused inner SpMV + dot + sketch kernel */
    int64_t n_inner_spmv;    /* its launches counted */
    double t_inner_axpy_ms;  /* total device time of the truncated-Arnoldi update kernel */
    int64_t n_inner_axpy;
    double t_qr_ms;          /* total device time of the sketched-QR update kernel */
    int64_t n_qr;
    double t_total_ms;       /* device time of the whole solve (first to last kernel) */
    /* per outer step j (arrays of length hist_cap, caller-owned, may be NULL), for tracing the bound of Eq. 5,
       ||r_j|| <= ||r~_{j-1}|| ||r_hat_j|| (r~ the FFOM residual, ||r~_{-1}|| = beta): */
    double* inner_res;       /* ||r_hat_j|| = ||v_j - A z_j||, the true residual of inner cycle j (v_j has unit
                                norm, so this is also its relative residual) */
    double* inner_rho;       /* the sketched residual rho_k = ||S v_j - S A B_k y_k|| the cycle ended with, its
                                estimate of ||r_hat_j|| (used by rule C3) */
    /* with SFGMRES_OPT_PROFILE = 2 (otherwise 0), over the inner cycles whose m steps all built a basis vector, for
       single-system solves that run each step as one launch: */
    double t_step_span_ms;   /* device time from before the first step launch to after the last, summed */
    int64_t n_step_span;     /* the step launches these spans hold */
} sfgmres_stats;

/* Filled by sfgmres_solve_batch when a non-NULL pointer is passed.  The arrays are caller-owned host arrays of
 * length problems = nsys * nrhs (or NULL), indexed by problem p = q * nrhs + r (system q, right-hand side r). */
typedef struct {
    int32_t problems;        /* set by the library: nsys * nrhs */
    int32_t lockstep_outer;  /* outer steps the batch ran (the largest per-problem count) */
    int64_t total_inner;     /* sum over problems and cycles of the inner basis size k */
    int32_t* status;         /* per-problem status: SFGMRES_OK, _NOT_CONVERGED, _BREAKDOWN or _ERR_NAN */
    int32_t* outer_iters;    /* per-problem FGMRES iterations */
    double* rel_res_true;    /* per-problem recomputed ||b - A x|| / ||b|| */
    double* rel_res_est;     /* per-problem last Givens estimate */
    int64_t kernel_launches; /* kernels this call launched */
    double t_total_ms;       /* device time of the whole solve (first to last kernel) */
    int32_t* inner_steps;    /* per-problem sum over its cycles of the inner basis size k (length problems, or NULL) */
} sfgmres_batch_stats;

typedef struct sfgmres_ctx* sfgmres_t;

/* Create a solver handle for the n x n matrix A given in CSR form (Section 1: A x = b, A large, sparse,
 * nonsymmetric), and the seed of the subspace embedding S (Eq. 1), which is drawn afresh from SplitMix64 for every
 * sketch size s but always from this seed.
 *   out        receives the handle (host pointer; *out is NULL on failure)
 *   n, nnz     order and number of stored entries; 1 <= n, 0 <= nnz < 2^31
 *   row_ptr    int64[n+1], nondecreasing, row_ptr[0] = 0, row_ptr[n] = nnz
 *   col_idx    int32[nnz], column indices in [0, n) (any order within a row; repeated entries are summed)
 *   vals       float64[nnz]
 *   flags      SFGMRES_CSR_HOST if the three arrays are host pointers, else 0 (device pointers)
 *   stream     cudaStream_t to run on (NULL: the library creates a non-blocking stream of its own)
 * The library copies the CSR arrays (the caller may free them on return) and validates them: a violation of the
 * rules above returns SFGMRES_ERR_INVALID_ARG.  Allocation failure returns SFGMRES_ERR_OOM. */
SFGMRES_API int sfgmres_create(sfgmres_t* out, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* vals, uint64_t sketch_seed, int32_t flags, void* stream);

/* Create a handle for a batch of nsys independent systems A_q x = b (q = 0 .. nsys-1) of uneven orders sys_n[q],
 * given as the block-diagonal matrix diag(A_0, ..., A_{nsys-1}) in one CSR: system q owns rows and columns
 * off_q .. off_q + sys_n[q] - 1 with off_q = sys_n[0] + ... + sys_n[q-1], and every stored entry of a row must lie
 * in its system's column range.  Every system is solved independently by the method of sfgmres_solve (its own
 * inner cycles, outer FGMRES, stop rules and convergence test); the systems share the handle's options and sketch
 * seed (system q's embedding is the one sfgmres_create would draw for order sys_n[q]).  sfgmres_create(n, ...) is
 * sfgmres_create_batch(1, &n, ...).
 *   nsys, sys_n    number of systems >= 1 and their orders (host int64[nsys], each >= 1, sum < 2^31 - 1)
 *   nnz, row_ptr, col_idx, vals, flags, stream    as for sfgmres_create, for the block-diagonal matrix
 * Returns SFGMRES_ERR_INVALID_ARG for an entry outside its system's block (in addition to the CSR rules). */
SFGMRES_API int sfgmres_create_batch(sfgmres_t* out, int32_t nsys, const int64_t* sys_n, int64_t nnz,
                                     const int64_t* row_ptr, const int32_t* col_idx, const double* vals,
                                     uint64_t sketch_seed, int32_t flags, void* stream);

/* Set / read an option (SFGMRES_OPT_*).  Values are passed as double.  Unknown keys or out-of-range values return
 * SFGMRES_ERR_INVALID_ARG and leave the option unchanged. */
SFGMRES_API int sfgmres_set_option(sfgmres_t h, int32_t key, double value);
SFGMRES_API int sfgmres_get_option(sfgmres_t h, int32_t key, double* value);

/* Solve A x = b by FGMRES (Algorithm 1) preconditioned with sGMRES cycles (Section 3), starting from x0.
 *   b, x0, x   n float64 each, device or host pointers (see Conventions); x0 may be NULL (zero initial guess)
 *              and may alias x.  x is written on every non-error return.
 *   m          maximum inner basis size (rule C1), 1 <= m <= 1024, m <= s
 *   s          sketch rows, zeta <= s <= 4096 (identity sketch: s == n <= 4096)
 *   k          Arnoldi truncation depth t of the inner basis, 0 <= k <= 8
 *   tol        target relative residual ||b - A x|| / ||b||, 0 < tol < 1
 *   st         optional statistics (may be NULL)
 * Special cases: ||b|| = 0 gives x = 0 and SFGMRES_OK; if ||b - A x0|| <= tol ||b|| then x = x0, 0 iterations.
 * The outer loop stops when the Givens estimate meets tol and the recomputed residual confirms it; otherwise it
 * continues until SFGMRES_OPT_MAX_OUTER iterations (SFGMRES_NOT_CONVERGED).  Returns a status code.  The handle
 * must hold a single system (sfgmres_create); batches use sfgmres_solve_batch. */
SFGMRES_API int sfgmres_solve(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s, int32_t k,
                  double tol, sfgmres_stats* st);

/* Solve A^T x = b with the same method, parameters, options and sketch as sfgmres_solve (A^T is formed on the
 * device on first use and kept).  This is the adjoint solve of the linear map b -> x = A^{-1} b: for a loss L(x),
 * dL/db = A^{-T} dL/dx.  Arguments, special cases and return values as for sfgmres_solve. */
SFGMRES_API int sfgmres_solve_transpose(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m,
                                        int32_t s, int32_t k, double tol, sfgmres_stats* st);

/* Solve every system of the handle for nrhs right-hand sides each: P = nsys * nrhs independent problems, all
 * advanced together (one inner step or one outer step of every unfinished problem per kernel launch; a problem
 * that has converged, broken down or failed is skipped from then on).
 *   nrhs       right-hand sides per system, >= 1 (nrhs * n < 2^31 - 1)
 *   b, x0, x   float64[nrhs * n] in problem order: problem p = q * nrhs + r (system q, right-hand side r) occupies
 *              the sys_n[q] entries starting at nrhs * off_q + r * sys_n[q].  Device or host pointers; x0 may be
 *              NULL and may alias x.  x is written on every non-error return.
 *   m, s, k, tol    as for sfgmres_solve (the same for every problem)
 *   flags      0, or SFGMRES_SOLVE_TRANSPOSE for A_q^T x = b
 *   st         optional per-problem statistics (may be NULL)
 * Returns SFGMRES_ERR_NAN if any problem met a non-finite value (that problem's x is x0; the others are valid),
 * else SFGMRES_NOT_CONVERGED if any problem did not converge, else SFGMRES_BREAKDOWN if any broke down, else
 * SFGMRES_OK; the per-problem outcomes are in st->status. */
SFGMRES_API int sfgmres_solve_batch(sfgmres_t h, int32_t nrhs, const double* b, const double* x0, double* x,
                                    int32_t m, int32_t s, int32_t k, double tol, int32_t flags,
                                    sfgmres_batch_stats* st);

/* Autotune the launch shape of the fused inner kernels for this handle: for each candidate row-block size (the
 * default rule's size and a ladder of multiples of 32 between 256 and 8192) and, for matrices with rows longer than
 * 16 entries, each sub-warp width of the inner SpMV (8 or 32 lanes per row), time short inner sGMRES cycles
 * (min(m, 8) steps, C1/C2 only, a constant unit start vector for every problem, best of two timed runs after a
 * warm-up) with nrhs right-hand sides per system, and keep the fastest per inner step.  The choice is stored in the options
 * SFGMRES_OPT_BLOCK_ROWS and SFGMRES_OPT_SPMV_VECTOR (the method's arithmetic is unchanged; only the order of block
 * partial sums follows the block size).  The paper has no counterpart: this picks GB300 tile shapes.
 *   nrhs, m, s, k       the solve parameters to tune for
 *   block_rows_out, spmv_vector_out (host int32, may be NULL): the chosen sizes
 *   step_ms_out         (host double, may be NULL): the measured time of one inner step (all problems), ms
 * Returns SFGMRES_OK or an error (the options are then left unchanged). */
SFGMRES_API int sfgmres_autotune(sfgmres_t h, int32_t nrhs, int32_t m, int32_t s, int32_t k, int32_t* block_rows_out,
                                 int32_t* spmv_vector_out, double* step_ms_out);

/* Replace the stored values of A (same sparsity pattern, same order as at sfgmres_create): vals is float64[nnz],
 * host or device.  The FP32 copy and the transpose's values follow. */
SFGMRES_API int sfgmres_update_values(sfgmres_t h, const double* vals);

/* out[p] += alpha * u[row(p)] * v[col(p)] for every stored entry p of A (device pointers; u, v: float64[n],
 * out: float64[nnz] in the stored order).  With u = A^{-T} dL/dx and v = x, alpha = -1 this accumulates the gradient
 * of L with respect to the stored values of A (differentiating x = A^{-1} b on the sparsity pattern only). */
SFGMRES_API int sfgmres_pattern_outer(sfgmres_t h, const double* u, const double* v, double alpha, double* out);

/* One sGMRES preconditioner application z = B_k y_k ~ A^{-1} v (Eq. 3 with r0 = v, x0 = 0; Section 3), with rules
 * C1 and C2 only (C3 needs an outer iteration).  Single-system handles only.  v must have unit 2-norm (it is the outer Arnoldi vector).
 *   v, z       n float64, device pointers
 *   m, s, k    as for sfgmres_solve
 *   basis      optional device float64[(m+1) * n], column-major: receives the normalised basis vectors b_1..b_kb
 *              (kb = k_out, plus one more vector when C2 dropped a column); NULL to skip
 *   y          optional device float64[m]: receives y_k (first k_out entries); NULL to skip
 *   k_out      host int32: receives k;   reason_out: host int32 (may be NULL): rule that ended the cycle
 * Returns SFGMRES_OK, or SFGMRES_BREAKDOWN when no column was accepted (z = 0). */
SFGMRES_API int sfgmres_inner_cycle(sfgmres_t h, const double* v, double* z, int32_t m, int32_t s, int32_t k, double* basis,
                        double* y, int32_t* k_out, int32_t* reason_out);

/* Restarted sGMRES (Algorithm 2, with one sGMRES cycle as the variable preconditioner M_c): starting from x_0,
 * r_c = b - A x_c, z_c = M_c^{-1} r_c (one cycle on r_c / ||r_c|| with rules C1 and C2, rescaled by ||r_c||) and
 * x_{c+1} = x_c + z_c, until ||r_c|| <= tol * ||b|| or max_cycles cycles have run.  The comparison method of the
 * paper's experiments: no outer minimisation, so its residuals may stagnate where FGMRES keeps decreasing.
 * Single-system handles only; the precision option applies to the cycles (x and r stay FP64).
 *   b, x0, x      n float64, device or host pointers (x0 may be NULL: zero; x may alias x0)
 *   m, s, k, tol  as for sfgmres_solve; max_cycles >= 0
 *   res_hist      optional host float64[max_cycles + 1]: ||r_c|| / ||b|| for c = 0 .. cycles_out
 *   cycles_out    optional host int32: cycles run
 * Returns SFGMRES_OK (converged), SFGMRES_NOT_CONVERGED (max_cycles reached), SFGMRES_BREAKDOWN (a cycle accepted
 * no column; x is the last iterate), or an error code. */
SFGMRES_API int sfgmres_solve_restarted(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m, int32_t s,
                                        int32_t k, double tol, int32_t max_cycles, double* res_hist,
                                        int32_t* cycles_out);

/* Multi-level FGMRES (the outlook of Section 5): FGMRES on A x = b whose preconditioner at step j is itself an FGMRES
 * run on A z = v_j (zero initial guess) of at most level_steps[0] outer steps, preconditioned in turn by an FGMRES run
 * of at most level_steps[1] steps, and so on for nlower levels; the lowest level is preconditioned by sGMRES cycles as
 * in sfgmres_solve.  Each level keeps its basis small, so the orthogonalisation cost O(n J^2) of one long outer
 * basis is spread over short ones, without restarting any level.  A lower level stops at its budget or once the
 * bound of Eq. 5 predicts that its parent meets the parent's target: with rule C3 on (SFGMRES_OPT_C3) the
 * preconditioner of step j is asked for the relative tolerance tol_parent / ||r~_{j-1}|| (the parent's target over its
 * FFOM residual of Eq. 4, beta before the first step: the test rule C3 applies to an sGMRES cycle); with C3 off every
 * lower level runs its whole budget.  A lower level always takes at least one step, stops on its Givens estimate and
 * returns its last iterate.  The top level's budget is SFGMRES_OPT_MAX_OUTER and it stops as sfgmres_solve does.
 *   b, x0, x, m, s, k, tol   as for sfgmres_solve (single-system handles)
 *   nlower           number of FGMRES levels below the top, 1..4
 *   level_steps      host int32[nlower]: outer-step budget of each lower level, top-most first, each in [1, 1024]
 *   st               optional statistics of the top level; inner_k[j] is the number of steps the level below took
 *                    for step j, inner_reason[j] 3 (it met its tolerance) or 1 (budget), inner_rho[j] its last
 *                    estimate, inner_res[j] the true ||v_j - A z_j||; total_inner counts the sGMRES steps of all
 *                    lowest-level cycles; the kernel timing fields stay 0
 * Returns a status code as sfgmres_solve does. */
SFGMRES_API int sfgmres_solve_multilevel(sfgmres_t h, const double* b, const double* x0, double* x, int32_t m,
                                         int32_t s, int32_t k, double tol, int32_t nlower,
                                         const int32_t* level_steps, sfgmres_stats* st);

/* The ILU(0) preconditioner of SFGMRES_OPT_PRECOND (built now if it is not already; the option itself need not be
 * set): colour (host int32[n], may be NULL) receives every row's colour, ncolours (host int32, may be NULL) their
 * number, lu (host float64[nnz], may be NULL) the factor values in the order of A's stored entries: for the entry
 * (i, j) of A, the entry (p(i), p(j)) of L (below the diagonal; L's unit diagonal is not stored) or of U (on and above
 * it), with p(i) the position of row i in the colour order (colour by colour, natural order within a colour).
 * Single-system handles.  Returns SFGMRES_ERR_INVALID_ARG for a zero pivot, a missing diagonal entry or repeated
 * entries. */
SFGMRES_API int sfgmres_precond_info(sfgmres_t h, int32_t* colour, int32_t* ncolours, double* lu);

/* c = S v for the handle's embedding with s rows (Eq. 1).  v: device float64[n], c: device float64[s].
 * Single-system handles only. */
SFGMRES_API int sfgmres_sketch_apply(sfgmres_t h, int32_t s, const double* v, double* c);

/* The nonzero pattern of S with s rows: for column j and slot l < zeta, rows[j*zeta + l] in [0, s) and
 * signs[j*zeta + l] in {+1, -1} (the value is sign / sqrt(zeta)).  rows: device int32[n*zeta],
 * signs: device int8[n*zeta].  Draw rule (SplitMix64, counter-based): slot q = j*zeta + l draws its row from
 * outputs 128q + 2a (attempt a = 0..63, first row not used by slots 0..l-1 of the column; cyclic probe after 64
 * collisions; row = ((h >> 32) * s) >> 32) and its sign from bit 63 of output 128q + 1.  Single-system handles
 * only. */
SFGMRES_API int sfgmres_sketch_pattern(sfgmres_t h, int32_t s, int32_t* rows, int8_t* signs);

/* c = S v without allocating anything, for callers that cannot call cudaMalloc (code whose device-memory plan is
 * fixed in advance, such as a captured or replayed sequence of work or a loop with a no-allocation rule, or an
 * application whose device memory belongs to another allocator).  The paper has no counterpart: it is the sketch
 * application of sfgmres_sketch_apply (same embedding for the same n, s, zeta and seed; results agree up to
 * summation rounding) without a handle.
 *   n, s, zeta     vector length, sketch rows and nonzeros per column: 1 <= zeta <= 16, zeta <= s <= 4096,
 *                  1 <= n <= 65536 * floor(2^20 / s); larger sizes return SFGMRES_ERR_INVALID_ARG
 *   sketch_seed    seed of the embedding
 *   v, c           device float64[n] input and float64[s] output, owned by the caller
 *   stream         cudaStream_t to enqueue on (NULL: the default stream); the call returns after enqueueing, and c
 *                  is ready when the stream reaches that point
 * Scratch: a fixed 8 MiB static device array (2^20 doubles) in the library, held on every GPU that loads the
 * library until the process exits.  All calls share it and it keeps the last call's contents; every call overwrites
 * the part it reads, so nothing needs to start at zero.  Calls whose work overlaps on the GPU (different streams,
 * different host threads) race on it and must be serialised by the caller.  The first call on a device does a
 * one-time set-up with that device current (it looks up the array's device address and raises the kernel's
 * shared-memory limit to what s = 4096 needs); make that first call before any stream capture.  Errors:
 * SFGMRES_ERR_INVALID_ARG (sizes, NULL), SFGMRES_ERR_CUDA (set-up or a launch of this call; an error left by
 * unrelated earlier work is not reported); sfgmres_last_error(NULL) describes them. */
SFGMRES_API int sfgmres_sketch_apply_noalloc(int64_t n, int32_t s, int32_t zeta, uint64_t sketch_seed,
                                             const double* v, double* c, void* stream);

/* y = A x in FP64 (device pointers, n each; for a batch handle A is the block-diagonal matrix). */
SFGMRES_API int sfgmres_spmv(sfgmres_t h, const double* x, double* y);

/* Release the handle and everything it owns.  NULL is accepted. */
SFGMRES_API int sfgmres_destroy(sfgmres_t h);

/* Description of the last error on this handle (h == NULL: of the last failed sfgmres_create in this thread).
 * The string stays valid until the next call on the same handle. */
SFGMRES_API const char* sfgmres_last_error(sfgmres_t h);

/* Library version string. */
SFGMRES_API const char* sfgmres_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SFGMRES_H */
