/*
 * lindblad_ss.h -- C ABI of the GB300 steady-state solver for open quantum
 * systems (Nation, "Steady-state solution methods for open quantum optical
 * systems", arXiv:1504.06768).
 *
 * Problem (section "Steady-state density matrix", Eq. ss / Eq. eigval):
 * given a time-independent Hamiltonian H and collapse operators C_k, all
 * d x d sparse complex matrices, find rho_ss with L rho_ss = 0 and
 * Tr rho_ss = 1, where L is the Lindblad superoperator of Eq. (lindblad)
 * acting on the column-stacked vector vec(rho) (vec(rho)[i + d*j] = rho[i,j]).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved doubles (re, im): a complex array of
 *   length m is a double array of length 2m.  FP32 variants use floats.
 * - Sparse matrices are CSR with int32 row pointers and column indices,
 *   columns sorted ascending and unique within a row.  nnz < 2^31.
 * - Views (ss_csr_view) are borrowed: the library copies what it needs and
 *   never keeps the caller's pointers after the call returns.
 * - Handles (ss_ctx, ss_mat, ss_prec) are owned by the library; free them
 *   with the matching *_free / *_destroy.  Matrices and factors live in the
 *   device memory of the context's GPU.
 * - Vector arguments documented as "device" must be device pointers on the
 *   context's GPU; "host" arguments are ordinary host memory.
 * - Work is issued on the context's CUDA stream.  A call returns after the
 *   work it started has completed, unless documented otherwise.
 * - Every function returns an ss_status and never aborts; on failure the
 *   reason is available from ss_last_error(ctx).  Output handles are set to
 *   NULL on failure.
 * - A context is not thread-safe: use one context per host thread.
 */
#ifndef LINDBLAD_SS_H
#define LINDBLAD_SS_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SS_OK = 0,
    SS_ERR_INVALID = 1,      /* bad argument (shape, pointer, option)              */
    SS_ERR_OOM = 2,          /* device allocation failed                           */
    SS_NOT_CONVERGED = 3,    /* iteration cap reached; outputs hold the last iterate */
    SS_BREAKDOWN = 4,        /* BiCGSTAB inner product vanished (section "Iterative
                                solvers": the residual became orthogonal to the
                                shadow residual)                                   */
    SS_ZERO_PIVOT = 5,       /* incomplete factorisation met a zero/missing pivot  */
    SS_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                 */
    SS_ERR_CUDA = 7,         /* a CUDA runtime call failed                          */
    SS_ERR_UNSUPPORTED = 8   /* valid request this build does not implement        */
} ss_status;

typedef enum {
    SS_METHOD_DIRECT = 0,          /* LU with partial pivoting of the RCM-ordered Eq. (linear) as a band (section
                                      "Direct factorization"); SS_ERR_UNSUPPORTED when the band is too wide */
    SS_METHOD_ITER_GMRES = 1,      /* "iterative-lgmres": restarted GMRES(m) on Eq. (linear), augmented
                                      with the corrections of the lgmres_k previous cycles (LGMRES,
                                      Baker, Jessup and Manteuffel 2005) when lgmres_k > 0        */
    SS_METHOD_ITER_BICGSTAB = 2,   /* "iterative-bicgstab": BiCGSTAB on Eq. (linear)         */
    SS_METHOD_INVERSE_POWER = 3,   /* doubly-iterative inverse power on L - sigma I          */
    SS_METHOD_AUTO = 4             /* the paper's choice (sections "Results" and "Conclusion"): the RCM
                                      bandwidths of L~ (Eq. linear) and of L - sigma I (Eq. inverse)
                                      are compared; (L)GMRES on L~ when B(L~) <= 1.5 B(L - sigma I),
                                      else the doubly-iterative inverse power with (L)GMRES inner
                                      solves.  FP64 only; info.method reports the choice          */
} ss_method;

typedef enum { SS_PRECOND_ILU0 = 0, SS_PRECOND_ILUT = 1 } ss_precond_kind;

typedef enum {
    SS_PREC_FP64 = 0,    /* everything in complex FP64                                    */
    SS_PREC_MIXED = 1    /* FP32 inner Krylov solve + FP32 factors, FP64 refinement       */
} ss_precision;

typedef enum { SS_KRYLOV_BICGSTAB = 0, SS_KRYLOV_GMRES = 1 } ss_krylov;

/* Borrowed CSR view of a square or rectangular complex matrix. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int32_t* row_ptr;   /* n_rows + 1 entries                                */
    const int32_t* col;       /* nnz entries                                        */
    const double* val;        /* 2 * nnz doubles, interleaved (re, im)              */
    int on_device;            /* 0: the three arrays are host memory; 1: device     */
} ss_csr_view;

typedef struct ss_ctx_s* ss_ctx;
typedef struct ss_mat_s* ss_mat;
typedef struct ss_prec_s* ss_prec;

/* Options of steady_state().  ss_options_default() fills the defaults shown. */
typedef struct {
    int method;            /* ss_method; default SS_METHOD_ITER_BICGSTAB                     */
    int precond;           /* ss_precond_kind; default SS_PRECOND_ILU0                       */
    int precision;         /* ss_precision; default SS_PREC_FP64                             */
    double tol;            /* accept when ||L rho||_2 <= tol, rho trace-normalised; 1e-10    */
    int maxiter;           /* Krylov iteration cap (section "Numerical Simulations"); 1000    */
    int restart;           /* GMRES restart length m; 30 (maximum 64)                         */
    double drop_tol;       /* ILUT drop tolerance d (relative to the row infinity norm); 1e-4 */
    double fill_factor;    /* ILUT fill factor p; 10                                         */
    double w;              /* weight of Eq. (linear); <= 0 selects mean_i |L_ii|              */
    double sigma;          /* shift of Eq. (inverse); 1e-15                                  */
    int use_rcm;           /* reverse Cuthill-McKee ordering of L~ + L~^T; 1                 */
    uint64_t seed;         /* inverse-power start vector (SplitMix64 counters); 0             */
    double inner_rtol;     /* SS_PREC_MIXED: relative tolerance of each FP32 inner solve; 1e-5 */
    int lgmres_k;          /* GMRES: corrections of earlier cycles added to each cycle (LGMRES);
                              0 = plain restarted GMRES; restart + lgmres_k <= 64                 */
    int warm_start;        /* 1: rho_out holds an initial guess on entry (the steady state of a
                              neighbouring point of a parameter sweep, say): the Krylov iteration
                              starts from it, scaled to unit trace (inverse power: the start
                              vector).  A guess of zero trace falls back to the zero start.  0   */
    int autotune;          /* steady_state_batched: 1 = choose the persistent solver's lanes per row
                              (of the two triangles and of L~) and its level staging by timing short
                              capped runs of candidate choices on the batch's first systems
                              (coordinate descent from the rule-based choice); the choice is kept per
                              context for batches of the same shape.  Results are those of the chosen
                              launch, to the same tolerance.  0: the rules                         */
} ss_options;

/* Per-solve diagnostics. */
typedef struct {
    int status;            /* ss_status of the solve                                   */
    int iters;             /* Krylov iterations (inner iterations for MIXED)           */
    int outer_iters;       /* inverse-power or refinement steps                        */
    double resid_Lrho;     /* FP64 ||L rho||_2 of the returned trace-normalised rho     */
    double w_used;         /* weight of Eq. (linear) (0 for inverse power)             */
    double condest;        /* ||M^{-1} e||_inf of the preconditioner                   */
    int64_t n, nnz;        /* size of L~ (or L - sigma I)                              */
    int64_t bandwidth, profile;  /* of the matrix after ordering                       */
    int64_t nnz_factors;   /* stored entries of the incomplete factors                 */
    int32_t levels_lower, levels_upper;  /* triangular-solve level counts               */
    double ms_setup, ms_solve;           /* wall time of setup and of the iteration      */
    int method;            /* ss_method that ran (the choice of SS_METHOD_AUTO)        */
    int64_t bw_modified, bw_shifted;     /* SS_METHOD_AUTO: RCM bandwidths compared; else 0 */
    int32_t tune_lanes_shift[3];         /* batched solver: lanes per row of the lower triangle, the
                                            upper triangle and L~ as log2 multiples of the rule's choice */
    int32_t tune_stage;                  /* 1: the level staging other than the rule's (see autotune)  */
    int32_t fp64_fallback;               /* MIXED single-system solve: 1 = an FP32 inner solve stalled
                                            (did not reach inner_rtol within its cap) and the remaining
                                            iterations ran in FP64 from the refined iterate            */
} ss_info;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is
 * borrowed and must outlive the context.  The library allocates device
 * memory from one memory pool per device, shared by its contexts, that
 * keeps freed blocks for later allocations until the process exits. */
ss_status ss_ctx_create(int device, void* cuda_stream, ss_ctx* out);
ss_status ss_ctx_destroy(ss_ctx ctx);
/* Replace the stream used by later calls. */
ss_status ss_ctx_set_stream(ss_ctx ctx, void* cuda_stream);
/* Message describing the last failure on this context ("" if none). */
const char* ss_last_error(ss_ctx ctx);
void ss_options_default(ss_options* opt);

/* ----------------------------------------------------------- matrices */

/* Assemble L (Eq. lindblad vectorised as in Eq. eigval):
 *   L = -i (I kron H - H^T kron I)
 *       + sum_k (conj(C_k) kron C_k - 1/2 I kron C_k^+C_k - 1/2 (C_k^+C_k)^T kron I)
 * H and the n_c operators in c_ops are d x d views (host or device).  The
 * result is an n x n matrix, n = d^2, built on the device from the Kronecker
 * structure; entries whose summed value is exactly zero are not stored.
 * Errors: SS_ERR_INVALID for non-square or mismatched views. */
ss_status assemble_liouvillian(ss_ctx ctx, const ss_csr_view* H, int n_c, const ss_csr_view* c_ops,
                               ss_mat* L_out);

/* Eq. (linear): L~ = L + w T, T = ones in row 0 at the columns i(d+1) of the
 * diagonal elements of rho; d = sqrt(n).  w <= 0 selects w = mean_i |L_ii|
 * (the weight of the numerical section); the value used is written to
 * *w_used (may be NULL).  The right-hand side of Eq. (linear) is w e_0. */
ss_status add_trace_row(ss_ctx ctx, ss_mat L, double w, ss_mat* out, double* w_used);

/* The trace-row systems of many Liouvillians at once: out[k] receives
 * L~_k = L_k + w_k T, L_k assembled from H[k] and the n_c[k] operators
 * c_ops[k] (Eq. lindblad, as assemble_liouvillian) and the trace row added as
 * add_trace_row does (Eq. linear), with w_k = w when w > 0, else
 * mean_i |(L_k)_ii|; each is entry for entry the matrix those two calls give.
 * w_used (may be NULL) receives the n_sys weights.  The operators of all
 * systems are stacked block-diagonally on the device, so the number of kernel
 * launches does not grow with n_sys.  out (n_sys handles, caller-allocated
 * array) is all NULL on failure.  Errors: as assemble_liouvillian; device
 * views must be 4-byte (indices) and 8-byte (values) aligned. */
ss_status assemble_trace_batched(ss_ctx ctx, int n_sys, const ss_csr_view* H, const int* n_c,
                                 const ss_csr_view* const* c_ops, double w, ss_mat* out, double* w_used);

/* Eq. (inverse): L - sigma I.  Every diagonal entry is stored afterwards. */
ss_status add_shift(ss_ctx ctx, ss_mat L, double sigma, ss_mat* out);

/* Reverse Cuthill-McKee ordering of the pattern of A + A^T (section "Direct
 * factorization"): breadth-first search from a node of minimum degree,
 * neighbours by increasing degree, per connected component, reversed.
 * Ties: the start node is the highest-index unvisited node of minimum
 * degree; neighbours are taken in ascending (degree, index); the degree
 * counts the stored diagonal.  perm_out (host, n int32) receives perm with
 * perm[new] = old.  bw_out / profile_out (may be NULL) receive the
 * bandwidth B and profile P of P A P^T. */
ss_status rcm_permute(ss_ctx ctx, ss_mat A, int32_t* perm_out, int64_t* bw_out, int64_t* profile_out);

/* out = P A P^T, out[r][c] = A[perm[r]][perm[c]]; perm is host memory, n int32. */
ss_status permute(ss_ctx ctx, ss_mat A, const int32_t* perm, ss_mat* out);

/* Bandwidth B = ub + lb + 1 and profile P = up + lp of A's stored pattern
 * (section "Direct factorization"). */
ss_status bandwidth_profile(ss_ctx ctx, ss_mat A, int64_t* bw_out, int64_t* profile_out);

/* Size of a matrix handle. */
ss_status ss_mat_shape(ss_mat A, int64_t* n_rows, int64_t* nnz);
/* Copy a matrix to caller buffers (host): row_ptr n+1, col nnz, val 2 nnz. */
ss_status ss_mat_export(ss_ctx ctx, ss_mat A, int32_t* row_ptr, int32_t* col, double* val);
/* Wrap a CSR view as a library matrix (copied to the device). */
ss_status ss_mat_import(ss_ctx ctx, const ss_csr_view* A, ss_mat* out);
void ss_mat_free(ss_mat A);

/* y = A x (complex FP64 CSR SpMV); x, y are device arrays of 2n doubles. */
ss_status spmv(ss_ctx ctx, ss_mat A, const double* x, double* y);
/* FP32 variant on A's FP32 copy (made on first use); x, y device, 2n floats. */
ss_status spmv_f32(ss_ctx ctx, ss_mat A, const float* x, float* y);

/* ------------------------------------------------------ preconditioner */

/* Incomplete LU of A (section "Iterative solvers"):
 *   kind SS_PRECOND_ILU0: no fill, computed on the device level by level;
 *   kind SS_PRECOND_ILUT: dual threshold -- entries of row i below
 *     drop_tol * ||a_i||_inf are dropped and each of the strict L and U parts
 *     keeps at most ceil(fill_factor * nnz(a_i) / 2) largest entries; no
 *     pivoting; computed on the host.
 * precision: SS_PREC_FP64, or SS_PREC_MIXED to also keep FP32 factors.
 * condest_out (may be NULL): ||M^{-1} e||_inf, e = ones.
 * Errors: SS_ZERO_PIVOT when a pivot is missing or zero. */
ss_status ilu_factor(ss_ctx ctx, ss_mat A, int kind, double drop_tol, double fill_factor,
                     int precision, ss_prec* out, double* condest_out);
/* z = U^{-1} L^{-1} r (level-scheduled sparse triangular solves); device, 2n doubles. */
ss_status precond_apply(ss_ctx ctx, ss_prec M, const double* r, double* z);
/* FP32 variant (needs precision SS_PREC_MIXED at factorisation). */
ss_status precond_apply_f32(ss_ctx ctx, ss_prec M, const float* r, float* z);
/* Factor sizes and level counts. */
ss_status ss_prec_info(ss_prec M, int64_t* nnz, int32_t* levels_lower, int32_t* levels_upper);
/* Copy the combined factors (strict lower = L with unit diagonal, rest = U)
 * into host buffers: row_ptr n+1, col nnz, val 2 nnz. */
ss_status ss_prec_export(ss_ctx ctx, ss_prec M, int32_t* row_ptr, int32_t* col, double* val);
void ss_prec_free(ss_prec M);

/* ------------------------------------------------------------ solvers */

/* Solve A x = b with right-preconditioned BiCGSTAB or GMRES(restart)
 * (section "Iterative solvers"), M from ilu_factor on the same A.  b and x
 * are device arrays (2n doubles); x holds the initial guess on entry.
 * Stops when the updated residual satisfies ||b - A x||_2 <= tol (absolute)
 * or after maxiter iterations (SS_NOT_CONVERGED); SS_BREAKDOWN when a
 * BiCGSTAB inner product vanishes.  *iters_out (may be NULL) receives the
 * iteration count, *resid_out (may be NULL) the final residual norm. */
ss_status krylov_solve(ss_ctx ctx, ss_mat A, ss_prec M, int krylov, const double* b, double* x,
                       double tol, int maxiter, int restart, int* iters_out, double* resid_out);

/* krylov_solve with SS_KRYLOV_GMRES augmented as LGMRES(restart, augment)
 * (Baker, Jessup and Manteuffel 2005): each restart cycle minimises
 * ||b - A x||_2 over M^{-1} applied to the Krylov space of the cycle's
 * residual plus the normalised corrections of the `augment` previous cycles
 * (each costs one product with A and no preconditioner application; both
 * kinds of step count as iterations).  augment = 0 is GMRES(restart).
 * Arguments and statuses as for krylov_solve.
 * Errors: SS_ERR_INVALID unless restart >= 1, augment >= 0 and
 * restart + augment <= 64. */
ss_status lgmres_solve(ss_ctx ctx, ss_mat A, ss_prec M, const double* b, double* x, double tol, int maxiter,
                       int restart, int augment, int* iters_out, double* resid_out);

/* ------------------------------------------------ host-side analysis */

/* The host steps of the path, callable without a GPU or a context (the same
 * code rcm_permute, ilu_factor and the level analysis of the triangular
 * solves run).  All arrays are host memory owned by the caller; the input is
 * an n x n CSR pattern with row_ptr[0] = 0, non-decreasing row pointers and
 * strictly ascending columns in [0, n) in every row, else SS_ERR_INVALID.
 *
 * ss_rcm_order_host: reverse Cuthill-McKee order of the pattern of A + A^T
 * (section "Direct factorization"; start node: the highest-index unvisited
 * node of minimum degree; neighbours in ascending (degree, index); one pass
 * per connected component; the sequence reversed).  perm_out[new] = old, n
 * entries. */
ss_status ss_rcm_order_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t* perm_out);

/* Level sets of the strict lower (lower != 0) or strict upper triangle:
 * level(i) = 1 + the largest level of the rows row i depends on (0 without
 * dependencies).  order_out (n entries) lists the rows by (level, row);
 * level_ptr_out (n + 1 entries available; *n_levels_out + 1 written) gives
 * the start of each level in order_out. */
ss_status ss_level_sets_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int lower,
                             int32_t* order_out, int32_t* level_ptr_out, int32_t* n_levels_out);

/* Elimination schedule of iLU(0) (section "Iterative solvers": incomplete
 * LU without fill, by IKJ elimination restricted to the pattern) for a CSR
 * pattern with ascending columns and every diagonal entry stored; the
 * batched solver factors each system from the schedule of its pattern.  For
 * the pivot at CSR position t of row i (k = col[t] < i) the updates are
 * the pairs p in [ptr_out[t], ptr_out[t + 1]): a[row_ptr[i] + tgt_out[p]] -=
 * l * a[src_out[p]] with l = a[t] / u_kk, in the order listed, after the
 * pivots before t; positions that are not pivots have empty ranges.
 * *count_out receives the number of pairs; when it exceeds `capacity`
 * nothing else is written and SS_ERR_INVALID is returned (call again with
 * enough room: ptr_out row_ptr[n] + 1 entries, tgt_out and src_out count
 * entries).  SS_ZERO_PIVOT: a diagonal entry is missing. */
ss_status ss_ilu0_schedule_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int64_t capacity,
                                int32_t* ptr_out, int32_t* tgt_out, int32_t* src_out, int64_t* count_out);

/* ILUT(drop_tol, fill_factor) without pivoting (section "Iterative
 * solvers"; the rules of ilu_factor with SS_PRECOND_ILUT) on a complex CSR
 * matrix (val: 2 * nnz doubles, interleaved).  Output: the combined factors
 * (strict lower part = L with unit diagonal, diagonal and upper part = U),
 * ascending columns.  *nnz_out receives their entry count; when it exceeds
 * `capacity` nothing else is written and SS_ERR_INVALID is returned (call
 * again with enough room: f_row_ptr n + 1, f_col nnz, f_val 2 nnz entries).
 * SS_ZERO_PIVOT with *zero_pivot_row = the row of a zero or missing pivot
 * (else -1). */
ss_status ss_ilut_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val, double drop_tol,
                       double fill_factor, int64_t capacity, int32_t* f_row_ptr, int32_t* f_col, double* f_val,
                       int64_t* nnz_out, int64_t* zero_pivot_row);

/* Weighted maximum bipartite matching (section "Direct factorization"): a
 * row permutation that makes the diagonal zero-free when A is structurally
 * nonsingular, trying to put large entries on it.  Columns are taken in
 * descending order of their largest |a_ij|^2 (ties: ascending column); each
 * runs a breadth-first search over alternating paths that tries the rows of
 * a column in descending |a_ij|^2 (ties: ascending row) and flips the path to
 * the first unmatched row.  match_out[j] (n entries) = the row assigned to
 * column j, or -1 when column j has no augmenting path; *matched_out = the
 * number of matched columns (n: A[match_out, :] has a zero-free diagonal).
 * val: 2 * nnz doubles, interleaved.  The device path does not apply it: the
 * trace-row Liouvillians of the workloads have a full diagonal. */
ss_status ss_mbm_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                      int32_t* match_out, int64_t* matched_out);

/* Largest system krylov_solve_noalloc accepts (complex unknowns). */
#define SS_NOALLOC_MAX_N 65536

/* krylov_solve with SS_KRYLOV_BICGSTAB (same iteration, same stop and
 * breakdown rules, same results) for callers that cannot allocate memory
 * during the call: a real-time or control loop with a fixed memory budget, or
 * a host that routes every device allocation through its own pool.  This
 * call makes no cudaMalloc/cudaFree or other allocation: its workspace (eight
 * Krylov vectors of up to SS_NOALLOC_MAX_N = 65,536 complex doubles, the
 * solver state and the reduction partials, about 8.3 MiB) is a fixed array in
 * the library's device memory that every GPU loading the library holds until
 * the process exits.  ss_ctx_create loads that array onto its device and
 * looks up its address (so with CUDA's lazy module loading the array comes
 * into existence there, and ss_ctx_create returns SS_ERR_OOM / SS_ERR_CUDA if
 * it cannot); no call of this function allocates it.  Every call shares the
 * array and overwrites what the previous call left there, and the host-side
 * mirror of the solver state is shared per device as well: calls on the same
 * GPU whose work could overlap (other streams, other host threads) race and
 * must be serialised by the caller.  The call synchronises the context's
 * stream (it reads the solver state back between chunks of iterations), so
 * it must not be issued on a stream that is being captured.  Arguments as
 * for krylov_solve; b and x are device arrays of 2n doubles, x holds the
 * initial guess.
 * Errors: SS_ERR_INVALID when n > SS_NOALLOC_MAX_N (use krylov_solve), plus
 * the statuses of krylov_solve.  The paper has no counterpart of this entry
 * point; it is an interface variant of the BiCGSTAB solve. */
ss_status krylov_solve_noalloc(ss_ctx ctx, ss_mat A, ss_prec M, const double* b, double* x, double tol,
                               int maxiter, int* iters_out, double* resid_out);

/* Full steady-state solve.  H and c_ops as for assemble_liouvillian.
 * rho_out: d*d complex (2 d^2 doubles), column-major, trace-normalised;
 * host memory if rho_on_device == 0, device memory otherwise.  info may be
 * NULL.  Returns SS_OK when ||L rho||_2 <= opt->tol; SS_NOT_CONVERGED or
 * SS_BREAKDOWN still write the last iterate to rho_out. */
ss_status steady_state(ss_ctx ctx, const ss_csr_view* H, int n_c, const ss_csr_view* c_ops,
                       const ss_options* opt, double* rho_out, int rho_on_device, ss_info* info);

/* Steady states of n_sys independent systems (parameter sweeps, uneven
 * Hilbert sizes).  System k is H[k] with the n_c[k] operators c_ops[k]; rho_out[k]
 * receives d_k * d_k complex values (column-major), host or device memory as
 * rho_on_device says; infos (may be NULL) receives n_sys entries.
 * With method = iterative-bicgstab and precond = iLU(0), systems with
 * n = d^2 up to 11,520 (FP64) or 19,200 (SS_PREC_MIXED) are solved together by
 * one persistent kernel launch: one thread block per system at a time runs the
 * iLU(0) factorisation, the preconditioned BiCGSTAB (FP64, or FP32 inner
 * iterations on r/||r|| refined in FP64 until ||L rho||_2 <= tol) and the
 * finalisation.  Systems sharing a sparsity pattern share one RCM ordering and
 * level schedule.  Other systems and options go through steady_state() one at
 * a time.  Host results (rho_on_device == 0) pass through pinned host memory
 * that the context keeps for later calls (grown to the largest batch's
 * results, freed by ss_ctx_destroy; pageable copies if it cannot be had).
 * Returns SS_OK when every system converged, otherwise the status of a
 * failing system (each info holds its own status). */
ss_status steady_state_batched(ss_ctx ctx, int n_sys, const ss_csr_view* H, const int* n_c,
                               const ss_csr_view* const* c_ops, const ss_options* opt,
                               double* const* rho_out, int rho_on_device, ss_info* infos);

/* -------------------------------------------------------------- serving */

/* A serving loop for steady-state requests (not part of the paper's method:
 * an interface around it).  Requests of different Hilbert sizes are
 * submitted at any time and solved while others are on the device: a worker
 * thread admits queued requests in arrival order whenever a batch slot is
 * free and the request's estimated device footprint fits the memory budget,
 * and runs them as one batch ("wave") of the persistent per-system solver of
 * steady_state_batched on the slot's own stream; several waves run side by
 * side, each system holding one SM, so a new wave fills the SMs an earlier
 * one leaves idle.  Pattern analyses (RCM ordering, level schedule) stay
 * resident across waves for requests with the same structure.  Requests
 * outside the persistent solver's scope (n beyond its limit, or options it
 * does not run) go to a second lane running steady_state() in FP64 on two
 * low-priority streams (its mixed form pays more iterations than it saves on
 * systems that large), while the waves run on high-priority streams.  A request's
 * result is the one the same system gets alone from steady_state_batched
 * (or from steady_state in the second lane). */
typedef struct ss_server_s* ss_server;

typedef struct {
    double hbm_budget_mb;   /* device memory admitted requests may hold (MiB); <= 0: 80 % of the free memory */
    int max_waves;          /* batches in flight at once (default 4) */
    int max_wave_systems;   /* systems per batch; <= 0: number of SMs / max_waves */
    int warm_start;         /* 1: a request of the persistent solver starts from the stored steady
                               state of the earlier request with the same sparsity pattern whose
                               L~ is closest (by the Frobenius norms of its diagonal and off-diagonal
                               parts): a parameter sweep then starts every point from a neighbour.
                               The result is the same steady state within the tolerance, not bit
                               for bit the result of a cold solve.  Default 0 */
} ss_server_options;

void ss_server_options_default(ss_server_options* so);
/* opt: the solve options of every request (NULL: defaults).  Starts the worker threads. */
ss_status ss_server_create(int device, const ss_options* opt, const ss_server_options* so, ss_server* out);
/* Finishes every submitted request, stops the workers and frees the server. */
ss_status ss_server_destroy(ss_server s);
/* Queues one system (host CSR views, copied before the call returns).
 * rho_out: host memory for d*d complex values (column-major), written when the
 * request completes; it must stay valid until then.  *ticket identifies the
 * request.  SS_ERR_OOM when its footprint exceeds the whole budget. */
ss_status ss_submit(ss_server s, const ss_csr_view* H, int n_c, const ss_csr_view* c_ops, double* rho_out,
                    uint64_t* ticket);
/* *done = 1 once the request has completed. */
ss_status ss_poll(ss_server s, uint64_t ticket, int* done);
/* Waits up to timeout_us (< 0: without limit).  Returns SS_ERR_TIMEOUT while the
 * request is pending (it stays queryable); once it has completed, returns its
 * solve status, fills info (may be NULL) and *latency_ms (submission to
 * completion, may be NULL) and forgets the ticket. */
ss_status ss_wait(ss_server s, uint64_t ticket, int64_t timeout_us, ss_info* info, double* latency_ms);
/* Waves launched, requests completed, memory held by admitted requests and the budget. */
ss_status ss_server_stats(ss_server s, uint64_t* waves, uint64_t* completed, double* in_use_mb, double* budget_mb);
const char* ss_server_last_error(ss_server s);

/* ---------------------------------------------------------- diagnostics */

/* Kernel classes of the per-launch profiler. */
typedef enum { SS_PROF_SPMV = 0, SS_PROF_TRSV_LOWER = 1, SS_PROF_TRSV_UPPER = 2, SS_PROF_BATCHED = 3 } ss_prof_kind;

/* When enabled, CUDA events are recorded on the context's stream around every
 * SpMV, triangular-solve and batched-solver launch issued through this context.  Not part of
 * the paper: a measurement aid for the bandwidth roofline. */
ss_status ss_profile_enable(ss_ctx ctx, int enable);
/* Synchronise the stream and return, for one kernel class, the number of
 * launches recorded since the last read and their summed device time in
 * milliseconds; the records of that class are then cleared. */
ss_status ss_profile_read(ss_ctx ctx, int kind, int64_t* launches, double* total_ms);
/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts). */
unsigned long long ss_launch_count(void);
/* The autotuner's search on a table of costs instead of measured runs (a
 * test of its logic; needs no GPU): cost_table[((l*4 + u)*4 + a)*2 + s] is the
 * cost of lanes-per-row shifts (l-1, u-1, a-1) and staging flag s.  Starting
 * from (0, 0, 0, 0), coordinate descent moves to a neighbour while the cost
 * drops by more than 1 %, evaluating each choice at most once and at most
 * max_probes choices.  best_out (4 values) receives the choice, *probes_out
 * (may be NULL) the evaluations made. */
ss_status ss_tune_search_host(const double* cost_table, int32_t max_probes, int32_t* best_out,
                              int32_t* probes_out);

/* Limit of every bounded device-side wait issued through this context: a
 * triangular solve waiting for a row it depends on, a staging barrier of the
 * batched solver.  Default 2 s; a wait that reaches it makes the call return
 * SS_ERR_TIMEOUT (the device stays usable).  Tests shorten it to make a
 * wait run out.  SS_ERR_INVALID for 0. */
ss_status ss_set_wait_limit(ss_ctx ctx, uint64_t limit_ns);
/* Failure-detection aid, not part of the paper's method: with restore == 0
 * the lower triangular solve of M stops computing row `row` (its value is
 * never written, so the rows depending on it wait until the wait limit and
 * precond_apply returns SS_ERR_TIMEOUT); restore != 0 undoes it.
 * SS_ERR_INVALID for a row outside M or a second skipped row. */
ss_status ss_diag_prec_skip_row(ss_ctx ctx, ss_prec M, int64_t row, int restore);

/* Failure-detection aid, not part of the paper's method: in later
 * steady_state_batched calls on this context whose triangular solves stage
 * their levels through the shared-memory ring (the FP64 form), every block's
 * staging number `seq` (counted from 0 over the levels it stages) arms its
 * barrier without issuing the copies, so the solving warps wait until the
 * wait limit, and the call reports SS_ERR_TIMEOUT for the systems of that
 * launch.  seq = -1 (the default) turns it off.  SS_ERR_INVALID below -1. */
ss_status ss_diag_batched_stall(ss_ctx ctx, int64_t seq);

/* Number of device and pinned-host memory allocations this library has made
 * in the process so far (all contexts): a call that allocates nothing leaves
 * it unchanged. */
unsigned long long ss_alloc_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LINDBLAD_SS_H */
