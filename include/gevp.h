/*
 * gevp.h -- C ABI of libgevp: sequences of dense complex Hermitian-definite generalized
 * eigenproblems A x = lambda B x on one GB300 (sm_103a).
 *
 * The problem is the one the paper poses for every k-point of every self-consistent
 * outer iteration of an FLAPW DFT cycle (Sec. "Introduction to Density Functional
 * Theory", Eq. 3 and the paragraph after it): A (the Hamiltonian) Hermitian, B (the
 * overlap) Hermitian positive definite, the lowest nev eigenpairs wanted. The paper's
 * Sec. "A new computational philosophy" treats the iterations as a sequence of
 * correlated problems and seeds an iterative eigensolver with the previous problem's
 * eigenvectors; its conclusions name an improved subspace iteration as the solver to
 * build. This library does that: Cholesky reduction C = L^-1 A L^-H, then Chebyshev-
 * filtered subspace iteration (CholQR2 orthonormalisation, Rayleigh-Ritz, residual
 * locking) seeded with the previous eigenvectors.
 *
 * Conventions (all functions):
 *  - Matrices are ROW-MAJOR, interleaved complex128 (C99 double complex / torch
 *    complex128, 16 bytes per element), with a leading dimension ld >= number of columns.
 *    A Hermitian matrix read column-major is its conjugate; the layout is fixed here.
 *  - A and B are read in full (both triangles); they must be Hermitian. Results are
 *    undefined if they are not.
 *  - Every matrix/vector argument is DEVICE memory owned by the caller unless the
 *    function name ends in _host. The library never frees caller memory.
 *  - All work is enqueued on the handle's stream. A function returns after the work is
 *    complete unless stated otherwise (the solver reads small status words back).
 *  - Functions never abort or trap; they return a gevp_status. gevp_last_error() gives
 *    a one-line message for the last failure on a handle.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Workspace belongs to the handle, is sized lazily, grows and is released by
 *    gevp_destroy.
 */
#ifndef GEVP_H
#define GEVP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gevp_ctx* gevp_handle;

typedef enum {
  GEVP_OK = 0,
  GEVP_ERR_INVALID_ARG = 1,     /* a size, pointer or leading dimension is invalid   */
  GEVP_ERR_NOT_HPD = 2,         /* B (or a Gram matrix) is not positive definite     */
  GEVP_ERR_NO_CONVERGENCE = 3,  /* iteration cap hit; best results are still written */
  GEVP_ERR_CUDA = 4,            /* a CUDA runtime call failed                        */
  GEVP_ERR_OOM = 5,             /* device workspace could not be allocated           */
  GEVP_ERR_TIMEOUT = 6,         /* a bounded device-side wait ran out                */
  GEVP_ERR_INVALID_VALUE = 7,   /* NaN or Inf found in an input matrix               */
  GEVP_ERR_UNSUPPORTED = 8      /* requested mode not available on this device       */
} gevp_status;

/* Precision of the Chebyshev filter (everything else is FP64). */
typedef enum {
  GEVP_PREC_FP64 = 0,   /* FP64 complex GEMM                                           */
  GEVP_PREC_FP32 = 1,   /* FP32-class: each operand split in three BF16 pieces, the six */
                        /* significant cross products on tcgen05, FP32 accumulation     */
  GEVP_PREC_BF16 = 2    /* BF16 planar operands, 3-product (Gauss) complex GEMM on      */
                        /* tcgen05 tensor cores, FP32 accumulation in TMEM              */
} gevp_prec;

typedef struct {
  int filter_prec;      /* gevp_prec the filter starts in; switches to FP64 on stall    */
  double tol;           /* target max_i ||A x_i - l_i B x_i|| / (||A|| ||x_i||); 1e-10  */
  int max_outer;        /* cap on outer (filter + Rayleigh-Ritz) iterations per problem */
  int deg_min, deg_max; /* Chebyshev degree range                                       */
  int nex;              /* guard vectors (at least 2 are used); m = min(n, nev + nex)  */
  uint64_t seed;        /* seed of the counter-based generator for random start blocks  */
  int b_fixed;          /* 1: every problem of the sequence has the same B              */
  int cold_start;       /* 1: every problem starts from a random block (no warm start)  */
  int lanczos_steps;    /* steps of the Lanczos bound estimator                         */
  int refine_iters;     /* refinement steps of the small eigensolver (>= 1)             */
  int keep_all_X;       /* 1: X receives every problem's eigenvectors (nprob*n*nev)     */
  int refresh_window;   /* 0: off. k > 0: after k consecutive warm-started problems that */
                        /* needed at least as many filter matvecs as the latest cold one, */
                        /* the next problem starts cold (the paper's refresh when progress */
                        /* flattens out, Sec. "A new computational philosophy")           */
  int reduce_slices;    /* 0: the products with an n x n operand (the reduction to standard */
                        /* form, W = C Q, X = L^-H Q, A X, B X) run on the FP64 pipe. 1..8: */
                        /* they are emulated on the tensor cores with that many 7-bit digits */
                        /* per entry (Ozaki scheme, exact digit products; 8 digits keep     */
                        /* FP64-class accuracy), see gevp_zgemm_emulated; the batched form  */
                        /* emulates them one k-point at a time. Requires n <= 30720.        */
} gevp_opts;

/* Per-problem counters and CUDA-event phase times (milliseconds). */
typedef struct {
  int outer_iters;      /* filter + orthonormalisation + Rayleigh-Ritz rounds           */
  int filter_steps;     /* Chebyshev matrix-block products                              */
  int switches;         /* filter precision switches to FP64                            */
  int orth_fallbacks;   /* shifted CholQR fallbacks                                     */
  int final_passes;     /* original-space residual checks                               */
  int converged;        /* 1 if every residual <= tol                                   */
  int64_t matvecs;      /* filter column-products (sum of active columns x degree)      */
  double flops_fp64;    /* executed-flop model, FP64 work                               */
  double flops_lowp;    /* executed-flop model, tensor-core filter work (complex, 8/MAC) */
  double max_resid;
  double orth_err;      /* max |Q^H Q - I| of the returned block (B-orthonormality of X)  */
  int cold;             /* 1 if this problem started from a random block                 */
  float ms_chol, ms_reduce, ms_bounds, ms_filter, ms_orth, ms_rr, ms_resid, ms_final, ms_total;
} gevp_stats;

/* Fills *o with the defaults: FP64 filter, tol 1e-10, max_outer 60, degrees 4..48,
 * nex 0 (callers set it), seed 10074400, b_fixed 0, cold_start 0, lanczos_steps 32,
 * refine_iters 3, keep_all_X 0, refresh_window 0, reduce_slices 8. */
void gevp_default_opts(gevp_opts* o);

/* Creates a handle on CUDA device `device` bound to `stream` (a cudaStream_t; NULL =
 * the legacy default stream). Returns GEVP_ERR_CUDA if the device cannot be used. */
gevp_status gevp_create(gevp_handle* h, int device, void* stream);
gevp_status gevp_destroy(gevp_handle h);
gevp_status gevp_set_stream(gevp_handle h, void* stream);
const char* gevp_status_string(gevp_status s);
const char* gevp_last_error(gevp_handle h);
const char* gevp_version(void);

/* Reduction to standard form (the first step after Eq. 3: B = L L^H, C = L^-1 A L^-H).
 *   A, B: n x n Hermitian (B HPD), read only.  L: n x n output, lower, strict upper = 0.
 *   C: n x n output, Hermitian (both triangles written).
 *   *info (host): 0, or the 1-based index of the first non-positive pivot of B (LAPACK
 *   potrf convention); then GEVP_ERR_NOT_HPD is returned and L, C are undefined. */
gevp_status gevp_reduce(gevp_handle h, int64_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                        void* L, int64_t ldl, void* C, int64_t ldc, int64_t* info);

/* Update of the standard form for a change of A confined to a few rows and columns. The
 * paper observes that most entries of the Hamiltonian change little from one iteration to
 * the next, so that only part of it needs to be regenerated (Sec. "Matrix generation").
 * With B (hence L) unchanged, C_new = L^-1 A_new L^-H = C_old + L^-1 dA L^-H, and when
 * dA = A_new - A_old vanishes outside the rows and the columns of an index set J (|J| = k),
 * the update is the Hermitian rank-2k product U V^H + V U^H with U = L^-1 E_J (the columns J
 * of L^-1), R = the rows J of dA and V = L^-1 R^H - U R_JJ / 2: O(n^2 k) work instead of the
 * 4 n^3 of a full reduction. The result equals the full reduction of A_new up to rounding.
 *   B: n x n HPD (ld ldb). reuse_factor 1: B is the matrix of the previous successful call
 *   on this handle (same pointer and contents) and its factorisation is reused; 0: B is
 *   factored (and kept for the next call).
 *   dA: n x n Hermitian difference (ld ldda), read only in the rows and columns listed; its
 *   other entries are ignored (treated as zero). rows: host array of k distinct indices in
 *   [0, n), 0 <= k <= n / 5 (beyond that a full reduction costs about as much).
 *   C: n x n (ld ldc) in: C_old = L^-1 A_old L^-H (Hermitian, both triangles); out: C_new,
 *   Hermitian (both triangles written).
 *   slices: 0 = FP64 pipe; 1..8 = the two n^2 k products emulated on the tensor cores as in
 *   gevp_zgemm_emulated (requires n <= 30720).
 *   *info (host): 0, or the potrf pivot of B (then GEVP_ERR_NOT_HPD). GEVP_ERR_INVALID_ARG
 *   for repeated or out-of-range rows or k > n / 5. Returns after the work is complete. */
gevp_status gevp_reduce_update(gevp_handle h, int64_t n, const void* B, int64_t ldb, int reuse_factor,
                               const void* dA, int64_t ldda, int k, const int64_t* rows, void* C, int64_t ldc,
                               int slices, int64_t* info);

/* The sequence solver (the paper's sequence {P_i} of correlated problems, each seeded
 * with the eigenvectors of the one before).
 *   A: host array of nprob device pointers, each n x n (ld lda). B: host array of nprob
 *   device pointers (ld ldb); when consecutive pointers are equal, or opts->b_fixed is
 *   set, the Cholesky factor is reused.
 *   X_prev: nullable, n x kprev (ld ldxp) eigenvector guesses for problem 0 (in the
 *   original space); kprev <= nev + nex.
 *   Outputs (device): Lambda[nprob * nev] ascending per problem; resid[nprob * nev] the
 *   original-space relative residuals ||A x - l B x|| / (||A||_est ||x||) with ||A||_est
 *   a Lanczos estimate of ||A||_2 from below; X: n x nev (ld ldx) eigenvectors of the
 *   last problem, B-orthonormal (or nprob such blocks, stride n*ldx, if keep_all_X).
 *   stats: nullable host array of nprob gevp_stats.
 *   Returns GEVP_ERR_NO_CONVERGENCE if some residual stays above tol (outputs written). */
gevp_status gevp_solve_sequence(gevp_handle h, int nprob, int64_t n, const void* const* A, int64_t lda,
                                const void* const* B, int64_t ldb, int nev, const void* X_prev, int64_t ldxp,
                                int kprev, const gevp_opts* opts, double* Lambda, void* X, int64_t ldx,
                                double* resid, gevp_stats* stats);

/* Same, with every array in HOST memory (A, B: host arrays of host pointers; Lambda,
 * resid, X host; pinned memory makes the copies asynchronous and fast). The copies to and
 * from the device are part of the call: every A (and each distinct B) is copied into a
 * device staging area owned by the handle, the sequence is solved there, and Lambda,
 * resid and X are copied back before the call returns. */
gevp_status gevp_solve_sequence_host(gevp_handle h, int nprob, int64_t n, const void* const* A, int64_t lda,
                                     const void* const* B, int64_t ldb, int nev, const gevp_opts* opts,
                                     double* Lambda, void* X, int64_t ldx, double* resid, gevp_stats* stats);

/* ---- batched (k-point) form --------------------------------------------------------- */

/* Counters of one gevp_solve_batched call. Times are CUDA-event milliseconds summed over
 * the steps of the sequence. */
typedef struct {
  int steps;            /* problems per k-point (the sequence length)                   */
  int rounds;           /* lock-step rounds (filter + CholQR + Rayleigh-Ritz), all steps */
  int max_rounds_step;  /* most rounds any one step needed                              */
  int graph_replays;    /* rounds executed as replays of the captured round graph      */
  int switches;         /* problems switched to the FP64 filter (all steps)            */
  int orth_fallbacks;   /* CholQR breakdowns repaired by a random restart              */
  int final_passes;     /* original-space checks, summed over problems and steps        */
  int converged;        /* 1 if every residual of every problem <= tol                 */
  int tile[8];          /* autotuner: grouped FP64 GEMM tile chosen per call class      */
  int deg_cap[8];       /* autotuner: filter degree cap per size bucket (last step)     */
  double max_resid;
  double flops_fp64, flops_lowp;   /* executed-flop model                              */
  float ms_chol, ms_reduce, ms_bounds, ms_rounds, ms_final, ms_total;
} gevp_batch_stats;

/* Many independent problem sequences of uneven size at once: the paper solves Eq. 3 for
 * every k-point of the Brillouin-zone sampling and every self-consistent iteration (the
 * paragraph after Eq. 3). nk k-points, each a sequence of nsteps problems
 * A_{k,l} x = lambda B_k x of order n[k] with B_k fixed along the sequence; each step l
 * is warm-started from step l-1's eigenvectors of the same k-point. All k-points advance
 * in lock-step rounds: every phase of a round is one launch for the whole batch (grouped
 * GEMMs over a global tile list, one CTA per problem for the small dense work, one
 * grouped tcgen05 launch per filter step), converged k-points are skipped by device
 * flags, and a round is captured once as a CUDA graph and replayed. An autotuner picks
 * the grouped GEMM tile per call class (timed on the first round of a new batch shape)
 * and the filter degree cap per size bucket (a cost model fed by measured times and the
 * Chebyshev convergence factors of the previous step).
 *   n, nev, nex: host arrays of nk (nex nullable: opts->nex for all, at least 2 used);
 *   m_k = min(n_k, nev_k + nex_k) <= 1024.
 *   A: host array of nk * nsteps device pointers, A[k * nsteps + l] (ld lda[k]);
 *   B: host array of nk device pointers (ld ldb[k]), HPD.
 *   X_prev: nullable host array of nk (entries nullable) device pointers, n_k x kprev[k]
 *   (ld ldxp[k]) start vectors for step 0 in the original space.
 *   Lambda, resid: host arrays of nk device pointers, each nsteps x nev_k.
 *   X: nullable host array of nk device pointers, n_k x nev_k (ld ldx[k]) eigenvectors of
 *   the last step (or nsteps such blocks, stride n_k * ldx[k], if opts->keep_all_X).
 *   opts: filter_prec FP64, FP32 or BF16 (low precision switches a k-point to FP64 when
 *   it stalls); tol, max_outer (rounds per step), deg_min, deg_max (<= 64), seed,
 *   cold_start, lanczos_steps, refine_iters as for gevp_solve_sequence; b_fixed is implied.
 *   stats: nullable.
 *   The handle keeps the batch's workspace, autotuner choices and round graph for the
 *   next call with the same shapes; a call with other shapes rebuilds them.
 *   Returns GEVP_ERR_NOT_HPD if some B_k is not HPD, GEVP_ERR_NO_CONVERGENCE if some
 *   residual stays above tol (all outputs written). */
gevp_status gevp_solve_batched(gevp_handle h, int nk, int nsteps, const int64_t* n, const int* nev, const int* nex,
                               const void* const* A, const int64_t* lda, const void* const* B, const int64_t* ldb,
                               const void* const* X_prev, const int64_t* ldxp, const int* kprev,
                               const gevp_opts* opts, double* const* Lambda, double* const* resid,
                               void* const* X, const int64_t* ldx, gevp_batch_stats* stats);

/* ---- individual steps of the solver (same kernels as the solver uses) ---------------- */

/* Scaled Chebyshev filter (Zhou, Saad, Tiago & Chelikowsky 2006), in place:
 *   Y <- p(C) Y,  p(t) = T_d((t-c)/e) / T_d((s-c)/e),  c = (lo+hi)/2, e = (hi-lo)/2,
 * for the n x m block Y (ld ldy), degree d >= 1, scaling point s < lo < hi.
 * prec: gevp_prec of the products. */
gevp_status gevp_chebyshev_filter(gevp_handle h, int64_t n, const void* C, int64_t ldc, void* Y, int64_t ldy,
                                  int m, int degree, double lo, double hi, double s, int prec);

/* The filter's contraction alone on the tensor cores: D = C Y (n x n times n x m) with
 * C and Y rounded to BF16 planes (real, imaginary, real + imaginary), the complex product
 * formed from three real products (Gauss) with FP32 accumulation, D written in FP64.
 * GEVP_ERR_UNSUPPORTED on devices other than sm_103. */
gevp_status gevp_matmul_tc(gevp_handle h, int64_t n, int m, const void* C, int64_t ldc, const void* Y, int64_t ldy,
                           void* D, int64_t ldd);

/* CholQR2 (Fukaya, Nakatsukasa, Yanagisawa & Yamamoto 2014): Y (n x m) <- Q with
 * Q^H Q = I and Y_in = Q R, R upper triangular with positive diagonal (written to R,
 * m x m, ld ldr, if non-null). GEVP_ERR_NOT_HPD if Y is rank deficient in FP64. */
gevp_status gevp_cholqr2(gevp_handle h, int64_t n, int m, void* Y, int64_t ldy, void* R, int64_t ldr);

/* Rayleigh-Ritz on span(Q) (Q n x m orthonormal, in place): G = Q^H C Q = Z diag(theta) Z^H,
 * Q <- Q Z, W = C Q (n x m output), theta ascending (device, m), res[i] = ||W_i - theta_i Q_i||. */
gevp_status gevp_rayleigh_ritz(gevp_handle h, int64_t n, int m, const void* C, int64_t ldc, void* Q, int64_t ldq,
                               void* W, int64_t ldw, double* theta, double* res);

/* Small dense Hermitian eigensolver: G (m x m) = Z diag(theta) Z^H, theta ascending. */
gevp_status gevp_heev_small(gevp_handle h, int m, const void* G, int64_t ldg, double* theta, void* Z, int64_t ldz);

/* Lanczos spectral bounds of Hermitian C: out (host, 5 doubles) = {lowest Ritz value,
 * highest Ritz value, upper bound of the spectrum, estimate of the count-th eigenvalue,
 * |beta_k|}. */
gevp_status gevp_spectral_bounds(gevp_handle h, int64_t n, const void* C, int64_t ldc, int k, int count,
                                 double* out);

/* Band energy E = sum_{i<nev} lambda_i, the sum of the occupied eigenvalues of each problem
 * (the band-structure term of the Kohn-Sham total energy whose eigenproblem is Eq. 3).
 *   Lambda: device nprob x nev (row p = problem p, as gevp_solve_sequence writes it);
 *   E: device nprob, E[p] summed in index order (deterministic). Enqueued on the handle's
 *   stream; returns without waiting. */
gevp_status gevp_band_energy(gevp_handle h, int nprob, int nev, const double* Lambda, double* E);

/* Band-energy gradient for E = sum_{i<nev} lambda_i (first-order perturbation theory):
 *   GA = gE * X X^H = dE/dA * gE,   GB = -gE * X diag(Lambda) X^H = dE/dB * gE,
 * X n x nev B-orthonormal eigenvectors (ld ldx), Lambda device (nev), gE a DEVICE scalar
 * (the incoming gradient, read on the device: no host synchronisation); GA, GB n x n (ld
 * ldg). Enqueued on the handle's stream; returns without waiting. */
gevp_status gevp_energy_backward(gevp_handle h, int64_t n, int nev, const void* X, int64_t ldx,
                                 const double* Lambda, const double* gE, void* GA, void* GB, int64_t ldg);

/* Entry-variation statistics between the Hamiltonians of consecutive self-consistent
 * iterations (Sec. "Matrix generation": the largest entry variation delta_{n+1} and the
 * entries of (A_{n+1} - A_n) / delta_{n+1} above a threshold fraction p_t, whose share
 * tells how much of the matrix would have to be regenerated).
 *   A_new, A_old: n x n device (ld lda, ldb). p_t: host array of nthr (<= 16) fractions.
 *   Outputs (host): *delta = max_ij |A_new - A_old|_ij; counts[k] = number of entries with
 *   |A_new - A_old|_ij > p_t[k] * delta. The comparison is made on squares in FP64,
 *   d2 = dr*dr + di*di (each product and the sum rounded separately) against
 *   (p*p) * delta^2, so the counts are exact for that arithmetic.
 *   mask: nullable device n x n bytes (row-major, ld n): 1 where the entry is above
 *   p_t[0] * delta, else 0.
 *   The handle keeps an n x n scratch of 8-byte words (the squared moduli), grown on
 *   demand. GEVP_ERR_INVALID_VALUE if a difference is NaN. Returns after the work is
 *   complete. */
gevp_status gevp_matrix_variation(gevp_handle h, int64_t n, const void* A_new, int64_t lda, const void* A_old,
                                  int64_t ldb, int nthr, const double* p_t, double* delta, int64_t* counts,
                                  void* mask);

/* Deviation angles between the eigenvectors of consecutive problems, and the re-indexing
 * that matches them (Sec. "A new computational philosophy", paragraph "Eigenvectors
 * evolution": eigenvalue order is not a reliable index from one iteration to the next, so
 * each old eigenvector is compared with the new one at the smallest angle; angles are
 * normalised so that 1.00 = pi/2).
 *   X_old: n x k_old, X_new: n x k_new (k_old <= k_new), device, row-major complex128
 *   (ld ldo, ldn), columns the eigenvectors. B: device n x n HPD (ld ldb), or NULL for the
 *   Euclidean inner product.
 *   c_ij = |x_old_i^H B x_new_j| / (||x_old_i||_B ||x_new_j||_B), clamped to [0, 1].
 *   cosines: nullable device k_old x k_new doubles (row-major, ld ldc) receiving c.
 *   perm: nullable host int64[k_old]. Given, it receives the re-indexing: the assignment of
 *   each old vector to a distinct new one minimising sum_i (1 - c_{i,perm[i]}), where a pair
 *   with |lam_old[i] - lam_new[j]| > window costs more than any assignment of pairs inside
 *   the window (so the fewest pairs possible lie outside it). The paper gives no algorithm;
 *   this is an optimal assignment (Hungarian method on the host, exact for the cosines in
 *   FP64; when several assignments tie, any one of them). NULL: no re-indexing, column i is
 *   matched with column i.
 *   lam_old, lam_new: host eigenvalues (k_old, k_new); required when window is finite,
 *   ignored when window = +INFINITY (no window). window >= 0.
 *   Outputs (host, each nullable): theta[i] = acos(c_{i,match(i)}) / (pi/2); *cost = sum of
 *   1 - c over matched pairs inside the window; *n_outside = matched pairs outside it.
 *   GEVP_ERR_INVALID_VALUE if a B-norm is zero or not finite. Device scratch of about
 *   16 n (k_old + k_new) + 24 k_old k_new bytes is kept by the handle (grown on demand).
 *   Returns after the work is complete. */
gevp_status gevp_deviation_angles(gevp_handle h, int64_t n, int k_old, int k_new, const void* X_old, int64_t ldo,
                                  const void* X_new, int64_t ldn, const void* B, int64_t ldb, const double* lam_old,
                                  const double* lam_new, double window, double* cosines, int64_t ldc, int64_t* perm,
                                  double* theta, double* cost, int64_t* n_outside);

/* The host step of the re-indexing above, on its own (no device, no handle): the
 * assignment of each of the ko rows of a ko x kn cost table (host, row-major, ld kn,
 * ko <= kn, finite entries) to a distinct column minimising the summed cost; perm (host,
 * ko) receives the column of each row. Hungarian method, shortest-augmenting-path form.
 * GEVP_ERR_INVALID_ARG on bad sizes, null pointers or a cost that is not finite. */
gevp_status gevp_assign_min_cost(int ko, int kn, const double* cost, int64_t* perm);

/* FP64 complex product emulated on the tensor cores (Ozaki scheme; beyond the paper, which
 * keeps every step in FP64): D (M x N) = op(A) op(B), op(X) = X (op 0) or X^H (op 1):
 * A is M x K (opA 0, lda >= K) or K x M (opA 1, lda >= M), B is K x N (opB 0, ldb >= N) or
 * N x K (opB 1, ldb >= K); device row-major complex128. Each row of op(A) and each column
 * of op(B) is scaled by a power of two so its
 * largest real or imaginary part lies in [1/4, 1/2), rounded to `slices` signed 7-bit
 * digits (1..8) and the digit planes are multiplied exactly in BF16 with FP32
 * accumulation (units of at most 2048 complex terms); pairs of digits whose weights sum
 * past the last digit are left out; the exact integer sums are combined in FP64.
 *   Error of entry (i, j): at most about 2K (slices + 3) 2^(-7 slices + 2) max_k|op(A)_ik|
 *   max_k|op(B)_kj| (FP64's own bound is K u sum_k |op(A)_ik||op(B)_kj|, u = 2^-53); with
 *   8 digits the two are of the same order.
 *   K <= 30720 (else GEVP_ERR_UNSUPPORTED); GEVP_ERR_INVALID_VALUE on NaN or Inf in A or B.
 *   Device scratch of slices * (4 M_pad + 6 N_pad) * K_pad bytes (M_pad, N_pad: M, N
 *   rounded up to 128; K_pad: K rounded up to 64) is kept by the handle. Needs an sm_103 device (GEVP_ERR_UNSUPPORTED otherwise).
 *   Returns after the work is complete. */
gevp_status gevp_zgemm_emulated(gevp_handle h, int opA, int opB, int M, int N, int K, const void* A, int64_t lda,
                                const void* B, int64_t ldb, void* D, int64_t ldd, int slices);

/* gevp_reduce with the two n^3 products of the reduction (T = L^-1 tril(A) with the
 * diagonal halved, M = T L^-H, C = M + M^H) emulated as in gevp_zgemm_emulated with
 * `slices` digits, and B factored recursively: for n > 256, n = n1 + n2 with
 * L21 = A21 L11^-H, L22 L22^H = B22 - L21 L21^H and (L^-1)21 = -L22^-1 L21 L11^-1, the
 * four off-diagonal products emulated, leaves of order <= 256 factored with their
 * inverses in one thread-block cluster each. n <= 30720. The same outputs (to FP64
 * rounding) and errors as gevp_reduce; `info` is the global index of the first
 * non-positive pivot met. */
gevp_status gevp_reduce_emulated(gevp_handle h, int64_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                                 void* L, int64_t ldl, void* C, int64_t ldc, int64_t* info, int slices);

/* Measured FP64 FMA, FP64 DMMA and FP32 FMA rates of this device in TFLOP/s (host out[3]). */
gevp_status gevp_probe_peaks(gevp_handle h, double* out);

/* ---- allocation-free variant ------------------------------------------------------- */

/* Size, in complex128 elements, of the fixed device scratch of the entry point below
 * (32 MiB on every device that loads the library, held until the process exits). */
#define GEVP_NOALLOC_MAX_ELEMS (1 << 21)

/* The FP64 Chebyshev filter of gevp_chebyshev_filter (prec GEVP_PREC_FP64), for callers
 * that must not allocate device memory when they call it: applications whose device
 * memory belongs to a pool allocator such as PyTorch's caching allocator (a library
 * cudaMalloc/cudaFree would bypass the pool, can fail while the pool holds the free memory,
 * and synchronises the device), and services that reserve a fixed memory budget at
 * start-up. The paper has no counterpart; it is a deployment variant of the same
 * computation.
 *   No handle: the work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *   stream) of the current device and the call returns without waiting for it. C, Y as in
 *   gevp_chebyshev_filter (device, row-major complex128, Y n x m overwritten in place).
 *   It calls no cudaMalloc, cudaFree or allocating library routine. Its scratch, two n x m
 *   blocks, is a fixed array in the library's device image: requires 2 n m <=
 *   GEVP_NOALLOC_MAX_ELEMS, else GEVP_ERR_INVALID_ARG is returned and nothing is enqueued.
 *   The first call on a device looks up the array's device address (once per device, with
 *   that device current) and caches it for the life of the process; make that first call
 *   before any stream capture, and do not use the entry point across a cudaDeviceReset
 *   (the cached address would be stale). Every call on a device shares the one array,
 *   which keeps the previous call's contents (each call writes every scratch element it
 *   reads first, so nothing needs clearing): calls whose work overlaps on the GPU (other
 *   streams, other host threads) race on it. If a CUDA error from earlier work is pending
 *   on the calling thread, GEVP_ERR_CUDA is returned, the error is left pending and nothing
 *   is enqueued. */
gevp_status gevp_chebyshev_filter_noalloc(void* stream, int64_t n, const void* C, int64_t ldc, void* Y, int64_t ldy,
                                          int m, int degree, double lo, double hi, double s);

/* Live timing of the product kernels, for measurement (off by default; process-wide).
 * enable 1 clears earlier records and starts recording: every launch of the FP64 complex
 * GEMM, of the emulated product and of the tall-skinny Gram kernel is bracketed by CUDA
 * events on its own stream; 0 stops. */
gevp_status gevp_kernel_timing(int enable);
/* out (host, 12 doubles): for class 0 (FP64 complex GEMM), class 1 (emulated product) and
 * class 2 (tall-skinny Gram kernel), four values each: launches, total milliseconds,
 * algorithmic flop (8 per complex multiply-add over the K ranges the tiles process, at
 * 64-, 128- resp. 16-row block granularity) and executed flop (class 1: the digit pairs'
 * BF16 real products, 36x the algorithmic at 8 digits). Waits for the recorded events. */
gevp_status gevp_kernel_timing_read(double* out);

/* Number of kernels the library launched since it was loaded, process-wide: every handle,
 * the handle-less entry points and every host thread (h is accepted for compatibility and
 * not used). For launch accounting. */
int64_t gevp_kernel_launches(gevp_handle h);

#ifdef __cplusplus
}
#endif
#endif /* GEVP_H */
