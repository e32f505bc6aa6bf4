// Internal declarations shared by the CUDA translation units of libgevp.
// All matrices are row-major; complex128 is interleaved (double2: x = real, y = imag).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <atomic>
#include <cstdint>
#include <cstddef>

namespace gevp {

// ---------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ double2 zmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__device__ __forceinline__ void zfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------- FP64 complex GEMM
// D = alpha * op(A) op(B) + beta * Cin + gamma * Ein   (real alpha, beta, gamma)
// op(X) = X (op = 0) or X^H (op = 1). op(A) is M x K, op(B) is K x N, D is M x N.
// tri flags let whole k-tiles that are known zero be skipped:
//   triA = 1: op(A) lower (op(A)[i][k] = 0 for k > i);  2: upper (0 for k < i)
//   triB = 1: op(B) lower (op(B)[k][j] = 0 for k < j);  2: upper (0 for k > j)
//   triD = 1: only tiles that intersect the lower triangle of D are computed
// maskB = 1 (opB = 0 only): op(B) is read as the lower triangle of B with its diagonal
//   halved and zeros above (the Hermitian split B = Bl + Bl^H).
// ksplit > 1: grid.z carries k-slices; slice z writes its partial product (no epilogue)
//   to D + z * M * N with ld = N, and zgemm_reduce_splits finishes the epilogue.
struct ZgemmArgs {
  int M, N, K;
  const double2* A; int64_t lda; int opA;
  const double2* B; int64_t ldb; int opB;
  double2* D; int64_t ldd;
  double alpha;
  const double2* Cin; int64_t ldc; double beta;
  const double2* Ein; int64_t lde; double gamma;
  int triA, triB, triD, maskB;
  int ksplit;
  int batch;
  int64_t sA, sB, sD, sC, sE;   // batch strides in elements
};

void zgemm(const ZgemmArgs& a, double2* split_ws, size_t split_ws_elems, cudaStream_t s);
// Scaled Chebyshev filter with FP64 products (see zgemm.cu); returns B1 or B2.
double2* cheb_filter_fp64(int64_t n, const double2* C, int64_t ldc, const double2* Y0, int64_t ld0, int ma, int deg,
                          double lo, double hi, double sc, double2* B1, double2* B2, int64_t ldb, double2* split_ws,
                          size_t split_elems, cudaStream_t s);
// Simple helper for the common case.
ZgemmArgs zg(int M, int N, int K, const double2* A, int64_t lda, int opA,
             const double2* B, int64_t ldb, int opB, double2* D, int64_t ldd, double alpha = 1.0);

// Grouped (ragged-batch) form: a device array of items, each one independent product with
// the same op/tri flags. tile_start/tiles_n are filled by zgemm_group_layout (host). If
// active != nullptr and *active == 0 the item is skipped; if coef != nullptr the scalars
// are read from device memory (alpha = coef[0], beta = coef[1], gamma = coef[2]).
struct ZgemmItem {
  int M, N, K;
  int tile_start, tiles_n;
  const double2* A; int64_t lda;
  const double2* B; int64_t ldb;
  double2* D; int64_t ldd;
  const double2* Cin; int64_t ldc;
  const double2* Ein; int64_t lde;
  double alpha, beta, gamma;
  const double* coef;
  const int* active;
};
struct ZgemmGroupFlags { int opA, opB, triA, triB, triD, maskB; };
int zgemm_group_tile(const ZgemmItem* items_host, int nitems);
int zgemm_group_layout(ZgemmItem* items_host, int nitems, int tile);   // returns total tiles
void zgemm_grouped(const ZgemmItem* items_dev, int nitems, int total_tiles, int tile, const ZgemmGroupFlags& f,
                   cudaStream_t s);

// ---------------------------------------------------------------- elementwise / misc
void herm_sum_inplace(int64_t n, double2* C, int64_t ldc, cudaStream_t s);  // C <- C + C^H
void zshift_diag(int64_t n, double2* A, int64_t lda, double sh, cudaStream_t s);
void zero_lower(int64_t n, double2* A, int64_t lda, cudaStream_t s);        // strict lower <- 0
void hermitize_lower(int64_t n, double2* C, int64_t ldc, cudaStream_t s);   // upper <- conj(lower), real diag
void hermitize_avg(int64_t n, double2* C, int64_t ldc, cudaStream_t s);     // C <- (C + C^H)/2
// lower triangle scaled by sign * (*scale) (device scalar), then upper <- conj(lower)
void hermitize_scale_lower(int64_t n, double2* C, int64_t ldc, const double* scale, double sign, cudaStream_t s);
// C <- C + D on the lower triangle, then upper <- conj(lower), real diagonal
void add_lower_herm(int64_t n, double2* C, int64_t ldc, const double2* D, int64_t ldd, cudaStream_t s);
// Out[i][t] = X[i][idx[t]] (rows x k) and Out[t][j] = X[idx[t]][j] (k x cols); idx device
void gather_cols(int64_t rows, int k, const double2* X, int64_t ldx, const int64_t* idx, double2* Out, int64_t ldo,
                 cudaStream_t s);
void gather_rows(int k, int64_t cols, const double2* X, int64_t ldx, const int64_t* idx, double2* Out, int64_t ldo,
                 cudaStream_t s);
// E[p] = sum of lam[p * nev + 0 .. nev - 1] in index order (device arrays)
void band_energy(int nprob, int nev, const double* lam, double* E, cudaStream_t s);
void zero_upper(int64_t n, double2* L, int64_t ldl, cudaStream_t s);        // strict upper <- 0
void zsub_lower(int64_t n, double2* A, int64_t lda, const double2* P, int64_t ldp, cudaStream_t s);  // A -= P, j <= i
void zneg(int64_t rows, int64_t cols, double2* X, int64_t ldx, cudaStream_t s);                      // X <- -X
void eye_deviation(int m, const double2* G, int64_t ldg, double* out_dev, cudaStream_t s);  // max |G - I|
void zcopy2d(int64_t rows, int64_t cols, const double2* src, int64_t lds, double2* dst, int64_t ldd, cudaStream_t s);
void zset_identity(int64_t rows, int64_t cols, double2* A, int64_t lda, cudaStream_t s);
void z_to_c(int64_t rows, int64_t cols, const double2* src, int64_t lds, float2* dst, int64_t ldd, cudaStream_t s);
void zrandn(int64_t rows, int64_t cols, double2* A, int64_t lda, uint64_t seed, cudaStream_t s);
void zcol_scale(int64_t rows, int64_t cols, double2* A, int64_t lda, const double* scale, cudaStream_t s);
int  check_finite(int64_t rows, int64_t cols, const double2* A, int64_t lda, int* dflag, cudaStream_t s);

// ---------------------------------------------------------------- factorizations
// Blocked lower Cholesky in place (strict upper zeroed). info_dev: 0 or 1-based pivot.
// Linv (n x n, ld ldi) receives the inverses of the 32 x 32 diagonal blocks of L.
void potrf_lower(int64_t n, double2* A, int64_t lda, int* info_dev, double2* Linv, int64_t ldi, cudaStream_t s);
// Lower-triangular inverse: Linv = L^-1 (Linv separate buffer, strict upper zeroed).
// diag_ready: Linv already holds the diagonal blocks' inverses (from potrf_lower).
void trtri_lower(int64_t n, const double2* L, int64_t ldl, double2* Linv, int64_t ldi, double2* ws,
                 size_t ws_elems, cudaStream_t s, bool diag_ready = false);
size_t trtri_ws_elems(int64_t n);

// ---------------------------------------------------------------- small Hermitian eigensolver
// G (m x m Hermitian, FP64) -> theta ascending (m), Z (m x m, columns = eigenvectors).
// FP32 parallel Jacobi followed by FP64 Ogita-Aishima refinement built from FP64 GEMMs.
struct HeevWork {
  float2* G32; float2* Z32; float* w32; int* perm;
  double2 *Z, *R, *S, *T, *E;   // m x m each
  double* lam;                  // m
  double2* split_ws; size_t split_ws_elems;
  double* scal;                 // small scalars
  unsigned* gcnt;               // zgram arrival counters (zgram_counters() words, zero)
};
size_t heev_ws_bytes(int m, size_t split_elems);
void heev_small(int m, const double2* G, int64_t ldg, double* theta, double2* Z, int64_t ldz,
                const HeevWork& w, int refine_iters, cudaStream_t s);
// FP32 Jacobi on a (possibly real) Hermitian matrix in FP32 (single CTA); sorted output.
void jacobi32(int m, float2* G, float2* Z, float* w, int* perm, int max_sweeps, cudaStream_t s);

// ---------------------------------------------------------------- Lanczos bounds (FP32)
struct LanczosOut { double lam_min, lam_max, upper, a_est, beta_last; };
struct LanczosWork { float2* V; float* ab; float2* w; float2* T32; float2* Z32; float* w32; int* perm; double* out; };
size_t lanczos_ws_bytes(int64_t n, int k);
// k-step Lanczos with full re-orthogonalisation on the FP32 copy of a Hermitian matrix.
// Writes to dev_out[0..4] = {theta_min, theta_max, upper bound, estimate of the count-th
// eigenvalue from the Ritz-weight density, |beta_k|}. count <= 0 skips the estimate.
void lanczos_bounds(int64_t n, const float2* M32, int64_t ldm, int k, int count, uint64_t seed,
                    const LanczosWork& w, double* dev_out, cudaStream_t s);

// ---------------------------------------------------------------- tall-skinny kernels
// res[i] = || W_i - theta_i Q_i ||_2 for columns i of n x m blocks (deterministic 2-stage).
void resid_norms(int64_t n, int m, const double2* W, int64_t ldw, const double2* Q, int64_t ldq,
                 const double* theta, double* res, double* partial, cudaStream_t s);
size_t resid_partial_elems(int64_t n, int m);
// Column dots for the final check: out[0][i] = Re(x_i^H ax_i), out[1][i] = Re(x_i^H bx_i),
// then (second call, mode 1) out[2][i] = ||ax_i - lam_i bx_i||^2, out[3][i] = ||x_i||^2.
void final_check(int64_t n, int m, const double2* X, const double2* AX, const double2* BX, int64_t ld,
                 double* lam_io, double* res_out, double normA, double* partial, cudaStream_t s);
// Cholesky-QR helpers
void gram_scale(int m, double2* W, int64_t ldw, double* dscale, cudaStream_t s); // W <- D W D, D = diag(W)^-1/2
// G = X^H Y (X n x mx, Y n x my; G mx x my, ld ldg) on the FP64 pipe, split over n with a
// fixed-order finish in the same launch; herm = 1: the result is Hermitian (mx = my), only
// its lower tiles are formed and both triangles written. part: partials scratch (may be
// null: no split), cnt: zgram_counters() words, zero on first use (left zero).
size_t zgram_counters();
void zgram(int64_t n, int mx, int my, const double2* X, int64_t ldx, const double2* Y, int64_t ldy, double2* G,
           int64_t ldg, int herm, double2* part, size_t part_elems, unsigned* cnt, cudaStream_t s);
// Li = L^-1 D (lower, ld ldi) and optionally Lf = D^-1 L (lower, upper triangle zeroed;
// the Cholesky factor of W + shift D^-2, of W itself for shift 0, and Li its inverse),
// where D W D + shift I = L L^H, W m x m (lower triangle read; Lf may be W), D =
// diag(W)^-1/2 (1 where a diagonal entry is not positive), in one thread-block cluster.
// *info <- info_base + the 1-based index of a non-positive pivot (atomicCAS from 0;
// nothing else is written then). false: not launchable (m > cholinv_max_order() or no
// cluster): nothing was enqueued.
int cholinv_max_order();
bool cholinv_small(int m, const double2* W, int64_t ldw, double shift, double2* Li, int64_t ldi, double2* Lf,
                   int64_t ldl, int* info, cudaStream_t s, int info_base = 0);
// Recursive Cholesky factorisation with the inverse, for the emulated-product mode: A
// (n x n, lower triangle read) -> L in place (upper triangle zeroed), Li <- L^-1. A block of
// order n > kCholLeaf splits as n1 + n2 (n1 a multiple of 128 near n / 2) with
// L21 = A21 L11^-H, L22 L22^H = A22 - L21 L21^H, (L^-1)21 = -L22^-1 L21 L11^-1 as emulated
// products; leaves of order <= kCholLeaf are factored and inverted by cholinv_small.
// Resources (CholRes): digit memory for one operand of up to n x n in the A role (memA,
// oz_operand_bytes(n, n, S, 2)) and one in the B role (memB, npl 3), an n x n scratch T
// (ld ldt), optional split-K partials, the products' status words (flags[0] error code,
// flags[1] non-finite entry), the pivot word and the stream (memA, memB, T unused for
// n <= kCholLeaf). Returns cudaSuccess when enqueued; cudaErrorNotSupported when nothing
// was enqueued (no cluster launch possible); another error after work was enqueued. A
// non-positive pivot sets *info to its global 1-based index (atomicCAS from 0); the later
// launches then run on stale blocks and the results are to be discarded, the status
// words possibly set by them with them.
constexpr int64_t kCholLeaf = 256;
struct CholRes {
  char* memA;
  char* memB;
  double2* T;
  int64_t ldt;
  double* ws;
  size_t ws_doubles;
  int* flags;
  int* info;
  int S;
  cudaStream_t s;
};
cudaError_t chol_recursive(int64_t n, double2* A, int64_t lda, double2* Li, int64_t ldi, const CholRes& r);

// ---------------------------------------------------------------- backward
// GA = gE X X^H, GB = -gE X diag(lam) X^H (lower tiles by GEMM, then Hermitian completion
// scaled by the device scalar *gE). XL: n x nev scratch.
void energy_backward_ws(int64_t n, int nev, const double2* X, int64_t ldx, const double* lam, const double* gE,
                        double2* GA, double2* GB, int64_t ldg, double2* XL, double2* split, size_t split_elems,
                        cudaStream_t s);

// ---------------------------------------------------------------- low-precision filter (tcgen05)
struct FilterTC;   // opaque, owned by the handle
bool tc_filter_supported();
cudaError_t filter_tc_reserve(FilterTC** f, int64_t n, int m, cudaStream_t s);
void filter_tc_release(FilterTC* f);
// nsplit: BF16 pieces per operand (1 = BF16 filter, 3 = FP32-class, see filter_tc.cu)
cudaError_t filter_tc_set_matrix(FilterTC* f, int64_t n, const double2* C, int64_t ldc, int nsplit, cudaStream_t s);
cudaError_t filter_tc_apply(FilterTC* f, int64_t n, int m, const double2* Y, int64_t ldy, double2* Yout,
                            int64_t ldo, int deg, double lo, double hi, double sc, int nsplit, int* err_host,
                            cudaStream_t s);
cudaError_t filter_tc_apply_corrected(FilterTC* f, int64_t n, int m, const double2* Q, int64_t ldq, const double2* W,
                                      int64_t ldw, const double* theta_dev, const double* theta_host, double2* Yout,
                                      int64_t ldo, int deg, double lo, double hi, double sc, int nsplit,
                                      cudaStream_t s);
cudaError_t filter_tc_product(FilterTC* f, int64_t n, int m, const double2* Y, int64_t ldy, double2* D, int64_t ldd,
                              int nsplit, int* err_host, cudaStream_t s);

// ---------------------------------------------------------------- batched (k-point) form
// One descriptor per problem of a batch, in device memory; batched kernels take the array
// and select their problem by a block index. Problems whose *active flag is zero return
// at once, so a launch sequence keeps its shape while problems converge. Every n x m
// block has ld = m, every m x m block ld = m, every n x n matrix ld = n.
constexpr int kBDegMax = 64;   // highest filter degree of the batched form
struct BDesc {
  int n, m, nev, kl;          // kl: Lanczos steps
  const double2* A; int64_t lda;
  const double2* B; int64_t ldb;
  double2 *L, *Linv, *C, *T;  // n x n
  float2* M32;                // n x n FP32 copy for Lanczos
  double2 *Q, *Y1, *Y2, *W, *Wt, *Xf;   // n x m
  double2 *G, *Zs, *Gw, *Gwi;           // m x m
  // small eigensolver
  float2 *G32, *Z32; float* w32; int* perm;
  double2 *hZ, *hR, *hS, *hT, *hE;      // m x m
  double *hlam, *hscal;
  // Lanczos
  float2 *V, *lvec, *T32, *LZ32; float *ab, *lw32; int* lperm;
  // per-column and per-problem scalars
  double *theta, *res, *lamf, *resf, *dscale, *partial;
  double* bounds;             // see bkernels.cu for the slot map
  double* fco;                // [kBDegMax][3] recurrence coefficients of the current round
  int* flags;                 // [0] active, [1] degree, [2] info, [3] state, [4] rounds,
                              // [5] fp64 filter, [6] filter active (tc), [7] filter active (fp64)
  int* stepact;               // [kBDegMax] FP64 filter: step j runs for this problem
  const int* active;          // = flags
  // tensor-core filter state
  int n_pad, ncols_pad, nchunk, nchunks, mtiles, ks, kbps, nseg;
  unsigned tmem_cols; int unit_start;
  const void* maps;           // 18 CUtensorMap (C pieces, then block pieces), 64-byte aligned
  __nv_bfloat16 *Cp, *Yp;
  float2 *S0, *S1, *S2, *S3, *tws;
  float* pcoef;               // [kBDegMax][ncols_pad]
  double* pfinal;             // [ncols_pad]
  int nsplit, pad_;
};

void bk_herm_sum(const BDesc* D, int np, int64_t nmax, cudaStream_t s);
void bk_to_c32(const BDesc* D, int np, int64_t nmax, int which, cudaStream_t s);
void bk_hermitize_lower_G(const BDesc* D, int np, int mmax, cudaStream_t s);
void bk_gram_scale(const BDesc* D, int np, double shift_factor, cudaStream_t s);
void bk_col_scale(const BDesc* D, int np, int64_t nm_max, int which, cudaStream_t s);
void bk_copy_nm(const BDesc* D, int np, int64_t nm_max, int from, int to, cudaStream_t s);
void bk_potrf_small(const BDesc* D, int np, cudaStream_t s);
void bk_trtri_small(const BDesc* D, int np, cudaStream_t s);
void bk_step_reset(const BDesc* D, int np, double tol, int filter64, cudaStream_t s);
void bk_lanczos(const BDesc* D, int np, int64_t nmax, int k, int use_count, int out_off, uint64_t seed,
                cudaStream_t s);
void bk_post_bounds(const BDesc* D, int np, cudaStream_t s);
void bk_heev_prep(const BDesc* D, int np, int mmax, cudaStream_t s);
void bk_oa_scalars(const BDesc* D, int np, cudaStream_t s);
void bk_oa_update(const BDesc* D, int np, int mmax, int only_orth, cudaStream_t s);
void bk_hermitize_avg_S(const BDesc* D, int np, int mmax, cudaStream_t s);
void bk_sort_pairs(const BDesc* D, int np, int zsel, cudaStream_t s);
void bk_resid(const BDesc* D, int np, int mmax, cudaStream_t s);
void bk_final_check(const BDesc* D, int np, int nevmax, cudaStream_t s);
void bk_final_status(const BDesc* D, int np, int* out, cudaStream_t s);
void bk_cheb_coef(const BDesc* D, int np, int deg_min, const int* deg_cap, cudaStream_t s);
void bk_fp64_select(const BDesc* D, int np, int64_t nm_max, cudaStream_t s);
void bk_round_status(const BDesc* D, int np, int* out, cudaStream_t s);
void bk_randn(const BDesc* D, int np, int64_t nm_max, uint64_t seed, const int* mask, cudaStream_t s);
void bk_force_final(const BDesc* D, int np, cudaStream_t s);
struct BOut { double* lam; double* res; double2* X; int64_t ldx; };
void bk_write_out(const BDesc* D, const BOut* O, int np, int64_t nm_max, cudaStream_t s);
size_t bk_partial_elems(int m);
// batched FP32 Jacobi: which = 0 -> G32 (m x m) into Z32/w32/perm; 1 -> T32 (k x k) into LZ32/lw32/lperm
void jacobi32_batched(const BDesc* D, int np, int which, int k, int mmax, int max_sweeps, cudaStream_t s);
void cluster_jacobi_batched(const BDesc* D, int np, int zsel, double rel, int max_sweeps, cudaStream_t s);

// grouped tensor-core filter (residual-corrected recurrence) over the problems of a batch
void tcg_geometry(int64_t n, int m, int* n_pad, int* ncols_pad, int* nchunk, int* nchunks);
int tcg_nseg(int nsplit);
size_t tcg_smem_bytes(int nchunk_max);
size_t tcg_map_bytes();                                  // bytes of one problem's tensor maps
bool tcg_encode_maps(const BDesc& d, void* maps_host);   // host copy of d's maps (Cp, Yp set)
void tcg_set_matrix(const BDesc* D, int np, int64_t npad2_max, cudaStream_t s);
struct TcgShape { int np, units, n_pad_max, ncols_pad_max, nchunk_max, steps; int64_t nc_max; };
cudaError_t tcg_prepare(int nchunk_max);
cudaError_t tcg_filter(const BDesc* D, const TcgShape& g, int* err, cudaStream_t s);

// ---------------------------------------------------------------- matrix variation
int variation_max_thresholds();
// ws: >= 48 words; [0] max of squared moduli (bits), [1] NaN flag, [2..] counts;
// d2: n * n words of scratch
void matrix_variation(int64_t n, const double2* A, int64_t lda, const double2* B, int64_t ldb, int nthr,
                      const double* p_dev, unsigned long long* ws, unsigned long long* d2, uint8_t* mask,
                      cudaStream_t s);

// ---------------------------------------------------------------- emulated FP64 GEMM
// An operand of the emulated product in digit form: `rows` rows of op(A) (npl = 2: planes
// re, im) or columns of op(B) (npl = 3: re, im, -im), each K entries split into S base-128
// digits, planes [npl][S][rows_pad][k_pad] BF16, followed by one exponent per row.
constexpr int kOzSlicesMax = 8;
struct OzOperand {
  __nv_bfloat16* planes = nullptr;
  int* ex = nullptr;
  int rows = 0, K = 0, rows_pad = 0, k_pad = 0, S = 0, npl = 0;
};
size_t oz_operand_bytes(int rows, int K, int S, int npl);
bool oz_supported();
// rows of X (cols = false; X is rows x K) or its columns (cols = true; X is K x rows) as
// operand rows, conjugated if conj, mask 1: k >= r with the diagonal halved, 2: k <= r,
// 3: k >= r; into digit form in `mem` (oz_operand_bytes); *bad = 1 on a non-finite entry
// active: nullable device flag, 0 = the launch does nothing (a converged batch problem)
cudaError_t oz_split(OzOperand& op, void* mem, int rows, int K, const double2* X, int64_t ldx, int conj, int mask,
                     int S, int npl, int* bad, cudaStream_t s, bool cols = false, const int* active = nullptr);
// D (A.rows x B.rows) = op(A) op(B); triA 1: op(A) lower; triB 1: op(B) lower, 2: upper
// ws (nullable, ws_doubles >= oz_split_k_doubles(M, N)): when the grid would leave SMs
// idle, K is cut into up to kOzSplitKMax slices whose FP64 partials are summed in slice order
constexpr int kOzSplitKMax = 8;
size_t oz_split_k_doubles(int M, int N);
cudaError_t oz_gemm(const OzOperand& A, const OzOperand& B, int triA, int triB, double2* D, int64_t ldd, int* err,
                    cudaStream_t s, const int* active = nullptr, double* ws = nullptr, size_t ws_doubles = 0);

// ---------------------------------------------------------------- deviation angles
// slices of the column-norm reduction (part needs slices * k doubles)
int deviation_norm_slices(int64_t n);
// nrm2[j] = Re(x_j^H w_j) for the columns of X, W (n x k)
void column_bnorms(int64_t n, int k, const double2* X, int64_t ldx, const double2* W, int64_t ldw, double* part,
                   double* nrm2, cudaStream_t s);
// c[i][j] = min(1, |O[i][j]| / sqrt(no2[i] nn2[j])); *bad = 1 on a norm that is not positive
void overlap_cosines(int ko, int kn, const double2* O, int64_t ldo, const double* no2, const double* nn2, double* c,
                     int64_t ldc, int* bad, cudaStream_t s);
// host: minimum-cost assignment of the ko rows of a ko x kn (ko <= kn) table to distinct columns
void assign_min_cost(int ko, int kn, const double* cost, int64_t* perm);

// handle access for the translation units outside the main driver
struct BatchPlan;
void batch_release(BatchPlan* p);
}  // namespace gevp
struct gevp_ctx;
namespace gevp {
cudaStream_t ctx_stream(gevp_ctx* h);
int ctx_device(gevp_ctx* h);
void ctx_set_error(gevp_ctx* h, const char* msg);
BatchPlan*& ctx_batch(gevp_ctx* h);

// ---------------------------------------------------------------- probes
void probe_peaks(double* fp64_fma_tflops, double* fp64_dmma_tflops, double* fp32_fma_tflops, cudaStream_t s);

// ---------------------------------------------------------------- launch accounting
// process-wide count of kernel launches (all handles, the handle-less entry points, all
// host threads)
extern std::atomic<int64_t> g_launches;
#define LAUNCH_NOTE(k) (::gevp::g_launches += (k))

// ---------------------------------------------------------------- live kernel timing
// Classes: 0 the FP64 complex GEMM (zgemm_kernel), 1 the emulated product (oz_gemm_kernel),
// 2 the tall-skinny Gram kernel (zgram_kernel).
// kt_begin records an event on s and returns it (only call when kt_enabled()); kt_end
// records the closing event with the launch's algorithmic and executed flop.
bool kt_enabled();
void* kt_begin(cudaStream_t s);
void kt_end(void* begin, int cls, double alg, double exec, cudaStream_t s);
double tiled_product_flops(int M, int N, int K, int triA, int triB, int triD);

// ---------------------------------------------------------------- error handling
#define GEVP_CUDA_TRY(x)                                   \
  do {                                                     \
    cudaError_t e__ = (x);                                 \
    if (e__ != cudaSuccess) return e__;                    \
  } while (0)

}  // namespace gevp
