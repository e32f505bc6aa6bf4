// Blocked right-looking complex Cholesky B = L L^H and blocked lower-triangular inverse.
// The serial diagonal-block work runs in one CTA per 32 x 32 block; the panel solve is
// spread one row per thread over many CTAs, and the trailing Hermitian update and the
// inverse's off-diagonal blocks are FP64 GEMMs over all SMs.
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

constexpr int NB = 32;

// Unblocked Cholesky of the kb x kb diagonal block at A (lower, in place). On a
// non-positive pivot the block is left partial and *info receives k0 + j + 1 (first
// failure only). Does nothing if *info is already set.
__global__ void potrf_diag_kernel(double2* A, int64_t lda, int kb, int64_t k0, int* info) {
  __shared__ double2 S[NB][NB + 1];
  __shared__ int fail;
  if (*info != 0) return;
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    int i = e / kb, j = e % kb;
    S[i][j] = (j <= i) ? A[i * lda + j] : make_double2(0.0, 0.0);
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      double d = S[j][j].x;
      if (!(d > 0.0)) {
        fail = 1;
        atomicCAS(info, 0, (int)(k0 + j + 1));
      } else {
        S[j][j] = make_double2(sqrt(d), 0.0);
      }
    }
    __syncthreads();
    if (fail) break;
    double inv = 1.0 / S[j][j].x;
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) S[i][j] = zscale(S[i][j], inv);
    __syncthreads();
    // trailing update of the lower part: S[i][l] -= S[i][j] conj(S[l][j]), j < l <= i
    int rem = kb - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      int i = j + 1 + e / rem, l = j + 1 + e % rem;
      if (l <= i) {
        double2 v = S[i][l];
        zfma(v, zscale(S[i][j], -1.0), zconj(S[l][j]));
        S[i][l] = v;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    int i = e / kb, j = e % kb;
    A[i * lda + j] = (j <= i) ? S[i][j] : make_double2(0.0, 0.0);
  }
}

// Panel solve X L11^H = A21 in place, one row of A21 per thread (rows independent).
template <int KB>
__global__ void trsm_panel_kernel(double2* A21, int64_t lda, int64_t rows, const double2* L11, int kb,
                                  const int* info) {
  __shared__ double2 Ls[KB][KB];
  __shared__ double dinv[KB];
  if (*info != 0) return;
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) Ls[e / kb][e % kb] = L11[(e / kb) * lda + (e % kb)];
  __syncthreads();
  for (int j = threadIdx.x; j < kb; j += blockDim.x) dinv[j] = 1.0 / Ls[j][j].x;
  __syncthreads();
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double2* row = A21 + r * lda;
  double2 x[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) {
    if (j < kb) {
      double2 s = row[j];
#pragma unroll
      for (int k = 0; k < KB; ++k)
        if (k < j) zfma(s, zscale(x[k], -1.0), zconj(Ls[j][k]));
      x[j] = zscale(s, dinv[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < KB; ++j)
    if (j < kb) row[j] = x[j];
}

// Inverse of the lower-triangular diagonal blocks (size <= NB) of L, written into Linv.
// One CTA per block; thread c forward-substitutes column c.
__global__ void trtri_diag_kernel(int64_t n, const double2* L, int64_t ldl, double2* Linv, int64_t ldi) {
  __shared__ double2 Ls[NB][NB + 1];
  __shared__ double2 Xs[NB][NB + 1];
  int64_t k0 = (int64_t)blockIdx.x * NB;
  int kb = (int)std::min<int64_t>(NB, n - k0);
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    int i = e / kb, j = e % kb;
    Ls[i][j] = L[(k0 + i) * ldl + k0 + j];
  }
  __syncthreads();
  int c = threadIdx.x;
  if (c < kb) {
    for (int i = 0; i < kb; ++i) {
      double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
      if (i < c) { Xs[i][c] = make_double2(0.0, 0.0); continue; }
      for (int k = c; k < i; ++k) zfma(s, zscale(Ls[i][k], -1.0), Xs[k][c]);
      // divide by the (real, positive) diagonal; tolerate a complex diagonal too
      double2 d = Ls[i][i];
      double den = zabs2(d);
      Xs[i][c] = zscale(zmul(s, zconj(d)), 1.0 / den);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    int i = e / kb, j = e % kb;
    Linv[(k0 + i) * ldi + k0 + j] = (j <= i) ? Xs[i][j] : make_double2(0.0, 0.0);
  }
}

void trtri_combine(int64_t n, const double2* L, int64_t ldl, double2* Linv, int64_t ldi, double2* T,
                   double2* split, size_t split_elems, cudaStream_t s) {
  if (n <= NB) return;
  int64_t n1 = ((n / 2 + NB - 1) / NB) * NB;
  int64_t n2 = n - n1;
  trtri_combine(n1, L, ldl, Linv, ldi, T, split, split_elems, s);
  trtri_combine(n2, L + n1 * ldl + n1, ldl, Linv + n1 * ldi + n1, ldi, T, split, split_elems, s);
  // T = L21 * Linv11 (n2 x n1); Linv11 lower
  ZgemmArgs a = zg((int)n2, (int)n1, (int)n1, L + n1 * ldl, ldl, 0, Linv, ldi, 0, T, n1);
  a.triB = 1;
  zgemm(a, split, split_elems, s);
  // Linv21 = -Linv22 * T ; Linv22 lower
  ZgemmArgs b = zg((int)n2, (int)n1, (int)n2, Linv + n1 * ldi + n1, ldi, 0, T, n1, 0, Linv + n1 * ldi, ldi, -1.0);
  b.triA = 1;
  zgemm(b, split, split_elems, s);
}

}  // namespace

size_t potrf_ws_elems(int64_t n) { return 0; }

size_t trtri_ws_elems(int64_t n) {
  int64_t n1 = ((n / 2 + NB - 1) / NB) * NB;
  int64_t n2 = n - n1;
  return (size_t)std::max<int64_t>(1, n1 * std::max<int64_t>(n2, 1));
}

void potrf_lower(int64_t n, double2* A, int64_t lda, int* info_dev, double2* ws, size_t ws_elems,
                 cudaStream_t s) {
  (void)ws; (void)ws_elems;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    int kb = (int)std::min<int64_t>(NB, n - k0);
    double2* Akk = A + k0 * lda + k0;
    potrf_diag_kernel<<<1, 256, 0, s>>>(Akk, lda, kb, k0, info_dev);
    LAUNCH_NOTE(1);
    int64_t rem = n - k0 - kb;
    if (rem <= 0) break;
    double2* A21 = A + (k0 + kb) * lda + k0;
    int threads = 32;
    int blocks = (int)((rem + threads - 1) / threads);
    trsm_panel_kernel<NB><<<blocks, threads, 0, s>>>(A21, lda, rem, Akk, kb, info_dev);
    LAUNCH_NOTE(1);
    // A22 -= L21 L21^H (lower tiles only)
    double2* A22 = A + (k0 + kb) * lda + (k0 + kb);
    ZgemmArgs g = zg((int)rem, (int)rem, kb, A21, lda, 0, A21, lda, 1, A22, lda, -1.0);
    g.Cin = A22; g.ldc = lda; g.beta = 1.0;
    g.triD = 1;
    zgemm(g, nullptr, 0, s);
  }
  zero_upper(n, A, lda, s);
}

void trtri_lower(int64_t n, const double2* L, int64_t ldl, double2* Linv, int64_t ldi, double2* ws,
                 size_t ws_elems, cudaStream_t s) {
  zero_upper(n, Linv, ldi, s);
  int nblk = (int)((n + NB - 1) / NB);
  trtri_diag_kernel<<<nblk, NB, 0, s>>>(n, L, ldl, Linv, ldi);
  LAUNCH_NOTE(1);
  // ws holds T (first trtri_ws_elems) and the split-K scratch after it
  size_t tel = trtri_ws_elems(n);
  double2* split = (ws_elems > tel) ? ws + tel : nullptr;
  size_t split_elems = (ws_elems > tel) ? ws_elems - tel : 0;
  trtri_combine(n, L, ldl, Linv, ldi, ws, split, split_elems, s);
}

}  // namespace gevp
