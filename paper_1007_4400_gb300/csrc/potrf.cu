// Blocked right-looking complex Cholesky B = L L^H and blocked lower-triangular inverse.
// The serial diagonal-block work runs in one CTA per 32 x 32 block, which also inverts
// the factored block while it is in shared memory; the panel solve X L11^H = A21 is then
// the product X = A21 L11^-H with every element computed in parallel (a row-per-thread
// substitution would leave almost all SMs idle: one SM retires only about two FP64 FMAs
// per clock on this part); the trailing Hermitian update and the inverse's off-diagonal
// blocks are FP64 GEMMs over all SMs.
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

constexpr int NB = 32;

// Unblocked Cholesky of the kb x kb diagonal block at A (lower, in place), and the
// inverse of the factored block written to Li (lower, zero above). On a non-positive
// pivot the block is left partial and *info receives k0 + j + 1 (first failure only).
// Does nothing if *info is already set.
__global__ void potrf_diag_kernel(double2* A, int64_t lda, int kb, int64_t k0, int* info, double2* Li,
                                  int64_t ldi) {
  __shared__ double2 S[NB][NB + 1];
  __shared__ double2 X[NB][NB + 1];
  __shared__ double rdiag[NB];
  __shared__ double pinv;   // 1 / pivot of the current column (one FP64 division per column)
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
        // one reciprocal square root, then the root as d * rsqrt(d)
        const double ri = rsqrt(d);
        S[j][j] = make_double2(d * ri, 0.0);
        pinv = ri;
      }
    }
    __syncthreads();
    if (fail) break;
    // FP64 division is an iterative sequence on the FP64 pipe (two FMAs per clock per SM
    // here): one thread forms the reciprocal, the others read it
    const double inv = pinv;
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
  if (fail) return;
  // inverse: row i of X = S^-1 from rows < i: X[i][i] = 1 / s_ii and, for c < i,
  // X[i][c] = -(1 / s_ii) sum_{k=c}^{i-1} S[i][k] X[k][c]. One warp per column, the lanes
  // splitting the sum: a product and a five-level shuffle reduction instead of a chain of
  // up to kb dependent FP64 operations per thread (the block otherwise waits at barriers)
  for (int j = tid; j < kb; j += blockDim.x) rdiag[j] = 1.0 / S[j][j].x;
  __syncthreads();
  const int lane = tid & 31, wid = tid >> 5, nw = (int)(blockDim.x >> 5);
  for (int i = 0; i < kb; ++i) {
    for (int c = wid; c <= i; c += nw) {
      double sx = 0.0, sy = 0.0;
      for (int k = c + lane; k < i; k += 32) {
        const double2 l = S[i][k], x = X[k][c];
        sx = fma(l.x, x.x, fma(-l.y, x.y, sx));
        sy = fma(l.x, x.y, fma(l.y, x.x, sy));
      }
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0) X[i][c] = c == i ? make_double2(rdiag[i], 0.0) : make_double2(-rdiag[i] * sx, -rdiag[i] * sy);
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    int i = e / kb, j = e % kb;
    Li[i * ldi + j] = (j <= i) ? X[i][j] : make_double2(0.0, 0.0);
  }
}

// Panel X = A21 L11^-H in place (solves X L11^H = A21), Li = L11^-1 lower:
// X[r][j] = sum_{k <= j} A21[r][k] conj(Li[j][k]). RB rows per CTA, staged in shared
// memory (every output of a row reads the row's first j + 1 inputs).
template <int RB>
__global__ void panel_apply_kernel(double2* A21, int64_t lda, int64_t rows, const double2* Li, int64_t ldi, int kb,
                                   const int* info) {
  __shared__ double2 Ls[NB][NB + 1];
  __shared__ double2 As[RB][NB + 1];
  if (*info != 0) return;
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int e = tid; e < kb * kb; e += blockDim.x) Ls[e / kb][e % kb] = Li[(e / kb) * ldi + (e % kb)];
  for (int e = tid; e < RB * kb; e += blockDim.x) {
    int rr = e / kb, k = e % kb;
    As[rr][k] = (r0 + rr < rows) ? A21[(r0 + rr) * lda + k] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int e = tid; e < RB * kb; e += blockDim.x) {
    int rr = e / kb, j = e % kb;
    if (r0 + rr >= rows) continue;
    double2 v = make_double2(0.0, 0.0);
    for (int k = 0; k <= j; ++k) zfma(v, As[rr][k], zconj(Ls[j][k]));
    A21[(r0 + rr) * lda + j] = v;
  }
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

size_t trtri_ws_elems(int64_t n) {
  int64_t n1 = ((n / 2 + NB - 1) / NB) * NB;
  int64_t n2 = n - n1;
  return (size_t)std::max<int64_t>(1, n1 * std::max<int64_t>(n2, 1));
}

void potrf_lower(int64_t n, double2* A, int64_t lda, int* info_dev, double2* Linv, int64_t ldi, cudaStream_t s) {
  constexpr int RB = 8;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    int kb = (int)std::min<int64_t>(NB, n - k0);
    double2* Akk = A + k0 * lda + k0;
    double2* Likk = Linv + k0 * ldi + k0;
    potrf_diag_kernel<<<1, 1024, 0, s>>>(Akk, lda, kb, k0, info_dev, Likk, ldi);
    LAUNCH_NOTE(1);
    int64_t rem = n - k0 - kb;
    if (rem <= 0) break;
    double2* A21 = A + (k0 + kb) * lda + k0;
    int blocks = (int)((rem + RB - 1) / RB);
    panel_apply_kernel<RB><<<blocks, RB * NB, 0, s>>>(A21, lda, rem, Likk, ldi, kb, info_dev);
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
                 size_t ws_elems, cudaStream_t s, bool diag_ready) {
  zero_upper(n, Linv, ldi, s);
  if (!diag_ready) {
    int nblk = (int)((n + NB - 1) / NB);
    trtri_diag_kernel<<<nblk, NB, 0, s>>>(n, L, ldl, Linv, ldi);
    LAUNCH_NOTE(1);
  }
  // ws holds T (first trtri_ws_elems) and the split-K scratch after it
  size_t tel = trtri_ws_elems(n);
  double2* split = (ws_elems > tel) ? ws + tel : nullptr;
  size_t split_elems = (ws_elems > tel) ? ws_elems - tel : 0;
  trtri_combine(n, L, ldl, Linv, ldi, ws, split, split_elems, s);
}

}  // namespace gevp
