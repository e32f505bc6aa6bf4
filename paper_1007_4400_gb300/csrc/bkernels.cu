// Batched kernels of the k-point form: one launch covers every problem of a batch, and
// the problem is selected by a block index. Problems whose active flag is zero return at
// once, so a launch sequence keeps its shape (and can be captured once as a CUDA graph)
// while problems converge and drop out.
//
// Per-problem scalars, BDesc::bounds (double):
//   [0..4]  Lanczos on C: theta_min, theta_max, upper bound, estimate of the m-th
//           eigenvalue, |beta_k|          [12..16] the same for A
//   [5] ||A||_2 estimate   [6] tolerance in the standard space   [7] ||C||_2 estimate
//   [8] largest residual of the previous round   [9] lo  [10] hi  [11] scaling point
//   [17] tolerance in the original space         [18] largest residual of this round
//   [19] largest residual at the start of the step
//   [20] Chebyshev convergence factor of the nev-th Ritz value
//   [21] largest residual predicted for the end of this round
// Per-problem flags, BDesc::flags (int):
//   [0] active (rounds still run)  [1] filter degree of this round  [2] Cholesky info
//   [3] state: 0 iterating, 1 converged in the standard space (final check pending),
//       2 done, 3 gave up   [4] rounds  [5] FP64 filter  [6] tensor-core filter runs
//   [7] FP64 filter runs  [8] CholQR failures  [9] filter steps  [10] precision switches
//   [11] final passes  [12] final check runs  [13] degree cap after filter stalls
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

__device__ __forceinline__ bool live(const BDesc& d) { return d.flags[0] != 0; }

__device__ double bsum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

__device__ double bmax_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double2* nm_block(const BDesc& d, int which) {
  switch (which) {
    case 0: return d.Y1;
    case 1: return d.Y2;
    case 2: return d.Q;
    case 3: return d.W;
    default: return d.Wt;
  }
}

// ---------------------------------------------------------------- elementwise
__global__ void b_herm_sum(const BDesc* D) {   // C <- C + C^H
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  int64_t n = d.n, total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (j < i) {
      double2 a = d.C[i * n + j], b = d.C[j * n + i];
      double2 v = make_double2(a.x + b.x, a.y - b.y);
      d.C[i * n + j] = v;
      d.C[j * n + i] = zconj(v);
    } else if (j == i) {
      d.C[i * n + i] = make_double2(2.0 * d.C[i * n + i].x, 0.0);
    }
  }
}

// FP32 copy of C (which = 0) or of A (which = 1) for the Lanczos bounds
__global__ void b_to_c32(const BDesc* D, int which) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  int64_t n = d.n, total = n * n;
  const double2* src = which == 0 ? d.C : d.A;
  int64_t lds = which == 0 ? n : d.lda;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    double2 v = src[i * lds + j];
    d.M32[e] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void b_hermitize_lower_G(const BDesc* D) {   // Gw: upper <- conj(lower), real diagonal
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  int m = d.m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int i = e / m, j = e % m;
    if (j > i) d.Gw[e] = zconj(d.Gw[j * m + i]);
    else if (j == i) d.Gw[e].y = 0.0;
  }
}

// Gw <- S Gw S (+ shift on the diagonal), S = diag(Gw)^-1/2 kept in dscale. The shift of
// shifted CholQR (Fukaya et al., SIAM J. Sci. Comput. 42, 2020) is
// 11 (n m + m (m + 1)) u ||Y S||_2^2 with ||Y S||_2^2 <= ||Y S||_F^2 = m.
__global__ void b_gram_scale(const BDesc* D, double shift_factor) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  int m = d.m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double v = d.Gw[i * m + i].x;
    d.dscale[i] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
  }
  __syncthreads();
  double sh = shift_factor * 11.0 * ((double)d.n * m + (double)m * (m + 1)) * 1.1102230246251565e-16 * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e / m, j = e % m;
    double2 v = zscale(d.Gw[e], d.dscale[i] * d.dscale[j]);
    if (i == j) v.x += sh;
    d.Gw[e] = v;
  }
}

__global__ void b_col_scale(const BDesc* D, int which) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  double2* Y = nm_block(d, which);
  int64_t m = d.m, total = (int64_t)d.n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = zscale(Y[e], d.dscale[e % m]);
}

__global__ void b_copy_nm(const BDesc* D, int from, int to) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  const double2* s = nm_block(d, from);
  double2* t = nm_block(d, to);
  int64_t total = (int64_t)d.n * d.m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    t[e] = s[e];
}

// ---------------------------------------------------------------- small dense FP64, one CTA per problem
// Cholesky of Gw in place (lower, strict upper zeroed); a failing pivot is recorded in
// flags[2] (1-based) and leaves the block unusable for this round.
__global__ void __launch_bounds__(1024) b_potrf_small(const BDesc* D) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  __shared__ int fail;
  __shared__ double pinv;   // 1 / pivot: one FP64 division per column, not one per thread
  const int m = d.m;
  double2* A = d.Gw;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      double v = A[j * m + j].x;
      if (!(v > 0.0)) fail = j + 1;
      else {
        const double r = sqrt(v);
        A[j * m + j] = make_double2(r, 0.0);
        pinv = 1.0 / r;
      }
    }
    __syncthreads();
    if (fail) break;
    const double inv = pinv;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i * m + j] = zscale(A[i * m + j], inv);
    __syncthreads();
    const int rem = m - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = j + 1 + e / rem, l = j + 1 + e % rem;
      if (l <= i) {
        double2 v = A[i * m + l], a = A[i * m + j], b = A[l * m + j];
        // v -= a conj(b)
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.y * b.x - a.x * b.y;
        A[i * m + l] = v;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && fail) d.flags[2] = fail;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x)
    if ((e % m) > (e / m)) A[e] = make_double2(0.0, 0.0);
}

// Gwi = Gw^-1 (lower triangular): row i of the inverse from rows < i, all columns in parallel.
__global__ void __launch_bounds__(1024) b_trtri_small(const BDesc* D) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  const int m = d.m;
  const double2* L = d.Gw;
  double2* X = d.Gwi;
  // reciprocals of the diagonal, one division per row (m <= 1024)
  __shared__ double rdiag[1024];
  for (int i = threadIdx.x; i < m; i += blockDim.x) rdiag[i] = 1.0 / L[i * m + i].x;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) X[e] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int i = 0; i < m; ++i) {
    const double inv = rdiag[i];
    for (int c = threadIdx.x; c <= i; c += blockDim.x) {
      double2 s = make_double2(c == i ? 1.0 : 0.0, 0.0);
      for (int k = c; k < i; ++k) {
        double2 l = L[i * m + k], x = X[k * m + c];
        s.x -= l.x * x.x - l.y * x.y;
        s.y -= l.x * x.y + l.y * x.x;
      }
      X[i * m + c] = zscale(s, inv);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Lanczos (FP32) on M32
constexpr int KMAX = 64;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void __launch_bounds__(1024) b_lanczos_init(const BDesc* D, uint64_t seed) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  __shared__ double red[32];
  const int64_t n = d.n;
  const uint64_t sd = seed + 0x2545F4914F6CDD1Dull * (uint64_t)blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    uint64_t h1 = mix64(sd ^ mix64(2 * (uint64_t)i)), h2 = mix64(sd ^ mix64(2 * (uint64_t)i + 1));
    float2 z = make_float2(((float)(h1 >> 40) + 0.5f) * (1.0f / 16777216.0f) - 0.5f,
                           ((float)(h2 >> 40) + 0.5f) * (1.0f / 16777216.0f) - 0.5f);
    d.V[i] = z;
    s += (double)z.x * z.x + (double)z.y * z.y;
  }
  s = bsum_d(s, red);
  const float inv = (float)(1.0 / sqrt(s));
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) d.V[i] = make_float2(d.V[i].x * inv, d.V[i].y * inv);
  if (threadIdx.x == 0) ((int*)(d.ab + 2 * KMAX))[0] = 0;
}

__global__ void b_matvec32(const BDesc* D, int j) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  if (((const int*)(d.ab + 2 * KMAX))[0] < j) return;   // broke down earlier
  const int64_t n = d.n;
  const float2* v = d.V + (int64_t)j * n;
  const int lane = threadIdx.x % 32;
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32; row < n;
       row += (int64_t)gridDim.x * (blockDim.x / 32)) {
    const float2* r = d.M32 + row * n;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t c = lane; c < n; c += 32) cfma(acc, r[c], v[c]);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) d.lvec[row] = acc;
  }
}

// two passes of classical Gram-Schmidt against V[0..j], then normalise into V[j+1]
__global__ void __launch_bounds__(1024) b_lanczos_update(const BDesc* D, int j) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  __shared__ float2 red[32][KMAX + 1];
  __shared__ float2 h[KMAX + 1];
  __shared__ float nrm;
  const int lane = threadIdx.x % 32, wp = threadIdx.x / 32, nw = blockDim.x / 32;
  int* keff = (int*)(d.ab + 2 * KMAX);
  if (*keff < j) return;
  const int64_t n = d.n;
  float2* w = d.lvec;
  for (int pass = 0; pass < 2; ++pass) {
    for (int c = 0; c <= j; ++c) {
      const float2* vc = d.V + (int64_t)c * n;
      float2 p = make_float2(0.f, 0.f);
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        float2 a = vc[i], b = w[i];
        p.x += a.x * b.x + a.y * b.y;
        p.y += a.x * b.y - a.y * b.x;
      }
      for (int o = 16; o > 0; o >>= 1) {
        p.x += __shfl_xor_sync(0xffffffffu, p.x, o);
        p.y += __shfl_xor_sync(0xffffffffu, p.y, o);
      }
      if (lane == 0) red[wp][c] = p;
    }
    __syncthreads();
    for (int c = threadIdx.x; c <= j; c += blockDim.x) {
      float2 t = make_float2(0.f, 0.f);
      for (int q = 0; q < nw; ++q) { t.x += red[q][c].x; t.y += red[q][c].y; }
      h[c] = t;
      if (pass == 0 && c == j) d.ab[2 * j] = t.x;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      float2 b = w[i];
      for (int c = 0; c <= j; ++c) {
        float2 a = d.V[(int64_t)c * n + i], hc = h[c];
        b.x -= a.x * hc.x - a.y * hc.y;
        b.y -= a.x * hc.y + a.y * hc.x;
      }
      w[i] = b;
    }
    __syncthreads();
  }
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) { float2 b = w[i]; s += b.x * b.x + b.y * b.y; }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[wp][0].x = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int q = 0; q < nw; ++q) t += red[q][0].x;
    nrm = sqrtf(t);
    d.ab[2 * j + 1] = nrm;
    float scale = fabsf(d.ab[2 * j]) + (j > 0 ? d.ab[2 * j - 1] : 0.f);
    *keff = (nrm > 1e-6f * scale && nrm > 0.f) ? j + 1 : -(j + 1);
  }
  __syncthreads();
  if (*keff < 0) return;
  const float inv = 1.f / nrm;
  float2* vn = d.V + (int64_t)(j + 1) * n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) { float2 b = w[i]; vn[i] = make_float2(b.x * inv, b.y * inv); }
}

// the k x k tridiagonal, padded far above the spectrum after a breakdown
__global__ void b_build_T(const BDesc* D, int k) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  int* kf = (int*)(d.ab + 2 * KMAX);
  const int ke = kf[0];
  int kk = ke < 0 ? -ke : (ke > k ? k : ke);
  if (kk < 1) kk = 1;
  __syncthreads();
  if (threadIdx.x == 0) kf[1] = kk;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    float v = 0.f;
    if (i >= kk || j >= kk) v = (i == j) ? 1e30f : 0.f;
    else if (i == j) v = d.ab[2 * i];
    else if (j == i + 1) v = d.ab[2 * i + 1];
    else if (i == j + 1) v = d.ab[2 * j + 1];
    d.T32[e] = make_float2(v, 0.f);
  }
}

__global__ void b_lanczos_finish(const BDesc* D, int k, int use_count, int out_off) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d) || threadIdx.x != 0) return;
  const int* kf = (const int*)(d.ab + 2 * KMAX);
  const int ke = kf[0], kk = kf[1];
  const double tmin = d.lw32[0], tmax = d.lw32[kk - 1];
  const double beta = (ke < 0) ? 0.0 : fabs((double)d.ab[2 * (kk - 1) + 1]);
  const double span = fmax(fabs(tmin), fabs(tmax));
  double* out = d.bounds + out_off;
  out[0] = tmin;
  out[1] = tmax;
  out[2] = tmax + beta + 1e-5 * span;
  out[4] = beta;
  double aest = tmax;
  if (use_count) {
    double cum = 0.0;
    for (int r = 0; r < kk; ++r) {
      float2 z0 = d.LZ32[d.lperm[r]];   // first row of the eigenvector matrix
      cum += ((double)z0.x * z0.x + (double)z0.y * z0.y) * (double)d.n;
      if (cum >= (double)d.m) { aest = d.lw32[r]; break; }
    }
  }
  out[3] = aest;
}

// start of a problem of the sequence: every problem iterates again
__global__ void b_step_reset(const BDesc* D, int np, double tol, int filter64) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const BDesc& d = D[p];
  for (int i = 0; i < 16; ++i) d.flags[i] = 0;
  d.flags[0] = 1;
  d.flags[5] = filter64;
  d.flags[13] = kBDegMax;
  d.bounds[8] = 1e300;
  d.bounds[17] = tol;
}

__global__ void b_post_bounds(const BDesc* D, int np) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const BDesc& d = D[p];
  if (!live(d)) return;
  double* b = d.bounds;
  b[7] = fmax(fabs(b[0]), fabs(b[2]));
  b[5] = fmax(fabs(b[12]), fabs(b[13]));
  b[6] = 0.1 * b[17] * b[7];
}

// ---------------------------------------------------------------- small eigensolver pieces
__global__ void b_g_to_c(const BDesc* D) {   // Hermitian part of G in FP32
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  const int m = d.m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int i = e / m, j = e % m;
    double2 a = d.G[i * m + j], b = d.G[j * m + i];
    d.G32[e] = make_float2((float)(0.5 * (a.x + b.x)), (float)(0.5 * (a.y - b.y)));
  }
}

__global__ void b_gather_z(const BDesc* D) {   // hZ[:, k] = Z32[:, perm[k]] in FP64
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  const int m = d.m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int i = e / m, k = e % m;
    float2 v = d.Z32[i * m + d.perm[k]];
    d.hZ[e] = make_double2(v.x, v.y);
  }
}

__global__ void b_frob(const BDesc* D) {   // hscal[1] = ||G||_F
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  __shared__ double red[32];
  const int m = d.m;
  double s = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) s += zabs2(d.G[e]);
  s = bsum_d(s, red);
  if (threadIdx.x == 0) d.hscal[1] = sqrt(s);
}

// Ogita-Aishima step: R = I - Z^H Z (hR), S = Z^H G Z (hS);
// lam_i = Re S_ii / (1 - Re R_ii), delta = 2 (||S - diag(lam)||_F + ||G||_F ||R||_F)
__global__ void b_oa_scalars(const BDesc* D) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  __shared__ double red[32];
  const int m = d.m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) d.hlam[i] = d.hS[i * m + i].x / (1.0 - d.hR[i * m + i].x);
  __syncthreads();
  double soff = 0.0, r2 = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e / m, j = e % m;
    double2 sv = d.hS[e];
    if (i == j) sv.x -= d.hlam[i];
    soff += zabs2(sv);
    r2 += zabs2(d.hR[e]);
  }
  soff = bsum_d(soff, red);
  r2 = bsum_d(r2, red);
  if (threadIdx.x == 0) d.hscal[0] = 2.0 * (sqrt(soff) + d.hscal[1] * sqrt(r2));
}

// correction E: R/2 on the diagonal and for pairs closer than delta (or all pairs in the
// orthonormality-only step), (S_ij + lam_j R_ij) / (lam_j - lam_i) elsewhere if <= 0.2
__global__ void b_oa_update(const BDesc* D, int only_orth) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  const int m = d.m;
  const double delta = only_orth ? 1e300 : d.hscal[0];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int i = e / m, j = e % m;
    double2 r = d.hR[e];
    double2 v = zscale(r, 0.5);
    double dl = d.hlam[j] - d.hlam[i];
    if (i != j && fabs(dl) > delta) {
      double2 sv = d.hS[e];
      double2 t = make_double2(sv.x + d.hlam[j] * r.x, sv.y + d.hlam[j] * r.y);
      if (sqrt(zabs2(t)) <= 0.2 * fabs(dl)) v = make_double2(t.x / dl, t.y / dl);
    }
    d.hE[e] = v;
  }
}

__global__ void b_hermitize_avg_S(const BDesc* D) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  const int m = d.m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int i = e / m, j = e % m;
    if (j < i) {
      double2 a = d.hS[i * m + j], b = d.hS[j * m + i];
      double2 v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      d.hS[i * m + j] = v;
      d.hS[j * m + i] = zconj(v);
    } else if (j == i) {
      d.hS[e].y = 0.0;
    }
  }
}

// theta ascending; Zs = Z with its columns in the same order (Z = hZ or hT)
__global__ void __launch_bounds__(1024) b_sort_pairs(const BDesc* D, int zsel) {
  const BDesc& d = D[blockIdx.x];
  if (!live(d)) return;
  __shared__ int rk[1024];
  const int m = d.m;
  const double2* Zin = zsel == 0 ? d.hZ : d.hT;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double li = d.hlam[i];
    int r = 0;
    for (int j = 0; j < m; ++j) r += (d.hlam[j] < li) || (d.hlam[j] == li && j < i);
    rk[i] = r;
    d.theta[r] = li;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e / m, k = e % m;
    d.Zs[i * m + rk[k]] = Zin[i * m + k];
  }
}

// ---------------------------------------------------------------- residual norms
constexpr int kNch = 64;   // row chunks of the two-stage column reductions

__global__ void b_resid_partial(const BDesc* D) {   // ||W_i - theta_i Q_i||^2 over a row chunk
  const BDesc& d = D[blockIdx.z];
  if (!live(d)) return;
  const int col = blockIdx.x * blockDim.x + threadIdx.x, ch = blockIdx.y;
  const int m = d.m;
  if (col >= m) return;
  const int64_t n = d.n, r0 = n * ch / kNch, r1 = n * (ch + 1) / kNch;
  const double th = d.theta[col];
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double2 w = d.W[r * m + col], q = d.Q[r * m + col];
    double dx = fma(-th, q.x, w.x), dy = fma(-th, q.y, w.y);
    s = fma(dx, dx, s);
    s = fma(dy, dy, s);
  }
  d.partial[(int64_t)ch * m + col] = s;
}

__global__ void b_resid_finish(const BDesc* D) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d)) return;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= d.m) return;
  double s = 0.0;
  for (int c = 0; c < kNch; ++c) s += d.partial[(int64_t)c * d.m + col];
  d.res[col] = sqrt(s);
}

// ---------------------------------------------------------------- final check (original space)
// On the first nev columns of Xf, AX (in Y1) and BX (in Y2), all with ld m:
// lam_i = Re(x^H A x) / Re(x^H B x), res_i = ||A x - lam_i B x|| / (||A||_2 ||x||).
__device__ __forceinline__ bool fin(const BDesc& d) { return d.flags[12] != 0; }

__global__ void b_final_pass0(const BDesc* D) {
  const BDesc& d = D[blockIdx.z];
  if (!fin(d)) return;
  const int col = blockIdx.x * blockDim.x + threadIdx.x, ch = blockIdx.y;
  if (col >= d.nev) return;
  const int m = d.m;
  const int64_t n = d.n, r0 = n * ch / kNch, r1 = n * (ch + 1) / kNch;
  double sa = 0.0, sb = 0.0, sx = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double2 x = d.Xf[r * m + col], a = d.Y1[r * m + col], b = d.Y2[r * m + col];
    sa += x.x * a.x + x.y * a.y;
    sb += x.x * b.x + x.y * b.y;
    sx += x.x * x.x + x.y * x.y;
  }
  const int64_t base = (int64_t)ch * 3 * d.nev;
  d.partial[base + col] = sa;
  d.partial[base + d.nev + col] = sb;
  d.partial[base + 2 * d.nev + col] = sx;
}

__global__ void b_final_finish0(const BDesc* D) {
  const BDesc& d = D[blockIdx.y];
  if (!fin(d)) return;
  const int col = blockIdx.x * blockDim.x + threadIdx.x, nev = d.nev;
  if (col >= nev) return;
  double sa = 0.0, sb = 0.0, sx = 0.0;
  for (int c = 0; c < kNch; ++c) {
    const int64_t base = (int64_t)c * 3 * nev;
    sa += d.partial[base + col];
    sb += d.partial[base + nev + col];
    sx += d.partial[base + 2 * nev + col];
  }
  d.lamf[col] = sa / sb;
  d.dscale[col] = sx;   // ||x||^2 (dscale is free here)
}

__global__ void b_final_pass1(const BDesc* D) {
  const BDesc& d = D[blockIdx.z];
  if (!fin(d)) return;
  const int col = blockIdx.x * blockDim.x + threadIdx.x, ch = blockIdx.y;
  if (col >= d.nev) return;
  const int m = d.m;
  const int64_t n = d.n, r0 = n * ch / kNch, r1 = n * (ch + 1) / kNch;
  const double l = d.lamf[col];
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double2 a = d.Y1[r * m + col], b = d.Y2[r * m + col];
    double dx = fma(-l, b.x, a.x), dy = fma(-l, b.y, a.y);
    s = fma(dx, dx, s);
    s = fma(dy, dy, s);
  }
  d.partial[(int64_t)ch * d.nev + col] = s;
}

__global__ void b_final_finish1(const BDesc* D) {
  const BDesc& d = D[blockIdx.y];
  if (!fin(d)) return;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= d.nev) return;
  double s = 0.0;
  for (int c = 0; c < kNch; ++c) s += d.partial[(int64_t)c * d.nev + col];
  d.resf[col] = sqrt(s) / (d.bounds[5] * sqrt(d.dscale[col]));
}

// after the final check: done, or re-open the problem with a 20x tighter standard-space
// tolerance and the FP64 filter (at most three final passes)
__global__ void b_final_status(const BDesc* D, int* out) {
  const int p = blockIdx.x;
  const BDesc& d = D[p];
  __shared__ double red[32];
  if (!fin(d)) {
    if (threadIdx.x == 0) out[p] = d.flags[3];
    return;
  }
  double mx = 0.0;
  for (int i = threadIdx.x; i < d.nev; i += blockDim.x) {
    double r = d.resf[i];
    mx = fmax(mx, r == r ? r : 1e300);
  }
  mx = bmax_d(mx, red);
  if (threadIdx.x == 0) {
    d.flags[12] = 0;
    d.flags[11] += 1;
    d.bounds[18] = mx;
    if (mx <= d.bounds[17]) {
      d.flags[3] = 2;
    } else if (d.flags[11] >= 3) {
      d.flags[3] = 3;
    } else {
      d.bounds[6] *= 0.05;
      if (!d.flags[5]) d.flags[10] += 1;
      d.flags[5] = 1;
      d.flags[3] = 0;
      d.flags[0] = 1;
      d.bounds[8] = 1e300;
    }
    out[p] = d.flags[3];
  }
}

// ---------------------------------------------------------------- per-round control
// Filter interval and degree from the current Ritz values (one CTA per problem):
//   lo = theta_{m-1}, hi = Lanczos upper bound, scaling point = min(theta_0, Lanczos min);
//   degree = smallest d with |T_d(t_i)| >= res_i / tol for every unconverged wanted
//   column (t_i = (theta_i - c) / e), clipped to [deg_min, cap]. Writes the three-term
//   coefficients, p_j(theta) for the residual-corrected filter, and the step masks.
__global__ void __launch_bounds__(256) b_cheb_coef(const BDesc* D, int deg_min, const int* deg_cap) {
  const BDesc& d = D[blockIdx.x];
  __shared__ double red[32];
  __shared__ double s_lo, s_hi, s_sc;
  __shared__ int s_deg;
  if (!live(d)) {
    if (threadIdx.x < kBDegMax) d.stepact[threadIdx.x] = 0;
    if (threadIdx.x == 0) { d.flags[6] = 0; d.flags[7] = 0; }
    return;
  }
  const int m = d.m, nev = d.nev;
  const int cap0 = max(deg_min, min(min(deg_cap[blockIdx.x], d.flags[13]), kBDegMax));
  if (threadIdx.x == 0) {
    double hi = d.bounds[2];
    double lo = d.theta[m - 1];
    double sc = fmin(d.theta[0], d.bounds[0]);
    if (!(lo > sc + 1e-3 * (hi - sc))) lo = sc + 0.5 * (hi - sc);
    if (!(hi > lo)) hi = lo + 1e-3 * d.bounds[7] + 1e-300;
    s_lo = lo;
    s_hi = hi;
    s_sc = sc;
    d.bounds[9] = lo;
    d.bounds[10] = hi;
    d.bounds[11] = sc;
  }
  __syncthreads();
  const double e = 0.5 * (s_hi - s_lo), c = 0.5 * (s_hi + s_lo), tolC = d.bounds[6];
  // highest degree whose dynamic range the filter carries: the guard columns near lo are
  // damped towards 1 / T_d(t_sc) relative to the column at the scaling point, and below
  // the filter's noise (FP32-class 1e-7, BF16 1e-3, FP64 1e-12) they degenerate
  int cap = cap0;
  {
    const double at = fabs((s_sc - c) / e);
    const double kappa = d.flags[5] ? 1e12 : (d.nsplit == 3 ? 1e7 : 1e3);
    if (at > 1.0) cap = max(deg_min, min(cap0, (int)floor(log(2.0 * kappa) / log(at + sqrt(at * at - 1.0)))));
  }
  double need = (double)deg_min;
  for (int i = threadIdx.x; i < nev; i += blockDim.x) {
    double r = d.res[i];
    if (!(r <= tolC)) {
      double at = fabs((d.theta[i] - c) / e);
      if (at <= 1.0 || !(r < 1e300)) need = fmax(need, (double)cap);
      else need = fmax(need, ceil(log(10.0 * r / tolC) / log(at + sqrt(at * at - 1.0))));   // 10x margin
    }
  }
  need = bmax_d(need, red);
  const int deg = (int)fmin(fmax(need, (double)deg_min), (double)cap);
  // largest residual Chebyshev theory predicts after this round (|T_deg(t_i)| gain for
  // every unconverged wanted pair outside the damped interval)
  double pred = 0.0;
  for (int i = threadIdx.x; i < nev; i += blockDim.x) {
    double r = d.res[i];
    const double at = fabs((d.theta[i] - c) / e);
    if (r > tolC && at > 1.0) r /= cosh(deg * acosh(fmin(at, 1e150)));
    pred = fmax(pred, r == r ? r : 1e300);
  }
  pred = bmax_d(pred, red);
  if (threadIdx.x == 0) {
    d.bounds[21] = pred;
    s_deg = deg;
    d.flags[1] = deg;
    d.flags[2] = 0;
    d.flags[9] += deg;
    const int f64 = d.flags[5] != 0;
    d.flags[6] = f64 ? 0 : 1;
    d.flags[7] = f64 ? 1 : 0;
    double sigma = e / (s_sc - c), sigma1 = sigma;
    for (int j = 0; j < deg; ++j) {
      double al, be, ga;
      if (j == 0) {
        al = sigma1 / e;
        be = -c * sigma1 / e;
        ga = 0.0;
      } else {
        double sn = 1.0 / (2.0 / sigma1 - sigma);
        al = 2.0 * sn / e;
        be = -al * c;
        ga = -sigma * sn;
        sigma = sn;
      }
      d.fco[3 * j] = al;
      d.fco[3 * j + 1] = be;
      d.fco[3 * j + 2] = ga;
    }
  }
  __syncthreads();
  if (threadIdx.x < kBDegMax) d.stepact[threadIdx.x] = (d.flags[7] && (int)threadIdx.x < deg) ? 1 : 0;
  if (d.pcoef) {
    // scalar recurrence at each Ritz value: pcoef[j][col] = alpha_j p_j(theta), pfinal = p_deg(theta)
    for (int col = threadIdx.x; col < d.ncols_pad; col += blockDim.x) {
      const double th = col < m ? d.theta[col] : 0.0;
      double pm1 = 0.0, p0 = 1.0;
      for (int j = 0; j < deg; ++j) {
        const double al = d.fco[3 * j], be = d.fco[3 * j + 1], ga = d.fco[3 * j + 2];
        d.pcoef[(size_t)j * d.ncols_pad + col] = col < m ? (float)(al * p0) : 0.f;
        double p1 = al * th * p0 + be * p0 + ga * pm1;
        pm1 = p0;
        p0 = p1;
      }
      d.pfinal[col] = col < m ? p0 : 0.0;
    }
  }
}

// FP64 filter: Y_k lives in slot k mod 3 of (Q, Y1, Y2); bring Y_deg to Y1
__global__ void b_fp64_select(const BDesc* D) {
  const BDesc& d = D[blockIdx.y];
  if (!live(d) || d.flags[7] == 0) return;
  const int slot = d.flags[1] % 3;
  if (slot == 1) return;
  const double2* s = slot == 0 ? d.Q : d.Y2;
  const int64_t total = (int64_t)d.n * d.m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    d.Y1[e] = s[e];
}

// after Rayleigh-Ritz: converged in the standard space -> final check; a low-precision
// filter that gained less than 4x in a round -> FP64 filter for this problem
__global__ void b_round_status(const BDesc* D, int* out) {
  const int p = blockIdx.x;
  const BDesc& d = D[p];
  __shared__ double red[32];
  if (!live(d)) {
    if (threadIdx.x == 0) out[p] = 0;
    return;
  }
  double mx = 0.0;
  for (int i = threadIdx.x; i < d.nev; i += blockDim.x) {
    double r = d.res[i];
    mx = fmax(mx, r == r ? r : 1e300);
  }
  mx = bmax_d(mx, red);
  if (threadIdx.x == 0) {
    const int info = d.flags[2];
    if (d.flags[4] == 0) d.bounds[19] = mx;   // largest residual at the start of the step
    // Chebyshev convergence factor of the nev-th Ritz value on the next round's interval
    {
      const int m = d.m;
      double hi = d.bounds[2], lo = d.theta[m - 1], sc = fmin(d.theta[0], d.bounds[0]);
      if (!(lo > sc + 1e-3 * (hi - sc))) lo = sc + 0.5 * (hi - sc);
      const double e = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
      const double t = fabs((d.theta[d.nev - 1] - c) / e);
      d.bounds[20] = (t > 1.0 && t < 1e300) ? t + sqrt(t * t - 1.0) : 1.0;
    }
    d.flags[4] += 1;
    d.bounds[18] = mx;
    if (info) d.flags[8] += 1;
    if (!info && mx <= d.bounds[6]) {
      d.flags[3] = 1;
      d.flags[0] = 0;
      d.flags[12] = 1;
    } else if (!info && !d.flags[5] && mx > 0.25 * d.bounds[8] && d.bounds[8] < 1e300 &&
               mx <= (d.nsplit == 3 ? 1e-3 : 1e-1) * d.bounds[7] &&   // below the cold-start zone
               mx > 25.0 * d.bounds[21]) {
      // the low-precision filter gained less than 4x where the Chebyshev factors of this
      // round promised more than 100x: it has reached its floor. The FP32-class floor
      // depends on the degree, so its cap is halved first (down to 16); BF16 -> FP64.
      if (d.nsplit == 3 && d.flags[13] > 16) {
        d.flags[13] = max(16, d.flags[13] / 2);
      } else {
        d.flags[5] = 1;
        d.flags[10] += 1;
      }
    }
    d.bounds[8] = mx;
    out[p] = d.flags[0] | (info ? 2 : 0);
  }
}

// round cap reached: the active problems go to the final check and are not re-opened
__global__ void b_force_final(const BDesc* D, int np) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const BDesc& d = D[p];
  if (d.flags[0] == 0) return;
  d.flags[0] = 0;
  d.flags[3] = 1;
  d.flags[12] = 1;
  d.flags[11] = max(d.flags[11], 2);
}

// complex normal block (counter-based splitmix64 + Box-Muller) in Y1 for masked problems
__global__ void b_randn(const BDesc* D, uint64_t seed, const int* mask) {
  const int p = blockIdx.y;
  const BDesc& d = D[p];
  if (mask ? mask[p] == 0 : !live(d)) return;
  const int64_t total = (int64_t)d.n * d.m;
  const uint64_t sd = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(p + 1));
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h1 = mix64(sd + 2 * (uint64_t)e), h2 = mix64(sd + 2 * (uint64_t)e + 1);
    double u1 = ((double)(h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
    double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    d.Y1[e] = make_double2(r * cs, r * sn);
  }
}

// outputs of one problem of the sequence: Lambda, residuals and (optionally) X
__global__ void b_write_out(const BDesc* D, const BOut* O) {
  const BDesc& d = D[blockIdx.y];
  const BOut& o = O[blockIdx.y];
  const int nev = d.nev, m = d.m;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < nev; i += blockDim.x) {
      o.lam[i] = d.lamf[i];
      o.res[i] = d.resf[i];
    }
  }
  if (!o.X) return;
  const int64_t total = (int64_t)d.n * nev;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / nev, c = e % nev;
    o.X[r * o.ldx + c] = d.Xf[r * m + c];
  }
}

}  // namespace

// --------------------------------------------------------------------------- launchers
namespace {
inline dim3 g2(int64_t per_problem, int nprob) {
  int64_t b = (per_problem + 255) / 256;
  b = std::max<int64_t>(1, std::min<int64_t>(b, 128));
  return dim3((unsigned)b, (unsigned)nprob);
}
}  // namespace

void bk_herm_sum(const BDesc* D, int np, int64_t nmax, cudaStream_t s) {
  b_herm_sum<<<g2(nmax * nmax, np), 256, 0, s>>>(D);
  LAUNCH_NOTE(1);
}
void bk_to_c32(const BDesc* D, int np, int64_t nmax, int which, cudaStream_t s) {
  b_to_c32<<<g2(nmax * nmax, np), 256, 0, s>>>(D, which);
  LAUNCH_NOTE(1);
}
void bk_hermitize_lower_G(const BDesc* D, int np, int mmax, cudaStream_t s) {
  b_hermitize_lower_G<<<g2((int64_t)mmax * mmax, np), 256, 0, s>>>(D);
  LAUNCH_NOTE(1);
}
void bk_gram_scale(const BDesc* D, int np, double shift_factor, cudaStream_t s) {
  b_gram_scale<<<np, 1024, 0, s>>>(D, shift_factor);
  LAUNCH_NOTE(1);
}
void bk_col_scale(const BDesc* D, int np, int64_t nm_max, int which, cudaStream_t s) {
  b_col_scale<<<g2(nm_max, np), 256, 0, s>>>(D, which);
  LAUNCH_NOTE(1);
}
void bk_copy_nm(const BDesc* D, int np, int64_t nm_max, int from, int to, cudaStream_t s) {
  b_copy_nm<<<g2(nm_max, np), 256, 0, s>>>(D, from, to);
  LAUNCH_NOTE(1);
}
void bk_potrf_small(const BDesc* D, int np, cudaStream_t s) {
  b_potrf_small<<<np, 1024, 0, s>>>(D);
  LAUNCH_NOTE(1);
}
void bk_trtri_small(const BDesc* D, int np, cudaStream_t s) {
  b_trtri_small<<<np, 1024, 0, s>>>(D);
  LAUNCH_NOTE(1);
}
void bk_step_reset(const BDesc* D, int np, double tol, int filter64, cudaStream_t s) {
  b_step_reset<<<(np + 63) / 64, 64, 0, s>>>(D, np, tol, filter64);
  LAUNCH_NOTE(1);
}
void bk_post_bounds(const BDesc* D, int np, cudaStream_t s) {
  b_post_bounds<<<(np + 63) / 64, 64, 0, s>>>(D, np);
  LAUNCH_NOTE(1);
}
void bk_lanczos(const BDesc* D, int np, int64_t nmax, int k, int use_count, int out_off, uint64_t seed,
                cudaStream_t s) {
  b_lanczos_init<<<np, 1024, 0, s>>>(D, seed);
  LAUNCH_NOTE(1);
  const int rows_per_block = 8;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nmax + rows_per_block - 1) / rows_per_block, 256));
  for (int j = 0; j < k; ++j) {
    b_matvec32<<<dim3(blocks, np), 32 * rows_per_block, 0, s>>>(D, j);
    b_lanczos_update<<<np, 1024, 0, s>>>(D, j);
    LAUNCH_NOTE(2);
  }
  b_build_T<<<np, 256, 0, s>>>(D, k);
  LAUNCH_NOTE(1);
  jacobi32_batched(D, np, 1, k, k, 30, s);
  b_lanczos_finish<<<np, 32, 0, s>>>(D, k, use_count, out_off);
  LAUNCH_NOTE(1);
}
void bk_heev_prep(const BDesc* D, int np, int mmax, cudaStream_t s) {
  b_g_to_c<<<g2((int64_t)mmax * mmax, np), 256, 0, s>>>(D);
  LAUNCH_NOTE(1);
  jacobi32_batched(D, np, 0, 0, mmax, 40, s);
  b_gather_z<<<g2((int64_t)mmax * mmax, np), 256, 0, s>>>(D);
  b_frob<<<np, 1024, 0, s>>>(D);
  LAUNCH_NOTE(2);
}
void bk_oa_scalars(const BDesc* D, int np, cudaStream_t s) {
  b_oa_scalars<<<np, 1024, 0, s>>>(D);
  LAUNCH_NOTE(1);
}
void bk_oa_update(const BDesc* D, int np, int mmax, int only_orth, cudaStream_t s) {
  b_oa_update<<<g2((int64_t)mmax * mmax, np), 256, 0, s>>>(D, only_orth);
  LAUNCH_NOTE(1);
}
void bk_hermitize_avg_S(const BDesc* D, int np, int mmax, cudaStream_t s) {
  b_hermitize_avg_S<<<g2((int64_t)mmax * mmax, np), 256, 0, s>>>(D);
  LAUNCH_NOTE(1);
}
void bk_sort_pairs(const BDesc* D, int np, int zsel, cudaStream_t s) {
  b_sort_pairs<<<np, 1024, 0, s>>>(D, zsel);
  LAUNCH_NOTE(1);
}
void bk_resid(const BDesc* D, int np, int mmax, cudaStream_t s) {
  b_resid_partial<<<dim3((mmax + 127) / 128, kNch, np), 128, 0, s>>>(D);
  b_resid_finish<<<dim3((mmax + 127) / 128, np), 128, 0, s>>>(D);
  LAUNCH_NOTE(2);
}
void bk_final_check(const BDesc* D, int np, int nevmax, cudaStream_t s) {
  dim3 g((nevmax + 127) / 128, kNch, np), f((nevmax + 127) / 128, np);
  b_final_pass0<<<g, 128, 0, s>>>(D);
  b_final_finish0<<<f, 128, 0, s>>>(D);
  b_final_pass1<<<g, 128, 0, s>>>(D);
  b_final_finish1<<<f, 128, 0, s>>>(D);
  LAUNCH_NOTE(4);
}
void bk_final_status(const BDesc* D, int np, int* out, cudaStream_t s) {
  b_final_status<<<np, 256, 0, s>>>(D, out);
  LAUNCH_NOTE(1);
}
void bk_cheb_coef(const BDesc* D, int np, int deg_min, const int* deg_cap, cudaStream_t s) {
  b_cheb_coef<<<np, 256, 0, s>>>(D, deg_min, deg_cap);
  LAUNCH_NOTE(1);
}
void bk_fp64_select(const BDesc* D, int np, int64_t nm_max, cudaStream_t s) {
  b_fp64_select<<<g2(nm_max, np), 256, 0, s>>>(D);
  LAUNCH_NOTE(1);
}
void bk_round_status(const BDesc* D, int np, int* out, cudaStream_t s) {
  b_round_status<<<np, 256, 0, s>>>(D, out);
  LAUNCH_NOTE(1);
}
void bk_force_final(const BDesc* D, int np, cudaStream_t s) {
  b_force_final<<<(np + 63) / 64, 64, 0, s>>>(D, np);
  LAUNCH_NOTE(1);
}
void bk_randn(const BDesc* D, int np, int64_t nm_max, uint64_t seed, const int* mask, cudaStream_t s) {
  b_randn<<<g2(nm_max, np), 256, 0, s>>>(D, seed, mask);
  LAUNCH_NOTE(1);
}
void bk_write_out(const BDesc* D, const BOut* O, int np, int64_t nm_max, cudaStream_t s) {
  b_write_out<<<g2(nm_max, np), 256, 0, s>>>(D, O);
  LAUNCH_NOTE(1);
}
size_t bk_partial_elems(int m) { return (size_t)kNch * 3 * std::max(m, 1); }

}  // namespace gevp
