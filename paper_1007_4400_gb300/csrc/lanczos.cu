// k-step Lanczos with full re-orthogonalisation on an FP32 copy of a Hermitian matrix, for
// the Chebyshev filter's interval: an upper bound of the spectrum (largest Ritz value plus
// the last residual norm |beta_k|, as in Zhou, Saad, Tiago & Chelikowsky 2006) and an
// estimate of the count-th eigenvalue from the Ritz values weighted by the squared first
// components of the tridiagonal's eigenvectors (a Lanczos quadrature of the spectral
// density). Bounds need a few digits only, so FP32 suffices; the matrix-vector product is
// HBM/L2 bound (one warp per row, coalesced row reads).
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

constexpr int KMAX = 64;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void matvec32_kernel(int64_t n, const float2* M, int64_t ldm, const float2* v, float2* w) {
  int64_t row = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x % 32;
  if (row >= n) return;
  const float2* r = M + row * ldm;
  float2 acc = make_float2(0.f, 0.f);
  for (int64_t j = lane; j < n; j += 32) cfma(acc, r[j], v[j]);
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) w[row] = acc;
}

__device__ float2 warp_sum2(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// V: (k+1) vectors of length n, vector-major. ab[2j] = alpha_j, ab[2j+1] = beta_j.
// ab[2*KMAX] (as int) = effective number of steps.
__global__ void __launch_bounds__(1024) lanczos_init_kernel(int64_t n, float2* V, uint64_t seed, float* ab) {
  __shared__ float red[32];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    uint64_t h1 = mix64(seed ^ mix64(2 * (uint64_t)i)), h2 = mix64(seed ^ mix64(2 * (uint64_t)i + 1));
    float u1 = ((float)(h1 >> 40) + 0.5f) * (1.0f / 16777216.0f);
    float u2 = ((float)(h2 >> 40) + 0.5f) * (1.0f / 16777216.0f);
    float2 z = make_float2(u1 - 0.5f, u2 - 0.5f);
    V[i] = z;
    s += z.x * z.x + z.y * z.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
    red[0] = rsqrtf(t);
    ((int*)ab)[2 * KMAX] = 0;
  }
  __syncthreads();
  float inv = red[0];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) { float2 z = V[i]; V[i] = make_float2(z.x * inv, z.y * inv); }
}

__global__ void __launch_bounds__(1024) lanczos_update_kernel(int64_t n, int j, float2* V, float2* w, float* ab) {
  __shared__ float2 red[32][KMAX + 1];
  __shared__ float2 h[KMAX + 1];
  __shared__ float nrm;
  const int lane = threadIdx.x % 32, wp = threadIdx.x / 32, nw = blockDim.x / 32;
  int* keff = (int*)(ab + 2 * KMAX);
  if (*keff < j) return;   // broke down earlier
  for (int pass = 0; pass < 2; ++pass) {
    for (int c = 0; c <= j; ++c) {
      const float2* vc = V + (int64_t)c * n;
      float2 p = make_float2(0.f, 0.f);
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        float2 a = vc[i], b = w[i];
        p.x += a.x * b.x + a.y * b.y;   // conj(a) * b
        p.y += a.x * b.y - a.y * b.x;
      }
      p = warp_sum2(p);
      if (lane == 0) red[wp][c] = p;
    }
    __syncthreads();
    for (int c = threadIdx.x; c <= j; c += blockDim.x) {
      float2 t = make_float2(0.f, 0.f);
      for (int q = 0; q < nw; ++q) { t.x += red[q][c].x; t.y += red[q][c].y; }
      h[c] = t;
      if (pass == 0 && c == j) ab[2 * j] = t.x;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      float2 b = w[i];
      for (int c = 0; c <= j; ++c) {
        float2 a = V[(int64_t)c * n + i], hc = h[c];
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
    ab[2 * j + 1] = nrm;
    float scale = fabsf(ab[2 * j]) + (j > 0 ? ab[2 * j - 1] : 0.f);
    if (nrm > 1e-6f * scale && nrm > 0.f) *keff = j + 1; else *keff = -(j + 1);  // negative: stop after j
  }
  __syncthreads();
  if (*keff < 0) return;
  float inv = 1.f / nrm;
  float2* vn = V + (int64_t)(j + 1) * n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) { float2 b = w[i]; vn[i] = make_float2(b.x * inv, b.y * inv); }
}

// T (k x k, stride k): the tridiagonal of the first kk steps, padded with a diagonal far
// above the spectrum for indices >= kk (kk < k only after a breakdown).
__global__ void build_T_kernel(int k, const float* ab, float2* T, int* kout, float big) {
  const int* keff = (const int*)(ab + 2 * KMAX);
  int ke = *keff;
  int kk = ke < 0 ? -ke : (ke > k ? k : ke);
  if (kk < 1) kk = 1;
  if (threadIdx.x == 0) *kout = kk;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    float v = 0.f;
    if (i >= kk || j >= kk) v = (i == j) ? big : 0.f;
    else if (i == j) v = ab[2 * i];
    else if (j == i + 1) v = ab[2 * i + 1];
    else if (i == j + 1) v = ab[2 * j + 1];
    T[e] = make_float2(v, 0.f);
  }
}

__global__ void lanczos_finish_kernel(int k, int64_t n, int count, const float* ab, const int* kout, const float* w,
                                      const int* perm, const float2* Z, double* out) {
  if (threadIdx.x != 0) return;
  int kk = *kout;
  double tmin = w[0], tmax = w[kk - 1];
  int ke = ((const int*)(ab + 2 * KMAX))[0];
  double beta = (ke < 0) ? 0.0 : fabs((double)ab[2 * (kk - 1) + 1]);
  double span = fmax(fabs(tmin), fabs(tmax));
  out[0] = tmin;
  out[1] = tmax;
  out[2] = tmax + beta + 1e-5 * span;
  out[4] = beta;
  double aest = tmax;
  if (count > 0) {
    double cum = 0.0;
    for (int r = 0; r < kk; ++r) {
      float2 z0 = Z[0 * k + perm[r]];
      cum += (double)(z0.x * z0.x + z0.y * z0.y) * (double)n;
      if (cum >= (double)count) { aest = w[r]; break; }
    }
  }
  out[3] = aest;
}

}  // namespace

size_t lanczos_ws_bytes(int64_t n, int k) {
  size_t b = 0;
  b += (size_t)(KMAX + 1) * n * sizeof(float2);   // V
  b += (2 * KMAX + 4) * sizeof(float);           // ab
  b += n * sizeof(float2);                        // w
  b += 2 * (size_t)KMAX * KMAX * sizeof(float2);  // T32, Z32
  b += KMAX * sizeof(float) + KMAX * sizeof(int) + 8 * sizeof(double) + 16 * 256;
  return b;
}

void lanczos_bounds(int64_t n, const float2* M32, int64_t ldm, int k, int count, uint64_t seed,
                    const LanczosWork& w, double* dev_out, cudaStream_t s) {
  k = std::max(1, std::min<int>(k, (int)std::min<int64_t>(n, KMAX)));
  lanczos_init_kernel<<<1, 1024, 0, s>>>(n, w.V, seed, w.ab);
  LAUNCH_NOTE(1);
  int rows_per_block = 8;
  int blocks = (int)((n + rows_per_block - 1) / rows_per_block);
  for (int j = 0; j < k; ++j) {
    matvec32_kernel<<<blocks, 32 * rows_per_block, 0, s>>>(n, M32, ldm, w.V + (int64_t)j * n, w.w);
    LAUNCH_NOTE(1);
    lanczos_update_kernel<<<1, 1024, 0, s>>>(n, j, w.V, w.w, w.ab);
    LAUNCH_NOTE(1);
  }
  int* kout = (int*)(w.ab + 2 * KMAX) + 1;
  build_T_kernel<<<1, 256, 0, s>>>(k, w.ab, w.T32, kout, 1e30f);
  LAUNCH_NOTE(1);
  jacobi32(k, w.T32, w.Z32, w.w32, w.perm, 30, s);
  lanczos_finish_kernel<<<1, 32, 0, s>>>(k, n, count, w.ab, kout, w.w32, w.perm, w.Z32, dev_out);
  LAUNCH_NOTE(1);
}

}  // namespace gevp
