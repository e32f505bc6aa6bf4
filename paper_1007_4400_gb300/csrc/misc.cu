// Elementwise and data-movement kernels (HBM-bound, grid-stride, coalesced along rows).
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t total) {
  int64_t b = (total + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// In place: C <- M + M^H for a square M stored in C (each pair (i, j), j < i, is read
// and written by one thread).
__global__ void herm_sum_inplace_kernel(int64_t n, double2* C, int64_t ldc) {
  int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (j < i) {
      double2 a = C[i * ldc + j], b = C[j * ldc + i];
      double2 v = make_double2(a.x + b.x, a.y - b.y);
      C[i * ldc + j] = v;
      C[j * ldc + i] = zconj(v);
    } else if (j == i) {
      C[i * ldc + i] = make_double2(2.0 * C[i * ldc + i].x, 0.0);
    }
  }
}

__global__ void zshift_diag_kernel(int64_t n, double2* A, int64_t lda, double sh) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    A[i * lda + i].x += sh;
}

__global__ void zero_lower_kernel(int64_t n, double2* A, int64_t lda) {
  int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (j < i) A[i * lda + j] = make_double2(0.0, 0.0);
  }
}

__global__ void hermitize_lower_kernel(int64_t n, double2* C, int64_t ldc) {
  int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (j > i) C[i * ldc + j] = zconj(C[j * ldc + i]);
    else if (j == i) C[i * ldc + i].y = 0.0;
  }
}

// lower triangle scaled by sign * (*scale) (a device scalar), upper <- conj(lower), real diagonal
__global__ void hermitize_scale_lower_kernel(int64_t n, double2* C, int64_t ldc, const double* scale, double sign) {
  const double f = sign * scale[0];
  int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (j > i) continue;
    double2 v = zscale(C[i * ldc + j], f);
    if (j == i) {
      C[i * ldc + i] = make_double2(v.x, 0.0);
    } else {
      C[i * ldc + j] = v;
      C[j * ldc + i] = zconj(v);
    }
  }
}

// E[p] = sum_i lam[p * nev + i], summed in index order (one thread per problem)
__global__ void band_energy_kernel(int nprob, int nev, const double* lam, double* E) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  double s = 0.0;
  for (int i = 0; i < nev; ++i) s += lam[(int64_t)p * nev + i];
  E[p] = s;
}

// C <- C + D on the lower triangle (diagonal real), mirrored to the upper one; each thread
// reads only lower entries, so the mirror writes never race with a read
__global__ void add_lower_herm_kernel(int64_t n, double2* C, int64_t ldc, const double2* D, int64_t ldd) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (j > i) continue;
    double2 v = zadd(C[i * ldc + j], D[i * ldd + j]);
    if (j == i) {
      C[i * ldc + i] = make_double2(v.x, 0.0);
    } else {
      C[i * ldc + j] = v;
      C[j * ldc + i] = zconj(v);
    }
  }
}

// Out[i][t] = X[i][idx[t]] (rows x k gather of columns)
__global__ void gather_cols_kernel(int64_t rows, int k, const double2* X, int64_t ldx, const int64_t* idx,
                                   double2* Out, int64_t ldo) {
  const int64_t total = rows * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const int t = (int)(e % k);
    Out[i * ldo + t] = X[i * ldx + idx[t]];
  }
}

// Out[t][j] = X[idx[t]][j] (k x cols gather of rows)
__global__ void gather_rows_kernel(int k, int64_t cols, const double2* X, int64_t ldx, const int64_t* idx,
                                   double2* Out, int64_t ldo) {
  const int64_t total = (int64_t)k * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / cols);
    const int64_t j = e % cols;
    Out[(int64_t)t * ldo + j] = X[idx[t] * ldx + j];
  }
}

__global__ void hermitize_avg_kernel(int64_t n, double2* C, int64_t ldc) {
  int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (j < i) {
      double2 a = C[i * ldc + j], b = C[j * ldc + i];
      double2 v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      C[i * ldc + j] = v;
      C[j * ldc + i] = zconj(v);
    } else if (j == i) {
      C[i * ldc + i].y = 0.0;
    }
  }
}

// A <- A - P on the lower triangle (j <= i) of an n x n block
__global__ void zsub_lower_kernel(int64_t n, double2* A, int64_t lda, const double2* P, int64_t ldp) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (j <= i) {
      const double2 a = A[i * lda + j], p = P[i * ldp + j];
      A[i * lda + j] = make_double2(a.x - p.x, a.y - p.y);
    }
  }
}

__global__ void zneg_kernel(int64_t rows, int64_t cols, double2* X, int64_t ldx) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    const double2 v = X[i * ldx + j];
    X[i * ldx + j] = make_double2(-v.x, -v.y);
  }
}

// out[0] = max_ij |G_ij - delta_ij| over an m x m block (one CTA; fixed reduction order)
__global__ void __launch_bounds__(1024) eye_dev_kernel(int m, const double2* G, int64_t ldg, double* out) {
  __shared__ double red[32];
  double mx = 0.0;
  const int64_t mm = (int64_t)m * m;
  for (int64_t e = threadIdx.x; e < mm; e += blockDim.x) {
    const int64_t i = e / m, j = e % m;
    double2 v = G[i * ldg + j];
    if (i == j) v.x -= 1.0;
    mx = fmax(mx, sqrt(v.x * v.x + v.y * v.y));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    out[0] = t;
  }
}

__global__ void zero_upper_kernel(int64_t n, double2* L, int64_t ldl) {
  int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (j > i) L[i * ldl + j] = make_double2(0.0, 0.0);
  }
}

__global__ void zcopy2d_kernel(int64_t rows, int64_t cols, const double2* s, int64_t lds, double2* d, int64_t ldd) {
  int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols, j = e % cols;
    d[i * ldd + j] = s[i * lds + j];
  }
}

__global__ void zset_identity_kernel(int64_t rows, int64_t cols, double2* A, int64_t lda) {
  int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols, j = e % cols;
    A[i * lda + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

__global__ void z_to_c_kernel(int64_t rows, int64_t cols, const double2* s, int64_t lds, float2* d, int64_t ldd) {
  int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols, j = e % cols;
    double2 v = s[i * lds + j];
    d[i * ldd + j] = make_float2((float)v.x, (float)v.y);
  }
}

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): a counter-based 64-bit mixer.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void zrandn_kernel(int64_t rows, int64_t cols, double2* A, int64_t lda, uint64_t seed) {
  int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols, j = e % cols;
    uint64_t h1 = splitmix64(seed ^ splitmix64(2 * (uint64_t)e));
    uint64_t h2 = splitmix64(seed ^ splitmix64(2 * (uint64_t)e + 1));
    double u1 = ((double)(h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = ((double)(h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double r = sqrt(-log(u1));            // Box-Muller with E|z|^2 = 1
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    A[i * lda + j] = make_double2(r * c, r * s);
  }
}

__global__ void zcol_scale_kernel(int64_t rows, int64_t cols, double2* A, int64_t lda, const double* sc) {
  int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols, j = e % cols;
    A[i * lda + j] = zscale(A[i * lda + j], sc[j]);
  }
}

__global__ void check_finite_kernel(int64_t rows, int64_t cols, const double2* A, int64_t lda, int* flag) {
  int64_t total = rows * cols;
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols, j = e % cols;
    double2 v = A[i * lda + j];
    if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

}  // namespace

void herm_sum_inplace(int64_t n, double2* C, int64_t ldc, cudaStream_t s) {
  herm_sum_inplace_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, C, ldc);
  LAUNCH_NOTE(1);
}
void zshift_diag(int64_t n, double2* A, int64_t lda, double sh, cudaStream_t s) {
  zshift_diag_kernel<<<grid_for(n), kThreads, 0, s>>>(n, A, lda, sh);
  LAUNCH_NOTE(1);
}
void zero_lower(int64_t n, double2* A, int64_t lda, cudaStream_t s) {
  zero_lower_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, A, lda);
  LAUNCH_NOTE(1);
}
void hermitize_lower(int64_t n, double2* C, int64_t ldc, cudaStream_t s) {
  hermitize_lower_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, C, ldc);
  LAUNCH_NOTE(1);
}
void hermitize_scale_lower(int64_t n, double2* C, int64_t ldc, const double* scale, double sign, cudaStream_t s) {
  hermitize_scale_lower_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, C, ldc, scale, sign);
  LAUNCH_NOTE(1);
}
void add_lower_herm(int64_t n, double2* C, int64_t ldc, const double2* D, int64_t ldd, cudaStream_t s) {
  if (n <= 0) return;
  add_lower_herm_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, C, ldc, D, ldd);
  LAUNCH_NOTE(1);
}
void gather_cols(int64_t rows, int k, const double2* X, int64_t ldx, const int64_t* idx, double2* Out, int64_t ldo,
                 cudaStream_t s) {
  if (rows <= 0 || k <= 0) return;
  gather_cols_kernel<<<grid_for(rows * k), kThreads, 0, s>>>(rows, k, X, ldx, idx, Out, ldo);
  LAUNCH_NOTE(1);
}
void gather_rows(int k, int64_t cols, const double2* X, int64_t ldx, const int64_t* idx, double2* Out, int64_t ldo,
                 cudaStream_t s) {
  if (cols <= 0 || k <= 0) return;
  gather_rows_kernel<<<grid_for((int64_t)k * cols), kThreads, 0, s>>>(k, cols, X, ldx, idx, Out, ldo);
  LAUNCH_NOTE(1);
}
void band_energy(int nprob, int nev, const double* lam, double* E, cudaStream_t s) {
  band_energy_kernel<<<(nprob + 127) / 128, 128, 0, s>>>(nprob, nev, lam, E);
  LAUNCH_NOTE(1);
}
void hermitize_avg(int64_t n, double2* C, int64_t ldc, cudaStream_t s) {
  hermitize_avg_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, C, ldc);
  LAUNCH_NOTE(1);
}
void zsub_lower(int64_t n, double2* A, int64_t lda, const double2* P, int64_t ldp, cudaStream_t s) {
  if (n <= 0) return;
  zsub_lower_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, A, lda, P, ldp);
  LAUNCH_NOTE(1);
}
void zneg(int64_t rows, int64_t cols, double2* X, int64_t ldx, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  zneg_kernel<<<grid_for(rows * cols), kThreads, 0, s>>>(rows, cols, X, ldx);
  LAUNCH_NOTE(1);
}
void eye_deviation(int m, const double2* G, int64_t ldg, double* out_dev, cudaStream_t s) {
  if (m <= 0) return;
  eye_dev_kernel<<<1, 1024, 0, s>>>(m, G, ldg, out_dev);
  LAUNCH_NOTE(1);
}
void zero_upper(int64_t n, double2* L, int64_t ldl, cudaStream_t s) {
  zero_upper_kernel<<<grid_for(n * n), kThreads, 0, s>>>(n, L, ldl);
  LAUNCH_NOTE(1);
}
void zcopy2d(int64_t rows, int64_t cols, const double2* src, int64_t lds, double2* dst, int64_t ldd, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  zcopy2d_kernel<<<grid_for(rows * cols), kThreads, 0, s>>>(rows, cols, src, lds, dst, ldd);
  LAUNCH_NOTE(1);
}
void zset_identity(int64_t rows, int64_t cols, double2* A, int64_t lda, cudaStream_t s) {
  zset_identity_kernel<<<grid_for(rows * cols), kThreads, 0, s>>>(rows, cols, A, lda);
  LAUNCH_NOTE(1);
}
void z_to_c(int64_t rows, int64_t cols, const double2* src, int64_t lds, float2* dst, int64_t ldd, cudaStream_t s) {
  z_to_c_kernel<<<grid_for(rows * cols), kThreads, 0, s>>>(rows, cols, src, lds, dst, ldd);
  LAUNCH_NOTE(1);
}
void zrandn(int64_t rows, int64_t cols, double2* A, int64_t lda, uint64_t seed, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  zrandn_kernel<<<grid_for(rows * cols), kThreads, 0, s>>>(rows, cols, A, lda, seed);
  LAUNCH_NOTE(1);
}
void zcol_scale(int64_t rows, int64_t cols, double2* A, int64_t lda, const double* scale, cudaStream_t s) {
  zcol_scale_kernel<<<grid_for(rows * cols), kThreads, 0, s>>>(rows, cols, A, lda, scale);
  LAUNCH_NOTE(1);
}
int check_finite(int64_t rows, int64_t cols, const double2* A, int64_t lda, int* dflag, cudaStream_t s) {
  check_finite_kernel<<<grid_for(rows * cols), kThreads, 0, s>>>(rows, cols, A, lda, dflag);
  LAUNCH_NOTE(1);
  return 0;
}

}  // namespace gevp
