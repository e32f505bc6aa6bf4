// Tall-skinny column reductions (residual norms, the final original-space check), the
// Gram-matrix scaling of CholQR, the band-energy backward and the peak probes.
//
// Column reductions over n x m row-major blocks: a CTA covers 128 consecutive columns
// (coalesced along the row) and a chunk of rows; chunk partials are summed in chunk
// order by a second kernel, so results are bitwise reproducible run to run.
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

constexpr int CT = 128;       // columns per CTA
constexpr int kChunks = 152;  // row chunks (one wave of CTAs per column block)

inline int nchunks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(kChunks, (n + 15) / 16)); }

__global__ void resid_partial_kernel(int64_t n, int m, const double2* W, int64_t ldw, const double2* Q, int64_t ldq,
                                     const double* theta, double* partial) {
  int col = blockIdx.x * CT + threadIdx.x;
  int ch = blockIdx.y, nch = gridDim.y;
  int64_t r0 = n * ch / nch, r1 = n * (ch + 1) / nch;
  if (col >= m) return;
  double th = theta[col];
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double2 w = W[r * ldw + col], q = Q[r * ldq + col];
    double dx = fma(-th, q.x, w.x), dy = fma(-th, q.y, w.y);
    s = fma(dx, dx, s);
    s = fma(dy, dy, s);
  }
  partial[(int64_t)ch * m + col] = s;
}

__global__ void col_finish_sqrt_kernel(int m, int nch, const double* partial, double* out) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= m) return;
  double s = 0.0;
  for (int c = 0; c < nch; ++c) s += partial[(int64_t)c * m + col];
  out[col] = sqrt(s);
}

// pass 0: partial[0] = Re x^H ax, partial[1] = Re x^H bx, partial[2] = ||x||^2
__global__ void final_pass0_kernel(int64_t n, int m, const double2* X, const double2* AX, const double2* BX,
                                   int64_t ld, double* partial) {
  int col = blockIdx.x * CT + threadIdx.x;
  int ch = blockIdx.y, nch = gridDim.y;
  int64_t r0 = n * ch / nch, r1 = n * (ch + 1) / nch;
  if (col >= m) return;
  double sa = 0.0, sb = 0.0, sx = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double2 x = X[r * ld + col], a = AX[r * ld + col], b = BX[r * ld + col];
    sa += x.x * a.x + x.y * a.y;
    sb += x.x * b.x + x.y * b.y;
    sx += x.x * x.x + x.y * x.y;
  }
  int64_t base = (int64_t)ch * 3 * m;
  partial[base + col] = sa;
  partial[base + m + col] = sb;
  partial[base + 2 * m + col] = sx;
}

// lam = (x^H A x)/(x^H B x); stash ||x||^2 and x^H B x in aux
__global__ void final_finish0_kernel(int m, int nch, const double* partial, double* lam, double* aux) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= m) return;
  double sa = 0.0, sb = 0.0, sx = 0.0;
  for (int c = 0; c < nch; ++c) {
    int64_t base = (int64_t)c * 3 * m;
    sa += partial[base + col];
    sb += partial[base + m + col];
    sx += partial[base + 2 * m + col];
  }
  lam[col] = sa / sb;
  aux[col] = sx;
  aux[m + col] = sb;
}

__global__ void final_pass1_kernel(int64_t n, int m, const double2* AX, const double2* BX, int64_t ld,
                                   const double* lam, double* partial) {
  int col = blockIdx.x * CT + threadIdx.x;
  int ch = blockIdx.y, nch = gridDim.y;
  int64_t r0 = n * ch / nch, r1 = n * (ch + 1) / nch;
  if (col >= m) return;
  double l = lam[col], s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double2 a = AX[r * ld + col], b = BX[r * ld + col];
    double dx = fma(-l, b.x, a.x), dy = fma(-l, b.y, a.y);
    s = fma(dx, dx, s);
    s = fma(dy, dy, s);
  }
  partial[(int64_t)ch * m + col] = s;
}

__global__ void final_finish1_kernel(int m, int nch, const double* partial, const double* aux, double normA,
                                     double* res) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= m) return;
  double s = 0.0;
  for (int c = 0; c < nch; ++c) s += partial[(int64_t)c * m + col];
  res[col] = sqrt(s) / (normA * sqrt(aux[col]));
}

__global__ void gram_dscale_kernel(int m, const double2* W, int64_t ldw, double* d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double v = W[(int64_t)i * ldw + i].x;
  d[i] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
}

__global__ void gram_apply_kernel(int m, double2* W, int64_t ldw, const double* d) {
  int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    W[(int64_t)i * ldw + j] = zscale(W[(int64_t)i * ldw + j], d[i] * d[j]);
  }
}

__global__ void scale_rows_by_lam_kernel(int64_t n, int nev, const double2* X, int64_t ldx, const double* lam,
                                         double2* XL) {
  int64_t total = n * nev;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / nev;
    int k = (int)(e % nev);
    XL[i * nev + k] = zscale(X[i * ldx + k], lam[k]);
  }
}

#define PROBE_ITERS 2048
__global__ void probe_fma64(double* out, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < PROBE_ITERS; i++) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void probe_fma32(float* out, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < PROBE_ITERS * 4; i++) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void probe_dmma(double* out) {
  double a = 1.0 + threadIdx.x * 1e-3, b = 0.5;
  double c[4][2];
  for (int j = 0; j < 4; j++) { c[j][0] = 0; c[j][1] = 0; }
  for (int i = 0; i < PROBE_ITERS / 4; i++) {
#pragma unroll
    for (int j = 0; j < 4; j++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[j][0]), "+d"(c[j][1]) : "d"(a), "d"(b));
  }
  double s = 0;
  for (int j = 0; j < 4; j++) s += c[j][0] + c[j][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

size_t resid_partial_elems(int64_t n, int m) { return (size_t)kChunks * 3 * std::max(m, 1) + 4 * (size_t)m + 64; }

void resid_norms(int64_t n, int m, const double2* W, int64_t ldw, const double2* Q, int64_t ldq, const double* theta,
                 double* res, double* partial, cudaStream_t s) {
  if (m <= 0) return;
  int nch = nchunks(n);
  dim3 g((m + CT - 1) / CT, nch);
  resid_partial_kernel<<<g, CT, 0, s>>>(n, m, W, ldw, Q, ldq, theta, partial);
  LAUNCH_NOTE(1);
  col_finish_sqrt_kernel<<<(m + 127) / 128, 128, 0, s>>>(m, nch, partial, res);
  LAUNCH_NOTE(1);
}

void final_check(int64_t n, int m, const double2* X, const double2* AX, const double2* BX, int64_t ld,
                 double* lam_io, double* res_out, double normA, double* partial, cudaStream_t s) {
  if (m <= 0) return;
  int nch = nchunks(n);
  dim3 g((m + CT - 1) / CT, nch);
  double* aux = partial + (size_t)kChunks * 3 * m;   // 2m doubles
  final_pass0_kernel<<<g, CT, 0, s>>>(n, m, X, AX, BX, ld, partial);
  LAUNCH_NOTE(1);
  final_finish0_kernel<<<(m + 127) / 128, 128, 0, s>>>(m, nch, partial, lam_io, aux);
  LAUNCH_NOTE(1);
  final_pass1_kernel<<<g, CT, 0, s>>>(n, m, AX, BX, ld, lam_io, partial);
  LAUNCH_NOTE(1);
  final_finish1_kernel<<<(m + 127) / 128, 128, 0, s>>>(m, nch, partial, aux, normA, res_out);
  LAUNCH_NOTE(1);
}

void gram_scale(int m, double2* W, int64_t ldw, double* dscale, cudaStream_t s) {
  gram_dscale_kernel<<<(m + 127) / 128, 128, 0, s>>>(m, W, ldw, dscale);
  LAUNCH_NOTE(1);
  int64_t total = (int64_t)m * m;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 4);
  gram_apply_kernel<<<blocks, 256, 0, s>>>(m, W, ldw, dscale);
  LAUNCH_NOTE(1);
}

void energy_backward_ws(int64_t n, int nev, const double2* X, int64_t ldx, const double* lam, const double* gE,
                        double2* GA, double2* GB, int64_t ldg, double2* XL, double2* split, size_t split_elems,
                        cudaStream_t s) {
  // GA = gE X X^H, GB = -gE (X diag(lam)) X^H ; lower tiles, then the Hermitian completion
  // applies the incoming gradient gE (a device scalar: no host synchronisation)
  ZgemmArgs a = zg((int)n, (int)n, nev, X, ldx, 0, X, ldx, 1, GA, ldg);
  a.triD = 1;
  zgemm(a, split, split_elems, s);
  hermitize_scale_lower(n, GA, ldg, gE, 1.0, s);
  int64_t total = n * nev;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  scale_rows_by_lam_kernel<<<blocks, 256, 0, s>>>(n, nev, X, ldx, lam, XL);
  LAUNCH_NOTE(1);
  ZgemmArgs b = zg((int)n, (int)n, nev, XL, nev, 0, X, ldx, 1, GB, ldg);
  b.triD = 1;
  zgemm(b, split, split_elems, s);
  hermitize_scale_lower(n, GB, ldg, gE, -1.0, s);
}

void probe_peaks(double* fp64_fma_tflops, double* fp64_dmma_tflops, double* fp32_fma_tflops, cudaStream_t s) {
  int blocks = 152 * 8, threads = 256;
  double* d = nullptr;
  cudaMalloc(&d, sizeof(double) * blocks * threads);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  probe_fma64<<<blocks, threads, 0, s>>>(d, 1.0000001, 1e-9);
  cudaEventRecord(e0, s);
  probe_fma64<<<blocks, threads, 0, s>>>(d, 1.0000001, 1e-9);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp64_fma_tflops = 2.0 * 8 * PROBE_ITERS * (double)blocks * threads / (ms * 1e-3) / 1e12;
  probe_dmma<<<blocks, threads, 0, s>>>(d);
  cudaEventRecord(e0, s);
  probe_dmma<<<blocks, threads, 0, s>>>(d);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp64_dmma_tflops = 512.0 * 4 * (PROBE_ITERS / 4) * ((double)blocks * threads / 32) / (ms * 1e-3) / 1e12;
  probe_fma32<<<blocks, threads, 0, s>>>((float*)d, 1.0000001f, 1e-9f);
  cudaEventRecord(e0, s);
  probe_fma32<<<blocks, threads, 0, s>>>((float*)d, 1.0000001f, 1e-9f);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp32_fma_tflops = 2.0 * 8 * PROBE_ITERS * 4 * (double)blocks * threads / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
}

}  // namespace gevp
