// Live timing of the product kernels, for measurement: while enabled, every launch of the
// FP64 complex GEMM, of the emulated product and of the tall-skinny Gram kernel is bracketed
// by a CUDA event pair recorded on its own stream, together with the launch's work (flop
// over the K ranges its tiles process). Reading waits for the events and sums per kernel class. Off by default; the
// cost when off is one branch per launch.
#include "gevp_internal.cuh"
#include "../../include/gevp.h"
#include <algorithm>
#include <mutex>
#include <vector>

namespace gevp {

constexpr int kKtClasses = 3;

namespace {

struct KtRec {
  int cls;
  cudaEvent_t e0, e1;
  double alg, exec;
};

struct KtState {
  std::mutex mu;
  bool on = false;
  std::vector<KtRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
};

KtState& kt() {
  static KtState st;
  return st;
}

}  // namespace

bool kt_enabled() { return kt().on; }

void* kt_begin(cudaStream_t s) {
  KtState& k = kt();
  // launches being captured into a graph are not timed
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  std::lock_guard<std::mutex> g(k.mu);
  cudaEvent_t e = k.get();
  if (e) cudaEventRecord(e, s);
  return e;
}

void kt_end(void* begin, int cls, double alg, double exec, cudaStream_t s) {
  KtState& k = kt();
  std::lock_guard<std::mutex> g(k.mu);
  if (!begin) return;
  cudaEvent_t e = k.get();
  if (!e) return;
  cudaEventRecord(e, s);
  k.recs.push_back({cls, (cudaEvent_t)begin, e, alg, exec});
}

// Work of a K-ranged tiled product at 64-block granularity: sum over 64 x 64 output blocks
// of rows x cols x (K range length), with the K range cut by the triangular structure
// (triA 1: k <= i, 2: k >= i; triB 1: k >= j, 2: k <= j) and, for triD, only blocks that
// meet the lower triangle.
double tiled_product_flops(int M, int N, int K, int triA, int triB, int triD) {
  const int b = 64;
  double f = 0.0;
  for (int i0 = 0; i0 < M; i0 += b) {
    const int i1 = std::min(M, i0 + b);
    for (int j0 = 0; j0 < N; j0 += b) {
      const int j1 = std::min(N, j0 + b);
      if (triD == 1 && j0 > i1 - 1) continue;
      int klo = 0, khi = K;
      if (triA == 1) khi = std::min(khi, i1);
      if (triA == 2) klo = std::max(klo, i0);
      if (triB == 1) klo = std::max(klo, j0);
      if (triB == 2) khi = std::min(khi, j1);
      if (khi > klo) f += 8.0 * (double)(i1 - i0) * (double)(j1 - j0) * (double)(khi - klo);
    }
  }
  return f;
}

}  // namespace gevp

extern "C" {

gevp_status gevp_kernel_timing(int enable) {
  gevp::KtState& k = gevp::kt();
  std::lock_guard<std::mutex> g(k.mu);
  if (enable) {
    k.recs.clear();
    k.used = 0;
  }
  k.on = enable != 0;
  return GEVP_OK;
}

gevp_status gevp_kernel_timing_read(double* out) {
  if (!out) return GEVP_ERR_INVALID_ARG;
  gevp::KtState& k = gevp::kt();
  std::lock_guard<std::mutex> g(k.mu);
  for (int i = 0; i < 4 * gevp::kKtClasses; ++i) out[i] = 0.0;
  for (const auto& r : k.recs) {
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return GEVP_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) return GEVP_ERR_CUDA;
    double* o = out + 4 * r.cls;
    o[0] += 1.0;
    o[1] += ms;
    o[2] += r.alg;
    o[3] += r.exec;
  }
  return GEVP_OK;
}

}  // extern "C"
