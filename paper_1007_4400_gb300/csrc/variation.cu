// Entry-variation statistics between consecutive Hamiltonians (the paper's Sec. "Matrix
// generation"): delta = max_ij |A_new - A_old|_ij and, per threshold fraction p, the
// number of entries whose variation exceeds p * delta (plus an optional byte mask).
//
// On this part an SM retires two FP64 FMAs per clock, so a pass that spends even a few
// FP64 operations per entry is bound by the FP64 pipe, not by HBM. The squared modulus
// d2 = dr*dr + di*di (each product and the sum rounded separately, as the definition
// fixes) costs five FP64 operations and is formed exactly once per entry: pass 1 stores
// its bit pattern and reduces the maximum as an integer (the IEEE ordering of
// non-negative doubles equals the unsigned ordering of their bit patterns); pass 2
// compares the stored bit patterns with the thresholds' as integers, with no FP64 work.
// Both passes walk rows with the threads on consecutive columns (coalesced, no 64-bit
// division per entry).
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

constexpr int kVarThreads = 256;
constexpr int kVarMaxThr = 16;

__device__ __forceinline__ unsigned long long var_d2_bits(double2 a, double2 b) {
  const double dr = __dsub_rn(a.x, b.x), di = __dsub_rn(a.y, b.y);
  return (unsigned long long)__double_as_longlong(__dadd_rn(__dmul_rn(dr, dr), __dmul_rn(di, di)));
}

// the bit pattern of every NaN is above that of +Inf
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

__global__ void __launch_bounds__(kVarThreads) var_max_kernel(int64_t n, const double2* A, int64_t lda,
                                                              const double2* B, int64_t ldb,
                                                              unsigned long long* d2, unsigned long long* ws) {
  __shared__ unsigned long long red[kVarThreads / 32];
  unsigned long long mx = 0;
  bool bad = false;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double2* a = A + i * lda;
    const double2* b = B + i * ldb;
    unsigned long long* o = d2 + i * n;
    for (int64_t j = threadIdx.x; j < n; j += kVarThreads) {
      const unsigned long long v = var_d2_bits(a[j], b[j]);
      o[j] = v;
      if (v > kInfBits) bad = true;
      else mx = v > mx ? v : mx;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, off);
    mx = t > mx ? t : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch((unsigned long long*)&ws[1], 1ull);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = red[0];
    for (int w = 1; w < kVarThreads / 32; ++w) m = red[w] > m ? red[w] : m;
    atomicMax(&ws[0], m);
  }
}

// NT: the smallest supported count of thresholds >= nthr (fewer counters, fewer registers)
template <int NT>
__global__ void __launch_bounds__(kVarThreads) var_count_kernel(int64_t n, const unsigned long long* d2,
                                                                const unsigned long long* ws_in, int nthr,
                                                                const double* p, unsigned long long* counts,
                                                                uint8_t* mask) {
  __shared__ unsigned long long thr[NT];
  __shared__ unsigned int red[kVarThreads / 32][NT];
  const double dmax2 = __longlong_as_double((long long)ws_in[0]);
  if (threadIdx.x < NT)
    thr[threadIdx.x] = threadIdx.x < nthr
                           ? (unsigned long long)__double_as_longlong(
                                 __dmul_rn(__dmul_rn(p[threadIdx.x], p[threadIdx.x]), dmax2))
                           : ~0ull;   // unused slots: nothing is above
  __syncthreads();
  unsigned long long tl[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) tl[t] = thr[t];
  unsigned int c[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) c[t] = 0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const unsigned long long* row = d2 + i * n;
    uint8_t* mrow = mask ? mask + i * n : nullptr;
    for (int j = threadIdx.x; j < n; j += kVarThreads) {
      const unsigned long long v = row[j];
#pragma unroll
      for (int t = 0; t < NT; ++t) c[t] += v > tl[t] ? 1u : 0u;
      if (mrow) mrow[j] = v > tl[0] ? 1 : 0;
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    unsigned int v = c[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < nthr) {
    unsigned long long sum = 0;
    for (int w = 0; w < kVarThreads / 32; ++w) sum += red[w][threadIdx.x];
    atomicAdd(&counts[threadIdx.x], sum);
  }
}

}  // namespace

int variation_max_thresholds() { return kVarMaxThr; }

// ws: >= 48 words ([0] max bits, [1] NaN flag, [2..17] counts, [32..47] thresholds = p_dev);
// d2: n * n words of scratch (the squared moduli).
void matrix_variation(int64_t n, const double2* A, int64_t lda, const double2* B, int64_t ldb, int nthr,
                      const double* p_dev, unsigned long long* ws, unsigned long long* d2, uint8_t* mask,
                      cudaStream_t s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rows_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(n, 8LL * sms));
  var_max_kernel<<<rows_blocks, kVarThreads, 0, s>>>(n, A, lda, B, ldb, d2, ws);
  unsigned long long* cnt = ws + 2;
  if (nthr <= 1) var_count_kernel<1><<<rows_blocks, kVarThreads, 0, s>>>(n, d2, ws, nthr, p_dev, cnt, mask);
  else if (nthr <= 4) var_count_kernel<4><<<rows_blocks, kVarThreads, 0, s>>>(n, d2, ws, nthr, p_dev, cnt, mask);
  else if (nthr <= 8) var_count_kernel<8><<<rows_blocks, kVarThreads, 0, s>>>(n, d2, ws, nthr, p_dev, cnt, mask);
  else var_count_kernel<16><<<rows_blocks, kVarThreads, 0, s>>>(n, d2, ws, nthr, p_dev, cnt, mask);
  LAUNCH_NOTE(2);
}

}  // namespace gevp
