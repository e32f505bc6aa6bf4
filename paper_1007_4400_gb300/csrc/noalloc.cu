// gevp_chebyshev_filter_noalloc: the FP64 Chebyshev filter for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the filter: code that
// runs while a CUDA graph is being captured (an allocation there is either illegal or
// becomes part of the graph), applications whose device memory is owned by a pool
// allocator such as PyTorch's caching allocator and must not be fragmented or raced by a
// library's own cudaMalloc/cudaFree (which also synchronise the device), and real-time or
// memory-budgeted services that reserve a fixed footprint at start-up. The regular
// gevp_chebyshev_filter needs a handle whose workspace grows with cudaMalloc; this entry
// point needs no handle and allocates nothing: its scratch (two n x m ping-pong blocks) is
// a fixed array in the library's device image.
#include "gevp_internal.cuh"
#include "../../include/gevp.h"

#include <mutex>

namespace {

// 2^21 complex128 = 32 MiB, shared by every call on a device. Every GPU that loads the
// library holds this array until the process exits.
constexpr size_t kScratchElems = (size_t)GEVP_NOALLOC_MAX_ELEMS;
static __device__ __align__(256) double2 g_filter_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once per device).
// The array's name in host code is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with the device current.
cudaError_t scratch_for_current_device(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_filter_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double2*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" gevp_status gevp_chebyshev_filter_noalloc(void* stream, int64_t n, const void* C, int64_t ldc, void* Y,
                                                     int64_t ldy, int m, int degree, double lo, double hi,
                                                     double s) {
  if (n < 0 || m < 0 || degree < 1 || !(hi > lo) || !(lo > s)) return GEVP_ERR_INVALID_ARG;
  if (n == 0 || m == 0) return GEVP_OK;
  if (!C || !Y || ldc < n || ldy < m) return GEVP_ERR_INVALID_ARG;
  if ((uint64_t)2 * (uint64_t)n * (uint64_t)m > (uint64_t)kScratchElems) return GEVP_ERR_INVALID_ARG;
  double2* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return GEVP_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  using namespace gevp;
  const double2* Cm = (const double2*)C;
  double2* B1 = scratch;
  double2* B2 = scratch + (size_t)n * m;
  const int64_t ldb = m;
  // scaled three-term recurrence (Zhou, Saad, Tiago & Chelikowsky 2006), each step one
  // FP64 complex GEMM with the recurrence fused into its epilogue; no split-K scratch
  double e = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
  double sigma = e / (s - c), sigma1 = sigma;
  ZgemmArgs a = zg((int)n, m, (int)n, Cm, ldc, 0, (const double2*)Y, ldy, 0, B1, ldb, sigma1 / e);
  a.Cin = (const double2*)Y; a.ldc = ldy; a.beta = -c * sigma1 / e;
  zgemm(a, nullptr, 0, st);
  const double2* prev = (const double2*)Y;
  int64_t ldp = ldy;
  double2* cur = B1;
  double2* nxt = B2;
  for (int i = 2; i <= degree; ++i) {
    double sn = 1.0 / (2.0 / sigma1 - sigma);
    double al = 2.0 * sn / e;
    ZgemmArgs g = zg((int)n, m, (int)n, Cm, ldc, 0, cur, ldb, 0, nxt, ldb, al);
    g.Cin = cur; g.ldc = ldb; g.beta = -al * c;
    g.Ein = prev; g.lde = ldp; g.gamma = -sigma * sn;
    zgemm(g, nullptr, 0, st);
    sigma = sn;
    double2* old = cur;
    prev = old;
    ldp = ldb;
    cur = nxt;
    nxt = old;
  }
  zcopy2d(n, m, cur, ldb, (double2*)Y, ldy, st);
  return cudaGetLastError() == cudaSuccess ? GEVP_OK : GEVP_ERR_CUDA;
}
