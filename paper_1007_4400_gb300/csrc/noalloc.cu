// gevp_chebyshev_filter_noalloc: the FP64 Chebyshev filter for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the filter:
// applications whose device memory is owned by a pool allocator such as PyTorch's caching
// allocator (a library's own cudaMalloc/cudaFree bypasses the pool, can fail when the pool
// holds the free memory, and synchronises the device), and real-time or memory-budgeted
// services that reserve a fixed footprint at start-up and may not grow it afterwards. The
// regular gevp_chebyshev_filter needs a handle whose workspace grows with cudaMalloc; this
// entry point needs no handle and allocates nothing: its scratch (two n x m ping-pong
// blocks) is a fixed array in the library's device image.
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
// from cudaGetSymbolAddress with the device current. The address is cached for the life of
// the process: after a cudaDeviceReset the device image is reloaded and the cached address
// is stale, so the entry point must not be used across a reset.
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
  // an error left pending by earlier, unrelated work on this thread stays with its owner:
  // report it without clearing it and enqueue nothing
  if (cudaPeekAtLastError() != cudaSuccess) return GEVP_ERR_CUDA;
  double2* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return GEVP_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // the handle path's recurrence (scaled three-term, one FP64 complex GEMM per step with the
  // recurrence in its epilogue), here without split-K scratch
  double2* out = gevp::cheb_filter_fp64(n, (const double2*)C, ldc, (const double2*)Y, ldy, m, degree, lo, hi, s,
                                        scratch, scratch + (size_t)n * m, m, nullptr, 0, st);
  if (cudaGetLastError() != cudaSuccess) return GEVP_ERR_CUDA;
  gevp::zcopy2d(n, m, out, m, (double2*)Y, ldy, st);
  return cudaGetLastError() == cudaSuccess ? GEVP_OK : GEVP_ERR_CUDA;
}
