// libgevp host driver: handle and workspace, the reduction to standard form, the
// Chebyshev-filtered subspace iteration with locking, the sequence driver with warm
// starts, and the C ABI declared in include/gevp.h.
//
// Per problem (the paper's P_i, Sec. "A new computational philosophy"):
//   1. B = L L^H and L^-1 (once while B is unchanged);
//   2. C = L^-1 A L^-H as T = L^-1 tril_half(A), M = T L^-H, C = M + M^H (4 n^3 flops:
//      both products skip the zero triangles);
//   3. spectral bounds by FP32 Lanczos on C (and an estimate of ||A||_2 for residuals);
//   4. start block: the previous problem's block (warm) or a random one (cold);
//   5. rounds of: Chebyshev filter on the active columns -> orthogonalise against the
//      locked columns + CholQR2 -> Rayleigh-Ritz -> residuals -> lock the leading
//      converged pairs, until nev pairs are locked;
//   6. X = L^-H Q, Rayleigh quotients and residuals on the original pencil (A, B).
#include "gevp_internal.cuh"
#include "../../include/gevp.h"

#include <algorithm>
#include <initializer_list>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace gevp;

namespace gevp {
std::atomic<int64_t> g_launches{0};
}

struct gevp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  // arena
  char* arena = nullptr;
  size_t arena_bytes = 0;
  int64_t cap_n = 0;
  int cap_m = 0;
  // n x n
  double2 *L = nullptr, *Linv = nullptr, *C = nullptr, *T = nullptr;
  float2* M32 = nullptr;
  // n x m (ld = cap_m)
  double2 *Q = nullptr, *Y1 = nullptr, *Y2 = nullptr, *W = nullptr, *Wt = nullptr, *Xf = nullptr;
  // m x m
  double2 *G = nullptr, *Zs = nullptr, *Gw = nullptr, *Gwi = nullptr, *P = nullptr;
  double2* split = nullptr;
  size_t split_elems = 0;
  double2* trtri_ws = nullptr;
  size_t trtri_elems = 0;
  HeevWork hw{};
  LanczosWork lw{};
  double *theta = nullptr, *res = nullptr, *dscale = nullptr, *partial = nullptr, *bounds = nullptr,
         *lam = nullptr, *resf = nullptr;
  int *info = nullptr, *flag = nullptr;
  unsigned* gcnt = nullptr;                 // arrival counters of the Gram kernel's split finish
  unsigned long long* vscratch = nullptr;   // matrix-variation reductions and thresholds
  unsigned long long* vd2 = nullptr;        // matrix-variation squared moduli (grown on demand)
  size_t vd2_bytes = 0;
  char* dvbuf = nullptr;                    // deviation-angle scratch (grown on demand)
  size_t dvbuf_bytes = 0;
  // emulated FP64 products of the reduction (digit form of L^-1 for both roles, and per
  // stream the digit forms of tril(A) and of T = L^-1 tril(A)); grown on demand
  int oz_slices = 0;                        // 0: FP64 pipe; 1..8: emulated with that many digits
  char* ozmem[2] = {nullptr, nullptr};      // [0] L^-1 operands + main-stream scratch, [1] side stream
  size_t ozmem_bytes[2] = {0, 0};
  gevp::OzOperand ozLA, ozLB, ozAB[2], ozTA[2];
  // solver products on the main stream: C (rows, per problem), A (rows, per final check),
  // B (rows, kept while the factorisation is), the block (columns, per product)
  gevp::OzOperand ozC, ozA, ozB, ozQ, ozLH;
  gevp::OzOperand ozQW, ozZ;                // the Rayleigh-Ritz rotation [Q; W] Z (rows, columns)
  gevp::OzOperand ozY, ozLiH;               // the CholQR product Y (L^-1 D)^H (rows, conjugated rows)
  gevp::OzOperand ozR, ozUV, ozVU;          // the localised update of the standard form
  // localised update: the B whose factorisation the last update call left (and its n, gen)
  const void* upd_B = nullptr;
  int64_t upd_n = 0, upd_gen = -1;
  int64_t* jidx = nullptr;                  // device copy of the changed rows
  size_t jidx_cap = 0;
  int64_t ozLH_gen = -1;                    // chol_gen the L^-H rows (ozLH) were split from
  double* ozws = nullptr;                   // split-K partials of the thin emulated products
  size_t ozws_doubles = 0;
  const void* ozC_src = nullptr;            // the C whose digits ozC holds (null: none)
  const void* ozB_src = nullptr;            // the B whose digits ozB holds, for chol_gen ozB_gen
  int64_t ozB_gen = -1;
  int64_t oz_l_gen = -1;                    // chol_gen the L^-1 operands were split from
  int oz_l_S = 0;
  int64_t chol_gen = 0;                     // incremented by every factorisation of B
  int* ozflags = nullptr;                   // device: [0] kernel error code, [1] non-finite entry
  // pinned host mirror
  double* hbuf = nullptr;
  size_t hbuf_elems = 0;
  // device staging of the host-buffer entry point (grown on demand)
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // warm-start state
  bool have_prev = false;
  int64_t prev_n = 0;
  int prev_m = 0;
  const void* prev_B = nullptr;
  bool chol_valid = false;
  // events
  std::vector<cudaEvent_t> evpool;
  std::string err;
  gevp::FilterTC* tc = nullptr;
  gevp::BatchPlan* batch = nullptr;   // state of the batched (k-point) entry point
  // sequence pipelining: the solver runs on a high-priority internal stream while a
  // low-priority side stream builds the next problem's standard form into a second set
  // of buffers (C2, its FP32 copy and bounds, the tensor-core planes in tc2)
  cudaStream_t hi = nullptr, side = nullptr;
  cudaEvent_t ev_main = nullptr, ev_side = nullptr, ev_user = nullptr;
  char* parena = nullptr;
  size_t parena_bytes = 0;
  double2 *C2 = nullptr, *T2 = nullptr, *split2 = nullptr;
  size_t split2_elems = 0;
  float2* M32b = nullptr;
  LanczosWork lw2{};
  double* bounds2 = nullptr;   // device: [0..4] bounds of C, [8..12] of A
  double* hb2 = nullptr;       // pinned copy
  gevp::FilterTC* tc2 = nullptr;
};

namespace gevp {
cudaStream_t ctx_stream(gevp_ctx* h) { return h->stream; }
int ctx_device(gevp_ctx* h) { return h->device; }
void ctx_set_error(gevp_ctx* h, const char* msg) { h->err = msg; }
BatchPlan*& ctx_batch(gevp_ctx* h) { return h->batch; }
}  // namespace gevp

namespace {

const char* kStatusNames[] = {"GEVP_OK", "GEVP_ERR_INVALID_ARG", "GEVP_ERR_NOT_HPD", "GEVP_ERR_NO_CONVERGENCE",
                              "GEVP_ERR_CUDA", "GEVP_ERR_OOM", "GEVP_ERR_TIMEOUT", "GEVP_ERR_INVALID_VALUE",
                              "GEVP_ERR_UNSUPPORTED"};

gevp_status cuda_fail(gevp_ctx* h, cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  h->err = buf;
  return e == cudaErrorMemoryAllocation ? GEVP_ERR_OOM : GEVP_ERR_CUDA;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

#define TRY(x)                         \
  do {                                 \
    gevp_status s_ = (x);              \
    if (s_ != GEVP_OK) return s_;      \
  } while (0)

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// Lay out (or only measure, when base == nullptr) every buffer for sizes (n, m).
size_t layout(gevp_ctx* h, char* base, int64_t n, int m) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += al(bytes);
    return p;
  };
  size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  h->L = (double2*)take(nn * 16);
  h->Linv = (double2*)take(nn * 16);
  h->C = (double2*)take(nn * 16);
  h->T = (double2*)take(nn * 16);
  h->M32 = (float2*)take(nn * 8);
  h->Q = (double2*)take(nm * 16);
  h->Y1 = (double2*)take(nm * 16);
  h->Y2 = (double2*)take(nm * 16);
  h->W = (double2*)take(nm * 16);
  h->Wt = (double2*)take(nm * 16);
  h->Xf = (double2*)take(nm * 16);
  h->G = (double2*)take(mm * 16);
  h->Zs = (double2*)take(mm * 16);
  h->Gw = (double2*)take(mm * 16);
  h->Gwi = (double2*)take(mm * 16);
  h->P = (double2*)take(mm * 16);
  h->split_elems = std::max<size_t>(64 * mm, 4 * nm);
  h->split_elems = std::max<size_t>(h->split_elems, 1 << 16);
  h->split = (double2*)take(h->split_elems * 16);
  int64_t tn = std::max<int64_t>(n, m);
  h->trtri_elems = trtri_ws_elems(tn) + std::max<size_t>(8 * (size_t)tn * 64, 1 << 16);
  h->trtri_ws = (double2*)take(h->trtri_elems * 16);
  // heev
  h->hw.G32 = (float2*)take(mm * 8);
  h->hw.Z32 = (float2*)take(mm * 8);
  h->hw.w32 = (float*)take(m * 4 + 64);
  h->hw.perm = (int*)take(m * 4 + 64);
  h->hw.Z = (double2*)take(mm * 16);
  h->hw.R = (double2*)take(mm * 16);
  h->hw.S = (double2*)take(mm * 16);
  h->hw.T = (double2*)take(mm * 16);
  h->hw.E = (double2*)take(mm * 16);
  h->hw.lam = (double*)take(m * 8 + 64);
  h->hw.scal = (double*)take(16 * 8 + 64 * 4);   // 16 scalars, then 64 floats of Jacobi reductions
  h->hw.split_ws = h->split;
  h->hw.split_ws_elems = h->split_elems;
  // lanczos (KMAX = 64)
  h->lw.V = (float2*)take((size_t)65 * n * 8);
  h->lw.ab = (float*)take(140 * 4);
  h->lw.w = (float2*)take((size_t)n * 8);
  h->lw.T32 = (float2*)take(64 * 64 * 8);
  h->lw.Z32 = (float2*)take(64 * 64 * 8);
  h->lw.w32 = (float*)take(64 * 4);
  h->lw.perm = (int*)take(64 * 4);
  h->lw.out = nullptr;
  h->theta = (double*)take(m * 8 + 64);
  h->res = (double*)take(m * 8 + 64);
  h->lam = (double*)take(m * 8 + 64);
  h->resf = (double*)take(m * 8 + 64);
  h->dscale = (double*)take(m * 8 + 64);
  h->partial = (double*)take(resid_partial_elems(n, m) * 8);
  h->bounds = (double*)take(16 * 8);
  h->info = (int*)take(64);
  h->flag = (int*)take(64);
  h->gcnt = (unsigned*)take(zgram_counters() * sizeof(unsigned));
  h->hw.gcnt = h->gcnt;
  h->vscratch = (unsigned long long*)take(64 * 8);
  return off;
}

gevp_status ensure(gevp_ctx* h, int64_t n, int m) {
  if (n <= h->cap_n && m <= h->cap_m && h->arena) return GEVP_OK;
  int64_t nn = std::max(n, h->cap_n);
  int mm = std::max(m, h->cap_m);
  // a change of the block width invalidates the warm-start block layout (ld = cap_m)
  h->have_prev = false;
  if (h->arena) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->arena);
    h->arena = nullptr;
  }
  size_t bytes = layout(h, nullptr, nn, mm);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    h->cap_n = 0;
    h->cap_m = 0;
    return cuda_fail(h, e, "workspace cudaMalloc");
  }
  h->arena = (char*)p;
  h->arena_bytes = bytes;
  layout(h, h->arena, nn, mm);
  CK(cudaMemsetAsync(h->gcnt, 0, zgram_counters() * sizeof(unsigned), h->stream));
  h->cap_n = nn;
  h->cap_m = mm;
  h->chol_valid = false;
  size_t hel = 8 * (size_t)mm + 64;
  if (hel > h->hbuf_elems) {
    if (h->hbuf) cudaFreeHost(h->hbuf);
    CK(cudaMallocHost(&h->hbuf, hel * sizeof(double)));
    h->hbuf_elems = hel;
  }
  return GEVP_OK;
}

// ---------------------------------------------------------------- phase timing
enum Phase { PH_CHOL, PH_REDUCE, PH_BOUNDS, PH_FILTER, PH_ORTH, PH_RR, PH_RESID, PH_FINAL, PH_N };

struct Timer {
  gevp_ctx* h;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  size_t used = 0;
  float ms[PH_N] = {0};
  explicit Timer(gevp_ctx* hh) : h(hh) {}
  cudaEvent_t ev() {
    if (used >= h->evpool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      h->evpool.push_back(e);
    }
    return h->evpool[used++];
  }
  void start() {
    cudaEvent_t e = ev();
    cudaEventRecord(e, h->stream);
    marks.push_back({-1, e});
  }
  void mark(int phase) {
    cudaEvent_t e = ev();
    cudaEventRecord(e, h->stream);
    marks.push_back({phase, e});
  }
  // call after the stream has been synchronised
  void resolve() {
    for (size_t i = 1; i < marks.size(); ++i) {
      if (marks[i].first < 0) continue;
      float t = 0.f;
      cudaEventElapsedTime(&t, marks[i - 1].second, marks[i].second);
      ms[marks[i].first] += t;
    }
    if (!marks.empty()) {
      auto last = marks.back();
      marks.clear();
      marks.push_back({-1, last.second});
    }
  }
};

gevp_status sync_read(gevp_ctx* h, const void* dsrc, void* hdst, size_t bytes) {
  CK(cudaMemcpyAsync(hdst, dsrc, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return GEVP_OK;
}

// several device-to-host reads with one synchronisation
struct ReadSpec {
  const void* dev;
  void* host;
  size_t bytes;
};
gevp_status sync_reads(gevp_ctx* h, std::initializer_list<ReadSpec> reads) {
  for (const ReadSpec& r : reads)
    if (r.bytes) CK(cudaMemcpyAsync(r.host, r.dev, r.bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return GEVP_OK;
}
gevp_status sync_read2(gevp_ctx* h, const void* d1, void* h1, size_t b1, const void* d2, void* h2, size_t b2) {
  return sync_reads(h, {{d1, h1, b1}, {d2, h2, b2}});
}

// ---------------------------------------------------------------- building blocks
bool factor_emulated(gevp_ctx* h, int64_t n, gevp_status* st);

// B = L L^H into h->L and L^-1 into h->Linv. With emulated products (oz_slices > 0) the
// recursive form of factor_emulated, else the blocked FP64 form (potrf.cu).
gevp_status factor_B(gevp_ctx* h, int64_t n, const double2* B, int64_t ldb, int64_t* info_out) {
  CK(cudaMemsetAsync(h->info, 0, sizeof(int), h->stream));
  zcopy2d(n, n, B, ldb, h->L, n, h->stream);
  gevp_status est = GEVP_OK;
  const bool emulated = h->oz_slices > 0 && factor_emulated(h, n, &est);
  if (est != GEVP_OK) return est;
  if (!emulated) potrf_lower(n, h->L, n, h->info, h->Linv, n, h->stream);
  int info = 0;
  TRY(sync_read(h, h->info, &info, sizeof(int)));
  if (info_out) *info_out = info;
  if (info != 0) {
    // the recursive form carries on past a failed leaf: its products may have flagged the
    // stale operands they met as non-finite
    if (emulated) CK(cudaMemsetAsync(h->ozflags, 0, 2 * sizeof(int), h->stream));
    h->chol_valid = false;
    char buf[96];
    snprintf(buf, sizeof buf, "B is not positive definite (pivot %d)", info);
    h->err = buf;
    return GEVP_ERR_NOT_HPD;
  }
  if (!emulated) trtri_lower(n, h->L, n, h->Linv, n, h->trtri_ws, h->trtri_elems, h->stream, true);
  h->chol_valid = true;
  ++h->chol_gen;
  return GEVP_OK;
}

// C = Linv A Linv^H into Cout (n x n, ld ldc), via T = Linv tril_half(A), M = T Linv^H,
// with the given scratch (T, split-K) on the given stream.
void reduce_into_ws(int64_t n, const double2* Linv, const double2* A, int64_t lda, double2* Cout, int64_t ldc,
                    double2* T, double2* split, size_t split_elems, cudaStream_t s) {
  ZgemmArgs a = zg((int)n, (int)n, (int)n, Linv, n, 0, A, lda, 0, T, n);
  a.triA = 1;
  a.maskB = 1;
  zgemm(a, split, split_elems, s);
  ZgemmArgs b = zg((int)n, (int)n, (int)n, T, n, 0, Linv, n, 1, Cout, ldc);
  b.triA = 1;
  b.triB = 2;
  zgemm(b, split, split_elems, s);
  herm_sum_inplace(n, Cout, ldc, s);
}

// The same reduction with the n^3 products emulated on the tensor cores (slices digits
// per entry): T = L^-1 tril_half(A) and M = T L^-H as digit-form products, then C = M + M^H.
// side 0 runs on the main stream, side 1 on the pipeline's side stream (own scratch). The
// digit forms of L^-1 are made once per factorisation of B, on the main stream.
// the device status words of the emulated products ([0] error code, [1] non-finite entry)
gevp_status oz_flags_ready(gevp_ctx* h) {
  if (h->ozflags) return GEVP_OK;
  void* p = nullptr;
  CK(cudaMalloc(&p, 2 * sizeof(int)));
  CK(cudaMemsetAsync(p, 0, 2 * sizeof(int), h->stream));
  h->ozflags = (int*)p;
  return GEVP_OK;
}

// device scratch of the emulated products: ozmem[side] of at least `need` bytes
gevp_status oz_reserve(gevp_ctx* h, int side, size_t need) {
  TRY(oz_flags_ready(h));
  if (need <= h->ozmem_bytes[side]) return GEVP_OK;
  // the other stream may still read this side's (or, for side 0, the shared) operands
  cudaDeviceSynchronize();
  if (h->ozmem[side]) cudaFree(h->ozmem[side]);
  h->ozmem[side] = nullptr;
  h->ozmem_bytes[side] = 0;
  if (side == 0) {
    h->oz_l_gen = -1;
    h->ozC_src = nullptr;
    h->ozB_src = nullptr;
    h->ozLH_gen = -1;
  }
  void* p = nullptr;
  CK(cudaMalloc(&p, need));
  h->ozmem[side] = (char*)p;
  h->ozmem_bytes[side] = need;
  return GEVP_OK;
}

// Main-stream digit scratch: [L^-1 rows | L^-H columns | reduction: tril(A) | T | A | B |
// L^-H rows (the back-transform's left operand)]
// (the solver's C digits reuse the T region and the block's digits the tril(A) region:
// the reduction of a problem is finished before its solve starts, on the same stream)
size_t oz_main_bytes(int64_t n, int S) {
  const size_t bA = gevp::oz_operand_bytes((int)n, (int)n, S, 2), bB = gevp::oz_operand_bytes((int)n, (int)n, S, 3);
  return 5 * bA + 2 * bB;
}
// 0 L^-1, 1 L^-H columns, 2 tril(A)/block, 3 T/C, 4 A, 5 B, 6 L^-H rows
char* oz_region(gevp_ctx* h, int64_t n, int which) {
  const int S = h->oz_slices;
  const size_t bA = gevp::oz_operand_bytes((int)n, (int)n, S, 2), bB = gevp::oz_operand_bytes((int)n, (int)n, S, 3);
  const size_t off[7] = {0, bA, bA + bB, bA + 2 * bB, 2 * bA + 2 * bB, 3 * bA + 2 * bB, 4 * bA + 2 * bB};
  return h->ozmem[0] + off[which];
}

// D (n x ncols, ld ldd) = M X with M one of the cached square operands (ozC, ozA, ozB) and
// X the n x ncols block (ld ldx), emulated on the main stream
gevp_status oz_times_block(gevp_ctx* h, const gevp::OzOperand& M, int64_t n, int ncols, const double2* X,
                           int64_t ldx, double2* D, int64_t ldd) {
  CK(gevp::oz_split(h->ozQ, oz_region(h, n, 2), ncols, (int)n, X, ldx, 0, 0, h->oz_slices, 3, h->ozflags + 1,
                    h->stream, true));
  CK(gevp::oz_gemm(M, h->ozQ, 0, 0, D, ldd, h->ozflags, h->stream, nullptr, h->ozws, h->ozws_doubles));
  return GEVP_OK;
}

// h->L (holding B) -> L, h->Linv -> L^-1 by chol_recursive (cholqr.cu), its digit operands
// in the first two regions of the main-stream scratch (the L^-1 digits, remade after it).
// false: not done (order above the emulated products' limit, or the cluster leaves not
// launchable: nothing was enqueued; *st set on a failure after work was enqueued).
bool factor_emulated(gevp_ctx* h, int64_t n, gevp_status* st) {
  *st = GEVP_OK;
  if (n > 30720) return false;
  const int S = h->oz_slices;
  gevp::CholRes r{};
  if (n > gevp::kCholLeaf) {
    if ((*st = oz_reserve(h, 0, oz_main_bytes(n, S))) != GEVP_OK) return false;
    // split-K partials for the products near the leaves (up to 512 x 512 at 4 slices)
    const size_t wd = gevp::oz_split_k_doubles(512, 512) / 2;
    if (h->ozws_doubles < wd) {
      if (h->ozws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ozws);
      }
      h->ozws = nullptr;
      h->ozws_doubles = 0;
      void* p = nullptr;
      if (cudaMalloc(&p, wd * sizeof(double)) != cudaSuccess) {
        *st = GEVP_ERR_OOM;
        return false;
      }
      h->ozws = (double*)p;
      h->ozws_doubles = wd;
    }
    r.memA = oz_region(h, n, 0);
    r.memB = oz_region(h, n, 1);
    r.T = h->T;
    r.ldt = n;
    r.ws = h->ozws;
    r.ws_doubles = h->ozws_doubles;
  }
  r.flags = h->ozflags;
  r.info = h->info;
  r.S = S;
  r.s = h->stream;
  const cudaError_t e = gevp::chol_recursive(n, h->L, n, h->Linv, n, r);
  if (e == cudaErrorNotSupported) return false;
  if (e != cudaSuccess) {
    *st = GEVP_ERR_CUDA;
    return false;
  }
  return true;
}

gevp_status reduce_emulated(gevp_ctx* h, int side, int64_t n, const double2* A, int64_t lda, double2* Cout,
                            int64_t ldc, double2* T, cudaStream_t s) {
  const int S = h->oz_slices;
  const int nn = (int)n;
  const size_t bA = gevp::oz_operand_bytes(nn, nn, S, 2), bB = gevp::oz_operand_bytes(nn, nn, S, 3);
  TRY(oz_reserve(h, side, side == 0 ? oz_main_bytes(n, S) : bA + bB));
  char* mem = h->ozmem[side];
  if (side == 0 && (h->oz_l_gen != h->chol_gen || h->oz_l_S != S)) {
    // L^-1 as the left operand (rows, lower) and L^-H as the right one (rows of L^-1, conjugated)
    CK(gevp::oz_split(h->ozLA, mem, nn, nn, h->Linv, n, 0, 2, S, 2, h->ozflags + 1, h->stream));
    CK(gevp::oz_split(h->ozLB, mem + bA, nn, nn, h->Linv, n, 1, 2, S, 3, h->ozflags + 1, h->stream));
    h->oz_l_gen = h->chol_gen;
    h->oz_l_S = S;
  }
  if (side == 0) mem += bA + bB;
  // columns of tril_half(A) are the conjugated rows of the Hermitian A from the diagonal on
  CK(gevp::oz_split(h->ozAB[side], mem, nn, nn, A, lda, 1, 1, S, 3, h->ozflags + 1, s));
  CK(gevp::oz_gemm(h->ozLA, h->ozAB[side], 1, 1, T, n, h->ozflags, s));
  CK(gevp::oz_split(h->ozTA[side], mem + bB, nn, nn, T, n, 0, 2, S, 2, h->ozflags + 1, s));
  CK(gevp::oz_gemm(h->ozTA[side], h->ozLB, 1, 2, Cout, ldc, h->ozflags, s));
  herm_sum_inplace(n, Cout, ldc, s);
  return GEVP_OK;
}

gevp_status reduce_into(gevp_ctx* h, int64_t n, const double2* A, int64_t lda, double2* Cout, int64_t ldc) {
  if (h->oz_slices > 0) return reduce_emulated(h, 0, n, A, lda, Cout, ldc, h->T, h->stream);
  reduce_into_ws(n, h->Linv, A, lda, Cout, ldc, h->T, h->split, h->split_elems, h->stream);
  return GEVP_OK;
}

// error code of an emulated-product kernel since the last check (0: none), then cleared
gevp_status oz_check(gevp_ctx* h) {
  if (!h->ozflags) return GEVP_OK;
  int f[2] = {0, 0};
  CK(cudaMemcpyAsync(f, h->ozflags, sizeof f, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (f[0] == 0 && f[1] == 0) return GEVP_OK;
  CK(cudaMemsetAsync(h->ozflags, 0, 2 * sizeof(int), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (f[0] != 0) {
    h->err = "a bounded wait of the emulated FP64 product ran out";
    return GEVP_ERR_TIMEOUT;
  }
  h->err = "NaN or Inf in an operand of the emulated FP64 product";
  return GEVP_ERR_INVALID_VALUE;
}

// Streams and buffers of the sequence pipeline (sized from the main arena's n and split).
gevp_status ensure_pipeline(gevp_ctx* h) {
  if (!h->hi) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, greatest));
    CK(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, least));
    CK(cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_side, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_user, cudaEventDisableTiming));
  }
  if (!h->hb2) CK(cudaMallocHost(&h->hb2, 24 * sizeof(double)));
  const int64_t n = h->cap_n;
  auto lay = [&](char* base) -> size_t {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
      char* p = base ? base + off : nullptr;
      off += al(bytes);
      return p;
    };
    h->C2 = (double2*)take((size_t)n * n * 16);
    h->T2 = (double2*)take((size_t)n * n * 16);
    h->M32b = (float2*)take((size_t)n * n * 8);
    h->split2 = (double2*)take(h->split_elems * 16);
    h->lw2.V = (float2*)take((size_t)65 * n * 8);
    h->lw2.ab = (float*)take(140 * 4);
    h->lw2.w = (float2*)take((size_t)n * 8);
    h->lw2.T32 = (float2*)take(64 * 64 * 8);
    h->lw2.Z32 = (float2*)take(64 * 64 * 8);
    h->lw2.w32 = (float*)take(64 * 4);
    h->lw2.perm = (int*)take(64 * 4);
    h->lw2.out = nullptr;
    h->bounds2 = (double*)take(24 * 8);
    return off;
  };
  const size_t need = lay(nullptr);
  if (!h->parena || need > h->parena_bytes) {
    if (h->parena) {
      cudaStreamSynchronize(h->side);
      cudaFree(h->parena);
      h->parena = nullptr;
    }
    void* p = nullptr;
    CK(cudaMalloc(&p, need));
    h->parena = (char*)p;
    h->parena_bytes = need;
  }
  lay(h->parena);
  h->split2_elems = h->split_elems;
  return GEVP_OK;
}

// One CholQR pass on the tall-skinny kernels: W = src^H src (lower tiles, one launch),
// Li = L^-1 D with D W D + sh I = L L^H (one cluster launch, *info set on a non-positive
// pivot), dst = src Li^H = src D L^-H. False if the cluster factorisation is not available
// for this order (nothing enqueued after the Gram matrix then).
// The product runs emulated on the tensor cores when the solve's products are (its digit
// operands in the block region of the main-stream scratch, free between the filter and the
// Rayleigh-Ritz rotation), else on the FP64 pipe.
bool cholqr_pass(gevp_ctx* h, int64_t n, int ma, const double2* src, int64_t lds, double2* dst, int64_t ldd, double sh,
                 int* info) {
  if (ma > cholinv_max_order()) return false;
  zgram(n, ma, ma, src, lds, src, lds, h->Gw, ma, 1, h->split, h->split_elems, h->gcnt, h->stream);
  if (!cholinv_small(ma, h->Gw, ma, sh, h->Gwi, ma, nullptr, 0, info, h->stream)) return false;
  const int S = h->oz_slices;
  if (S > 0 && h->ozmem[0] && h->ozmem_bytes[0] >= oz_main_bytes(n, S) &&
      gevp::oz_operand_bytes((int)n, ma, S, 2) + gevp::oz_operand_bytes(ma, ma, S, 3) <=
          gevp::oz_operand_bytes((int)n, (int)n, S, 3)) {
    // dst = Y (L^-1 D)^H: the columns of (L^-1 D)^H are the conjugated rows of the lower L^-1 D
    char* mem = oz_region(h, n, 2);
    if (gevp::oz_split(h->ozY, mem, (int)n, ma, src, lds, 0, 0, S, 2, h->ozflags + 1, h->stream) == cudaSuccess &&
        gevp::oz_split(h->ozLiH, mem + gevp::oz_operand_bytes((int)n, ma, S, 2), ma, ma, h->Gwi, ma, 1, 2, S, 3,
                       h->ozflags + 1, h->stream) == cudaSuccess &&
        gevp::oz_gemm(h->ozY, h->ozLiH, 0, 2, dst, ldd, h->ozflags, h->stream, nullptr, h->ozws, h->ozws_doubles) ==
            cudaSuccess)
      return true;
    cudaGetLastError();
  }
  ZgemmArgs q = zg((int)n, ma, ma, src, lds, 0, h->Gwi, ma, 1, dst, ldd);
  q.triB = 2;
  zgemm(q, h->split, h->split_elems, h->stream);
  return true;
}

// Orthonormalise Y (n x ma, ld ldy) against Q[:, 0:nlock] and by CholQR2; result in Out.
// The usual case, two plain passes that both succeed, is enqueued at once (the first into
// the free block Xf, the second into Out, so Y is still intact if a pass fails) with a
// single status read after both. Otherwise a pass whose Gram matrix is not numerically
// positive definite is repeated as shifted CholQR (Fukaya et al. 2020); the result is
// accepted only after two consecutive plain passes (so a shifted pass is always followed
// by CholQR2). A block that stays rank deficient is replaced by fresh random columns
// (projected against the locked ones).
// pending (nullable): the two-pass fast path is only enqueued and *pending set to 1; the
// caller reads the passes' statuses h->info[0..1] later (with its next read) and, if either
// is set, calls again with allow_fast = false (Y is left intact by the fast path).
gevp_status orthonormalize(gevp_ctx* h, int64_t n, int nlock, double2* Y, int64_t ldy, int ma, double2* Out,
                           int64_t ldo, gevp_stats* st, uint64_t seed = 0, int* pending = nullptr,
                           bool allow_fast = true) {
  const int64_t ldq = h->cap_m;
  const bool fast = ma <= cholinv_max_order();
  if (pending) *pending = 0;
  for (int restart = 0; restart < 2; ++restart) {
    for (int pass = 0; pass < 2 && nlock > 0; ++pass) {
      zgram(n, nlock, ma, h->Q, ldq, Y, ldy, h->P, ma, 0, h->split, h->split_elems, h->gcnt, h->stream);
      ZgemmArgs u = zg((int)n, ma, nlock, h->Q, ldq, 0, h->P, ma, 0, Y, ldy, -1.0);
      u.Cin = Y; u.ldc = ldy; u.beta = 1.0;
      zgemm(u, h->split, h->split_elems, h->stream);
    }
    if (fast && allow_fast && restart == 0) {
      CK(cudaMemsetAsync(h->info, 0, 2 * sizeof(int), h->stream));
      if (cholqr_pass(h, n, ma, Y, ldy, h->Xf, ldq, 0.0, h->info) &&
          cholqr_pass(h, n, ma, h->Xf, ldq, Out, ldo, 0.0, h->info + 1)) {
        if (st) st->flops_fp64 += 2 * 8.0 * (double)n * ma * ma;
        if (pending) {
          *pending = 1;
          return GEVP_OK;
        }
        int inf[2] = {0, 0};
        TRY(sync_read(h, h->info, inf, sizeof inf));
        if (inf[0] == 0 && inf[1] == 0) return GEVP_OK;
      }
    }
    double2* src = Y;
    int64_t lds = ldy;
    double2* dst = Out;
    int64_t ldd = ldo;
    int plain_ok = 0;
    bool failed = false;
    for (int pass = 0; pass < 6 && plain_ok < 2; ++pass) {
      bool shifted = false;
      bool clustered = false;
      int attempt = 0;
      for (; attempt < 3; ++attempt) {
        double sh = 0.0;
        if (shifted) {
          // s = 11 (n m + m (m+1)) u ||Y D||_2^2 with ||Y D||_F^2 = m, grown 100x per retry
          double u = 1.1102230246251565e-16;
          sh = 11.0 * ((double)n * ma + (double)ma * (ma + 1)) * u * ma * std::pow(100.0, attempt - 1);
        }
        CK(cudaMemsetAsync(h->info, 0, sizeof(int), h->stream));
        clustered = false;
        if (fast) {
          zgram(n, ma, ma, src, lds, src, lds, h->Gw, ma, 1, h->split, h->split_elems, h->gcnt, h->stream);
          clustered = cholinv_small(ma, h->Gw, ma, sh, h->Gwi, ma, nullptr, 0, h->info, h->stream);
        }
        if (!clustered) {
          ZgemmArgs g = zg(ma, ma, (int)n, src, lds, 1, src, lds, 0, h->Gw, ma);
          g.triD = 1;
          zgemm(g, h->split, h->split_elems, h->stream);
          hermitize_lower(ma, h->Gw, ma, h->stream);
          gram_scale(ma, h->Gw, ma, h->dscale, h->stream);
          if (shifted) zshift_diag(ma, h->Gw, ma, sh, h->stream);
          potrf_lower(ma, h->Gw, ma, h->info, h->Gwi, ma, h->stream);
        }
        int info = 0;
        TRY(sync_read(h, h->info, &info, sizeof(int)));
        if (info == 0) break;
        shifted = true;
        if (st) st->orth_fallbacks++;
      }
      if (attempt == 3) { failed = true; break; }
      plain_ok = shifted ? 0 : plain_ok + 1;
      if (!clustered) {
        trtri_lower(ma, h->Gw, ma, h->Gwi, ma, h->trtri_ws, h->trtri_elems, h->stream, true);
        zcol_scale(n, ma, src, lds, h->dscale, h->stream);
      }
      ZgemmArgs q = zg((int)n, ma, ma, src, lds, 0, h->Gwi, ma, 1, dst, ldd);
      q.triB = 2;
      zgemm(q, h->split, h->split_elems, h->stream);
      if (st) st->flops_fp64 += 8.0 * (double)n * ma * ma;
      std::swap(src, dst);
      std::swap(lds, ldd);
    }
    if (!failed && plain_ok >= 2) {
      if (src != Out) zcopy2d(n, ma, src, lds, Out, ldo, h->stream);
      return GEVP_OK;
    }
    // rank deficient: restart the block from random columns
    zrandn(n, ma, Y, ldy, 0x9E3779B97F4A7C15ull ^ (seed + 7919ull * (uint64_t)(restart + 1)), h->stream);
    if (st) st->orth_fallbacks += 100;
  }
  h->err = "CholQR: block stays rank deficient";
  return GEVP_ERR_NOT_HPD;
}

// Out = C Qa (n x ma, ld of the block), emulated when C's digits are held
gevp_status times_C(gevp_ctx* h, int64_t n, int ma, const double2* C, int64_t ldc, const double2* Qa, double2* Out) {
  const int64_t ld = h->cap_m;
  if (h->oz_slices > 0 && h->ozC_src == (const void*)C) {
    TRY(oz_times_block(h, h->ozC, n, ma, Qa, ld, Out, ld));
  } else {
    ZgemmArgs w = zg((int)n, ma, (int)n, C, ldc, 0, Qa, ld, 0, Out, ld);
    zgemm(w, h->split, h->split_elems, h->stream);
  }
  return GEVP_OK;
}

// Rayleigh-Ritz on the active columns Q[:, nlock:nlock+ma]; updates Q, W, theta, res there.
gevp_status rayleigh_ritz(gevp_ctx* h, int64_t n, int nlock, int ma, const double2* C, int64_t ldc,
                          int refine, gevp_stats* st) {
  const int64_t ld = h->cap_m;
  double2* Qa = h->Q + nlock;
  TRY(times_C(h, n, ma, C, ldc, Qa, h->Wt));
  // G = Q^H C Q is Hermitian: its lower tiles only, both triangles written
  zgram(n, ma, ma, Qa, ld, h->Wt, ld, h->G, ma, 1, h->split, h->split_elems, h->gcnt, h->stream);
  heev_small(ma, h->G, ma, h->theta + nlock, h->Zs, ma, h->hw, refine, h->stream);
  // [Q W] <- [Q Wt] Z. Emulated (when C's products are): the two blocks stacked into the
  // free n x n scratch T as one 2n x ma operand, so that one product fills the SMs; else one
  // FP64 launch (a batch of two products sharing Z). Q's result goes through T or Xf (free
  // until the final check), so that the filtered block in Y1/Y2 stays intact.
  const int S = h->oz_slices;
  const size_t qw_bytes = S > 0 ? gevp::oz_operand_bytes(2 * (int)n, ma, S, 2) + gevp::oz_operand_bytes(ma, ma, S, 3)
                                : 0;
  // (the emulated operands' memory is reserved for this n while C's digits are held)
  if (S > 0 && h->ozC_src == (const void*)C && 2 * n * (int64_t)ma <= n * n &&
      qw_bytes <= gevp::oz_operand_bytes((int)n, (int)n, S, 3)) {
    zcopy2d(n, ma, Qa, ld, h->T, ma, h->stream);
    zcopy2d(n, ma, h->Wt, ld, h->T + n * ma, ma, h->stream);
    char* mem = oz_region(h, n, 2);
    CK(gevp::oz_split(h->ozQW, mem, 2 * (int)n, ma, h->T, ma, 0, 0, S, 2, h->ozflags + 1, h->stream));
    CK(gevp::oz_split(h->ozZ, mem + gevp::oz_operand_bytes(2 * (int)n, ma, S, 2), ma, ma, h->Zs, ma, 0, 0, S, 3,
                      h->ozflags + 1, h->stream, true));
    CK(gevp::oz_gemm(h->ozQW, h->ozZ, 0, 0, h->T, ma, h->ozflags, h->stream, nullptr, h->ozws, h->ozws_doubles));
    zcopy2d(n, ma, h->T, ma, Qa, ld, h->stream);
    zcopy2d(n, ma, h->T + n * ma, ma, h->W + nlock, ld, h->stream);
  } else {
    ZgemmArgs q = zg((int)n, ma, ma, Qa, ld, 0, h->Zs, ma, 0, h->Xf, ld);
    q.batch = 2;
    q.sA = h->Wt - Qa;
    q.sD = (h->W + nlock) - h->Xf;
    zgemm(q, h->split, h->split_elems, h->stream);
    zcopy2d(n, ma, h->Xf, ld, Qa, ld, h->stream);
  }
  resid_norms(n, ma, h->W + nlock, ld, Qa, ld, h->theta + nlock, h->res + nlock, h->partial, h->stream);
  if (st) st->flops_fp64 += 8.0 * ((double)n * n * ma + 3.0 * n * ma * ma) + 32.0 * refine * (double)ma * ma * ma;
  return GEVP_OK;
}

// Chebyshev filter on Y0 (n x ma, ld ld0) with FP64 products; returns the output buffer.
double2* filter_fp64(gevp_ctx* h, int64_t n, const double2* C, int64_t ldc, const double2* Y0, int64_t ld0, int ma,
                     int deg, double lo, double hi, double sc, double2* B1, double2* B2, int64_t ldb) {
  return cheb_filter_fp64(n, C, ldc, Y0, ld0, ma, deg, lo, hi, sc, B1, B2, ldb, h->split, h->split_elems, h->stream);
}

gevp_status lanczos(gevp_ctx* h, int64_t n, const double2* M, int64_t ldm, int k, int count, uint64_t seed,
                    double* host_out) {
  z_to_c(n, n, M, ldm, h->M32, n, h->stream);
  lanczos_bounds(n, h->M32, n, k, count, seed, h->lw, h->bounds, h->stream);
  return sync_read(h, h->bounds, host_out, 5 * sizeof(double));
}

// GEVP_TRACE set in the environment: one line per solver round on stderr
bool trace_on() {
  static const bool on = std::getenv("GEVP_TRACE") != nullptr;
  return on;
}

struct SolveState {
  int m, nev;
  int nlock = 0;
  bool have_theta = false;
  std::vector<double> theta, res;
  double upper = 0, lower_est = 0, a_est = 0, normC = 1, normA = 1;
};

int choose_degree(const SolveState& S, double lo, double hi, double tolC, int dmin, int dmax) {
  double e = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
  int d = dmin;
  for (int i = S.nlock; i < S.nev; ++i) {
    double r = S.res[i];
    if (r <= tolC) continue;
    double t = (S.theta[i] - c) / e;
    double at = std::fabs(t);
    if (at <= 1.0) { d = dmax; break; }
    double rho = at + std::sqrt(at * at - 1.0);
    // aim 10x below the tolerance: a degree that only just reaches it leaves the pairs
    // closest to the damped interval crawling over several extra rounds
    int di = (int)std::ceil(std::log(10.0 * r / tolC) / std::log(rho));
    d = std::max(d, di);
  }
  return std::min(std::max(d, dmin), dmax);
}

// Highest degree whose dynamic range the filter can carry. The scaled filter keeps the
// column at the scaling point sc at 1 and damps the guard columns near lo towards
// 1 / T_d(t_sc); once that falls below the filter's relative noise, the guard columns
// degenerate into noise and the last wanted pairs (which need them) stop converging.
// kappa ~ the inverse noise level of the filter's arithmetic: FP32-class 1e7, BF16 1e3,
// FP64 1e12 (CholQR's limit). The residual-corrected filter (corrected) rounds relative to
// the defect p(C) Q - Q p(Theta), whose norm is the residual level rather than the block's,
// so its guard columns carry a wider range: 100x for the low-precision modes (measured on
// the n 2048 and n 6144 sequences: beyond about 1000x the BF16 filter stalls and the
// solver falls back to FP64).
int range_degree_cap(double sc, double lo, double hi, int prec, bool corrected) {
  const double e = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
  const double at = std::fabs((sc - c) / e);
  if (!(at > 1.0)) return 1 << 20;
  double kappa = prec == GEVP_PREC_FP32 ? 1e7 : (prec == GEVP_PREC_BF16 ? 1e3 : 1e12);
  if (corrected && prec != GEVP_PREC_FP64) kappa *= 100.0;
  return (int)std::floor(std::log(2.0 * kappa) / std::log(at + std::sqrt(at * at - 1.0)));
}

// Largest residual among the unlocked wanted pairs that Chebyshev theory predicts after a
// filter of degree deg: an unconverged pair's residual shrinks by |T_deg(t_i)| (t_i its
// Ritz value mapped to the damped interval; no gain when |t_i| <= 1).
double predicted_max_res(const SolveState& S, double lo, double hi, double tolC, int deg) {
  double e = 0.5 * (hi - lo), c = 0.5 * (hi + lo), pred = 0.0;
  for (int i = S.nlock; i < S.nev; ++i) {
    double r = S.res[i];
    double at = std::fabs((S.theta[i] - c) / e);
    if (r > tolC && at > 1.0) r /= std::cosh(deg * std::acosh(std::min(at, 1e150)));
    pred = std::max(pred, r);
  }
  return pred;
}

// ||Q^H Q - I||_max over the first nev columns of Q (= ||X^H B X - I|| up to the rounding of
// L^-1) into h->partial[0]: the Gram kernel (Hermitian), its deviation reduced on the device
void orth_enqueue(gevp_ctx* h, int64_t n, int nev) {
  zgram(n, nev, nev, h->Q, h->cap_m, h->Q, h->cap_m, h->Gwi, nev, 1, h->split, h->split_elems, h->gcnt, h->stream);
  eye_deviation(nev, h->Gwi, nev, h->partial, h->stream);
}

// Solve one problem whose standard form is already in h->C. Q holds the start block
// (orthonormal, all m columns) when warm; otherwise it is drawn here.
gevp_status solve_one(gevp_ctx* h, int64_t n, const double2* A, int64_t lda, const double2* B, int64_t ldb,
                      int nev, int m, bool warm, const gevp_opts& o, int prob_index, Timer& tm, gevp_stats* st,
                      double* Lam_out, double2* X_out, int64_t ldx, double* res_out, const double* pre = nullptr,
                      bool tc_ready = false) {
  const int64_t ld = h->cap_m;
  SolveState S;
  S.m = m;
  S.nev = nev;
  S.theta.assign(m, 0.0);
  S.res.assign(m, 0.0);
  double hb[16];
  // bounds of C, and an estimate of ||A||_2 for the final residuals (pre: computed ahead
  // on the side stream, by the same kernels with the same seeds)
  if (pre) std::memcpy(hb, pre, 5 * sizeof(double));
  else TRY(lanczos(h, n, h->C, n, o.lanczos_steps, m, o.seed + 7919ull * prob_index, hb));
  S.lower_est = hb[0];
  S.upper = hb[2];
  S.a_est = hb[3];
  S.normC = std::max(std::fabs(hb[0]), std::fabs(hb[2]));
  if (pre) std::memcpy(hb, pre + 8, 5 * sizeof(double));
  else TRY(lanczos(h, n, A, lda, o.lanczos_steps, 0, o.seed + 104729ull * prob_index + 1, hb));
  S.normA = std::max(std::fabs(hb[0]), std::fabs(hb[1]));
  int prec = o.filter_prec;
  const int nsplit = (prec == GEVP_PREC_FP32) ? 3 : 1;
  if (prec != GEVP_PREC_FP64 && !tc_ready) {
    CK(filter_tc_reserve(&h->tc, n, m, h->stream));
    CK(filter_tc_set_matrix(h->tc, n, h->C, n, nsplit, h->stream));
  }
  // emulated products: the digits of C for every W = C Q of this problem
  const bool oz = h->oz_slices > 0;
  bool oz_a_ready = false;
  if (oz) {
    TRY(oz_reserve(h, 0, oz_main_bytes(n, h->oz_slices)));
    CK(gevp::oz_split(h->ozC, oz_region(h, n, 3), (int)n, (int)n, h->C, n, 0, 0, h->oz_slices, 2, h->ozflags + 1,
                      h->stream));
    h->ozC_src = h->C;
    // split-K partials of the n x m products (W = C Q, the back-transform, A X, B X)
    const size_t wd = gevp::oz_split_k_doubles((int)n, m);
    if (wd > h->ozws_doubles) {
      if (h->ozws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ozws);
      }
      h->ozws = nullptr;
      h->ozws_doubles = 0;
      void* p = nullptr;
      CK(cudaMalloc(&p, wd * sizeof(double)));
      h->ozws = (double*)p;
      h->ozws_doubles = wd;
    }
  }
  tm.mark(PH_BOUNDS);
  if (!warm) {
    zrandn(n, m, h->Y1, ld, o.seed * 1000003ull + (uint64_t)prob_index, h->stream);
    TRY(orthonormalize(h, n, 0, h->Y1, ld, m, h->Q, ld, st));
    tm.mark(PH_ORTH);
  }
  if (warm || m == n) {
    // warm start (the Rayleigh-Ritz pairs of the start block against this C: its residual
    // R = C Q - Q Theta, which drives the corrected low-precision filter, then has no
    // component inside span Q), or a block that spans the whole space (then this
    // projection is exact)
    TRY(rayleigh_ritz(h, n, 0, m, h->C, n, o.refine_iters, st));
    TRY(sync_read2(h, h->theta, S.theta.data(), m * sizeof(double), h->res, S.res.data(), m * sizeof(double)));
    S.have_theta = true;
    tm.mark(PH_RR);
  }
  double tolC = 0.1 * o.tol * S.normC;
  double orth_val = -1.0;   // max |Q^H Q - I| of the block the last final check saw
  int final_pass = 0;
  double prev_maxres = 1e300;
  bool converged = false;
  int deg_cap = o.deg_max;   // lowered when the FP32-class filter reaches its floor
  for (int it = 0;; ++it) {
    if (S.have_theta) {
      while (S.nlock < nev && S.res[S.nlock] <= tolC) S.nlock++;
    }
    if (S.nlock >= nev) {
      // ---- final check in the original space
      if (oz) {
        // X = L^-H Q: the rows of L^-H (upper) are the conjugated columns of L^-1, made
        // once per factorisation
        if (h->ozLH_gen != h->chol_gen || h->ozLH.S != h->oz_slices) {
          CK(gevp::oz_split(h->ozLH, oz_region(h, n, 6), (int)n, (int)n, h->Linv, n, 1, 3, h->oz_slices, 2,
                            h->ozflags + 1, h->stream, true));
          h->ozLH_gen = h->chol_gen;
        }
        CK(gevp::oz_split(h->ozQ, oz_region(h, n, 2), nev, (int)n, h->Q, ld, 0, 0, h->oz_slices, 3, h->ozflags + 1,
                          h->stream, true));
        CK(gevp::oz_gemm(h->ozLH, h->ozQ, 2, 0, h->Xf, ld, h->ozflags, h->stream, nullptr, h->ozws, h->ozws_doubles));
      } else {
        ZgemmArgs x = zg((int)n, nev, (int)n, h->Linv, n, 1, h->Q, ld, 0, h->Xf, ld);
        x.triA = 2;
        zgemm(x, h->split, h->split_elems, h->stream);
      }
      if (oz) {
        // A X and B X emulated: A's digits once per problem, B's while it stays factorised
        if (!oz_a_ready) {
          CK(gevp::oz_split(h->ozA, oz_region(h, n, 4), (int)n, (int)n, A, lda, 0, 0, h->oz_slices, 2,
                            h->ozflags + 1, h->stream));
          oz_a_ready = true;
        }
        if (h->ozB_src != (const void*)B || h->ozB_gen != h->chol_gen) {
          CK(gevp::oz_split(h->ozB, oz_region(h, n, 5), (int)n, (int)n, B, ldb, 0, 0, h->oz_slices, 2,
                            h->ozflags + 1, h->stream));
          h->ozB_src = B;
          h->ozB_gen = h->chol_gen;
        }
        CK(gevp::oz_split(h->ozQ, oz_region(h, n, 2), nev, (int)n, h->Xf, ld, 0, 0, h->oz_slices, 3, h->ozflags + 1,
                          h->stream, true));
        CK(gevp::oz_gemm(h->ozA, h->ozQ, 0, 0, h->Y1, ld, h->ozflags, h->stream, nullptr, h->ozws, h->ozws_doubles));
        CK(gevp::oz_gemm(h->ozB, h->ozQ, 0, 0, h->Y2, ld, h->ozflags, h->stream, nullptr, h->ozws, h->ozws_doubles));
      } else {
        ZgemmArgs ax = zg((int)n, nev, (int)n, A, lda, 0, h->Xf, ld, 0, h->Y1, ld);
        zgemm(ax, h->split, h->split_elems, h->stream);
        ZgemmArgs bx = zg((int)n, nev, (int)n, B, ldb, 0, h->Xf, ld, 0, h->Y2, ld);
        zgemm(bx, h->split, h->split_elems, h->stream);
      }
      // Y1/Y2 share ld; final_check wants one ld for X, AX, BX
      final_check(n, nev, h->Xf, h->Y1, h->Y2, ld, h->lam, h->resf, S.normA, h->partial, h->stream);
      if (st) st->flops_fp64 += 8.0 * (double)n * n * nev * 2.5;
      // the returned block's orthonormality, read with the residuals (kept if they pass)
      if (st) orth_enqueue(h, n, nev);
      std::vector<double> rf(nev);
      double ov = -1.0;
      TRY(sync_reads(h, {{h->resf, rf.data(), nev * sizeof(double)}, {h->partial, &ov, st ? sizeof ov : 0}}));
      orth_val = ov;
      tm.mark(PH_FINAL);
      final_pass++;
      double mx = 0;
      int first_bad = nev;
      for (int i = 0; i < nev; ++i) {
        // a NaN residual fails (and is reported): every comparison with NaN is false
        if (!(rf[i] <= mx)) mx = rf[i];
        if (!(rf[i] <= o.tol) && first_bad == nev) first_bad = i;
      }
      if (st) { st->final_passes = final_pass; st->max_resid = mx; }
      if (first_bad == nev) { converged = true; break; }
      if (final_pass >= 3 || it >= o.max_outer) break;
      // tighten the C-space tolerance and re-open the failing pairs
      tolC *= 0.05;
      S.nlock = first_bad;
      if (prec != GEVP_PREC_FP64 && st) st->switches++;
      prec = GEVP_PREC_FP64;
      continue;
    }
    if (it >= o.max_outer) break;
    orth_val = -1.0;   // Q changes in this round
    // ---- filter the active columns
    int ma = m - S.nlock;
    double hi = S.upper;
    double lo = S.have_theta ? S.theta[m - 1] : S.a_est;
    double sc = S.have_theta ? std::min(S.theta[0], S.lower_est) : S.lower_est;
    if (!(lo > sc + 1e-3 * (hi - sc))) lo = sc + 0.5 * (hi - sc);
    if (!(hi > lo)) hi = lo + 1e-3 * S.normC + 1e-300;
    const int cap = std::max(o.deg_min, std::min(deg_cap, range_degree_cap(sc, lo, hi, prec, S.have_theta)));
    int deg = S.have_theta ? choose_degree(S, lo, hi, tolC, o.deg_min, cap) : std::min(cap, 10);
    const double pred = S.have_theta ? predicted_max_res(S, lo, hi, tolC, deg) : 0.0;
    double2* Yf;
    if (prec != GEVP_PREC_FP64) {
      if (S.have_theta) {
        // residual-corrected: the tensor cores filter the defect driven by R = W - Q Theta
        CK(filter_tc_apply_corrected(h->tc, n, ma, h->Q + S.nlock, ld, h->W + S.nlock, ld, h->theta + S.nlock,
                                     S.theta.data() + S.nlock, h->Y1, ld, deg, lo, hi, sc, nsplit,
                                     h->stream));
        if (st) st->flops_lowp += 8.0 * (double)n * n * ma * (deg - 1);
      } else {
        CK(filter_tc_apply(h->tc, n, ma, h->Q + S.nlock, ld, h->Y1, ld, deg, lo, hi, sc, nsplit, nullptr,
                           h->stream));
        if (st) st->flops_lowp += 8.0 * (double)n * n * ma * deg;
      }
      Yf = h->Y1;
    } else {
      Yf = filter_fp64(h, n, h->C, n, h->Q + S.nlock, ld, ma, deg, lo, hi, sc, h->Y1, h->Y2, ld);
      if (st) st->flops_fp64 += 8.0 * (double)n * n * ma * deg;
    }
    if (st) {
      st->filter_steps += deg;
      st->matvecs += (int64_t)deg * ma;
    }
    tm.mark(PH_FILTER);
    const uint64_t oseed = o.seed + 31ull * it + 7ull * prob_index;
    int pend = 0;
    TRY(orthonormalize(h, n, S.nlock, Yf, ld, ma, h->Q + S.nlock, ld, st, oseed, &pend));
    tm.mark(PH_ORTH);
    TRY(rayleigh_ritz(h, n, S.nlock, ma, h->C, n, o.refine_iters, st));
    // one status read per round: the Ritz values, residuals and the CholQR passes' pivots
    int orth_info[2] = {0, 0};
    TRY(sync_reads(h, {{h->theta + S.nlock, S.theta.data() + S.nlock, ma * sizeof(double)},
                       {h->res + S.nlock, S.res.data() + S.nlock, ma * sizeof(double)},
                       {h->info, orth_info, pend ? sizeof orth_info : 0}}));
    if (pend && (orth_info[0] != 0 || orth_info[1] != 0)) {
      // a CholQR pass met a non-positive pivot: the projection above used a bad basis.
      // Orthonormalise the (intact) filtered block again with the shifted fallback and
      // project again
      TRY(orthonormalize(h, n, S.nlock, Yf, ld, ma, h->Q + S.nlock, ld, st, oseed, nullptr, false));
      TRY(rayleigh_ritz(h, n, S.nlock, ma, h->C, n, o.refine_iters, st));
      TRY(sync_read2(h, h->theta + S.nlock, S.theta.data() + S.nlock, ma * sizeof(double), h->res + S.nlock,
                     S.res.data() + S.nlock, ma * sizeof(double)));
    }
    tm.mark(PH_RR);
    S.have_theta = true;
    if (st) st->outer_iters++;
    double mr = 0;
    for (int i = S.nlock; i < nev; ++i) mr = std::max(mr, S.res[i]);
    // precision switch: the low-precision filter has reached its floor (less than 4x
    // progress in a round where the Chebyshev factors promised more than 100x) -> FP64
    // for the rest of this problem. Slow progress that theory predicts (Ritz values close
    // to the damped interval) is no reason to switch: FP64 would not converge faster.
    // The prediction assumes settled Ritz values; while residuals are still large (the
    // first rounds of a cold start) it is no test of the filter's precision, so a stall
    // only counts below 1e-3 ||C|| for the FP32-class filter (its floor is near 1e-8) and
    // below 1e-1 ||C|| for BF16.
    const double stall_zone = (prec == GEVP_PREC_FP32 ? 1e-3 : 1e-1) * S.normC;
    if (prec != GEVP_PREC_FP64 && mr <= stall_zone && mr > 0.25 * prev_maxres &&
        (pred <= 0.0 || mr > 25.0 * pred)) {
      // The FP32-class filter's floor depends on the degree (its rounding is amplified
      // along the recurrence): first halve the degree cap, down to 16; BF16's floor does
      // not depend on it, so BF16 switches at once.
      if (prec == GEVP_PREC_FP32 && deg_cap > 16) {
        deg_cap = std::max(16, deg_cap / 2);
      } else {
        prec = GEVP_PREC_FP64;
        if (st) st->switches++;
      }
    }
    if (trace_on())
      std::fprintf(stderr, "gevp: problem %d round %d prec %d deg %d cap %d lo %.6g hi %.6g sc %.6g nlock %d maxres %.3e "
                   "pred %.3e zone %.3e\n", prob_index, it, prec, deg, cap, lo, hi, sc, S.nlock, mr, pred, stall_zone);
    prev_maxres = mr;
  }
  if (st) {
    if (orth_val < 0.0) {   // no final check of the current block (the round limit)
      orth_enqueue(h, n, nev);
      TRY(sync_read(h, h->partial, &orth_val, sizeof orth_val));
    }
    st->orth_err = orth_val;
  }
  CK(cudaMemcpyAsync(Lam_out, h->lam, nev * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(res_out, h->resf, nev * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (X_out) zcopy2d(n, nev, h->Xf, ld, X_out, ldx, h->stream);
  if (st) st->converged = converged ? 1 : 0;
  h->ozC_src = nullptr;   // C's digits are this problem's only
  return converged ? GEVP_OK : GEVP_ERR_NO_CONVERGENCE;
}

bool bad_ld(int64_t ld, int64_t cols) { return ld < cols || ld <= 0; }

// Standard form, spectral bounds and tensor-core planes of problem idx (matrix A) on the
// side stream into C2 / bounds2 / tc2, ordered after everything already enqueued on the
// main stream (which includes the last use of those buffers by the problem before). The
// kernels and seeds are those of the main path, so the results are identical.
gevp_status prefetch_problem(gevp_ctx* h, int64_t n, int m, const double2* A, int64_t lda, const gevp_opts& o,
                             int idx) {
  CK(cudaEventRecord(h->ev_main, h->stream));
  CK(cudaStreamWaitEvent(h->side, h->ev_main, 0));
  if (h->oz_slices > 0)
    TRY(reduce_emulated(h, 1, n, A, lda, h->C2, n, h->T2, h->side));
  else
    reduce_into_ws(n, h->Linv, A, lda, h->C2, n, h->T2, h->split2, h->split2_elems, h->side);
  z_to_c(n, n, h->C2, n, h->M32b, n, h->side);
  lanczos_bounds(n, h->M32b, n, o.lanczos_steps, m, o.seed + 7919ull * idx, h->lw2, h->bounds2, h->side);
  z_to_c(n, n, A, lda, h->M32b, n, h->side);
  lanczos_bounds(n, h->M32b, n, o.lanczos_steps, 0, o.seed + 104729ull * idx + 1, h->lw2, h->bounds2 + 8, h->side);
  CK(cudaMemcpyAsync(h->hb2, h->bounds2, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->side));
  if (o.filter_prec != GEVP_PREC_FP64) {
    CK(filter_tc_reserve(&h->tc2, n, m, h->side));
    CK(filter_tc_set_matrix(h->tc2, n, h->C2, n, o.filter_prec == GEVP_PREC_FP32 ? 3 : 1, h->side));
  }
  CK(cudaEventRecord(h->ev_side, h->side));
  return GEVP_OK;
}

// For the duration of a sequence solve: work on the internal high-priority stream (after
// the caller's stream), and on every exit hand back to the caller's stream, wait for the
// side stream and give the double-buffered standard form its original roles.
struct PipelineScope {
  gevp_ctx* h;
  cudaStream_t user;
  bool swapped = false;
  PipelineScope(gevp_ctx* hh) : h(hh), user(hh->stream) {
    cudaEventRecord(h->ev_user, user);
    cudaStreamWaitEvent(h->hi, h->ev_user, 0);
    h->stream = h->hi;
  }
  void swap_buffers() {
    std::swap(h->C, h->C2);
    std::swap(h->tc, h->tc2);
    swapped = !swapped;
  }
  ~PipelineScope() {
    cudaStreamSynchronize(h->side);
    cudaEventRecord(h->ev_user, h->stream);
    cudaStreamWaitEvent(user, h->ev_user, 0);
    h->stream = user;
    if (swapped) swap_buffers();
  }
};

}  // namespace

// ===================================================================== C ABI
extern "C" {

void gevp_default_opts(gevp_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->filter_prec = GEVP_PREC_FP64;
  o->tol = 1e-10;
  o->max_outer = 60;
  o->deg_min = 4;
  // filter steps are cheap next to a Rayleigh-Ritz round (an n x n x m FP64 product and
  // an m x m eigensolve); a cap of 48 gave the fewest rounds on the warm sequences, while
  // higher degrees make the guard columns of the filtered block nearly dependent
  o->deg_max = 48;
  o->nex = 0;
  o->seed = 10074400ull;
  o->b_fixed = 0;
  o->cold_start = 0;
  o->lanczos_steps = 32;
  o->refine_iters = 3;
  o->keep_all_X = 0;
  // the reduction's n^3 products emulated with 8 digits: FP64-class accuracy, about 17x
  // the FP64 pipe's rate at n = 2048
  o->reduce_slices = 8;
}

const char* gevp_status_string(gevp_status s) {
  int i = (int)s;
  if (i < 0 || i > 8) return "GEVP_UNKNOWN";
  return kStatusNames[i];
}

const char* gevp_version(void) { return "gevp-gb300 0.1 (sm_103a)"; }

const char* gevp_last_error(gevp_handle h) { return h ? h->err.c_str() : "null handle"; }

int64_t gevp_kernel_launches(gevp_handle h) { (void)h; return gevp::g_launches.load(); }

gevp_status gevp_create(gevp_handle* out, int device, void* stream) {
  if (!out) return GEVP_ERR_INVALID_ARG;
  *out = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return GEVP_ERR_CUDA;
  gevp_ctx* h = new gevp_ctx();
  h->device = device;
  h->stream = (cudaStream_t)stream;
  e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete h; return GEVP_ERR_CUDA; }
  *out = h;
  return GEVP_OK;
}

gevp_status gevp_destroy(gevp_handle h) {
  if (!h) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->hi) cudaStreamSynchronize(h->hi);
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->tc) gevp::filter_tc_release(h->tc);
  if (h->tc2) gevp::filter_tc_release(h->tc2);
  if (h->batch) gevp::batch_release(h->batch);
  if (h->parena) cudaFree(h->parena);
  if (h->vd2) cudaFree(h->vd2);
  if (h->dvbuf) cudaFree(h->dvbuf);
  for (int i = 0; i < 2; ++i)
    if (h->ozmem[i]) cudaFree(h->ozmem[i]);
  if (h->ozflags) cudaFree(h->ozflags);
  if (h->ozws) cudaFree(h->ozws);
  if (h->jidx) cudaFree(h->jidx);
  if (h->hb2) cudaFreeHost(h->hb2);
  for (cudaEvent_t e : {h->ev_main, h->ev_side, h->ev_user})
    if (e) cudaEventDestroy(e);
  if (h->hi) cudaStreamDestroy(h->hi);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->stage) cudaFree(h->stage);
  if (h->arena) cudaFree(h->arena);
  if (h->hbuf) cudaFreeHost(h->hbuf);
  for (auto e : h->evpool) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
  return GEVP_OK;
}

gevp_status gevp_set_stream(gevp_handle h, void* stream) {
  if (!h) return GEVP_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return GEVP_OK;
}

gevp_status gevp_reduce(gevp_handle h, int64_t n, const void* A, int64_t lda, const void* B, int64_t ldb, void* L,
                        int64_t ldl, void* C, int64_t ldc, int64_t* info) {
  if (!h || n < 0 || !info) return GEVP_ERR_INVALID_ARG;
  *info = 0;
  if (n == 0) return GEVP_OK;
  if (!A || !B || !L || !C || bad_ld(lda, n) || bad_ld(ldb, n) || bad_ld(ldl, n) || bad_ld(ldc, n))
    return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, n, 1));
  TRY(factor_B(h, n, (const double2*)B, ldb, info));
  TRY(reduce_into(h, n, (const double2*)A, lda, (double2*)C, ldc));
  zcopy2d(n, n, h->L, n, (double2*)L, ldl, h->stream);
  h->chol_valid = false;   // the caller's next solve refactors
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return GEVP_OK;
}

gevp_status gevp_reduce_update(gevp_handle h, int64_t n, const void* B, int64_t ldb, int reuse_factor,
                               const void* dA, int64_t ldda, int k, const int64_t* rows, void* C, int64_t ldc,
                               int slices, int64_t* info) {
  if (!h || n < 0 || k < 0 || !info || slices < 0 || slices > gevp::kOzSlicesMax) return GEVP_ERR_INVALID_ARG;
  *info = 0;
  if (n == 0) return GEVP_OK;
  if (!B || !C || bad_ld(ldb, n) || bad_ld(ldc, n)) return GEVP_ERR_INVALID_ARG;
  if (k > 0 && (!dA || !rows || bad_ld(ldda, n))) return GEVP_ERR_INVALID_ARG;
  if ((int64_t)5 * k > n) return GEVP_ERR_INVALID_ARG;
  {
    std::vector<char> seen((size_t)n, 0);
    for (int t = 0; t < k; ++t) {
      if (rows[t] < 0 || rows[t] >= n || seen[(size_t)rows[t]]) return GEVP_ERR_INVALID_ARG;
      seen[(size_t)rows[t]] = 1;
    }
  }
  if (k == 0) return GEVP_OK;
  if (slices > 0 && n > 30720) {
    h->err = "emulated product: n above 30720";
    return GEVP_ERR_UNSUPPORTED;
  }
  cudaSetDevice(h->device);
  if (slices > 0 && !gevp::oz_supported()) {
    h->err = "emulated FP64 products need an sm_103 device";
    return GEVP_ERR_UNSUPPORTED;
  }
  TRY(ensure(h, n, k));
  if (!(reuse_factor && h->chol_valid && h->upd_B == B && h->upd_n == n && h->upd_gen == h->chol_gen)) {
    h->upd_B = nullptr;
    TRY(factor_B(h, n, (const double2*)B, ldb, info));
    h->upd_B = B;
    h->upd_n = n;
    h->upd_gen = h->chol_gen;
  }
  if ((size_t)k > h->jidx_cap) {
    if (h->jidx) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->jidx);
    }
    h->jidx = nullptr;
    h->jidx_cap = 0;
    void* p = nullptr;
    CK(cudaMalloc(&p, (size_t)k * sizeof(int64_t)));
    h->jidx = (int64_t*)p;
    h->jidx_cap = (size_t)k;
  }
  CK(cudaMemcpyAsync(h->jidx, rows, (size_t)k * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));   // rows is pageable host memory of the caller
  // scratch in T (n x n): UV = [U V] and VU = [V U] (n x 2k each), R = rows J of dA (k x n);
  // R_JJ (k x k) in G
  const int64_t k2 = 2 * (int64_t)k;
  double2* UV = h->T;
  double2* VU = h->T + n * k2;
  double2* R = h->T + 2 * n * k2;
  double2* RJJ = h->G;
  cudaStream_t s = h->stream;
  gather_cols(n, k, h->Linv, n, h->jidx, UV, k2, s);                       // U = L^-1 E_J
  gather_rows(k, n, (const double2*)dA, ldda, h->jidx, R, n, s);          // R = E_J^T dA
  gather_cols(k, k, R, n, h->jidx, RJJ, k, s);                             // R_JJ
  const int keep = h->oz_slices;
  h->oz_slices = slices;
  gevp_status st = GEVP_OK;
  if (slices > 0) {
    // W = L^-1 R^H (L^-1 rows, lower; columns of R^H = conjugated rows of R), emulated
    const int S = slices;
    const int nn = (int)n;
    const size_t bA = gevp::oz_operand_bytes(nn, nn, S, 2);
    st = oz_reserve(h, 0, oz_main_bytes(n, S));
    if (st == GEVP_OK && (h->oz_l_gen != h->chol_gen || h->oz_l_S != S)) {
      char* mem = h->ozmem[0];
      if (gevp::oz_split(h->ozLA, mem, nn, nn, h->Linv, n, 0, 2, S, 2, h->ozflags + 1, s) != cudaSuccess ||
          gevp::oz_split(h->ozLB, mem + bA, nn, nn, h->Linv, n, 1, 2, S, 3, h->ozflags + 1, s) != cudaSuccess)
        st = cuda_fail(h, cudaGetLastError(), "oz_split");
      h->oz_l_gen = h->chol_gen;
      h->oz_l_S = S;
    }
    if (st == GEVP_OK &&
        (gevp::oz_split(h->ozR, oz_region(h, n, 2), k, nn, R, n, 1, 0, S, 3, h->ozflags + 1, s) != cudaSuccess ||
         gevp::oz_gemm(h->ozLA, h->ozR, 1, 0, UV + k, k2, h->ozflags, s, nullptr, h->ozws, h->ozws_doubles) !=
             cudaSuccess))
      st = cuda_fail(h, cudaGetLastError(), "oz_gemm");
  } else {
    ZgemmArgs w = zg((int)n, k, (int)n, h->Linv, n, 0, R, n, 1, UV + k, k2);
    w.triA = 1;
    zgemm(w, h->split, h->split_elems, s);
  }
  if (st == GEVP_OK) {
    // V = W - U R_JJ / 2 (in place over W)
    ZgemmArgs v = zg((int)n, k, k, UV, k2, 0, RJJ, k, 0, UV + k, k2, -0.5);
    v.Cin = UV + k; v.ldc = k2; v.beta = 1.0;
    zgemm(v, h->split, h->split_elems, s);
    zcopy2d(n, k, UV + k, k2, VU, k2, s);
    zcopy2d(n, k, UV, k2, VU + k, k2, s);
    // C += [U V] [V U]^H = U V^H + V U^H, lower triangle, then its Hermitian completion
    if (slices > 0) {
      const int nn = (int)n;
      // [U V] rows in the T/C region, the conjugated rows of [V U] from the A region on
      // (up to three regions' room: the cached digits of B and of L^-H are invalidated)
      h->ozB_src = nullptr;
      h->ozB_gen = -1;
      h->ozLH_gen = -1;
      if (gevp::oz_split(h->ozUV, oz_region(h, n, 3), nn, (int)k2, UV, k2, 0, 0, slices, 2, h->ozflags + 1, s) !=
              cudaSuccess ||
          gevp::oz_split(h->ozVU, oz_region(h, n, 4), nn, (int)k2, VU, k2, 1, 0, slices, 3, h->ozflags + 1, s) !=
              cudaSuccess ||
          gevp::oz_gemm(h->ozUV, h->ozVU, 0, 0, h->C, n, h->ozflags, s) != cudaSuccess)
        st = cuda_fail(h, cudaGetLastError(), "oz_gemm");
      if (st == GEVP_OK) add_lower_herm(n, (double2*)C, ldc, h->C, n, s);
    } else {
      ZgemmArgs u = zg((int)n, (int)n, (int)k2, UV, k2, 0, VU, k2, 1, (double2*)C, ldc);
      u.Cin = (const double2*)C; u.ldc = ldc; u.beta = 1.0;
      u.triD = 1;
      zgemm(u, h->split, h->split_elems, s);
      hermitize_lower(n, (double2*)C, ldc, s);
    }
  }
  h->oz_slices = keep;
  if (st != GEVP_OK) return st;
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (slices > 0) TRY(oz_check(h));
  return GEVP_OK;
}

gevp_status gevp_solve_sequence(gevp_handle h, int nprob, int64_t n, const void* const* A, int64_t lda,
                                const void* const* B, int64_t ldb, int nev, const void* X_prev, int64_t ldxp,
                                int kprev, const gevp_opts* opts, double* Lambda, void* X, int64_t ldx,
                                double* resid, gevp_stats* stats) {
  if (!h || nprob < 0 || n < 0 || nev < 0) return GEVP_ERR_INVALID_ARG;
  if (nprob == 0 || n == 0 || nev == 0) return GEVP_OK;
  gevp_opts o;
  if (opts) o = *opts; else gevp_default_opts(&o);
  // at least two guard vectors: with none, the nev-th Ritz value sits at the edge of the
  // damped interval and its convergence factor tends to one
  int m = nev + std::max(2, o.nex);
  if (m > n) m = (int)n;
  if (nev > n || !A || !B || !Lambda || !resid || bad_ld(lda, n) || bad_ld(ldb, n)) return GEVP_ERR_INVALID_ARG;
  if (X && bad_ld(ldx, nev)) return GEVP_ERR_INVALID_ARG;
  if (X_prev && (kprev < 1 || kprev > m || bad_ld(ldxp, kprev))) return GEVP_ERR_INVALID_ARG;
  if (m > 1024) { h->err = "block width nev + nex above 1024"; return GEVP_ERR_UNSUPPORTED; }
  if (o.refine_iters < 1) o.refine_iters = 1;
  if (o.filter_prec < 0 || o.filter_prec > 2) return GEVP_ERR_INVALID_ARG;
  if (o.filter_prec != GEVP_PREC_FP64 && !tc_filter_supported()) {
    h->err = "tensor-core filter needs an sm_103 device";
    return GEVP_ERR_UNSUPPORTED;
  }
  if (o.deg_min < 1) o.deg_min = 1;
  if (o.deg_max < o.deg_min) o.deg_max = o.deg_min;
  if (o.lanczos_steps < 4) o.lanczos_steps = 4;
  if (o.reduce_slices < 0 || o.reduce_slices > gevp::kOzSlicesMax) return GEVP_ERR_INVALID_ARG;
  if (o.reduce_slices > 0 && !gevp::oz_supported()) {
    h->err = "emulated FP64 products need an sm_103 device";
    return GEVP_ERR_UNSUPPORTED;
  }
  if (o.reduce_slices > 0 && n > 30720) {
    h->err = "emulated product: n above 30720";
    return GEVP_ERR_UNSUPPORTED;
  }
  for (int l = 0; l < nprob; ++l)
    if (!A[l] || !B[l]) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  // the emulated products serve this solve only (the per-step entry points stay FP64)
  struct OzScope {
    gevp_ctx* h;
    ~OzScope() { h->oz_slices = 0; }
  } oz_scope{h};
  h->oz_slices = o.reduce_slices;
  TRY(ensure(h, n, m));
  TRY(ensure_pipeline(h));
  PipelineScope pipe(h);
  const int64_t ld = h->cap_m;
  // input sanity: NaN/Inf in any A or in B
  CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  for (int l = 0; l < nprob; ++l) {
    check_finite(n, n, (const double2*)A[l], lda, h->flag, h->stream);
    if (l == 0 || B[l] != B[l - 1]) check_finite(n, n, (const double2*)B[l], ldb, h->flag, h->stream);
  }
  int bad = 0;
  TRY(sync_read(h, h->flag, &bad, sizeof(int)));
  if (bad) { h->err = "NaN or Inf in an input matrix"; return GEVP_ERR_INVALID_VALUE; }

  gevp_status overall = GEVP_OK;
  bool warm_ok = false;   // Q holds a usable start block for this n, m
  bool have_pre = false;  // C2 / bounds2 / tc2 hold problem l's standard form
  int64_t cold_mv = -1;   // filter matvecs of the latest cold-started problem
  int flat = 0;           // consecutive warm problems that saved nothing over it
  bool refresh = false;   // the next problem starts cold
  for (int l = 0; l < nprob; ++l) {
    Timer tm(h);
    tm.start();
    gevp_stats local{};
    gevp_stats* st = stats ? &stats[l] : &local;
    std::memset(st, 0, sizeof(*st));
    const double2* Al = (const double2*)A[l];
    const double2* Bl = (const double2*)B[l];
    bool same_B = (l > 0) && (o.b_fixed || B[l] == B[l - 1]) && h->chol_valid;
    bool refactor = !same_B;
    if (refactor) {
      // keep the previous eigenvector block in the original space for the warm start
      if (warm_ok && h->chol_valid) {
        ZgemmArgs x = zg((int)n, m, (int)n, h->Linv, n, 1, h->Q, ld, 0, h->Xf, ld);
        x.triA = 2;
        zgemm(x, h->split, h->split_elems, h->stream);
      }
      int64_t info = 0;
      gevp_status s = factor_B(h, n, Bl, ldb, &info);
      if (s != GEVP_OK) return s;
      tm.mark(PH_CHOL);
      if (warm_ok) {
        // Y0 = L^H X_prev_block, then orthonormalise
        ZgemmArgs y = zg((int)n, m, (int)n, h->L, n, 1, h->Xf, ld, 0, h->Y1, ld);
        y.triA = 2;
        zgemm(y, h->split, h->split_elems, h->stream);
      }
    }
    double pre_hb[16];
    const bool used_pre = have_pre;
    if (have_pre) {
      // built on the side stream while the previous problem was being solved
      CK(cudaStreamWaitEvent(h->stream, h->ev_side, 0));
      CK(cudaEventSynchronize(h->ev_side));
      std::memcpy(pre_hb, h->hb2, 16 * sizeof(double));
      pipe.swap_buffers();
      have_pre = false;
    } else {
      TRY(reduce_into(h, n, Al, lda, h->C, n));
    }
    st->flops_fp64 += 4.0 * (double)n * n * n;
    tm.mark(PH_REDUCE);
    // the next problem's standard form overlaps with this problem's solve (same B only)
    if (l + 1 < nprob && (o.b_fixed || B[l + 1] == B[l])) {
      TRY(prefetch_problem(h, n, m, (const double2*)A[l + 1], lda, o, l + 1));
      have_pre = true;
    }
    bool warm = false;
    if (!o.cold_start && !refresh) {
      if (l == 0 && X_prev) {
        // seed from the caller's vectors: Y0[:, :kprev] = L^H X_prev, rest random
        zrandn(n, m, h->Y1, ld, o.seed + 17, h->stream);
        ZgemmArgs y = zg((int)n, kprev, (int)n, h->L, n, 1, (const double2*)X_prev, ldxp, 0, h->Y1, ld);
        y.triA = 2;
        zgemm(y, h->split, h->split_elems, h->stream);
        TRY(orthonormalize(h, n, 0, h->Y1, ld, m, h->Q, ld, st));
        warm = true;
      } else if (warm_ok) {
        if (refactor) TRY(orthonormalize(h, n, 0, h->Y1, ld, m, h->Q, ld, st));
        warm = true;
      }
    }
    gevp_status s = solve_one(h, n, Al, lda, Bl, ldb, nev, m, warm, o, l, tm,
                              st, Lambda + (int64_t)l * nev,
                              X ? ((o.keep_all_X ? (double2*)X + (int64_t)l * n * ldx
                                                 : (l == nprob - 1 ? (double2*)X : nullptr)))
                                : nullptr,
                              ldx, resid + (int64_t)l * nev, used_pre ? pre_hb : nullptr,
                              used_pre && o.filter_prec != GEVP_PREC_FP64);
    if (s != GEVP_OK && s != GEVP_ERR_NO_CONVERGENCE) return s;
    if (s == GEVP_ERR_NO_CONVERGENCE) overall = s;
    warm_ok = true;
    st->cold = warm ? 0 : 1;
    if (o.refresh_window > 0) {
      // refresh: warm starts that no longer save filter work over the latest cold solve
      if (!warm) {
        cold_mv = st->matvecs;
        flat = 0;
        refresh = false;
      } else if (cold_mv >= 0 && st->matvecs >= cold_mv) {
        if (++flat >= o.refresh_window) refresh = true;
      } else {
        flat = 0;
      }
    }
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    tm.mark(PH_FINAL);
    CK(cudaStreamSynchronize(h->stream));
    tm.resolve();
    st->ms_chol = tm.ms[PH_CHOL];
    st->ms_reduce = tm.ms[PH_REDUCE];
    st->ms_bounds = tm.ms[PH_BOUNDS];
    st->ms_filter = tm.ms[PH_FILTER];
    st->ms_orth = tm.ms[PH_ORTH];
    st->ms_rr = tm.ms[PH_RR];
    st->ms_resid = tm.ms[PH_RESID];
    st->ms_final = tm.ms[PH_FINAL];
    float tot = 0;
    for (int p = 0; p < PH_N; ++p) tot += tm.ms[p];
    st->ms_total = tot;
  }
  if (h->oz_slices > 0) TRY(oz_check(h));
  if (overall != GEVP_OK) h->err = "some residual stayed above tol";
  return overall;
}

gevp_status gevp_solve_sequence_host(gevp_handle h, int nprob, int64_t n, const void* const* A, int64_t lda,
                                     const void* const* B, int64_t ldb, int nev, const gevp_opts* opts,
                                     double* Lambda, void* X, int64_t ldx, double* resid, gevp_stats* stats) {
  if (!h || nprob < 0 || n < 0 || nev < 0) return GEVP_ERR_INVALID_ARG;
  if (nprob == 0 || n == 0 || nev == 0) return GEVP_OK;
  if (!A || !B || !Lambda || !resid || bad_ld(lda, n) || bad_ld(ldb, n) || (X && bad_ld(ldx, nev)))
    return GEVP_ERR_INVALID_ARG;
  for (int l = 0; l < nprob; ++l)
    if (!A[l] || !B[l]) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  gevp_opts o;
  if (opts) o = *opts; else gevp_default_opts(&o);
  // distinct B matrices (consecutive equal pointers share one device copy)
  std::vector<int> bslot(nprob);
  int nb = 0;
  for (int l = 0; l < nprob; ++l) bslot[l] = (l > 0 && B[l] == B[l - 1]) ? bslot[l - 1] : nb++;
  const size_t mat = (size_t)n * n * sizeof(double2);
  const size_t out_x = X ? (size_t)(o.keep_all_X ? nprob : 1) * n * nev * sizeof(double2) : 0;
  const size_t need = (size_t)(nprob + nb) * mat + 2 * (size_t)nprob * nev * sizeof(double) + out_x + 4096;
  if (need > h->stage_bytes) {
    if (h->stage) { cudaStreamSynchronize(h->stream); cudaFree(h->stage); h->stage = nullptr; }
    CK(cudaMalloc(&h->stage, need));
    h->stage_bytes = need;
  }
  char* p = (char*)h->stage;
  std::vector<const void*> dA(nprob), dB(nprob), dBs(nb);
  // host -> device: one copy per matrix, rows packed to ld = n
  for (int l = 0; l < nprob; ++l) {
    dA[l] = p;
    CK(cudaMemcpy2DAsync(p, n * sizeof(double2), A[l], lda * sizeof(double2), n * sizeof(double2), n,
                         cudaMemcpyHostToDevice, h->stream));
    p += mat;
  }
  for (int l = 0; l < nprob; ++l) {
    if (l == 0 || bslot[l] != bslot[l - 1]) {
      dBs[bslot[l]] = p;
      CK(cudaMemcpy2DAsync(p, n * sizeof(double2), B[l], ldb * sizeof(double2), n * sizeof(double2), n,
                           cudaMemcpyHostToDevice, h->stream));
      p += mat;
    }
    dB[l] = dBs[bslot[l]];
  }
  double* dLam = (double*)p;
  p += (size_t)nprob * nev * sizeof(double);
  double* dRes = (double*)p;
  p += (size_t)nprob * nev * sizeof(double);
  double2* dX = X ? (double2*)p : nullptr;
  gevp_status s = gevp_solve_sequence(h, nprob, n, dA.data(), n, dB.data(), n, nev, nullptr, 0, 0, &o, dLam, dX, nev,
                                      dRes, stats);
  if (s != GEVP_OK && s != GEVP_ERR_NO_CONVERGENCE) return s;
  CK(cudaMemcpyAsync(Lambda, dLam, (size_t)nprob * nev * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(resid, dRes, (size_t)nprob * nev * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (X) {
    int blocks = o.keep_all_X ? nprob : 1;
    for (int b = 0; b < blocks; ++b)
      CK(cudaMemcpy2DAsync((double2*)X + (size_t)b * n * ldx, ldx * sizeof(double2), dX + (size_t)b * n * nev,
                           nev * sizeof(double2), nev * sizeof(double2), n, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return s;
}

gevp_status gevp_chebyshev_filter(gevp_handle h, int64_t n, const void* C, int64_t ldc, void* Y, int64_t ldy, int m,
                                  int degree, double lo, double hi, double s, int prec) {
  if (!h || n < 0 || m < 0 || degree < 1 || !(hi > lo) || !(lo > s)) return GEVP_ERR_INVALID_ARG;
  if (n == 0 || m == 0) return GEVP_OK;
  if (!C || !Y || bad_ld(ldc, n) || bad_ld(ldy, m)) return GEVP_ERR_INVALID_ARG;
  if (prec < 0 || prec > 2) return GEVP_ERR_UNSUPPORTED;
  cudaSetDevice(h->device);
  TRY(ensure(h, n, m));
  const int64_t ld = h->cap_m;
  if (prec != GEVP_PREC_FP64) {
    if (!tc_filter_supported()) return GEVP_ERR_UNSUPPORTED;
    const int nsplit = (prec == GEVP_PREC_FP32) ? 3 : 1;
    CK(filter_tc_reserve(&h->tc, n, m, h->stream));
    CK(filter_tc_set_matrix(h->tc, n, (const double2*)C, ldc, nsplit, h->stream));
    int err = 0;
    CK(filter_tc_apply(h->tc, n, m, (const double2*)Y, ldy, (double2*)Y, ldy, degree, lo, hi, s, nsplit, &err,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (err) { h->err = "tensor-core filter: a bounded wait expired"; return GEVP_ERR_TIMEOUT; }
    return GEVP_OK;
  }
  double2* out = filter_fp64(h, n, (const double2*)C, ldc, (const double2*)Y, ldy, m, degree, lo, hi, s, h->Y1,
                             h->Y2, ld);
  zcopy2d(n, m, out, ld, (double2*)Y, ldy, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return GEVP_OK;
}

gevp_status gevp_matmul_tc(gevp_handle h, int64_t n, int m, const void* C, int64_t ldc, const void* Y, int64_t ldy,
                           void* D, int64_t ldd) {
  if (!h || n < 0 || m < 0) return GEVP_ERR_INVALID_ARG;
  if (n == 0 || m == 0) return GEVP_OK;
  if (!C || !Y || !D || bad_ld(ldc, n) || bad_ld(ldy, m) || bad_ld(ldd, m)) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  if (!tc_filter_supported()) return GEVP_ERR_UNSUPPORTED;
  CK(filter_tc_reserve(&h->tc, n, m, h->stream));
  CK(filter_tc_set_matrix(h->tc, n, (const double2*)C, ldc, 1, h->stream));
  int err = 0;
  CK(filter_tc_product(h->tc, n, m, (const double2*)Y, ldy, (double2*)D, ldd, 1, &err, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  if (err) { h->err = "tensor-core product: a bounded wait expired"; return GEVP_ERR_TIMEOUT; }
  return GEVP_OK;
}

gevp_status gevp_cholqr2(gevp_handle h, int64_t n, int m, void* Y, int64_t ldy, void* R, int64_t ldr) {
  if (!h || n < 0 || m < 0 || m > n) return GEVP_ERR_INVALID_ARG;
  if (n == 0 || m == 0) return GEVP_OK;
  if (!Y || bad_ld(ldy, m) || (R && bad_ld(ldr, m))) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, n, m));
  const int64_t ld = h->cap_m;
  h->have_prev = false;
  zcopy2d(n, m, (const double2*)Y, ldy, h->Y2, ld, h->stream);
  zcopy2d(n, m, (const double2*)Y, ldy, h->Wt, ld, h->stream);   // keep the input for R
  TRY(orthonormalize(h, n, 0, h->Y2, ld, m, h->Y1, ld, nullptr));
  zcopy2d(n, m, h->Y1, ld, (double2*)Y, ldy, h->stream);
  if (R) {
    // R = Q^H Y_in: upper triangular up to rounding; the strict lower part is set to 0
    ZgemmArgs r = zg(m, m, (int)n, h->Y1, ld, 1, h->Wt, ld, 0, (double2*)R, ldr);
    zgemm(r, h->split, h->split_elems, h->stream);
    zero_lower(m, (double2*)R, ldr, h->stream);
  }
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return GEVP_OK;
}

gevp_status gevp_rayleigh_ritz(gevp_handle h, int64_t n, int m, const void* C, int64_t ldc, void* Q, int64_t ldq,
                               void* W, int64_t ldw, double* theta, double* res) {
  if (!h || n < 0 || m < 0 || m > n) return GEVP_ERR_INVALID_ARG;
  if (n == 0 || m == 0) return GEVP_OK;
  if (!C || !Q || !W || !theta || !res || bad_ld(ldc, n) || bad_ld(ldq, m) || bad_ld(ldw, m))
    return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, n, m));
  const int64_t ld = h->cap_m;
  h->have_prev = false;
  zcopy2d(n, m, (const double2*)Q, ldq, h->Q, ld, h->stream);
  TRY(rayleigh_ritz(h, n, 0, m, (const double2*)C, ldc, 3, nullptr));
  zcopy2d(n, m, h->Q, ld, (double2*)Q, ldq, h->stream);
  zcopy2d(n, m, h->W, ld, (double2*)W, ldw, h->stream);
  CK(cudaMemcpyAsync(theta, h->theta, m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(res, h->res, m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return GEVP_OK;
}

gevp_status gevp_heev_small(gevp_handle h, int m, const void* G, int64_t ldg, double* theta, void* Z, int64_t ldz) {
  if (!h || m < 0 || m > 1024) return GEVP_ERR_INVALID_ARG;
  if (m == 0) return GEVP_OK;
  if (!G || !theta || !Z || bad_ld(ldg, m) || bad_ld(ldz, m)) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, std::max<int64_t>(m, h->cap_n), m));
  heev_small(m, (const double2*)G, ldg, theta, (double2*)Z, ldz, h->hw, 3, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return GEVP_OK;
}

gevp_status gevp_spectral_bounds(gevp_handle h, int64_t n, const void* C, int64_t ldc, int k, int count,
                                 double* out) {
  if (!h || n <= 0 || !C || !out || bad_ld(ldc, n) || k < 1) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, n, 1));
  TRY(lanczos(h, n, (const double2*)C, ldc, k, count, 10074400ull, out));
  return GEVP_OK;
}

gevp_status gevp_band_energy(gevp_handle h, int nprob, int nev, const double* Lambda, double* E) {
  if (!h || nprob < 0 || nev < 0) return GEVP_ERR_INVALID_ARG;
  if (nprob == 0) return GEVP_OK;
  if (!E || (nev > 0 && !Lambda)) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  gevp::band_energy(nprob, nev, Lambda, E, h->stream);
  CK(cudaGetLastError());
  return GEVP_OK;
}

gevp_status gevp_energy_backward(gevp_handle h, int64_t n, int nev, const void* X, int64_t ldx, const double* Lambda,
                                 const double* gE, void* GA, void* GB, int64_t ldg) {
  if (!h || n < 0 || nev < 0 || nev > n) return GEVP_ERR_INVALID_ARG;
  if (n == 0) return GEVP_OK;
  if (!X || !Lambda || !gE || !GA || !GB || bad_ld(ldx, nev) || bad_ld(ldg, n)) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, n, std::max(nev, 1)));
  gevp::energy_backward_ws(n, nev, (const double2*)X, ldx, Lambda, gE, (double2*)GA, (double2*)GB, ldg, h->T,
                           h->split, h->split_elems, h->stream);
  CK(cudaGetLastError());
  return GEVP_OK;
}

gevp_status gevp_matrix_variation(gevp_handle h, int64_t n, const void* A_new, int64_t lda, const void* A_old,
                                  int64_t ldb, int nthr, const double* p_t, double* delta, int64_t* counts,
                                  void* mask) {
  if (!h || n < 0 || !delta || nthr < 0 || nthr > variation_max_thresholds()) return GEVP_ERR_INVALID_ARG;
  if (nthr > 0 && (!p_t || !counts)) return GEVP_ERR_INVALID_ARG;
  *delta = 0.0;
  for (int t = 0; t < nthr; ++t) counts[t] = 0;
  if (n == 0) return GEVP_OK;
  if (!A_new || !A_old || bad_ld(lda, n) || bad_ld(ldb, n)) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, std::max<int64_t>(1, h->cap_n), std::max(1, h->cap_m)));
  unsigned long long* ws = h->vscratch;
  double* p_dev = (double*)(ws + 32);
  const size_t need = (size_t)n * n * sizeof(unsigned long long);
  if (need > h->vd2_bytes) {
    if (h->vd2) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->vd2);
      h->vd2 = nullptr;
      h->vd2_bytes = 0;
    }
    void* p = nullptr;
    CK(cudaMalloc(&p, need));
    h->vd2 = (unsigned long long*)p;
    h->vd2_bytes = need;
  }
  CK(cudaMemsetAsync(ws, 0, 32 * sizeof(unsigned long long), h->stream));
  if (nthr > 0) CK(cudaMemcpyAsync(p_dev, p_t, nthr * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  gevp::matrix_variation(n, (const double2*)A_new, lda, (const double2*)A_old, ldb, nthr, p_dev, ws, h->vd2,
                         (uint8_t*)mask, h->stream);
  unsigned long long out[32];
  TRY(sync_read(h, ws, out, sizeof(out)));
  if (out[1] != 0) {
    h->err = "NaN in a matrix difference";
    return GEVP_ERR_INVALID_VALUE;
  }
  double dmax2;
  std::memcpy(&dmax2, &out[0], sizeof(double));
  *delta = std::sqrt(dmax2);
  for (int t = 0; t < nthr; ++t) counts[t] = (int64_t)out[2 + t];
  return GEVP_OK;
}

gevp_status gevp_deviation_angles(gevp_handle h, int64_t n, int k_old, int k_new, const void* X_old, int64_t ldo,
                                  const void* X_new, int64_t ldn, const void* B, int64_t ldb, const double* lam_old,
                                  const double* lam_new, double window, double* cosines, int64_t ldc, int64_t* perm,
                                  double* theta, double* cost, int64_t* n_outside) {
  if (!h || n < 0 || k_old < 0 || k_new < k_old || !(window >= 0.0)) return GEVP_ERR_INVALID_ARG;
  const bool windowed = std::isfinite(window);
  if (windowed && (!lam_old || !lam_new)) return GEVP_ERR_INVALID_ARG;
  if (cost) *cost = 0.0;
  if (n_outside) *n_outside = 0;
  if (k_old == 0) return GEVP_OK;
  if (n == 0 || !X_old || !X_new || bad_ld(ldo, k_old) || bad_ld(ldn, k_new)) return GEVP_ERR_INVALID_ARG;
  if ((B && bad_ld(ldb, n)) || (cosines && bad_ld(ldc, k_new))) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  TRY(ensure(h, std::max<int64_t>(1, h->cap_n), std::max(1, h->cap_m)));
  const int64_t ko = k_old, kn = k_new;
  const int slices = gevp::deviation_norm_slices(n);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t wbytes = B ? up((size_t)n * (ko + kn) * sizeof(double2)) : 0;
  const size_t obytes = up((size_t)ko * kn * sizeof(double2));
  const size_t cbytes = up((size_t)ko * kn * sizeof(double));
  const size_t pbytes = up((size_t)slices * kn * sizeof(double));
  const size_t nbytes = up((size_t)(ko + kn) * sizeof(double));
  const size_t need = wbytes + obytes + cbytes + pbytes + nbytes + 256;
  if (need > h->dvbuf_bytes) {
    if (h->dvbuf) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->dvbuf);
      h->dvbuf = nullptr;
      h->dvbuf_bytes = 0;
    }
    void* p = nullptr;
    CK(cudaMalloc(&p, need));
    h->dvbuf = (char*)p;
    h->dvbuf_bytes = need;
  }
  char* q = h->dvbuf;
  double2* Wo = (double2*)q;
  double2* Wn = Wo + (size_t)n * ko;
  q += wbytes;
  double2* O = (double2*)q;
  q += obytes;
  double* cosb = (double*)q;
  q += cbytes;
  double* part = (double*)q;
  q += pbytes;
  double* nrm = (double*)q;
  q += nbytes;
  int* bad = (int*)q;
  const double2* Xo = (const double2*)X_old;
  const double2* Xn = (const double2*)X_new;
  const double2* Wop = Xo;
  const double2* Wnp = Xn;
  int64_t ldwo = ldo, ldwn = ldn;
  if (B) {
    // W = B X for both blocks (FP64 complex GEMMs); with B = I the blocks are their own W
    gevp::zgemm(gevp::zg((int)n, (int)ko, (int)n, (const double2*)B, ldb, 0, Xo, ldo, 0, Wo, ko), h->split,
                h->split_elems, h->stream);
    gevp::zgemm(gevp::zg((int)n, (int)kn, (int)n, (const double2*)B, ldb, 0, Xn, ldn, 0, Wn, kn), h->split,
                h->split_elems, h->stream);
    Wop = Wo;
    Wnp = Wn;
    ldwo = ko;
    ldwn = kn;
  }
  // O = X_old^H (B X_new), the B-norms, the cosine table
  gevp::zgemm(gevp::zg((int)ko, (int)kn, (int)n, Xo, ldo, 1, Wnp, ldwn, 0, O, kn), h->split, h->split_elems,
              h->stream);
  gevp::column_bnorms(n, (int)ko, Xo, ldo, Wop, ldwo, part, nrm, h->stream);
  gevp::column_bnorms(n, (int)kn, Xn, ldn, Wnp, ldwn, part, nrm + ko, h->stream);
  CK(cudaMemsetAsync(bad, 0, sizeof(int), h->stream));
  gevp::overlap_cosines((int)ko, (int)kn, O, kn, nrm, nrm + ko, cosb, kn, bad, h->stream);
  CK(cudaGetLastError());
  if (cosines)
    CK(cudaMemcpy2DAsync(cosines, ldc * sizeof(double), cosb, kn * sizeof(double), kn * sizeof(double), ko,
                         cudaMemcpyDeviceToDevice, h->stream));
  int hbad = 0;
  TRY(sync_read(h, bad, &hbad, sizeof(int)));
  if (hbad) {
    h->err = "an eigenvector has a B-norm that is zero or not finite";
    return GEVP_ERR_INVALID_VALUE;
  }
  if (!perm && !theta && !cost && !n_outside) return GEVP_OK;
  std::vector<double> c((size_t)ko * kn);
  TRY(sync_read(h, cosb, c.data(), c.size() * sizeof(double)));
  auto outside = [&](int64_t i, int64_t j) { return windowed && std::fabs(lam_old[i] - lam_new[j]) > window; };
  std::vector<int64_t> match(ko);
  if (perm) {
    // a pair outside the window costs more than any assignment of pairs inside it
    const double far = (double)ko + 1.0;
    std::vector<double> w((size_t)ko * kn);
    for (int64_t i = 0; i < ko; ++i)
      for (int64_t j = 0; j < kn; ++j) w[i * kn + j] = outside(i, j) ? far : 1.0 - c[i * kn + j];
    gevp::assign_min_cost((int)ko, (int)kn, w.data(), match.data());
    for (int64_t i = 0; i < ko; ++i) perm[i] = match[i];
  } else {
    for (int64_t i = 0; i < ko; ++i) match[i] = i;
  }
  double tot = 0.0;
  int64_t nout = 0;
  const double half_pi = 2.0 * std::atan(1.0);
  for (int64_t i = 0; i < ko; ++i) {
    const double ci = c[i * kn + match[i]];
    if (theta) theta[i] = std::acos(ci) / half_pi;
    if (outside(i, match[i])) ++nout;
    else tot += 1.0 - ci;
  }
  if (cost) *cost = tot;
  if (n_outside) *n_outside = nout;
  return GEVP_OK;
}

gevp_status gevp_assign_min_cost(int ko, int kn, const double* cost, int64_t* perm) {
  if (ko < 0 || kn < ko || (ko > 0 && (!cost || !perm))) return GEVP_ERR_INVALID_ARG;
  for (int64_t e = 0; e < (int64_t)ko * kn; ++e)
    if (!std::isfinite(cost[e])) return GEVP_ERR_INVALID_ARG;
  if (ko > 0) gevp::assign_min_cost(ko, kn, cost, perm);
  return GEVP_OK;
}

gevp_status gevp_zgemm_emulated(gevp_handle h, int opA, int opB, int M, int N, int K, const void* A, int64_t lda,
                                const void* B, int64_t ldb, void* D, int64_t ldd, int slices) {
  if (!h || M < 0 || N < 0 || K < 0 || slices < 1 || slices > gevp::kOzSlicesMax) return GEVP_ERR_INVALID_ARG;
  if ((opA != 0 && opA != 1) || (opB != 0 && opB != 1)) return GEVP_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return GEVP_OK;
  if (!D || bad_ld(ldd, N)) return GEVP_ERR_INVALID_ARG;
  if (K > 0 && (!A || !B || bad_ld(lda, opA ? M : K) || bad_ld(ldb, opB ? K : N))) return GEVP_ERR_INVALID_ARG;
  if (K > 30720) {
    h->err = "emulated product: K above 30720";
    return GEVP_ERR_UNSUPPORTED;
  }
  cudaSetDevice(h->device);
  if (!gevp::oz_supported()) {
    h->err = "emulated FP64 products need an sm_103 device";
    return GEVP_ERR_UNSUPPORTED;
  }
  if (K == 0) {
    CK(cudaMemset2DAsync(D, ldd * sizeof(double2), 0, (size_t)N * sizeof(double2), M, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GEVP_OK;
  }
  const size_t bA = gevp::oz_operand_bytes(M, K, slices, 2), bB = gevp::oz_operand_bytes(N, K, slices, 3);
  TRY(oz_reserve(h, 1, bA + bB));
  gevp::OzOperand a, b;
  // rows of op(A): rows of A, or conjugated columns; columns of op(B): columns of B, or
  // conjugated rows
  CK(gevp::oz_split(a, h->ozmem[1], M, K, (const double2*)A, lda, opA, 0, slices, 2, h->ozflags + 1, h->stream,
                    opA == 1));
  CK(gevp::oz_split(b, h->ozmem[1] + bA, N, K, (const double2*)B, ldb, opB, 0, slices, 3, h->ozflags + 1,
                    h->stream, opB == 0));
  CK(gevp::oz_gemm(a, b, 0, 0, (double2*)D, ldd, h->ozflags, h->stream));
  return oz_check(h);
}

gevp_status gevp_reduce_emulated(gevp_handle h, int64_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                                 void* L, int64_t ldl, void* C, int64_t ldc, int64_t* info, int slices) {
  if (!h || slices < 1 || slices > gevp::kOzSlicesMax) return GEVP_ERR_INVALID_ARG;
  if (n > 30720) {
    h->err = "emulated product: n above 30720";
    return GEVP_ERR_UNSUPPORTED;
  }
  cudaSetDevice(h->device);
  if (n > 0 && !gevp::oz_supported()) {
    h->err = "emulated FP64 products need an sm_103 device";
    return GEVP_ERR_UNSUPPORTED;
  }
  const int keep = h->oz_slices;
  h->oz_slices = slices;
  gevp_status st = gevp_reduce(h, n, A, lda, B, ldb, L, ldl, C, ldc, info);
  if (st == GEVP_OK) st = oz_check(h);
  h->oz_slices = keep;
  return st;
}

gevp_status gevp_probe_peaks(gevp_handle h, double* out) {
  if (!h || !out) return GEVP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  probe_peaks(&out[0], &out[1], &out[2], h->stream);
  CK(cudaGetLastError());
  return GEVP_OK;
}

}  // extern "C"
