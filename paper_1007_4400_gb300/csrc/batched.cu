// Batched k-point driver (gevp_solve_batched): nk independent problem sequences of uneven
// order advance in lock-step rounds, one launch per phase for the whole batch.
//
// The paper's Eq. 3 is solved for every k-point and every self-consistent iteration;
// the k-points are independent. On one GPU, solving them one after another leaves most
// SMs idle in every phase that is small per problem (the m x m eigensolver, CholQR's
// small Cholesky, Lanczos, the tall-skinny products), and pays a host round trip per
// round and problem. Here every phase covers all k-points at once:
//   - FP64 products are grouped GEMMs over one global tile list (zgemm_grouped.cu);
//   - small dense work runs one CTA per problem (bkernels.cu, heev.cu);
//   - the low-precision filter is one grouped tcgen05 launch per step (filter_tc.cu);
//   - per-problem control (filter interval and degree, convergence, precision switch)
//     is computed on the device and gates each problem through device flags.
// A round (filter, CholQR3, Rayleigh-Ritz, status) therefore has a fixed launch
// sequence; it is captured once as a CUDA graph and replayed, with one 4-byte-per-problem
// status read per round. Step structure per k-point (B_k fixed along the sequence):
// Cholesky of B_k once per call; per step: C = L^-1 A L^-H (grouped), Lanczos bounds,
// start block (previous step's Ritz vectors, or random / caller's vectors at step 0),
// Rayleigh-Ritz, rounds until every wanted residual is below tol in the standard space,
// final residuals in the original space (re-opening a problem with a tighter tolerance
// and the FP64 filter if they miss tol).
//
// Autotuner: (1) every grouped GEMM call of a new batch shape is timed with 32 x 32 and
// 64 x 64 tiles on its first execution and keeps the faster; (2) after each step the
// filter degree cap of every size bucket is set by minimising the modelled time of the
// next step, R (T_rest + sum_b d_b T_step share_b), over the number of rounds R, where
// d_b(R) is the degree at which the Chebyshev factor rho_b of the bucket's slowest wanted
// Ritz value reduces its largest starting residual to tol in R rounds (T_rest, T_step
// measured on the first round, rho_b and the residuals from the step just solved).
#include "gevp_internal.cuh"
#include "../../include/gevp.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace gevp {

namespace {

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr int kNB = 24;        // doubles of per-problem bounds
constexpr int kNF = 16;        // ints of per-problem flags
constexpr int kBuckets = 8;    // size buckets of the degree autotuner (n / 512)

enum CallClass { CC_REDUCE, CC_CQ, CC_GRAM, CC_TALL, CC_SMALL, CC_FINAL, CC_FILTER, CC_N };

struct GCall {
  std::vector<ZgemmItem> items;
  ZgemmGroupFlags f{};
  int cls = 0;
  int tile = 32;
  int total = 0;
  size_t off = 0;   // index of the first item in the device pool
  bool tuned = false;
};

ZgemmItem item(int M, int N, int K, const double2* A, int64_t lda, const double2* B, int64_t ldb, double2* D,
               int64_t ldd, const int* active) {
  ZgemmItem it{};
  it.M = M; it.N = N; it.K = K;
  it.A = A; it.lda = lda;
  it.B = B; it.ldb = ldb;
  it.D = D; it.ldd = ldd;
  it.alpha = 1.0;
  it.active = active;
  return it;
}

}  // namespace

struct BatchPlan {
  // shape key
  int np = 0, prec = 0, nsplit = 0, deg_steps = 0, refine = 0, kl = 0;
  std::vector<int64_t> n;
  std::vector<int> m, nev;
  bool tc = false;
  int64_t nmax = 0;
  int mmax = 0, nevmax = 0;
  // device memory
  char* arena = nullptr;
  size_t arena_bytes = 0;
  BDesc* dD = nullptr;
  BDesc* hD = nullptr;            // pinned
  double* dBounds = nullptr;
  int* dFlags = nullptr;
  double* hBounds = nullptr;      // pinned
  int* hFlags = nullptr;          // pinned
  int *dStatus = nullptr, *hStatus = nullptr;
  int *dDegcap = nullptr, *hDegcap = nullptr;
  int *dMask = nullptr, *hMask = nullptr;
  int *dInfo = nullptr, *hInfo = nullptr;
  int *dErr = nullptr, *hErr = nullptr;
  BOut *dOut = nullptr, *hOut = nullptr;
  double2* ident = nullptr;
  double2* trtri_ws = nullptr;
  size_t trtri_elems = 0;
  ZgemmItem* pool = nullptr;
  size_t pool_items = 0;
  ZgemmItem* tune_pool = nullptr;
  size_t tune_items = 0;
  // calls
  std::vector<GCall> calls;
  int c_red1 = -1, c_red2 = -1, c_xf = -1, c_ax = -1, c_bx = -1, c_wt = -1, c_g = -1, c_qz = -1, c_wz = -1;
  int c_gram[3] = {-1, -1, -1}, c_apply[3] = {-1, -1, -1};
  int c_R[2], c_E[2], c_S[2], c_Zn[2], c_Ef[2], c_Sf[2];
  std::vector<int> c_filt;
  // tensor-core filter shape
  TcgShape tg{};
  // round graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool tuned = false, measured = false;
  // autotuner state
  float t_step = 0.f, t_rest = 0.f;   // ms per filter step (whole batch), ms per round besides the filter
  std::vector<int> bucket;
  int cap_bucket[kBuckets];
  // emulated reduction: digit forms of every k-point's L^-1 (left operand) and L^-H (right
  // operand), made once per call, plus one k-point's worth of scratch for tril(A) and T
  int oz_S = 0;
  int oz_key = 0;   // reduce_slices the plan (and its captured round) was built for
  char* oz_mem = nullptr;
  size_t oz_bytes = 0;
  std::vector<OzOperand> ozLA, ozLB;
  OzOperand ozAB, ozTA;
  char* oz_scratch = nullptr;
  // W = C Q of every round: the digits of each k-point's C (made once per step) and one
  // k-point's block (made per round, inside the captured round)
  std::vector<OzOperand> ozC;
  OzOperand ozQ;
  char* oz_cq = nullptr;
  size_t oz_cq_bytes = 0;
  char* oz_qs = nullptr;   // the block's digits (inside oz_cq)
  // the final check's X = L^-H Q, A X, B X: digits of every k-point's L^-H (rows) and B
  // (rows), made once per call, and one k-point's A (per check)
  std::vector<OzOperand> ozLH, ozBd;
  OzOperand ozAd;
  char* oz_fin = nullptr;
  size_t oz_fin_bytes = 0;
  char* oz_ad = nullptr;   // A's digits (inside oz_fin)
  double* oz_ws = nullptr;  // split-K partials of one k-point's thin product
  size_t oz_ws_doubles = 0;
  int* oz_flags = nullptr;   // device: [0] kernel error code, [1] non-finite entry
  std::vector<cudaEvent_t> ev;
};

void batch_release(BatchPlan* P) {
  if (!P) return;
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->arena) cudaFree(P->arena);
  if (P->oz_mem) cudaFree(P->oz_mem);
  if (P->oz_cq) cudaFree(P->oz_cq);
  if (P->oz_fin) cudaFree(P->oz_fin);
  if (P->oz_ws) cudaFree(P->oz_ws);
  if (P->hD) cudaFreeHost(P->hD);
  for (auto e : P->ev) cudaEventDestroy(e);
  delete P;
}

namespace {

// ---------------------------------------------------------------- plan

gevp_status build_plan(gevp_ctx* h, BatchPlan* P, std::string& err) {
  const int np = P->np;
  const bool tc = P->tc;
  // tensor-core geometry, split-K across the batch
  std::vector<int> n_pad(np), ncols_pad(np), nchunk(np), nchunks(np), ks(np, 1), kbps(np, 1);
  int64_t base_units = 0;
  if (tc) {
    for (int p = 0; p < np; ++p) {
      tcg_geometry(P->n[p], P->m[p], &n_pad[p], &ncols_pad[p], &nchunk[p], &nchunks[p]);
      base_units += (int64_t)(n_pad[p] / 128) * nchunks[p];
    }
    int ks_all = base_units >= 152 ? 1 : (int)std::min<int64_t>(16, (2 * 152 + base_units - 1) / base_units);
    for (int p = 0; p < np; ++p) {
      int nkb = n_pad[p] / 64;
      int k = std::max(1, std::min(ks_all, nkb / 2));
      kbps[p] = (nkb + k - 1) / k;
      ks[p] = (nkb + kbps[p] - 1) / kbps[p];
    }
  }
  // ---- arena layout (two passes: measure, then place)
  int64_t tn = P->nmax;
  P->trtri_elems = trtri_ws_elems(tn) + std::max<size_t>(8 * (size_t)tn * 64, 1 << 16);
  auto layout = [&](char* base) -> size_t {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
      char* q = base ? base + off : nullptr;
      off += al256(bytes);
      return q;
    };
    P->dBounds = (double*)take((size_t)np * kNB * 8);
    P->dFlags = (int*)take((size_t)np * kNF * 4);
    P->dStatus = (int*)take((size_t)np * 4);
    P->dDegcap = (int*)take((size_t)np * 4);
    P->dMask = (int*)take((size_t)np * 4);
    P->dInfo = (int*)take((size_t)np * 4);
    P->dErr = (int*)take(64);
    take(64);
    P->dOut = (BOut*)take((size_t)np * sizeof(BOut));
    P->dD = (BDesc*)take((size_t)np * sizeof(BDesc));
    P->ident = (double2*)take((size_t)P->mmax * P->mmax * 16);
    P->trtri_ws = (double2*)take(P->trtri_elems * 16);
    for (int p = 0; p < np; ++p) {
      BDesc& d = P->hD[p];
      const int64_t n = P->n[p];
      const int m = P->m[p];
      const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
      d.L = (double2*)take(nn * 16);
      d.Linv = (double2*)take(nn * 16);
      d.C = (double2*)take(nn * 16);
      d.T = (double2*)take(nn * 16);
      d.M32 = (float2*)take(nn * 8);
      d.Q = (double2*)take(nm * 16);
      d.Y1 = (double2*)take(nm * 16);
      d.Y2 = (double2*)take(nm * 16);
      d.W = (double2*)take(nm * 16);
      d.Wt = (double2*)take(nm * 16);
      d.Xf = (double2*)take(nm * 16);
      d.G = (double2*)take(mm * 16);
      d.Zs = (double2*)take(mm * 16);
      d.Gw = (double2*)take(mm * 16);
      d.Gwi = (double2*)take(mm * 16);
      d.G32 = (float2*)take(mm * 8);
      d.Z32 = (float2*)take(mm * 8);
      d.w32 = (float*)take((size_t)m * 4);
      d.perm = (int*)take((size_t)m * 4);
      d.hZ = (double2*)take(mm * 16);
      d.hR = (double2*)take(mm * 16);
      d.hS = (double2*)take(mm * 16);
      d.hT = (double2*)take(mm * 16);
      d.hE = (double2*)take(mm * 16);
      d.hlam = (double*)take((size_t)m * 8);
      d.hscal = (double*)take(16 * 8);
      d.V = (float2*)take((size_t)65 * n * 8);
      d.lvec = (float2*)take((size_t)n * 8);
      d.T32 = (float2*)take(64 * 64 * 8);
      d.LZ32 = (float2*)take(64 * 64 * 8);
      d.ab = (float*)take(140 * 4);
      d.lw32 = (float*)take(64 * 4);
      d.lperm = (int*)take(64 * 4);
      d.theta = (double*)take((size_t)m * 8);
      d.res = (double*)take((size_t)m * 8);
      d.lamf = (double*)take((size_t)m * 8);
      d.resf = (double*)take((size_t)m * 8);
      d.dscale = (double*)take((size_t)m * 8);
      d.partial = (double*)take(bk_partial_elems(m) * 8);
      d.fco = (double*)take((size_t)kBDegMax * 3 * 8);
      d.stepact = (int*)take((size_t)kBDegMax * 4);
      if (tc) {
        const size_t np2 = (size_t)n_pad[p] * n_pad[p], nc = (size_t)ncols_pad[p] * n_pad[p];
        d.Cp = (__nv_bfloat16*)take((size_t)P->nsplit * 3 * np2 * 2);
        d.Yp = (__nv_bfloat16*)take((size_t)P->nsplit * 3 * nc * 2);
        d.S0 = (float2*)take(nc * 8);
        d.S1 = (float2*)take(nc * 8);
        d.S2 = (float2*)take(nc * 8);
        d.S3 = (float2*)take(nc * 8);
        d.tws = (float2*)take((size_t)ks[p] * nc * 8);
        d.pcoef = (float*)take((size_t)kBDegMax * ncols_pad[p] * 4);
        d.pfinal = (double*)take((size_t)ncols_pad[p] * 8);
        d.maps = take(tcg_map_bytes());
      }
    }
    return off;
  };
  size_t bytes = layout(nullptr);
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bytes);
  if (e != cudaSuccess) {
    err = "batched workspace cudaMalloc failed";
    return e == cudaErrorMemoryAllocation ? GEVP_ERR_OOM : GEVP_ERR_CUDA;
  }
  P->arena = (char*)mem;
  P->arena_bytes = bytes;
  layout(P->arena);
  cudaStream_t s = ctx_stream(h);
  cudaMemsetAsync(P->arena, 0, bytes, s);
  // ---- descriptors
  int unit = 0;
  for (int p = 0; p < np; ++p) {
    BDesc& d = P->hD[p];
    d.n = (int)P->n[p];
    d.m = P->m[p];
    d.nev = P->nev[p];
    d.kl = P->kl;
    d.bounds = P->dBounds + (size_t)p * kNB;
    d.flags = P->dFlags + (size_t)p * kNF;
    d.active = d.flags;
    d.nsplit = P->nsplit;
    if (tc) {
      d.n_pad = n_pad[p];
      d.ncols_pad = ncols_pad[p];
      d.nchunk = nchunk[p];
      d.nchunks = nchunks[p];
      d.mtiles = n_pad[p] / 128;
      d.ks = ks[p];
      d.kbps = kbps[p];
      d.nseg = tcg_nseg(P->nsplit);
      unsigned tcols = 32;
      while (tcols < 3u * (unsigned)nchunk[p]) tcols *= 2;
      d.tmem_cols = tcols;
      d.unit_start = unit;
      unit += d.mtiles * d.nchunks * d.ks;
    } else {
      d.pcoef = nullptr;
      d.pfinal = nullptr;
      d.ncols_pad = 0;
    }
  }
  if (tc) {
    P->tg.np = np;
    P->tg.units = unit;
    P->tg.n_pad_max = *std::max_element(n_pad.begin(), n_pad.end());
    P->tg.ncols_pad_max = *std::max_element(ncols_pad.begin(), ncols_pad.end());
    P->tg.nchunk_max = *std::max_element(nchunk.begin(), nchunk.end());
    P->tg.steps = P->deg_steps;
    int64_t ncm = 0;
    for (int p = 0; p < np; ++p) ncm = std::max<int64_t>(ncm, (int64_t)ncols_pad[p] * n_pad[p]);
    P->tg.nc_max = ncm;
    e = tcg_prepare(P->tg.nchunk_max);
    if (e != cudaSuccess) { err = "tensor-core filter: shared memory attribute refused"; return GEVP_ERR_CUDA; }
    const size_t mb = tcg_map_bytes();
    std::vector<char> maps(mb * np);
    for (int p = 0; p < np; ++p) {
      if (!tcg_encode_maps(P->hD[p], maps.data() + mb * p)) {
        err = "cuTensorMapEncodeTiled failed for the batched filter";
        return GEVP_ERR_UNSUPPORTED;
      }
      // ordered after the arena clear on the same stream
      e = cudaMemcpyAsync((void*)P->hD[p].maps, maps.data() + mb * p, mb, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) { err = "tensor map upload failed"; return GEVP_ERR_CUDA; }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { err = "tensor map upload failed"; return GEVP_ERR_CUDA; }
  }
  zset_identity(P->mmax, P->mmax, P->ident, P->mmax, s);
  // ---- grouped GEMM calls with fixed pointers (the round) and per-step ones
  auto add = [&](int cls, ZgemmGroupFlags f) -> int {
    GCall c;
    c.cls = cls;
    c.f = f;
    P->calls.push_back(c);
    return (int)P->calls.size() - 1;
  };
  auto fl = [](int opA, int opB, int triA, int triB, int triD, int maskB) {
    ZgemmGroupFlags f{opA, opB, triA, triB, triD, maskB};
    return f;
  };
  P->c_red1 = add(CC_REDUCE, fl(0, 0, 1, 0, 0, 1));
  P->c_red2 = add(CC_REDUCE, fl(0, 1, 1, 2, 0, 0));
  P->c_xf = add(CC_FINAL, fl(1, 0, 2, 0, 0, 0));
  P->c_ax = add(CC_FINAL, fl(0, 0, 0, 0, 0, 0));
  P->c_bx = add(CC_FINAL, fl(0, 0, 0, 0, 0, 0));
  P->c_wt = add(CC_CQ, fl(0, 0, 0, 0, 0, 0));
  P->c_g = add(CC_GRAM, fl(1, 0, 0, 0, 0, 0));
  P->c_qz = add(CC_TALL, fl(0, 0, 0, 0, 0, 0));
  P->c_wz = add(CC_TALL, fl(0, 0, 0, 0, 0, 0));
  for (int k = 0; k < 3; ++k) {
    P->c_gram[k] = add(CC_GRAM, fl(1, 0, 0, 0, 1, 0));
    P->c_apply[k] = add(CC_TALL, fl(0, 1, 0, 2, 0, 0));
  }
  for (int par = 0; par < 2; ++par) {
    P->c_R[par] = add(CC_SMALL, fl(1, 0, 0, 0, 0, 0));
    P->c_E[par] = add(CC_SMALL, fl(0, 0, 0, 0, 0, 0));
    P->c_S[par] = add(CC_SMALL, fl(1, 0, 0, 0, 0, 0));
    P->c_Zn[par] = add(CC_SMALL, fl(0, 0, 0, 0, 0, 0));
    P->c_Ef[par] = add(CC_SMALL, fl(0, 0, 0, 0, 0, 0));
    P->c_Sf[par] = add(CC_SMALL, fl(1, 0, 0, 0, 0, 0));
  }
  P->c_filt.clear();
  for (int j = 0; j < P->deg_steps; ++j) P->c_filt.push_back(add(CC_FILTER, fl(0, 0, 0, 0, 0, 0)));
  const int mmax = P->mmax;
  for (int p = 0; p < np; ++p) {
    const BDesc& d = P->hD[p];
    const int n = d.n, m = d.m, nev = d.nev;
    const int* act = d.flags;
    const int* fin = d.flags + 12;
    // reduction: A pointer set per step
    P->calls[P->c_red1].items.push_back(item(n, n, n, d.Linv, n, nullptr, 0, d.T, n, act));
    P->calls[P->c_red2].items.push_back(item(n, n, n, d.T, n, d.Linv, n, d.C, n, act));
    P->calls[P->c_xf].items.push_back(item(n, nev, n, d.Linv, n, d.Q, m, d.Xf, m, fin));
    P->calls[P->c_ax].items.push_back(item(n, nev, n, nullptr, 0, d.Xf, m, d.Y1, m, fin));
    P->calls[P->c_bx].items.push_back(item(n, nev, n, nullptr, 0, d.Xf, m, d.Y2, m, fin));
    P->calls[P->c_wt].items.push_back(item(n, m, n, d.C, n, d.Q, m, d.Wt, m, act));
    P->calls[P->c_g].items.push_back(item(m, m, n, d.Q, m, d.Wt, m, d.G, m, act));
    P->calls[P->c_qz].items.push_back(item(n, m, m, d.Q, m, d.Zs, m, d.Y1, m, act));
    P->calls[P->c_wz].items.push_back(item(n, m, m, d.Wt, m, d.Zs, m, d.W, m, act));
    double2* src[3] = {d.Y1, d.Y2, d.Y1};
    double2* dst[3] = {d.Y2, d.Y1, d.Q};
    for (int k = 0; k < 3; ++k) {
      P->calls[P->c_gram[k]].items.push_back(item(m, m, n, src[k], m, src[k], m, d.Gw, m, act));
      P->calls[P->c_apply[k]].items.push_back(item(n, m, m, src[k], m, d.Gwi, m, dst[k], m, act));
    }
    double2* Zp[2] = {d.hZ, d.hT};
    for (int par = 0; par < 2; ++par) {
      double2* Z = Zp[par];
      double2* Zn = Zp[1 - par];
      ZgemmItem r = item(m, m, m, Z, m, Z, m, d.hR, m, act);
      r.alpha = -1.0;
      r.Cin = P->ident;
      r.ldc = mmax;
      r.beta = 1.0;
      P->calls[P->c_R[par]].items.push_back(r);
      P->calls[P->c_E[par]].items.push_back(item(m, m, m, d.G, m, Z, m, d.hE, m, act));
      P->calls[P->c_S[par]].items.push_back(item(m, m, m, Z, m, d.hE, m, d.hS, m, act));
      ZgemmItem zn = item(m, m, m, Z, m, d.hE, m, Zn, m, act);
      zn.Cin = Z;
      zn.ldc = m;
      zn.beta = 1.0;
      P->calls[P->c_Zn[par]].items.push_back(zn);
      P->calls[P->c_Ef[par]].items.push_back(item(m, m, m, d.G, m, Z, m, d.hE, m, act));
      P->calls[P->c_Sf[par]].items.push_back(item(m, m, m, Z, m, d.hE, m, d.hS, m, act));
    }
    double2* slot[3] = {d.Q, d.Y1, d.Y2};
    for (int j = 0; j < P->deg_steps; ++j) {
      ZgemmItem f = item(n, m, n, d.C, n, slot[j % 3], m, slot[(j + 1) % 3], m, d.stepact + j);
      f.Cin = slot[j % 3];
      f.ldc = m;
      if (j >= 1) {
        f.Ein = slot[(j + 2) % 3];
        f.lde = m;
      }
      f.coef = d.fco + 3 * j;
      P->calls[P->c_filt[j]].items.push_back(f);
    }
  }
  // device item pool (room for a caller-vector call too)
  size_t total = 0, largest = 0;
  for (auto& c : P->calls) {
    c.off = total;
    total += c.items.size();
    largest = std::max(largest, c.items.size());
  }
  P->pool_items = total + np;
  P->tune_items = largest;
  e = cudaMalloc(&P->pool, (P->pool_items + P->tune_items) * sizeof(ZgemmItem));
  if (e != cudaSuccess) { err = "item pool cudaMalloc failed"; return GEVP_ERR_OOM; }
  P->tune_pool = P->pool + P->pool_items;
  for (auto& c : P->calls) {
    c.tile = zgemm_group_tile(c.items.data(), (int)c.items.size());
    c.total = zgemm_group_layout(c.items.data(), (int)c.items.size(), c.tile);
  }
  P->bucket.resize(np);
  for (int p = 0; p < np; ++p) P->bucket[p] = (int)std::min<int64_t>(kBuckets - 1, P->n[p] / 512);
  for (int b = 0; b < kBuckets; ++b) P->cap_bucket[b] = P->deg_steps;
  return GEVP_OK;
}

// upload the items of one call (pointer fields may have changed)
cudaError_t upload_call(BatchPlan* P, GCall& c, cudaStream_t s) {
  if (c.items.empty()) return cudaSuccess;
  c.total = zgemm_group_layout(c.items.data(), (int)c.items.size(), c.tile);
  return cudaMemcpyAsync(P->pool + c.off, c.items.data(), c.items.size() * sizeof(ZgemmItem),
                         cudaMemcpyHostToDevice, s);
}

cudaEvent_t evt(BatchPlan* P, size_t i) {
  while (P->ev.size() <= i) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    P->ev.push_back(e);
  }
  return P->ev[i];
}

// one grouped GEMM call; on its first run for a new shape both tiles are timed
void launch(BatchPlan* P, int ci, cudaStream_t s, bool tune) {
  GCall& c = P->calls[ci];
  const int ni = (int)c.items.size();
  if (ni == 0) return;
  if (tune && !c.tuned) {
    float best = 1e30f;
    int best_tile = c.tile;
    for (int t : {32, 64}) {
      std::vector<ZgemmItem> tmp = c.items;
      int tot = zgemm_group_layout(tmp.data(), ni, t);
      cudaMemcpyAsync(P->tune_pool, tmp.data(), ni * sizeof(ZgemmItem), cudaMemcpyHostToDevice, s);
      cudaEventRecord(evt(P, 0), s);
      zgemm_grouped(P->tune_pool, ni, tot, t, c.f, s);
      cudaEventRecord(evt(P, 1), s);
      cudaEventSynchronize(evt(P, 1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, evt(P, 0), evt(P, 1));
      if (ms < best) { best = ms; best_tile = t; }
    }
    c.tile = best_tile;
    c.tuned = true;
    upload_call(P, c, s);
    return;   // the timed runs computed the result
  }
  zgemm_grouped(P->pool + c.off, ni, c.total, c.tile, c.f, s);
}

// ---------------------------------------------------------------- phases
void enqueue_orth(BatchPlan* P, cudaStream_t s, bool tune) {
  const int np = P->np;
  const int64_t nm = P->nmax * P->mmax;
  const int src_idx[3] = {0, 1, 0};   // nm blocks: 0 Y1, 1 Y2, 2 Q
  for (int k = 0; k < 3; ++k) {
    launch(P, P->c_gram[k], s, tune);
    bk_hermitize_lower_G(P->dD, np, P->mmax, s);
    // the first pass is shifted CholQR (always positive definite for cond(Y) up to about
    // 1/u), the two plain ones that follow restore orthonormality to FP64 rounding
    bk_gram_scale(P->dD, np, k == 0 ? 1.0 : 0.0, s);
    bk_potrf_small(P->dD, np, s);
    bk_trtri_small(P->dD, np, s);
    bk_col_scale(P->dD, np, nm, src_idx[k], s);
    launch(P, P->c_apply[k], s, tune);
  }
}

void enqueue_rr(BatchPlan* P, cudaStream_t s, bool tune) {
  const int np = P->np, mmax = P->mmax;
  if (P->oz_S > 0 && (int)P->ozC.size() == np) {
    // W = C Q emulated per k-point; a converged k-point's launches do nothing
    for (int k = 0; k < np; ++k) {
      const BDesc& d = P->hD[k];
      oz_split(P->ozQ, P->oz_qs, d.m, d.n, d.Q, d.m, 0, 0, P->oz_S, 3, P->oz_flags + 1, s, true, d.flags);
      oz_gemm(P->ozC[k], P->ozQ, 0, 0, d.Wt, d.m, P->oz_flags, s, d.flags, P->oz_ws, P->oz_ws_doubles);
    }
  } else {
    launch(P, P->c_wt, s, tune);
  }
  launch(P, P->c_g, s, tune);
  bk_heev_prep(P->dD, np, mmax, s);
  for (int it = 0; it <= P->refine; ++it) {
    const int par = it & 1;
    launch(P, P->c_R[par], s, tune);
    launch(P, P->c_E[par], s, tune);
    launch(P, P->c_S[par], s, tune);
    bk_oa_scalars(P->dD, np, s);
    bk_oa_update(P->dD, np, mmax, it == P->refine ? 1 : 0, s);
    launch(P, P->c_Zn[par], s, tune);
  }
  const int zsel = (P->refine + 1) & 1;
  launch(P, P->c_Ef[zsel], s, tune);
  launch(P, P->c_Sf[zsel], s, tune);
  bk_hermitize_avg_S(P->dD, np, mmax, s);
  cluster_jacobi_batched(P->dD, np, zsel, 1e-15, 12, s);
  bk_sort_pairs(P->dD, np, zsel, s);
  launch(P, P->c_qz, s, tune);
  bk_copy_nm(P->dD, np, P->nmax * mmax, 0, 2, s);   // Q <- Y1
  launch(P, P->c_wz, s, tune);
  bk_resid(P->dD, np, mmax, s);
}

cudaError_t enqueue_filter(BatchPlan* P, cudaStream_t s, bool tune, int deg_min) {
  const int np = P->np;
  bk_cheb_coef(P->dD, np, deg_min, P->dDegcap, s);
  if (P->tc) {
    cudaError_t e = tcg_filter(P->dD, P->tg, P->dErr, s);
    if (e != cudaSuccess) return e;
  }
  for (int j = 0; j < P->deg_steps; ++j) launch(P, P->c_filt[j], s, tune);
  bk_fp64_select(P->dD, np, P->nmax * P->mmax, s);
  return cudaGetLastError();
}

void enqueue_status(BatchPlan* P, cudaStream_t s) {
  bk_round_status(P->dD, P->np, P->dStatus, s);
  cudaMemcpyAsync(P->hStatus, P->dStatus, P->np * sizeof(int), cudaMemcpyDeviceToHost, s);
}

// ---------------------------------------------------------------- degree autotuner
void tune_degrees(BatchPlan* P, const gevp_opts& o) {
  const int np = P->np;
  double share[kBuckets] = {0}, L[kBuckets] = {0}, lrho[kBuckets], tot = 0;
  bool used[kBuckets] = {false};
  for (int b = 0; b < kBuckets; ++b) lrho[b] = 1e300;
  for (int p = 0; p < np; ++p) {
    const double* bd = P->hBounds + (size_t)p * kNB;
    const int b = P->bucket[p];
    double w = (double)P->n[p] * P->n[p] * P->m[p];
    share[b] += w;
    tot += w;
    used[b] = true;
    double r0 = bd[19], tolC = bd[6];
    double l = (r0 > tolC && tolC > 0) ? std::log(r0 / tolC) : 0.0;
    L[b] = std::max(L[b], 1.2 * l);
    double rho = bd[20];
    lrho[b] = std::min(lrho[b], rho > 1.0 ? std::log(rho) : 1e-3);
  }
  // largest residual reduction one round of the filter can deliver, by its precision
  const double lcap = P->prec == GEVP_PREC_FP64 ? std::log(1e13) : (P->prec == GEVP_PREC_FP32 ? std::log(1e5)
                                                                                             : std::log(30.0));
  const double Tf = std::max(P->t_step, 1e-3f), Tr = std::max(P->t_rest, 1e-3f);
  double best = 1e300;
  int bestR = -1;
  int caps[kBuckets];
  for (int R = 1; R <= 8; ++R) {
    double cost = Tr;
    int c[kBuckets];
    bool ok = true;
    for (int b = 0; b < kBuckets; ++b) {
      c[b] = o.deg_min;
      if (!used[b] || L[b] <= 0) continue;
      if (lcap * R < L[b]) { ok = false; break; }
      double d = std::ceil(L[b] / (R * lrho[b]));
      if (d > P->deg_steps) { ok = false; break; }
      c[b] = std::max(o.deg_min, (int)d);
      cost += c[b] * Tf * share[b] / std::max(tot, 1e-300);
    }
    if (!ok) continue;
    cost *= R;
    if (cost < best) {
      best = cost;
      bestR = R;
      std::memcpy(caps, c, sizeof(caps));
    }
  }
  for (int b = 0; b < kBuckets; ++b) P->cap_bucket[b] = bestR > 0 ? caps[b] : P->deg_steps;
}

}  // namespace

}  // namespace gevp

using namespace gevp;

extern "C" gevp_status gevp_solve_batched(gevp_handle h, int nk, int nsteps, const int64_t* n, const int* nev,
                                          const int* nex, const void* const* A, const int64_t* lda,
                                          const void* const* B, const int64_t* ldb, const void* const* X_prev,
                                          const int64_t* ldxp, const int* kprev, const gevp_opts* opts,
                                          double* const* Lambda, double* const* resid, void* const* X,
                                          const int64_t* ldx, gevp_batch_stats* stats) {
  if (!h || nk < 0 || nsteps < 0) return GEVP_ERR_INVALID_ARG;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (nk == 0 || nsteps == 0) return GEVP_OK;
  if (!n || !nev || !A || !lda || !B || !ldb || !Lambda || !resid) return GEVP_ERR_INVALID_ARG;
  gevp_opts o;
  if (opts) o = *opts; else gevp_default_opts(&o);
  if (o.filter_prec < 0 || o.filter_prec > 2) return GEVP_ERR_INVALID_ARG;
  if (o.deg_min < 1) o.deg_min = 1;
  o.deg_max = std::min(std::max(o.deg_max, o.deg_min), kBDegMax);
  if (o.refine_iters < 1) o.refine_iters = 1;
  if (o.lanczos_steps < 4) o.lanczos_steps = 4;
  if (o.max_outer < 1) o.max_outer = 1;
  std::vector<int> m(nk);
  int64_t nmin = INT64_MAX;
  for (int k = 0; k < nk; ++k) {
    if (n[k] < 2 || nev[k] < 1 || nev[k] > n[k] || n[k] > (1 << 30) / 2) return GEVP_ERR_INVALID_ARG;
    if (lda[k] < n[k] || ldb[k] < n[k] || !B[k]) return GEVP_ERR_INVALID_ARG;
    int ex = std::max(2, nex ? nex[k] : o.nex);
    m[k] = (int)std::min<int64_t>(n[k], (int64_t)nev[k] + ex);
    if (m[k] > 1024) { ctx_set_error(h, "block width nev + nex above 1024"); return GEVP_ERR_UNSUPPORTED; }
    if (!Lambda[k] || !resid[k]) return GEVP_ERR_INVALID_ARG;
    if (X && X[k] && (!ldx || ldx[k] < nev[k])) return GEVP_ERR_INVALID_ARG;
    if (X_prev && X_prev[k] && (!ldxp || !kprev || kprev[k] < 1 || kprev[k] > m[k] || ldxp[k] < kprev[k]))
      return GEVP_ERR_INVALID_ARG;
    for (int l = 0; l < nsteps; ++l)
      if (!A[(size_t)k * nsteps + l]) return GEVP_ERR_INVALID_ARG;
    nmin = std::min(nmin, n[k]);
  }
  const bool tc = o.filter_prec != GEVP_PREC_FP64;
  if (tc && !tc_filter_supported()) {
    ctx_set_error(h, "tensor-core filter needs an sm_103 device");
    return GEVP_ERR_UNSUPPORTED;
  }
  cudaSetDevice(ctx_device(h));
  cudaStream_t s = ctx_stream(h);
  const int nsplit = o.filter_prec == GEVP_PREC_FP32 ? 3 : 1;
  const int kl = (int)std::min<int64_t>(std::min(o.lanczos_steps, 64), nmin);

  // ---- plan (reused while the shapes and modes are unchanged)
  BatchPlan*& P = ctx_batch(h);
  // the captured round graph embeds the emulated products or the grouped FP64 one
  const int oz_want = (o.reduce_slices > 0 && oz_supported()) ? o.reduce_slices : 0;
  bool same = P && P->np == nk && P->prec == o.filter_prec && P->deg_steps == o.deg_max &&
              P->refine == o.refine_iters && P->kl == kl && P->oz_key == oz_want;
  if (same)
    for (int k = 0; k < nk && same; ++k) same = P->n[k] == n[k] && P->m[k] == m[k] && P->nev[k] == nev[k];
  if (!same) {
    if (P) {
      cudaStreamSynchronize(s);
      batch_release(P);
      P = nullptr;
    }
    P = new BatchPlan();
    P->np = nk;
    P->oz_key = oz_want;
    P->prec = o.filter_prec;
    P->nsplit = nsplit;
    P->tc = tc;
    P->deg_steps = o.deg_max;
    P->refine = o.refine_iters;
    P->kl = kl;
    P->n.assign(n, n + nk);
    P->m = m;
    P->nev.assign(nev, nev + nk);
    P->nmax = *std::max_element(P->n.begin(), P->n.end());
    P->mmax = *std::max_element(m.begin(), m.end());
    P->nevmax = *std::max_element(P->nev.begin(), P->nev.end());
    // pinned host mirrors
    size_t hb = al256((size_t)nk * sizeof(BDesc)) + al256((size_t)nk * kNB * 8) + al256((size_t)nk * kNF * 4) +
                5 * al256((size_t)nk * 4) + al256((size_t)nk * sizeof(BOut));
    char* hp = nullptr;
    if (cudaMallocHost(&hp, hb) != cudaSuccess) {
      delete P;
      P = nullptr;
      return GEVP_ERR_OOM;
    }
    std::memset(hp, 0, hb);
    P->hD = (BDesc*)hp; hp += al256((size_t)nk * sizeof(BDesc));
    P->hBounds = (double*)hp; hp += al256((size_t)nk * kNB * 8);
    P->hFlags = (int*)hp; hp += al256((size_t)nk * kNF * 4);
    P->hStatus = (int*)hp; hp += al256((size_t)nk * 4);
    P->hDegcap = (int*)hp; hp += al256((size_t)nk * 4);
    P->hMask = (int*)hp; hp += al256((size_t)nk * 4);
    P->hInfo = (int*)hp; hp += al256((size_t)nk * 4);
    P->hErr = (int*)hp; hp += al256((size_t)nk * 4);
    P->hOut = (BOut*)hp;
    std::string err;
    gevp_status st = build_plan(h, P, err);
    if (st != GEVP_OK) {
      ctx_set_error(h, err.c_str());
      batch_release(P);
      P = nullptr;
      return st;
    }
  }
  const int np = nk;
  const int64_t nm_max = P->nmax * P->mmax;
  gevp_batch_stats local{};
  gevp_batch_stats* bs = stats ? stats : &local;
  bs->steps = nsteps;
  auto fail = [&](cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    ctx_set_error(h, buf);
    return e == cudaErrorMemoryAllocation ? GEVP_ERR_OOM : GEVP_ERR_CUDA;
  };
#define BCK(x)                              \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return fail(e_, #x); \
  } while (0)
  enum { EV_T0 = 2, EV_CHOL, EV_RED, EV_BND, EV_RND0, EV_RND1, EV_FIN0, EV_FIN1, EV_F0, EV_F1, EV_END };
  BCK(cudaEventRecord(evt(P, EV_T0), s));

  // digit memory of the emulated products (o.reduce_slices digits per entry): the L^-1
  // operands of every k-point and a scratch pair; the factorisations below use the front
  // of it before the L^-1 operands are split there
  P->oz_S = P->nmax <= 30720 ? P->oz_key : 0;
  if (P->oz_S > 0) {
    const int S = P->oz_S;
    size_t need = 256, scratch = 0;
    for (int k = 0; k < np; ++k) {
      const int nk_ = (int)n[k];
      need += oz_operand_bytes(nk_, nk_, S, 2) + oz_operand_bytes(nk_, nk_, S, 3);
      scratch = std::max(scratch, oz_operand_bytes(nk_, nk_, S, 2) + oz_operand_bytes(nk_, nk_, S, 3));
    }
    need += scratch;
    if (need > P->oz_bytes) {
      if (P->oz_mem) cudaFree(P->oz_mem);
      P->oz_mem = nullptr;
      P->oz_bytes = 0;
      BCK(cudaMalloc(&P->oz_mem, need));
      P->oz_bytes = need;
    }
    P->oz_flags = (int*)P->oz_mem;
    BCK(cudaMemsetAsync(P->oz_flags, 0, 2 * sizeof(int), s));
  }

  // ---- Cholesky of every B_k (sequence-invariant): recursive with emulated off-diagonal
  // products when the products are emulated, else blocked on the FP64 pipe
  BCK(cudaMemsetAsync(P->dInfo, 0, np * sizeof(int), s));
  for (int k = 0; k < np; ++k) {
    BDesc& d = P->hD[k];
    zcopy2d(n[k], n[k], (const double2*)B[k], ldb[k], d.L, n[k], s);
    cudaError_t ce = cudaErrorNotSupported;
    if (P->oz_S > 0) {
      CholRes r{};
      r.memA = P->oz_mem + 256;
      r.memB = r.memA + oz_operand_bytes((int)n[k], (int)n[k], P->oz_S, 2);
      r.T = d.T;
      r.ldt = n[k];
      r.ws = P->oz_ws;
      r.ws_doubles = P->oz_ws_doubles;
      r.flags = P->oz_flags;
      r.info = P->dInfo + k;
      r.S = P->oz_S;
      r.s = s;
      ce = chol_recursive(n[k], d.L, n[k], d.Linv, n[k], r);
      if (ce != cudaSuccess && ce != cudaErrorNotSupported) return fail(ce, "chol_recursive");
    }
    if (ce == cudaErrorNotSupported) {
      potrf_lower(n[k], d.L, n[k], P->dInfo + k, d.Linv, n[k], s);
      trtri_lower(n[k], d.L, n[k], d.Linv, n[k], P->trtri_ws, P->trtri_elems, s, true);
    }
  }
  BCK(cudaMemcpyAsync(P->hInfo, P->dInfo, np * sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaEventRecord(evt(P, EV_CHOL), s));
  BCK(cudaStreamSynchronize(s));
  for (int k = 0; k < np; ++k)
    if (P->hInfo[k] != 0) {
      char buf[96];
      snprintf(buf, sizeof buf, "B of k-point %d is not positive definite (pivot %d)", k, P->hInfo[k]);
      ctx_set_error(h, buf);
      return GEVP_ERR_NOT_HPD;
    }
  if (P->oz_S > 0) {
    const int S = P->oz_S;
    char* q = P->oz_mem + 256;
    P->ozLA.assign(np, OzOperand{});
    P->ozLB.assign(np, OzOperand{});
    for (int k = 0; k < np; ++k) {
      const BDesc& d = P->hD[k];
      const int nk_ = (int)n[k];
      BCK(oz_split(P->ozLA[k], q, nk_, nk_, d.Linv, n[k], 0, 2, S, 2, P->oz_flags + 1, s));
      q += oz_operand_bytes(nk_, nk_, S, 2);
      BCK(oz_split(P->ozLB[k], q, nk_, nk_, d.Linv, n[k], 1, 2, S, 3, P->oz_flags + 1, s));
      q += oz_operand_bytes(nk_, nk_, S, 3);
    }
    P->oz_scratch = q;
    // digits of C (one per k-point) and of one block (the largest)
    size_t cq = 256, qs = 0;
    for (int k = 0; k < np; ++k) {
      cq += oz_operand_bytes((int)n[k], (int)n[k], S, 2);
      qs = std::max(qs, oz_operand_bytes(P->hD[k].m, (int)n[k], S, 3));
    }
    cq += qs;
    if (cq > P->oz_cq_bytes) {
      if (P->oz_cq) cudaFree(P->oz_cq);
      P->oz_cq = nullptr;
      P->oz_cq_bytes = 0;
      BCK(cudaMalloc(&P->oz_cq, cq));
      P->oz_cq_bytes = cq;
    }
    P->oz_qs = P->oz_cq + (cq - qs);
    P->ozC.assign(np, OzOperand{});
    // L^-H and B digits for the final check, and room for one A
    size_t fb = 256, ab = 0;
    for (int k = 0; k < np; ++k) {
      fb += 2 * oz_operand_bytes((int)n[k], (int)n[k], S, 2);
      ab = std::max(ab, oz_operand_bytes((int)n[k], (int)n[k], S, 2));
    }
    fb += ab;
    if (fb > P->oz_fin_bytes) {
      if (P->oz_fin) cudaFree(P->oz_fin);
      P->oz_fin = nullptr;
      P->oz_fin_bytes = 0;
      BCK(cudaMalloc(&P->oz_fin, fb));
      P->oz_fin_bytes = fb;
    }
    P->ozLH.assign(np, OzOperand{});
    P->ozBd.assign(np, OzOperand{});
    char* f = P->oz_fin;
    for (int k = 0; k < np; ++k) {
      const BDesc& d = P->hD[k];
      const int nk_ = (int)n[k];
      // rows of L^-H (upper) = conjugated columns of L^-1
      BCK(oz_split(P->ozLH[k], f, nk_, nk_, d.Linv, n[k], 1, 3, S, 2, P->oz_flags + 1, s, true));
      f += oz_operand_bytes(nk_, nk_, S, 2);
      BCK(oz_split(P->ozBd[k], f, nk_, nk_, (const double2*)B[k], ldb[k], 0, 0, S, 2, P->oz_flags + 1, s));
      f += oz_operand_bytes(nk_, nk_, S, 2);
    }
    P->oz_ad = f;
    size_t wd = 0;
    for (int k = 0; k < np; ++k) wd = std::max(wd, oz_split_k_doubles((int)n[k], P->hD[k].m));
    if (wd > P->oz_ws_doubles) {
      if (P->oz_ws) cudaFree(P->oz_ws);
      P->oz_ws = nullptr;
      P->oz_ws_doubles = 0;
      BCK(cudaMalloc(&P->oz_ws, wd * sizeof(double)));
      P->oz_ws_doubles = wd;
    }
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, evt(P, EV_T0), evt(P, EV_CHOL));
  bs->ms_chol += ms;

  // caller's start vectors: Y1[:, :kprev] = L^H X_prev (step 0)
  GCall xcall;
  xcall.f = ZgemmGroupFlags{1, 0, 2, 0, 0, 0};
  if (X_prev && !o.cold_start)
    for (int k = 0; k < np; ++k)
      if (X_prev[k]) {
        const BDesc& d = P->hD[k];
        xcall.items.push_back(item((int)n[k], kprev[k], (int)n[k], d.L, n[k], (const double2*)X_prev[k], ldxp[k],
                                   d.Y1, d.m, d.flags));
      }
  if (!xcall.items.empty()) {
    xcall.tile = zgemm_group_tile(xcall.items.data(), (int)xcall.items.size());
    xcall.total = zgemm_group_layout(xcall.items.data(), (int)xcall.items.size(), xcall.tile);
    xcall.off = P->pool_items - np;
    BCK(cudaMemcpyAsync(P->pool + xcall.off, xcall.items.data(), xcall.items.size() * sizeof(ZgemmItem),
                        cudaMemcpyHostToDevice, s));
  }

  gevp_status overall = GEVP_OK;
  double maxres = 0.0;
  for (int l = 0; l < nsteps; ++l) {
    // ---- per-step pointers: A_{k,l} into the descriptors, the reduction and the final check
    for (int k = 0; k < np; ++k) {
      BDesc& d = P->hD[k];
      d.A = (const double2*)A[(size_t)k * nsteps + l];
      d.lda = lda[k];
      d.B = (const double2*)B[k];
      d.ldb = ldb[k];
      P->calls[P->c_red1].items[k].B = d.A;
      P->calls[P->c_red1].items[k].ldb = d.lda;
      P->calls[P->c_ax].items[k].A = d.A;
      P->calls[P->c_ax].items[k].lda = d.lda;
      P->calls[P->c_bx].items[k].A = d.B;
      P->calls[P->c_bx].items[k].lda = d.ldb;
      P->hDegcap[k] = P->cap_bucket[P->bucket[k]];
      BOut& ob = P->hOut[k];
      ob.lam = Lambda[k] + (size_t)l * nev[k];
      ob.res = resid[k] + (size_t)l * nev[k];
      ob.X = nullptr;
      ob.ldx = 0;
      if (X && X[k] && (o.keep_all_X || l == nsteps - 1)) {
        ob.X = (double2*)X[k] + (o.keep_all_X ? (size_t)l * n[k] * ldx[k] : 0);
        ob.ldx = ldx[k];
      }
    }
    BCK(cudaMemcpyAsync(P->dD, P->hD, np * sizeof(BDesc), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(P->dDegcap, P->hDegcap, np * sizeof(int), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(P->dOut, P->hOut, np * sizeof(BOut), cudaMemcpyHostToDevice, s));
    for (int c : {P->c_red1, P->c_ax, P->c_bx}) BCK(upload_call(P, P->calls[c], s));
    const bool tune = !P->tuned;
    BCK(cudaEventRecord(evt(P, EV_T0), s));
    bk_step_reset(P->dD, np, o.tol, tc ? 0 : 1, s);
    // ---- reduction C = L^-1 A L^-H for every k-point
    if (P->oz_S > 0) {
      // emulated: T = L^-1 tril_half(A), M = T L^-H per k-point (each product fills the GPU)
      for (int k = 0; k < np; ++k) {
        const BDesc& d = P->hD[k];
        const int nk_ = (int)n[k], S = P->oz_S;
        char* base = P->oz_scratch;
        BCK(oz_split(P->ozAB, base, nk_, nk_, d.A, d.lda, 1, 1, S, 3, P->oz_flags + 1, s));
        BCK(oz_gemm(P->ozLA[k], P->ozAB, 1, 1, d.T, n[k], P->oz_flags, s));
        BCK(oz_split(P->ozTA, base + oz_operand_bytes(nk_, nk_, S, 3), nk_, nk_, d.T, n[k], 0, 2, S, 2,
                     P->oz_flags + 1, s));
        BCK(oz_gemm(P->ozTA, P->ozLB[k], 1, 2, d.C, n[k], P->oz_flags, s));
      }
    } else {
      launch(P, P->c_red1, s, tune);
      launch(P, P->c_red2, s, tune);
    }
    bk_herm_sum(P->dD, np, P->nmax, s);
    if (P->oz_S > 0) {
      // the digits of every C for the rounds' W = C Q
      char* q = P->oz_cq;
      for (int k = 0; k < np; ++k) {
        const BDesc& d = P->hD[k];
        BCK(oz_split(P->ozC[k], q, (int)n[k], (int)n[k], d.C, n[k], 0, 0, P->oz_S, 2, P->oz_flags + 1, s));
        q += oz_operand_bytes((int)n[k], (int)n[k], P->oz_S, 2);
      }
    }
    BCK(cudaEventRecord(evt(P, EV_RED), s));
    // ---- bounds of C (and ||A||_2)
    bk_to_c32(P->dD, np, P->nmax, 0, s);
    bk_lanczos(P->dD, np, P->nmax, kl, 1, 0, o.seed + 7919ull * l, s);
    bk_to_c32(P->dD, np, P->nmax, 1, s);
    bk_lanczos(P->dD, np, P->nmax, kl, 0, 12, o.seed + 104729ull * l + 1, s);
    bk_post_bounds(P->dD, np, s);
    if (tc) tcg_set_matrix(P->dD, np, (int64_t)P->tg.n_pad_max * P->tg.n_pad_max, s);
    // ---- start block
    if (l == 0 || o.cold_start) {
      bk_randn(P->dD, np, nm_max, o.seed * 1000003ull + (uint64_t)l, nullptr, s);
      if (l == 0 && !xcall.items.empty())
        zgemm_grouped(P->pool + xcall.off, (int)xcall.items.size(), xcall.total, xcall.tile, xcall.f, s);
      enqueue_orth(P, s, tune);
    }
    enqueue_rr(P, s, tune);
    enqueue_status(P, s);
    BCK(cudaEventRecord(evt(P, EV_BND), s));
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(s));
    cudaEventElapsedTime(&ms, evt(P, EV_T0), evt(P, EV_RED));
    bs->ms_reduce += ms;
    cudaEventElapsedTime(&ms, evt(P, EV_RED), evt(P, EV_BND));
    bs->ms_bounds += ms;
    int rounds = 0;
    for (;;) {
      bool any_active = false, any_fail = false;
      for (int k = 0; k < np; ++k) {
        any_active |= (P->hStatus[k] & 1) != 0;
        any_fail |= (P->hStatus[k] & 2) != 0;
        P->hMask[k] = (P->hStatus[k] & 2) ? 1 : 0;
      }
      if (any_fail) {
        // a CholQR Gram matrix lost definiteness: restart those k-points from random
        // blocks (the others only repeat an orthonormalisation of orthonormal columns)
        BCK(cudaMemcpyAsync(P->dMask, P->hMask, np * sizeof(int), cudaMemcpyHostToDevice, s));
        bk_randn(P->dD, np, nm_max, o.seed * 7777ull + 131ull * rounds + l, P->dMask, s);
        enqueue_orth(P, s, false);
        enqueue_rr(P, s, false);
        enqueue_status(P, s);
        BCK(cudaStreamSynchronize(s));
        bs->orth_fallbacks++;
        if (++rounds > 4 * o.max_outer) break;
        continue;
      }
      if (!any_active) {
        // ---- original-space check of the k-points that converged
        BCK(cudaEventRecord(evt(P, EV_FIN0), s));
        if (P->oz_S > 0 && (int)P->ozLH.size() == np) {
          // emulated per k-point; launches of k-points without a pending check do nothing
          const int S = P->oz_S;
          for (int k = 0; k < np; ++k) {
            const BDesc& d = P->hD[k];
            const int* fin = d.flags + 12;
            BCK(oz_split(P->ozQ, P->oz_qs, d.nev, d.n, d.Q, d.m, 0, 0, S, 3, P->oz_flags + 1, s, true, fin));
            BCK(oz_gemm(P->ozLH[k], P->ozQ, 2, 0, d.Xf, d.m, P->oz_flags, s, fin, P->oz_ws, P->oz_ws_doubles));
            BCK(oz_split(P->ozAd, P->oz_ad, d.n, d.n, d.A, d.lda, 0, 0, S, 2, P->oz_flags + 1, s, false, fin));
            BCK(oz_split(P->ozQ, P->oz_qs, d.nev, d.n, d.Xf, d.m, 0, 0, S, 3, P->oz_flags + 1, s, true, fin));
            BCK(oz_gemm(P->ozAd, P->ozQ, 0, 0, d.Y1, d.m, P->oz_flags, s, fin, P->oz_ws, P->oz_ws_doubles));
            BCK(oz_gemm(P->ozBd[k], P->ozQ, 0, 0, d.Y2, d.m, P->oz_flags, s, fin, P->oz_ws, P->oz_ws_doubles));
          }
        } else {
          launch(P, P->c_xf, s, tune);
          launch(P, P->c_ax, s, tune);
          launch(P, P->c_bx, s, tune);
        }
        bk_final_check(P->dD, np, P->nevmax, s);
        bk_final_status(P->dD, np, P->dStatus, s);
        BCK(cudaMemcpyAsync(P->hStatus, P->dStatus, np * sizeof(int), cudaMemcpyDeviceToHost, s));
        BCK(cudaEventRecord(evt(P, EV_FIN1), s));
        BCK(cudaStreamSynchronize(s));
        cudaEventElapsedTime(&ms, evt(P, EV_FIN0), evt(P, EV_FIN1));
        bs->ms_final += ms;
        bool reopened = false;
        for (int k = 0; k < np; ++k) {
          if (P->hStatus[k] == 0) reopened = true;
          P->hStatus[k] = P->hStatus[k] == 0 ? 1 : 0;   // re-opened k-points are active again
        }
        if (!reopened) break;
        continue;
      }
      if (rounds >= o.max_outer) {
        // round cap: check what the active k-points have (they are not re-opened)
        bk_force_final(P->dD, np, s);
        for (int k = 0; k < np; ++k) P->hStatus[k] = 0;
        continue;
      }
      // ---- one lock-step round
      BCK(cudaEventRecord(evt(P, EV_RND0), s));
      if (P->gexec) {
        BCK(cudaGraphLaunch(P->gexec, s));
        bs->graph_replays++;
      } else if (!P->tuned || !P->measured) {
        // first round of a new shape: every grouped GEMM is timed with both tiles; second
        // round: the filter / rest split for the degree model; from the third on, the
        // round is captured once and replayed
        const bool tr_tune = !P->tuned;
        BCK(cudaEventRecord(evt(P, EV_F0), s));
        cudaError_t fe = enqueue_filter(P, s, tr_tune, o.deg_min);
        if (fe != cudaSuccess) return fail(fe, "batched filter launch");
        BCK(cudaEventRecord(evt(P, EV_F1), s));
        enqueue_orth(P, s, tr_tune);
        enqueue_rr(P, s, tr_tune);
        enqueue_status(P, s);
        BCK(cudaEventRecord(evt(P, EV_END), s));
        BCK(cudaStreamSynchronize(s));
        if (!tr_tune) {
          float tf = 0.f, tr = 0.f;
          cudaEventElapsedTime(&tf, evt(P, EV_F0), evt(P, EV_F1));
          cudaEventElapsedTime(&tr, evt(P, EV_F1), evt(P, EV_END));
          BCK(cudaMemcpy(P->hFlags, P->dFlags, (size_t)np * kNF * 4, cudaMemcpyDeviceToHost));
          int dmax = 1;
          for (int k = 0; k < np; ++k) dmax = std::max(dmax, P->hFlags[(size_t)k * kNF + 1]);
          P->t_step = tf / dmax;
          P->t_rest = tr;
          P->measured = true;
        }
        P->tuned = true;
      } else {
        // capture the round once: coefficients, filter, CholQR3, Rayleigh-Ritz, status
        cudaStream_t cs;
        BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
          cudaError_t fe = enqueue_filter(P, cs, false, o.deg_min);
          enqueue_orth(P, cs, false);
          enqueue_rr(P, cs, false);
          enqueue_status(P, cs);
          ce = cudaStreamEndCapture(cs, &P->graph);
          if (fe != cudaSuccess) ce = fe;
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&P->gexec, P->graph, 0);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) return fail(ce, "round graph capture");
        BCK(cudaGraphLaunch(P->gexec, s));
        bs->graph_replays++;
      }
      BCK(cudaEventRecord(evt(P, EV_RND1), s));
      BCK(cudaStreamSynchronize(s));
      BCK(cudaGetLastError());
      cudaEventElapsedTime(&ms, evt(P, EV_RND0), evt(P, EV_RND1));
      bs->ms_rounds += ms;
      rounds++;
      bs->rounds++;
      if (P->tc) {
        BCK(cudaMemcpy(P->hErr, P->dErr, sizeof(int), cudaMemcpyDeviceToHost));
        if (P->hErr[0]) {
          ctx_set_error(h, "batched tensor-core filter: a bounded wait expired");
          return GEVP_ERR_TIMEOUT;
        }
      }
    }
    bs->max_rounds_step = std::max(bs->max_rounds_step, rounds);
    // ---- outputs of this step
    bk_write_out(P->dD, P->dOut, np, (int64_t)P->nmax * P->nevmax, s);
    BCK(cudaMemcpyAsync(P->hBounds, P->dBounds, (size_t)np * kNB * 8, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(P->hFlags, P->dFlags, (size_t)np * kNF * 4, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    for (int k = 0; k < np; ++k) {
      const int* f = P->hFlags + (size_t)k * kNF;
      const double* bd = P->hBounds + (size_t)k * kNB;
      if (f[3] != 2) overall = GEVP_ERR_NO_CONVERGENCE;
      bs->switches += f[10];
      bs->final_passes += f[11];
      maxres = std::max(maxres, bd[18]);
      const double nn = (double)n[k], mm = (double)m[k];
      const int rr = f[4];
      bs->flops_fp64 += 4.0 * nn * nn * nn + rr * (8.0 * nn * nn * mm + 48.0 * nn * mm * mm) +
                        2.5 * 8.0 * nn * nn * nev[k] * std::max(1, f[11]);
      const double fl = 8.0 * nn * nn * mm * f[9];
      if (f[5] && !tc) bs->flops_fp64 += fl; else bs->flops_lowp += fl;
    }
    // ---- degree caps for the next step
    if (l + 1 < nsteps) tune_degrees(P, o);
  }
  BCK(cudaEventRecord(evt(P, EV_END), s));
  BCK(cudaStreamSynchronize(s));
  if (P->oz_S > 0) {
    int f[2] = {0, 0};
    BCK(cudaMemcpy(f, P->oz_flags, sizeof f, cudaMemcpyDeviceToHost));
    if (f[0]) {
      ctx_set_error(h, "a bounded wait of the emulated FP64 product ran out");
      return GEVP_ERR_TIMEOUT;
    }
  }
  bs->converged = overall == GEVP_OK ? 1 : 0;
  bs->max_resid = maxres;
  for (int c = 0; c < 8; ++c) bs->tile[c] = 0;
  for (auto& c : P->calls)
    if (c.cls < 8) bs->tile[c.cls] = c.tile;
  for (int b = 0; b < kBuckets; ++b) bs->deg_cap[b] = P->cap_bucket[b];
  bs->ms_total = bs->ms_chol + bs->ms_reduce + bs->ms_bounds + bs->ms_rounds + bs->ms_final;
  if (overall != GEVP_OK) ctx_set_error(h, "some residual stayed above tol");
  return overall;
#undef BCK
}
