// FP64 complex GEMM with fused three-term epilogue, triangular k-tile skipping, split-K
// and uniform batching. On this part FP64 issues at about 1.7 FMA per clock per SM, so
// the kernel is bound by the FP64 pipe at every shape used here; what matters is that
// every one of the 152 SMs is busy, which the host-side tiling choice below arranges
// (tile size and split-K picked so that the grid covers the SMs in full waves).
#include "gevp_internal.cuh"
#include <algorithm>
#include <cmath>

namespace gevp {

namespace {

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
zgemm_kernel(ZgemmArgs p, double2* ws) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int z = blockIdx.z;
  const int b = z / p.ksplit, slice = z % p.ksplit;

  if (p.triD == 1 && n0 > m0 + BM - 1) return;

  const double2* A = p.A + (int64_t)b * p.sA;
  const double2* B = p.B + (int64_t)b * p.sB;

  int kb = 0, ke = p.K;
  if (p.triA == 1) ke = min(ke, m0 + BM);
  if (p.triA == 2) kb = max(kb, m0);
  if (p.triB == 1 || p.maskB) kb = max(kb, n0);
  if (p.triB == 2) ke = min(ke, n0 + BN);
  if (p.ksplit > 1) {
    int len = ke > kb ? ke - kb : 0;
    int per = ((len + p.ksplit - 1) / p.ksplit + BK - 1) / BK * BK;
    int s0 = kb + slice * per;
    int s1 = min(ke, s0 + per);
    kb = s0;
    ke = s1;
  }

  double2 acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = make_double2(0.0, 0.0);

  for (int k0 = kb; k0 < ke; k0 += BK) {
    // ---- load op(A) tile (BM x BK) into As[k][m]
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (p.opA == 0) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      int gm = m0 + mm, gk = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (gm < p.M && gk < ke) {
        if (p.opA == 0) v = A[(int64_t)gm * p.lda + gk];
        else v = zconj(A[(int64_t)gk * p.lda + gm]);
      }
      As[kk][mm] = v;
    }
    // ---- load op(B) tile (BK x BN) into Bs[k][n]
    for (int e = tid; e < BK * BN; e += NT) {
      int kk, nn;
      if (p.opB == 0) { kk = e / BN; nn = e % BN; } else { nn = e / BK; kk = e % BK; }
      int gk = k0 + kk, gn = n0 + nn;
      double2 v = make_double2(0.0, 0.0);
      if (gn < p.N && gk < ke) {
        if (p.opB == 0) {
          v = B[(int64_t)gk * p.ldb + gn];
          if (p.maskB) {
            if (gk < gn) v = make_double2(0.0, 0.0);
            else if (gk == gn) v = zscale(v, 0.5);
          }
        } else {
          v = zconj(B[(int64_t)gn * p.ldb + gk]);
        }
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[TM], bb[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) a[r] = As[kk][ty * TM + r];
#pragma unroll
      for (int c = 0; c < TN; ++c) bb[c] = Bs[kk][tx * TN + c];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) zfma(acc[r][c], a[r], bb[c]);
    }
    __syncthreads();
  }

  if (p.ksplit > 1) {
    double2* out = ws + ((int64_t)b * p.ksplit + slice) * (int64_t)p.M * p.N;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      int gm = m0 + ty * TM + r;
      if (gm >= p.M) continue;
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        int gn = n0 + tx * TN + c;
        if (gn < p.N) out[(int64_t)gm * p.N + gn] = acc[r][c];
      }
    }
    return;
  }
  double2* D = p.D + (int64_t)b * p.sD;
  const double2* Cin = p.Cin ? p.Cin + (int64_t)b * p.sC : nullptr;
  const double2* Ein = p.Ein ? p.Ein + (int64_t)b * p.sE : nullptr;
#pragma unroll
  for (int r = 0; r < TM; ++r) {
    int gm = m0 + ty * TM + r;
    if (gm >= p.M) continue;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      int gn = n0 + tx * TN + c;
      if (gn >= p.N) continue;
      double2 v = zscale(acc[r][c], p.alpha);
      if (Cin) {
        double2 cv = Cin[(int64_t)gm * p.ldc + gn];
        v.x = fma(p.beta, cv.x, v.x);
        v.y = fma(p.beta, cv.y, v.y);
      }
      if (Ein) {
        double2 ev = Ein[(int64_t)gm * p.lde + gn];
        v.x = fma(p.gamma, ev.x, v.x);
        v.y = fma(p.gamma, ev.y, v.y);
      }
      D[(int64_t)gm * p.ldd + gn] = v;
    }
  }
}

// Sum the k-slices in a fixed order (deterministic) and apply the epilogue.
__global__ void zgemm_reduce_kernel(ZgemmArgs p, const double2* ws, int BM, int BN) {
  int64_t total = (int64_t)p.M * p.N;
  int b = blockIdx.y;
  double2* D = p.D + (int64_t)b * p.sD;
  const double2* Cin = p.Cin ? p.Cin + (int64_t)b * p.sC : nullptr;
  const double2* Ein = p.Ein ? p.Ein + (int64_t)b * p.sE : nullptr;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int gm = (int)(e / p.N), gn = (int)(e % p.N);
    if (p.triD == 1 && (gn / BN) * BN > (gm / BM) * BM + BM - 1) continue;
    double2 s = make_double2(0.0, 0.0);
    const double2* w = ws + (int64_t)b * p.ksplit * total + e;
    for (int z = 0; z < p.ksplit; ++z) s = zadd(s, w[(int64_t)z * total]);
    double2 v = zscale(s, p.alpha);
    if (Cin) {
      double2 cv = Cin[(int64_t)gm * p.ldc + gn];
      v.x = fma(p.beta, cv.x, v.x);
      v.y = fma(p.beta, cv.y, v.y);
    }
    if (Ein) {
      double2 ev = Ein[(int64_t)gm * p.lde + gn];
      v.x = fma(p.gamma, ev.x, v.x);
      v.y = fma(p.gamma, ev.y, v.y);
    }
    D[(int64_t)gm * p.ldd + gn] = v;
  }
}

constexpr int kSMs = 152;

}  // namespace

ZgemmArgs zg(int M, int N, int K, const double2* A, int64_t lda, int opA, const double2* B, int64_t ldb, int opB,
             double2* D, int64_t ldd, double alpha) {
  ZgemmArgs a{};
  a.M = M; a.N = N; a.K = K;
  a.A = A; a.lda = lda; a.opA = opA;
  a.B = B; a.ldb = ldb; a.opB = opB;
  a.D = D; a.ldd = ldd; a.alpha = alpha;
  a.Cin = nullptr; a.ldc = 0; a.beta = 0.0;
  a.Ein = nullptr; a.lde = 0; a.gamma = 0.0;
  a.triA = a.triB = a.triD = a.maskB = 0;
  a.ksplit = 1; a.batch = 1;
  a.sA = a.sB = a.sD = a.sC = a.sE = 0;
  return a;
}

void zgemm(const ZgemmArgs& in, double2* split_ws, size_t split_ws_elems, cudaStream_t s) {
  ZgemmArgs p = in;
  if (p.M <= 0 || p.N <= 0) return;
  if (p.batch < 1) p.batch = 1;
  // Every SM has the same (slow) FP64 pipe, so time ~ the busiest SM's share of FMAs.
  // For each tile size (64, 32, 16) and split-K factor, estimate
  //   waves = ceil(active_tiles * ksplit / SMs),  cost = waves * bm * bn * (K / ksplit)
  // and take the cheapest (ties to larger tiles, which cost fewer shared-memory reads).
  auto active_tiles = [&](int bm, int bn) {
    int64_t tm = (p.M + bm - 1) / bm, tn = (p.N + bn - 1) / bn;
    int64_t t = tm * tn;
    if (p.triD == 1) {
      t = 0;
      for (int64_t i = 0; i < tm; ++i) t += std::min<int64_t>(tn, (i * bm + bm - 1) / bn + 1);
    }
    return t * p.batch;
  };
  const int sizes[3] = {64, 32, 16};
  int best_b = 64, best_ks = 1;
  double best_cost = 1e300;
  int kmax_split = (p.ksplit > 0 ? p.ksplit : 1);
  for (int si = 0; si < 3; ++si) {
    int b = sizes[si];
    int64_t t = active_tiles(b, b);
    for (int ks = 1; ks <= 64; ks *= 2) {
      if (ks > 1) {
        if (p.ksplit > 1 || !split_ws) break;
        if (p.K / ks < 64) break;
        if ((size_t)ks * p.M * p.N * p.batch > split_ws_elems) break;
      }
      int ksu = (p.ksplit > 1) ? kmax_split : ks;
      double waves = std::ceil((double)(t * ksu) / kSMs);
      double kslice = std::ceil((double)std::max(p.K, 1) / ksu);
      double cost = waves * b * b * kslice + (ksu > 1 ? 0.02 * (double)p.M * p.N * ksu / kSMs : 0.0);
      if (cost < best_cost * 0.97) {
        best_cost = cost;
        best_b = b;
        best_ks = ksu;
      }
      if (p.ksplit > 1) break;
    }
  }
  p.ksplit = best_ks;
  int bm = best_b, bn = best_b;
  dim3 grid((p.N + bn - 1) / bn, (p.M + bm - 1) / bm, p.batch * p.ksplit);
  void* kt0 = kt_enabled() ? kt_begin(s) : nullptr;
  if (bm == 64) zgemm_kernel<64, 64, 8, 4, 4><<<grid, 256, 0, s>>>(p, split_ws);
  else if (bm == 32) zgemm_kernel<32, 32, 8, 2, 2><<<grid, 256, 0, s>>>(p, split_ws);
  else zgemm_kernel<16, 16, 16, 1, 1><<<grid, 256, 0, s>>>(p, split_ws);
  LAUNCH_NOTE(1);
  if (kt0) {
    const int tb = p.maskB ? 1 : p.triB;
    const double f = p.batch * tiled_product_flops(p.M, p.N, p.K, p.triA, tb, p.triD);
    kt_end(kt0, 0, f, f, s);
  }
  if (p.ksplit > 1) {
    int64_t total = (int64_t)p.M * p.N;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 4 * kSMs);
    zgemm_reduce_kernel<<<dim3(blocks, p.batch), 256, 0, s>>>(p, split_ws, bm, bn);
    LAUNCH_NOTE(1);
  }
}

// Scaled Chebyshev filter (Zhou, Saad, Tiago & Chelikowsky 2006) with FP64 products: Y0
// (n x ma, ld ld0) through deg steps of the three-term recurrence, each step one complex
// GEMM with the recurrence fused into its epilogue, ping-ponging between B1 and B2 (ld
// ldb); returns the buffer holding the result. split_ws may be null (no split-K).
double2* cheb_filter_fp64(int64_t n, const double2* C, int64_t ldc, const double2* Y0, int64_t ld0, int ma, int deg,
                          double lo, double hi, double sc, double2* B1, double2* B2, int64_t ldb, double2* split_ws,
                          size_t split_elems, cudaStream_t s) {
  double e = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
  double sigma = e / (sc - c), sigma1 = sigma;
  ZgemmArgs a = zg((int)n, ma, (int)n, C, ldc, 0, Y0, ld0, 0, B1, ldb, sigma1 / e);
  a.Cin = Y0; a.ldc = ld0; a.beta = -c * sigma1 / e;
  zgemm(a, split_ws, split_elems, s);
  const double2* prev = Y0;
  int64_t ldp = ld0;
  double2* cur = B1;
  double2* nxt = B2;
  for (int i = 2; i <= deg; ++i) {
    double sn = 1.0 / (2.0 / sigma1 - sigma);
    double al = 2.0 * sn / e;
    ZgemmArgs g = zg((int)n, ma, (int)n, C, ldc, 0, cur, ldb, 0, nxt, ldb, al);
    g.Cin = cur; g.ldc = ldb; g.beta = -al * c;
    g.Ein = prev; g.lde = ldp; g.gamma = -sigma * sn;
    zgemm(g, split_ws, split_elems, s);
    sigma = sn;
    double2* old = cur;
    prev = old;
    ldp = ldb;
    cur = nxt;
    nxt = old;   // overwrites the step before 'cur' next time (allowed: read-then-write per element)
  }
  return cur;
}

}  // namespace gevp
