// Grouped (ragged-batch) FP64 complex GEMM: one launch computes a list of independent
// products D_g = alpha_g op(A_g) op(B_g) + beta_g Cin_g + gamma_g Ein_g of different sizes
// (one per k-point problem of a batch). The host lays the tiles of all products out as one
// global tile list (prefix sums in ZgemmItem::tile_start); a persistent grid of CTAs walks
// that list, so small and large problems share the 152 SMs. Each item may point at a
// device flag: when it is zero the item's tiles are skipped (a converged problem), which
// keeps the launch shape fixed from one round to the next. The scalars may come from
// device memory (coef), so a launch sequence can be captured once and replayed.
#include "gevp_internal.cuh"
#include <algorithm>

namespace gevp {

namespace {

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
zgemm_group_kernel(const ZgemmItem* __restrict__ items, int nitems, int total_tiles, ZgemmGroupFlags f) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    // the item owning global tile t: the last item with tile_start <= t
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) / 2;
      if (items[mid].tile_start <= t) lo = mid; else hi = mid - 1;
    }
    const ZgemmItem& it = items[lo];
    if (it.active && *it.active == 0) continue;
    const int local = t - it.tile_start;
    const int m0 = (local / it.tiles_n) * BM, n0 = (local % it.tiles_n) * BN;
    if (f.triD == 1 && n0 > m0 + BM - 1) continue;
    int kb = 0, ke = it.K;
    if (f.triA == 1) ke = min(ke, m0 + BM);
    if (f.triA == 2) kb = max(kb, m0);
    if (f.triB == 1 || f.maskB) kb = max(kb, n0);
    if (f.triB == 2) ke = min(ke, n0 + BN);
    double2 acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
      for (int c = 0; c < TN; ++c) acc[r][c] = make_double2(0.0, 0.0);
    for (int k0 = kb; k0 < ke; k0 += BK) {
      for (int e = tid; e < BM * BK; e += NT) {
        int mm, kk;
        if (f.opA == 0) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
        int gm = m0 + mm, gk = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (gm < it.M && gk < ke) {
          if (f.opA == 0) v = it.A[(int64_t)gm * it.lda + gk];
          else v = zconj(it.A[(int64_t)gk * it.lda + gm]);
        }
        As[kk][mm] = v;
      }
      for (int e = tid; e < BK * BN; e += NT) {
        int kk, nn;
        if (f.opB == 0) { kk = e / BN; nn = e % BN; } else { nn = e / BK; kk = e % BK; }
        int gk = k0 + kk, gn = n0 + nn;
        double2 v = make_double2(0.0, 0.0);
        if (gn < it.N && gk < ke) {
          if (f.opB == 0) {
            v = it.B[(int64_t)gk * it.ldb + gn];
            if (f.maskB) {
              if (gk < gn) v = make_double2(0.0, 0.0);
              else if (gk == gn) v = zscale(v, 0.5);
            }
          } else {
            v = zconj(it.B[(int64_t)gn * it.ldb + gk]);
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
    double alpha = it.alpha, beta = it.beta, gamma = it.gamma;
    if (it.coef) {
      alpha = it.coef[0];
      beta = it.coef[1];
      gamma = it.coef[2];
    }
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      int gm = m0 + ty * TM + r;
      if (gm >= it.M) continue;
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        int gn = n0 + tx * TN + c;
        if (gn >= it.N) continue;
        double2 v = zscale(acc[r][c], alpha);
        if (it.Cin) {
          double2 cv = it.Cin[(int64_t)gm * it.ldc + gn];
          v.x = fma(beta, cv.x, v.x);
          v.y = fma(beta, cv.y, v.y);
        }
        if (it.Ein) {
          double2 ev = it.Ein[(int64_t)gm * it.lde + gn];
          v.x = fma(gamma, ev.x, v.x);
          v.y = fma(gamma, ev.y, v.y);
        }
        it.D[(int64_t)gm * it.ldd + gn] = v;
      }
    }
  }
}

}  // namespace

int zgemm_group_tile(const ZgemmItem* items_host, int nitems) {
  // 32 x 32 tiles unless every product is large enough for 64 x 64 to fill the SMs
  int64_t t64 = 0;
  for (int i = 0; i < nitems; ++i)
    t64 += (int64_t)((items_host[i].M + 63) / 64) * ((items_host[i].N + 63) / 64);
  return t64 >= 4 * 152 ? 64 : 32;
}

int zgemm_group_layout(ZgemmItem* items_host, int nitems, int tile) {
  int total = 0;
  for (int i = 0; i < nitems; ++i) {
    ZgemmItem& it = items_host[i];
    it.tiles_n = (it.N + tile - 1) / tile;
    int tm = (it.M + tile - 1) / tile;
    it.tile_start = total;
    total += (it.M > 0 && it.N > 0) ? tm * it.tiles_n : 0;
  }
  return total;
}

void zgemm_grouped(const ZgemmItem* items_dev, int nitems, int total_tiles, int tile, const ZgemmGroupFlags& f,
                   cudaStream_t s) {
  if (total_tiles <= 0 || nitems <= 0) return;
  int grid = std::min(total_tiles, 152 * 4);
  if (tile == 64) zgemm_group_kernel<64, 64, 8, 4, 4><<<grid, 256, 0, s>>>(items_dev, nitems, total_tiles, f);
  else zgemm_group_kernel<32, 32, 8, 2, 2><<<grid, 256, 0, s>>>(items_dev, nitems, total_tiles, f);
  LAUNCH_NOTE(1);
}

}  // namespace gevp
