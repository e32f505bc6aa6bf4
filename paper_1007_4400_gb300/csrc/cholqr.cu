// Tall-skinny kernels of the orthonormalisation (CholQR) and the Rayleigh-Ritz projection.
//
// zgram: G = X^H Y for n x mx and n x my blocks with n >> m (the Gram matrix Y^H Y of
//   CholQR, the projection Q^H W of Rayleigh-Ritz, the overlaps Q_lock^H Y). On this part
//   one SM retires about 1.7 FP64 FMAs per clock, so the product is FP64-pipe bound and
//   the whole job is to keep all 152 SMs busy with little else: the m x m result is cut
//   into 16 x 16 tiles (only the lower ones when the result is Hermitian, half the
//   flops), n into slices so that the CTAs cover the SMs several times over, and the
//   slices of a tile are summed in slice order by whichever CTA of that tile finishes
//   last (a per-tile arrival counter), so there is no second launch and the sum is
//   deterministic. A Hermitian result is written to both triangles.
//
// cholinv: the Cholesky factor L of D W D + shift I (W the Gram matrix, lower triangle
//   read; D = diag(W)^-1/2 the column scaling of CholQR) and its inverse, for m up to a
//   few hundred, in the CTAs of one thread-block cluster. A one-CTA factorisation would
//   take close to a millisecond at m = 140 (m^3/3 complex multiply-adds at two FP64 FMAs
//   per clock); the blocked right-looking form over all SMs spends most of its time in
//   launches and serial diagonal blocks. Here the rows are dealt cyclically to the P CTAs
//   (row i to CTA i mod P) and held in shared memory with the rows of the inverse; column
//   j of the factor and row j of the inverse are exchanged through distributed shared
//   memory, one cluster barrier per column:
//     step j: every CTA reads the pivot a_jj, the column A[j+1:m, j] and the row S[j, 0:j]
//     (values final after step j-1), then updates its own rows i > j:
//       A[i, e] -= A[i, j] conj(A[e, j]) / a_jj   (j < e <= i; the trailing Cholesky update)
//       S[i, e] -= A[i, j] S[j, e] / a_jj         (e <= j; the inverse, L X = I, right-looking)
//     L[i, j] = A[i, j] / sqrt(a_jj) and (L^-1)[i, e] = S[i, e] / sqrt(a_ii) are read off at
//     the end. Within a step the reads (column j, row j, the pivot) and the writes
//     (columns > j of A, rows > j of S) never meet, so one barrier per step suffices. The
//     barrier is split: a step first updates what the next step reads (column j + 1 with
//     the next pivot, row j + 1 of S), arrives, updates the rest while the other CTAs catch
//     up, and waits only before the next gather; the gathered values are double-buffered,
//     so a thread gathering step j + 1 never overwrites what another still reads for j.
//   The output Li = L^-1 D (columns scaled by D) makes Y Li^H = Y D L^-H, the orthonormal
//   factor of one CholQR pass, a single product; it is also the inverse of D^-1 L, the
//   Cholesky factor of W itself (shift 0), which is written out on request (the leaves
//   of the recursive factorisation of B). A non-positive pivot stops the cluster (every
//   CTA reads the same pivot, so the decision is uniform) and sets *info to its 1-based
//   index plus a caller's offset. W may share memory with that factor's output: every
//   CTA reads its rows of W before the first cluster barrier and writes the factor after
//   the last.
#include "gevp_internal.cuh"
#include <cooperative_groups.h>
#include <algorithm>

namespace gevp {

namespace {

constexpr int GT = 16;   // zgram output tile edge
constexpr int GK = 16;   // rows staged per step

__global__ void __launch_bounds__(256) zgram_kernel(int64_t n, int mx, int my, const double2* __restrict__ X,
                                                    int64_t ldx, const double2* __restrict__ Y, int64_t ldy,
                                                    double2* G, int64_t ldg, int herm, int ntj, int slices,
                                                    int64_t per, double2* part, unsigned* cnt) {
  __shared__ double2 Xs[GK][GT];
  __shared__ double2 Ys[GK][GT];
  __shared__ int last;
  const int tile = blockIdx.x;
  const int ti = tile / ntj, tj = tile % ntj;
  if (herm && tj > ti) return;
  const int slice = blockIdx.y;
  const int tid = threadIdx.x;
  const int ty = tid / GT, tx = tid % GT;
  const int64_t k0 = (int64_t)slice * per;
  const int64_t k1 = min(n, k0 + per);
  const int lr = tid / GT, lc = tid % GT;   // staging: row lr, column lc of the tile
  const int xc = ti * GT + lc, yc = tj * GT + lc;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t k = k0; k < k1; k += GK) {
    const int64_t kr = k + lr;
    Xs[lr][lc] = (kr < k1 && xc < mx) ? X[kr * ldx + xc] : make_double2(0.0, 0.0);
    Ys[lr][lc] = (kr < k1 && yc < my) ? Y[kr * ldy + yc] : make_double2(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) zfma(acc, zconj(Xs[kk][ty]), Ys[kk][tx]);
    __syncthreads();
  }
  const int i = ti * GT + ty, j = tj * GT + tx;
  if (slices > 1) {
    part[((int64_t)tile * slices + slice) * (GT * GT) + tid] = acc;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&cnt[tile], 1u) == (unsigned)(slices - 1));
    __syncthreads();
    if (!last) return;
    __threadfence();
    acc = make_double2(0.0, 0.0);
    const double2* p = part + (int64_t)tile * slices * (GT * GT) + tid;
    for (int s = 0; s < slices; ++s) acc = zadd(acc, __ldcg(p + (int64_t)s * (GT * GT)));
    if (tid == 0) cnt[tile] = 0u;   // ready for the next launch (stream order)
  }
  if (i >= mx || j >= my) return;
  if (!herm) {
    G[(int64_t)i * ldg + j] = acc;
    return;
  }
  if (j > i) return;   // the diagonal tile's upper half comes from the lower one
  if (j == i) {
    G[(int64_t)i * ldg + i] = make_double2(acc.x, 0.0);
  } else {
    G[(int64_t)i * ldg + j] = acc;
    G[(int64_t)j * ldg + i] = zconj(acc);
  }
}

constexpr int CT = 256;          // threads per cholinv CTA
constexpr int kCholInvMax = 288; // largest order (shared-memory bound at 16 CTAs)

// split cluster barrier: arrive (release) and, later, wait (acquire) for the phase
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

template <int P>
__global__ void __launch_bounds__(CT, 1) cholinv_cluster_kernel(int m, const double2* W, int64_t ldw,
                                                                double shift, double2* Li, int64_t ldi,
                                                                double2* Lf, int64_t ldl, int* info, int info_base) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double2 csm[];
  // gathered values of step j in buffer j & 1: a thread may gather step j + 1 while another
  // still finishes step j's update
  __shared__ double2 cbuf[2][kCholInvMax];   // column j of A (raw), rows > j
  __shared__ double2 xbuf[2][kCholInvMax];   // row j of S (raw), columns <= j
  __shared__ double2 cs[2][kCholInvMax / 8]; // own rows' -A[i, j] / a_jj
  __shared__ double dsc[kCholInvMax];     // D
  __shared__ double piv[kCholInvMax];     // sqrt(a_jj)
  __shared__ double2 pinfo[kCholInvMax / 8];   // own rows: (pivot a_ii, rsqrt(a_ii)) once final
  __shared__ double2* rA[P];
  __shared__ double2* rS[P];
  __shared__ double2* rPI[P];
  __shared__ double apiv;
  const int tid = threadIdx.x;
  const int rank = (int)cl.block_rank();
  const int R = (m + P - 1) / P;
  double2* Arow = csm;            // [R][m]: own rows i = rank + P t of the matrix being factored
  double2* Srow = csm + R * m;    // [R][m]: own rows of the inverse's accumulator
  if (tid < P) {
    rA[tid] = cl.map_shared_rank(Arow, tid);
    rS[tid] = cl.map_shared_rank(Srow, tid);
    rPI[tid] = cl.map_shared_rank(pinfo, tid);
  }
  for (int i = tid; i < m; i += CT) {
    const double v = W[(int64_t)i * ldw + i].x;
    dsc[i] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
  }
  __syncthreads();
  for (int e = tid; e < R * m; e += CT) {
    const int t = e / m, c = e % m, i = rank + P * t;
    double2 a = make_double2(0.0, 0.0), s = make_double2(0.0, 0.0);
    if (i < m && c <= i) {
      a = zscale(W[(int64_t)i * ldw + c], dsc[i] * dsc[c]);
      if (c == i) a = make_double2(a.x + shift, 0.0);
      if (c == i) s = make_double2(1.0, 0.0);
    }
    Arow[e] = a;
    Srow[e] = s;
  }
  // the first pivot is final from the start: its owner (rank 0, local row 0; this thread
  // wrote that entry above) prepares its reciprocal square root
  if (rank == 0 && tid == 0) {
    const double a0 = Arow[0].x;
    pinfo[0] = make_double2(a0, a0 > 0.0 ? rsqrt(a0) : 0.0);
  }
  cl.sync();
  bool failed = false;
  for (int j = 0; j < m; ++j) {
    const int oj = j % P, tjj = j / P, bsel = j & 1;
    double2* cb = cbuf[bsel];
    double2* xb = xbuf[bsel];
    double2* cm = cs[bsel];
    // own rows below the pivot: i = rank + P t > j, t in [t0, t1)
    const int t0 = j >= rank ? (j - rank) / P + 1 : 0;
    int t1 = R;
    while (t1 > t0 && rank + P * (t1 - 1) >= m) --t1;
    const int nr = t1 - t0;
    // everything step j reads is final once every CTA has arrived after step j - 1's
    // first part (column j, row j of the inverse, the pivot)
    if (j > 0) cluster_wait();
    // gather column j and row j of the inverse (raw values); the threads of own rows also
    // form the row's multiplier -A[i][j] / a_jj from the pivot's reciprocal square root,
    // prepared by the pivot's owner when it became final
    for (int l = tid; l < m; l += CT) {
      if (l > j) {
        const double2 c = rA[l % P][(l / P) * m + j];
        cb[l] = c;
        if (l % P == rank) {
          const double ri = rPI[oj][tjj].y;
          cm[l / P - t0] = zscale(c, -(ri * ri));
        }
      } else {
        xb[l] = rS[oj][tjj * m + l];
      }
    }
    if (tid == 0) {
      const double2 pv = rPI[oj][tjj];
      apiv = pv.x;
      piv[j] = pv.x * pv.y;
    }
    __syncthreads();
    const double a = apiv;   // the same value in every CTA: a uniform decision
    if (!(a > 0.0)) {
      if (rank == 0 && tid == 0) atomicCAS(info, 0, info_base + j + 1);
      failed = true;
      break;
    }
    // first part: what step j + 1 reads. Column j + 1 of the own rows below the pivot (with
    // the next pivot and its reciprocal square root), and row j + 1 of the inverse if it is
    // an own row
    const int own_next = ((j + 1) % P == rank && j + 1 < m) ? (j + 1) / P : -1;
    const int nfirst = nr + (own_next >= 0 ? j + 1 : 0);
    for (int q = tid; q < nfirst; q += CT) {
      if (q < nr) {
        const int t = t0 + q, e = j + 1;
        double2 v = Arow[t * m + e];
        zfma(v, cm[q], zconj(cb[e]));
        Arow[t * m + e] = v;
        if (rank + P * t == j + 1) pinfo[t] = make_double2(v.x, v.x > 0.0 ? rsqrt(v.x) : 0.0);
      } else {
        const int e = q - nr, t = own_next;
        double2 v = Srow[t * m + e];
        zfma(v, cm[t - t0], xb[e]);
        Srow[t * m + e] = v;
      }
    }
    cluster_arrive();
    // the rest of the update, while the other CTAs finish their first parts
    for (int idx = tid; idx < nr * m; idx += CT) {
      const int tt = idx / m, e = idx % m, t = t0 + tt, i = rank + P * t;
      if (e > i || e == j + 1 || (i == j + 1 && e <= j)) continue;
      const double2 li = cm[tt];
      if (e <= j) {
        double2 v = Srow[t * m + e];
        zfma(v, li, xb[e]);
        Srow[t * m + e] = v;
      } else {
        double2 v = Arow[t * m + e];
        zfma(v, li, zconj(cb[e]));
        Arow[t * m + e] = v;
      }
    }
  }
  if (failed) {
    cl.sync();   // no CTA leaves while another may still read its shared memory
    return;
  }
  cluster_wait();   // the last step's gathers are over in every CTA
  __syncthreads();  // and every thread of this one finished its update
  // read off L and L^-1 D for the own rows
  for (int e = tid; e < R * m; e += CT) {
    const int t = e / m, c = e % m, i = rank + P * t;
    if (i >= m) continue;
    double2 x = make_double2(0.0, 0.0);
    if (c <= i) x = zscale(Srow[e], dsc[c] / piv[i]);
    Li[(int64_t)i * ldi + c] = x;
    if (Lf) {
      // the factor of W + shift D^-2: D^-1 times the factor of D W D + shift I
      double2 l = make_double2(0.0, 0.0);
      if (c < i) l = zscale(Arow[e], 1.0 / (piv[c] * dsc[i]));
      else if (c == i) l = make_double2(piv[i] / dsc[i], 0.0);
      Lf[(int64_t)i * ldl + c] = l;
    }
  }
}

template <int P>
size_t cholinv_smem(int m) {
  return (size_t)2 * ((m + P - 1) / P) * m * sizeof(double2);
}

template <int P>
bool cholinv_launch(int m, const double2* W, int64_t ldw, double shift, double2* Li, int64_t ldi, double2* Lf,
                    int64_t ldl, int* info, int info_base, cudaStream_t s) {
  const size_t smem = cholinv_smem<P>(m);
  if (smem > 200 * 1024) return false;
  static int ready = 0;   // 0 unknown, 1 usable, -1 not launchable on this device
  if (ready < 0) return false;
  if (ready == 0) {
    ready = -1;
    if (P > 8 && cudaFuncSetAttribute(cholinv_cluster_kernel<P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                     cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaFuncSetAttribute(cholinv_cluster_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t probe = {};
    probe.gridDim = dim3(P, 1, 1);
    probe.blockDim = dim3(CT, 1, 1);
    probe.dynamicSmemBytes = 200 * 1024;
    cudaLaunchAttribute pa[1];
    pa[0].id = cudaLaunchAttributeClusterDimension;
    pa[0].val.clusterDim.x = P;
    pa[0].val.clusterDim.y = 1;
    pa[0].val.clusterDim.z = 1;
    probe.attrs = pa;
    probe.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, cholinv_cluster_kernel<P>, &probe) != cudaSuccess ||
        nclusters < 1) {
      cudaGetLastError();
      return false;
    }
    ready = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P, 1, 1);
  cfg.blockDim = dim3(CT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, cholinv_cluster_kernel<P>, m, W, ldw, shift, Li, ldi, Lf, ldl, info, info_base) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  LAUNCH_NOTE(1);
  return true;
}

constexpr int kSMs = 152;

}  // namespace

int cholinv_max_order() { return kCholInvMax; }

bool cholinv_small(int m, const double2* W, int64_t ldw, double shift, double2* Li, int64_t ldi, double2* Lf,
                   int64_t ldl, int* info, cudaStream_t s, int info_base) {
  if (m < 1 || m > kCholInvMax) return false;
  if (cholinv_launch<16>(m, W, ldw, shift, Li, ldi, Lf, ldl, info, info_base, s)) return true;
  return cholinv_launch<8>(m, W, ldw, shift, Li, ldi, Lf, ldl, info, info_base, s);
}

namespace {

// The recursion of chol_recursive: a block of order n splits as n1 + n2 (n1 a multiple of
// 128 near n / 2):
//   [A11 .  ]   [L11  .  ] [L11^H L21^H]
//   [A21 A22] = [L21 L22 ] [  .   L22^H],   L21 = A21 L11^-H,  A22 - L21 L21^H = L22 L22^H,
//   (L^-1)21 = -L22^-1 L21 L11^-1,
// the four off-diagonal products emulated, leaves of order <= kCholLeaf factored and
// inverted in one cluster launch each.
struct CholRec {
  const CholRes& r;
  cudaError_t err = cudaSuccess;

  bool product(OzOperand& a, OzOperand& b, int triA, int triB, double2* D, int64_t ldd) {
    const bool ws = r.ws && oz_split_k_doubles(a.rows, b.rows) <= r.ws_doubles;
    err = oz_gemm(a, b, triA, triB, D, ldd, r.flags, r.s, nullptr, ws ? r.ws : nullptr, ws ? r.ws_doubles : 0);
    return err == cudaSuccess;
  }
  bool split(OzOperand& op, bool roleA, int rows, int K, const double2* X, int64_t ldx, int conj, int mask,
             bool cols) {
    err = oz_split(op, roleA ? r.memA : r.memB, rows, K, X, ldx, conj, mask, r.S, roleA ? 2 : 3, r.flags + 1, r.s,
                   cols);
    return err == cudaSuccess;
  }
  // false with err == cudaSuccess: a leaf could not be launched (nothing enqueued if k0 == 0)
  bool run(int64_t n, double2* A, int64_t lda, double2* Li, int64_t ldi, int64_t k0) {
    if (n <= kCholLeaf) return cholinv_small((int)n, A, lda, 0.0, Li, ldi, A, lda, r.info, r.s, (int)k0);
    const int64_t n1 = std::max<int64_t>(128, (n / 2) / 128 * 128), n2 = n - n1;
    double2 *A21 = A + n1 * lda, *A22 = A21 + n1, *Li21 = Li + n1 * ldi, *Li22 = Li21 + n1;
    OzOperand a, b;
    const int i1 = (int)n1, i2 = (int)n2;
    if (!run(n1, A, lda, Li, ldi, k0)) return false;
    // L21 = A21 L11^-H: the columns of L11^-H are the conjugated rows of L11^-1 (k <= j)
    if (!split(a, true, i2, i1, A21, lda, 0, 0, false) || !split(b, false, i1, i1, Li, ldi, 1, 2, false) ||
        !product(a, b, 0, 2, A21, lda))
      return false;
    // A22 -= L21 L21^H (lower triangle), the product through the scratch T
    if (!split(a, true, i2, i1, A21, lda, 0, 0, false) || !split(b, false, i2, i1, A21, lda, 1, 0, false) ||
        !product(a, b, 0, 0, r.T, r.ldt))
      return false;
    zsub_lower(n2, A22, lda, r.T, r.ldt, r.s);
    if (!run(n2, A22, lda, Li22, ldi, k0 + n1)) {
      if (err == cudaSuccess) err = cudaErrorLaunchFailure;   // the first leaf launched: this one should too
      return false;
    }
    // T = L21 L11^-1 (the columns of the lower L11^-1 from their diagonal down), then
    // (L^-1)21 = -L22^-1 T
    if (!split(a, true, i2, i1, A21, lda, 0, 0, false) || !split(b, false, i1, i1, Li, ldi, 0, 3, true) ||
        !product(a, b, 0, 1, r.T, r.ldt))
      return false;
    if (!split(a, true, i2, i2, Li22, ldi, 0, 2, false) || !split(b, false, i1, i2, r.T, r.ldt, 0, 0, true) ||
        !product(a, b, 1, 0, Li21, ldi))
      return false;
    zneg(n2, n1, Li21, ldi, r.s);
    return true;
  }
};

}  // namespace

cudaError_t chol_recursive(int64_t n, double2* A, int64_t lda, double2* Li, int64_t ldi, const CholRes& r) {
  if (n < 1 || cholinv_max_order() < kCholLeaf) return cudaErrorNotSupported;
  if (n > kCholLeaf) zero_upper(n, Li, ldi, r.s);   // the leaves and products fill the lower part
  CholRec rec{r};
  if (!rec.run(n, A, lda, Li, ldi, 0)) return rec.err == cudaSuccess ? cudaErrorNotSupported : rec.err;
  if (n > kCholLeaf) zero_upper(n, A, lda, r.s);
  return cudaSuccess;
}

size_t zgram_counters() { return 4096; }

void zgram(int64_t n, int mx, int my, const double2* X, int64_t ldx, const double2* Y, int64_t ldy, double2* G,
           int64_t ldg, int herm, double2* part, size_t part_elems, unsigned* cnt, cudaStream_t s) {
  if (mx <= 0 || my <= 0) return;
  const int nti = (mx + GT - 1) / GT, ntj = (my + GT - 1) / GT;
  const int64_t tiles = (int64_t)nti * ntj;
  const int64_t active = herm ? (int64_t)nti * (nti + 1) / 2 : tiles;
  // slices: about eight CTAs per SM over the active tiles (the FP64 pipe is the limit, so
  // the point is an even spread), at least 2 GK rows each, within the partials' room and
  // the counters
  int64_t slices = (8 * kSMs + active - 1) / active;
  slices = std::min<int64_t>(slices, std::max<int64_t>(1, n / (2 * GK)));
  if (tiles > (int64_t)zgram_counters() || !part) slices = 1;
  while (slices > 1 && (size_t)(tiles * slices * GT * GT) > part_elems) slices /= 2;
  if (n == 0) slices = 1;
  int64_t per = (n + slices - 1) / slices;
  per = (per + GK - 1) / GK * GK;
  slices = n > 0 ? (n + per - 1) / per : 1;
  dim3 grid((unsigned)tiles, (unsigned)slices);
  void* kt0 = kt_enabled() ? kt_begin(s) : nullptr;
  zgram_kernel<<<grid, GT * GT, 0, s>>>(n, mx, my, X, ldx, Y, ldy, G, ldg, herm, ntj, (int)slices, per, part, cnt);
  LAUNCH_NOTE(1);
  if (kt0) {
    // work: 8 flop per complex multiply-add of the tiles formed (16 x 16 granularity)
    const double f = 8.0 * (double)active * (GT * GT) * (double)n;
    kt_end(kt0, 2, f, f, s);
  }
}

}  // namespace gevp
