// Small dense Hermitian eigensolver for the Rayleigh-Ritz projection (m <= a few hundred).
//
// One SM executes FP64 at about 1.7 FMA per clock on this part, so an FP64 Jacobi in one
// CTA would take milliseconds. Instead:
//   1. parallel-ordered two-sided Jacobi in FP32 (FP32 runs at 128 FMA per clock per SM),
//      giving eigenvectors accurate to about 1e-6: one CTA below m = 32, the eight CTAs
//      of a thread-block cluster sharing G through distributed shared memory up to
//      m = 256, all SMs (cooperative launch) above. The cluster form runs no sweep when
//      G is already nearly diagonal (the projection of an almost converged block: the
//      refinement starts from Z = I, see jacobi32_cluster_kernel);
//   2. Ogita & Aishima's iterative refinement for symmetric/Hermitian eigenvector
//      matrices (Japan J. Ind. Appl. Math. 35, 2018), which converges quadratically and
//      consists of four FP64 GEMMs per step spread over all SMs. Pairs closer than the
//      refinement's threshold, and pairs whose first-order correction would exceed 0.2,
//      are left for later steps; the last step corrects only the orthonormality (a
//      symmetric Newton-Schulz step);
//   3. S = Z^H G Z in FP64 and exact FP64 Jacobi rotations, in one CTA, on the few pairs of
//      S whose coupling is still above 1e-15 ||G||_F (near-degenerate clusters the
//      refinement cannot separate); eigenvalues = diag(S).
// FP32 Jacobi uses hypot for |g_pq| (the squares of tiny couplings are denormal and would
// make the phase, hence the rotation, non-unitary) and skips couplings below FP32
// significance relative to the diagonal.
#include "gevp_internal.cuh"
#include <cooperative_groups.h>
#include <algorithm>

namespace gevp {

namespace {

constexpr int JT = 1024;   // threads of the Jacobi CTA

// split cluster barrier: arrive (release) and, later, wait (acquire) for the phase
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

__device__ __forceinline__ void block_pair(int step, int k, int np, int* p, int* q) {
  // circle method: position 0 fixed, the other np-1 players rotate by one per round
  auto player = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + step) % (np - 1)); };
  int a = player(k), b = player(np - 1 - k);
  *p = a < b ? a : b;
  *q = a < b ? b : a;
}

__device__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// L2 = true: load through L2 only (the multi-CTA variant; other CTAs wrote these
// elements in the previous round and L1 is not coherent across SMs)
template <bool L2>
__device__ __forceinline__ float2 ld2(const float2* p) {
  if constexpr (L2) return __ldcg(p);
  else return *p;
}

// Element access to G for the Jacobi rounds: a plain matrix (shared or global memory, the
// one-CTA forms), a global matrix read through L2 (the cooperative form: other CTAs wrote
// it and L1 is not coherent across SMs), or row bands held in the shared memory of the CTAs
// of a thread-block cluster (the cluster form; rows [c mb, (c + 1) mb) in CTA c).
struct GPlain {
  float2* g;
  int m;
  __device__ __forceinline__ float2 ld(int i, int j) const { return g[i * m + j]; }
  __device__ __forceinline__ void st(int i, int j, float2 v) const { g[i * m + j] = v; }
};
struct GL2 {
  float2* g;
  int m;
  __device__ __forceinline__ float2 ld(int i, int j) const { return __ldcg(g + i * m + j); }
  __device__ __forceinline__ void st(int i, int j, float2 v) const { g[i * m + j] = v; }
};
struct GBand {
  float2* const* band;   // per cluster rank: the generic address of that CTA's band
  int m, mb;
  __device__ __forceinline__ float2* at(int i, int j) const { return band[i / mb] + (i % mb) * m + j; }
  __device__ __forceinline__ float2 ld(int i, int j) const { return *at(i, j); }
  __device__ __forceinline__ void st(int i, int j, float2 v) const { *at(i, j) = v; }
};

// Rotation of pair k of round `step`: U = [[c, s], [-s conj(ph), c conj(ph)]] acting on
// columns (p, q), stored as (c, s, Re ph, Im ph); identity for the dummy index q = m of
// odd orders and for couplings below FP32 significance relative to the diagonal.
template <class Acc>
__device__ __forceinline__ void jacobi_pair_params(const Acc& G, int m, int np, int step, int k, float4* U,
                                                   int (*PQ)[2]) {
  int p, q;
  block_pair(step, k, np, &p, &q);
  PQ[k][0] = p;
  PQ[k][1] = q;
  float4 u = make_float4(1.f, 0.f, 1.f, 0.f);
  if (q < m) {
    float2 apq = G.ld(p, q);
    // |g_pq| without under/overflow: the phase g_pq / |g_pq| must stay unit-modulus
    // or the rotation stops being unitary (squares of tiny off-diagonals are denormal)
    float r = hypotf(apq.x, apq.y);
    float app = G.ld(p, p).x, aqq = G.ld(q, q).x;
    if (r > 1e-30f && r > 1e-10f * (fabsf(app) + fabsf(aqq))) {
      float tau = (aqq - app) / (2.f * r);
      float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
      float c = rsqrtf(1.f + t * t);
      u = make_float4(c, t * c, apq.x / r, apq.y / r);
    }
  }
  U[k] = u;
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Task e of one rotation step. The pairs of a round are disjoint, so G <- U^H G U splits
// into independent 2 x 2 blocks G[{p,q},{r,s}] <- U_a^H G[{p,q},{r,s}] U_b (tasks
// e < npairs^2, a = row pair, b = column pair), and Z <- Z U into independent row pieces
// (tasks after those). Every element of G is read from G and written to Gout once per
// step (Gout = G in place, or the other buffer of a ping-pong pair).
template <class Acc, bool ZL2>
__device__ __forceinline__ void jacobi_apply(const Acc& G, const Acc& Gout, float2* Z, int m, int npairs, int e,
                                             const float4* U, const int (*PQ)[2]) {
  if (e < npairs * npairs) {
    const int a = e / npairs, b = e % npairs;
    const int p = PQ[a][0], q = PQ[a][1], r = PQ[b][0], s = PQ[b][1];
    const bool qv = q < m, sv = s < m;
    const float4 ua = U[a], ub = U[b];
    const float2 z0 = make_float2(0.f, 0.f);
    float2 gpr = G.ld(p, r);
    float2 gps = sv ? G.ld(p, s) : z0;
    float2 gqr = qv ? G.ld(q, r) : z0;
    float2 gqs = (qv && sv) ? G.ld(q, s) : z0;
    // columns (r, s) with U_b: x_r' = c x_r - s conj(ph) x_s, x_s' = s x_r + c conj(ph) x_s
    {
      const float c = ub.x, sn = ub.y;
      const float2 phc = make_float2(ub.z, -ub.w);
      float2 t = cmulf(gps, phc);
      float2 nr = make_float2(c * gpr.x - sn * t.x, c * gpr.y - sn * t.y);
      float2 ns = make_float2(sn * gpr.x + c * t.x, sn * gpr.y + c * t.y);
      gpr = nr;
      gps = ns;
      t = cmulf(gqs, phc);
      nr = make_float2(c * gqr.x - sn * t.x, c * gqr.y - sn * t.y);
      ns = make_float2(sn * gqr.x + c * t.x, sn * gqr.y + c * t.y);
      gqr = nr;
      gqs = ns;
    }
    // rows (p, q) with U_a^H: r_p' = c r_p - s ph r_q, r_q' = s r_p + c ph r_q
    {
      const float c = ua.x, sn = ua.y;
      const float2 ph = make_float2(ua.z, ua.w);
      float2 t = cmulf(ph, gqr);
      float2 np_ = make_float2(c * gpr.x - sn * t.x, c * gpr.y - sn * t.y);
      float2 nq_ = make_float2(sn * gpr.x + c * t.x, sn * gpr.y + c * t.y);
      gpr = np_;
      gqr = nq_;
      t = cmulf(ph, gqs);
      np_ = make_float2(c * gps.x - sn * t.x, c * gps.y - sn * t.y);
      nq_ = make_float2(sn * gps.x + c * t.x, sn * gps.y + c * t.y);
      gps = np_;
      gqs = nq_;
    }
    if (a == b) {   // the rotated pair: exact zero coupling, real diagonal
      gps = z0;
      gqr = z0;
      gpr.y = 0.f;
      gqs.y = 0.f;
    }
    Gout.st(p, r, gpr);
    if (sv) Gout.st(p, s, gps);
    if (qv) Gout.st(q, r, gqr);
    if (qv && sv) Gout.st(q, s, gqs);
  } else {
    const int t = e - npairs * npairs;
    const int i = t / npairs, b = t % npairs;
    const int r = PQ[b][0], s = PQ[b][1];
    if (s >= m) return;
    const float4 u = U[b];
    const float c = u.x, sn = u.y;
    const float2 phc = make_float2(u.z, -u.w);
    const float2 zr = ld2<ZL2>(Z + i * m + r), zs = cmulf(ld2<ZL2>(Z + i * m + s), phc);
    Z[i * m + r] = make_float2(c * zr.x - sn * zs.x, c * zr.y - sn * zs.y);
    Z[i * m + s] = make_float2(sn * zr.x + c * zs.x, sn * zr.y + c * zs.y);
  }
}

// G (m x m, FP32 complex, Hermitian) is destroyed; Z receives eigenvectors (columns);
// w receives eigenvalues sorted ascending and perm the column order (w[k] = G[perm[k]]).
// Executed by one CTA of JT threads. Gs: shared-memory room for G (m * m), or nullptr to
// work on G in global memory; every rotation step reads and writes all of G, so keeping
// it on chip halves the step's memory traffic (Z stays in global memory).
__device__ void jacobi32_body(int m, float2* Gg, float2* Z, float* w, int* perm, int max_sweeps, float2* Gs) {
  __shared__ float4 U[512];       // per pair: (c, s, Re ph, Im ph)
  __shared__ int PQ[512][2];
  __shared__ float red[32];
  const int tid = threadIdx.x;
  float2* G = Gg;
  if (Gs) {
    for (int e = tid; e < m * m; e += JT) Gs[e] = Gg[e];
    __syncthreads();
    G = Gs;
  }
  for (int e = tid; e < m * m; e += JT) Z[e] = make_float2((e / m) == (e % m) ? 1.f : 0.f, 0.f);
  int np = (m % 2) ? m + 1 : m;
  int npairs = np / 2;
  float fro2 = 0.f;
  for (int e = tid; e < m * m; e += JT) { float2 g = G[e]; fro2 += g.x * g.x + g.y * g.y; }
  fro2 = block_sum(fro2, red);
  // sweep until the off-diagonal norm reaches the FP32 noise level or stops falling
  const float tol2 = 1e-16f * fro2;   // (1e-8 ||G||_F)^2
  float off_prev = 3.0e38f;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    float off = 0.f;
    for (int e = tid; e < m * m; e += JT) {
      int i = e / m, j = e % m;
      if (i != j) { float2 g = G[e]; off += g.x * g.x + g.y * g.y; }
    }
    off = block_sum(off, red);
    // converged, or stagnated at the FP32 noise level (early sweeps on clustered spectra
    // can reduce the off-norm slowly, so slow progress alone is not a reason to stop)
    if (off <= tol2 || (off > 0.9f * off_prev && off <= 1e-12f * fro2)) break;
    off_prev = off;
    for (int step = 0; step < np - 1; ++step) {
      const GPlain Ga{G, m};
      for (int k = tid; k < npairs; k += JT) jacobi_pair_params(Ga, m, np, step, k, U, PQ);
      __syncthreads();
      for (int e = tid; e < npairs * npairs + m * npairs; e += JT)
        jacobi_apply<GPlain, false>(Ga, Ga, Z, m, npairs, e, U, PQ);
      __syncthreads();
    }
  }
  // sort ascending by rank (ties by index)
  for (int i = tid; i < m; i += JT) {
    float wi = G[i * m + i].x;
    int r = 0;
    for (int j = 0; j < m; ++j) {
      float wj = G[j * m + j].x;
      r += (wj < wi) || (wj == wi && j < i);
    }
    perm[r] = i;
    w[r] = wi;
  }
}

constexpr int kJacobiSmemMax = 160;   // largest m whose G (m * m FP32 complex) is kept in shared memory

// Multi-CTA variant for orders above the one-CTA shared-memory size: the same rounds, each
// CTA computing every rotation of a round (redundantly, from G in global memory) and
// applying its share of the 2 x 2 block and Z tasks, with one grid barrier per round
// (cooperative launch: all CTAs are resident). The rounds alternate between G and Gb
// (m x m each): a round reads one and writes the other, so a CTA still computing the
// round's rotations never sees entries another CTA has already rotated. red: 2 +
// max_sweeps floats, zero on entry. G and Gb are both destroyed.
__global__ void __launch_bounds__(JT) jacobi32_coop_kernel(int m, float2* G, float2* Gb, float2* Z, float* w,
                                                           int* perm, int max_sweeps, float* red_g) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ float4 U[512];
  __shared__ int PQ[512][2];
  __shared__ float red[32];
  const int tid = threadIdx.x;
  const int gtid = blockIdx.x * JT + tid, gsz = gridDim.x * JT;
  for (int e = gtid; e < m * m; e += gsz) Z[e] = make_float2((e / m) == (e % m) ? 1.f : 0.f, 0.f);
  const int np = (m % 2) ? m + 1 : m;
  const int npairs = np / 2;
  float f = 0.f;
  for (int e = gtid; e < m * m; e += gsz) { float2 g = G[e]; f += g.x * g.x + g.y * g.y; }
  f = block_sum(f, red);
  if (tid == 0) atomicAdd(&red_g[0], f);
  grid.sync();
  const float fro2 = __ldcg(&red_g[0]);
  const float tol2 = 1e-16f * fro2;
  float off_prev = 3.0e38f;
  float2* Gc = G;    // the current matrix; rounds write the other buffer
  float2* Gn = Gb;
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    float off = 0.f;
    for (int e = gtid; e < m * m; e += gsz) {
      int i = e / m, j = e % m;
      if (i != j) { float2 g = __ldcg(Gc + e); off += g.x * g.x + g.y * g.y; }
    }
    off = block_sum(off, red);
    if (tid == 0) atomicAdd(&red_g[1 + sweep], off);
    grid.sync();
    off = __ldcg(&red_g[1 + sweep]);   // the same value in every CTA: a uniform decision
    if (off <= tol2 || (off > 0.9f * off_prev && off <= 1e-12f * fro2)) break;
    off_prev = off;
    for (int step = 0; step < np - 1; ++step) {
      const GL2 Ac{Gc, m}, An{Gn, m};
      for (int k = tid; k < npairs; k += JT) jacobi_pair_params(Ac, m, np, step, k, U, PQ);
      __syncthreads();
      for (int e = gtid; e < npairs * npairs + m * npairs; e += gsz)
        jacobi_apply<GL2, true>(Ac, An, Z, m, npairs, e, U, PQ);
      grid.sync();
      float2* t = Gc;
      Gc = Gn;
      Gn = t;
    }
  }
  if (blockIdx.x != 0) return;
  for (int i = tid; i < m; i += JT) {
    float wi = __ldcg(Gc + i * m + i).x;
    int r = 0;
    for (int j = 0; j < m; ++j) {
      float wj = __ldcg(Gc + j * m + j).x;
      r += (wj < wi) || (wj == wi && j < i);
    }
    perm[r] = i;
    w[r] = wi;
  }
}

// Cluster form for mid-size orders: the rounds of jacobi32_body spread over the kJC CTAs
// of one thread-block cluster. G lives in the CTAs' shared memory as row bands (two
// buffers: a round reads one and writes the other, so CTAs still computing the round's
// rotations never see rotated entries), read and written through distributed shared
// memory; one cluster barrier per round instead of one CTA doing every 2 x 2 block. Z is
// held as row bands too: the update Z <- Z U mixes two columns within each row, so every
// CTA rotates its own rows in its own shared memory (two thirds of a round's tasks, which
// no longer go through L2), and writes its band to Z at the end. The round's barrier is
// split around that work: a CTA arrives once its share of G is written and waits only
// after rotating its rows of Z (the rotations are double-buffered by round parity). The
// arithmetic of every element is that of jacobi32_body, so the results are identical. Gin
// (m x m) is read, not modified.
constexpr int kJC = 8;
constexpr int kJClusterMax = 256;

__global__ void __launch_bounds__(JT, 1) jacobi32_cluster_kernel(int m, const float2* Gin, float2* Z, float* w,
                                                                 int* perm, int max_sweeps, int may_skip) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ float2 jband[];   // [2][mb][m] G bands, then [mb][m] the Z band
  // rotations of round k in buffer k & 1: a thread may compute round k + 1's while another
  // still rotates its rows of Z with round k's
  __shared__ float4 U2[2][512];
  __shared__ int PQ2[2][512][2];
  __shared__ float red[32];
  __shared__ float part[64];          // this CTA's partial sums: [0] ||G||_F^2, [1 + sweep] off-norm
  __shared__ float dg[kJClusterMax];  // the diagonal of G
  __shared__ int coupled;             // this CTA's rows hold a coupling the refinement cannot start from
  __shared__ float2* bandp[2][kJC];   // generic addresses of every CTA's two bands
  const int tid = threadIdx.x;
  const int rank = (int)cl.block_rank();
  const int mb = (m + kJC - 1) / kJC;
  if (tid < kJC) {
    bandp[0][tid] = cl.map_shared_rank(jband, tid);
    bandp[1][tid] = cl.map_shared_rank(jband + mb * m, tid);
  }
  // own band of G into buffer 0 (rows past m are never addressed)
  const int r0 = rank * mb;
  for (int e = tid; e < mb * m; e += JT) {
    const int r = r0 + e / m;
    jband[e] = r < m ? Gin[r * m + (e % m)] : make_float2(0.f, 0.f);
  }
  const int gtid = rank * JT + tid, gsz = kJC * JT;
  const int rows = max(0, min(mb, m - r0));
  float2* zband = jband + 2 * mb * m;   // own rows r0 .. r0 + rows - 1 of Z
  for (int e = tid; e < rows * m; e += JT) zband[e] = make_float2((r0 + e / m) == (e % m) ? 1.f : 0.f, 0.f);
  const int np = (m % 2) ? m + 1 : m;
  const int npairs = np / 2;
  float f = 0.f;
  for (int e = tid; e < rows * m; e += JT) { float2 g = jband[e]; f += g.x * g.x + g.y * g.y; }
  for (int j = tid; j < m; j += JT) dg[j] = Gin[j * m + j].x;
  if (tid == 0) coupled = 0;
  f = block_sum(f, red);
  if (tid == 0) part[0] = f;
  cl.sync();
  // every CTA sums the partials in the same order: the same decisions everywhere
  auto cluster_sum = [&](int slot) {
    float t = 0.f;
    for (int c = 0; c < kJC; ++c) t += *cl.map_shared_rank(&part[slot], c);
    return t;
  };
  const float fro2 = cluster_sum(0);
  const float tol2 = 1e-16f * fro2;
  float off_prev = 3.0e38f;
  int cur = 0;
  if (max_sweeps > 62) max_sweeps = 62;
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    float off = 0.f;
    const float2* Gc = jband + cur * mb * m;
    for (int e = tid; e < rows * m; e += JT) {
      const int i = r0 + e / m, j = e % m;
      if (i != j) { float2 g = Gc[e]; off += g.x * g.x + g.y * g.y; }
    }
    off = block_sum(off, red);
    if (tid == 0) part[1 + sweep] = off;
    cl.sync();
    off = cluster_sum(1 + sweep);
    if (off <= tol2 || (off > 0.9f * off_prev && off <= 1e-12f * fro2)) break;
    if (sweep == 0 && may_skip) {
      // Nearly diagonal already (the projection of a block that has almost converged):
      // every coupling at most 1e-3 of its diagonal gap (gaps below eta0 = 1e-6 ||G||_F
      // counted as eta0: clusters, which FP32 sweeps cannot resolve either), and at most
      // 1e-5 of it for gaps between eta0 and delta = 2 ||offdiag(G)||_F. The FP64
      // refinement started from Z = I has the clustering threshold delta in its first step:
      // it corrects the pairs farther apart than delta there (to about 1e-6), those between
      // eta0 and delta in its second step (to about 1e-10), and, converging quadratically,
      // reaches FP64 accuracy in its last step as it would from the sweeps' result; the
      // clusters go to the exact rotations after it. No sweep is run.
      const float eta0 = 1e-6f * sqrtf(fro2), delta = 2.f * sqrtf(off);
      bool c = false;
      for (int e = tid; e < rows * m; e += JT) {
        const int i = r0 + e / m, j = e % m;
        if (i == j) continue;
        const float2 g = Gc[e];
        const float gap = fabsf(dg[i] - dg[j]);
        const float a = hypotf(g.x, g.y);
        c |= a > 1e-3f * fmaxf(gap, eta0) || (gap > eta0 && gap <= delta && a > 1e-5f * gap);
      }
      if (__any_sync(0xffffffffu, c) && (tid & 31) == 0) coupled = 1;
      cl.sync();
      int any = 0;
      for (int r = 0; r < kJC; ++r) any |= *cl.map_shared_rank(&coupled, r);
      if (!any) break;
    }
    off_prev = off;
    for (int step = 0; step < np - 1; ++step) {
      const GBand Ac{bandp[cur], m, mb}, An{bandp[cur ^ 1], m, mb};
      float4* U = U2[step & 1];
      int(*PQ)[2] = PQ2[step & 1];
      for (int k = tid; k < npairs; k += JT) jacobi_pair_params(Ac, m, np, step, k, U, PQ);
      __syncthreads();
      for (int e = gtid; e < npairs * npairs; e += gsz) jacobi_apply<GBand, true>(Ac, An, Z, m, npairs, e, U, PQ);
      // the round's G is written: arrive, and rotate the own rows of Z (columns r, s of each
      // pair, this CTA's shared memory only) while the other CTAs finish theirs
      cluster_arrive();
      for (int t = tid; t < rows * npairs; t += JT) {
        const int il = t / npairs, b = t % npairs;
        const int r = PQ[b][0], sc = PQ[b][1];
        if (sc >= m) continue;
        const float4 u = U[b];
        const float c = u.x, sn = u.y;
        const float2 phc = make_float2(u.z, -u.w);
        float2* zrow = zband + il * m;
        const float2 zr = zrow[r], zs = cmulf(zrow[sc], phc);
        zrow[r] = make_float2(c * zr.x - sn * zs.x, c * zr.y - sn * zs.y);
        zrow[sc] = make_float2(sn * zr.x + c * zs.x, sn * zr.y + c * zs.y);
      }
      cluster_wait();
      cur ^= 1;
    }
  }
  if (rank == 0) {
    const GBand Ac{bandp[cur], m, mb};
    for (int i = tid; i < m; i += JT) {
      const float wi = Ac.ld(i, i).x;
      int r = 0;
      for (int j = 0; j < m; ++j) {
        const float wj = Ac.ld(j, j).x;
        r += (wj < wi) || (wj == wi && j < i);
      }
      perm[r] = i;
      w[r] = wi;
    }
  }
  for (int e = tid; e < rows * m; e += JT) Z[(int64_t)r0 * m + e] = zband[e];
  // no CTA leaves while rank 0 may still read its shared memory
  cl.sync();
}

__global__ void __launch_bounds__(JT) jacobi32_kernel(int m, float2* G, float2* Z, float* w, int* perm,
                                                      int max_sweeps) {
  extern __shared__ float2 jsm[];
  jacobi32_body(m, G, Z, w, perm, max_sweeps, m <= kJacobiSmemMax ? jsm : nullptr);
}

// one CTA per problem of a batch: which = 0 -> the Rayleigh-Ritz matrix, 1 -> Lanczos T;
// smem_m: the launch provided shared-memory room for matrices up to smem_m x smem_m
__global__ void __launch_bounds__(JT) jacobi32_batched_kernel(const BDesc* D, int which, int k, int max_sweeps,
                                                              int smem_m) {
  extern __shared__ float2 jsm[];
  const BDesc& d = D[blockIdx.x];
  if (d.active && *d.active == 0) return;
  if (which == 0) jacobi32_body(d.m, d.G32, d.Z32, d.w32, d.perm, max_sweeps, d.m <= smem_m ? jsm : nullptr);
  else jacobi32_body(k, d.T32, d.LZ32, d.lw32, d.lperm, max_sweeps, k <= smem_m ? jsm : nullptr);
}

// dynamic shared memory of a Jacobi launch on matrices up to m x m (0: global memory)
size_t jacobi_smem(int m) {
  static bool set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !set[dev]) {
    const int bytes = kJacobiSmemMax * kJacobiSmemMax * (int)sizeof(float2);
    cudaFuncSetAttribute(jacobi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(jacobi32_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    set[dev] = true;
  }
  return m <= kJacobiSmemMax ? (size_t)m * m * sizeof(float2) : 0;
}

// Z64[:, k] = Z32[:, perm[k]]
__global__ void gather_z_kernel(int m, const float2* Z32, const int* perm, double2* Z, int64_t ldz) {
  int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), k = (int)(e % m);
    float2 v = Z32[i * m + perm[k]];
    Z[i * ldz + k] = make_double2(v.x, v.y);
  }
}

__global__ void g_to_c_kernel(int m, const double2* G, int64_t ldg, float2* G32) {
  int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    double2 a = G[i * ldg + j], b = G[j * ldg + i];   // Hermitian part
    G32[e] = make_float2((float)(0.5 * (a.x + b.x)), (float)(0.5 * (a.y - b.y)));
  }
}

__device__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// Ogita-Aishima: lam_i = Re S_ii / (1 - Re R_ii); delta = 2 (||S - diag(lam)||_F + ||G||_F ||R||_F).
// scal[0] = delta, scal[1] = ||G||_F (input, computed once). The kernels are given the Gram
// matrix Zg = Z^H Z and use R = I - Zg.
// The same scalars over many CTAs (one SM retires about two FP64 FMAs per clock, so the
// m^2 sums of one CTA take tens of microseconds): per-block partial sums, then one thread
// adds them in block order (deterministic). lam is written by the diagonal's owners.
__device__ __forceinline__ double2 oa_r(const double2* Zg, int64_t e, int i, int j) {
  const double2 g = Zg[e];
  return make_double2((i == j ? 1.0 : 0.0) - g.x, -g.y);
}

__global__ void __launch_bounds__(256) oa_partial_kernel(int m, const double2* Zg, const double2* S, double* lam,
                                                         double* part) {
  __shared__ double red[32];
  double soff = 0.0, r2 = 0.0;
  const int64_t mm = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mm; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    double2 sv = S[e];
    const double2 rv = oa_r(Zg, e, i, j);
    if (i == j) {
      const double li = sv.x / (1.0 - rv.x);
      lam[i] = li;
      sv.x -= li;
    }
    soff += zabs2(sv);
    r2 += zabs2(rv);
  }
  soff = block_sum_d(soff, red);
  r2 = block_sum_d(r2, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = soff;
    part[2 * blockIdx.x + 1] = r2;
  }
}

__global__ void oa_finish_kernel(int nblk, const double* part, double* scal) {
  if (threadIdx.x != 0) return;
  double soff = 0.0, r2 = 0.0;
  for (int b = 0; b < nblk; ++b) {
    soff += part[2 * b];
    r2 += part[2 * b + 1];
  }
  scal[0] = 2.0 * (sqrt(soff) + scal[1] * sqrt(r2));
}

// ||G||_F over many CTAs: per-block partial sums of |g|^2, then out = sqrt(sum) in block order
__global__ void __launch_bounds__(256) frob_partial_kernel(int m, const double2* G, int64_t ldg, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  const int64_t mm = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mm; e += (int64_t)gridDim.x * blockDim.x)
    s += zabs2(G[(e / m) * ldg + (e % m)]);
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void frob_finish_kernel(int nblk, const double* part, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b];
  out[0] = sqrt(s);
}

__global__ void oa_update_kernel(int m, const double2* Zg, const double2* S, const double* lam, const double* scal,
                                 double2* E, int only_orth, double emax) {
  int64_t total = (int64_t)m * m;
  double delta = only_orth ? 1e300 : scal[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    double2 r = oa_r(Zg, e, i, j);
    double2 v;
    double d = lam[j] - lam[i];
    v = zscale(r, 0.5);
    if (i != j && fabs(d) > delta) {
      double2 sv = S[e];
      double2 t = make_double2(sv.x + lam[j] * r.x, sv.y + lam[j] * r.y);
      // first-order correction only where it is small (|E_ij| <= emax); larger couplings
      // are left to the next step (or to the exact rotations after the last), which keeps
      // the iteration from diverging
      if (sqrt(zabs2(t)) <= emax * fabs(d)) v = make_double2(t.x / d, t.y / d);
    }
    E[e] = v;
  }
}


// Zn = Z + Z E with the product Z E in FP32 (FP32 FMA runs 64x faster than FP64 here). E
// is the refinement's correction: its entries are at most 0.2 and shrink quadratically, so
// the FP32 product's error (about 1e-7 |E|) is far below the quadratic error the next step
// removes anyway; every step recomputes Z^H Z and Z^H G Z in FP64 from the new Z, and the
// sum with Z is in FP64, so the iteration still converges to FP64 accuracy.
__global__ void __launch_bounds__(256) zupd32_kernel(int m, const double2* Z, const double2* E, double2* Zn) {
  __shared__ float2 Zs[16][17];
  __shared__ float2 Es[16][17];
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  float2 acc = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < m; k0 += 16) {
    const int kz = k0 + tx, ke = k0 + ty;
    double2 z = (i < m && kz < m) ? Z[(int64_t)i * m + kz] : make_double2(0.0, 0.0);
    double2 e = (ke < m && j < m) ? E[(int64_t)ke * m + j] : make_double2(0.0, 0.0);
    Zs[ty][tx] = make_float2((float)z.x, (float)z.y);
    Es[ty][tx] = make_float2((float)e.x, (float)e.y);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) cfma(acc, Zs[ty][kk], Es[kk][tx]);
    __syncthreads();
  }
  if (i < m && j < m) {
    const double2 z = Z[(int64_t)i * m + j];
    Zn[(int64_t)i * m + j] = make_double2(z.x + (double)acc.x, z.y + (double)acc.y);
  }
}

// Clusters the refinement leaves mixed (pairs closer than its threshold): S = Z^H G Z is
// diagonal apart from those couplings. One CTA finds the pairs with |s_pq| above tol and
// applies exact FP64 Jacobi rotations to them (S two-sided, Z on the right), a few at a
// time, for a few sweeps; typically a handful of rotations. lam <- diag(S).
__device__ void cluster_jacobi_body(int m, double2* S, double2* Z, double* lam, const double* fro, double rel,
                                    int max_sweeps) {
  const double tol = rel * fro[0];
  // FP32 Jacobi leaves eigenvalue errors of order 1e-4 ||G|| at m ~ 300 (accumulated
  // rounding of many rotations), so dense clusters can leave several hundred couplings
  constexpr int kMaxPairs = 1024;
  __shared__ int PI[kMaxPairs], PJ[kMaxPairs];
  __shared__ int npairs;
  __shared__ double2 ucs[3];   // c, s (real), ph
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) npairs = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int i = e / m, j = e % m;
      if (j <= i) continue;
      double2 v = S[e];
      if (hypot(v.x, v.y) > tol) {
        int k = atomicAdd(&npairs, 1);
        if (k < kMaxPairs) { PI[k] = i; PJ[k] = j; }
      }
    }
    __syncthreads();
    int np = min(npairs, kMaxPairs);
    if (np == 0) break;
    for (int k = 0; k < np; ++k) {
      int p = PI[k], q = PJ[k];
      if (threadIdx.x == 0) {
        double2 apq = S[p * m + q];
        double r = hypot(apq.x, apq.y);
        double c = 1.0, s = 0.0;
        double2 ph = make_double2(1.0, 0.0);
        if (r > 0.0) {
          double app = S[p * m + p].x, aqq = S[q * m + q].x;
          double tau = (aqq - app) / (2.0 * r);
          double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
          ph = make_double2(apq.x / r, apq.y / r);
        }
        ucs[0] = make_double2(c, 0.0);
        ucs[1] = make_double2(s, 0.0);
        ucs[2] = ph;
      }
      __syncthreads();
      const double c = ucs[0].x, s = ucs[1].x;
      const double2 ph = ucs[2], phc = zconj(ph);
      // columns p, q of S and Z: [x_p, x_q] <- [c x_p - s conj(ph) x_q, s x_p + c conj(ph) x_q]
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 a = S[i * m + p], b = zmul(S[i * m + q], phc);
        S[i * m + p] = make_double2(c * a.x - s * b.x, c * a.y - s * b.y);
        S[i * m + q] = make_double2(s * a.x + c * b.x, s * a.y + c * b.y);
        double2 za = Z[i * m + p], zb = zmul(Z[i * m + q], phc);
        Z[i * m + p] = make_double2(c * za.x - s * zb.x, c * za.y - s * zb.y);
        Z[i * m + q] = make_double2(s * za.x + c * zb.x, s * za.y + c * zb.y);
      }
      __syncthreads();
      // rows p, q of S: [r_p; r_q] <- [c r_p - s ph r_q; s r_p + c ph r_q]
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double2 a = S[p * m + j], b = zmul(ph, S[q * m + j]);
        double2 np_ = make_double2(c * a.x - s * b.x, c * a.y - s * b.y);
        double2 nq_ = make_double2(s * a.x + c * b.x, s * a.y + c * b.y);
        if (j == q) np_ = make_double2(0.0, 0.0);
        if (j == p) nq_ = make_double2(0.0, 0.0);
        if (j == p) np_.y = 0.0;
        if (j == q) nq_.y = 0.0;
        S[p * m + j] = np_;
        S[q * m + j] = nq_;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = S[i * m + i].x;
}

__global__ void __launch_bounds__(1024) cluster_jacobi_kernel(int m, double2* S, double2* Z, double* lam,
                                                              const double* fro, double rel, int max_sweeps) {
  cluster_jacobi_body(m, S, Z, lam, fro, rel, max_sweeps);
}

__global__ void __launch_bounds__(1024) cluster_jacobi_batched_kernel(const BDesc* D, int zsel, double rel,
                                                                      int max_sweeps) {
  const BDesc& d = D[blockIdx.x];
  if (d.active && *d.active == 0) return;
  cluster_jacobi_body(d.m, d.hS, zsel == 0 ? d.hZ : d.hT, d.hlam, d.hscal + 1, rel, max_sweeps);
}

// final ordering: theta ascending, Z columns permuted accordingly
__global__ void sort_pairs_kernel(int m, const double* lam, const double2* Zin, double* theta, double2* Z,
                                  int64_t ldz) {
  __shared__ int rk[1024];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double li = lam[i];
    int r = 0;
    for (int j = 0; j < m; ++j) r += (lam[j] < li) || (lam[j] == li && j < i);
    rk[i] = r;
    theta[r] = li;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e / m, k = e % m;
    Z[i * ldz + rk[k]] = Zin[i * m + k];
  }
}

}  // namespace

size_t heev_ws_bytes(int m, size_t split_elems) {
  size_t mm = (size_t)m * m;
  size_t b = 0;
  b += 2 * mm * sizeof(float2) + m * sizeof(float) + m * sizeof(int);
  b += 5 * mm * sizeof(double2) + m * sizeof(double) + 8 * sizeof(double);
  b += split_elems * sizeof(double2);
  return b + 16 * 256;
}

// Cooperative multi-CTA Jacobi for large m; false if it cannot be launched (then the
// caller runs the one-CTA kernel).
bool jacobi32_coop(int m, float2* G, float2* Gb, float2* Z, float* w, int* perm, int max_sweeps, float* red,
                   cudaStream_t s) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi32_coop_kernel, JT, 0) != cudaSuccess ||
      per_sm < 1)
    return false;
  const int np = (m % 2) ? m + 1 : m, npairs = np / 2;
  const int64_t tasks = (int64_t)npairs * npairs + (int64_t)m * npairs;
  int grid = (int)std::min<int64_t>((int64_t)per_sm * sms, (tasks + JT - 1) / JT);
  grid = std::max(grid, 1);
  if (max_sweeps > 62) max_sweeps = 62;
  if (cudaMemsetAsync(red, 0, 64 * sizeof(float), s) != cudaSuccess) return false;
  void* args[] = {&m, &G, &Gb, &Z, &w, &perm, &max_sweeps, &red};
  if (cudaLaunchCooperativeKernel((const void*)jacobi32_coop_kernel, grid, JT, args, 0, s) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  LAUNCH_NOTE(1);
  return true;
}

// Cluster Jacobi for 32 <= m <= kJClusterMax; false if it cannot be launched (then the
// caller runs the one-CTA kernel).
bool jacobi32_cluster(int m, const float2* G, float2* Z, float* w, int* perm, int max_sweeps, int may_skip,
                      cudaStream_t s) {
  if (m < 32 || m > kJClusterMax) return false;
  const int mb = (m + kJC - 1) / kJC;
  const size_t smem = (size_t)3 * mb * m * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(jacobi32_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(3 * ((kJClusterMax + kJC - 1) / kJC) * kJClusterMax * sizeof(float2))) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kJC, 1, 1);
  cfg.blockDim = dim3(JT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kJC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, jacobi32_cluster_kernel, m, G, Z, w, perm, max_sweeps, may_skip) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  LAUNCH_NOTE(1);
  return true;
}

void jacobi32(int m, float2* G, float2* Z, float* w, int* perm, int max_sweeps, cudaStream_t s) {
  jacobi32_kernel<<<1, JT, jacobi_smem(m), s>>>(m, G, Z, w, perm, max_sweeps);
  LAUNCH_NOTE(1);
}

// mmax: the largest matrix order among the problems (k for the Lanczos matrices)
void jacobi32_batched(const BDesc* D, int np, int which, int k, int mmax, int max_sweeps, cudaStream_t s) {
  // problems with m <= 160 keep G on chip even when the batch's largest m is above that
  const int cap = std::min(which == 0 ? mmax : k, kJacobiSmemMax);
  const size_t sm = jacobi_smem(cap);
  jacobi32_batched_kernel<<<np, JT, sm, s>>>(D, which, k, max_sweeps, sm > 0 ? cap : 0);
  LAUNCH_NOTE(1);
}

void cluster_jacobi_batched(const BDesc* D, int np, int zsel, double rel, int max_sweeps, cudaStream_t s) {
  cluster_jacobi_batched_kernel<<<np, 1024, 0, s>>>(D, zsel, rel, max_sweeps);
  LAUNCH_NOTE(1);
}

void heev_small(int m, const double2* G, int64_t ldg, double* theta, double2* Zout, int64_t ldz,
                const HeevWork& w, int refine_iters, cudaStream_t s) {
  if (m <= 0) return;
  int64_t mm = (int64_t)m * m;
  int blocks = (int)std::min<int64_t>((mm + 255) / 256, 152 * 4);
  g_to_c_kernel<<<blocks, 256, 0, s>>>(m, G, ldg, w.G32);
  LAUNCH_NOTE(1);
  // large orders on all SMs (cooperative launch); otherwise, or if that launch is not
  // possible, one CTA
  // 32 <= m <= 256 on the eight CTAs of a cluster; larger orders on all SMs (cooperative
  // launch; the FP64 scratch E, unused until the refinement, holds its second FP32 buffer);
  // small ones, or when neither launch is possible, in one CTA
  // (the sweeps may be skipped for a nearly diagonal G when the refinement has the three
  // steps that its start from Z = I needs)
  bool done = jacobi32_cluster(m, w.G32, w.Z32, w.w32, w.perm, 40, refine_iters >= 3 ? 1 : 0, s);
  if (!done && m > kJacobiSmemMax)
    done = jacobi32_coop(m, w.G32, (float2*)w.E, w.Z32, w.w32, w.perm, 40, (float*)(w.scal + 16), s);
  if (!done) {
    jacobi32_kernel<<<1, JT, jacobi_smem(m), s>>>(m, w.G32, w.Z32, w.w32, w.perm, 40);
    LAUNCH_NOTE(1);
  }
  gather_z_kernel<<<blocks, 256, 0, s>>>(m, w.Z32, w.perm, w.Z, m);
  LAUNCH_NOTE(1);
  // partial sums in E (free until the refinement's first product writes it)
  const int nblk = (int)std::min<int64_t>(64, std::max<int64_t>(1, ((int64_t)m * m + 255) / 256));
  double* part = (double*)w.E;
  frob_partial_kernel<<<nblk, 256, 0, s>>>(m, G, ldg, part);
  frob_finish_kernel<<<1, 32, 0, s>>>(nblk, part, w.scal + 1);
  LAUNCH_NOTE(2);
  double2* Z = w.Z;
  double2* Zn = w.T;   // ping-pong partner
  const dim3 ugrid((m + 15) / 16, (m + 15) / 16);
  for (int it = 0; it <= refine_iters; ++it) {
    const bool only_orth = it == refine_iters;
    // R = I - Z^H Z (the kernels below are given Z^H Z; Hermitian: lower tiles only)
    zgram(m, m, m, Z, m, Z, m, w.R, m, 1, w.split_ws, w.split_ws_elems, w.gcnt, s);
    if (!only_orth) {
      // E <- G Z (E used as scratch), S = Z^H (G Z) (Hermitian: lower tiles only)
      ZgemmArgs b = zg(m, m, m, G, ldg, 0, Z, m, 0, w.E, m);
      zgemm(b, w.split_ws, w.split_ws_elems, s);
      zgram(m, m, m, Z, m, w.E, m, w.S, m, 1, w.split_ws, w.split_ws_elems, w.gcnt, s);
      // partial sums in E: the product G Z it held has been consumed by S = Z^H (G Z)
      oa_partial_kernel<<<nblk, 256, 0, s>>>(m, w.R, w.S, w.lam, part);
      oa_finish_kernel<<<1, 32, 0, s>>>(nblk, part, w.scal);
      LAUNCH_NOTE(2);
    }
    // the last step corrects only the orthonormality (E = R/2 everywhere: a symmetric
    // Newton-Schulz step), which needs neither S nor the eigenvalue estimates; the
    // eigenvalues come from S = Z^H G Z of the final Z below
    // a correction of size e leaves an error of about e^2 for the next step: 0.2 in the
    // first step and while two or more correcting steps follow, 1e-4 before the last one,
    // 1e-8 in it, so that what the refinement corrects reaches FP64 accuracy; a pair that
    // needs more (a near-degenerate pair that the earlier corrections coupled) goes to the
    // rotations
    const int rem = refine_iters - 1 - it;
    const double emax = (rem >= 2 || it == 0) ? 0.2 : (rem == 1 ? 1e-4 : 1e-8);
    oa_update_kernel<<<blocks, 256, 0, s>>>(m, w.R, w.S, w.lam, w.scal, w.E, only_orth ? 1 : 0, emax);
    LAUNCH_NOTE(1);
    // Zn = Z + Z E (the correction's product in FP32)
    zupd32_kernel<<<ugrid, 256, 0, s>>>(m, Z, w.E, Zn);
    LAUNCH_NOTE(1);
    std::swap(Z, Zn);
  }
  // resolve what the refinement left mixed: S = Z^H G Z, exact rotations on its remaining
  // couplings (near-degenerate clusters), eigenvalues = diag(S)
  ZgemmArgs b2 = zg(m, m, m, G, ldg, 0, Z, m, 0, w.E, m);
  zgemm(b2, w.split_ws, w.split_ws_elems, s);
  zgram(m, m, m, Z, m, w.E, m, w.S, m, 1, w.split_ws, w.split_ws_elems, w.gcnt, s);
  cluster_jacobi_kernel<<<1, 1024, 0, s>>>(m, w.S, Z, w.lam, w.scal + 1, 1e-15, 12);
  LAUNCH_NOTE(1);
  sort_pairs_kernel<<<1, 1024, 0, s>>>(m, w.lam, Z, theta, Zout, ldz);
  LAUNCH_NOTE(1);
}

}  // namespace gevp
