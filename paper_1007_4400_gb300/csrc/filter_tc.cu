// Chebyshev filter steps on the tcgen05 tensor cores.
//
// Complex product by the three-real-product (Gauss) formula with FP32 accumulation in TMEM:
//   T1 = Cr Yr,  T2 = Ci Yi,  T3 = (Cr + Ci)(Yr + Yi),   Re = T1 - T2,  Im = T3 - T1 - T2,
// followed by the scaled three-term recurrence Y_{j+1} = alpha C Y_j + beta Y_j + gamma Y_{j-1}
// with the recurrence state kept in FP32.
//
// Precision. Each real operand x is stored as nsplit BF16 pieces x = x0 + x1 + x2 + ...
// (x0 = bf16(x), x1 = bf16(x - x0), ...). nsplit = 1 is the BF16 filter. nsplit = 3 keeps
// the six products x_a y_b with a + b <= 2 (about 24 significant bits, FP32 class); the
// products are extra segments of the K loop accumulating into the same TMEM accumulators,
// so the kernel is unchanged apart from which tensor map each segment loads.
//
// Layout (all K-major, as the MMA wants both operands): the planes of C are n_pad x n_pad
// row-major BF16 (row i = output row, contiguous k); the block Y is stored transposed,
// Y^T planes ncols x n_pad (row c = column c of Y, contiguous k), and so is the FP32 state.
// Padding rows/columns are zero, so the padded K contributes nothing.
//
// One CTA: 128 rows of C (UMMA M = 128) x one chunk of up to 160 columns of Y (N), over a
// slice of K (split-K across grid.z, so that n = 2048 still fills the 152 SMs). Warp 0
// lane 0 issues TMA loads (128B-swizzled boxes, 2-stage mbarrier pipeline), warp 1 lane 0
// issues the MMAs (3 per 16-wide K step into three TMEM accumulators of N columns each),
// then all four warps read TMEM back (warp w owns lanes 32w..32w+31) and write the FP32
// partial product transposed (coalesced along rows). A second kernel sums the split-K
// partials in a fixed order (deterministic) and applies the recurrence.
//
// Every mbarrier wait is bounded; on expiry the kernel records an error code, skips the
// rest of its work, frees its TMEM and returns.
#include "gevp_internal.cuh"
#include "tc_ptx.cuh"
#include <cuda.h>
#include <algorithm>
#include <cstring>
#include <vector>

namespace gevp {

namespace {

constexpr int TM = 128;
constexpr int TK = 64;
constexpr int STAGES = 2;
constexpr int NMAX = 160;
constexpr int MAXSPLIT = 3;
constexpr int MAXSEG = 6;

// segments (a piece, b piece) with a + b <= nsplit - 1
__constant__ int kSegA[MAXSEG] = {0, 0, 1, 0, 1, 2};
__constant__ int kSegB[MAXSEG] = {0, 1, 0, 2, 1, 0};
inline int nseg_for(int nsplit) { return nsplit == 1 ? 1 : (nsplit == 2 ? 3 : 6); }

struct TcMaps {
  CUtensorMap a[MAXSPLIT * 3];   // C planes: [piece][re, im, re+im]
  CUtensorMap b[MAXSPLIT * 3];   // Y^T planes
};

struct TcParams {
  int n_pad;
  int nchunk;
  int kb_per_split;
  int ncols_pad;      // rows of the Y^T planes (multiple of nchunk)
  int nseg;
  uint32_t tmem_cols; // power of two >= 3 * nchunk
  float2* ws;         // [ksplit][ncols_pad][n_pad]
  int* err;
};

// One output tile: rows m0..m0+127 of C times columns c0..c0+nchunk-1 of the block over
// K slice z. amaps/bmaps: the tensor maps of the pieces of C and of the block (kernel
// parameter space or global memory).
__device__ __forceinline__ void tc_tile(const CUtensorMap* amaps, const CUtensorMap* bmaps, const TcParams& p,
                                        int m0, int c0, int z) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_sh;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nkb_total = p.n_pad / TK;
  const int kb0 = z * p.kb_per_split;
  const int kb1 = min(kb0 + p.kb_per_split, nkb_total);
  const int nkb = max(0, kb1 - kb0);
  // K-block-major: all segments of one K block back to back, so the C piece a segment
  // reloads (piece 0 serves three segments, piece 1 two) is still in L2
  const int niter = nkb * p.nseg;
  const uint32_t a_bytes = TM * TK * 2;
  const uint32_t b_bytes = (uint32_t)p.nchunk * TK * 2;
  const uint32_t stage_bytes = 3 * a_bytes + 3 * b_bytes;
  auto tile = [&](int s, int which) -> uint8_t* {
    uint8_t* base = smem + (size_t)s * stage_bytes;
    return which < 3 ? base + which * a_bytes : base + 3 * a_bytes + (which - 3) * b_bytes;
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_sh;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int i = 0; i < niter; ++i, issued = i) {
      int s = i % STAGES;
      uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (i >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, p.err, 1)) break;
      mbar_expect_tx(&full[s], stage_bytes);
      const int seg = i % p.nseg;
      const int kx = (kb0 + i / p.nseg) * TK;
      const CUtensorMap* A = amaps + 3 * kSegA[seg];
      const CUtensorMap* B = bmaps + 3 * kSegB[seg];
      tma_load_2d(tile(s, 0), A + 0, kx, m0, &full[s]);
      tma_load_2d(tile(s, 1), A + 1, kx, m0, &full[s]);
      tma_load_2d(tile(s, 2), A + 2, kx, m0, &full[s]);
      tma_load_2d(tile(s, 3), B + 0, kx, c0, &full[s]);
      tma_load_2d(tile(s, 4), B + 1, kx, c0, &full[s]);
      tma_load_2d(tile(s, 5), B + 2, kx, c0, &full[s]);
    }
    // every copy issued has landed before the CTA leaves (bounded; immediate unless a wait
    // elsewhere gave up)
    for (int i = max(0, issued - STAGES); i < issued; ++i)
      mbar_wait(&full[i % STAGES], (uint32_t)(i / STAGES) & 1u, p.err, 4);
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(TM, p.nchunk);
    for (int i = 0; i < niter; ++i) {
      int s = i % STAGES;
      uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, p.err, 2)) break;
      fence_after();
      const uint64_t dr = sdesc(su32(tile(s, 0))), di = sdesc(su32(tile(s, 1))), ds = sdesc(su32(tile(s, 2)));
      const uint64_t er = sdesc(su32(tile(s, 3))), ei = sdesc(su32(tile(s, 4))), es = sdesc(su32(tile(s, 5)));
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk) {
        uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        uint64_t off = (uint64_t)(kk * 32) >> 4;   // 16 bf16 = 32 B along K inside the swizzle row
        umma(tmem, dr + off, er + off, idesc, acc);
        umma(tmem + (uint32_t)p.nchunk, di + off, ei + off, idesc, acc);
        umma(tmem + 2u * (uint32_t)p.nchunk, ds + off, es + off, idesc, acc);
      }
      umma_commit(&empty[s]);
    }
    umma_commit(&done);
  }
  __syncwarp();
  const bool have = __all_sync(0xffffffffu, mbar_wait(&done, 0, p.err, 3) ? 1 : 0) != 0;
  fence_after();
  const int row = m0 + warp * 32 + lane;
  float2* out = p.ws + (size_t)z * p.ncols_pad * p.n_pad;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  for (int cc = 0; cc < p.nchunk; cc += 16) {
    uint32_t t1[16], t2[16], t3[16];
    if (have && niter > 0) {
      tmem_ld16(tmem + lane_base + (uint32_t)cc, t1);
      tmem_ld16(tmem + lane_base + (uint32_t)(p.nchunk + cc), t2);
      tmem_ld16(tmem + lane_base + (uint32_t)(2 * p.nchunk + cc), t3);
      tmem_wait_ld();
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) t1[j] = t2[j] = t3[j] = 0u;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float a = __uint_as_float(t1[j]), b = __uint_as_float(t2[j]), c = __uint_as_float(t3[j]);
      int col = c0 + cc + j;
      if (row < p.n_pad && col < p.ncols_pad) out[(size_t)col * p.n_pad + row] = make_float2(a - b, c - a - b);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

__global__ void __launch_bounds__(128, 1) cheb_tc_kernel(const __grid_constant__ TcMaps maps, TcParams p) {
  tc_tile(maps.a, maps.b, p, blockIdx.x * TM, blockIdx.y * p.nchunk, blockIdx.z);
}

// Split v into nsplit BF16 pieces written at stride `ps` (piece p at base + p * ps).
__device__ __forceinline__ void split_store(double v, int nsplit, __nv_bfloat16* base, size_t ps, int64_t e) {
  double r = v;
  for (int p = 0; p < nsplit; ++p) {
    __nv_bfloat16 h = __double2bfloat16(r);
    base[(size_t)p * ps + e] = h;
    r -= (double)__bfloat162float(h);
  }
}

// The same pieces for a value that is already FP32, in FP32 arithmetic: each piece is the
// nearest BF16 of the remainder, and the remainder minus its nearest BF16 is exact in FP32
// (the two are within a factor of two: Sterbenz), so the pieces equal split_store's
// bit for bit without FP64 instructions (the FP64 pipe is 1/64 of the FP32 rate here).
__device__ __forceinline__ void split_store_f32(float v, int nsplit, __nv_bfloat16* base, size_t ps, int64_t e) {
  float r = v;
  for (int p = 0; p < nsplit; ++p) {
    __nv_bfloat16 h = __float2bfloat16_rn(r);
    base[(size_t)p * ps + e] = h;
    r -= __bfloat162float(h);
  }
}

struct YPlanes {
  __nv_bfloat16* base;   // [piece][part re, im, re+im][ncols_pad][n_pad]
  size_t plane;          // ncols_pad * n_pad
  int nsplit;
  __device__ __forceinline__ void store(int64_t e, float2 y) const {
    split_store_f32(y.x, nsplit, base, 3 * plane, e);
    split_store_f32(y.y, nsplit, base + plane, 3 * plane, e);
    // the exact sum of two FP32 values needs up to 25 significant bits: split in FP64
    split_store((double)y.x + (double)y.y, nsplit, base + 2 * plane, 3 * plane, e);
  }
};

// Sum split-K partials (fixed order) and apply the recurrence; write the FP32 state and
// the BF16 pieces of the new block. All arrays are transposed (column-major in Y).
// ksplit = 0 means the product term is zero (first step of the corrected filter).
// With R non-null the forcing term pc[col] * R[col][row] is added (residual-corrected
// filter: the recurrence runs on the defect D_j = p_j(C) Q - Q p_j(Theta)).
__device__ __forceinline__ void tc_epilogue_body(int n, int ncols, int n_pad, int ncols_pad, int ksplit,
                                                 const float2* ws, const float2* cur, const float2* prev, float2* outp,
                                                 const YPlanes& yp, float alpha, float beta, float gamma,
                                                 const float2* R, const float* pc) {
  int64_t total = (int64_t)ncols_pad * n_pad;
  int64_t plane = total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int col = (int)(e / n_pad), row = (int)(e % n_pad);
    float2 y = make_float2(0.f, 0.f);
    if (col < ncols && row < n) {
      float2 acc = make_float2(0.f, 0.f);
      for (int z = 0; z < ksplit; ++z) {
        float2 v = ws[(int64_t)z * plane + e];
        acc.x += v.x;
        acc.y += v.y;
      }
      y.x = alpha * acc.x;
      y.y = alpha * acc.y;
      if (cur) {
        float2 c = cur[e];
        y.x += beta * c.x;
        y.y += beta * c.y;
      }
      if (prev) {
        float2 q = prev[e];
        y.x += gamma * q.x;
        y.y += gamma * q.y;
      }
      if (R) {
        float2 r = R[e];
        float w = pc[col];
        y.x += w * r.x;
        y.y += w * r.y;
      }
    }
    outp[e] = y;
    yp.store(e, y);
  }
}

__global__ void cheb_tc_epilogue(int n, int ncols, int n_pad, int ncols_pad, int ksplit, const float2* ws,
                                 const float2* cur, const float2* prev, float2* outp, YPlanes yp, float alpha,
                                 float beta, float gamma, const float2* R, const float* pc) {
  tc_epilogue_body(n, ncols, n_pad, ncols_pad, ksplit, ws, cur, prev, outp, yp, alpha, beta, gamma, R, pc);
}

// R^T = (W - Q diag(theta))^T in FP32 (residual of the Rayleigh-Ritz pairs), transposed.
__device__ __forceinline__ void resid_to_state_body(int n, int m, int n_pad, int ncols_pad, const double2* Q,
                                                    int64_t ldq, const double2* W, int64_t ldw, const double* theta,
                                                    float2* Rt, int r0, int c0) {
  __shared__ float2 t[32][33];
  int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int k = ty; k < 32; k += 8) {
    int r = r0 + k, c = c0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (r < n && c < m) {
      double2 q = Q[(int64_t)r * ldq + c], w = W[(int64_t)r * ldw + c];
      double th = theta[c];
      v = make_float2((float)(w.x - th * q.x), (float)(w.y - th * q.y));
    }
    t[k][tx] = v;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int c = c0 + k, r = r0 + tx;
    if (c < ncols_pad && r < n_pad) Rt[(int64_t)c * n_pad + r] = t[tx][k];
  }
}

__global__ void resid_to_state(int n, int m, int n_pad, int ncols_pad, const double2* Q, int64_t ldq,
                               const double2* W, int64_t ldw, const double* theta, float2* Rt) {
  resid_to_state_body(n, m, n_pad, ncols_pad, Q, ldq, W, ldw, theta, Rt, blockIdx.x * 32, blockIdx.y * 32);
}

// Y = Q diag(pd) + D (FP64 out, row-major): the filtered block from the defect D^T.
__device__ __forceinline__ void defect_to_y_body(int n, int m, int n_pad, const float2* Dt, const double2* Q,
                                                 int64_t ldq, const double* pd, double2* Y, int64_t ldy, int r0,
                                                 int c0) {
  __shared__ float2 t[32][33];
  int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int k = ty; k < 32; k += 8) {
    int c = c0 + k, r = r0 + tx;
    t[k][tx] = (c < m && r < n) ? Dt[(int64_t)c * n_pad + r] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int r = r0 + k, c = c0 + tx;
    if (r < n && c < m) {
      float2 d = t[tx][k];
      double2 q = Q[(int64_t)r * ldq + c];
      double p = pd[c];
      Y[(int64_t)r * ldy + c] = make_double2(fma(q.x, p, (double)d.x), fma(q.y, p, (double)d.y));
    }
  }
}

__global__ void defect_to_y(int n, int m, int n_pad, const float2* Dt, const double2* Q, int64_t ldq,
                            const double* pd, double2* Y, int64_t ldy) {
  defect_to_y_body(n, m, n_pad, Dt, Q, ldq, pd, Y, ldy, blockIdx.x * 32, blockIdx.y * 32);
}

// C (FP64, n x n) -> BF16 pieces [piece][re, im, re+im][n_pad][n_pad] (zero padding).
__global__ void c_to_planes(int64_t n, int n_pad, const double2* C, int64_t ldc, __nv_bfloat16* planes, int nsplit) {
  int64_t total = (int64_t)n_pad * n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n_pad, j = e % n_pad;
    double2 v = (i < n && j < n) ? C[i * ldc + j] : make_double2(0.0, 0.0);
    split_store(v.x, nsplit, planes, 3 * (size_t)total, e);
    split_store(v.y, nsplit, planes + total, 3 * (size_t)total, e);
    split_store(v.x + v.y, nsplit, planes + 2 * total, 3 * (size_t)total, e);
  }
}

// Y (FP64 row-major n x m, ld) -> transposed FP32 state + BF16 pieces (ncols_pad x n_pad),
// through a 32 x 32 shared-memory tile for coalescing on both sides.
__global__ void y_to_state(int n, int m, int n_pad, int ncols_pad, const double2* Y, int64_t ldy, float2* st,
                           YPlanes yp) {
  __shared__ float2 t[32][33];
  int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 256 threads: ty 0..7
  for (int k = ty; k < 32; k += 8) {
    int r = r0 + k, c = c0 + tx;
    double2 v = (r < n && c < m) ? Y[(int64_t)r * ldy + c] : make_double2(0.0, 0.0);
    t[k][tx] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int c = c0 + k, r = r0 + tx;
    if (c < ncols_pad && r < n_pad) {
      float2 v = t[tx][k];
      int64_t e = (int64_t)c * n_pad + r;
      st[e] = v;
      yp.store(e, v);
    }
  }
}

__global__ void state_to_y(int n, int m, int n_pad, const float2* st, double2* Y, int64_t ldy) {
  __shared__ float2 t[32][33];
  int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int k = ty; k < 32; k += 8) {
    int c = c0 + k, r = r0 + tx;
    t[k][tx] = (c < m && r < n) ? st[(int64_t)c * n_pad + r] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int r = r0 + k, c = c0 + tx;
    if (r < n && c < m) {
      float2 v = t[tx][k];
      Y[(int64_t)r * ldy + c] = make_double2(v.x, v.y);
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool encode_2d(CUtensorMap* map, void* base, uint64_t inner, uint64_t outer, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

constexpr int kKsplitMax = 16;
constexpr int kDegMax = 64;

int pad_to(int x, int a) { return (x + a - 1) / a * a; }

void chunking(int m, int* nchunks, int* nchunk) {
  int k = (m + NMAX - 1) / NMAX;
  int c = pad_to((m + k - 1) / k, 16);
  *nchunks = k;
  *nchunk = c;
}

}  // namespace

struct FilterTC {
  int n_pad = 0, ncols_pad = 0;
  int c_nsplit = 0;                 // pieces of C currently stored
  __nv_bfloat16* Cp = nullptr;      // [MAXSPLIT][3][n_pad][n_pad]
  __nv_bfloat16* Yp = nullptr;      // [MAXSPLIT][3][ncols_pad][n_pad]
  float2 *S0 = nullptr, *S1 = nullptr, *S2 = nullptr, *S3 = nullptr, *ws = nullptr;
  float* pcoef = nullptr;           // device: [kDegMax][ncols_pad]
  double* pfinal = nullptr;         // device: [ncols_pad]
  float* h_pcoef = nullptr;         // pinned host staging
  double* h_pfinal = nullptr;
  int* err = nullptr;
  size_t bytes = 0;
  void* arena = nullptr;
};

bool tc_filter_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && get_encode() != nullptr;
}

// Zero fill on stream s: a plain cudaMemset runs on the legacy default stream, which is
// not ordered with the library's non-blocking streams, and could land after the planes
// that s writes next.
cudaError_t filter_tc_reserve(FilterTC** pf, int64_t n, int m, cudaStream_t s) {
  if (!*pf) *pf = new FilterTC();
  FilterTC* f = *pf;
  int n_pad = pad_to((int)n, TM);
  int nchunks, nchunk;
  chunking(m, &nchunks, &nchunk);
  int ncols_pad = nchunks * nchunk;
  if (n_pad <= f->n_pad && ncols_pad <= f->ncols_pad && f->arena) return cudaSuccess;
  n_pad = std::max(n_pad, f->n_pad);
  ncols_pad = std::max(ncols_pad, f->ncols_pad);
  if (f->arena) cudaFree(f->arena);
  f->arena = nullptr;
  f->c_nsplit = 0;
  size_t np2 = (size_t)n_pad * n_pad, nc = (size_t)ncols_pad * n_pad;
  auto al = [](size_t b) { return (b + 1023) & ~(size_t)1023; };
  size_t bytes = al((size_t)MAXSPLIT * 3 * np2 * 2) + al((size_t)MAXSPLIT * 3 * nc * 2) + 4 * al(nc * 8) +
                 al((size_t)kKsplitMax * nc * 8) + al((size_t)kDegMax * ncols_pad * 4) + al((size_t)ncols_pad * 8) +
                 1024;
  cudaError_t e = cudaMalloc(&f->arena, bytes);
  if (e != cudaSuccess) { f->arena = nullptr; f->n_pad = f->ncols_pad = 0; return e; }
  e = cudaMemsetAsync(f->arena, 0, bytes, s);
  if (e != cudaSuccess) return e;
  char* p = (char*)f->arena;
  f->Cp = (__nv_bfloat16*)p; p += al((size_t)MAXSPLIT * 3 * np2 * 2);
  f->Yp = (__nv_bfloat16*)p; p += al((size_t)MAXSPLIT * 3 * nc * 2);
  f->S0 = (float2*)p; p += al(nc * 8);
  f->S1 = (float2*)p; p += al(nc * 8);
  f->S2 = (float2*)p; p += al(nc * 8);
  f->S3 = (float2*)p; p += al(nc * 8);
  f->ws = (float2*)p; p += al((size_t)kKsplitMax * nc * 8);
  f->pcoef = (float*)p; p += al((size_t)kDegMax * ncols_pad * 4);
  f->pfinal = (double*)p; p += al((size_t)ncols_pad * 8);
  if (f->h_pcoef) cudaFreeHost(f->h_pcoef);
  if (f->h_pfinal) cudaFreeHost(f->h_pfinal);
  f->h_pcoef = nullptr;
  f->h_pfinal = nullptr;
  cudaMallocHost(&f->h_pcoef, (size_t)kDegMax * ncols_pad * 4);
  cudaMallocHost(&f->h_pfinal, (size_t)ncols_pad * 8);
  f->err = (int*)p;
  f->n_pad = n_pad;
  f->ncols_pad = ncols_pad;
  f->bytes = bytes;
  return cudaSuccess;
}

void filter_tc_release(FilterTC* f) {
  if (!f) return;
  if (f->h_pcoef) cudaFreeHost(f->h_pcoef);
  if (f->h_pfinal) cudaFreeHost(f->h_pfinal);
  if (f->arena) cudaFree(f->arena);
  delete f;
}

// Convert C (FP64) into its BF16 pieces; once per problem.
cudaError_t filter_tc_set_matrix(FilterTC* f, int64_t n, const double2* C, int64_t ldc, int nsplit, cudaStream_t s) {
  int64_t total = (int64_t)f->n_pad * f->n_pad;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  c_to_planes<<<blocks, 256, 0, s>>>(n, f->n_pad, C, ldc, f->Cp, nsplit);
  LAUNCH_NOTE(1);
  f->c_nsplit = nsplit;
  return cudaGetLastError();
}

namespace {

// Shared driver of the plain and the residual-corrected filter.
cudaError_t run_filter(FilterTC* f, int64_t n, int m, const double2* Y, int64_t ldy, const double2* W, int64_t ldw,
                       const double* theta_dev, const double* theta_host, double2* Yout, int64_t ldo, int deg,
                       double lo, double hi, double sc, int nsplit, int* err_host, cudaStream_t s) {
  if (deg < 1 || deg > kDegMax || nsplit < 1 || nsplit > MAXSPLIT || f->c_nsplit < nsplit) return cudaErrorInvalidValue;
  const bool corrected = (W != nullptr);
  int nchunks, nchunk;
  chunking(m, &nchunks, &nchunk);
  const int n_pad = f->n_pad;
  const int ncols_pad = f->ncols_pad;
  const size_t cplane = (size_t)n_pad * n_pad, yplane = (size_t)ncols_pad * n_pad;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int pc = 0; pc < nsplit; ++pc)
    for (int part = 0; part < 3; ++part) {
      if (!encode_2d(&maps.a[3 * pc + part], f->Cp + (3 * pc + part) * cplane, n_pad, n_pad, TK, TM) ||
          !encode_2d(&maps.b[3 * pc + part], f->Yp + (3 * pc + part) * yplane, n_pad, ncols_pad, TK, nchunk))
        return cudaErrorNotSupported;
    }
  YPlanes yp{f->Yp, yplane, nsplit};
  const int mtiles = n_pad / TM;
  const int nkb = n_pad / TK;
  int base = mtiles * nchunks;
  int ks = std::max(1, std::min(std::min(kKsplitMax, nkb / 2), 152 / std::max(base, 1)));
  int kbps = (nkb + ks - 1) / ks;
  ks = (nkb + kbps - 1) / kbps;
  TcParams p;
  p.n_pad = n_pad;
  p.nchunk = nchunk;
  p.kb_per_split = kbps;
  p.ncols_pad = ncols_pad;
  p.nseg = nseg_for(nsplit);
  p.ws = f->ws;
  p.err = f->err;
  p.tmem_cols = 32;
  while (p.tmem_cols < 3u * (uint32_t)nchunk) p.tmem_cols *= 2;
  const uint32_t stage_bytes = 3 * TM * TK * 2 + 3 * (uint32_t)nchunk * TK * 2;
  const size_t smem = (size_t)STAGES * stage_bytes + 1024;
  cudaFuncSetAttribute(cheb_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaMemsetAsync(f->err, 0, sizeof(int), s);
  // recurrence coefficients (the same for the block and for the scalars p_j(theta))
  double e = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
  double sigma = e / (sc - c), sigma1 = sigma;
  std::vector<double> al(deg), be(deg), ga(deg);
  for (int j = 0; j < deg; ++j) {
    if (j == 0) {
      al[0] = sigma1 / e;
      be[0] = -c * sigma1 / e;
      ga[0] = 0.0;
    } else {
      double sn = 1.0 / (2.0 / sigma1 - sigma);
      al[j] = 2.0 * sn / e;
      be[j] = -al[j] * c;
      ga[j] = -sigma * sn;
      sigma = sn;
    }
  }
  dim3 tg((n_pad + 31) / 32, (ncols_pad + 31) / 32);
  int64_t total = (int64_t)ncols_pad * n_pad;
  int eblocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  dim3 grid(mtiles, nchunks, ks);
  float2* prev = nullptr;
  float2* cur = f->S0;
  float2* nxt = f->S1;
  float2* spare = f->S2;
  int j0 = 0;
  if (corrected) {
    // scalar recurrence p_j(theta_c) on the host: pcoef[j][c] = alpha_j p_j(theta_c), pfinal = p_deg
    for (int col = 0; col < m; ++col) {
      double th = theta_host[col];
      double pm1 = 0.0, p0 = 1.0;
      for (int j = 0; j < deg; ++j) {
        f->h_pcoef[(size_t)j * ncols_pad + col] = (float)(al[j] * p0);
        double p1 = al[j] * th * p0 + be[j] * p0 + ga[j] * pm1;
        pm1 = p0;
        p0 = p1;
      }
      f->h_pfinal[col] = p0;
    }
    cudaMemcpyAsync(f->pcoef, f->h_pcoef, (size_t)deg * ncols_pad * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(f->pfinal, f->h_pfinal, (size_t)ncols_pad * 8, cudaMemcpyHostToDevice, s);
    resid_to_state<<<tg, 256, 0, s>>>((int)n, m, n_pad, ncols_pad, Y, ldy, W, ldw, theta_dev, f->S3);
    LAUNCH_NOTE(1);
    // D_1 = alpha_0 R (no product: D_0 = 0)
    cheb_tc_epilogue<<<eblocks, 256, 0, s>>>((int)n, m, n_pad, ncols_pad, 0, f->ws, nullptr, nullptr, cur, yp, 0.f, 0.f,
                                             0.f, f->S3, f->pcoef);
    LAUNCH_NOTE(1);
    j0 = 1;
  } else {
    y_to_state<<<tg, 256, 0, s>>>((int)n, m, n_pad, ncols_pad, Y, ldy, f->S0, yp);
    LAUNCH_NOTE(1);
  }
  for (int j = j0; j < deg; ++j) {
    cheb_tc_kernel<<<grid, 128, smem, s>>>(maps, p);
    LAUNCH_NOTE(1);
    const float2* Rj = corrected ? f->S3 : nullptr;
    const float* pcj = corrected ? f->pcoef + (size_t)j * ncols_pad : nullptr;
    cheb_tc_epilogue<<<eblocks, 256, 0, s>>>((int)n, m, n_pad, ncols_pad, ks, f->ws, cur, prev, nxt, yp, (float)al[j],
                                             (float)be[j], (float)ga[j], Rj, pcj);
    LAUNCH_NOTE(1);
    float2* old_prev = prev ? prev : spare;
    prev = cur;
    cur = nxt;
    nxt = old_prev;
  }
  if (corrected) defect_to_y<<<tg, 256, 0, s>>>((int)n, m, n_pad, cur, Y, ldy, f->pfinal, Yout, ldo);
  else state_to_y<<<tg, 256, 0, s>>>((int)n, m, n_pad, cur, Yout, ldo);
  LAUNCH_NOTE(1);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (err_host) cudaMemcpyAsync(err_host, f->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  return cudaSuccess;
}

}  // namespace

// Y (FP64 n x m, ld ldy) -> p(C) Y written to Yout (FP64, ld ldo); the same polynomial as
// the FP64 filter: degree deg, damped interval [lo, hi], scaling point sc.
cudaError_t filter_tc_apply(FilterTC* f, int64_t n, int m, const double2* Y, int64_t ldy, double2* Yout,
                            int64_t ldo, int deg, double lo, double hi, double sc, int nsplit, int* err_host,
                            cudaStream_t s) {
  return run_filter(f, n, m, Y, ldy, nullptr, 0, nullptr, nullptr, Yout, ldo, deg, lo, hi, sc, nsplit, err_host, s);
}

// Residual-corrected filter: Y = p(C) Q computed as Q p(Theta) + D, where the defect
//   D_{j+1} = alpha_j C D_j + beta_j D_j + gamma_j D_{j-1} + alpha_j R diag(p_j(Theta)),  D_0 = 0,
// follows from C Q = Q Theta + R (R = W - Q Theta, the FP64 Rayleigh-Ritz residual). The
// products C D_j run on the tensor cores; their rounding is relative to ||D||, which
// shrinks with ||R||, so the filtered block stays accurate to about u ||R|| instead of
// u ||Y||. theta (host) are the Ritz values of the columns of Q.
cudaError_t filter_tc_apply_corrected(FilterTC* f, int64_t n, int m, const double2* Q, int64_t ldq, const double2* W,
                                      int64_t ldw, const double* theta_dev, const double* theta_host, double2* Yout,
                                      int64_t ldo, int deg, double lo, double hi, double sc, int nsplit,
                                      cudaStream_t s) {
  return run_filter(f, n, m, Q, ldq, W, ldw, theta_dev, theta_host, Yout, ldo, deg, lo, hi, sc, nsplit, nullptr, s);
}

// One plain product D = C Y for tests of the tensor-core GEMM: a degree-1 filter with
// e = 1, c = 0 and scaling point 1 gives alpha = 1, beta = 0 exactly.
cudaError_t filter_tc_product(FilterTC* f, int64_t n, int m, const double2* Y, int64_t ldy, double2* D, int64_t ldd,
                              int nsplit, int* err_host, cudaStream_t s) {
  return run_filter(f, n, m, Y, ldy, nullptr, 0, nullptr, nullptr, D, ldd, 1, -1.0, 1.0, 1.0, nsplit, err_host, s);
}

// ===================================================================== grouped form
// The residual-corrected filter for every problem of a k-point batch at once: one launch
// per recurrence step covers the output tiles of all problems (a global tile list with a
// prefix sum per problem, BDesc::unit_start), and one launch per step applies the
// recurrence to all problems. The coefficients, the degree and the activity of each
// problem are read from device memory (BDesc::fco, pcoef, pfinal, flags), so the launch
// sequence is the same in every round and is captured once. The tensor maps live in
// global memory, 18 per problem.
namespace {

__device__ __forceinline__ bool tcg_runs(const BDesc& d, int j) { return d.flags[6] != 0 && j < d.flags[1]; }

__global__ void __launch_bounds__(128, 1) cheb_tcg_kernel(const BDesc* D, int np, int j, int* err) {
  const int u = blockIdx.x;
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (D[mid].unit_start <= u) lo = mid; else hi = mid - 1;
  }
  const BDesc& d = D[lo];
  if (!tcg_runs(d, j)) return;
  const int local = u - d.unit_start;
  const int per_z = d.mtiles * d.nchunks;
  const int z = local / per_z, r = local % per_z;
  if (z >= d.ks) return;
  TcParams p;
  p.n_pad = d.n_pad;
  p.nchunk = d.nchunk;
  p.kb_per_split = d.kbps;
  p.ncols_pad = d.ncols_pad;
  p.nseg = d.nseg;
  p.tmem_cols = d.tmem_cols;
  p.ws = d.tws;
  p.err = err;
  const CUtensorMap* maps = (const CUtensorMap*)d.maps;
  tc_tile(maps, maps + MAXSPLIT * 3, p, (r / d.nchunks) * TM, (r % d.nchunks) * d.nchunk, z);
}

// j = 0: D_1 = alpha_0 R; j >= 1: D_{j+1} from the split-K partials of C D_j. D_k is kept
// in S[(k - 1) mod 3].
__global__ void tcg_epilogue(const BDesc* D, int j) {
  const BDesc& d = D[blockIdx.y];
  if (!tcg_runs(d, j)) return;
  float2* S[3] = {d.S0, d.S1, d.S2};
  float2* outp = S[j % 3];
  const float2* cur = j >= 1 ? S[(j - 1) % 3] : nullptr;
  const float2* prev = j >= 2 ? S[(j - 2) % 3] : nullptr;
  const float al = j >= 1 ? (float)d.fco[3 * j] : 0.f;
  const float be = j >= 1 ? (float)d.fco[3 * j + 1] : 0.f;
  const float ga = j >= 1 ? (float)d.fco[3 * j + 2] : 0.f;
  YPlanes yp{d.Yp, (size_t)d.ncols_pad * d.n_pad, d.nsplit};
  tc_epilogue_body(d.n, d.m, d.n_pad, d.ncols_pad, j >= 1 ? d.ks : 0, d.tws, cur, prev, outp, yp, al, be, ga, d.S3,
                   d.pcoef + (size_t)j * d.ncols_pad);
}

__global__ void tcg_resid_to_state(const BDesc* D) {
  const BDesc& d = D[blockIdx.z];
  if (d.flags[6] == 0) return;
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  if (r0 >= d.n_pad || c0 >= d.ncols_pad) return;
  resid_to_state_body(d.n, d.m, d.n_pad, d.ncols_pad, d.Q, d.m, d.W, d.m, d.theta, d.S3, r0, c0);
}

// Y1 = Q diag(p_deg(theta)) + D_deg
__global__ void tcg_defect_to_y(const BDesc* D) {
  const BDesc& d = D[blockIdx.z];
  if (d.flags[6] == 0) return;
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  if (r0 >= d.n || c0 >= d.m) return;
  float2* S[3] = {d.S0, d.S1, d.S2};
  const int deg = d.flags[1];
  defect_to_y_body(d.n, d.m, d.n_pad, S[(deg - 1) % 3], d.Q, d.m, d.pfinal, d.Y1, d.m, r0, c0);
}

__global__ void tcg_c_to_planes(const BDesc* D) {
  const BDesc& d = D[blockIdx.y];
  if (d.flags[0] == 0) return;
  const int64_t n = d.n, n_pad = d.n_pad, total = n_pad * n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n_pad, k = e % n_pad;
    double2 v = (i < n && k < n) ? d.C[i * n + k] : make_double2(0.0, 0.0);
    split_store(v.x, d.nsplit, d.Cp, 3 * (size_t)total, e);
    split_store(v.y, d.nsplit, d.Cp + total, 3 * (size_t)total, e);
    split_store(v.x + v.y, d.nsplit, d.Cp + 2 * total, 3 * (size_t)total, e);
  }
}

}  // namespace

void tcg_geometry(int64_t n, int m, int* n_pad, int* ncols_pad, int* nchunk, int* nchunks) {
  *n_pad = pad_to((int)n, TM);
  chunking(m, nchunks, nchunk);
  *ncols_pad = *nchunks * *nchunk;
}

int tcg_nseg(int nsplit) { return nseg_for(nsplit); }

size_t tcg_smem_bytes(int nchunk_max) {
  return (size_t)STAGES * (3 * TM * TK * 2 + 3 * (size_t)nchunk_max * TK * 2) + 1024;
}

size_t tcg_map_bytes() { return sizeof(CUtensorMap) * MAXSPLIT * 3 * 2; }

bool tcg_encode_maps(const BDesc& d, void* maps_host) {
  CUtensorMap* a = (CUtensorMap*)maps_host;
  CUtensorMap* b = a + MAXSPLIT * 3;
  std::memset(maps_host, 0, tcg_map_bytes());
  const size_t cplane = (size_t)d.n_pad * d.n_pad, yplane = (size_t)d.ncols_pad * d.n_pad;
  for (int pc = 0; pc < d.nsplit; ++pc)
    for (int part = 0; part < 3; ++part) {
      if (!encode_2d(&a[3 * pc + part], d.Cp + (3 * pc + part) * cplane, d.n_pad, d.n_pad, TK, TM) ||
          !encode_2d(&b[3 * pc + part], d.Yp + (3 * pc + part) * yplane, d.n_pad, d.ncols_pad, TK, d.nchunk))
        return false;
    }
  return true;
}

void tcg_set_matrix(const BDesc* D, int np, int64_t npad2_max, cudaStream_t s) {
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((npad2_max + 255) / 256, 256));
  tcg_c_to_planes<<<dim3(blocks, np), 256, 0, s>>>(D);
  LAUNCH_NOTE(1);
}

cudaError_t tcg_prepare(int nchunk_max) {
  return cudaFuncSetAttribute(cheb_tcg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tcg_smem_bytes(nchunk_max));
}

// The launch sequence of one filter application (no host synchronisation, capturable);
// tcg_prepare must have been called for this nchunk_max first.
cudaError_t tcg_filter(const BDesc* D, const TcgShape& g, int* err, cudaStream_t s) {
  const size_t smem = tcg_smem_bytes(g.nchunk_max);
  dim3 tg((g.n_pad_max + 31) / 32, (g.ncols_pad_max + 31) / 32, g.np);
  int eb = (int)std::max<int64_t>(1, std::min<int64_t>((g.nc_max + 255) / 256, 64));
  tcg_resid_to_state<<<tg, 256, 0, s>>>(D);
  tcg_epilogue<<<dim3(eb, g.np), 256, 0, s>>>(D, 0);
  LAUNCH_NOTE(2);
  for (int j = 1; j < g.steps; ++j) {
    cheb_tcg_kernel<<<g.units, 128, smem, s>>>(D, g.np, j, err);
    tcg_epilogue<<<dim3(eb, g.np), 256, 0, s>>>(D, j);
    LAUNCH_NOTE(2);
  }
  tcg_defect_to_y<<<tg, 256, 0, s>>>(D);
  LAUNCH_NOTE(1);
  return cudaGetLastError();
}

}  // namespace gevp
