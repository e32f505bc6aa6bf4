// FP64 complex matrix products emulated on the tcgen05 tensor cores (Ozaki scheme):
// D = op(A) op(B) with FP64-class accuracy from exact BF16 products. On this part an SM
// retires two FP64 FMAs per clock but thousands of BF16 tensor flops, so the n^3 products
// of the reduction to standard form, and the n^2 m products with an n x n operand, run far
// faster this way than on the FP64 pipe.
//
//  1. Splitting. Every row i of op(A) is scaled by 2^-e_i so that its largest real or
//     imaginary part lies in [1/4, 1/2), rounded to the integer q = round(a 2^(7S))
//     (|q| <= 2^(7S-1)) and written as S signed base-128 digits, a = 2^e_i sum_s d_s 2^-7s,
//     |d_s| <= 64. Columns of op(B) likewise, with exponents f_j. Digits are small integers,
//     exact in BF16. The rounding leaves at most 2^(e_i - 7S - 1) per entry.
//  2. Digit products on the tensor cores. |d d'| <= 2^12, so an FP32 accumulation over at
//     most 4096 products is exact (every partial sum is an integer of magnitude <= 2^24).
//     The complex product is the real product of the embedding [[Ar, -Ai], [Ai, Ar]]
//     [Br; Bi] = [Re; Im], 2K real terms per output, so K is cut into exact units of at
//     most 2048 complex terms. Only digit pairs with s + t <= S + 1 are formed: the pairs
//     left out weigh less than the rounding of step 1.
//  3. Summation. The products of one level L = s + t share the scale 2^-7L and are summed
//     exactly as 32-bit integers; the levels are combined by a Horner recurrence in FP64
//     (one rounding per level), from the smallest level up, and the result is scaled by
//     2^(e_i + f_j).
// Error per entry, relative to 2^(e_i + f_j) <= 16 max_k|a_ik| max_k|b_kj|: about
// 2K (S + 3) 2^(-7S - 2) in the worst case (K complex terms), the FP64 product's bound
// K u sum_k |a_ik||b_kj| being of the same order for S = 8.
//
// GEMM kernel: one CTA per 128 x 128 tile of the real or the imaginary part of D (128 x 144
// for a D of 129..144 columns, with one accumulator, see oz_gemm_kernel). Warp 8
// issues TMA loads (3D maps: k, row, digit; 128-byte swizzle; six stages), warp 9 issues
// the MMAs of one unit (digit pair, K chunk) into one of two TMEM accumulators (128
// columns each) while warps 0-7 drain the other: each thread owns one row and 64 columns,
// converts the exact FP32 sums to integers and adds them up per level; at the end of a
// level the FP64 Horner state, kept in the upper 256 TMEM columns, is updated. When a
// tile's K range is short (S K <= 2048: the thin products with K = m), all pairs of a
// level accumulate in one buffer, still exactly, and are drained once per level. A grid that
// would leave SMs idle (a short M or N) cuts K into slices whose FP64 partials a second
// kernel sums in slice order; a device flag can make a launch a no-op (a converged batch
// problem inside a captured graph). All waits are bounded; on expiry the kernel records an
// error code, stops issuing work, waits (bounded) for the copies it issued, frees its TMEM
// and returns. Operand rows come from the rows of a matrix or, through a transposing
// splitter, from its columns.
#include "gevp_internal.cuh"
#include "tc_ptx.cuh"
#include <cuda.h>
#include <algorithm>
#include <cstring>

namespace gevp {

namespace {

constexpr int OZ_TM = 128;
constexpr int OZ_TN = 128;   // the usual tile width (a wider one serves 129..144 columns)
constexpr int OZ_TK = 64;
constexpr int OZ_ST = 6;
constexpr int OZ_KCHUNK = 2048;
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = (OZ_EPI_WARPS + 2) * 32;
constexpr int OZ_MAXPAIRS = kOzSlicesMax * (kOzSlicesMax + 1) / 2;
constexpr uint32_t OZ_A_BYTES = OZ_TM * OZ_TK * 2;   // one 128 x 64 BF16 box of A
// a stage: the A box and a TN x 64 box of B (both multiples of the 1024-byte swizzle atom)
__host__ __device__ constexpr uint32_t oz_stage_bytes(int TN) { return OZ_A_BYTES + (uint32_t)TN * OZ_TK * 2; }
constexpr size_t oz_smem(int TN) { return (size_t)OZ_ST * oz_stage_bytes(TN) + 1024; }

struct OzMaps {
  CUtensorMap a[2];   // op(A) digit planes: re, im
  CUtensorMap b[3];   // op(B)^T digit planes: re, im, -im
};

struct OzParams {
  int M, N;        // complex output size
  int mt;          // 128-row tiles of one part
  int k_pad;       // padded K (multiple of 64)
  int S;           // digits per entry
  int triA;        // 1: op(A)[i][k] = 0 for k > i;  2: op(A)[i][k] = 0 for k < i
  int triB;        // 1: op(B)[k][j] = 0 for k < j;  2: op(B)[k][j] = 0 for k > j
  const int* ea;   // row exponents of op(A)
  const int* eb;   // column exponents of op(B)
  double2* D;
  int64_t ldd;
  int* err;
  const int* active;   // nullable device flag: 0 = skip the whole launch (a converged problem)
  double* ws;          // split K: this slice's partial, [z][part][M][N] (null: write D)
  int kspan;           // split K: the K range of one slice (a multiple of 64)
};

// TN: tile width (128, or 144 for 129..144 columns in one tile); NBUF: TMEM accumulator
// buffers (two of TN columns with the Horner state of TN values in the upper 256 columns;
// one for TN = 144, whose Horner state takes 288 columns)
template <int TN, int NBUF>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const __grid_constant__ OzMaps maps, OzParams p) {
  static_assert(NBUF * TN + 2 * TN <= 512, "TMEM: accumulators and Horner state exceed 512 columns");
  constexpr int CPT = TN / 2;   // columns of one epilogue thread
  constexpr uint32_t STAGE = oz_stage_bytes(TN);
  if (p.active && *p.active == 0) return;   // uniform: before any barrier or TMEM allocation
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[OZ_ST], empty[OZ_ST], tfull[2], tempty[2];
  __shared__ uint32_t tmem_sh;
  __shared__ uint8_t pair_s[OZ_MAXPAIRS], pair_t[OZ_MAXPAIRS], pair_last[OZ_MAXPAIRS];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // the real- and imaginary-part tiles of the same rows are launched next to each other:
  // they read the same B tiles (first half of the embedding's K) while both are in L2
  const int part = blockIdx.y & 1;   // 0: real part of D, 1: imaginary part
  const int m0 = (blockIdx.y >> 1) * OZ_TM;
  const int n0 = blockIdx.x * TN;
  // K range of the tile from the triangular structure, in whole 64-blocks
  int klo = 0, khi = p.k_pad;
  if (p.triA == 1) khi = min(khi, m0 + OZ_TM);
  if (p.triA == 2) klo = max(klo, m0);
  if (p.triB == 1) klo = max(klo, n0);
  // (whole 64-blocks: n0 + TN is not a multiple of 64 for TN = 144, and the K entries past
  // the triangle up to the next block boundary are zero digits of the masked operand)
  if (p.triB == 2) khi = min(khi, (n0 + TN + OZ_TK - 1) / OZ_TK * OZ_TK);
  if (p.ws) {   // split K: this CTA's slice
    klo = max(klo, (int)blockIdx.z * p.kspan);
    khi = min(khi, ((int)blockIdx.z + 1) * p.kspan);
  }
  const int klen = max(0, khi - klo);
  const int nchunk = (klen + OZ_KCHUNK - 1) / OZ_KCHUNK;
  const int npairs = p.S * (p.S + 1) / 2;
  const int nunits = npairs * nchunk;
  // A short K range (the thin products, K = m): all digit pairs of one level accumulate in
  // the same TMEM buffer and are drained once per level instead of once per pair. Exact
  // while a level's sum stays an FP32 integer: at most S pairs x 2 klen real products of
  // at most 2^12 each, S klen <= 2048.
  const bool grouped = nchunk == 1 && p.S * klen <= 2048;
  auto chunk_blocks = [&](int c) {   // 64-blocks of chunk c (one part of the embedding)
    const int a = klo + c * OZ_KCHUNK;
    return (min(khi, a + OZ_KCHUNK) - a) / OZ_TK;
  };

  if (threadIdx.x == 0) {
    // pairs by level L = s + t from S + 1 down to 2, s ascending inside a level
    int i = 0;
    for (int L = p.S + 1; L >= 2; --L)
      for (int s = 1; s < L; ++s, ++i) {
        pair_s[i] = (uint8_t)s;
        pair_t[i] = (uint8_t)(L - s);
        pair_last[i] = (uint8_t)(s == L - 1);
      }
    for (int s = 0; s < OZ_ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], OZ_EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_sh;

  if (warp == OZ_EPI_WARPS && lane == 0) {
    // producer: for block kh (embedding half) of a unit, the real-part tile multiplies
    // A planes re | im with B planes re | -im, the imaginary-part tile im | re with re | im
    int it = 0;
    bool ok = true;
    for (int u = 0; u < nunits && ok; ++u) {
      const int pi = u / nchunk, c = u % nchunk;
      const int sa = pair_s[pi] - 1, tb = pair_t[pi] - 1;
      const int nb = chunk_blocks(c);
      const int kbase = klo + c * OZ_KCHUNK;
      for (int i = 0; i < 2 * nb; ++i, ++it) {
        const int st = it % OZ_ST;
        if (it >= OZ_ST && !mbar_wait(&empty[st], ((uint32_t)(it / OZ_ST) & 1u) ^ 1u, p.err, 21)) {
          ok = false;
          break;
        }
        const int kh = i / nb, kx = kbase + (i % nb) * OZ_TK;
        const int pa = part ^ kh;
        const int pb = kh == 0 ? 0 : (part == 0 ? 2 : 1);
        uint8_t* sa_tile = smem + (size_t)st * STAGE;
        mbar_expect_tx(&full[st], STAGE);
        tma_load_3d(sa_tile, &maps.a[pa], kx, m0, sa, &full[st]);
        tma_load_3d(sa_tile + OZ_A_BYTES, &maps.b[pb], kx, n0, tb, &full[st]);
      }
    }
    // every copy issued has landed before the CTA leaves (normally they were all consumed;
    // after a wait elsewhere gave up they may still be in flight): bounded waits on the
    // last issue of every stage
    for (int i = max(0, it - OZ_ST); i < it; ++i) mbar_wait(&full[i % OZ_ST], (uint32_t)(i / OZ_ST) & 1u, p.err, 25);
  } else if (warp == OZ_EPI_WARPS + 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(OZ_TM, TN);
    int it = 0, grp = 0;   // accumulation groups: the units, or the levels when grouped
    bool ok = true;
    for (int u = 0; u < nunits && ok; ++u) {
      const int pi = u / nchunk;
      const bool gs = !grouped || pair_s[pi] == 1, ge = !grouped || pair_last[pi];
      const int buf = grp % NBUF;
      if (gs && grp >= NBUF && !mbar_wait(&tempty[buf], (uint32_t)((grp / NBUF) - 1) & 1u, p.err, 22)) break;
      fence_after();
      const uint32_t dt = tmem + (uint32_t)(buf * TN);
      const int nb2 = 2 * chunk_blocks(u % nchunk);
      for (int i = 0; i < nb2; ++i, ++it) {
        const int st = it % OZ_ST;
        if (!mbar_wait(&full[st], (uint32_t)(it / OZ_ST) & 1u, p.err, 23)) {
          ok = false;
          break;
        }
        fence_after();
        const uint8_t* base = smem + (size_t)st * STAGE;
        const uint64_t da = sdesc(su32(base)), db = sdesc(su32(base + OZ_A_BYTES));
#pragma unroll
        for (int kk = 0; kk < OZ_TK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;
          umma(dt, da + off, db + off, idesc, (i > 0 || kk > 0 || !gs) ? 1u : 0u);
        }
        umma_commit(&empty[st]);
      }
      if (!ok) break;
      if (ge) {
        umma_commit(&tfull[buf]);
        ++grp;
      }
    }
  } else if (warp < OZ_EPI_WARPS) {
    const int q = warp & 3, ch = warp >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const uint32_t col0 = (uint32_t)(ch * CPT);
    const uint32_t hcol = (uint32_t)(NBUF * TN) + 2u * col0;   // FP64 Horner state: 2 TMEM columns per value
    const int row = m0 + q * 32 + lane;
    const bool row_ok = row < p.M;
    const int er = row_ok ? p.ea[row] : 0;
    // output: interleaved complex D (double 2 (row ldd + col) + part), or this slice's
    // partial (double row N + col of plane (z, part) of the workspace)
    double* Dd = p.ws ? p.ws + ((size_t)blockIdx.z * 2 + part) * (size_t)p.M * p.N : (double*)p.D;
    const int64_t ostr = p.ws ? 1 : 2, opart = p.ws ? 0 : part, old = p.ws ? p.N : p.ldd;
    int acc[CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[j] = 0;
    bool first_level = true, ok = true;
    int grp = 0;
    for (int u = 0; u < nunits; ++u) {
      // (grouped: the buffer holds a level's running sum until its last pair)
      if (grouped && !pair_last[u / nchunk]) continue;
      const int buf = grp % NBUF;
      ok = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], (uint32_t)(grp / NBUF) & 1u, p.err, 24) ? 1 : 0) != 0;
      if (!ok) break;
      ++grp;
      fence_after();
      // (CPT = 72: the fifth load's last 8 columns are not this thread's and are ignored)
#pragma unroll
      for (int g = 0; g < (CPT + 15) / 16; ++g) {
        uint32_t r[16];
        tmem_ld16(tmem + lane_base + (uint32_t)(buf * TN) + col0 + 16u * g, r);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (16 * g + j < CPT) acc[16 * g + j] += __float2int_rn(__uint_as_float(r[j]));
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      const int pi = u / nchunk;
      if (u % nchunk != nchunk - 1 || !pair_last[pi]) continue;
      // end of a level: h <- h 2^-7 + I_L (FP64), kept in TMEM until the last level
      const bool last_level = (pi == npairs - 1);
#pragma unroll
      for (int g = 0; g < CPT / 8; ++g) {
        uint32_t hv[16];
        if (!first_level) {
          tmem_ld16(tmem + lane_base + hcol + 16u * g, hv);
          tmem_wait_ld();
        }
        double h8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const double prev = first_level ? 0.0 : __hiloint2double((int)hv[2 * j + 1], (int)hv[2 * j]);
          h8[j] = fma(prev, 0x1p-7, (double)acc[8 * g + j]);
          acc[8 * g + j] = 0;
        }
        if (!last_level) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            hv[2 * j] = (uint32_t)__double2loint(h8[j]);
            hv[2 * j + 1] = (uint32_t)__double2hiint(h8[j]);
          }
          tmem_st16(tmem + lane_base + hcol + 16u * g, hv);
        } else if (row_ok) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = n0 + (int)col0 + 8 * g + j;
            if (col < p.N) Dd[ostr * ((int64_t)row * old + col) + opart] = ldexp(h8[j], er + p.eb[col] - 14);
          }
        }
      }
      if (!last_level) tmem_wait_st();
      first_level = false;
    }
    if (nunits == 0 && row_ok) {
      for (int j = 0; j < CPT; ++j) {
        const int col = n0 + (int)col0 + j;
        if (col < p.N) Dd[ostr * ((int64_t)row * old + col) + opart] = 0.0;
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// D = sum over the K slices of their partials (real and imaginary planes), in slice order
__global__ void oz_sum_slices_kernel(int M, int N, int nz, const double* ws, double2* D, int64_t ldd,
                                     const int* active) {
  if (active && *active == 0) return;
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int z = 0; z < nz; ++z) {
      re += ws[(size_t)(2 * z) * total + e];
      im += ws[(size_t)(2 * z + 1) * total + e];
    }
    D[(e / N) * ldd + (e % N)] = make_double2(re, im);
  }
}

// Digits of one operand row r (a row of op(A), or a column of op(B)), entries k < K. The
// row is row r of the stored X (oz_split_rows_kernel) or its column r
// (oz_split_cols_kernel), conjugated if conj; mask 1 keeps k >= r with the diagonal halved
// (a column of the lower triangle of a Hermitian matrix, tril(A) with its diagonal split
// between A and A^H), mask 2 keeps k <= r, mask 3 keeps k >= r. Writes the exponent of the
// row and the S digits of the real part, the imaginary part and (npl = 3) the negated
// imaginary part into planes [npl][S][rows_pad][k_pad]; rows and entries past the operand
// are zero. A row with a non-finite entry sets *bad.
__device__ __forceinline__ double2 oz_masked(double2 v, int r, int k, int conj, int mask) {
  if ((mask == 1 && k < r) || (mask == 2 && k > r) || (mask == 3 && k < r)) return make_double2(0.0, 0.0);
  if (conj) v.y = -v.y;
  if (mask == 1 && k == r) v = make_double2(0.5 * v.x, 0.5 * v.y);
  return v;
}

__device__ __forceinline__ double2 oz_entry(const double2* X, int64_t ldx, int r, int k, int K, int conj, int mask) {
  if (k >= K) return make_double2(0.0, 0.0);
  return oz_masked(X[(int64_t)r * ldx + k], r, k, conj, mask);
}

// The splitting works on the IEEE-754 fields with integer instructions only: one SM
// retires about two FP64 operations per clock on this part, and a conversion, a scaling
// and a maximum per entry on the FP64 pipe made the splitter several times slower than
// its memory traffic.
//
// |v| as an ordered integer key: for finite values the order of the keys is the order of
// the magnitudes; an exponent field of all ones (Inf or NaN) is reported as non-finite.
__device__ __forceinline__ unsigned long long oz_abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ bool oz_key_finite(unsigned long long key) { return (key >> 52) != 0x7FF; }

// floor(log2 |x|) of the value with magnitude key `key` (> 0, finite), as ilogb.
__device__ __forceinline__ int oz_key_ilogb(unsigned long long key) {
  const int E = (int)(key >> 52);
  return E != 0 ? E - 1023 : (63 - __clzll((long long)key)) - 1074;
}

// round(x 2^shift) to the nearest integer, ties to even, for finite x with
// |x 2^shift| < 2^62: x = M 2^k' with the integer significand M < 2^53, so the result is
// M shifted left, or shifted right with the dropped bits deciding the rounding. The same
// value as converting ldexp(x, shift) with round-to-nearest-even, without FP64
// instructions. A non-finite x gives 0 (its row is reported as bad).
__device__ __forceinline__ long long oz_round_scaled(double x, int shift) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0x7FF) return 0;
  unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  int k = shift - 1074;                    // subnormal: x = M 2^-1074
  if (E != 0) {
    M |= 1ull << 52;
    k = E - 1075 + shift;
  }
  unsigned long long q;
  if (k >= 0) {
    q = M << k;
  } else if (k < -63) {
    q = 0;                                 // |x 2^shift| < 2^-10
  } else {
    const int r = -k;
    q = M >> r;
    const unsigned long long rem = M & ((1ull << (r - 1) << 1) - 1), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}

__device__ __forceinline__ void oz_digits_q(long long q, int S, __nv_bfloat16* out, size_t plane) {
  for (int s = S - 1; s >= 1; --s) {
    const long long d = ((q + 64) & 127) - 64;
    out[(size_t)s * plane] = __int2bfloat16_rn((int)d);
    q = (q - d) >> 7;
  }
  out[0] = __int2bfloat16_rn((int)q);
}

// the digits of x, of -x (npl = 3: the negated imaginary part) from the same rounding:
// rounding to nearest even is odd-symmetric, so round(-x 2^shift) = -round(x 2^shift)
__device__ __forceinline__ void oz_digits(double x, int shift, int S, __nv_bfloat16* out, size_t plane) {
  oz_digits_q(oz_round_scaled(x, shift), S, out, plane);
}

__global__ void __launch_bounds__(256) oz_split_rows_kernel(int rows, int K, const double2* X, int64_t ldx, int conj,
                                                            int mask, int S, int npl, int rows_pad, int k_pad,
                                                            __nv_bfloat16* planes, int* ex, int* bad,
                                                            const int* active) {
  if (active && *active == 0) return;
  __shared__ unsigned long long red[8];
  const int r = blockIdx.x;
  unsigned long long mx = 0;   // largest magnitude key of the finite entries
  bool nonfinite = false;
  if (r < rows)
    for (int k = threadIdx.x; k < K; k += 256) {
      const double2 v = oz_entry(X, ldx, r, k, K, conj, mask);
      const unsigned long long kx = oz_abs_key(v.x), ky = oz_abs_key(v.y);
      if (!oz_key_finite(kx) || !oz_key_finite(ky)) nonfinite = true;
      else mx = max(mx, max(kx, ky));
    }
  if (__any_sync(0xffffffffu, nonfinite) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = red[0];
  for (int w = 1; w < 8; ++w) mx = max(mx, red[w]);
  // 2^e > 2 max|entry|: the scaled row lies below 1/2
  const int e = mx > 0 ? oz_key_ilogb(mx) + 2 : 0;
  if (threadIdx.x == 0 && r < rows) ex[r] = e;
  const int shift = 7 * S - e;
  const size_t plane = (size_t)rows_pad * k_pad;
  const size_t pstride = (size_t)S * plane;
  for (int k = threadIdx.x; k < k_pad; k += 256) {
    const double2 v = r < rows ? oz_entry(X, ldx, r, k, K, conj, mask) : make_double2(0.0, 0.0);
    const size_t o = (size_t)r * k_pad + k;
    const long long qy = oz_round_scaled(v.y, shift);
    oz_digits(v.x, shift, S, planes + o, plane);
    oz_digits_q(qy, S, planes + pstride + o, plane);
    if (npl == 3) oz_digits_q(-qy, S, planes + 2 * pstride + o, plane);
  }
}

// Columns of X (K rows x R columns, ld ldx) as operand rows. Pass 1: the exponent of each
// column (threads across consecutive columns, coalesced). Pass 2: a 32 x 32 tile of X
// staged in shared memory and written out transposed, so the digit stores run along k.
constexpr int OZ_CT = 32;

// ex[j] starts at kExpNone; each block (32 columns x one slice of rows) raises it to the
// exponent of its slice's largest entry (the exponent of a maximum is the maximum of the
// exponents); a column with no nonzero entry keeps kExpNone, read as 0.
constexpr int kExpNone = (int)0x80808080;   // the cudaMemset byte pattern 0x80
constexpr int OZ_CE_ROWS = 256;             // rows per slice

__global__ void __launch_bounds__(256) oz_cols_exp_kernel(int R, int K, const double2* X, int64_t ldx, int conj,
                                                          int mask, int* ex, int* bad, const int* active) {
  if (active && *active == 0) return;
  __shared__ unsigned long long red[8][OZ_CT];
  const int j = blockIdx.x * OZ_CT + threadIdx.x;
  const int k0 = blockIdx.y * OZ_CE_ROWS, k1 = min(K, k0 + OZ_CE_ROWS);
  unsigned long long mx = 0;
  bool nonfinite = false;
  if (j < R)
    for (int k = k0 + threadIdx.y; k < k1; k += 8) {
      const double2 v = oz_masked(X[(int64_t)k * ldx + j], j, k, conj, mask);
      const unsigned long long kx = oz_abs_key(v.x), ky = oz_abs_key(v.y);
      if (!oz_key_finite(kx) || !oz_key_finite(ky)) nonfinite = true;
      else mx = max(mx, max(kx, ky));
    }
  if (nonfinite) atomicExch(bad, 1);
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && j < R) {
    for (int t = 1; t < 8; ++t) mx = max(mx, red[t][threadIdx.x]);
    if (mx > 0) atomicMax(&ex[j], oz_key_ilogb(mx) + 2);
  }
}

__global__ void __launch_bounds__(256) oz_cols_digits_kernel(int R, int K, const double2* X, int64_t ldx, int conj,
                                                             int mask, int S, int npl, int rows_pad, int k_pad,
                                                             __nv_bfloat16* planes, const int* ex,
                                                             const int* active) {
  if (active && *active == 0) return;
  __shared__ double2 tile[OZ_CT][OZ_CT + 1];   // [k][j]
  const int k0 = blockIdx.x * OZ_CT, j0 = blockIdx.y * OZ_CT;
  for (int i = threadIdx.y; i < OZ_CT; i += 8) {
    const int k = k0 + i, j = j0 + threadIdx.x;
    tile[i][threadIdx.x] = (k < K && j < R) ? oz_masked(X[(int64_t)k * ldx + j], j, k, conj, mask)
                                            : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const size_t plane = (size_t)rows_pad * k_pad;
  const size_t pstride = (size_t)S * plane;
  const int k = k0 + threadIdx.x;
  if (k >= k_pad) return;
  for (int jj = threadIdx.y; jj < OZ_CT; jj += 8) {
    const int j = j0 + jj;
    if (j >= rows_pad) break;
    const double2 v = tile[threadIdx.x][jj];
    const int e = j < R ? ex[j] : 0;
    const int shift = 7 * S - (e == kExpNone ? 0 : e);
    const size_t o = (size_t)j * k_pad + k;
    const long long qy = oz_round_scaled(v.y, shift);
    oz_digits(v.x, shift, S, planes + o, plane);
    oz_digits_q(qy, S, planes + pstride + o, plane);
    if (npl == 3) oz_digits_q(-qy, S, planes + 2 * pstride + o, plane);
  }
}

// columns with no nonzero entry: exponent 0 (the product kernel scales by 2^(e_i + f_j))
__global__ void oz_exp_fix_kernel(int R, int* ex, const int* active) {
  if (active && *active == 0) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < R && ex[j] == kExpNone) ex[j] = 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn oz_encode() {
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

// 3D map over the digit planes of one part: (k, row, digit), box 64 x box_rows x 1
bool oz_map(CUtensorMap* map, void* base, int k_pad, int rows_pad, int S, int box_rows) {
  EncodeTiledFn enc = oz_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)k_pad, (cuuint64_t)rows_pad, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)k_pad * 2, (cuuint64_t)rows_pad * k_pad * 2};
  cuuint32_t box[3] = {OZ_TK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t oz_operand_bytes(int rows, int K, int S, int npl) {
  const size_t rp = (size_t)(rows + OZ_TM - 1) / OZ_TM * OZ_TM;
  const size_t kp = (size_t)(K + OZ_TK - 1) / OZ_TK * OZ_TK;
  return (size_t)npl * S * rp * kp * 2 + ((size_t)rows * 4 + 255) / 256 * 256;
}

bool oz_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && oz_encode() != nullptr;
}

cudaError_t oz_split(OzOperand& op, void* mem, int rows, int K, const double2* X, int64_t ldx, int conj, int mask,
                     int S, int npl, int* bad, cudaStream_t s, bool cols, const int* active) {
  if (S < 1 || S > kOzSlicesMax || (npl != 2 && npl != 3)) return cudaErrorInvalidValue;
  op.rows = rows;
  op.K = K;
  op.S = S;
  op.npl = npl;
  op.rows_pad = (rows + OZ_TM - 1) / OZ_TM * OZ_TM;
  op.k_pad = (K + OZ_TK - 1) / OZ_TK * OZ_TK;
  op.planes = (__nv_bfloat16*)mem;
  op.ex = (int*)((char*)mem + (size_t)npl * S * op.rows_pad * op.k_pad * 2);
  if (rows == 0) return cudaSuccess;
  if (!cols) {
    oz_split_rows_kernel<<<op.rows_pad, 256, 0, s>>>(rows, K, X, ldx, conj, mask, S, npl, op.rows_pad, op.k_pad,
                                                     op.planes, op.ex, bad, active);
    LAUNCH_NOTE(1);
  } else {
    cudaMemsetAsync(op.ex, 0x80, (size_t)rows * sizeof(int), s);
    dim3 egrid((rows + OZ_CT - 1) / OZ_CT, std::max(1, (K + OZ_CE_ROWS - 1) / OZ_CE_ROWS));
    oz_cols_exp_kernel<<<egrid, dim3(OZ_CT, 8), 0, s>>>(rows, K, X, ldx, conj, mask, op.ex, bad, active);
    dim3 grid((op.k_pad + OZ_CT - 1) / OZ_CT, (op.rows_pad + OZ_CT - 1) / OZ_CT);
    oz_cols_digits_kernel<<<grid, dim3(OZ_CT, 8), 0, s>>>(rows, K, X, ldx, conj, mask, S, npl, op.rows_pad, op.k_pad,
                                                          op.planes, op.ex, active);
    oz_exp_fix_kernel<<<(rows + 255) / 256, 256, 0, s>>>(rows, op.ex, active);
    LAUNCH_NOTE(3);
  }
  return cudaGetLastError();
}

size_t oz_split_k_doubles(int M, int N) { return (size_t)kOzSplitKMax * 2 * M * N; }

cudaError_t oz_gemm(const OzOperand& A, const OzOperand& B, int triA, int triB, double2* D, int64_t ldd, int* err,
                    cudaStream_t s, const int* active, double* ws, size_t ws_doubles) {
  if (A.K != B.K || A.S != B.S || A.npl != 2 || B.npl != 3 || A.k_pad != B.k_pad) return cudaErrorInvalidValue;
  // the integer sums of one level hold at most S products of 2^24 per K chunk
  if (A.k_pad > 15 * OZ_KCHUNK) return cudaErrorInvalidValue;
  if (A.rows == 0 || B.rows == 0) return cudaSuccess;
  // 129..144 columns (the Rayleigh-Ritz block W = C Q at m = 140) in one 144-wide tile with
  // a single accumulator instead of a second 128-wide tile that is mostly padding (the
  // operand's rows are padded to 256, so the 144-row box stays inside them)
  const int tn = (B.rows > OZ_TN && B.rows <= 144) ? 144 : OZ_TN;
  const int ntile = (B.rows + tn - 1) / tn;
  OzMaps maps;
  std::memset(&maps, 0, sizeof maps);
  const size_t pa = (size_t)A.S * A.rows_pad * A.k_pad, pb = (size_t)B.S * B.rows_pad * B.k_pad;
  for (int i = 0; i < 2; ++i)
    if (!oz_map(&maps.a[i], A.planes + i * pa, A.k_pad, A.rows_pad, A.S, OZ_TM)) return cudaErrorInvalidValue;
  for (int i = 0; i < 3; ++i)
    if (!oz_map(&maps.b[i], B.planes + i * pb, B.k_pad, B.rows_pad, B.S, tn)) return cudaErrorInvalidValue;
  OzParams p;
  p.M = A.rows;
  p.N = B.rows;
  p.mt = A.rows_pad / OZ_TM;
  p.k_pad = A.k_pad;
  p.S = A.S;
  p.triA = triA;
  p.triB = triB;
  p.ea = A.ex;
  p.eb = B.ex;
  p.D = D;
  p.ldd = ldd;
  p.err = err;
  p.active = active;
  p.ws = nullptr;
  p.kspan = p.k_pad;
  int nz = 1;
  if (ws) {
    // grids that leave SMs idle (short M or N) cut K into slices until about one wave
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ctas = ntile * 2 * p.mt;
    const int kb = p.k_pad / OZ_TK;
    int want = std::min(std::min(kOzSplitKMax, kb), sms / std::max(ctas, 1));
    if (want >= 2) {
      p.kspan = (kb + want - 1) / want * OZ_TK;
      nz = (p.k_pad + p.kspan - 1) / p.kspan;
      if ((size_t)nz * 2 * p.M * p.N <= ws_doubles) p.ws = ws;
      else nz = 1, p.kspan = p.k_pad;
    }
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<OZ_TN, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)oz_smem(OZ_TN));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(oz_gemm_kernel<144, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem(144));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(ntile, 2 * p.mt, nz);
  void* kt0 = kt_enabled() ? kt_begin(s) : nullptr;
  if (tn == 144) oz_gemm_kernel<144, 1><<<grid, OZ_THREADS, oz_smem(144), s>>>(maps, p);
  else oz_gemm_kernel<OZ_TN, 2><<<grid, OZ_THREADS, oz_smem(OZ_TN), s>>>(maps, p);
  LAUNCH_NOTE(1);
  if (kt0) {
    // algorithmic: the complex product over the K ranges the tiles process (8 flop per
    // complex multiply-add); executed: the digit pairs' real products of the embedding
    double alg = 0.0;
    for (int mt = 0; mt < p.mt; ++mt)
      for (int nt = 0; nt < ntile; ++nt) {
        const int m0 = mt * OZ_TM, n0 = nt * tn;
        int klo = 0, khi = p.k_pad;
        if (triA == 1) khi = std::min(khi, m0 + OZ_TM);
        if (triA == 2) klo = std::max(klo, m0);
        if (triB == 1) klo = std::max(klo, n0);
        if (triB == 2) khi = std::min(khi, (n0 + tn + OZ_TK - 1) / OZ_TK * OZ_TK);
        const int rows = std::min(OZ_TM, p.M - m0), cols = std::min(tn, p.N - n0);
        if (khi > klo && rows > 0 && cols > 0) alg += 8.0 * rows * cols * (double)(khi - klo);
      }
    const double pairs = (double)p.S * (p.S + 1) / 2;
    kt_end(kt0, 1, alg, alg * pairs, s);
  }
  if (p.ws) {
    const int64_t total = (int64_t)p.M * p.N;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4 * 152);
    oz_sum_slices_kernel<<<blocks, 256, 0, s>>>(p.M, p.N, nz, p.ws, D, ldd, active);
    LAUNCH_NOTE(1);
  }
  return cudaGetLastError();
}

}  // namespace gevp
