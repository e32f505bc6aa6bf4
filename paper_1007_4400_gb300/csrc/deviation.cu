// Deviation angles between the eigenvectors of consecutive problems of a sequence and the
// re-indexing that matches them (Sec. "A new computational philosophy", paragraph
// "Eigenvectors evolution"): the cosine of the angle between x_old_i and x_new_j in the B
// inner product is c_ij = |x_old_i^H B x_new_j| / (||x_old_i||_B ||x_new_j||_B), and the
// normalised deviation angle of a matched pair is acos(c) / (pi / 2) (1.00 = pi / 2).
//
// The device part is the O(n^2 k) work: W = B X (FP64 complex GEMM, issued by the caller),
// the B-norms as column dot products Re(x_j^H w_j), and the k_old x k_new cosine table.
// The paper gives no algorithm for the matching; here it is the optimal assignment of old
// to new vectors under the cost 1 - c_ij, pairs whose eigenvalues differ by more than an
// energy window costing more than any assignment of pairs inside it. That is a small
// sequential combinatorial problem (k <= a few thousand) solved on the host by the
// shortest-augmenting-path form of the Hungarian method (Kuhn-Munkres with dual
// potentials), started from the row minima, which already match almost every row when the
// eigenvectors moved little.
#include "gevp_internal.cuh"
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

namespace gevp {

namespace {

constexpr int kNormCols = 32;   // columns per block (one warp across consecutive columns)
constexpr int kNormRows = 8;    // row lanes per block

// part[s * k + j] = sum over the rows of slice s of Re(conj(X[r][j]) * W[r][j])
__global__ void __launch_bounds__(kNormCols* kNormRows) dev_bnorm_partial_kernel(int64_t n, int k, const double2* X,
                                                                                 int64_t ldx, const double2* W,
                                                                                 int64_t ldw, int64_t rows_per,
                                                                                 double* part) {
  __shared__ double red[kNormRows][kNormCols];
  const int j = blockIdx.x * kNormCols + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = std::min<int64_t>(n, r0 + rows_per);
  double acc = 0.0;
  if (j < k)
    for (int64_t r = r0 + threadIdx.y; r < r1; r += kNormRows) {
      const double2 x = X[r * ldx + j], w = W[r * ldw + j];
      acc = fma(x.x, w.x, acc);
      acc = fma(x.y, w.y, acc);
    }
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && j < k) {
    double s = red[0][threadIdx.x];
    for (int t = 1; t < kNormRows; ++t) s += red[t][threadIdx.x];
    part[(int64_t)blockIdx.y * k + j] = s;
  }
}

__global__ void dev_bnorm_final_kernel(int k, int slices, const double* part, double* nrm2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int t = 0; t < slices; ++t) s += part[(int64_t)t * k + j];
  nrm2[j] = s;
}

// c[i][j] = min(1, |O[i][j]| / (sqrt(no2[i]) sqrt(nn2[j]))); bad = 1 if a norm is not a
// positive finite number
__global__ void dev_cos_kernel(int ko, int kn, const double2* O, int64_t ldo, const double* no2, const double* nn2,
                               double* c, int64_t ldc, int* bad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= kn) return;
  const double a = no2[i], b = nn2[j];
  if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b)) {
    *bad = 1;
    c[(int64_t)i * ldc + j] = 0.0;
    return;
  }
  const double2 o = O[(int64_t)i * ldo + j];
  const double v = hypot(o.x, o.y) / (sqrt(a) * sqrt(b));
  if (!isfinite(v)) *bad = 1;
  c[(int64_t)i * ldc + j] = v < 1.0 ? v : 1.0;
}

}  // namespace

int deviation_norm_slices(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(64, (n + 255) / 256));
}

void column_bnorms(int64_t n, int k, const double2* X, int64_t ldx, const double2* W, int64_t ldw, double* part,
                   double* nrm2, cudaStream_t s) {
  if (k <= 0) return;
  const int slices = deviation_norm_slices(n);
  const int64_t rows_per = (n + slices - 1) / slices;
  dim3 grid((k + kNormCols - 1) / kNormCols, slices);
  dev_bnorm_partial_kernel<<<grid, dim3(kNormCols, kNormRows), 0, s>>>(n, k, X, ldx, W, ldw, rows_per, part);
  dev_bnorm_final_kernel<<<(k + 255) / 256, 256, 0, s>>>(k, slices, part, nrm2);
  LAUNCH_NOTE(2);
}

void overlap_cosines(int ko, int kn, const double2* O, int64_t ldo, const double* no2, const double* nn2, double* c,
                     int64_t ldc, int* bad, cudaStream_t s) {
  if (ko <= 0 || kn <= 0) return;
  dim3 grid((kn + 127) / 128, ko);
  dev_cos_kernel<<<grid, 128, 0, s>>>(ko, kn, O, ldo, no2, nn2, c, ldc, bad);
  LAUNCH_NOTE(1);
}

// Minimum-cost assignment of every row of the ko x kn (ko <= kn) cost table to a distinct
// column (row-major, ld kn): perm[i] = column of row i. Hungarian method in its
// shortest-augmenting-path form: dual potentials u (rows) and v (columns) with
// u_i + v_j <= cost_ij everywhere and equality on matched pairs; each free row is joined by
// a Dijkstra-like search over reduced costs that ends at a free column, the potentials of
// the searched part move by the distances found, and the path's matching is flipped.
// Started from u_i = min_j cost_ij, v = 0 and every row matched to its first minimum
// column when that column is still free (all such pairs are tight).
void assign_min_cost(int ko, int kn, const double* cost, int64_t* perm) {
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> u(ko, 0.0), v(kn, 0.0), dist(kn);
  std::vector<int> col_of(ko, -1), row_of(kn, -1), prev(kn), order;
  std::vector<char> done(kn);
  order.reserve(kn);
  for (int i = 0; i < ko; ++i) {
    const double* ci = cost + (int64_t)i * kn;
    int jm = 0;
    for (int j = 1; j < kn; ++j)
      if (ci[j] < ci[jm]) jm = j;
    u[i] = ci[jm];
    if (row_of[jm] < 0) {
      row_of[jm] = i;
      col_of[i] = jm;
    }
  }
  for (int i0 = 0; i0 < ko; ++i0) {
    if (col_of[i0] >= 0) continue;
    // search from row i0: dist[j] = least reduced cost of reaching column j
    std::fill(dist.begin(), dist.end(), inf);
    std::fill(done.begin(), done.end(), 0);
    order.clear();
    int i = i0, jfree = -1;
    double dcur = 0.0;   // distance of the row being expanded
    while (true) {
      const double* ci = cost + (int64_t)i * kn;
      for (int j = 0; j < kn; ++j) {
        if (done[j]) continue;
        const double d = dcur + ci[j] - u[i] - v[j];
        if (d < dist[j]) {
          dist[j] = d;
          prev[j] = i;
        }
      }
      int jb = -1;
      for (int j = 0; j < kn; ++j)
        if (!done[j] && (jb < 0 || dist[j] < dist[jb])) jb = j;
      done[jb] = 1;
      order.push_back(jb);
      if (row_of[jb] < 0) {
        jfree = jb;
        break;
      }
      i = row_of[jb];
      dcur = dist[jb];
    }
    // potentials: every settled column j moves by dist[jfree] - dist[j] (v down, the row
    // matched to it up), which keeps all reduced costs non-negative and makes the path tight
    const double dend = dist[jfree];
    u[i0] += dend;
    for (int j : order) {
      if (j == jfree) continue;
      const double t = dend - dist[j];
      v[j] -= t;
      u[row_of[j]] += t;
    }
    // flip the alternating path back from the free column
    int j = jfree;
    while (true) {
      const int r = prev[j];
      const int jn = col_of[r];
      row_of[j] = r;
      col_of[r] = j;
      if (r == i0) break;
      j = jn;
    }
  }
  for (int i = 0; i < ko; ++i) perm[i] = col_of[i];
}

}  // namespace gevp
