/*
 * gevp_oracle.c -- plain, slow, FP64 CPU oracle for the Hermitian-definite generalized
 * eigenproblem A x = lambda B x (the per-k-point problem of the paper's FLAPW cycle,
 * Eq. 3 and the sentence that follows it: A Hermitian, B Hermitian positive definite).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may link, load or call
 * this file; only the tests, the package entry point's smoke check and the CPU-baseline
 * leg of the benchmark use it. It shares no code, header or constant with the CUDA path.
 *
 * What it computes is the plain definition: the full spectrum of the pencil, of which the
 * lowest nev pairs are kept, with B-orthonormal eigenvectors (X^H B X = I) and lambda
 * ascending. Steps (all row-major, interleaved complex128, unblocked, textbook):
 *   1. B = L L^H, lower Cholesky with a pivot check (LAPACK potrf convention for info).
 *   2. C = L^-1 A L^-H by forward substitution on the columns of A, then on the rows,
 *      followed by C <- (C + C^H)/2.
 *   3. Eigenpairs of C by either
 *        (a) complex two-sided cyclic Jacobi in a parallel round-robin ordering
 *            (Golub & Van Loan Sec. 8.5, with the 2x2 Hermitian block turned real by a
 *            diagonal phase), or
 *        (b) Householder reduction to a real symmetric tridiagonal T (zlarfg-style
 *            reflectors with real beta), Sturm-count bisection for the lowest nev
 *            eigenvalues and inverse iteration with in-cluster re-orthogonalisation
 *            (Wilkinson / Peters-Wilkinson), back-transformed through the reflectors.
 *   4. Sort ascending (ties stable by index), keep nev, X = L^-H Y.
 * Extra checkers: the inertia of A - sigma B by a Bunch-Kaufman LDL^H (Sylvester's law
 * of inertia: the count of negative pivots equals the number of eigenvalues of the
 * pencil below sigma), and the band-energy gradient dE/dA = X X^H, dE/dB = -X Lambda X^H
 * for E = sum of the lowest nev eigenvalues (first-order perturbation theory).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define IDX(i, j, ld) ((int64_t)(i) * (ld) + (j))

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static double abs2(cplx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* ---- 1. Cholesky B = L L^H (lower). Returns 0, or the 1-based index of the first
 *         pivot that is not positive (L is then partial). ------------------------- */
int64_t orc_potrf(int64_t n, const cplx *B, cplx *L) {
  memset(L, 0, sizeof(cplx) * (size_t)(n * n));
  for (int64_t j = 0; j < n; ++j) {
    double d = creal(B[IDX(j, j, n)]);
    for (int64_t k = 0; k < j; ++k) d -= abs2(L[IDX(j, k, n)]);
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    L[IDX(j, j, n)] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      cplx s = B[IDX(i, j, n)];
      for (int64_t k = 0; k < j; ++k) s -= L[IDX(i, k, n)] * conj(L[IDX(j, k, n)]);
      L[IDX(i, j, n)] = s / ljj;
    }
  }
  return 0;
}

/* Solve L W = R in place (L lower, n x n; R n x ncol, row-major, ld = ncol). */
static void forward_subst(int64_t n, const cplx *L, cplx *R, int64_t ncol) {
  for (int64_t i = 0; i < n; ++i) {
    cplx *ri = R + i * ncol;
    for (int64_t k = 0; k < i; ++k) {
      cplx lik = L[IDX(i, k, n)];
      if (lik == 0) continue;
      const cplx *rk = R + k * ncol;
#pragma omp parallel for schedule(static) if (ncol > 256)
      for (int64_t j = 0; j < ncol; ++j) ri[j] -= lik * rk[j];
    }
    cplx inv = 1.0 / L[IDX(i, i, n)];
    for (int64_t j = 0; j < ncol; ++j) ri[j] *= inv;
  }
}

/* Solve L^H X = Y in place (back substitution with the upper factor L^H). */
static void backward_subst_LH(int64_t n, const cplx *L, cplx *Y, int64_t ncol) {
  for (int64_t i = n - 1; i >= 0; --i) {
    cplx *yi = Y + i * ncol;
    /* row i of L^H is conj(L[k, i]) for k >= i */
    for (int64_t k = i + 1; k < n; ++k) {
      cplx u = conj(L[IDX(k, i, n)]);
      if (u == 0) continue;
      const cplx *yk = Y + k * ncol;
      for (int64_t j = 0; j < ncol; ++j) yi[j] -= u * yk[j];
    }
    cplx inv = 1.0 / conj(L[IDX(i, i, n)]);
    for (int64_t j = 0; j < ncol; ++j) yi[j] *= inv;
  }
}

void orc_solve_LH(int64_t n, const cplx *L, cplx *Y, int64_t ncol) { backward_subst_LH(n, L, Y, ncol); }

/* ---- 2. C = L^-1 A L^-H, then its Hermitian part. -------------------------------- */
void orc_reduce(int64_t n, const cplx *A, const cplx *L, cplx *C) {
  cplx *W = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  memcpy(W, A, sizeof(cplx) * (size_t)(n * n));
  forward_subst(n, L, W, n);               /* W = L^-1 A */
  /* C = W L^-H  <=>  C^H = L^-1 W^H */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) C[IDX(i, j, n)] = conj(W[IDX(j, i, n)]);
  forward_subst(n, L, C, n);               /* C now holds (W L^-H)^H */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) W[IDX(i, j, n)] = conj(C[IDX(j, i, n)]);
  /* Hermitian part */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      C[IDX(i, j, n)] = 0.5 * (W[IDX(i, j, n)] + conj(W[IDX(j, i, n)]));
  free(W);
}

/* ---- 3a. Hermitian two-sided Jacobi, parallel round-robin ordering. -------------
 * M (n x n Hermitian) is overwritten; w receives all n eigenvalues (unsorted, in the
 * order of V's columns), V the eigenvectors (columns). Returns the number of sweeps. */
int orc_jacobi(int64_t n, cplx *M, double *w, cplx *V, int max_sweeps, double tol) {
  memset(V, 0, sizeof(cplx) * (size_t)(n * n));
  for (int64_t i = 0; i < n; ++i) V[IDX(i, i, n)] = 1.0;
  if (n == 1) { w[0] = creal(M[0]); return 0; }
  double fro = 0.0;
  for (int64_t i = 0; i < n * n; ++i) fro += abs2(M[i]);
  fro = sqrt(fro);
  int64_t np = (n % 2) ? n + 1 : n;          /* players; np-1 is a bye when n is odd */
  int64_t npairs = np / 2;
  int64_t *ring = (int64_t *)malloc(sizeof(int64_t) * (size_t)np);
  int64_t *P = (int64_t *)malloc(sizeof(int64_t) * (size_t)npairs);
  int64_t *Qx = (int64_t *)malloc(sizeof(int64_t) * (size_t)npairs);
  cplx *U = (cplx *)malloc(sizeof(cplx) * (size_t)(4 * npairs)); /* u11 u12 u21 u22 */
  for (int64_t i = 0; i < np; ++i) ring[i] = i;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j)
        if (i != j) off += abs2(M[IDX(i, j, n)]);
    if (sqrt(off) <= tol * fro) break;
    for (int64_t step = 0; step < np - 1; ++step) {
      /* pairs of this round: (ring[k], ring[np-1-k]) */
      for (int64_t k = 0; k < npairs; ++k) {
        int64_t a = ring[k], b = ring[np - 1 - k];
        P[k] = a < b ? a : b;
        Qx[k] = a < b ? b : a;
      }
      /* rotation parameters from the current 2x2 blocks */
      for (int64_t k = 0; k < npairs; ++k) {
        int64_t p = P[k], q = Qx[k];
        cplx *u = U + 4 * k;
        u[0] = 1; u[1] = 0; u[2] = 0; u[3] = 1;
        if (q >= n) continue;                  /* bye */
        cplx apq = M[IDX(p, q, n)];
        double r = cabs(apq);
        if (r == 0.0) continue;
        double app = creal(M[IDX(p, p, n)]), aqq = creal(M[IDX(q, q, n)]);
        cplx ph = apq / r;                     /* e^{i phi} */
        /* real symmetric 2x2 [[app, r],[r, aqq]]: Golub-Van Loan sym.schur2 */
        double tau = (aqq - app) / (2.0 * r);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* U = diag(1, conj(ph)) * [[c, s], [-s, c]] */
        u[0] = c;
        u[1] = s;
        u[2] = -s * conj(ph);
        u[3] = c * conj(ph);
      }
      /* columns: M <- M U, V <- V U (rows independent) */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = 0; k < npairs; ++k) {
          int64_t p = P[k], q = Qx[k];
          if (q >= n) continue;
          const cplx *u = U + 4 * k;
          cplx mp = M[IDX(i, p, n)], mq = M[IDX(i, q, n)];
          M[IDX(i, p, n)] = mp * u[0] + mq * u[2];
          M[IDX(i, q, n)] = mp * u[1] + mq * u[3];
          cplx vp = V[IDX(i, p, n)], vq = V[IDX(i, q, n)];
          V[IDX(i, p, n)] = vp * u[0] + vq * u[2];
          V[IDX(i, q, n)] = vp * u[1] + vq * u[3];
        }
      }
      /* rows: M <- U^H M (pairs independent) */
#pragma omp parallel for schedule(static)
      for (int64_t k = 0; k < npairs; ++k) {
        int64_t p = P[k], q = Qx[k];
        if (q >= n) continue;
        const cplx *u = U + 4 * k;
        cplx c11 = conj(u[0]), c12 = conj(u[2]), c21 = conj(u[1]), c22 = conj(u[3]);
        for (int64_t j = 0; j < n; ++j) {
          cplx mp = M[IDX(p, j, n)], mq = M[IDX(q, j, n)];
          M[IDX(p, j, n)] = c11 * mp + c12 * mq;
          M[IDX(q, j, n)] = c21 * mp + c22 * mq;
        }
        M[IDX(p, q, n)] = 0;
        M[IDX(q, p, n)] = 0;
        M[IDX(p, p, n)] = creal(M[IDX(p, p, n)]);
        M[IDX(q, q, n)] = creal(M[IDX(q, q, n)]);
      }
      /* rotate the ring, keeping ring[0] fixed */
      int64_t last = ring[np - 1];
      for (int64_t i = np - 1; i > 1; --i) ring[i] = ring[i - 1];
      ring[1] = last;
    }
  }
  for (int64_t i = 0; i < n; ++i) w[i] = creal(M[IDX(i, i, n)]);
  free(ring); free(P); free(Qx); free(U);
  return sweep;
}

/* ---- 3b. Householder tridiagonalisation (lower), in place. -----------------------
 * On exit d (n) and e (n-1) hold the real tridiagonal T = Q^H M Q, and the reflector
 * vectors v_k (v_k[0] = 1 implicit) sit below the subdiagonal of column k of M, with
 * H_k = I - tau_k v_k v_k^H acting on rows/columns k+1..n-1, Q = H_0 H_1 ... H_{n-2}. */
void orc_tridiag(int64_t n, cplx *M, double *d, double *e, cplx *tau) {
  cplx *p = (cplx *)malloc(sizeof(cplx) * (size_t)n);
  for (int64_t k = 0; k + 1 < n; ++k) {
    int64_t m = n - k - 1;                     /* length of x = M[k+1:, k] */
    cplx alpha = M[IDX(k + 1, k, n)];
    double xn2 = 0.0;
    for (int64_t i = k + 2; i < n; ++i) xn2 += abs2(M[IDX(i, k, n)]);
    cplx tk;
    double beta;
    if (xn2 == 0.0 && cimag(alpha) == 0.0) {
      tk = 0.0;
      beta = creal(alpha);
    } else {
      beta = -copysign(sqrt(abs2(alpha) + xn2), creal(alpha));
      tk = (beta - alpha) / beta;
      cplx sc = 1.0 / (alpha - beta);
      for (int64_t i = k + 2; i < n; ++i) M[IDX(i, k, n)] *= sc;
    }
    tau[k] = tk;
    e[k] = beta;
    M[IDX(k + 1, k, n)] = 1.0;                  /* v[0] = 1 while applying */
    if (tk != 0.0) {
      /* p = tau * M22 * v  (M22 = M[k+1:, k+1:], Hermitian; use the full block) */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < m; ++i) {
        cplx s = 0;
        const cplx *row = M + (k + 1 + i) * n + (k + 1);
        for (int64_t j = 0; j < m; ++j) s += row[j] * M[IDX(k + 1 + j, k, n)];
        p[i] = tk * s;
      }
      /* w = p - (1/2)(tau * p^H v) v ; s = tau * (p^H v) is real */
      cplx ph_v = 0;
      for (int64_t i = 0; i < m; ++i) ph_v += conj(p[i]) * M[IDX(k + 1 + i, k, n)];
      cplx half = -0.5 * tk * ph_v;
      for (int64_t i = 0; i < m; ++i) p[i] += half * M[IDX(k + 1 + i, k, n)];
      /* M22 -= v w^H + w v^H */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < m; ++i) {
        cplx vi = M[IDX(k + 1 + i, k, n)], wi = p[i];
        cplx *row = M + (k + 1 + i) * n + (k + 1);
        for (int64_t j = 0; j < m; ++j) {
          cplx vj = M[IDX(k + 1 + j, k, n)];
          row[j] -= vi * conj(p[j]) + wi * conj(vj);
        }
      }
    }
    d[k] = creal(M[IDX(k, k, n)]);
  }
  d[n - 1] = creal(M[IDX(n - 1, n - 1, n)]);
  free(p);
}

/* Number of eigenvalues of the real symmetric tridiagonal (d, e) strictly below x. */
static int64_t sturm_count(int64_t n, const double *d, const double *e, double x, double pivmin) {
  int64_t cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int64_t i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

/* Eigenvalues k0..k0+cnt-1 (0-based, ascending) of T by bisection. */
static void tridiag_bisect(int64_t n, const double *d, const double *e, int64_t cnt, double *lam) {
  double lo = d[0], hi = d[0], tnorm = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    if (d[i] - r < lo) lo = d[i] - r;
    if (d[i] + r > hi) hi = d[i] + r;
    if (fabs(d[i]) + r > tnorm) tnorm = fabs(d[i]) + r;
  }
  double pivmin = 1e-300 + 1e-290 * tnorm;
#pragma omp parallel for schedule(dynamic)
  for (int64_t k = 0; k < cnt; ++k) {
    double a = lo - 1e-12 * tnorm - 1e-300, b = hi + 1e-12 * tnorm + 1e-300;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (a + b);
      if (mid <= a || mid >= b) break;
      if (sturm_count(n, d, e, mid, pivmin) > k) b = mid; else a = mid;
      if (b - a <= 2.0 * 2.2e-16 * fmax(fabs(a), fabs(b)) + 1e-300) break;
    }
    lam[k] = 0.5 * (a + b);
  }
}

/* Inverse iteration on (T - lam I) by Gaussian elimination with partial pivoting on the
 * tridiagonal; z (n) on entry holds the start vector, on exit the eigenvector. */
static void tridiag_inverse_step(int64_t n, const double *d, const double *e, double lam, double tnorm,
                                 double *z, double *wk) {
  /* wk: 5n doubles: main diag u, first super u1, second super u2, multipliers l, pivot flags */
  double *u = wk, *u1 = wk + n, *u2 = wk + 2 * n, *l = wk + 3 * n, *piv = wk + 4 * n;
  double eps = 2.2e-16 * tnorm + 1e-300;
  for (int64_t i = 0; i < n; ++i) { u[i] = d[i] - lam; u1[i] = (i + 1 < n) ? e[i] : 0.0; u2[i] = 0.0; }
  for (int64_t i = 0; i + 1 < n; ++i) {
    /* rows i and i+1; row i+1 has sub e[i], diag u[i+1], super u1[i+1] */
    double sub = e[i];
    if (fabs(sub) > fabs(u[i])) {
      /* swap rows i and i+1 */
      double mult = u[i] / sub;
      double ni = sub, n1 = u[i + 1], n2 = u1[i + 1];
      double oi1 = u1[i], oi2 = u2[i];
      u[i] = ni; u1[i] = n1; u2[i] = n2;
      l[i] = mult; piv[i] = 1.0;
      u[i + 1] = oi1 - mult * n1;
      u1[i + 1] = oi2 - mult * n2;
    } else {
      double mult = (u[i] != 0.0) ? sub / u[i] : 0.0;
      l[i] = mult; piv[i] = 0.0;
      u[i + 1] -= mult * u1[i];
      u1[i + 1] -= mult * u2[i];
    }
  }
  /* forward: apply row ops to z */
  for (int64_t i = 0; i + 1 < n; ++i) {
    if (piv[i] != 0.0) { double t = z[i]; z[i] = z[i + 1]; z[i + 1] = t - l[i] * z[i]; }
    else z[i + 1] -= l[i] * z[i];
  }
  /* back substitution on upper triangular with 2 superdiagonals */
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = z[i];
    if (i + 1 < n) s -= u1[i] * z[i + 1];
    if (i + 2 < n) s -= u2[i] * z[i + 2];
    double p = u[i];
    if (fabs(p) < eps) p = (p >= 0 ? eps : -eps);
    z[i] = s / p;
  }
}

/* Lowest nev eigenpairs of Hermitian C (n x n, untouched) by 3b. Y is n x nev row-major. */
void orc_heev_tridiag(int64_t n, const cplx *C, int64_t nev, double *lam, cplx *Y) {
  cplx *M = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  memcpy(M, C, sizeof(cplx) * (size_t)(n * n));
  double *d = (double *)malloc(sizeof(double) * (size_t)n);
  double *e = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
  cplx *tau = (cplx *)malloc(sizeof(cplx) * (size_t)(n > 1 ? n - 1 : 1));
  if (n > 1) orc_tridiag(n, M, d, e, tau); else d[0] = creal(M[0]);
  tridiag_bisect(n, d, e, nev, lam);
  double tnorm = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    if (r > tnorm) tnorm = r;
  }
  double ortol = 1e-3 * tnorm;
  double *Z = (double *)malloc(sizeof(double) * (size_t)(n * nev)); /* column k at Z + k*n */
  double *wk = (double *)malloc(sizeof(double) * (size_t)(5 * n));
  int64_t cluster_start = 0;
  for (int64_t k = 0; k < nev; ++k) {
    if (k > 0 && lam[k] - lam[k - 1] > ortol) cluster_start = k;
    /* separate coincident eigenvalues slightly, as LAPACK's stein does */
    double lk = lam[k];
    if (k > cluster_start && lk - lam[k - 1] < 10.0 * 2.2e-16 * tnorm) lk = lam[k - 1] + 10.0 * 2.2e-16 * tnorm;
    double *z = Z + k * n;
    for (int64_t i = 0; i < n; ++i) z[i] = 1.0 + 0.1 * sin(0.7 * (double)(i + 1) * (double)(k + 1) + 0.3);
    for (int it = 0; it < 5; ++it) {
      /* re-orthogonalise against earlier vectors of the cluster (MGS) */
      for (int64_t j = cluster_start; j < k; ++j) {
        double *zj = Z + j * n;
        double dot = 0.0;
        for (int64_t i = 0; i < n; ++i) dot += zj[i] * z[i];
        for (int64_t i = 0; i < n; ++i) z[i] -= dot * zj[i];
      }
      double nrm = 0.0;
      for (int64_t i = 0; i < n; ++i) nrm += z[i] * z[i];
      nrm = sqrt(nrm);
      for (int64_t i = 0; i < n; ++i) z[i] /= nrm;
      tridiag_inverse_step(n, d, e, lk, tnorm, z, wk);
    }
    for (int64_t j = cluster_start; j < k; ++j) {
      double *zj = Z + j * n;
      double dot = 0.0;
      for (int64_t i = 0; i < n; ++i) dot += zj[i] * z[i];
      for (int64_t i = 0; i < n; ++i) z[i] -= dot * zj[i];
    }
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) nrm += z[i] * z[i];
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < n; ++i) z[i] /= nrm;
  }
  /* back-transform y = H_0 H_1 ... H_{n-2} z  (apply H_{n-2} first) */
#pragma omp parallel for schedule(dynamic)
  for (int64_t k = 0; k < nev; ++k) {
    cplx *y = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) y[i] = Z[k * n + i];
    for (int64_t r = n - 2; r >= 0; --r) {
      cplx t = tau[r];
      if (t == 0.0) continue;
      /* v = (1, M[r+2:, r]) on rows r+1.. ; y <- y - t v (v^H y) */
      cplx s = y[r + 1];
      for (int64_t i = r + 2; i < n; ++i) s += conj(M[IDX(i, r, n)]) * y[i];
      s *= t;
      y[r + 1] -= s;
      for (int64_t i = r + 2; i < n; ++i) y[i] -= s * M[IDX(i, r, n)];
    }
    for (int64_t i = 0; i < n; ++i) Y[IDX(i, k, nev)] = y[i];
    free(y);
  }
  free(M); free(d); free(e); free(tau); free(Z); free(wk);
}

/* All eigenpairs of Hermitian C by Jacobi, sorted ascending; lowest nev returned. */
int orc_heev_jacobi(int64_t n, const cplx *C, int64_t nev, double *lam, cplx *Y) {
  cplx *M = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  memcpy(M, C, sizeof(cplx) * (size_t)(n * n));
  int sweeps = orc_jacobi(n, M, w, V, 40, 1e-15);
  /* stable insertion sort of indices by eigenvalue */
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  for (int64_t i = 1; i < n; ++i) {
    int64_t t = ord[i];
    int64_t j = i - 1;
    while (j >= 0 && w[ord[j]] > w[t]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = t;
  }
  for (int64_t k = 0; k < nev; ++k) {
    lam[k] = w[ord[k]];
    for (int64_t i = 0; i < n; ++i) Y[IDX(i, k, nev)] = V[IDX(i, ord[k], n)];
  }
  free(M); free(V); free(w); free(ord);
  return sweeps;
}

/* ---- Full oracle solve: lowest nev pairs of A x = lambda B x. ---------------------
 * method 0 = Jacobi, 1 = tridiagonal. X is n x nev (row-major), B-orthonormal.
 * Returns 0, or -info (info = 1-based failing Cholesky pivot) when B is not HPD. */
int64_t orc_solve(int64_t n, const cplx *A, const cplx *B, int64_t nev, int method, double *lam, cplx *X) {
  cplx *L = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  int64_t info = orc_potrf(n, B, L);
  if (info) { free(L); return -info; }
  cplx *C = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  orc_reduce(n, A, L, C);
  if (method == 0) orc_heev_jacobi(n, C, nev, lam, X);
  else orc_heev_tridiag(n, C, nev, lam, X);
  backward_subst_LH(n, L, X, nev);          /* X = L^-H Y */
  free(L); free(C);
  return 0;
}

/* Per-column residual ||A x_i - lam_i B x_i||_2 / (normA * ||x_i||_2). */
void orc_residuals(int64_t n, const cplx *A, const cplx *B, int64_t nev, const double *lam,
                   const cplx *X, double normA, double *res) {
#pragma omp parallel for schedule(dynamic)
  for (int64_t k = 0; k < nev; ++k) {
    double r2 = 0.0, x2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      cplx ax = 0, bx = 0;
      for (int64_t j = 0; j < n; ++j) {
        cplx xj = X[IDX(j, k, nev)];
        ax += A[IDX(i, j, n)] * xj;
        bx += B[IDX(i, j, n)] * xj;
      }
      r2 += abs2(ax - lam[k] * bx);
      x2 += abs2(X[IDX(i, k, nev)]);
    }
    res[k] = sqrt(r2) / (normA * sqrt(x2));
  }
}

/* ---- Inertia: number of negative eigenvalues of the Hermitian matrix A - sigma B,
 * via Bunch-Kaufman symmetric-pivoted LDL^H (Golub & Van Loan Sec. 4.4). Also returns
 * the number of exactly zero pivots in *nzero. By Sylvester's law (B HPD) the count
 * equals the number of eigenvalues of the pencil below sigma. -------------------- */
static void sym_swap(int64_t n, cplx *M, int64_t i, int64_t j) {
  if (i == j) return;
  for (int64_t k = 0; k < n; ++k) { cplx t = M[IDX(i, k, n)]; M[IDX(i, k, n)] = M[IDX(j, k, n)]; M[IDX(j, k, n)] = t; }
  for (int64_t k = 0; k < n; ++k) { cplx t = M[IDX(k, i, n)]; M[IDX(k, i, n)] = M[IDX(k, j, n)]; M[IDX(k, j, n)] = t; }
}

int64_t orc_inertia(int64_t n, const cplx *A, const cplx *B, double sigma, int64_t *nzero) {
  cplx *M = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  for (int64_t i = 0; i < n * n; ++i) M[i] = A[i] - sigma * B[i];
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  int64_t neg = 0, zero = 0, k = 0;
  while (k < n) {
    double lam = 0.0;
    int64_t r = k;
    for (int64_t i = k + 1; i < n; ++i) {
      double a = cabs(M[IDX(i, k, n)]);
      if (a > lam) { lam = a; r = i; }
    }
    double akk = fabs(creal(M[IDX(k, k, n)]));
    if (lam == 0.0) {
      double dk = creal(M[IDX(k, k, n)]);
      if (dk < 0) ++neg; else if (dk == 0) ++zero;
      ++k;
      continue;
    }
    int two = 0;
    if (akk < alpha * lam) {
      double sig = 0.0;
      for (int64_t j = k; j < n; ++j)
        if (j != r) { double a = cabs(M[IDX(j, r, n)]); if (a > sig) sig = a; }
      if (akk * sig >= alpha * lam * lam) {
        /* 1x1 at k */
      } else if (fabs(creal(M[IDX(r, r, n)])) >= alpha * sig) {
        sym_swap(n, M, k, r);
      } else {
        sym_swap(n, M, k + 1, r);
        two = 1;
      }
    }
    if (!two) {
      double dk = creal(M[IDX(k, k, n)]);
      if (dk < 0) ++neg; else if (dk == 0) ++zero;
#pragma omp parallel for schedule(static)
      for (int64_t i = k + 1; i < n; ++i) {
        cplx f = M[IDX(i, k, n)] / dk;
        for (int64_t j = k + 1; j < n; ++j) M[IDX(i, j, n)] -= f * conj(M[IDX(j, k, n)]);
      }
      k += 1;
    } else {
      double a = creal(M[IDX(k, k, n)]), c = creal(M[IDX(k + 1, k + 1, n)]);
      cplx b = M[IDX(k + 1, k, n)];           /* E = [[a, conj(b)], [b, c]] */
      double det = a * c - abs2(b);
      if (det < 0) ++neg;
      else if (det > 0) { if (a + c < 0) neg += 2; }
      else { ++zero; if (a + c < 0) ++neg; }
      /* E^-1 = (1/det) [[c, -conj(b)], [-b, a]] ; M22 -= Cb E^-1 Cb^H */
#pragma omp parallel for schedule(static)
      for (int64_t i = k + 2; i < n; ++i) {
        cplx ci0 = M[IDX(i, k, n)], ci1 = M[IDX(i, k + 1, n)];
        cplx g0 = (ci0 * c - ci1 * b) / det;          /* row i of Cb E^-1 */
        cplx g1 = (-ci0 * conj(b) + ci1 * a) / det;
        for (int64_t j = k + 2; j < n; ++j)
          M[IDX(i, j, n)] -= g0 * conj(M[IDX(j, k, n)]) + g1 * conj(M[IDX(j, k + 1, n)]);
      }
      k += 2;
    }
  }
  free(M);
  if (nzero) *nzero = zero;
  return neg;
}

/* ---- Band-energy gradient: GA = gE X X^H, GB = -gE X diag(lam) X^H. ---------------- */
void orc_energy_grad(int64_t n, int64_t nev, const cplx *X, const double *lam, double gE, cplx *GA, cplx *GB) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      cplx sa = 0, sb = 0;
      for (int64_t k = 0; k < nev; ++k) {
        cplx p = X[IDX(i, k, nev)] * conj(X[IDX(j, k, nev)]);
        sa += p;
        sb += lam[k] * p;
      }
      GA[IDX(i, j, n)] = gE * sa;
      GB[IDX(i, j, n)] = -gE * sb;
    }
}

/* Extreme eigenvalues of a Hermitian matrix (for ||A||_2 = max |lambda|), by 3b. */
void orc_eig_extremes(int64_t n, const cplx *M0, double *lmin, double *lmax) {
  cplx *M = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
  memcpy(M, M0, sizeof(cplx) * (size_t)(n * n));
  double *d = (double *)malloc(sizeof(double) * (size_t)n);
  double *e = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n : 1));
  cplx *tau = (cplx *)malloc(sizeof(cplx) * (size_t)(n > 1 ? n : 1));
  if (n > 1) orc_tridiag(n, M, d, e, tau); else d[0] = creal(M[0]);
  double *all = (double *)malloc(sizeof(double) * (size_t)n);
  /* bisection for the first and the last */
  double lam[1];
  tridiag_bisect(n, d, e, 1, lam);
  *lmin = lam[0];
  /* largest: negate T */
  for (int64_t i = 0; i < n; ++i) d[i] = -d[i];
  tridiag_bisect(n, d, e, 1, lam);
  *lmax = -lam[0];
  free(M); free(d); free(e); free(tau); free(all);
}
