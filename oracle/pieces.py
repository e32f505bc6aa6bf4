"""Plain numpy definitions of the individual steps of the block subspace solver.

TEST INFRASTRUCTURE ONLY. Each function is the textbook definition of one step that the
CUDA path implements (in FP64 unless stated), written without blocking, fusion or
reordering, so that a per-kernel parity test can compare element by element:

* ``chebyshev_filter`` -- the scaled three-term Chebyshev recurrence of Zhou, Saad, Tiago
  & Chelikowsky (J. Comput. Phys. 219, 2006): Y = p(C) Y0 with
  p(t) = T_d((t - c)/e) / T_d((s - c)/e), c = (lo + hi)/2, e = (hi - lo)/2, s the
  scaling point below the damped interval [lo, hi].
* ``cholqr2`` -- CholQR applied twice (Fukaya, Nakatsukasa, Yanagisawa & Yamamoto 2014).
* ``rayleigh_ritz`` -- G = Q^H C Q, G = Z diag(theta) Z^H, Q <- Q Z, W = C Q.
* ``residual_norms`` -- ||W_i - theta_i Q_i||_2.

The paper names "an improved version of the subspace iteration method" as the solver to
build for the fast iterations seeded by the previous problem's eigenvectors (Sec.
"Summary and conclusions"); these are its steps. Matrix products use numpy (a library
primitive); the small Hermitian eigensolve and the Cholesky use the C oracle.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as _o


def cheb_T(d: int, x):
    """Chebyshev polynomial T_d(x) by its closed form (cos/cosh), for pins."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(d * np.arccos(x[inside]))
    xo = x[~inside]
    sgn = np.where(xo < 0, (-1.0) ** d, 1.0)
    out[~inside] = sgn * np.cosh(d * np.arccosh(np.abs(xo)))
    return out


def cheb_scalar(d: int, t, lo: float, hi: float, s: float):
    """p(t) = T_d((t-c)/e) / T_d((s-c)/e): the filter polynomial at scalar points."""
    c, e = 0.5 * (hi + lo), 0.5 * (hi - lo)
    return cheb_T(d, (np.asarray(t) - c) / e) / cheb_T(d, np.array([(s - c) / e]))[0]


def chebyshev_filter(Cm, Y0, deg: int, lo: float, hi: float, s: float):
    """Scaled Chebyshev recurrence (degree ``deg`` >= 1) applied to the block Y0."""
    Cm = np.asarray(Cm, dtype=np.complex128)
    X = np.array(Y0, dtype=np.complex128)
    e = 0.5 * (hi - lo)
    c = 0.5 * (hi + lo)
    sigma = e / (s - c)
    sigma1 = sigma
    Y = (Cm @ X - c * X) * (sigma1 / e)
    for _ in range(2, deg + 1):
        sigma_new = 1.0 / (2.0 / sigma1 - sigma)
        Yt = (Cm @ Y - c * Y) * (2.0 * sigma_new / e) - (sigma * sigma_new) * X
        X, Y, sigma = Y, Yt, sigma_new
    return Y


def gram(Y):
    Y = np.asarray(Y, dtype=np.complex128)
    return Y.conj().T @ Y


def cholqr(Y):
    """One CholQR pass: W = Y^H Y = R^H R (R upper, positive diagonal), Q = Y R^-1."""
    W = gram(Y)
    Lw, info = _o.potrf(W)
    if info:
        raise np.linalg.LinAlgError(f"Gram matrix not positive definite (pivot {info})")
    R = Lw.conj().T
    # Q = Y R^-1  <=>  R^H Q^H = Y^H  (forward substitution with the lower factor Lw)
    Qh = np.linalg.solve(Lw, Y.conj().T)
    return Qh.conj().T, R


def cholqr2(Y):
    Q1, R1 = cholqr(Y)
    Q, R2 = cholqr(Q1)
    return Q, R2 @ R1


def rayleigh_ritz(Cm, Q):
    """Ritz values (ascending) and vectors of C on span(Q) (Q orthonormal)."""
    Cm = np.asarray(Cm, dtype=np.complex128)
    Q = np.asarray(Q, dtype=np.complex128)
    W = Cm @ Q
    G = Q.conj().T @ W
    G = 0.5 * (G + G.conj().T)
    theta, Z = _o.heev(G, method="jacobi")
    Qn = Q @ Z
    return theta, Qn, Cm @ Qn


def residual_norms(W, Q, theta):
    W = np.asarray(W)
    Q = np.asarray(Q)
    return np.linalg.norm(W - Q * np.asarray(theta)[None, :], axis=0)


def lanczos_upper_bound_ok(Cm, b: float) -> bool:
    """True if b bounds the spectrum of C from above (checked with the oracle)."""
    lo, hi = _o.eig_extremes(Cm)
    return b >= hi - 1e-12 * max(abs(lo), abs(hi))


def principal_sines(X1, X2, B=None):
    """Sines of the principal angles between span(X1) and span(X2) in the B inner
    product (B = I if None): the paper's subspace deviation angle applied to clusters.
    Computed as the singular values of (I - Q2 Q2^H) Q1, which stays accurate for small
    angles (unlike sqrt(1 - cos^2))."""
    X1 = np.asarray(X1, dtype=np.complex128)
    X2 = np.asarray(X2, dtype=np.complex128)
    if B is not None:
        Lb, info = _o.potrf(B)
        if info:
            raise np.linalg.LinAlgError("B not HPD")
        X1 = Lb.conj().T @ X1
        X2 = Lb.conj().T @ X2
    q1, _ = np.linalg.qr(X1)
    q2, _ = np.linalg.qr(X2)
    D = q1 - q2 @ (q2.conj().T @ q1)
    s = np.linalg.svd(D, compute_uv=False)
    return np.clip(s, 0.0, 1.0)


def deviation_angles(X_old, X_new, B):
    """Normalised deviation angle (1.00 = pi/2) between matched columns in the B inner
    product: theta_i = acos(|x_old_i^H B x_new_i| / (||x_old_i||_B ||x_new_i||_B)) / (pi/2)."""
    BXn = np.asarray(B) @ np.asarray(X_new)
    BXo = np.asarray(B) @ np.asarray(X_old)
    num = np.abs(np.sum(np.conj(X_old) * BXn, axis=0))
    no = np.sqrt(np.abs(np.sum(np.conj(X_old) * BXo, axis=0)))
    nn = np.sqrt(np.abs(np.sum(np.conj(X_new) * BXn, axis=0)))
    c = np.clip(num / (no * nn), 0.0, 1.0)
    return np.arccos(c) / (math.pi / 2)


def matrix_variation(A_new, A_old, thresholds):
    """The paper's entry-variation statistics between consecutive Hamiltonians (Sec.
    "Matrix generation"): delta = the largest entry variation max_ij |A_new - A_old|_ij,
    and for each threshold fraction p the number of entries whose variation exceeds
    p * delta. Compared as squares in FP64 with the operations in this order and no fused
    multiply-add: d2 = dr*dr + di*di, delta2 = max d2, an entry counts for p when
    d2 > (p*p) * delta2. Returns (delta, counts, mask for thresholds[0])."""
    D = np.asarray(A_new, dtype=np.complex128) - np.asarray(A_old, dtype=np.complex128)
    dr, di = D.real, D.imag
    d2 = dr * dr + di * di
    delta2 = float(d2.max()) if d2.size else 0.0
    counts = []
    for p in thresholds:
        thr2 = (float(p) * float(p)) * delta2
        counts.append(int(np.count_nonzero(d2 > thr2)))
    mask = (d2 > (float(thresholds[0]) * float(thresholds[0])) * delta2) if len(thresholds) else None
    return math.sqrt(delta2), counts, mask


def overlap_cosines(X_old, X_new, B):
    """c_ij = |x_old_i^H B x_new_j| / (||x_old_i||_B ||x_new_j||_B): the cosines of the
    angles between every old and every new eigenvector in the B inner product."""
    B = np.asarray(B)
    X_old = np.asarray(X_old)
    X_new = np.asarray(X_new)
    O = X_old.conj().T @ (B @ X_new)
    no = np.sqrt(np.abs(np.sum(np.conj(X_old) * (B @ X_old), axis=0)))
    nn = np.sqrt(np.abs(np.sum(np.conj(X_new) * (B @ X_new), axis=0)))
    return np.clip(np.abs(O) / np.outer(no, nn), 0.0, 1.0)


def reindex(X_old, X_new, B, lam_old, lam_new, window=np.inf):
    """Re-indexing of the new eigenvectors against the old (Sec. "A new computational
    philosophy", paragraph "Eigenvectors evolution": each eigenvector is compared with the
    one at the next iteration that it deviates least from; the paper names the criterion,
    angle minimisation, but gives no algorithm). Reading: the assignment perm of every old
    vector to a distinct new one minimising sum_i (1 - c_{i, perm[i]}), where a pair whose
    eigenvalues differ by more than `window` costs k_old + 1, more than any assignment of
    pairs inside the window. Solved with scipy's linear_sum_assignment (a library
    primitive). Returns (perm, cost of the pairs inside the window, pairs outside it)."""
    from scipy.optimize import linear_sum_assignment
    c = overlap_cosines(X_old, X_new, B)
    ko = c.shape[0]
    far = np.abs(np.asarray(lam_old)[:, None] - np.asarray(lam_new)[None, :]) > window
    cost = np.where(far, ko + 1.0, 1.0 - c)
    r, col = linear_sum_assignment(cost)
    perm = np.empty(len(r), dtype=np.int64)
    perm[r] = col
    out = far[np.arange(ko), perm]
    inside = float((1.0 - c[np.arange(ko), perm])[~out].sum())
    return perm, inside, int(out.sum())
