"""Pins of the oracle's step definitions (filter, CholQR2, Rayleigh-Ritz, angles)."""
import math

import numpy as np
import pytest

from tests.conftest import crandn, rand_herm, rand_hpd


def test_filter_closed_form_on_diagonal(orc):
    # for diagonal C the filter is the scalar polynomial p(lambda_j) on each row
    from oracle import pieces
    lam = np.linspace(-2, 50, 30)
    Cm = np.diag(lam).astype(np.complex128)
    rng = np.random.default_rng(11)
    Y0 = crandn(rng, 30, 5)
    lo, hi, s = 3.0, 50.0, -2.0
    for d in (1, 2, 7, 16):
        Y = pieces.chebyshev_filter(Cm, Y0, d, lo, hi, s)
        p = pieces.cheb_scalar(d, lam, lo, hi, s)
        assert np.allclose(Y, p[:, None] * Y0, rtol=1e-12, atol=1e-12)
    # p(s) = 1 by construction and |p| <= 1/|T_d((s-c)/e)| on [lo, hi]
    assert pieces.cheb_scalar(9, np.array([s]), lo, hi, s)[0] == pytest.approx(1.0)
    inside = np.linspace(lo, hi, 101)
    c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
    bound = 1.0 / abs(pieces.cheb_T(9, np.array([(s - c) / e]))[0])
    assert np.abs(pieces.cheb_scalar(9, inside, lo, hi, s)).max() <= bound * (1 + 1e-12)


def test_cheb_T_closed_form():
    from oracle import pieces
    x = np.array([-1.7, -1.0, -0.3, 0.0, 0.6, 1.0, 2.5])
    # T_3(x) = 4x^3 - 3x, T_4(x) = 8x^4 - 8x^2 + 1
    assert np.allclose(pieces.cheb_T(3, x), 4 * x**3 - 3 * x, rtol=1e-13, atol=1e-13)
    assert np.allclose(pieces.cheb_T(4, x), 8 * x**4 - 8 * x**2 + 1, rtol=1e-13, atol=1e-13)


def test_cholqr2_is_the_unique_qr(orc):
    from oracle import pieces
    rng = np.random.default_rng(12)
    Y = crandn(rng, 200, 17) @ np.diag(np.logspace(0, 4, 17))
    Q, R = pieces.cholqr2(Y)
    assert np.abs(Q.conj().T @ Q - np.eye(17)).max() < 1e-13
    assert np.abs(Q @ R - Y).max() < 1e-12 * np.abs(Y).max()
    Qn, Rn = np.linalg.qr(Y)
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    Qn, Rn = Qn * ph, (Rn.T * ph.conj()).T
    assert np.abs(Q - Qn).max() < 1e-10
    assert np.allclose(np.triu(R), R)


def test_rayleigh_ritz_exact_subspace(orc):
    from oracle import pieces
    rng = np.random.default_rng(13)
    n, k = 60, 6
    lam = np.sort(rng.uniform(-1, 10, n))
    Qf, _ = np.linalg.qr(crandn(rng, n, n))
    Cm = (Qf * lam) @ Qf.conj().T
    Cm = 0.5 * (Cm + Cm.conj().T)
    # a rotated basis of the invariant subspace of eigenvalues 2..7
    Z, _ = np.linalg.qr(crandn(rng, k, k))
    Q = Qf[:, 2:2 + k] @ Z
    th, Qn, W = pieces.rayleigh_ritz(Cm, Q)
    assert np.abs(th - lam[2:2 + k]).max() < 1e-12
    assert pieces.residual_norms(W, Qn, th).max() < 1e-12


def test_deviation_angles_known_rotation():
    from oracle import pieces
    n = 10
    B = np.eye(n, dtype=np.complex128)
    X0 = np.eye(n, dtype=np.complex128)[:, :2]
    t = 0.3
    X1 = X0.copy()
    X1[:, 0] = math.cos(t) * X0[:, 0] + math.sin(t) * np.eye(n)[:, 5]
    ang = pieces.deviation_angles(X0, X1, B)
    assert ang[0] == pytest.approx(t / (math.pi / 2), rel=1e-12)
    assert ang[1] == pytest.approx(0.0, abs=1e-7)


def test_principal_sines_B_inner_product(orc):
    from oracle import pieces
    rng = np.random.default_rng(14)
    n = 30
    from tests.conftest import rand_hpd
    B = rand_hpd(rng, n, 50)
    X = crandn(rng, n, 3)
    s = pieces.principal_sines(X, X @ crandn(rng, 3, 3), B)
    assert s.max() < 1e-7


def test_matrix_variation_hand_case():
    """delta and the counts on a difference whose entries are known exactly: moduli
    5 (3+4i), 1 (exactly at p = 0.2 of delta), 0.5 (exactly at p = 0.1), 0.25 (at p = 0.05):
    entries exactly at a threshold are not above it (the comparison is strict);
    0.25j, 0 elsewhere."""
    from oracle import pieces
    A_old = np.zeros((4, 4), dtype=np.complex128)
    A_new = A_old.copy()
    A_new[0, 1], A_new[1, 0] = 3 + 4j, 3 - 4j
    A_new[2, 2] = 1.0
    A_new[3, 0], A_new[0, 3] = 0.5, 0.5
    A_new[1, 3], A_new[3, 1] = 0.25j, -0.25j
    A_old[2, 3] = A_new[2, 3] = 7.0 - 2.0j          # unchanged entry, nonzero
    delta, counts, mask = pieces.matrix_variation(A_new, A_old, [0.1, 0.0, 0.05, 0.2, 1.0])
    assert delta == 5.0
    assert counts == [3, 7, 5, 2, 0]   # p = 0.2: threshold 1.0, the diagonal 1 is not above it
    assert mask.sum() == 3 and mask[0, 1] and mask[1, 0] and mask[2, 2]


def test_matrix_variation_invariants():
    """Counts fall as the threshold rises, count(0) is the number of changed entries, the
    largest entry defines delta (count at p = 1 is zero), and a Hermitian difference gives
    counts of the same parity as its changed diagonal entries."""
    from oracle import pieces
    rng = np.random.default_rng(5)
    n = 37
    A = crandn(rng, n, n)
    A = A + A.conj().T
    P = crandn(rng, n, n) * (rng.random((n, n)) < 0.2)
    P = P + P.conj().T
    ps = [0.0, 0.01, 0.1, 0.3, 0.7, 1.0]
    delta, counts, _ = pieces.matrix_variation(A + 1e-3 * P, A, ps)
    assert all(a >= b for a, b in zip(counts, counts[1:]))
    changed = np.count_nonzero((A + 1e-3 * P) != A)
    assert counts[0] == changed and counts[-1] == 0
    diag_changed = np.count_nonzero(np.diag(A + 1e-3 * P) != np.diag(A))
    assert (counts[0] - diag_changed) % 2 == 0
    assert abs(delta - np.abs((A + 1e-3 * P) - A).max()) <= 1e-15 * delta


def test_reindex_recovers_a_permutation():
    """New eigenvectors that are a permuted, re-phased copy of the old: the assignment
    returns the permutation and every matched angle is zero."""
    from oracle import pieces
    rng = np.random.default_rng(3)
    n, k = 40, 9
    B = rand_hpd(rng, n, cond=30.0)
    X, _ = np.linalg.qr(crandn(rng, n, k))
    perm = rng.permutation(k)
    ph = np.exp(1j * rng.uniform(0, 2 * np.pi, k))
    Xn = X[:, perm] * ph
    inv = np.argsort(perm)
    got, cost, nout = pieces.reindex(X, Xn, B, np.arange(k), np.arange(k)[perm])
    assert np.array_equal(got, inv)
    assert abs(cost) < 1e-12 and nout == 0
    c = pieces.overlap_cosines(X, Xn, B)
    assert np.allclose(c[np.arange(k), got], 1.0, atol=1e-12)


def test_reindex_optimal_against_brute_force():
    """The assignment equals the optimum over all permutations (tiny k), with no window and
    with an energy window that forbids the unrestricted optimum: the new vectors are a
    shuffled, perturbed copy of the old, while the new eigenvalues stay in place, so the
    window admits only the pairs i -> i."""
    import itertools
    from oracle import pieces
    rng = np.random.default_rng(4)
    n, k = 30, 5
    B = rand_hpd(rng, n, cond=10.0)
    Xo = crandn(rng, n, k)
    sh = np.array([1, 2, 3, 4, 0])
    Xn = Xo[:, sh] + 0.6 * crandn(rng, n, k)
    lo = np.array([0.0, 0.2, 0.4, 0.6, 0.8])
    ln = lo + 0.01
    c = pieces.overlap_cosines(Xo, Xn, B)
    perms = {}
    for window in (np.inf, 0.05):
        far = np.abs(lo[:, None] - ln[None, :]) > window
        # lexicographic: fewest pairs outside the window, then the least cost inside it
        best = min((sum(far[i, p[i]] for i in range(k)),
                    sum(0.0 if far[i, p[i]] else 1 - c[i, p[i]] for i in range(k)))
                   for p in itertools.permutations(range(k)))
        perm, cost, nout = pieces.reindex(Xo, Xn, B, lo, ln, window)
        assert nout == best[0] == 0
        assert abs(cost - best[1]) <= 1e-12 * max(1.0, best[1])
        assert sorted(perm) == list(range(k))
        perms[window] = perm
    assert np.array_equal(perms[np.inf], np.argsort(sh))
    assert np.array_equal(perms[0.05], np.arange(k))


def test_overlap_cosines_known_angles():
    """Vectors at known angles in the B inner product: with B = L L^H, y = L^-H e, the
    cosine of y_old = L^-H e_1 and y_new = L^-H (cos phi e_1 + sin phi e_2) is cos phi
    whatever the scaling of either vector; using B the wrong way (B^-1, B^T on complex data,
    or no B) gives another value."""
    from oracle import pieces
    rng = np.random.default_rng(5)
    n = 12
    B = rand_hpd(rng, n, cond=50.0)
    L = np.linalg.cholesky(B)
    Linv_h = np.linalg.inv(L).conj().T
    phis = np.array([0.0, 0.3, 1.1, np.pi / 2])
    E = np.zeros((n, 4), dtype=complex)
    E[0] = 1.0
    Xo = Linv_h @ E * 2.5
    F = np.zeros((n, 4), dtype=complex)
    F[0] = np.cos(phis)
    F[1] = np.sin(phis) * np.exp(0.7j)
    Xn = Linv_h @ F * 0.3j
    c = pieces.overlap_cosines(Xo, Xn, B)
    assert np.allclose(np.diag(c), np.abs(np.cos(phis)), atol=1e-12)
    th = pieces.deviation_angles(Xo, Xn, B)
    assert np.allclose(th[:3], phis[:3] / (np.pi / 2), atol=1e-7)
    assert not np.allclose(np.diag(pieces.overlap_cosines(Xo, Xn, np.eye(n))), np.abs(np.cos(phis)), atol=1e-3)
