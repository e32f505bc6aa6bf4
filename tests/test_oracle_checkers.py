"""Pins of the oracle's checkers against known NONZERO values.

Every parity claim of the GPU tests ("residual <= 1e-10", "eigenvectors within a small
principal angle of the oracle's") rests on three oracle functions: the original-space
residual ``orc_residuals`` (C), ``pieces.residual_norms`` and ``pieces.principal_sines``.
A pin at an exact solution (where the right answer is 0) passes for many wrong versions
of them, so each is pinned here at a value that is not zero and derived by hand or from a
closed form, and each test shows that plausible mistakes (a missing square root, B left
out or used the wrong way, the wrong normalisation, a transposed operand) move the value
far outside the tolerance. The residual is the relative residual of a computed pair of the
paper's A x = lambda B x (the sentence after Eq. 3); the principal angles are the paper's
deviation angle between eigenvectors of consecutive iterations (Sec. "A new computational
philosophy") taken over subspaces in the B inner product.
"""
import math
import os

import numpy as np
import pytest

from tests.conftest import crandn, rand_hpd

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_residual_fixture():
    rows = {"A": [], "B": [], "X": []}
    scal = {}
    for line in open(os.path.join(GOLDEN, "residual_2x2.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, *vals = line.split()
        if tag in rows:
            v = [float(x) for x in vals]
            rows[tag].append([complex(v[2 * j], v[2 * j + 1]) for j in range(len(v) // 2)])
        else:
            scal[tag] = np.array([float(x) for x in vals])
    return (np.array(rows["A"]), np.array(rows["B"]), np.array(rows["X"]), scal["lambda"],
            float(scal["normA"][0]), scal["resid"])


def test_residuals_golden_nonzero(orc):
    A, B, X, lam, normA, want = _read_residual_fixture()
    got = orc.residuals(A, B, lam, X, normA)
    assert np.abs(got - want).max() <= 4e-16 * want.max()


def test_residuals_planted_mistakes_fail(orc):
    """Each plausible mistake in the residual gives a value the golden pin rejects.
    Mutations that are input-level are made by calling the oracle on the mutated inputs;
    the output-level ones (a missing square root, normA squared) are the oracle's output
    transformed exactly as the mistake would transform it."""
    A, B, X, lam, normA, want = _read_residual_fixture()
    good = orc.residuals(A, B, lam, X, normA)
    xn = np.linalg.norm(X, axis=0)
    mutants = {
        "A transposed (its conjugate)": orc.residuals(A.T.copy(), B, lam, X, normA),
        "B left out": orc.residuals(A, np.eye(2, dtype=complex), lam, X, normA),
        "missing sqrt on the residual": (good * normA * xn) ** 2 / (normA * xn),
        "normA squared": good / normA,
        "divided by ||x||^2": good / xn,
    }
    # (B = diag(2, 1) is real, so B transposed cannot be seen here; the n = 40 pencil below
    # makes it visible)
    for name, bad in mutants.items():
        assert np.abs(bad - want).max() > 1e-3 * want.max(), name


def test_residuals_closed_form_perturbed_eigenvector(orc):
    """n = 40 pencil with a known spectrum, B = L L^H, A = L Q diag(lam) Q^H L^H (the
    closed-form construction of the survey's pins). For x = L^-H Q (e_i + t e_j) and the
    value lam_i: A x - lam_i B x = t (lam_j - lam_i) L Q e_j exactly, so
    r = |t| |lam_j - lam_i| ||L Q e_j|| / (normA ||x||). A complex t and a B far from the
    identity make a transposed or conjugated operand, or B left out, visible."""
    rng = np.random.default_rng(41)
    n = 40
    lam = np.sort(rng.uniform(-2, 50, n))
    G = crandn(rng, n, n)
    Q, R = np.linalg.qr(G)
    Q = Q * (np.diag(R) / np.abs(np.diag(R)))
    L = np.tril(crandn(rng, n, n) * (0.3 / math.sqrt(n)), -1) + np.diag(rng.uniform(0.5, 2.0, n))
    B = L @ L.conj().T
    A = L @ (Q * lam) @ Q.conj().T @ L.conj().T
    A = 0.5 * (A + A.conj().T)
    B = 0.5 * (B + B.conj().T)
    Linv_h = np.linalg.inv(L).conj().T
    pairs = [(0, 5, 0.3 - 0.2j), (3, 1, 1e-3j), (10, 39, -2.0), (7, 8, 0.5 + 0.5j)]
    X = np.zeros((n, len(pairs)), dtype=complex)
    lam_x = np.zeros(len(pairs))
    want = np.zeros(len(pairs))
    normA = 60.0
    for k, (i, j, t) in enumerate(pairs):
        X[:, k] = Linv_h @ (Q[:, i] + t * Q[:, j])
        lam_x[k] = lam[i]
        want[k] = abs(t) * abs(lam[j] - lam[i]) * np.linalg.norm(L @ Q[:, j]) / (normA * np.linalg.norm(X[:, k]))
    got = orc.residuals(A, B, lam_x, X, normA)
    # the closed form holds up to the rounding of forming A and B (n u ||A|| scale)
    assert np.abs(got - want).max() <= 1e-12 * want.max()
    assert want.min() > 1e-6
    # B used the wrong way: transposed (= conjugated, B Hermitian) or left out
    for bad_B in (B.T.copy(), np.eye(n, dtype=complex)):
        bad = orc.residuals(A, bad_B, lam_x, X, normA)
        assert np.abs(bad - want).max() > 1e-3 * want.max()
    bad = orc.residuals(A.T.copy(), B, lam_x, X, normA)
    assert np.abs(bad - want).max() > 1e-3 * want.max()


def _ritz_case():
    """C Hermitian 3 x 3 with span(e1, e2) not invariant:
         C = [[1, 1/2, 0], [1/2, 2, i/4], [0, -i/4, 3]],  Q = [e1, e2].
    G = Q^H C Q = [[1, 1/2], [1/2, 2]] has the Ritz values (3 -+ sqrt 2)/2 and unit Ritz
    vectors z with |z_2| = sin(pi/8) (lower value) and cos(pi/8) (upper): the lower one
    solves (1 - theta) z_1 + z_2 / 2 = 0, so z_2 / z_1 = -(sqrt 2 - 1) = -tan(pi/8). The
    part of C Q z outside span(Q) is row 3 of C times z, (0, -i/4) . z, so the residual
    ||C Q z - theta Q z|| is |z_2| / 4."""
    Cm = np.array([[1, 0.5, 0], [0.5, 2, 0.25j], [0, -0.25j, 3]], dtype=np.complex128)
    Q = np.eye(3, dtype=np.complex128)[:, :2]
    theta = np.array([(3 - math.sqrt(2)) / 2, (3 + math.sqrt(2)) / 2])
    res = np.array([math.sin(math.pi / 8), math.cos(math.pi / 8)]) / 4
    return Cm, Q, theta, res


def test_rayleigh_ritz_residual_norms_closed_form(orc):
    from oracle import pieces
    Cm, Q, theta_w, res_w = _ritz_case()
    th, Qn, W = pieces.rayleigh_ritz(Cm, Q)
    assert np.abs(th - theta_w).max() <= 1e-15 * 3
    r = pieces.residual_norms(W, Qn, th)
    assert np.abs(r - res_w).max() <= 1e-15
    # planted mistakes: the residual of the unrotated basis, theta applied by rows, the
    # squared norm, the Ritz values left out
    assert np.abs(pieces.residual_norms(Cm @ Q, Q, th) - res_w).max() > 1e-3
    bad_rows = np.linalg.norm(W - (Qn.T * th[:, None]).T[::-1], axis=0)
    assert np.abs(bad_rows - res_w).max() > 1e-3
    assert np.abs(r ** 2 - res_w).max() > 1e-3
    assert np.abs(pieces.residual_norms(W, Qn, 0 * th) - res_w).max() > 1e-3


def test_residual_norms_known_columns():
    """W - Q diag(theta) with known columns: Q = [e1, e2] in C^3, theta = (2, 5),
    W = [[2, 0], [0, 5], [3i, 4]]: the residual columns are (0, 0, 3i) and (0, 0, 4), norms
    3 and 4. theta applied to the rows of Q instead of its columns (a broadcasting mistake)
    gives other norms."""
    from oracle import pieces
    Q = np.eye(3, dtype=np.complex128)[:, :2]
    W = np.array([[2, 0], [0, 5], [3j, 4]], dtype=np.complex128)
    theta = np.array([2.0, 5.0])
    assert np.array_equal(pieces.residual_norms(W, Q, theta), np.array([3.0, 4.0]))
    W2 = W.copy()
    W2[0, 1] = 1.0   # residual column (1, 0, 4): sqrt(17)
    assert pieces.residual_norms(W2, Q, theta)[1] == pytest.approx(math.sqrt(17.0), rel=1e-15)


def test_principal_sines_planted_angles_B_inner_product(orc):
    """Two 3-dimensional subspaces at planted principal angles in the B inner product:
    with B = L L^H, X1 = L^-H [e1, e2, e3] M1 and X2 = L^-H F M2, where the columns of F are
    cos(phi_k) e_k + sin(phi_k) e_{k+3} (k = 1..3) and M1, M2 are arbitrary invertible
    mixings. L^H maps the B inner product to the Euclidean one, so the principal angles are
    exactly phi_k and the sines sin(phi_k) (descending). B left out, or B^-1 in its place,
    gives other values; so does a version that ignores the mixing (no QR of the bases)."""
    from oracle import pieces
    rng = np.random.default_rng(17)
    n = 24
    B = rand_hpd(rng, n, cond=200.0)
    L = np.linalg.cholesky(B)
    Linv_h = np.linalg.inv(L).conj().T
    phis = np.array([1.2, 0.45, 0.01])
    E = np.eye(n, dtype=np.complex128)
    F = np.zeros((n, 3), dtype=np.complex128)
    for k, ph in enumerate(phis):
        F[:, k] = math.cos(ph) * E[:, k] + math.sin(ph) * np.exp(0.3j * (k + 1)) * E[:, k + 3]
    M1 = crandn(rng, 3, 3) + 2 * np.eye(3)
    M2 = crandn(rng, 3, 3) + 2 * np.eye(3)
    X1 = Linv_h @ E[:, :3] @ M1
    X2 = Linv_h @ F @ M2
    want = np.sort(np.sin(phis))[::-1]
    s = np.sort(pieces.principal_sines(X1, X2, B))[::-1]
    assert np.abs(s - want).max() <= 1e-12
    # symmetric in its arguments
    s21 = np.sort(pieces.principal_sines(X2, X1, B))[::-1]
    assert np.abs(s21 - want).max() <= 1e-12
    # B used wrongly
    for bad in (pieces.principal_sines(X1, X2, None), pieces.principal_sines(X1, X2, np.linalg.inv(B))):
        assert np.abs(np.sort(bad)[::-1] - want).max() > 1e-3
    # a version without orthonormal bases (the raw projection of the mixed columns)
    P = L.conj().T @ X2
    raw = np.linalg.svd((L.conj().T @ X1) - P @ np.linalg.lstsq(P, L.conj().T @ X1, rcond=None)[0],
                        compute_uv=False)
    assert np.abs(np.sort(raw)[::-1] - want).max() > 1e-3
