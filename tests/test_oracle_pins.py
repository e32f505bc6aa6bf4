"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself:
closed forms, invariants, textbook special cases, brute force on tiny inputs and
finite differences. The problem is the paper's A x = lambda B x with A Hermitian and B
Hermitian positive definite (the sentence after Eq. 3)."""
import math

import numpy as np
import pytest

from tests.conftest import crandn, rand_herm, rand_hpd


def test_potrf_reconstructs(orc):
    rng = np.random.default_rng(1)
    B = rand_hpd(rng, 37, cond=1e3)
    L, info = orc.potrf(B)
    assert info == 0
    assert np.allclose(np.triu(L, 1), 0)
    d = np.diag(L)
    assert np.all(d.real > 0) and np.allclose(d.imag, 0)
    assert np.abs(L @ L.conj().T - B).max() <= 1e-13 * np.abs(B).max()


@pytest.mark.parametrize("diag,expect", [([1.0, 2.0, -1.0, 3.0], 3), ([0.0, 1.0], 1), ([2.0, 3.0], 0)])
def test_potrf_info_convention(orc, diag, expect):
    # LAPACK potrf: info = 1-based index of the first non-positive leading minor's pivot
    B = np.diag(np.array(diag, dtype=np.complex128))
    _, info = orc.potrf(B)
    assert info == expect


def test_reduce_congruence(orc):
    rng = np.random.default_rng(2)
    n = 29
    A, B = rand_herm(rng, n), rand_hpd(rng, n, 1e2)
    L, _ = orc.potrf(B)
    Cm = orc.reduce(A, L)
    assert np.abs(Cm - Cm.conj().T).max() == 0.0
    assert np.abs(L @ Cm @ L.conj().T - A).max() <= 1e-12 * np.abs(A).max()


def _known(rng, n, lam):
    Q, R = np.linalg.qr(crandn(rng, n, n))
    Q = Q * (np.diag(R) / np.abs(np.diag(R)))
    Cm = (Q * lam) @ Q.conj().T
    return 0.5 * (Cm + Cm.conj().T), Q


@pytest.mark.parametrize("method", ["jacobi", "tridiag"])
def test_heev_closed_form(orc, method):
    rng = np.random.default_rng(3)
    n = 40
    lam = np.sort(rng.uniform(-2, 50, n))
    Cm, Q = _known(rng, n, lam)
    w, V = orc.heev(Cm, n if method == "jacobi" else 12, method=method)
    k = len(w)
    assert np.abs(w - lam[:k]).max() <= 1e-13 * 50
    # eigenvector residuals and orthonormality
    assert np.abs(Cm @ V - V * w).max() <= 1e-12 * 50
    assert np.abs(V.conj().T @ V - np.eye(k)).max() <= 1e-12
    # matches the generating vectors up to a phase (eigenvalues are simple)
    ov = np.abs(np.sum(np.conj(Q[:, :k]) * V, axis=0))
    assert np.all(ov > 1 - 1e-10)


def test_heev_degenerate_subspace(orc):
    # an exactly degenerate eigenvalue: only the eigenspace is unique (paper, Fig. 1 caption)
    rng = np.random.default_rng(4)
    n = 20
    lam = np.array([-1.0, 0.5, 0.5, 0.5] + list(np.linspace(1, 9, n - 4)))
    Cm, Q = _known(rng, n, lam)
    for method in ("jacobi", "tridiag"):
        w, V = orc.heev(Cm, 4, method=method)
        assert np.abs(w - lam[:4]).max() < 1e-13 * 9
        P1 = Q[:, 1:4] @ Q[:, 1:4].conj().T
        P2 = V[:, 1:4] @ V[:, 1:4].conj().T
        assert np.abs(P1 - P2).max() < 1e-10


def test_tridiag_matches_jacobi(orc):
    rng = np.random.default_rng(5)
    Cm = rand_herm(rng, 64)
    w1, V1 = orc.heev(Cm, 10, method="jacobi")
    w2, V2 = orc.heev(Cm, 10, method="tridiag")
    assert np.abs(w1 - w2).max() < 1e-13 * np.abs(w1).max()
    assert np.all(np.abs(np.sum(np.conj(V1) * V2, axis=0)) > 1 - 1e-10)


def test_solve_known_spectrum_pencil(orc):
    from paper_1007_4400_gb300 import synth
    s = synth.make_sequence(0, 96, 1, 10, 4)
    A, B = s.A[0].numpy(), s.B.numpy()
    for method in ("jacobi", "tridiag"):
        lam, X = orc.solve(A, B, 10, method=method)
        # Weyl bound on the rounding of forming A: generous multiple of n u ||A|| ||L^-1||^2
        assert np.abs(lam - s.lam0[:10]).max() <= 1e-12 * np.abs(s.lam0).max()
        assert np.abs(X.conj().T @ B @ X - np.eye(10)).max() < 1e-12
        nA = orc.norm2_hermitian(A)
        assert orc.residuals(A, B, lam, X, nA).max() < 1e-13
        for i in range(10):
            xt = s.x0_true(i).numpy()[:, 0]
            c = abs(np.vdot(xt, B @ X[:, i]))
            assert c > 1 - 1e-9


def test_n1_is_ratio(orc):
    lam, X = orc.solve(np.array([[3.0 + 0j]]), np.array([[4.0 + 0j]]), 1)
    assert lam[0] == pytest.approx(0.75, abs=1e-15)
    assert abs(abs(X[0, 0]) ** 2 * 4.0 - 1) < 1e-15


def test_n2_quadratic(orc):
    # det(A - lam B) = 0 written out for 2x2 Hermitian A, B
    A = np.array([[2.0, 1 - 2j], [1 + 2j, -3.0]])
    B = np.array([[3.0, 0.5 + 0.25j], [0.5 - 0.25j, 2.0]])
    a2 = (B[0, 0] * B[1, 1] - abs(B[0, 1]) ** 2).real
    a1 = -(A[0, 0] * B[1, 1] + A[1, 1] * B[0, 0] - 2 * (A[0, 1] * np.conj(B[0, 1])).real).real
    a0 = (A[0, 0] * A[1, 1] - abs(A[0, 1]) ** 2).real
    disc = math.sqrt(a1 * a1 - 4 * a2 * a0)
    roots = sorted([(-a1 - disc) / (2 * a2), (-a1 + disc) / (2 * a2)])
    lam, _ = orc.solve(A, B, 2)
    assert np.allclose(lam, roots, atol=1e-14, rtol=1e-14)


def test_diagonal_identity(orc):
    d = np.array([3.0, -1.0, 7.0, 0.5, -4.0])
    lam, X = orc.solve(np.diag(d).astype(np.complex128), np.eye(5, dtype=np.complex128), 5)
    assert np.array_equal(lam, np.sort(d))
    assert np.allclose(np.abs(X), np.eye(5)[:, np.argsort(d)])


@pytest.mark.parametrize("n", [3, 5, 6])
def test_tiny_brute_force_determinant(orc, n):
    # every computed lambda is a root of det(A - lambda B); the count is n
    rng = np.random.default_rng(10 + n)
    A, B = rand_herm(rng, n), rand_hpd(rng, n, 5.0)
    lam, _ = orc.solve(A, B, n)
    for l in lam:
        M = A - l * B
        d = abs(np.linalg.det(M))
        scale = np.prod(np.linalg.svd(M, compute_uv=False)[:-1]) * np.linalg.norm(A, 2)
        assert d <= 1e-12 * scale
    # roots of the characteristic polynomial of B^-1 A (numpy's poly/roots as comparator)
    ref = np.sort(np.roots(np.poly(np.linalg.solve(B, A))).real)
    assert np.allclose(lam, ref, atol=1e-9 * np.abs(ref).max())


def test_inertia_counts_closed_form(orc):
    from paper_1007_4400_gb300 import synth
    s = synth.make_sequence(0, 80, 1, 8, 4)
    A, B = s.A[0].numpy(), s.B.numpy()
    lam = s.lam0
    for k in (0, 1, 7, 8, 40, 79):
        sig = 0.5 * (lam[k] + lam[k + 1]) if k + 1 < len(lam) else lam[-1] + 1
        neg, zero = orc.inertia(A, B, sig)
        assert zero == 0
        assert neg == k + 1


def test_inertia_forces_2x2_pivots(orc):
    # zero diagonal: Bunch-Kaufman must take 2x2 pivots; eigenvalues of [[0,1],[1,0]] are +-1
    A = np.kron(np.eye(3), np.array([[0.0, 1.0], [1.0, 0.0]])).astype(np.complex128)
    B = np.eye(6, dtype=np.complex128)
    assert orc.inertia(A, B, 0.0) == (3, 0)
    assert orc.inertia(A, B, -2.0) == (0, 0)
    assert orc.inertia(A, B, 2.0) == (6, 0)


def test_norm2(orc):
    rng = np.random.default_rng(6)
    A = rand_herm(rng, 50)
    assert orc.norm2_hermitian(A) == pytest.approx(np.abs(np.linalg.eigvalsh(A)).max(), rel=1e-13)


def _energy(orc, A, B, nev):
    lam, _ = orc.solve(A, B, nev)
    return lam.sum()


def test_energy_gradient_fd(orc):
    # dE[dA] = Re tr(G_A^H dA) with G_A = X X^H; dE[dB] = Re tr(G_B^H dB) with G_B = -X L X^H
    rng = np.random.default_rng(7)
    n, nev = 16, 4
    lam0 = np.concatenate([np.linspace(-2, 1, nev), np.linspace(2, 9, n - nev)])
    from paper_1007_4400_gb300 import synth
    L = synth.draw_L(rng, n)
    Q, _ = np.linalg.qr(crandn(rng, n, n))
    A = L @ Q @ np.diag(lam0) @ Q.conj().T @ L.conj().T
    A = 0.5 * (A + A.conj().T)
    B = L @ L.conj().T
    lam, X = orc.solve(A, B, nev)
    GA, GB = orc.energy_grad(X, lam)
    h = 1e-6
    for t in range(4):
        P = rand_herm(rng, n)
        fd = (_energy(orc, A + h * P, B, nev) - _energy(orc, A - h * P, B, nev)) / (2 * h)
        an = np.real(np.sum(np.conj(GA) * P))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        Pb = 0.1 * rand_herm(rng, n)
        fdb = (_energy(orc, A, B + h * Pb, nev) - _energy(orc, A, B - h * Pb, nev)) / (2 * h)
        anb = np.real(np.sum(np.conj(GB) * Pb))
        assert abs(fdb - anb) <= 1e-6 * max(1.0, abs(anb))


def test_energy_gradient_degenerate_occupied(orc):
    # an exactly degenerate pair inside the occupied block, gap at nev: gradient finite and FD-exact
    rng = np.random.default_rng(8)
    n, nev = 12, 4
    lam0 = np.array([-1.0, 0.3, 0.3, 0.8] + list(np.linspace(2, 6, n - 4)))
    Q, _ = np.linalg.qr(crandn(rng, n, n))
    A = (Q * lam0) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    B = np.eye(n, dtype=np.complex128)
    lam, X = orc.solve(A, B, nev)
    GA, _ = orc.energy_grad(X, lam)
    assert np.all(np.isfinite(GA))
    P0 = Q[:, :nev] @ Q[:, :nev].conj().T
    assert np.abs(GA - P0).max() < 1e-10     # the occupied-space projector
    h = 1e-6
    P = rand_herm(rng, n)
    fd = (_energy(orc, A + h * P, B, nev) - _energy(orc, A - h * P, B, nev)) / (2 * h)
    assert abs(fd - np.real(np.sum(np.conj(GA) * P))) < 1e-6


def test_oracle_pin_catches_planted_sign_error(orc):
    # a plausible mistake (conjugating the wrong factor in the reduction) is detected by the
    # congruence pin: use C' = L^-1 A^T L^-H, which equals C only for real A
    rng = np.random.default_rng(9)
    n = 12
    A, B = rand_herm(rng, n), rand_hpd(rng, n)
    L, _ = orc.potrf(B)
    bad = orc.reduce(A.T.copy(), L)
    assert np.abs(L @ bad @ L.conj().T - A).max() > 1e-3


def _read_golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    A, B, lam = [], [], None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, *vals = line.split()
        if tag in ("A", "B"):
            v = [float(x) for x in vals]
            (A if tag == "A" else B).append([complex(v[2 * j], v[2 * j + 1]) for j in range(len(v) // 2)])
        elif tag == "lambda":
            lam = np.array([float(x) for x in vals])
    return np.array(A), np.array(B), lam


@pytest.mark.parametrize("name", ["pencil_2x2.txt", "pencil_3x3_block.txt"])
def test_golden_pencils(orc, name):
    """Hand-derived spectra stored in tests/golden (each file gives its derivation)."""
    A, B, lam = _read_golden(name)
    assert np.array_equal(A, A.conj().T) and np.array_equal(B, B.conj().T)
    for method in ("jacobi", "tridiag"):
        w, X = orc.solve(A, B, len(lam), method=method)
        assert np.abs(w - lam).max() <= 1e-14 * np.abs(lam).max()
        assert np.abs(A @ X - (B @ X) * w).max() <= 1e-13 * np.abs(lam).max()
