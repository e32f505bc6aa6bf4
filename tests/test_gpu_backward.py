"""Differentiable form: E = sum of the lowest nev eigenvalues through torch.autograd with
the library's backward kernel (dE/dA = X X^H, dE/dB = -X Lambda X^H), checked against
central finite differences of the GPU solver and against the oracle's gradient."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _pencil(n, nev, seed, degenerate=False):
    from paper_1007_4400_gb300 import synth
    rng = synth.rng_for(4, seed)
    L = synth.draw_L(rng, n)
    Q = synth.haar_unitary(rng, n).numpy()
    lam = synth.clustered_spectrum(rng, n, nev)
    if degenerate:
        lam[1] = lam[2]
    A = (L @ Q) * lam @ (L @ Q).conj().T
    A = 0.5 * (A + A.conj().T)
    B = L @ L.conj().T
    B = 0.5 * (B + B.conj().T)
    return A, B


def _energy(A, B, nev, nex):
    from paper_1007_4400_gb300 import gevp
    r = gevp.solve_sequence([A], B, nev, nex=nex)
    assert r.status == 0
    return float(r.Lambda[0].sum())


@pytest.mark.parametrize("degenerate", [False, True])
def test_autograd_matches_oracle_and_fd(cuda, orc, degenerate):
    from paper_1007_4400_gb300 import gevp
    n, nev, nex = 160, 12, 6
    A_np, B_np = _pencil(n, nev, 3 + int(degenerate), degenerate)
    A = torch.from_numpy(A_np).to(cuda).requires_grad_(True)
    B = torch.from_numpy(B_np).to(cuda).requires_grad_(True)
    E = gevp.band_energy(A, B, nev, nex=nex)
    E.backward()
    GA, GB = A.grad.cpu().numpy(), B.grad.cpu().numpy()
    assert np.all(np.isfinite(GA)) and np.all(np.isfinite(GB))
    lam_r, X_r = orc.solve(A_np, B_np, nev, method="jacobi")
    GAr, GBr = orc.energy_grad(X_r, lam_r)
    assert np.abs(GA - GAr).max() <= 1e-10 * np.abs(GAr).max()
    assert np.abs(GB - GBr).max() <= 1e-10 * np.abs(GBr).max()
    assert float(E.detach()) == pytest.approx(lam_r.sum(), rel=1e-12, abs=1e-12 * np.abs(lam_r).max())
    # central finite differences along random Hermitian directions (step 1e-6)
    rng = np.random.default_rng(11)
    h = 1e-6
    Ad = A.detach()
    Bd = B.detach()
    for _ in range(4):
        P = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        P = torch.from_numpy(0.5 * (P + P.conj().T)).to(cuda)
        fd = (_energy(Ad + h * P, Bd, nev, nex) - _energy(Ad - h * P, Bd, nev, nex)) / (2 * h)
        an = float(torch.real(torch.sum(torch.conj(A.grad) * P)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        Pb = 0.01 * P
        fdb = (_energy(Ad, Bd + h * Pb, nev, nex) - _energy(Ad, Bd - h * Pb, nev, nex)) / (2 * h)
        anb = float(torch.real(torch.sum(torch.conj(B.grad) * Pb)))
        assert abs(fdb - anb) <= 1e-6 * max(1.0, abs(anb))


def test_autograd_matches_oracle_n1024(cuda, orc):
    """The oracle's gradient at a size where the oracle's full solve takes seconds."""
    from paper_1007_4400_gb300 import gevp
    n, nev, nex = 1024, 50, 20
    A_np, B_np = _pencil(n, nev, 21)
    A = torch.from_numpy(A_np).to(cuda).requires_grad_(True)
    B = torch.from_numpy(B_np).to(cuda).requires_grad_(True)
    E = gevp.band_energy(A, B, nev, nex=nex, filter_prec="fp32")
    E.backward()
    lam_r, X_r = orc.solve(A_np, B_np, nev, method="tridiag")
    GAr, GBr = orc.energy_grad(X_r, lam_r)
    GA, GB = A.grad.cpu().numpy(), B.grad.cpu().numpy()
    # Both gradients are sums of nev outer products of eigenvectors, whose errors are of
    # the order of the residuals (~1e-12 ||A||) over the eigenvalue gaps; at n = 1024 that
    # is ~1e-10 relative in the entries of -X Lambda X^H. A wrong formula (a dropped
    # conjugate, sign or Lambda) differs at O(1), so 1e-9 still separates right from wrong.
    assert np.abs(GA - GAr).max() <= 1e-9 * np.abs(GAr).max()
    assert np.abs(GB - GBr).max() <= 1e-9 * np.abs(GBr).max()


@pytest.mark.slow
def test_autograd_full_size_n4096(cuda):
    """The differentiation workload at full size (n 4096, nev 200, nex 50, clustered
    spectrum near the gap, FP32-class tensor-core filter): central differences (step
    1e-6) along 16 random Hermitian directions of A and 4 of B, and the trace identities
    tr(G_A B) = nev and tr(G_B A) = -sum lambda^2 that hold at any size."""
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.workload("grad_n4096", device=cuda)
    nev, nex = s.nev, s.nex
    A = s.A[0].clone().requires_grad_(True)
    B = s.B.clone().requires_grad_(True)
    E = gevp.band_energy(A, B, nev, nex=nex, filter_prec="fp32")
    E.backward()
    GA, GB = A.grad, B.grad
    r = gevp.solve_sequence([A.detach()], B.detach(), nev, nex=nex, filter_prec="fp32")
    lam = r.Lambda[0]
    X = r.X
    assert abs(float(torch.real(torch.sum(GA * B.detach().T))) - nev) <= 1e-9 * nev
    lam2 = float((lam * lam).sum())
    assert abs(float(torch.real(torch.sum(GB * A.detach().T))) + lam2) <= 1e-9 * lam2
    rng = np.random.default_rng(4096)
    h = 1e-6
    lmax = float(lam.abs().max())
    Ad, Bd = A.detach(), B.detach()

    def energy(Ax, Bx):
        rr = gevp.solve_sequence([Ax], Bx, nev, nex=nex, filter_prec="fp32", X_prev=X)
        assert rr.status == 0
        return float(rr.Lambda[0].sum())

    # eigenvalue noise of a converged solve is ~1e-14 relative per eigenvalue
    noise = 2 * nev * 2e-14 * lmax / h
    for i in range(20):
        P = rng.standard_normal((s.n, s.n)) + 1j * rng.standard_normal((s.n, s.n))
        P = torch.from_numpy(0.5 * (P + P.conj().T)).to(cuda)
        if i < 16:
            fd = (energy(Ad + h * P, Bd) - energy(Ad - h * P, Bd)) / (2 * h)
            an = float(torch.real(torch.sum(torch.conj(GA) * P)))
        else:
            P = 1e-3 * P
            fd = (energy(Ad, Bd + h * P) - energy(Ad, Bd - h * P)) / (2 * h)
            an = float(torch.real(torch.sum(torch.conj(GB) * P)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + noise, (i, fd, an)
