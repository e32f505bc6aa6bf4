"""The seeded generator's stated properties: the realised conditioning of B for the
plain and the ill-conditioned workloads, the known spectrum of problem 0, the drift of
the sequence, and the k-point batch sizes."""
import math

import numpy as np


def _condB(L):
    s = np.linalg.svd(L, compute_uv=False)
    return (s[0] / s[-1]) ** 2


def test_condition_of_B():
    from paper_1007_4400_gb300 import synth
    # recipe of the plain workloads: diag U[0.5, 2], off-diagonals 0.3/sqrt(n) complex normal
    c0 = _condB(synth.draw_L(synth.rng_for(0, 0), 256))
    assert 5.0 < c0 < 100.0
    # ill-conditioned workload: log-uniform diagonal in [6e-3, 2], rows scaled: about 1e5
    c2 = _condB(synth.draw_L(synth.rng_for(2, 0), 256, diag=(6e-3, 2.0), log_uniform_diag=True))
    assert 3e4 < c2 < 5e5


def test_sequence_spectrum_and_drift():
    from paper_1007_4400_gb300 import synth
    s = synth.make_sequence(1, 64, 4, 8, 4)
    A0, B = s.A[0].numpy(), s.B.numpy()
    L = s.L_true.numpy()
    Li = np.linalg.inv(L)
    ev = np.linalg.eigvalsh(Li @ A0 @ Li.conj().T)
    assert np.abs(ev - s.lam0).max() <= 1e-10 * np.abs(s.lam0).max()
    for l in range(3):
        d = s.A[l + 1].numpy() - s.A[l].numpy()
        assert abs(np.linalg.norm(d, 2) - 0.1 * 0.6 ** l) <= 1e-9
        assert np.abs(d - d.conj().T).max() == 0.0


def test_kpoint_sizes():
    from paper_1007_4400_gb300 import synth
    sz = synth.batched_sizes(64)
    assert len(sz) == 64
    for n, nev, nex in sz:
        assert 800 <= n <= 3000 and nev == int(round(0.06 * n)) and nex == math.ceil(0.4 * nev)


def test_lanczos_norm_estimate():
    """The spectral-norm estimate used to scale the perturbations of the largest workload."""
    import torch
    from paper_1007_4400_gb300 import synth
    rng = synth.rng_for(9, 1)
    P = synth.hermitian_part(torch.from_numpy(synth._cnormal(rng, (900, 900))))
    exact = float(torch.linalg.eigvalsh(P).abs().max())
    assert abs(synth._norm2_lanczos(P) - exact) <= 1e-3 * exact


def test_deviation_angles_shrink_along_the_sequence(orc):
    """The sequences behave as the paper reports for its SCF runs (Sec. "A new computational
    philosophy", paragraph "Eigenvectors evolution"): the deviation angles of the matched
    eigenvectors of consecutive problems are small and shrink as the sequence advances.
    Oracle eigenvectors, the oracle's re-indexing."""
    from oracle import pieces
    from paper_1007_4400_gb300 import synth
    n, nev = 120, 10
    s = synth.make_sequence(1, n, 6, nev, 4)
    B = s.B.numpy()
    X = []
    lam = []
    for a in s.A:
        lr, xr = orc.solve(a.numpy(), B, nev, method="jacobi")
        lam.append(lr)
        X.append(xr)
    means = []
    for l in range(len(X) - 1):
        perm, _, nout = pieces.reindex(X[l], X[l + 1], B, lam[l], lam[l + 1])
        c = pieces.overlap_cosines(X[l], X[l + 1], B)[np.arange(nev), perm]
        theta = np.arccos(np.clip(c, 0.0, 1.0)) / (math.pi / 2)
        means.append(theta.mean())
    assert max(means) < 0.2
    assert all(b < a for a, b in zip(means, means[1:]))
