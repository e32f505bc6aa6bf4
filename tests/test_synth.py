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
