"""Parity of the deviation angles and the re-indexing (gevp_deviation_angles) with the
oracle: the cosine table element by element, the matching by its cost (several
assignments can be optimal: the one returned must be valid and reach the oracle's
optimum), the pairs outside the energy window exactly, and the angles of the matched
pairs. Sizes span several GEMM tiles with ragged edges; one case uses the eigenvectors
of consecutive problems of a solved sequence, one the full precision-form size with
sampled entries checked one by one."""
import math

import numpy as np
import pytest
import torch

from tests.conftest import crandn, rand_hpd

pytestmark = pytest.mark.gpu


def T(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _check(cuda, Xo, Xn, B, lo=None, ln=None, window=math.inf):
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    r = gevp.deviation_angles(T(Xo, cuda), T(Xn, cuda), None if B is None else T(B, cuda), lo, ln, window,
                              want_cosines=True)
    Bo = np.eye(Xo.shape[0]) if B is None else B
    c_ref = pieces.overlap_cosines(Xo, Xn, Bo)
    c = r["cosines"].cpu().numpy()
    assert np.abs(c - c_ref).max() <= 1e-12
    ko, kn = c_ref.shape
    lo_ = np.zeros(ko) if lo is None else np.asarray(lo)
    ln_ = np.zeros(kn) if ln is None else np.asarray(ln)
    perm_ref, cost_ref, nout_ref = pieces.reindex(Xo, Xn, Bo, lo_, ln_, window)
    perm = r["perm"]
    assert len(set(perm.tolist())) == ko and perm.min() >= 0 and perm.max() < kn
    far = np.abs(lo_[:, None] - ln_[None, :]) > window
    out = far[np.arange(ko), perm]
    assert int(out.sum()) == nout_ref == r["n_outside"]
    cost = float((1.0 - c_ref[np.arange(ko), perm])[~out].sum())
    assert abs(cost - cost_ref) <= 1e-10 * max(1.0, cost_ref)
    assert abs(r["cost"] - cost_ref) <= 1e-10 * max(1.0, cost_ref)
    # theta = acos(c) / (pi / 2) of the matched pairs: compare through the cosine, which
    # is well conditioned where the angle is small
    assert np.abs(np.cos(r["theta"] * math.pi / 2) - c_ref[np.arange(ko), perm]).max() <= 1e-12
    return r, perm_ref


@pytest.mark.parametrize("n,ko,kn", [(700, 37, 45), (129, 1, 1), (96, 64, 64), (1030, 150, 161)])
def test_random_vectors_vs_oracle(cuda, n, ko, kn):
    rng = np.random.default_rng(70 + n + ko)
    B = rand_hpd(rng, n, cond=1e3)
    Xo = crandn(rng, n, ko)
    Xn = crandn(rng, n, kn)
    Xn[:, :ko] += 3.0 * Xo   # a dominant partner for every old vector, at varied angles
    _check(cuda, Xo, Xn, B)


def test_permuted_rephased_copy(cuda):
    rng = np.random.default_rng(71)
    n, k = 500, 60
    B = rand_hpd(rng, n, cond=100.0)
    Xo = crandn(rng, n, k)
    sh = rng.permutation(k)
    Xn = Xo[:, sh] * np.exp(1j * rng.uniform(0, 2 * np.pi, k)) * rng.uniform(0.5, 2.0, k)
    r, _ = _check(cuda, Xo, Xn, B)
    assert np.array_equal(r["perm"], np.argsort(sh))
    assert r["theta"].max() < 1e-6


def test_energy_window_forbids_the_unrestricted_optimum(cuda):
    # new vectors are a shuffled, perturbed copy of the old while the eigenvalues stay in
    # place: without a window the matching follows the vectors, with a narrow one it must
    # keep i -> i
    rng = np.random.default_rng(72)
    n, k = 300, 24
    B = rand_hpd(rng, n, cond=30.0)
    Xo = crandn(rng, n, k)
    sh = np.roll(np.arange(k), 1)
    Xn = Xo[:, sh] + 0.4 * crandn(rng, n, k)
    lo = np.arange(k) * 0.1
    ln = lo + 0.003
    r0, _ = _check(cuda, Xo, Xn, B)
    assert np.array_equal(r0["perm"], np.argsort(sh))
    r1, _ = _check(cuda, Xo, Xn, B, lo, ln, window=0.01)
    assert np.array_equal(r1["perm"], np.arange(k)) and r1["n_outside"] == 0


def test_euclidean_inner_product(cuda):
    rng = np.random.default_rng(73)
    Xo = crandn(rng, 257, 20)
    Xn = Xo + 0.2 * crandn(rng, 257, 20)
    _check(cuda, Xo, Xn, None)


def test_without_reindexing(cuda):
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(74)
    n, k = 400, 30
    B = rand_hpd(rng, n, cond=10.0)
    Xo = crandn(rng, n, k)
    Xn = Xo + 0.3 * crandn(rng, n, k)
    r = gevp.deviation_angles(T(Xo, cuda), T(Xn, cuda), T(B, cuda), reindex=False)
    assert r["perm"] is None
    th_ref = pieces.deviation_angles(Xo, Xn, B)
    assert np.abs(np.cos(r["theta"] * math.pi / 2) - np.cos(th_ref * math.pi / 2)).max() <= 1e-12


def test_zero_vector_is_an_error(cuda):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(75)
    Xo = crandn(rng, 64, 4)
    Xn = crandn(rng, 64, 4)
    Xn[:, 2] = 0.0
    with pytest.raises(gevp.GevpError) as e:
        gevp.deviation_angles(T(Xo, cuda), T(Xn, cuda))
    assert e.value.status == 7   # GEVP_ERR_INVALID_VALUE


def test_consecutive_eigenvectors_of_a_sequence(cuda):
    """The eigenvectors of consecutive problems of a solved sequence: every old vector has
    a partner at a small angle, and the matching agrees with the oracle's."""
    from paper_1007_4400_gb300 import gevp, synth
    n, nev, nex = 600, 24, 10
    s = synth.make_sequence(1, n, 3, nev, nex, device=cuda)
    res = gevp.solve_sequence(s.A, s.B, nev, nex=nex, keep_all_X=True)
    assert res.status == 0
    X = res.X.cpu().numpy()
    lam = res.Lambda.cpu().numpy()
    B = s.B.cpu().numpy()
    gap = float(np.diff(lam[0]).max())
    for l in (0, 1):
        r, _ = _check(cuda, X[l], X[l + 1], B, lam[l], lam[l + 1], window=gap)
        assert np.median(r["theta"]) < 0.5


def test_full_size_sampled(cuda):
    """n = 6144, 360 x 360 vectors (the precision form's block): the device table at
    sampled entries against the definition computed one entry at a time."""
    from paper_1007_4400_gb300 import gevp
    n, k = 6144, 360
    g = torch.Generator(device="cpu").manual_seed(76)
    def rnd(*shape):
        return torch.complex(torch.randn(*shape, generator=g, dtype=torch.float64),
                             torch.randn(*shape, generator=g, dtype=torch.float64))
    # HPD with its spectrum inside about [1.6, 4.4]: 3 I plus a scaled Hermitian Gaussian
    E = rnd(n, n) / (2.0 * math.sqrt(n))
    B = (E + E.conj().T + 3.0 * torch.eye(n, dtype=torch.complex128)).numpy()
    Xo = rnd(n, k).numpy()
    Xn = Xo + 0.5 * rnd(n, k).numpy()
    r = gevp.deviation_angles(T(Xo, cuda), T(Xn, cuda), T(B, cuda), want_cosines=True)
    c = r["cosines"].cpu().numpy()
    rng = np.random.default_rng(77)
    rows = rng.integers(0, k, 12)
    cols = np.concatenate([rows[:6], rng.integers(0, k, 6)])
    for i, j in zip(rows, cols):
        bo, bn = B @ Xo[:, i], B @ Xn[:, j]
        ref = abs(np.vdot(Xo[:, i], bn)) / math.sqrt(np.vdot(Xo[:, i], bo).real * np.vdot(Xn[:, j], bn).real)
        assert abs(c[i, j] - min(ref, 1.0)) <= 1e-12
    assert len(set(r["perm"].tolist())) == k
    assert np.array_equal(r["perm"], np.arange(k))
