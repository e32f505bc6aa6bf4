"""Per-step parity of the CUDA kernels (through the C ABI) with the FP64 oracle's
definitions, on seeded inputs spanning several tiles and ragged tails."""
import numpy as np
import pytest
import torch

from tests.conftest import crandn, rand_herm, rand_hpd

pytestmark = pytest.mark.gpu


def T(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n", [1, 2, 17, 64, 127, 200])
def test_reduce_parity(cuda, orc, n):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(100 + n)
    A, B = rand_herm(rng, n), rand_hpd(rng, n, 1e3)
    L, C = gevp.reduce(T(A, cuda), T(B, cuda))
    Lr, info = orc.potrf(B)
    assert info == 0
    Cr = orc.reduce(A, Lr)
    assert relmax(L.cpu().numpy(), Lr) < 1e-13
    assert relmax(C.cpu().numpy(), Cr) < 1e-12
    assert np.array_equal(np.triu(L.cpu().numpy(), 1), np.zeros((n, n)))


def test_reduce_not_hpd(cuda):
    from paper_1007_4400_gb300 import gevp
    B = np.diag(np.array([1.0, 2.0, -1.0, 3.0] + [1.0] * 60)).astype(np.complex128)
    A = np.eye(64, dtype=np.complex128)
    with pytest.raises(gevp.GevpError) as e:
        gevp.reduce(T(A, cuda), T(B, cuda))
    assert e.value.status == 2 and "pivot 3" in str(e.value)


@pytest.mark.parametrize("n,m,deg", [(200, 13, 1), (200, 13, 2), (333, 40, 9), (64, 64, 5)])
def test_filter_parity(cuda, orc, n, m, deg):
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(200 + n + m + deg)
    lam = np.sort(rng.uniform(-2, 50, n))
    Q, _ = np.linalg.qr(crandn(rng, n, n))
    Cm = (Q * lam) @ Q.conj().T
    Cm = 0.5 * (Cm + Cm.conj().T)
    Y0 = crandn(rng, n, m)
    lo, hi, s = 5.0, 50.5, -2.5
    Yg = gevp.chebyshev_filter(T(Cm, cuda), T(Y0, cuda), deg, lo, hi, s).cpu().numpy()
    Yr = pieces.chebyshev_filter(Cm, Y0, deg, lo, hi, s)
    assert relmax(Yg, Yr) < 1e-12


# m 288: the largest order of the cluster factorisation; m 289: the blocked path
@pytest.mark.parametrize("n,m", [(300, 21), (1000, 48), (517, 140), (900, 288), (900, 289)])
def test_cholqr2_parity(cuda, orc, n, m):
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(300 + m)
    Y = crandn(rng, n, m) @ np.diag(np.logspace(0, 3, m))
    Qg, Rg = gevp.cholqr2(T(Y, cuda), want_R=True)
    Qg, Rg = Qg.cpu().numpy(), Rg.cpu().numpy()
    Qr, Rr = pieces.cholqr2(Y)
    assert np.abs(Qg.conj().T @ Qg - np.eye(m)).max() < 1e-13
    assert relmax(Qg, Qr) < 1e-10
    assert relmax(Rg, Rr) < 1e-10


# one CTA below 32, the eight-CTA cluster form for 32..256, the cooperative form above
@pytest.mark.parametrize("m", [1, 2, 3, 17, 31, 32, 33, 64, 140, 159, 161, 200, 201, 255, 256, 257, 301])
def test_heev_small_parity(cuda, orc, m):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(400 + m)
    G = rand_herm(rng, m) * 10
    th, Z = gevp.heev_small(T(G, cuda))
    th, Z = th.cpu().numpy(), Z.cpu().numpy()
    w, V = orc.heev(G, method="jacobi")
    scale = np.abs(w).max()
    assert np.abs(th - w).max() <= 1e-12 * scale
    assert np.abs(Z.conj().T @ Z - np.eye(m)).max() < 1e-13
    assert np.abs(G @ Z - Z * th).max() <= 1e-12 * scale


@pytest.mark.parametrize("m", [48, 140, 300, 333])
def test_heev_small_clustered_wide(cuda, orc, m):
    # the shape of a cold-start Rayleigh-Ritz projection: a dense cluster of small values,
    # a near-degenerate pair and a wide sparse tail; Z must stay orthonormal to FP64 level
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(4200 + m)
    k = int(0.7 * m)
    lam = np.concatenate([np.sort(rng.uniform(-2, 2, k)), [3.0, 3.0 + 1e-9],
                          np.sort(rng.uniform(5, 60, m - k - 2))])
    Q, _ = np.linalg.qr(crandn(rng, m, m))
    G = (Q * lam) @ Q.conj().T
    G = 0.5 * (G + G.conj().T)
    th, Z = gevp.heev_small(T(G, cuda))
    th, Z = th.cpu().numpy(), Z.cpu().numpy()
    assert np.abs(Z.conj().T @ Z - np.eye(m)).max() < 1e-13
    assert np.abs(th - np.sort(lam)).max() <= 1e-12 * 60
    assert np.abs(G @ Z - Z * th).max() <= 1e-12 * 60


def test_heev_small_degenerate(cuda, orc):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(41)
    m = 50
    lam = np.concatenate([[-3.0], [1.0] * 3, np.linspace(2, 9, m - 4)])
    Q, _ = np.linalg.qr(crandn(rng, m, m))
    G = (Q * lam) @ Q.conj().T
    G = 0.5 * (G + G.conj().T)
    th, Z = gevp.heev_small(T(G, cuda))
    th, Z = th.cpu().numpy(), Z.cpu().numpy()
    assert np.abs(th - lam).max() < 1e-12 * 9
    P1 = Q[:, 1:4] @ Q[:, 1:4].conj().T
    P2 = Z[:, 1:4] @ Z[:, 1:4].conj().T
    assert np.abs(P1 - P2).max() < 1e-10


@pytest.mark.parametrize("m,eps", [(140, 1e-5), (140, 5e-4), (64, 1e-7), (256, 1e-4), (140, 3e-2)])
def test_heev_small_nearly_diagonal(cuda, orc, m, eps):
    """The projection of a nearly converged block: a diagonal plus couplings of eps times
    the gaps, unsorted, with a near-degenerate pair whose coupling is tiny. For eps 1e-5
    and 1e-7 the cluster eigensolver starts the FP64 refinement from Z = I without FP32
    sweeps (the couplings are below 1e-3 of the gaps and no gap lies between 1e-6 ||G||_F
    and 2 ||offdiag G||_F); the larger eps take the sweeps. Both must give the oracle's
    eigenpairs; in the first the later corrections couple the near-degenerate pair, which
    the refinement must then leave to the exact rotations."""
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(4300 + m + int(-np.log10(eps)))
    d = rng.permutation(np.concatenate([np.linspace(-2.0, 2.0, m - 2), [0.3 + 1e-9, 0.3 + 2e-9]]))
    gaps = np.abs(d[:, None] - d[None, :]) + np.eye(m)
    E = crandn(rng, m, m)
    E = 0.5 * (E + E.conj().T)
    np.fill_diagonal(E, 0.0)
    G = np.diag(d).astype(np.complex128) + eps * np.minimum(gaps, 1.0) * E / np.abs(E).max()
    near = np.where(np.abs(d - 0.3) < 1e-8)[0]
    G[near[0], near[1]] = G[near[1], near[0]] = 1e-12
    th, Z = gevp.heev_small(T(G, cuda))
    th, Z = th.cpu().numpy(), Z.cpu().numpy()
    w, V = orc.heev(G, method="jacobi")
    assert np.abs(th - w).max() <= 1e-13 * 2.0
    assert np.abs(Z.conj().T @ Z - np.eye(m)).max() < 1e-13
    assert np.abs(G @ Z - Z * th).max() <= 1e-13 * 2.0


@pytest.mark.parametrize("n,m", [(256, 24), (611, 48)])
def test_rayleigh_ritz_parity(cuda, orc, n, m):
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(500 + n)
    lam = np.sort(rng.uniform(-2, 50, n))
    Qf, _ = np.linalg.qr(crandn(rng, n, n))
    Cm = (Qf * lam) @ Qf.conj().T
    Cm = 0.5 * (Cm + Cm.conj().T)
    Q0, _ = np.linalg.qr(Qf[:, :m] + 1e-3 * crandn(rng, n, m))
    th, Qg, Wg, rs = gevp.rayleigh_ritz(T(Cm, cuda), T(Q0, cuda))
    thr, Qr, Wr = pieces.rayleigh_ritz(Cm, Q0)
    assert np.abs(th.cpu().numpy() - thr).max() <= 1e-12 * 50
    ov = np.abs(np.sum(np.conj(Qr) * Qg.cpu().numpy(), axis=0))
    assert np.all(ov > 1 - 1e-9)
    rr = pieces.residual_norms(Wr, Qr, thr)
    assert np.abs(rs.cpu().numpy() - rr).max() <= 1e-11 * 50


def test_spectral_bounds(cuda, orc):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(600)
    n = 500
    lam = np.sort(rng.uniform(-2, 50, n))
    Q, _ = np.linalg.qr(crandn(rng, n, n))
    Cm = (Q * lam) @ Q.conj().T
    Cm = 0.5 * (Cm + Cm.conj().T)
    lo_ritz, hi_ritz, upper, aest, beta = gevp.spectral_bounds(T(Cm, cuda), 32, 48)
    assert upper >= lam[-1]
    assert lo_ritz >= lam[0] - 1e-4 * 50 and hi_ritz <= lam[-1] + 1e-4 * 50
    assert lam[0] - 1 <= aest <= lam[-1] + 1


@pytest.mark.parametrize("n,nev", [(100, 7), (300, 40)])
def test_energy_backward_parity(cuda, orc, n, nev):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(700 + n)
    X = crandn(rng, n, nev)
    lam = np.sort(rng.uniform(-2, 5, nev))
    GA, GB = gevp.energy_backward(T(X, cuda), T(lam, cuda), 0.7)
    GAr, GBr = orc.energy_grad(X, lam, 0.7)
    assert relmax(GA.cpu().numpy(), GAr) < 1e-13
    assert relmax(GB.cpu().numpy(), GBr) < 1e-13


def test_energy_backward_device_scalar_gradient(cuda, orc):
    """The incoming gradient is read on the device (a one-element tensor): the same result
    as the oracle's gradient scaled by it, negative and zero scales included."""
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(711)
    n, nev = 150, 11
    X = crandn(rng, n, nev)
    lam = np.sort(rng.uniform(-2, 5, nev))
    GA1, GB1 = orc.energy_grad(X, lam, 1.0)
    for g in (-1.75, 0.0, 3.0):
        gE = torch.tensor([g], dtype=torch.float64, device=cuda)
        GA, GB = gevp.energy_backward(T(X, cuda), T(lam, cuda), gE)
        GAr, GBr = orc.energy_grad(X, lam, g)
        tol = 1e-13 * max(1.0, abs(g))
        assert np.abs(GA.cpu().numpy() - GAr).max() <= tol * np.abs(GA1).max()
        assert np.abs(GB.cpu().numpy() - GBr).max() <= tol * np.abs(GB1).max()


def test_band_energy_sums_in_index_order(cuda):
    """gevp_band_energy: E[p] = sum of row p of Lambda, summed in index order (bit-exact
    against the same sequential sum on the host), empty rows give 0."""
    import functools
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(712)
    lam = rng.uniform(-2, 50, (5, 37)) * 10.0 ** rng.integers(-8, 8, (5, 37))
    E = gevp.band_energy_of(T(lam, cuda)).cpu().numpy()
    for p in range(lam.shape[0]):
        assert E[p] == functools.reduce(lambda a, b: a + b, lam[p].tolist(), 0.0)
    E0 = gevp.band_energy_of(torch.zeros((3, 0), dtype=torch.float64, device=cuda)).cpu().numpy()
    assert np.array_equal(E0, np.zeros(3))
