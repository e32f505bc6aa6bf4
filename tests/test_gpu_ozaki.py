"""Parity of the FP64 products emulated on the tensor cores (gevp_zgemm_emulated,
gevp_reduce_emulated, and the sequence solver with the emulated reduction) with the
oracle: bit-exact on inputs whose digits represent them exactly, within the stated error
bound on random data (the bound is written out here from the splitting's arithmetic),
the reduction against the oracle's reduction, and the solver's eigenpairs against the
closed-form spectrum and the oracle at the precision form's full size."""
import math

import numpy as np
import pytest
import torch

from tests.conftest import crandn, rand_herm, rand_hpd

pytestmark = pytest.mark.gpu


def T(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def scale(A, B):
    """max_k |A_ik| x max_k |B_jk| over real and imaginary parts: the unit of the bound"""
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
    rb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=1)
    return np.outer(ra, rb)


def bound(K, S):
    """Worst case per entry, in units of scale(): each entry of A, B is rounded to within
    2^(-7S-1) of its row's 2^e (2^e <= 4 max), the pairs past the last digit weigh at most
    (S + 1) 2^(-7S-2) per term, 2K real terms, and 16 from the two power-of-two scales."""
    return 16 * 2 * K * (S + 3) * 2.0 ** (-7 * S - 2)


# (2048, 140, 140): the solver's thin products (K = m), whose digit pairs of one level
# accumulate in one tensor-memory buffer; (257, 300, 1000) also takes that form per split-K
# slice (K slices of 128); the last two keep one buffer per pair. N from 129 to 144 runs
# in one 144-wide tile with a single accumulator: (128, 129, 2100), (2048, 140, 140),
# (300, 144, 2048), the solver's W = C Q shape
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 70, 64), (2048, 140, 140), (257, 300, 1000), (128, 129, 2100),
                                   (300, 144, 2048), (64, 200, 4177)])
@pytest.mark.parametrize("S", [1, 3, 8])
def test_exact_on_small_integers(cuda, M, N, K, S):
    # entries in {-2..2} + i{-2..2}: one digit holds them, every product and sum is exact
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(1000 + M + N + K + S)
    A = rng.integers(-2, 3, (M, K)) + 1j * rng.integers(-2, 3, (M, K))
    B = rng.integers(-2, 3, (N, K)) + 1j * rng.integers(-2, 3, (N, K))
    D = gevp.zgemm_emulated(T(A, cuda), T(B, cuda), slices=S).cpu().numpy()
    assert np.array_equal(D, A @ B.conj().T)


@pytest.mark.parametrize("M,N,K", [(200, 130, 700), (4096, 140, 140), (2048, 140, 2048), (129, 257, 2048),
                                   (300, 64, 2049), (96, 96, 5000)])
def test_random_within_bound(cuda, M, N, K):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(2000 + M + N + K)
    A = crandn(rng, M, K) * np.exp(rng.uniform(-6, 6, (M, 1)))   # rows of different magnitudes
    B = crandn(rng, N, K)
    B[:, : K // 3] *= 1e-3                                        # and a wide range inside rows
    ref = A @ B.conj().T
    sc = scale(A, B)
    for S in (6, 8):
        D = gevp.zgemm_emulated(T(A, cuda), T(B, cuda), slices=S).cpu().numpy()
        err = np.abs(D - ref) / sc
        assert err.max() <= bound(K, S) + 1e-15
        if S == 8:
            # typical size: the roundings are independent, so about sqrt(2K) of them add up
            assert err.max() <= 64 * math.sqrt(2 * K) * 2.0 ** (-7 * S)


@pytest.mark.parametrize("opA,opB", [("N", "N"), ("C", "C"), ("C", "N"), ("N", "C")])
def test_op_variants(cuda, opA, opB):
    # rows of op(A) and columns of op(B) come from rows or (transposed) columns of the
    # stored matrices; every combination against the plain product
    from paper_1007_4400_gb300 import gevp
    M, N, K = 150, 97, 777
    rng = np.random.default_rng(2500 + len(opA + opB) + (opA == "C") * 7 + (opB == "C") * 13)
    opa = crandn(rng, M, K) * np.exp(rng.uniform(-3, 3, (M, 1)))
    opb = crandn(rng, K, N) * np.exp(rng.uniform(-3, 3, (1, N)))
    A = opa if opA == "N" else opa.conj().T
    B = opb if opB == "N" else opb.conj().T
    D = gevp.zgemm_emulated(T(A, cuda), T(B, cuda), slices=8, opA=opA, opB=opB).cpu().numpy()
    ref = opa @ opb
    err = np.abs(D - ref) / scale(opa, opb.T)
    assert err.max() <= 64 * math.sqrt(2 * K) * 2.0 ** -56


def test_zero_rows_and_empty_k(cuda):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(3000)
    A = crandn(rng, 50, 90)
    A[7] = 0.0
    B = crandn(rng, 40, 90)
    D = gevp.zgemm_emulated(T(A, cuda), T(B, cuda)).cpu().numpy()
    assert np.array_equal(D[7], np.zeros(40))
    assert np.abs(D - A @ B.conj().T).max() <= 1e-13 * np.abs(A).max() * np.abs(B).max() * 90
    E = gevp.zgemm_emulated(torch.zeros((3, 0), dtype=torch.complex128, device=cuda),
                            torch.zeros((4, 0), dtype=torch.complex128, device=cuda)).cpu().numpy()
    assert np.array_equal(E, np.zeros((3, 4)))


def test_nan_is_an_error(cuda):
    from paper_1007_4400_gb300 import gevp
    A = torch.ones((10, 20), dtype=torch.complex128, device=cuda)
    A[3, 4] = complex(float("nan"), 0.0)
    with pytest.raises(gevp.GevpError) as e:
        gevp.zgemm_emulated(A, torch.ones((5, 20), dtype=torch.complex128, device=cuda))
    assert e.value.status == 7


# 130 and 144: the right operands of the reduction's second product (L^-H, triangular)
# have 129..144 rows and run in one 144-wide tile, whose triangle ends inside a K block
@pytest.mark.parametrize("n", [1, 17, 130, 144, 200, 333])
def test_reduce_emulated_vs_oracle(cuda, orc, n):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(4000 + n)
    A, B = rand_herm(rng, n), rand_hpd(rng, n, 1e3)
    L, C = gevp.reduce(T(A, cuda), T(B, cuda), slices=8)
    Lr, info = orc.potrf(B)
    assert info == 0
    Cr = orc.reduce(A, Lr)
    C = C.cpu().numpy()
    assert np.abs(C - Cr).max() / np.abs(Cr).max() < 1e-12
    assert np.array_equal(C, C.conj().T)


# the emulated mode factors B recursively: leaves of order <= 256 in one cluster launch,
# the off-diagonal blocks of L and L^-1 from emulated products. 256: one leaf; 300: one
# split (128 + 172); 700 and 1100: two and three levels with ragged leaves.
@pytest.mark.parametrize("n", [256, 300, 700, 1100])
def test_emulated_factor_vs_oracle(cuda, orc, n):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(4100 + n)
    A, B = rand_herm(rng, n), rand_hpd(rng, n, 1e3)
    L, C = gevp.reduce(T(A, cuda), T(B, cuda), slices=8)
    L = L.cpu().numpy()
    Lr, info = orc.potrf(B)
    assert info == 0
    assert np.array_equal(np.triu(L, 1), np.zeros_like(L))
    assert np.abs(L - Lr).max() <= 1e-13 * np.abs(Lr).max()
    # the reduction used the recursive form's L^-1: C against the oracle's
    Cr = orc.reduce(A, Lr)
    assert np.abs(C.cpu().numpy() - Cr).max() <= 1e-12 * np.abs(Cr).max()


@pytest.mark.parametrize("n,k", [(600, 400), (600, 17), (200, 150)])
def test_emulated_factor_not_hpd(cuda, n, k):
    """A non-positive pivot in a later leaf, in the first leaf and in a single leaf: the
    global 1-based index is reported, the handle stays usable."""
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(4200 + n + k)
    B = rand_hpd(rng, n, 10.0)
    B[k, :] = 0.0
    B[:, k] = 0.0
    B[k, k] = -1.0
    A = np.eye(n, dtype=np.complex128)
    with pytest.raises(gevp.GevpError) as e:
        gevp.reduce(T(A, cuda), T(B, cuda), slices=8)
    assert e.value.status == 2 and f"pivot {k + 1}" in str(e.value)
    B2 = rand_hpd(rng, n, 10.0)
    L, _ = gevp.reduce(T(A, cuda), T(B2, cuda), slices=8)
    Lh = L.cpu().numpy()
    assert np.abs(Lh @ Lh.conj().T - B2).max() <= 1e-13 * np.abs(B2).max() * n


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solver_with_emulated_reduction(cuda, orc, prec):
    from paper_1007_4400_gb300 import gevp, synth
    n, nev, nex = 700, 30, 12
    s = synth.make_sequence(1, n, 4, nev, nex, device=cuda)
    r = gevp.solve_sequence(s.A, s.B, nev, nex=nex, filter_prec=prec, reduce_slices=8, keep_all_X=True)
    assert r.status == 0, r.stats
    lam = r.Lambda.cpu().numpy()
    assert np.abs(lam[0] - s.lam0[:nev]).max() <= 1e-12 * np.abs(s.lam0).max()
    assert float(r.resid.max()) <= 1e-10
    B = s.B.cpu().numpy()
    for l in (1, 3):
        lr, _ = orc.solve(s.A[l].cpu().numpy(), B, nev, method="jacobi")
        assert np.abs(lam[l] - lr).max() <= 1e-12 * np.abs(lr).max()


@pytest.mark.slow
def test_emulated_reduction_full_size(cuda, orc):
    """n = 6144, cond(B) ~ 1.3e5, clustered spectrum (the precision form's first problems):
    the congruence L C L^H = A at sampled entries, and the solver with the emulated
    reduction against the closed-form spectrum, its residuals and B-orthonormality."""
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.workload("scf_seq_n6144_cond1e5", device=cuda, nprob=3)
    L, C = gevp.reduce(s.A[0], s.B, slices=8)
    Lh, Ch, A0 = L.cpu().numpy(), C.cpu().numpy(), s.A[0].cpu().numpy()
    rng = np.random.default_rng(5)
    nA = np.abs(A0).max()
    for i, j in zip(rng.integers(0, 6144, 10), rng.integers(0, 6144, 10)):
        v = Lh[i] @ Ch @ Lh[j].conj()
        assert abs(v - A0[i, j]) <= 1e-11 * nA * 6144
    r = gevp.solve_sequence(s.A, s.B, s.nev, nex=s.nex, filter_prec="fp32", reduce_slices=8)
    assert r.status == 0, r.stats
    lam = r.Lambda.cpu().numpy()
    assert np.abs(lam[0] - s.lam0[:s.nev]).max() <= 1e-12 * np.abs(s.lam0).max()
    assert r.resid.max().item() <= 1e-10
    X = r.X.cpu().numpy()
    B = s.B.cpu().numpy()
    assert np.abs(X.conj().T @ (B @ X) - np.eye(s.nev)).max() < 1e-9
