"""The tcgen05 BF16 planar three-product filter: exactness on BF16-representable data,
accuracy on random data, the filter polynomial against the FP64 oracle within BF16
tolerance, and the mixed-precision solver against the FP64 oracle at full accuracy."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def T(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _tc_product(cuda, Cm, Y):
    import ctypes as C
    from paper_1007_4400_gb300 import gevp
    L = gevp.load()
    if not hasattr(L, "_mm_set"):
        L.gevp_matmul_tc.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_int64]
        L.gevp_matmul_tc.restype = C.c_int
        L._mm_set = True
    Ct, Yt = T(Cm, cuda), T(Y, cuda)
    D = torch.empty_like(Yt)
    h = gevp._handle(cuda)
    st = L.gevp_matmul_tc(h, Ct.shape[0], Yt.shape[1], C.c_void_p(Ct.data_ptr()), Ct.stride(0),
                          C.c_void_p(Yt.data_ptr()), Yt.stride(0), C.c_void_p(D.data_ptr()), D.stride(0))
    gevp._check(st, h)
    return D.cpu().numpy()


@pytest.mark.parametrize("n,m", [(128, 16), (256, 48), (300, 140), (520, 200), (64, 1)])
def test_tc_product_exact_on_small_integers(cuda, n, m):
    # BF16-exact inputs with FP32-exact sums: the tensor-core product must equal C Y exactly
    rng = np.random.default_rng(900 + n + m)
    Cm = rng.integers(-2, 3, (n, n)) + 1j * rng.integers(-2, 3, (n, n))
    Y = rng.integers(-2, 3, (n, m)) + 1j * rng.integers(-2, 3, (n, m))
    D = _tc_product(cuda, Cm.astype(np.complex128), Y.astype(np.complex128))
    assert np.array_equal(D, Cm @ Y)


def test_tc_product_random_accuracy(cuda):
    rng = np.random.default_rng(901)
    n, m = 1000, 144
    Cm = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Y = (rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m)))
    D = _tc_product(cuda, Cm, Y)
    ref = Cm @ Y
    err = np.linalg.norm(D - ref) / np.linalg.norm(ref)
    assert err < 1e-2


@pytest.mark.parametrize("deg", [1, 4, 12])
def test_tc_filter_vs_oracle(cuda, deg):
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(902 + deg)
    n, m = 384, 40
    lam = np.sort(rng.uniform(-2, 50, n))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Cm = (Q * lam) @ Q.conj().T
    Cm = 0.5 * (Cm + Cm.conj().T)
    Y0 = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    lo, hi, s = 5.0, 50.5, -2.5
    Yg = gevp.chebyshev_filter(T(Cm, cuda), T(Y0, cuda), deg, lo, hi, s, prec="bf16").cpu().numpy()
    Yr = pieces.chebyshev_filter(Cm, Y0, deg, lo, hi, s)
    err = np.linalg.norm(Yg - Yr) / np.linalg.norm(Yr)
    assert err < 5e-2


@pytest.mark.parametrize("deg", [1, 4, 12])
def test_fp32_class_filter_vs_oracle(cuda, deg):
    # three BF16 pieces per operand, six cross products: about FP32 accuracy
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(912 + deg)
    n, m = 384, 40
    lam = np.sort(rng.uniform(-2, 50, n))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Cm = (Q * lam) @ Q.conj().T
    Cm = 0.5 * (Cm + Cm.conj().T)
    Y0 = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    lo, hi, s = 5.0, 50.5, -2.5
    Yg = gevp.chebyshev_filter(T(Cm, cuda), T(Y0, cuda), deg, lo, hi, s, prec="fp32").cpu().numpy()
    Yr = pieces.chebyshev_filter(Cm, Y0, deg, lo, hi, s)
    err = np.linalg.norm(Yg - Yr) / np.linalg.norm(Yr)
    assert err < 2e-5


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_lowp_cold_and_warm_full_accuracy(cuda, orc, prec):
    from paper_1007_4400_gb300 import gevp, synth
    n, nev, nex = 600, 24, 10
    s = synth.make_sequence(1, n, 4, nev, nex, device=cuda)
    r = gevp.solve_sequence(s.A, s.B, nev, nex=nex, filter_prec=prec, keep_all_X=True)
    assert r.status == 0, r.stats
    lam = r.Lambda.cpu().numpy()
    assert np.abs(lam[0] - s.lam0[:nev]).max() <= 1e-12 * np.abs(s.lam0).max()
    assert float(r.resid.max()) <= 1e-10
    for st in r.stats:
        assert st["orth_err"] < 1e-12
    B = s.B.cpu().numpy()
    for l in (1, 3):
        A = s.A[l].cpu().numpy()
        lr, _ = orc.solve(A, B, nev, method="jacobi")
        assert np.abs(lam[l] - lr).max() <= 1e-12 * np.abs(lr).max()


def test_bf16_solver_full_accuracy(cuda, orc):
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.workload("single_n512", device=cuda)
    r = gevp.solve_sequence(s.A, s.B, s.nev, nex=s.nex, cold_start=1, filter_prec="bf16")
    assert r.status == 0, r.stats
    lam = r.Lambda[0].cpu().numpy()
    assert np.abs(lam - s.lam0[:s.nev]).max() <= 1e-12 * np.abs(s.lam0).max()
    assert float(r.resid.max()) <= 1e-10
    assert r.stats[0]["flops_lowp"] > 0
    A, B = s.A[0].cpu().numpy(), s.B.cpu().numpy()
    X = r.X.cpu().numpy()
    assert orc.residuals(A, B, lam, X, orc.norm2_hermitian(A)).max() <= 1e-10


def test_bf16_sequence_matches_fp64(cuda, orc):
    from paper_1007_4400_gb300 import gevp, synth
    n, nev, nex = 400, 20, 8
    s = synth.make_sequence(1, n, 5, nev, nex, device=cuda)
    rb = gevp.solve_sequence(s.A, s.B, nev, nex=nex, filter_prec="bf16")
    rf = gevp.solve_sequence(s.A, s.B, nev, nex=nex)
    assert rb.status == 0 and rf.status == 0
    lb, lf = rb.Lambda.cpu().numpy(), rf.Lambda.cpu().numpy()
    assert np.abs(lb - lf).max() <= 1e-12 * np.abs(lf).max()
    assert float(rb.resid.max()) <= 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_precision_form_full_size(cuda, orc, prec):
    """The precision form at full size: n = 6144, nev = 300, nex = 60, cond(B) ~ 1.3e5, the
    spectrum clustered below a 0.05 gap, the first five problems of the 20-step sequence
    with the FP32-class or BF16 tensor-core filter. Problem 0 against its closed-form
    spectrum; every residual below 1e-10; on the last problem the oracle's residuals of
    the returned eigenvectors and their B-orthonormality."""
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.workload("scf_seq_n6144_cond1e5", device=cuda, nprob=5)
    r = gevp.solve_sequence(s.A, s.B, s.nev, nex=s.nex, filter_prec=prec)
    assert r.status == 0, r.stats
    lam = r.Lambda.cpu().numpy()
    scale = np.abs(s.lam0).max()
    assert np.abs(lam[0] - s.lam0[:s.nev]).max() <= 1e-12 * scale
    assert r.resid.max().item() <= 1e-10
    A = s.A[-1].cpu().numpy()
    B = s.B.cpu().numpy()
    X = r.X.cpu().numpy()
    # the largest column norm bounds ||A||_2 from below, so this check is at least as strict
    # as the definition (the oracle's exact norm needs a full tridiagonalisation here)
    nA = float(np.linalg.norm(A, axis=0).max())
    assert orc.residuals(A, B, lam[-1], X, nA).max() <= 1e-10
    assert np.abs(X.conj().T @ (B @ X) - np.eye(s.nev)).max() < 1e-9
