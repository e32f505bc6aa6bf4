"""The localised update of the standard form (gevp_reduce_update) through the C ABI.

The paper notes that most entries of the Hamiltonian change little between iterations
(Sec. "Matrix generation"). With B fixed, C_new = L^-1 A_new L^-H = C_old + L^-1 dA L^-H, and
a change dA confined to the rows and columns J gives a rank-2|J| update. Checked against the
oracle's full reduction of A_new (the plain definition) element by element, on the FP64
pipe and emulated, with entries of dA outside the rows and columns J filled with garbage
(they must be ignored), the factor reused across calls, and the argument checks."""
import numpy as np
import pytest
import torch

from tests.conftest import crandn, rand_herm, rand_hpd

pytestmark = pytest.mark.gpu


def _localised(rng, n, J):
    """A Hermitian change supported on the rows and columns J, and a copy with garbage
    outside them."""
    D = rand_herm(rng, n)
    mask = np.zeros((n, n), dtype=bool)
    mask[J, :] = True
    mask[:, J] = True
    dA = np.where(mask, D, 0.0)
    garbage = np.where(mask, D, 1e3 * crandn(rng, n, n))
    return dA, garbage


@pytest.mark.parametrize("slices", [0, 8])
@pytest.mark.parametrize("n,k", [(300, 13), (129, 1), (517, 100)])
def test_update_matches_full_reduction(cuda, orc, n, k, slices):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(1300 + n + k)
    A, B = rand_herm(rng, n), rand_hpd(rng, n, 1e3)
    J = np.sort(rng.choice(n, size=k, replace=False))
    dA, dA_garbage = _localised(rng, n, J)
    L, info = orc.potrf(B)
    assert info == 0
    C_old = orc.reduce(A, L)
    want = orc.reduce(A + dA, L)
    Cg = torch.from_numpy(C_old.copy()).to(cuda)
    gevp.reduce_update(Cg, torch.from_numpy(B).to(cuda), torch.from_numpy(dA_garbage).to(cuda), J, slices=slices)
    got = Cg.cpu().numpy()
    assert np.array_equal(got, got.conj().T)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_update_reuses_the_factor(cuda, orc):
    """Two consecutive changes with the factor of the first call reused: the result equals
    the oracle's reduction of the twice-changed matrix."""
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(1401)
    n = 260
    A, B = rand_herm(rng, n), rand_hpd(rng, n, 1e2)
    L, _ = orc.potrf(B)
    J1, J2 = np.array([3, 77, 200]), np.array([5, 77, 140, 259])
    d1, _ = _localised(rng, n, J1)
    d2, _ = _localised(rng, n, J2)
    Bt = torch.from_numpy(B).to(cuda)
    Cg = torch.from_numpy(orc.reduce(A, L)).to(cuda)
    gevp.reduce_update(Cg, Bt, torch.from_numpy(d1).to(cuda), J1)
    gevp.reduce_update(Cg, Bt, torch.from_numpy(d2).to(cuda), J2, reuse_factor=True)
    want = orc.reduce(A + d1 + d2, L)
    assert np.abs(Cg.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()


def test_update_argument_checks(cuda):
    from paper_1007_4400_gb300 import gevp
    n = 50
    rng = np.random.default_rng(1402)
    B = torch.from_numpy(rand_hpd(rng, n)).to(cuda)
    Cg = torch.zeros((n, n), dtype=torch.complex128, device=cuda)
    dA = torch.zeros_like(Cg)
    for bad_rows in ([1, 1], [-1], [n], list(range(11))):   # repeated, out of range, k > n / 5
        with pytest.raises(gevp.GevpError) as e:
            gevp.reduce_update(Cg, B, dA, bad_rows)
        assert e.value.status == 1
    # no rows: C unchanged
    C0 = torch.from_numpy(rand_herm(rng, n)).to(cuda)
    C1 = gevp.reduce_update(C0.clone(), B, dA, [])
    assert torch.equal(C0, C1)


@pytest.mark.slow
def test_update_full_size_against_full_emulated_reduction(cuda):
    """n = 2048 with 64 changed rows and columns: the update from the reduction of A_old
    equals the full (emulated) reduction of A_new, which test_gpu_ozaki pins to the oracle."""
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.make_sequence(1, 2048, 1, 100, 40, device=cuda)
    rng = np.random.default_rng(1403)
    J = np.sort(rng.choice(2048, size=64, replace=False))
    dA, _ = _localised(rng, 2048, J)
    dA = torch.from_numpy(0.01 * dA).to(cuda)
    _, C_old = gevp.reduce(s.A[0], s.B, slices=8)
    _, C_full = gevp.reduce(s.A[0] + dA, s.B, slices=8)
    C_upd = gevp.reduce_update(C_old.clone(), s.B, dA, J, slices=8)
    assert (C_upd - C_full).abs().max().item() <= 1e-12 * C_full.abs().max().item()
