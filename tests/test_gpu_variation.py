"""Parity of the matrix-variation kernel (gevp_matrix_variation) with the oracle's
definition: the largest entry variation and the counts above p * delta must agree exactly
(integer results, and the FP64 arithmetic of the comparison is fixed by the definition)."""
import numpy as np
import pytest
import torch

from tests.conftest import crandn

pytestmark = pytest.mark.gpu

PS = [0.1, 0.0, 0.01, 0.05, 0.2, 0.5, 0.99, 1.0]


def _check(A_new, A_old, cuda, ps=PS, ld_pad=0):
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    n = A_new.shape[0]
    def dev(M):
        if ld_pad:
            big = torch.zeros((n, n + ld_pad), dtype=torch.complex128, device=cuda)
            big[:, :n] = torch.from_numpy(M).to(cuda)
            return big[:, :n]
        return torch.from_numpy(np.ascontiguousarray(M)).to(cuda)
    d, c, mask = gevp.matrix_variation(dev(A_new), dev(A_old), ps, want_mask=True)
    dr, cr, mr = pieces.matrix_variation(A_new, A_old, ps)
    assert d == dr
    assert c == cr
    assert np.array_equal(mask.cpu().numpy().astype(bool), mr)


def test_hand_case_exact(cuda):
    A_old = np.zeros((4, 4), dtype=np.complex128)
    A_new = A_old.copy()
    A_new[0, 1], A_new[1, 0] = 3 + 4j, 3 - 4j
    A_new[2, 2] = 1.0
    A_new[3, 0], A_new[0, 3] = 0.5, 0.5
    A_new[1, 3], A_new[3, 1] = 0.25j, -0.25j
    _check(A_new, A_old, cuda)


@pytest.mark.parametrize("n,pad", [(1, 0), (2, 0), (37, 3), (300, 0), (1023, 5)])
def test_sequence_differences(cuda, n, pad):
    from paper_1007_4400_gb300 import synth
    s = synth.make_sequence(1, n, 3, max(1, n // 20), 2)
    for l in range(2):
        _check(s.A[l + 1].numpy(), s.A[l].numpy(), cuda, ld_pad=pad)


def test_structured_difference_with_ties(cuda):
    # a difference with many equal moduli (ties at every threshold) and unchanged blocks
    rng = np.random.default_rng(7)
    n = 257
    A = crandn(rng, n, n)
    A = A + A.conj().T
    D = np.zeros_like(A)
    D[:40, :40] = 0.5 * (1 + 1j)
    D[100:, 100:] = (rng.integers(-4, 5, (n - 100, n - 100)) + 1j * rng.integers(-4, 5, (n - 100, n - 100))) / 8
    D = D + D.conj().T
    _check(A + D, A, cuda, ps=[0.1, 0.25, 0.5, 0.7071067811865476, 1.0])


def test_full_size_bench_sequence(cuda):
    """The consecutive Hamiltonians of the n = 2048 benchmark sequence."""
    from paper_1007_4400_gb300 import synth
    s = synth.workload("scf_seq_n2048", nprob=3)
    for l in range(2):
        _check(s.A[l + 1].numpy(), s.A[l].numpy(), cuda)


def test_nan_and_errors(cuda):
    from paper_1007_4400_gb300 import gevp
    A = torch.eye(16, dtype=torch.complex128, device=cuda)
    B = A.clone()
    B[3, 4] = float("nan")
    with pytest.raises(gevp.GevpError) as e:
        gevp.matrix_variation(B, A, [0.1])
    assert e.value.status == 7
    with pytest.raises(gevp.GevpError) as e:
        gevp.matrix_variation(A, A, [0.1] * 17)
    assert e.value.status == 1
    d, c, _ = gevp.matrix_variation(A, A, [0.0, 0.5])
    assert d == 0.0 and c == [0, 0]
