"""End-to-end parity of the sequence solver (C ABI) with the FP64 oracle: eigenvalues,
original-space residuals, B-orthonormality and eigenspace angles, cold and warm starts,
edge cases, and the full-size SCF sequence (sampled problems + properties)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL_RES = 1e-10      # relative residual target
TOL_LAM = 1e-12      # |lambda - lambda*| / max_j |lambda*_j|


def _check_problem(orc, A, B, lam_g, X_g, res_g, nev, method="auto", lam_true=None):
    from oracle import pieces
    lam_r, X_r = orc.solve(A, B, nev, method=method)
    scale = np.abs(lam_r).max() if lam_true is None else np.abs(lam_true).max()
    assert np.abs(lam_g - lam_r).max() <= TOL_LAM * max(scale, np.abs(lam_g).max())
    if lam_true is not None:
        assert np.abs(lam_g - lam_true[:nev]).max() <= TOL_LAM * np.abs(lam_true).max()
    assert res_g.max() <= TOL_RES
    nA = orc.norm2_hermitian(A)
    res_exact = orc.residuals(A, B, lam_g, X_g, nA)
    assert res_exact.max() <= TOL_RES
    assert np.abs(X_g.conj().T @ B @ X_g - np.eye(nev)).max() < 1e-10
    # eigenspace angles per cluster (B inner product)
    gaps = np.diff(lam_r)
    start = 0
    for i in range(nev):
        end_cluster = (i == nev - 1) or gaps[i] > 1e-8 * np.abs(lam_r).max()
        if end_cluster:
            s = pieces.principal_sines(X_g[:, start:i + 1], X_r[:, start:i + 1], B)
            gap = np.abs(np.diff(lam_r[max(0, start - 1):min(nev, i + 2)])).min() if nev > 1 else 1.0
            assert s.max() < max(1e-8, 1e-9 / max(gap, 1e-3))
            start = i + 1


def test_single_problem_n512_cold(cuda, orc):
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.workload("single_n512", device=cuda)
    r = gevp.solve_sequence(s.A, s.B, s.nev, nex=s.nex, cold_start=1)
    assert r.status == 0, r.stats
    _check_problem(orc, s.A[0].cpu().numpy(), s.B.cpu().numpy(), r.Lambda[0].cpu().numpy(),
                   r.X.cpu().numpy(), r.resid[0].cpu().numpy(), s.nev, method="jacobi", lam_true=s.lam0)


def test_sequence_warm_matches_cold_and_saves_work(cuda, orc):
    from paper_1007_4400_gb300 import gevp, synth
    n, nev, nex, nprob = 300, 16, 8, 6
    s = synth.make_sequence(1, n, nprob, nev, nex, device=cuda)
    warm = gevp.solve_sequence(s.A, s.B, nev, nex=nex, keep_all_X=True)
    cold = gevp.solve_sequence(s.A, s.B, nev, nex=nex, cold_start=1)
    assert warm.status == 0 and cold.status == 0
    lw, lc = warm.Lambda.cpu().numpy(), cold.Lambda.cpu().numpy()
    assert np.abs(lw - lc).max() <= TOL_LAM * np.abs(lc).max()
    assert sum(st["matvecs"] for st in warm.stats[1:]) < sum(st["matvecs"] for st in cold.stats[1:])
    B = s.B.cpu().numpy()
    for l in range(nprob):
        _check_problem(orc, s.A[l].cpu().numpy(), B, lw[l], warm.X[l].cpu().numpy(),
                       warm.resid[l].cpu().numpy(), nev, method="jacobi",
                       lam_true=s.lam0 if l == 0 else None)


@pytest.mark.parametrize("n,nev,nex", [(2, 1, 1), (37, 5, 3), (130, 33, 0), (65, 64, 1)])
def test_edge_sizes(cuda, orc, n, nev, nex):
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.make_sequence(0, n, 2, nev, nex, device=cuda)
    r = gevp.solve_sequence(s.A, s.B, nev, nex=nex, keep_all_X=True)
    assert r.status == 0, r.stats
    for l in range(2):
        _check_problem(orc, s.A[l].cpu().numpy(), s.B.cpu().numpy(), r.Lambda[l].cpu().numpy(),
                       r.X[l].cpu().numpy(), r.resid[l].cpu().numpy(), nev, method="jacobi")


def test_changing_B_warm_start(cuda, orc):
    # B differs per problem: the Cholesky factor is recomputed and the warm start maps
    # the previous eigenvectors through the new factor
    from paper_1007_4400_gb300 import gevp, synth
    n, nev, nex = 200, 10, 6
    s0 = synth.make_sequence(0, n, 1, nev, nex, device=cuda)
    s1 = synth.make_sequence(0, n, 1, nev, nex, device=cuda, problem_index=1)
    As = [s0.A[0], s0.A[0] + 0.01 * s1.A[0] / s1.A[0].abs().max()]
    As[1] = 0.5 * (As[1] + As[1].conj().T)
    Bs = [s0.B, s0.B + 0.01 * torch.eye(n, dtype=torch.complex128, device=cuda)]
    r = gevp.solve_sequence(As, Bs, nev, nex=nex, keep_all_X=True)
    assert r.status == 0
    for l in range(2):
        _check_problem(orc, As[l].cpu().numpy(), Bs[l].cpu().numpy(), r.Lambda[l].cpu().numpy(),
                       r.X[l].cpu().numpy(), r.resid[l].cpu().numpy(), nev, method="jacobi")


def test_seed_with_exact_eigenvectors(cuda, orc):
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.make_sequence(0, 256, 1, 12, 6, device=cuda)
    A, B = s.A[0].cpu().numpy(), s.B.cpu().numpy()
    lam, X = orc.solve(A, B, 18, method="jacobi")
    r = gevp.solve_sequence(s.A, s.B, 12, nex=6, X_prev=torch.from_numpy(X).to(cuda))
    assert r.status == 0
    assert r.stats[0]["outer_iters"] <= 1
    assert np.abs(r.Lambda[0].cpu().numpy() - lam[:12]).max() <= TOL_LAM * np.abs(lam).max()


def test_errors_not_hpd_and_nan(cuda):
    from paper_1007_4400_gb300 import gevp
    n = 40
    A = torch.eye(n, dtype=torch.complex128, device=cuda)
    Bbad = torch.eye(n, dtype=torch.complex128, device=cuda)
    Bbad[5, 5] = -1.0
    with pytest.raises(gevp.GevpError) as e:
        gevp.solve_sequence([A], Bbad, 4, nex=2)
    assert e.value.status == 2
    An = A.clone()
    An[3, 7] = float("nan")
    with pytest.raises(gevp.GevpError) as e:
        gevp.solve_sequence([An], A, 4, nex=2)
    assert e.value.status == 7


@pytest.mark.slow
def test_full_size_scf_sequence_n2048(cuda, orc):
    """The benchmark workload in its bench configuration: 20 problems, n = 2048,
    nev = 100, nex = 40, warm start. Problem 0 against its closed-form spectrum,
    every problem's residual and B-orthonormality, the oracle's full solve on problems
    {1, last}, and Sylvester inertia (no missed eigenvalue) on problems {7, last}."""
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.workload("scf_seq_n2048", device=cuda)
    r = gevp.solve_sequence(s.A, s.B, s.nev, nex=s.nex, keep_all_X=True)
    assert r.status == 0
    lam = r.Lambda.cpu().numpy()
    res = r.resid.cpu().numpy()
    assert res.max() <= TOL_RES
    assert np.abs(lam[0] - s.lam0[:s.nev]).max() <= TOL_LAM * np.abs(s.lam0).max()
    B = s.B.cpu().numpy()
    last = len(s.A) - 1
    for l in range(len(s.A)):
        X = r.X[l].cpu().numpy()
        assert np.abs(X.conj().T @ B @ X - np.eye(s.nev)).max() < 1e-9
    for l in (1, last):
        A = s.A[l].cpu().numpy()
        lam_r, _ = orc.solve(A, B, s.nev, method="tridiag")
        assert np.abs(lam[l] - lam_r).max() <= TOL_LAM * np.abs(lam_r).max() * 1.0 + 1e-12 * 50
    for l in (7, last):
        A = s.A[l].cpu().numpy()
        sig = 0.5 * (lam[l][-1] + lam[l][-1] + 0.0)
        # a point between lambda_nev and the next eigenvalue: use the (nev+1)-th from the oracle
        lam_r, _ = orc.solve(A, B, s.nev + 1, method="tridiag")
        sig = 0.5 * (lam_r[s.nev - 1] + lam_r[s.nev])
        neg, zero = orc.inertia(A, B, sig)
        assert zero == 0 and neg == s.nev
        assert lam[l][-1] < sig


def test_host_entry_point_matches_device(cuda):
    from paper_1007_4400_gb300 import gevp, synth
    s = synth.make_sequence(1, 256, 3, 12, 6, device="cpu")
    rd = gevp.solve_sequence([a.to(cuda) for a in s.A], s.B.to(cuda), 12, nex=6)
    rh = gevp.solve_sequence_host([a.pin_memory() for a in s.A], s.B.pin_memory(), 12, nex=6)
    assert rh.status == 0
    assert torch.equal(rh.Lambda, rd.Lambda.cpu())
    assert torch.equal(rh.resid, rd.resid.cpu())
    assert torch.equal(rh.X, rd.X.cpu())


def _refresh_rule_holds(stats, window):
    """Replays the refresh rule on the per-problem counters: after `window` consecutive warm
    problems with at least the matvecs of the latest cold one, the next problem is cold."""
    cold_mv, flat, refresh = -1, 0, False
    for i, st in enumerate(stats):
        if i > 0 and st["cold"] != (1 if refresh else 0):
            return False
        if st["cold"]:
            cold_mv, flat, refresh = st["matvecs"], 0, False
        elif cold_mv >= 0 and st["matvecs"] >= cold_mv:
            flat += 1
            refresh = flat >= window
        else:
            flat = 0
    return True


@pytest.mark.parametrize("eps0,decay", [(0.1, 0.6), (40.0, 1.0)])
def test_refresh_policy(cuda, orc, eps0, decay):
    """The slowly drifting SCF sequence never refreshes (every warm start saves work); a
    sequence of unrelated problems (drift as large as the spectrum) follows the rule, and
    every problem is solved to tolerance either way."""
    from paper_1007_4400_gb300 import gevp, synth
    n, nev, nex = 300, 16, 8
    s = synth.make_sequence(1, n, 6, nev, nex, device=cuda, eps0=eps0, decay=decay)
    r = gevp.solve_sequence(s.A, s.B, nev, nex=nex, refresh_window=1, keep_all_X=True)
    assert r.status == 0
    assert r.stats[0]["cold"] == 1
    assert _refresh_rule_holds(r.stats, 1)
    if eps0 < 1:
        assert [st["cold"] for st in r.stats] == [1, 0, 0, 0, 0, 0]
    B = s.B.cpu().numpy()
    for l in (1, 5):
        _check_problem(orc, s.A[l].cpu().numpy(), B, r.Lambda[l].cpu().numpy(), r.X[l].cpu().numpy(),
                       r.resid[l].cpu().numpy(), nev, method="jacobi")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cholqr_breakdown_inside_the_rounds(cuda, orc, prec):
    """A spectrum with one cluster of wanted values far below a single, highly degenerate
    unwanted value: the filter drives the whole block towards the 4-dimensional wanted
    space, the Gram matrix of the filtered block is numerically singular, and the plain
    CholQR pass inside a round fails. The solver must notice it (the status of the pass is
    read with the round's Ritz values), repeat the orthonormalisation with the shifted
    fallback, and still return the oracle's eigenpairs."""
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(881)
    n, nev, nex = 64, 4, 4
    lam = np.concatenate([[-2.0, -1.9, -1.8, -1.7], np.full(n - 4, 50.0)])
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * (np.diag(R) / np.abs(np.diag(R)))
    L = np.tril(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), -1) * (0.3 / np.sqrt(n))
    L = L + np.diag(rng.uniform(0.5, 2.0, n))
    B = L @ L.conj().T
    B = 0.5 * (B + B.conj().T)
    A = L @ (Q * lam) @ Q.conj().T @ L.conj().T
    A = 0.5 * (A + A.conj().T)
    r = gevp.solve_sequence([torch.from_numpy(A).to(cuda)], torch.from_numpy(B).to(cuda), nev, nex=nex,
                            cold_start=1, filter_prec=prec, deg_min=24)
    assert r.status == 0, r.stats
    if prec == "fp64":
        # the FP64 filter drives the block to numerical rank deficiency; the FP32-class
        # filter's own rounding keeps it just above (the same spectrum, no fallback needed)
        assert r.stats[0]["orth_fallbacks"] > 0
    _check_problem(orc, A, B, r.Lambda[0].cpu().numpy(), r.X.cpu().numpy(), r.resid[0].cpu().numpy(), nev,
                   method="jacobi", lam_true=lam)
