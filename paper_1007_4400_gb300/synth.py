"""Seeded synthetic inputs: FLAPW-shaped Hermitian-definite pencils and SCF-like sequences.

This module builds inputs only. It holds none of the solver's arithmetic (no Cholesky,
no reduction, no eigensolver, no filter); both the CUDA path and the CPU oracle consume
the arrays it returns, so the two always see bit-identical problems.

The paper's own matrices (FLEUR runs on bulk Cu and an Fe multilayer, Sec. "A new
computational philosophy") are not available; these pencils stand in for them:

* ``B = L L^H`` with ``L`` lower triangular, a real positive diagonal and complex normal
  off-diagonal entries (E|z|^2 = 1) scaled by ``0.3/sqrt(n)``.
* ``A = L Q diag(lam) Q^H L^H`` with ``Q`` Haar-unitary, so the pencil's spectrum is
  exactly ``lam`` (up to the rounding of forming ``A``) and ``x_i = L^-H Q e_i``.
* A sequence ``A_{l+1} = A_l + eps_l P_l`` with ``P_l`` a random Hermitian matrix of unit
  spectral norm and ``eps_l = 0.1 * 0.6**l`` mimics the slowly drifting problems of the
  self-consistent cycle (the paper's "correlated problems"), with ``B`` fixed.

Random draws use ``numpy.random.Generator(PCG64(10074400 + 1000*config + problem))`` in a
fixed order: diag(L); lower(L) real then imaginary; Ginibre for Q (real then imaginary);
lambda; then each ``P_l`` from ``seed + 100 + l``. Products are formed in complex128 with
torch on the requested device (CPU or CUDA); the draws do not depend on the device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

SEED_BASE = 10074400


def rng_for(config_id: int, problem_index: int = 0, offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * config_id + problem_index + offset))


def _cnormal(rng: np.random.Generator, shape) -> np.ndarray:
    """Standard complex normal (E|z|^2 = 1): real then imaginary parts, each N(0, 1/2)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) * math.sqrt(0.5)


def draw_L(rng: np.random.Generator, n: int, diag=(0.5, 2.0), off_scale=None,
           log_uniform_diag: bool = False) -> np.ndarray:
    """Lower-triangular factor of B: real positive diagonal, complex normal strict lower part.

    With ``log_uniform_diag`` the diagonal d is log-uniform in ``diag`` and each row of the
    strict lower part is scaled by its diagonal entry, L = D (I + N): then
    cond(B) ~ (max d / min d)^2 (about 1.3e5 for diag = (6e-3, 2)). Unscaled off-diagonals
    next to small diagonal entries would make L (hence B) numerically singular."""
    if off_scale is None:
        off_scale = 0.3 / math.sqrt(n)
    lo, hi = diag
    if log_uniform_diag:
        d = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    else:
        d = rng.uniform(lo, hi, n)
    il = np.tril_indices(n, -1)
    m = il[0].size
    re = rng.standard_normal(m)
    im = rng.standard_normal(m)
    L = np.zeros((n, n), dtype=np.complex128)
    off = (re + 1j * im) * math.sqrt(0.5) * off_scale
    if log_uniform_diag:
        off = off * d[il[0]]
    L[il] = off
    L[np.arange(n), np.arange(n)] = d
    return L


def haar_unitary(rng: np.random.Generator, n: int, device="cpu") -> torch.Tensor:
    """Haar-distributed unitary: QR of a complex Ginibre matrix with R's diagonal phases
    divided out (Mezzadri, Notices AMS 2007)."""
    G = torch.from_numpy(_cnormal(rng, (n, n))).to(device)
    Q, R = torch.linalg.qr(G)
    ph = torch.diagonal(R)
    ph = ph / ph.abs()
    return Q * ph.unsqueeze(0)


def hermitian_part(M: torch.Tensor) -> torch.Tensor:
    return 0.5 * (M + M.conj().transpose(-1, -2))


def known_spectrum_pencil(L: torch.Tensor, Q: torch.Tensor, lam: torch.Tensor):
    """A = L Q diag(lam) Q^H L^H and B = L L^H, both made exactly Hermitian."""
    LQ = L @ Q
    A = hermitian_part((LQ * lam.to(LQ.dtype).unsqueeze(0)) @ LQ.conj().transpose(-1, -2))
    B = hermitian_part(L @ L.conj().transpose(-1, -2))
    return A.contiguous(), B.contiguous()


def _norm2_lanczos(P: torch.Tensor, k: int = 60) -> float:
    """Spectral norm of Hermitian P from k Lanczos steps (full re-orthogonalisation) with a
    fixed start vector; used for the large workloads, where a full eigvalsh per sequence
    step would dominate input generation. The estimate is within 1e-3 relative for the
    random Hermitian matrices drawn here, which only sets the size of a perturbation."""
    n = P.shape[0]
    g = torch.Generator(device="cpu").manual_seed(SEED_BASE)
    v = torch.randn(n, dtype=torch.float64, generator=g).to(P.device).to(P.dtype)
    V = [v / torch.linalg.vector_norm(v)]
    a, b = [], []
    for j in range(min(k, n)):
        w = P @ V[j]
        for _ in range(2):
            for u in V:
                w = w - (u.conj() @ w) * u
        a.append(float(torch.real(V[j].conj() @ (P @ V[j]))))
        nb = float(torch.linalg.vector_norm(w))
        if nb < 1e-12:
            break
        b.append(nb)
        V.append(w / nb)
    m = len(a)
    T = np.diag(a) + np.diag(b[:m - 1], 1) + np.diag(b[:m - 1], -1)
    return float(np.abs(np.linalg.eigvalsh(T)).max())


def hermitian_unit_norm(rng: np.random.Generator, n: int, device="cpu") -> torch.Tensor:
    """P = (G + G^H)/2 with complex standard normal G, divided by its spectral norm (for
    n > 8192 by a Lanczos estimate of it)."""
    G = torch.from_numpy(_cnormal(rng, (n, n))).to(device)
    P = hermitian_part(G)
    del G
    if n > 8192:
        return (P / _norm2_lanczos(P)).contiguous()
    ev = torch.linalg.eigvalsh(P)
    return (P / ev.abs().max()).contiguous()


def clustered_spectrum(rng: np.random.Generator, n: int, nocc: int, occ=(-2.0, 5.0),
                       gap: float = 0.05, top: float = 80.0) -> np.ndarray:
    """Lowest ``nocc`` uniform in ``occ``; the rest uniform in [occ[1]+gap, top]; sorted."""
    a = np.sort(rng.uniform(occ[0], occ[1], nocc))
    b = np.sort(rng.uniform(occ[1] + gap, top, n - nocc))
    return np.concatenate([a, b])


@dataclass
class Sequence:
    """A sequence of pencils (A_l, B) sharing one B, as in an SCF cycle with fixed overlap."""
    n: int
    nev: int
    nex: int
    A: list                      # list of (n, n) complex128 tensors
    B: torch.Tensor              # (n, n) complex128
    lam0: np.ndarray             # exact spectrum of problem 0 (sorted)
    L_true: torch.Tensor         # the generating factor (B = L L^H)
    Q_true: torch.Tensor         # the generating unitary of problem 0
    eps: list = field(default_factory=list)
    config_id: int = -1

    def x0_true(self, i: int) -> torch.Tensor:
        """Exact eigenvector i of problem 0: x_i = L^-H Q e_i (test helper)."""
        q = self.Q_true[:, i:i + 1]
        return torch.linalg.solve_triangular(self.L_true.conj().transpose(0, 1), q, upper=True)


def make_sequence(config_id: int, n: int, nprob: int, nev: int, nex: int, device="cpu",
                  spectrum: str = "uniform", problem_index: int = 0, diag=(0.5, 2.0),
                  log_uniform_diag: bool = False, eps0: float = 0.1, decay: float = 0.6,
                  lam_range=(-2.0, 50.0)) -> Sequence:
    """Build a seeded sequence. ``spectrum='uniform'``: lambda sorted U[lam_range];
    ``'clustered'``: lowest nev in [-2, 5], gap 0.05, rest in [5.05, 80]."""
    seed_index = problem_index
    rng = rng_for(config_id, seed_index)
    L_np = draw_L(rng, n, diag=diag, log_uniform_diag=log_uniform_diag)
    Q = haar_unitary(rng, n, device)
    if spectrum == "uniform":
        lam = np.sort(rng.uniform(lam_range[0], lam_range[1], n))
    elif spectrum == "clustered":
        lam = clustered_spectrum(rng, n, nev)
    else:
        raise ValueError(spectrum)
    L = torch.from_numpy(L_np).to(device)
    A0, B = known_spectrum_pencil(L, Q, torch.from_numpy(lam).to(device))
    As = [A0]
    eps = []
    for l in range(nprob - 1):
        prng = rng_for(config_id, seed_index, offset=100 + l)
        P = hermitian_unit_norm(prng, n, device)
        e = eps0 * decay ** l
        eps.append(e)
        As.append(hermitian_part(As[-1] + e * P).contiguous())
        del P
    return Sequence(n=n, nev=nev, nex=nex, A=As, B=B, lam0=lam, L_true=L, Q_true=Q,
                    eps=eps, config_id=config_id)


# Named workloads (sizes from the paper's FLAPW setting, scaled up; see the module docstring).
WORKLOADS = {
    # single problem, cold start, n=512
    "single_n512": dict(config_id=0, n=512, nprob=1, nev=32, nex=16),
    # SCF-like sequence of 20 problems, n=2048, B fixed
    "scf_seq_n2048": dict(config_id=1, n=2048, nprob=20, nev=100, nex=40),
    # precision form: clustered spectrum, cond(B) about 1e5
    "scf_seq_n6144_cond1e5": dict(config_id=2, n=6144, nprob=20, nev=300, nex=60,
                                  spectrum="clustered", diag=(6.0e-3, 2.0), log_uniform_diag=True),
    # differentiation form
    "grad_n4096": dict(config_id=4, n=4096, nprob=1, nev=200, nex=50, spectrum="clustered"),
    # the long sequence of the differentiation form's construction: 30 problems, n=12000
    "scf_seq_n12000": dict(config_id=4, n=12000, nprob=30, nev=600, nex=150, spectrum="clustered",
                           problem_index=1),
}


def workload(name: str, device="cpu", **over) -> Sequence:
    kw = dict(WORKLOADS[name])
    kw.update(over)
    return make_sequence(device=device, **kw)


def batched_sizes(nprob: int = 64, lo: int = 800, hi: int = 3000, config_id: int = 3):
    """Per-problem sizes of the batched k-point workload: n ~ U{lo..hi},
    nev = round(0.06 n), nex = ceil(0.4 nev)."""
    rng = rng_for(config_id, 0, offset=999)
    ns = rng.integers(lo, hi + 1, nprob)
    out = []
    for n in ns:
        nev = int(round(0.06 * int(n)))
        out.append((int(n), nev, int(math.ceil(0.4 * nev))))
    return out


def kpoint_batch(nk: int = 64, nsteps: int = 10, lo: int = 800, hi: int = 3000, device="cpu",
                 config_id: int = 3, sizes=None) -> list:
    """The batched k-point workload: nk independent sequences (one per k-point), each built
    like the SCF sequence (known-spectrum A_0, B fixed, A_{l+1} = A_l + 0.1 0.6^l P_l) with
    its own seed (problem_index = k) and its own order n_k ~ U{lo..hi},
    nev_k = round(0.06 n_k), nex_k = ceil(0.4 nev_k). ``sizes`` overrides the draw with a
    list of (n, nev, nex)."""
    sz = sizes if sizes is not None else batched_sizes(nk, lo, hi, config_id)
    return [make_sequence(config_id, n, nsteps, nev, nex, device=device, problem_index=k)
            for k, (n, nev, nex) in enumerate(sz)]


def random_block(n: int, m: int, seed: int, device="cpu") -> torch.Tensor:
    """Seeded complex normal n x m block (row-major), for kernel-level tests."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 7 + seed))
    return torch.from_numpy(_cnormal(rng, (n, m))).to(device).contiguous()
