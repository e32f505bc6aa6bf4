"""Python binding of libgevp (ctypes over the C ABI in include/gevp.h).

Argument marshalling only: every step runs in the library's CUDA kernels. Tensors must be
CUDA complex128 (or float64 for eigenvalues/residuals); PyTorch supplies device memory and
the current stream. There is no CPU fallback: if the library cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import _build

_LIB = None
_LOCK = threading.Lock()
_HANDLES: dict = {}

STATUS = ["GEVP_OK", "GEVP_ERR_INVALID_ARG", "GEVP_ERR_NOT_HPD", "GEVP_ERR_NO_CONVERGENCE", "GEVP_ERR_CUDA",
          "GEVP_ERR_OOM", "GEVP_ERR_TIMEOUT", "GEVP_ERR_INVALID_VALUE", "GEVP_ERR_UNSUPPORTED"]
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}


class GevpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        self.name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{self.name}: {msg}")


class GevpOpts(C.Structure):
    _fields_ = [("filter_prec", C.c_int), ("tol", C.c_double), ("max_outer", C.c_int), ("deg_min", C.c_int),
                ("deg_max", C.c_int), ("nex", C.c_int), ("seed", C.c_uint64), ("b_fixed", C.c_int),
                ("cold_start", C.c_int), ("lanczos_steps", C.c_int), ("refine_iters", C.c_int),
                ("keep_all_X", C.c_int), ("refresh_window", C.c_int),
                ("reduce_slices", C.c_int)]


class GevpStats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("filter_steps", C.c_int), ("switches", C.c_int),
                ("orth_fallbacks", C.c_int), ("final_passes", C.c_int), ("converged", C.c_int),
                ("matvecs", C.c_int64), ("flops_fp64", C.c_double), ("flops_lowp", C.c_double),
                ("max_resid", C.c_double), ("orth_err", C.c_double), ("cold", C.c_int),
                ("ms_chol", C.c_float), ("ms_reduce", C.c_float), ("ms_bounds", C.c_float),
                ("ms_filter", C.c_float), ("ms_orth", C.c_float), ("ms_rr", C.c_float), ("ms_resid", C.c_float),
                ("ms_final", C.c_float), ("ms_total", C.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class GevpBatchStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("rounds", C.c_int), ("max_rounds_step", C.c_int), ("graph_replays", C.c_int),
                ("switches", C.c_int), ("orth_fallbacks", C.c_int), ("final_passes", C.c_int),
                ("converged", C.c_int), ("tile", C.c_int * 8), ("deg_cap", C.c_int * 8), ("max_resid", C.c_double),
                ("flops_fp64", C.c_double), ("flops_lowp", C.c_double),
                ("ms_chol", C.c_float), ("ms_reduce", C.c_float), ("ms_bounds", C.c_float),
                ("ms_rounds", C.c_float), ("ms_final", C.c_float), ("ms_total", C.c_float)]

    def as_dict(self) -> dict:
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if k in ("tile", "deg_cap") else v
        return d


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgevp.so (building it first if needed). Raises if it cannot be loaded."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.LIB
        if build_if_missing and (not os.path.exists(path) or _build._stale()):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgevp is not built ({path}); run paper_1007_4400_gb300._build.build()")
        L = C.CDLL(path)
        vp, i64, i32, f64 = C.c_void_p, C.c_int64, C.c_int, C.c_double
        L.gevp_create.argtypes = [C.POINTER(vp), i32, vp]
        L.gevp_destroy.argtypes = [vp]
        L.gevp_set_stream.argtypes = [vp, vp]
        L.gevp_status_string.restype = C.c_char_p
        L.gevp_status_string.argtypes = [i32]
        L.gevp_last_error.restype = C.c_char_p
        L.gevp_last_error.argtypes = [vp]
        L.gevp_version.restype = C.c_char_p
        L.gevp_default_opts.argtypes = [C.POINTER(GevpOpts)]
        L.gevp_default_opts.restype = None
        L.gevp_reduce.argtypes = [vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, C.POINTER(i64)]
        L.gevp_solve_sequence.argtypes = [vp, i32, i64, C.POINTER(vp), i64, C.POINTER(vp), i64, i32, vp, i64, i32,
                                          C.POINTER(GevpOpts), vp, vp, i64, vp, C.POINTER(GevpStats)]
        L.gevp_solve_sequence_host.argtypes = [vp, i32, i64, C.POINTER(vp), i64, C.POINTER(vp), i64, i32,
                                               C.POINTER(GevpOpts), vp, vp, i64, vp, C.POINTER(GevpStats)]
        L.gevp_solve_batched.argtypes = [vp, i32, i32, vp, vp, vp, C.POINTER(vp), vp, C.POINTER(vp), vp,
                                         C.POINTER(vp), vp, vp, C.POINTER(GevpOpts), C.POINTER(vp), C.POINTER(vp),
                                         C.POINTER(vp), vp, C.POINTER(GevpBatchStats)]
        L.gevp_chebyshev_filter.argtypes = [vp, i64, vp, i64, vp, i64, i32, i32, f64, f64, f64, i32]
        L.gevp_cholqr2.argtypes = [vp, i64, i32, vp, i64, vp, i64]
        L.gevp_rayleigh_ritz.argtypes = [vp, i64, i32, vp, i64, vp, i64, vp, i64, vp, vp]
        L.gevp_heev_small.argtypes = [vp, i32, vp, i64, vp, vp, i64]
        L.gevp_spectral_bounds.argtypes = [vp, i64, vp, i64, i32, i32, C.POINTER(f64)]
        L.gevp_energy_backward.argtypes = [vp, i64, i32, vp, i64, vp, vp, vp, vp, i64]
        L.gevp_band_energy.argtypes = [vp, i32, i32, vp, vp]
        L.gevp_reduce_update.argtypes = [vp, i64, vp, i64, i32, vp, i64, i32, C.POINTER(i64), vp, i64, i32,
                                         C.POINTER(i64)]
        L.gevp_probe_peaks.argtypes = [vp, C.POINTER(f64)]
        L.gevp_matrix_variation.argtypes = [vp, i64, vp, i64, vp, i64, i32, C.POINTER(f64), C.POINTER(f64),
                                            C.POINTER(i64), vp]
        L.gevp_deviation_angles.argtypes = [vp, i64, i32, i32, vp, i64, vp, i64, vp, i64, C.POINTER(f64),
                                            C.POINTER(f64), f64, vp, i64, C.POINTER(i64), C.POINTER(f64),
                                            C.POINTER(f64), C.POINTER(i64)]
        L.gevp_assign_min_cost.argtypes = [i32, i32, C.POINTER(f64), C.POINTER(i64)]
        L.gevp_zgemm_emulated.argtypes = [vp, i32, i32, i32, i32, i32, vp, i64, vp, i64, vp, i64, i32]
        L.gevp_reduce_emulated.argtypes = [vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, C.POINTER(i64), i32]
        L.gevp_kernel_timing.argtypes = [i32]
        L.gevp_kernel_timing_read.argtypes = [C.POINTER(f64)]
        L.gevp_kernel_launches.argtypes = [vp]
        L.gevp_kernel_launches.restype = i64
        for name in ("gevp_create", "gevp_destroy", "gevp_set_stream", "gevp_reduce", "gevp_solve_sequence",
                     "gevp_solve_sequence_host", "gevp_solve_batched", "gevp_chebyshev_filter", "gevp_cholqr2", "gevp_rayleigh_ritz",
                     "gevp_heev_small", "gevp_spectral_bounds", "gevp_energy_backward", "gevp_band_energy", "gevp_reduce_update",
                     "gevp_probe_peaks",
                     "gevp_matrix_variation", "gevp_deviation_angles", "gevp_assign_min_cost",
                     "gevp_zgemm_emulated", "gevp_reduce_emulated", "gevp_kernel_timing",
                     "gevp_kernel_timing_read"):
            getattr(L, name).restype = i32
        _LIB = L
        return L


def _handle(device: torch.device):
    L = load()
    idx = device.index if device.index is not None else torch.cuda.current_device()
    h = _HANDLES.get(idx)
    if h is None:
        hv = C.c_void_p()
        with torch.cuda.device(idx):
            st = L.gevp_create(C.byref(hv), idx, C.c_void_p(torch.cuda.current_stream().cuda_stream))
        _check(st, None)
        h = hv
        _HANDLES[idx] = h
    with torch.cuda.device(idx):
        L.gevp_set_stream(h, C.c_void_p(torch.cuda.current_stream(idx).cuda_stream))
    return h


def _check(st: int, h) -> None:
    if st != 0:
        msg = load().gevp_last_error(h).decode() if h is not None else ""
        raise GevpError(st, msg)


def _mat(t: torch.Tensor, name: str, dtype=torch.complex128) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() == 2 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major with unit column stride")
    return t


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def default_opts(**kw) -> GevpOpts:
    o = GevpOpts()
    load().gevp_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "filter_prec" and isinstance(v, str):
            v = PREC[v]
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def reduce(A: torch.Tensor, B: torch.Tensor, slices: int = 0):
    """(L, C) with B = L L^H and C = L^-1 A L^-H (see gevp_reduce). slices > 0: the n^3
    products emulated on the tensor cores with that many digits (gevp_reduce_emulated)."""
    _mat(A, "A"); _mat(B, "B")
    n = A.shape[0]
    h = _handle(A.device)
    L_ = torch.empty_like(A)
    C_ = torch.empty_like(A)
    info = C.c_int64(0)
    if slices > 0:
        st = load().gevp_reduce_emulated(h, n, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(L_), n, _ptr(C_),
                                         n, C.byref(info), int(slices))
    else:
        st = load().gevp_reduce(h, n, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(L_), n, _ptr(C_), n,
                                C.byref(info))
    _check(st, h)
    return L_, C_


def zgemm_emulated(A: torch.Tensor, B: torch.Tensor, slices: int = 8, opA: str = "N", opB: str = "C") -> torch.Tensor:
    """op(A) op(B) (complex128; op "N" = X, "C" = X^H) emulated on the tensor cores with
    `slices` 7-bit digits per entry (gevp_zgemm_emulated). The default is A B^H."""
    _mat(A, "A"); _mat(B, "B")
    oa, ob = {"N": 0, "C": 1}[opA], {"N": 0, "C": 1}[opB]
    M, K = (A.shape[1], A.shape[0]) if oa else (A.shape[0], A.shape[1])
    Kb, N = (B.shape[1], B.shape[0]) if ob else (B.shape[0], B.shape[1])
    if Kb != K:
        raise ValueError("op(A) and op(B) do not conform")
    h = _handle(A.device)
    D = torch.empty((M, N), dtype=torch.complex128, device=A.device)
    st = load().gevp_zgemm_emulated(h, oa, ob, M, N, K, _ptr(A), max(A.stride(0), 1), _ptr(B), max(B.stride(0), 1),
                                    _ptr(D), max(N, 1), int(slices))
    _check(st, h)
    return D


@dataclass
class SequenceResult:
    Lambda: torch.Tensor     # (nprob, nev) float64
    X: torch.Tensor          # (n, nev) or (nprob, n, nev) complex128
    resid: torch.Tensor      # (nprob, nev) float64
    stats: list              # per-problem dicts
    status: int


def solve_sequence(A_list, B, nev: int, X_prev=None, keep_all_X: bool = False, check: bool = True, **opts):
    """Solve the sequence A_l x = lambda B_l x (l = 0..len(A_list)-1) for the lowest nev
    pairs with warm starts (gevp_solve_sequence). B: one tensor (fixed) or a list."""
    As = list(A_list)
    Bs = list(B) if isinstance(B, (list, tuple)) else [B] * len(As)
    if len(Bs) != len(As):
        raise ValueError("A_list and B lists differ in length")
    for i, a in enumerate(As):
        _mat(a, f"A[{i}]")
    for i, b in enumerate(Bs):
        _mat(b, f"B[{i}]")
    n = As[0].shape[0]
    lda, ldb = As[0].stride(0), Bs[0].stride(0)
    if any(a.stride(0) != lda or a.shape != (n, n) for a in As) or any(b.stride(0) != ldb for b in Bs):
        raise ValueError("all A (and all B) must share shape and leading dimension")
    dev = As[0].device
    h = _handle(dev)
    nprob = len(As)
    o = default_opts(keep_all_X=1 if keep_all_X else 0, **opts)
    if not isinstance(B, (list, tuple)):
        o.b_fixed = 1
    Lam = torch.empty((nprob, nev), dtype=torch.float64, device=dev)
    res = torch.empty((nprob, nev), dtype=torch.float64, device=dev)
    X = torch.empty(((nprob, n, nev) if keep_all_X else (n, nev)), dtype=torch.complex128, device=dev)
    Ap = (C.c_void_p * nprob)(*[a.data_ptr() for a in As])
    Bp = (C.c_void_p * nprob)(*[b.data_ptr() for b in Bs])
    stats = (GevpStats * nprob)()
    kprev, ldxp = 0, 0
    if X_prev is not None:
        _mat(X_prev, "X_prev")
        kprev, ldxp = X_prev.shape[1], X_prev.stride(0)
    st = load().gevp_solve_sequence(h, nprob, n, Ap, lda, Bp, ldb, nev, _ptr(X_prev), ldxp, kprev, C.byref(o),
                                    _ptr(Lam), _ptr(X), nev, _ptr(res), stats)
    if check and st not in (0, 3):
        _check(st, h)
    return SequenceResult(Lam, X, res, [s.as_dict() for s in stats], st)


def solve_sequence_host(A_list, B, nev: int, keep_all_X: bool = False, device=None, check: bool = True, **opts):
    """gevp_solve_sequence_host: host (CPU, ideally pinned) complex128 inputs and outputs;
    the library copies to and from its device staging inside the call."""
    As = list(A_list)
    Bs = list(B) if isinstance(B, (list, tuple)) else [B] * len(As)
    for t in As + Bs:
        if t.is_cuda or t.dtype != torch.complex128 or t.stride(1) != 1:
            raise TypeError("host entry point takes CPU complex128 row-major tensors")
    n = As[0].shape[0]
    nprob = len(As)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    h = _handle(dev)
    o = default_opts(keep_all_X=1 if keep_all_X else 0, **opts)
    if not isinstance(B, (list, tuple)):
        o.b_fixed = 1
    Lam = torch.empty((nprob, nev), dtype=torch.float64).pin_memory()
    res = torch.empty((nprob, nev), dtype=torch.float64).pin_memory()
    X = torch.empty(((nprob, n, nev) if keep_all_X else (n, nev)), dtype=torch.complex128).pin_memory()
    Ap = (C.c_void_p * nprob)(*[a.data_ptr() for a in As])
    Bp = (C.c_void_p * nprob)(*[b.data_ptr() for b in Bs])
    stats = (GevpStats * nprob)()
    st = load().gevp_solve_sequence_host(h, nprob, n, Ap, As[0].stride(0), Bp, Bs[0].stride(0), nev, C.byref(o),
                                         _ptr(Lam), _ptr(X), nev, _ptr(res), stats)
    if check and st not in (0, 3):
        _check(st, h)
    return SequenceResult(Lam, X, res, [s.as_dict() for s in stats], st)


@dataclass
class BatchedResult:
    Lambda: list             # per k-point (nsteps, nev_k) float64
    resid: list              # per k-point (nsteps, nev_k) float64
    X: list                  # per k-point (n_k, nev_k) or (nsteps, n_k, nev_k) complex128
    stats: dict
    status: int


def solve_batched(A, B, nev, nex=None, X_prev=None, keep_all_X: bool = False, want_X: bool = True,
                  check: bool = True, **opts):
    """gevp_solve_batched: A[k][l] (k-point k, step l) and B[k] CUDA complex128 tensors of
    order n_k; nev (and nex) an int or a per-k-point list. All k-points advance in lock-step
    rounds inside the library; returns per-k-point Lambda, resid and X."""
    nk = len(A)
    nsteps = len(A[0]) if nk else 0
    if len(B) != nk or any(len(a) != nsteps for a in A):
        raise ValueError("A must be nk lists of nsteps tensors and B a list of nk tensors")
    nev_l = [int(nev)] * nk if isinstance(nev, int) else [int(v) for v in nev]
    nex_l = None if nex is None else ([int(nex)] * nk if isinstance(nex, int) else [int(v) for v in nex])
    ns = []
    for k in range(nk):
        _mat(B[k], f"B[{k}]")
        nk_ = B[k].shape[0]
        ns.append(nk_)
        for l in range(nsteps):
            _mat(A[k][l], f"A[{k}][{l}]")
            if A[k][l].shape != (nk_, nk_) or A[k][l].stride(0) != A[k][0].stride(0):
                raise ValueError(f"A[{k}] must be {nk_} x {nk_} with one leading dimension")
    dev = B[0].device
    h = _handle(dev)
    o = default_opts(keep_all_X=1 if keep_all_X else 0, b_fixed=1, **opts)
    i64a = lambda v: (C.c_int64 * nk)(*v)
    i32a = lambda v: (C.c_int * nk)(*v)
    Lam = [torch.empty((nsteps, nev_l[k]), dtype=torch.float64, device=dev) for k in range(nk)]
    res = [torch.empty((nsteps, nev_l[k]), dtype=torch.float64, device=dev) for k in range(nk)]
    Xs = None
    if want_X:
        Xs = [torch.empty(((nsteps, ns[k], nev_l[k]) if keep_all_X else (ns[k], nev_l[k])), dtype=torch.complex128,
                          device=dev) for k in range(nk)]
    Ap = (C.c_void_p * (nk * nsteps))(*[A[k][l].data_ptr() for k in range(nk) for l in range(nsteps)])
    Bp = (C.c_void_p * nk)(*[b.data_ptr() for b in B])
    xp = ldxp = kp = None
    if X_prev is not None:
        for k, x in enumerate(X_prev):
            if x is not None:
                _mat(x, f"X_prev[{k}]")
        xp = (C.c_void_p * nk)(*[(x.data_ptr() if x is not None else 0) for x in X_prev])
        ldxp = i64a([(x.stride(0) if x is not None else 0) for x in X_prev])
        kp = i32a([(x.shape[1] if x is not None else 0) for x in X_prev])
    stats = GevpBatchStats()
    st = load().gevp_solve_batched(
        h, nk, nsteps, i64a(ns), i32a(nev_l), (i32a(nex_l) if nex_l is not None else None), Ap,
        i64a([A[k][0].stride(0) for k in range(nk)]), Bp, i64a([b.stride(0) for b in B]), xp, ldxp, kp, C.byref(o),
        (C.c_void_p * nk)(*[t.data_ptr() for t in Lam]), (C.c_void_p * nk)(*[t.data_ptr() for t in res]),
        ((C.c_void_p * nk)(*[t.data_ptr() for t in Xs]) if Xs is not None else None),
        (i64a([nev_l[k] for k in range(nk)]) if Xs is not None else None), C.byref(stats))
    if check and st not in (0, 3):
        _check(st, h)
    return BatchedResult(Lam, res, Xs, stats.as_dict(), st)


def chebyshev_filter(Cm: torch.Tensor, Y: torch.Tensor, degree: int, lo: float, hi: float, s: float,
                     prec: str = "fp64") -> torch.Tensor:
    """Y <- p(C) Y in place (scaled Chebyshev filter); returns Y."""
    _mat(Cm, "C"); _mat(Y, "Y")
    h = _handle(Cm.device)
    st = load().gevp_chebyshev_filter(h, Cm.shape[0], _ptr(Cm), Cm.stride(0), _ptr(Y), Y.stride(0), Y.shape[1],
                                      int(degree), float(lo), float(hi), float(s), PREC[prec])
    _check(st, h)
    return Y


def cholqr2(Y: torch.Tensor, want_R: bool = False):
    """Q (in place in Y) and optionally R with Y_in = Q R."""
    _mat(Y, "Y")
    h = _handle(Y.device)
    m = Y.shape[1]
    R = torch.zeros((m, m), dtype=torch.complex128, device=Y.device) if want_R else None
    st = load().gevp_cholqr2(h, Y.shape[0], m, _ptr(Y), Y.stride(0), _ptr(R), m if want_R else 0)
    _check(st, h)
    return (Y, R) if want_R else Y


def rayleigh_ritz(Cm: torch.Tensor, Q: torch.Tensor):
    """(theta, Q <- Q Z in place, W = C Q, res)."""
    _mat(Cm, "C"); _mat(Q, "Q")
    h = _handle(Q.device)
    n, m = Q.shape
    W = torch.empty_like(Q)
    th = torch.empty(m, dtype=torch.float64, device=Q.device)
    rs = torch.empty(m, dtype=torch.float64, device=Q.device)
    st = load().gevp_rayleigh_ritz(h, n, m, _ptr(Cm), Cm.stride(0), _ptr(Q), Q.stride(0), _ptr(W), m, _ptr(th),
                                   _ptr(rs))
    _check(st, h)
    return th, Q, W, rs


def heev_small(G: torch.Tensor):
    _mat(G, "G")
    h = _handle(G.device)
    m = G.shape[0]
    th = torch.empty(m, dtype=torch.float64, device=G.device)
    Z = torch.empty_like(G)
    st = load().gevp_heev_small(h, m, _ptr(G), G.stride(0), _ptr(th), _ptr(Z), m)
    _check(st, h)
    return th, Z


def spectral_bounds(Cm: torch.Tensor, k: int = 32, count: int = 0):
    _mat(Cm, "C")
    h = _handle(Cm.device)
    out = (C.c_double * 5)()
    st = load().gevp_spectral_bounds(h, Cm.shape[0], _ptr(Cm), Cm.stride(0), int(k), int(count), out)
    _check(st, h)
    return list(out)


def reduce_update(Cm: torch.Tensor, B: torch.Tensor, dA: torch.Tensor, rows, slices: int = 8,
                  reuse_factor: bool = False) -> torch.Tensor:
    """Cm (in place) <- Cm + L^-1 dA L^-H for a change dA of A confined to the given rows
    and columns (gevp_reduce_update); returns Cm."""
    _mat(Cm, "C"); _mat(B, "B"); _mat(dA, "dA")
    n = Cm.shape[0]
    h = _handle(Cm.device)
    rs = [int(r) for r in rows]
    ra = (C.c_int64 * max(len(rs), 1))(*rs)
    info = C.c_int64(0)
    st = load().gevp_reduce_update(h, n, _ptr(B), B.stride(0), 1 if reuse_factor else 0, _ptr(dA), dA.stride(0),
                                   len(rs), ra, _ptr(Cm), Cm.stride(0), int(slices), C.byref(info))
    _check(st, h)
    return Cm


def energy_backward(X: torch.Tensor, Lambda: torch.Tensor, gE=1.0):
    """(GA, GB) = (gE X X^H, -gE X diag(Lambda) X^H). gE: a number or a one-element float64
    tensor on X's device (read there by the library, no host synchronisation)."""
    _mat(X, "X")
    _mat(Lambda, "Lambda", torch.float64)
    h = _handle(X.device)
    n, nev = X.shape
    if isinstance(gE, torch.Tensor):
        g = gE.detach().to(device=X.device, dtype=torch.float64).reshape(1).contiguous()
    else:
        g = torch.tensor([float(gE)], dtype=torch.float64, device=X.device)
    lam = Lambda.contiguous()
    GA = torch.empty((n, n), dtype=torch.complex128, device=X.device)
    GB = torch.empty_like(GA)
    st = load().gevp_energy_backward(h, n, nev, _ptr(X), X.stride(0), _ptr(lam), _ptr(g), _ptr(GA), _ptr(GB), n)
    _check(st, h)
    return GA, GB


def band_energy_of(Lambda: torch.Tensor) -> torch.Tensor:
    """E[p] = sum of row p of Lambda (nprob x nev, device), computed by the library."""
    _mat(Lambda, "Lambda", torch.float64)
    lam = Lambda.contiguous()
    h = _handle(lam.device)
    nprob, nev = lam.shape
    E = torch.empty((nprob,), dtype=torch.float64, device=lam.device)
    st = load().gevp_band_energy(h, nprob, nev, _ptr(lam), _ptr(E))
    _check(st, h)
    return E


def matrix_variation(A_new: torch.Tensor, A_old: torch.Tensor, thresholds=(0.1,), want_mask: bool = False):
    """(delta, counts, mask) of gevp_matrix_variation: the largest entry variation between
    two consecutive matrices and the number of entries varying by more than p * delta."""
    _mat(A_new, "A_new"); _mat(A_old, "A_old")
    n = A_new.shape[0]
    h = _handle(A_new.device)
    k = len(thresholds)
    p = (C.c_double * max(k, 1))(*[float(x) for x in thresholds])
    delta = C.c_double(0.0)
    counts = (C.c_int64 * max(k, 1))()
    mask = torch.empty((n, n), dtype=torch.uint8, device=A_new.device) if want_mask else None
    st = load().gevp_matrix_variation(h, n, _ptr(A_new), A_new.stride(0), _ptr(A_old), A_old.stride(0), k, p,
                                      C.byref(delta), counts, _ptr(mask))
    _check(st, h)
    return delta.value, [int(counts[i]) for i in range(k)], mask


def deviation_angles(X_old: torch.Tensor, X_new: torch.Tensor, B: torch.Tensor = None, lam_old=None, lam_new=None,
                     window: float = math.inf, reindex: bool = True, want_cosines: bool = False) -> dict:
    """gevp_deviation_angles: the normalised deviation angles (1.00 = pi/2) between the old
    and the new eigenvectors in the B inner product, after re-indexing the new ones against
    the old (reindex=True) or column by column. Returns a dict with perm (None without
    re-indexing), theta, cost, n_outside and cosines (device k_old x k_new, or None)."""
    _mat(X_old, "X_old"); _mat(X_new, "X_new")
    if B is not None:
        _mat(B, "B")
    n, ko = X_old.shape
    kn = X_new.shape[1]
    h = _handle(X_old.device)
    f64p = C.POINTER(C.c_double)
    if math.isfinite(window):
        lo = (C.c_double * max(ko, 1))(*[float(x) for x in lam_old])
        ln = (C.c_double * max(kn, 1))(*[float(x) for x in lam_new])
    else:
        lo = ln = None
    cos = torch.empty((ko, kn), dtype=torch.float64, device=X_old.device) if want_cosines else None
    perm = (C.c_int64 * max(ko, 1))() if reindex else None
    theta = (C.c_double * max(ko, 1))()
    cost = C.c_double(0.0)
    nout = C.c_int64(0)
    st = load().gevp_deviation_angles(h, n, ko, kn, _ptr(X_old), X_old.stride(0), _ptr(X_new), X_new.stride(0),
                                      _ptr(B), B.stride(0) if B is not None else 0, lo, ln, float(window),
                                      _ptr(cos), kn, perm, theta, C.byref(cost), C.byref(nout))
    _check(st, h)
    return {"perm": np.array(perm[:ko], dtype=np.int64) if reindex else None,
            "theta": np.array(theta[:ko]), "cost": cost.value, "n_outside": int(nout.value), "cosines": cos}


def assign_min_cost(cost) -> np.ndarray:
    """gevp_assign_min_cost (host only): the column of each row in the minimum-cost
    assignment of the rows of a ko x kn (ko <= kn) table to distinct columns."""
    c = np.ascontiguousarray(cost, dtype=np.float64)
    ko, kn = c.shape
    perm = np.zeros(max(ko, 1), dtype=np.int64)
    st = load().gevp_assign_min_cost(ko, kn, c.ctypes.data_as(C.POINTER(C.c_double)),
                                     perm.ctypes.data_as(C.POINTER(C.c_int64)))
    if st != 0:
        raise ValueError(f"gevp_assign_min_cost: status {st}")
    return perm[:ko]


def probe_peaks(device=None) -> dict:
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    h = _handle(dev)
    out = (C.c_double * 3)()
    st = load().gevp_probe_peaks(h, out)
    _check(st, h)
    return {"fp64_fma_tflops": out[0], "fp64_dmma_tflops": out[1], "fp32_fma_tflops": out[2]}


def kernel_timing(enable: bool) -> None:
    """Start (clearing earlier records) or stop live timing of the GEMM kernels."""
    st = load().gevp_kernel_timing(1 if enable else 0)
    if st != 0:
        raise GevpError(st, "gevp_kernel_timing")


def kernel_timing_read() -> dict:
    """Per kernel class: launches, total ms, algorithmic and executed flop."""
    out = (C.c_double * 12)()
    st = load().gevp_kernel_timing_read(out)
    if st != 0:
        raise GevpError(st, "gevp_kernel_timing_read")
    names = ("zgemm_kernel", "oz_gemm_kernel", "zgram_kernel")
    return {names[c]: {"launches": int(out[4 * c]), "ms": out[4 * c + 1], "alg_flop": out[4 * c + 2],
                       "exec_flop": out[4 * c + 3]} for c in range(3)}


def kernel_launches(device=None) -> int:
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    return int(load().gevp_kernel_launches(_handle(dev)))


class GevpEnergy(torch.autograd.Function):
    """E = sum of the lowest nev eigenvalues of A x = lambda B x, differentiable in A and B.

    backward: dE/dA = X X^H, dE/dB = -X Lambda X^H (first-order perturbation theory for a
    B-orthonormal X), computed by the library's backward kernel. For complex inputs torch
    expects the conjugate Wirtinger gradient; for Hermitian perturbations the real-valued
    directional derivative is Re tr(G^H dA) with G = X X^H, which is what is returned.
    """

    @staticmethod
    def forward(ctx, A, B, nev, opts):
        r = solve_sequence([A], B, nev, **(opts or {}))
        ctx.save_for_backward(r.X, r.Lambda[0])
        ctx.result = r
        return band_energy_of(r.Lambda[:1])[0]

    @staticmethod
    def backward(ctx, gE):
        X, lam = ctx.saved_tensors
        GA, GB = energy_backward(X, lam, gE)
        return GA, GB, None, None


def band_energy(A, B, nev, **opts):
    return GevpEnergy.apply(A, B, nev, opts)
