"""ctypes front end of the C oracle (``gevp_oracle.c``), on numpy complex128 arrays.

TEST INFRASTRUCTURE ONLY (see the package docstring). Every array is row-major,
interleaved complex128. Functions follow the steps of the plain definition of the
problem the paper poses for each k-point and SCF iteration: A x = lambda B x with A
Hermitian and B Hermitian positive definite, lowest ``nev`` pairs.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_c128p = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = C.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_potrf.argtypes = [_i64, _c128p, _c128p]
        L.orc_potrf.restype = _i64
        L.orc_reduce.argtypes = [_i64, _c128p, _c128p, _c128p]
        L.orc_reduce.restype = None
        L.orc_solve_LH.argtypes = [_i64, _c128p, _c128p, _i64]
        L.orc_solve_LH.restype = None
        L.orc_heev_jacobi.argtypes = [_i64, _c128p, _i64, _f64p, _c128p]
        L.orc_heev_jacobi.restype = C.c_int
        L.orc_heev_tridiag.argtypes = [_i64, _c128p, _i64, _f64p, _c128p]
        L.orc_heev_tridiag.restype = None
        L.orc_solve.argtypes = [_i64, _c128p, _c128p, _i64, C.c_int, _f64p, _c128p]
        L.orc_solve.restype = _i64
        L.orc_residuals.argtypes = [_i64, _c128p, _c128p, _i64, _f64p, _c128p, C.c_double, _f64p]
        L.orc_residuals.restype = None
        L.orc_inertia.argtypes = [_i64, _c128p, _c128p, C.c_double, C.POINTER(_i64)]
        L.orc_inertia.restype = _i64
        L.orc_energy_grad.argtypes = [_i64, _i64, _c128p, _f64p, C.c_double, _c128p, _c128p]
        L.orc_energy_grad.restype = None
        L.orc_eig_extremes.argtypes = [_i64, _c128p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_eig_extremes.restype = None
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _c(a) -> np.ndarray:
    a = np.asarray(a)
    if hasattr(a, "numpy"):
        a = a.numpy()
    return np.ascontiguousarray(a, dtype=np.complex128)


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def potrf(B):
    """Lower Cholesky factor of B; returns (L, info) with info the 1-based failing pivot."""
    B = _c(B)
    n = B.shape[0]
    L = np.zeros_like(B)
    info = lib().orc_potrf(n, B, L)
    return L, int(info)


def reduce(A, L):
    """C = L^-1 A L^-H (Hermitian part)."""
    A, L = _c(A), _c(L)
    n = A.shape[0]
    Cm = np.zeros_like(A)
    lib().orc_reduce(n, A, L, Cm)
    return Cm


def solve_LH(L, Y):
    """X = L^-H Y (back substitution)."""
    L, X = _c(L), _c(Y).copy()
    lib().orc_solve_LH(L.shape[0], L, X, X.shape[1])
    return X


def heev(Cm, nev=None, method="jacobi"):
    """Lowest nev eigenpairs (ascending) of a Hermitian matrix."""
    Cm = _c(Cm)
    n = Cm.shape[0]
    nev = n if nev is None else int(nev)
    lam = np.zeros(nev)
    Y = np.zeros((n, nev), dtype=np.complex128)
    if method == "jacobi":
        lib().orc_heev_jacobi(n, Cm, nev, lam, Y)
    elif method == "tridiag":
        lib().orc_heev_tridiag(n, Cm, nev, lam, Y)
    else:
        raise ValueError(method)
    return lam, Y


def solve(A, B, nev, method="auto"):
    """Lowest nev eigenpairs of the pencil (A, B): lam ascending, X B-orthonormal."""
    A, B = _c(A), _c(B)
    n = A.shape[0]
    if method == "auto":
        method = "jacobi" if n <= 512 else "tridiag"
    lam = np.zeros(int(nev))
    X = np.zeros((n, int(nev)), dtype=np.complex128)
    rc = lib().orc_solve(n, A, B, int(nev), 0 if method == "jacobi" else 1, lam, X)
    if rc < 0:
        raise np.linalg.LinAlgError(f"B is not positive definite (pivot {-rc})")
    return lam, X


def residuals(A, B, lam, X, normA):
    """||A x_i - lam_i B x_i||_2 / (normA ||x_i||_2) per column."""
    A, B, X = _c(A), _c(B), _c(X)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    r = np.zeros(X.shape[1])
    lib().orc_residuals(A.shape[0], A, B, X.shape[1], lam, X, float(normA), r)
    return r


def inertia(A, B, sigma):
    """(number of negative, number of zero) pivots of LDL^H(A - sigma B)."""
    A, B = _c(A), _c(B)
    nz = _i64(0)
    neg = lib().orc_inertia(A.shape[0], A, B, float(sigma), C.byref(nz))
    return int(neg), int(nz.value)


def energy_grad(X, lam, gE=1.0):
    """(dE/dA, dE/dB) = (gE X X^H, -gE X diag(lam) X^H) for E = sum(lam)."""
    X = _c(X)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    n, k = X.shape
    GA = np.zeros((n, n), dtype=np.complex128)
    GB = np.zeros((n, n), dtype=np.complex128)
    lib().orc_energy_grad(n, k, X, lam, float(gE), GA, GB)
    return GA, GB


def eig_extremes(M):
    M = _c(M)
    lo, hi = C.c_double(0), C.c_double(0)
    lib().orc_eig_extremes(M.shape[0], M, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def norm2_hermitian(M) -> float:
    lo, hi = eig_extremes(M)
    return max(abs(lo), abs(hi))


def cpu_info() -> dict:
    import platform
    info = {"cpu_count": os.cpu_count(), "affinity": len(os.sched_getaffinity(0)),
            "machine": platform.machine(), "omp_threads": get_threads()}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    info["model"] = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return info
