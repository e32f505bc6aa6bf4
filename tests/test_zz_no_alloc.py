"""The allocation-free FP64 Chebyshev filter (gevp_chebyshev_filter_noalloc) through the C
ABI, against the oracle's scaled Chebyshev recurrence and against the handle-based
gevp_chebyshev_filter, on consecutive calls.

This entry point exists for callers that must not allocate device memory when they call
it: applications whose device memory is owned by a pool allocator (a library cudaMalloc
would bypass the pool, can fail while the pool holds the free memory, and synchronises the
device) and services with a fixed memory budget. Its scratch is a fixed device array in
the library, shared by every call and keeping the previous call's contents, so the calls
below run back to back with different sizes (the second smaller than the first, then a
degree-1 call and a call with padded leading dimensions) to show that nothing of one call
leaks into the next. Collected last (file name) so that a failure here cannot hide another
test's failure in a run that stops at the first failure."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(L, stream, Cm, Y, deg, lo, hi, s, n=None, m=None):
    f = L.gevp_chebyshev_filter_noalloc
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                  C.c_double, C.c_double, C.c_double]
    f.restype = C.c_int
    n = Cm.shape[0] if n is None else n
    m = Y.shape[1] if m is None else m
    return f(C.c_void_p(stream), n, C.c_void_p(Cm.data_ptr()), Cm.stride(0), C.c_void_p(Y.data_ptr()),
             Y.stride(0), m, deg, lo, hi, s)


def _problem(rng, n):
    lam = np.sort(rng.uniform(-2, 50, n))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Cm = (Q * lam) @ Q.conj().T
    return 0.5 * (Cm + Cm.conj().T)


def test_noalloc_filter_matches_oracle_and_handle_filter():
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    dev = torch.device("cuda", 0)
    L = gevp.load()
    stream = torch.cuda.current_stream(dev).cuda_stream
    rng = np.random.default_rng(77)
    lo, hi, s = 5.0, 50.5, -2.5
    # (n, m, degree, extra leading-dimension padding of C, of Y)
    cases = [(517, 40, 12, 0, 0), (300, 24, 7, 0, 0), (211, 9, 1, 0, 0), (260, 17, 5, 13, 6)]
    for call, (n, m, deg, padc, pady) in enumerate(cases):
        Cn = _problem(rng, n)
        Y0n = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
        want = pieces.chebyshev_filter(Cn, Y0n, deg, lo, hi, s)
        Cbuf = torch.zeros((n, n + padc), dtype=torch.complex128, device=dev)
        Cbuf[:, :n] = torch.from_numpy(Cn).to(dev)
        Ybuf = torch.full((n, m + pady), 7.0 + 7.0j, dtype=torch.complex128, device=dev)
        Ybuf[:, :m] = torch.from_numpy(Y0n).to(dev)
        st = _noalloc(L, stream, Cbuf, Ybuf, deg, lo, hi, s, n=n, m=m)
        torch.cuda.synchronize()
        assert st == 0, f"call {call}: status {st}"
        got = Ybuf[:, :m].cpu().numpy()
        # oracle: the recurrence's products round differently; the bound is FP64 rounding
        # of the degree-deg recurrence relative to the block's size
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 1e-12, f"call {call}: relative difference to the oracle {err:.2e}"
        # padding columns of Y are left alone
        if pady:
            assert bool((Ybuf[:, m:] == 7.0 + 7.0j).all())
        ref = gevp.chebyshev_filter(Cbuf[:, :n].contiguous(), torch.from_numpy(Y0n).to(dev), deg, lo, hi, s,
                                    prec="fp64")
        err2 = (Ybuf[:, :m] - ref).abs().max().item() / ref.abs().max().item()
        assert err2 < 1e-12, f"call {call}: relative difference to gevp_chebyshev_filter {err2:.2e}"


def test_noalloc_filter_rejects_oversize():
    from paper_1007_4400_gb300 import gevp
    dev = torch.device("cuda", 0)
    L = gevp.load()
    n, m = 4096, 300          # 2 n m > 2^21 complex128 of fixed scratch
    Cm = torch.zeros((8, 8), dtype=torch.complex128, device=dev)
    Y = torch.zeros((8, 8), dtype=torch.complex128, device=dev)
    f = L.gevp_chebyshev_filter_noalloc
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                  C.c_double, C.c_double, C.c_double]
    f.restype = C.c_int
    st = f(None, n, C.c_void_p(Cm.data_ptr()), n, C.c_void_p(Y.data_ptr()), m, m, 3, 5.0, 50.0, -2.0)
    assert st == 1   # GEVP_ERR_INVALID_ARG, nothing enqueued
