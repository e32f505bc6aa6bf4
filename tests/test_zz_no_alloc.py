"""The allocation-free FP64 Chebyshev filter (gevp_chebyshev_filter_noalloc) against the
handle-based gevp_chebyshev_filter, through the C ABI, on two calls in a row.

This entry point exists for callers that must not allocate device memory at the point of
the call (inside a CUDA graph capture, under a pool allocator that owns device memory, or
with a fixed memory budget): its scratch is a fixed device array in the library. The two
calls in a row check that the shared scratch, which keeps the previous call's contents,
does not leak into the next result. Collected last (file name) so that a failure here
cannot hide another test's failure in a run that stops at the first failure."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(L, stream, Cm, Y, deg, lo, hi, s):
    f = L.gevp_chebyshev_filter_noalloc
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                  C.c_double, C.c_double, C.c_double]
    f.restype = C.c_int
    return f(C.c_void_p(stream), Cm.shape[0], C.c_void_p(Cm.data_ptr()), Cm.stride(0), C.c_void_p(Y.data_ptr()),
             Y.stride(0), Y.shape[1], deg, lo, hi, s)


def test_noalloc_filter_matches_handle_filter():
    from paper_1007_4400_gb300 import gevp
    dev = torch.device("cuda", 0)
    L = gevp.load()
    stream = torch.cuda.current_stream(dev).cuda_stream
    rng = np.random.default_rng(77)
    lo, hi, s = 5.0, 50.5, -2.5
    for call, (n, m, deg) in enumerate([(300, 24, 7), (517, 40, 12)]):
        lam = np.sort(rng.uniform(-2, 50, n))
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        Cm = torch.from_numpy(0.5 * ((Q * lam) @ Q.conj().T + ((Q * lam) @ Q.conj().T).conj().T)).to(dev)
        Y0 = torch.from_numpy(rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))).to(dev)
        ref = gevp.chebyshev_filter(Cm, Y0.clone(), deg, lo, hi, s, prec="fp64")
        Y = Y0.clone()
        st = _noalloc(L, stream, Cm, Y, deg, lo, hi, s)
        torch.cuda.synchronize()
        assert st == 0, f"call {call}: status {st}"
        err = (Y - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-12, f"call {call}: relative difference {err:.2e}"


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
