"""The arithmetic of the emulated FP64 product (Ozaki scheme), checked on the CPU with a
numpy model written from the scheme's definition (it shares no code with the CUDA path):
rows scaled into [1/4, 1/2) and rounded to S signed base-128 digits with |d| <= 64; the
digit products of one unit (at most 2048 complex terms, 4096 real terms of the embedding)
summed exactly in FP32 (every partial sum an integer of magnitude <= 2^24); pairs with
s + t <= S + 1 kept; levels combined by an FP64 Horner recurrence. The stated error bound
2K (S + 3) 2^(-7S + 2) max|a_i.| max|b_.j| must hold, including on adversarial inputs that
put every digit at its extreme."""
import math

import numpy as np
import pytest


def split(X, S):
    mx = np.maximum(np.abs(X.real), np.abs(X.imag)).max(axis=1)
    e = np.zeros(X.shape[0], dtype=np.int64)
    nz = mx > 0
    e[nz] = np.floor(np.log2(mx[nz])).astype(np.int64) + 2
    assert np.all(mx[nz] * 2.0 ** -e[nz] < 0.5) and np.all(mx[nz] * 2.0 ** -e[nz] >= 0.25)

    def digits(x):
        q = np.rint(np.ldexp(x, (7 * S - e)[:, None])).astype(np.int64)
        assert np.abs(q).max() <= 2 ** (7 * S - 1)
        D = np.zeros((S,) + x.shape, dtype=np.int64)
        for s in range(S - 1, 0, -1):
            d = ((q + 64) & 127) - 64
            D[s] = d
            q = (q - d) >> 7
        D[0] = q
        return D

    return e, digits(X.real), digits(X.imag)


def emulate(A, B, S, kchunk=2048, grouped=False):
    """A B^H through the scheme; also returns the largest |partial sum| seen in a unit.
    grouped: the pairs of one level share one running sum (the accumulator of a level, for
    S K <= 2048), instead of one per pair."""
    ea, Ar, Ai = split(A, S)
    eb, Br, Bi = split(B.conj(), S)
    K = A.shape[1]
    worst = 0
    out = []
    for part in (0, 1):
        h = None
        for L in range(S + 1, 1, -1):
            I = np.zeros((A.shape[0], B.shape[0]), dtype=np.int64)
            run = np.zeros(I.shape, dtype=np.int64)
            for s in range(1, L):
                t = L - s
                for k0 in range(0, K, kchunk):
                    sl = slice(k0, min(K, k0 + kchunk))
                    if part == 0:
                        terms = [(Ar[s - 1][:, sl], Br[t - 1][:, sl]), (Ai[s - 1][:, sl], -Bi[t - 1][:, sl])]
                    else:
                        terms = [(Ai[s - 1][:, sl], Br[t - 1][:, sl]), (Ar[s - 1][:, sl], Bi[t - 1][:, sl])]
                    # the running sum of a unit (or of the level), term by term, in the
                    # order the MMA adds them
                    if not grouped:
                        run = np.zeros(I.shape, dtype=np.int64)
                    for X, Y in terms:
                        for kk in range(X.shape[1]):
                            run += np.outer(X[:, kk], Y[:, kk])
                            worst = max(worst, int(np.abs(run).max()))
                    if not grouped:
                        I += run
            if grouped:
                I = run
            assert np.abs(I).max() < 2 ** 31   # the level sum fits the kernel's int32
            h = I.astype(float) if h is None else h * 2.0 ** -7 + I
        out.append(np.ldexp(h, ea[:, None] + eb[None, :] - 14))
    return out[0] + 1j * out[1], worst


def bound(A, B, S):
    K = A.shape[1]
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
    rb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=1)
    return 2 * K * (S + 3) * 2.0 ** (-7 * S + 2) * np.outer(ra, rb)


@pytest.mark.parametrize("S", [2, 4, 8])
def test_random_within_the_stated_bound(S):
    rng = np.random.default_rng(60 + S)
    A = (rng.standard_normal((6, 150)) + 1j * rng.standard_normal((6, 150))) * np.exp(rng.uniform(-8, 8, (6, 1)))
    B = rng.standard_normal((5, 150)) + 1j * rng.standard_normal((5, 150))
    D, worst = emulate(A, B, S)
    assert worst <= 2 ** 24
    assert np.all(np.abs(D - A @ B.conj().T) <= bound(A, B, S) + 1e-300)


def test_extreme_digits_keep_fp32_sums_exact():
    # every entry at the top of its row's range with the sign pattern that makes every
    # digit product +-64^2 and every partial sum grow monotonically: the worst case for
    # the FP32 accumulation of a 2048-term unit
    S, K = 3, 2048
    x = (0.5 - 2.0 ** -22) * np.ones(K)
    A = (x + 1j * x)[None, :]
    B = (x - 1j * x)[None, :]
    D, worst = emulate(A, B, S)
    assert worst <= 2 ** 24
    ref = A @ B.conj().T
    assert np.abs(D - ref).max() <= bound(A, B, S).max()


def test_integer_inputs_are_exact():
    rng = np.random.default_rng(61)
    A = rng.integers(-2, 3, (4, 300)) + 1j * rng.integers(-2, 3, (4, 300))
    B = rng.integers(-2, 3, (3, 300)) + 1j * rng.integers(-2, 3, (3, 300))
    for S in (1, 8):
        D, _ = emulate(A, B, S)
        assert np.array_equal(D, A @ B.conj().T)


def test_chunked_units_equal_one_pass_for_short_k():
    # cutting K into exact units changes nothing when every sum is exact
    rng = np.random.default_rng(62)
    A = rng.standard_normal((3, 200)) + 1j * rng.standard_normal((3, 200))
    B = rng.standard_normal((2, 200)) + 1j * rng.standard_normal((2, 200))
    D1, _ = emulate(A, B, 8, kchunk=2048)
    D2, _ = emulate(A, B, 8, kchunk=64)
    assert np.array_equal(D1, D2)


def test_level_grouped_accumulation_stays_exact():
    # S K <= 2048: all digit pairs of a level accumulate in one FP32 buffer; S pairs of
    # 2K real products of at most 2^12 stay within 2^24 (exact FP32 integers), including
    # for the extreme-digit input, and give the same product as one running sum per pair
    for S, K in ((8, 256), (4, 512), (3, 600)):
        x = (0.5 - 2.0 ** -22) * np.ones(K)
        A = (x + 1j * x)[None, :]
        B = (x - 1j * x)[None, :]
        Dg, worst = emulate(A, B, S, grouped=True)
        assert worst <= 2 ** 24
        Dp, _ = emulate(A, B, S)
        assert np.array_equal(Dg, Dp)
    rng = np.random.default_rng(63)
    A = (rng.standard_normal((4, 256)) + 1j * rng.standard_normal((4, 256))) * np.exp(rng.uniform(-5, 5, (4, 1)))
    B = rng.standard_normal((3, 256)) + 1j * rng.standard_normal((3, 256))
    Dg, worst = emulate(A, B, 8, grouped=True)
    assert worst <= 2 ** 24
    assert np.array_equal(Dg, emulate(A, B, 8)[0])
    assert np.all(np.abs(Dg - A @ B.conj().T) <= bound(A, B, 8) + 1e-300)
