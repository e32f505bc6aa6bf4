"""Element-wise checks of the tcgen05 filter product at the bench shape (n = 2048, m = 140,
split-K 8), through the C ABI.

The low-precision filter rounds every real operand to BF16 pieces (one piece for the BF16
filter; three for the FP32-class one, x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1),
of which the products with piece indices a + b <= 2 are formed), with Y first rounded to
FP32 (its recurrence state), and forms the complex product by three real products (Gauss):
T1 = Cr Yr, T2 = Ci Yi, T3 = (Cr + Ci)(Yr + Yi), Re = T1 - T2, Im = T3 - T1 - T2, accumulated
in FP32. The reference below is the exact product of those rounded pieces (BF16 x BF16
products are exact in FP64 and K = 2048 FP64 sums add < 1e-12 relative), so the GPU result
may differ from it only by FP32 accumulation: per entry at most
    (terms + slices + 8) 2^-23 (S1 + S2 + S3),   S = sum_k |piece of C| |piece of Y|
over the three real products (2^-23 also covers truncating accumulation). A wrong tile, a
missing or doubled split-K slice or a piece pairing error moves entries far outside this.
A second per-entry check bounds the distance to the true FP64 product C Y by the rounding
the precision mode itself makes (2^-8 of S for BF16, 2^-21 for the FP32 class) plus the
accumulation bound. Multi-step filters are compared with the oracle's scaled recurrence per
block of 128 rows (one MMA tile) and column, so that a localised error cannot hide in a
norm over the whole block.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _round_sig(x, bits):
    """Round to `bits` significant bits, nearest, ties to even (exponent range unbounded)."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(np.ldexp(m, bits)), e - bits)


def _pieces(x, nsplit):
    out, r = [], np.array(x, dtype=np.float64)
    for _ in range(nsplit):
        h = _round_sig(r, 8)
        out.append(h)
        r = r - h
    return out


def _model(Cm, Y, nsplit):
    """Exact product of the rounded pieces, and the per-entry accumulation bound."""
    cr, ci = Cm.real.copy(), Cm.imag.copy()
    cs = cr + ci
    y32 = Y.astype(np.complex64)
    yr = y32.real.astype(np.float64)
    yi = y32.imag.astype(np.float64)
    ys = yr + yi   # exact: a sum of two FP32 values
    P = {k: _pieces(v, nsplit) for k, v in (("cr", cr), ("ci", ci), ("cs", cs), ("yr", yr), ("yi", yi), ("ys", ys))}
    segs = [(a, b) for a in range(nsplit) for b in range(nsplit) if a + b <= nsplit - 1]
    T = {}
    S = 0.0
    for c, y, name in (("cr", "yr", 1), ("ci", "yi", 2), ("cs", "ys", 3)):
        T[name] = sum(P[c][a] @ P[y][b] for a, b in segs)
        S = S + sum(np.abs(P[c][a]) @ np.abs(P[y][b]) for a, b in segs)
    ref = (T[1] - T[2]) + 1j * (T[3] - T[1] - T[2])
    return ref, S, len(segs)


def _hermitian(rng, n, lo=-2.0, hi=50.0):
    lam = np.sort(rng.uniform(lo, hi, n))
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, _ = np.linalg.qr(G)
    Cm = (Q * lam) @ Q.conj().T
    return 0.5 * (Cm + Cm.conj().T)


@pytest.mark.parametrize("prec,nsplit", [("bf16", 1), ("fp32", 3)])
def test_tc_product_elementwise_bench_shape(cuda, prec, nsplit):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(2048 + nsplit)
    n, m = 2048, 140
    Cm = _hermitian(rng, n)
    Y = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    # degree-1 filter with c = 0, e = 1, s = -2: Y1 = -(1/2) C Y exactly (a power-of-two
    # scale and a zero multiple of Y in the FP32 epilogue)
    Y1 = gevp.chebyshev_filter(torch.from_numpy(Cm).to(cuda), torch.from_numpy(Y).to(cuda), 1, -1.0, 1.0, -2.0,
                               prec=prec).cpu().numpy()
    D = -2.0 * Y1
    ref, S, nseg = _model(Cm, Y, nsplit)
    K, slices = n, 8
    acc_bound = (nseg * K + slices + 8) * 2.0 ** -23 * S
    d = np.maximum(np.abs(D.real - ref.real), np.abs(D.imag - ref.imag))
    assert np.all(d <= acc_bound), f"worst excess {np.max(d / acc_bound):.3g}x of the accumulation bound"
    # against the true product: the precision mode's own rounding plus accumulation
    true = Cm @ Y
    u_mode = 2.0 ** -8 if nsplit == 1 else 2.0 ** -21
    d2 = np.maximum(np.abs(D.real - true.real), np.abs(D.imag - true.imag))
    assert np.all(d2 <= 1.02 * u_mode * S + acc_bound)
    # the realistic error is far below the bounds: the check would see a lost slice
    assert np.max(d) < 1e-2 * np.max(acc_bound)


@pytest.mark.parametrize("prec,deg,tol", [("bf16", 4, 5e-2), ("bf16", 12, 5e-2), ("fp32", 4, 1e-4),
                                          ("fp32", 12, 1e-4)])
def test_tc_filter_blockwise_bench_shape(cuda, prec, deg, tol):
    """The recurrence at the bench shape against the oracle: the whole block within the
    precision mode's tolerance, and no block of 128 rows (one MMA tile) in any column more
    than 10x the median block error: a lost, doubled or misplaced tile or split-K slice
    stands out against the median, which a localised error does not move."""
    from oracle import pieces
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(3000 + deg + len(prec))
    n, m = 2048, 140
    Cm = _hermitian(rng, n)
    Y0 = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    lo, hi, s = 5.0, 50.5, -2.5
    Yg = gevp.chebyshev_filter(torch.from_numpy(Cm).to(cuda), torch.from_numpy(Y0).to(cuda), deg, lo, hi, s,
                               prec=prec).cpu().numpy()
    Yr = pieces.chebyshev_filter(Cm, Y0, deg, lo, hi, s)
    glob = np.linalg.norm(Yg - Yr) / np.linalg.norm(Yr)
    assert glob < tol
    E = (Yg - Yr).reshape(n // 128, 128, m)
    R = Yr.reshape(n // 128, 128, m)
    rel = np.linalg.norm(E, axis=1) / np.linalg.norm(R, axis=1)
    med = np.median(rel)
    assert rel.max() < 10 * med, f"worst block {np.unravel_index(rel.argmax(), rel.shape)}: {rel.max() / med:.3g}x median"
