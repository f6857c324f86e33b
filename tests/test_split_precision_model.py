"""Numerics of the split tensor-core contraction, emulated on the CPU.

The split-BF16 correlator writes each FP32 operand as three BF16 slices
(x = x0 + x1 + x2, 8 significant bits each) and sums the six slice products
whose weight is at least 2^-16 (a0 b0, a0 b1, a1 b0, a1 b1, a0 b2, a2 b0).
The tensor cores form each slice product exactly and accumulate in FP32.
The alternative on TF32 units (11 significant bits, half the BF16 rate) at
the same cost is two slices with three products (a0 b0, a0 b1, a1 b0):
three products at half rate equal six BF16 products.  This test emulates
both bit by bit on operands drawn like the workload's (snapshot sums of
conj(a) b over ny x ny pairs per wavenumber) and measures each against FP64.
Measured: both stay within a few 1e-7 of the largest value (FP32
accumulation alone gives about 1e-7), so a TF32 split of equal cost would
match BF16 x 3, not beat it; a single TF32 product (a0 b0 only) does not
reach 1e-6.
"""
import numpy as np

import synthetic as S


def _round(x, bits):
    """x (float32 array) rounded to `bits` significant bits, nearest-even."""
    m, e = np.frexp(x.astype(np.float64))
    scale = float(2 ** bits)
    return np.ldexp(np.round(m * scale) / scale, e).astype(np.float32)


def _slices(x, bits, n):
    out, r = [], x.astype(np.float32)
    for _ in range(n):
        s = _round(r, bits)
        out.append(s)
        r = (r - s).astype(np.float32)
    return out


def _contract(a, b, bits, nsl, pairs):
    """sum_s conj(a[s, y]) b[s, y'] with the real parts of the complex
    product split into slices; slice products exact (float64, which holds
    them), accumulated in float32 over snapshots and products."""
    ar, ai = _slices(a.real, bits, nsl), _slices(a.imag, bits, nsl)
    br, bi = _slices(b.real, bits, nsl), _slices(b.imag, bits, nsl)
    ny = a.shape[1]
    re = np.zeros((ny, ny), np.float32)
    im = np.zeros((ny, ny), np.float32)
    for s in range(a.shape[0]):
        for i, j in pairs:
            # conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
            pr = np.outer(ar[i][s], br[j][s]).astype(np.float64) + np.outer(ai[i][s], bi[j][s])
            pi = np.outer(ar[i][s], bi[j][s]).astype(np.float64) - np.outer(ai[i][s], br[j][s])
            re = (re + pr.astype(np.float32)).astype(np.float32)
            im = (im + pi.astype(np.float32)).astype(np.float32)
    return re.astype(np.float64) + 1j * im.astype(np.float64)


BF16X3 = (8, 3, [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 0)])
TF32X2 = (11, 2, [(0, 0), (0, 1), (1, 0)])
TF32X1 = (11, 1, [(0, 0)])


def test_tf32_split_of_equal_cost_matches_bf16x3():
    wl = S.small(16, 16, 33, 16, wid=44)
    coef = S.coefficients(wl)                       # [ns][4][ny][nz][nxh]
    worst = {"bf16x3": 0.0, "tf32x2": 0.0, "tf32x1": 0.0}
    for kz, kx in ((0, 1), (1, 0), (3, 2), (7, 5), (15, 8)):
        a = coef[:, 0, :, kz, kx].astype(np.complex64)     # u at the first plane of each pair
        b = coef[:, 1, :, kz, kx].astype(np.complex64)     # v at the second
        a64, b64 = a.astype(np.complex128), b.astype(np.complex128)
        exact = np.einsum("sy,sz->yz", np.conj(a64), b64)
        scale = np.abs(exact).max()
        for name, (bits, nsl, pairs) in (("bf16x3", BF16X3), ("tf32x2", TF32X2), ("tf32x1", TF32X1)):
            err = np.abs(_contract(a, b, bits, nsl, pairs) - exact).max() / scale
            worst[name] = max(worst[name], err)
    assert worst["bf16x3"] < 1e-6 and worst["tf32x2"] < 1e-6, worst
    assert 1 / 3 < worst["tf32x2"] / worst["bf16x3"] < 3, worst
    assert worst["tf32x1"] > 1e-6, worst
