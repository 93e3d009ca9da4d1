"""The FP32 error bounds that the certified decisions rely on, checked on CPU.

The stencil stage's FP32 operation sequences (row filters, column filters,
scaling) are replayed in NumPy float32, each fused multiply-add taken as one
rounding of the exact product-sum. They run on random and adversarial frames
and are compared with the exact integer values (or FP64 ones for float
frames). At every pixel the error must stay within the delta the kernels use,
even with the maximum of L taken over the pixel's own 5x5 window (a tile's
maximum is never smaller)."""
import numpy as np
import pytest

from oracle import ringdet as O
from oracle import soft as S
from paper_1310_1371_gb300 import synth

U = 2.0 ** -24
f32 = np.float32


def fma(a, b, c):
    """a b + c rounded once to float32 (the float32 product is exact in float64)."""
    return (np.float64(a) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def row_filters(Lf):
    l0, l1, l2, l3, l4 = (Lf[:, k:Lf.shape[1] - 4 + k] for k in range(5))
    e = l0 + l4
    rs = fma(6.0, l2, fma(4.0, l1 + l3, e))
    rd2 = fma(-2.0, l2, e)
    rd1 = fma(2.0, l3 - l1, l4 - l0)
    return rs, rd2, rd1


def rows(R):
    return [R[k:R.shape[0] - 4 + k, :] for k in range(5)]


def hess32(Lf, invD):
    rs, rd2, rd1 = row_filters(Lf)
    x0, x1, x2, x3, x4 = rows(rd2)
    y0, y1, y2, y3, y4 = rows(rs)
    z0, z1, z2, z3, z4 = rows(rd1)
    hxx = fma(6.0, x2, fma(4.0, x1 + x3, x0 + x4))
    hyy = fma(-2.0, y2, y0 + y4)
    hxy = fma(2.0, z3 - z1, z4 - z0)
    return hxx * invD, hyy * invD, hxy * invD


def grad32(Lf, invD):
    rs, _, rd1 = row_filters(Lf)
    x0, x1, x2, x3, x4 = rows(rd1)
    y0, y1, y2, y3, y4 = rows(rs)
    gx = fma(6.0, x2, fma(4.0, x1 + x3, x0 + x4))
    gy = fma(2.0, y3 - y1, y4 - y0)
    return gx * invD, gy * invD


def window_max(A):
    """max over each interior pixel's 5x5 window."""
    H, W = A.shape
    return np.max(np.stack([A[dy:H - 4 + dy, dx:W - 4 + dx] for dy in range(5) for dx in range(5)]), axis=0)


def frames():
    rng = np.random.default_rng(31)
    yield rng.integers(0, 65536, (96, 96), dtype=np.uint16)                     # full-range noise
    cb = (np.indices((96, 96)).sum(0) % 2 * 65535).astype(np.uint16)             # checkerboard
    yield cb
    yield (65535 - rng.integers(0, 8, (96, 96))).astype(np.uint16)               # high offset, tiny detail
    yield rng.integers(0, 256, (96, 96), dtype=np.uint8)
    yield synth.plain_full(seed=[1002, 0]).image[300:428, 300:428]
    yield synth.plain_small(seed=1001).image[60:188, 60:188]


@pytest.mark.parametrize("k", range(6))
def test_hessian_bound(k):
    img = list(frames())[k]
    Lp, Ssum = O.smooth_int(img, 2.0)
    D = 64.0 * Ssum * Ssum
    Lf = Lp.astype(np.float32)
    fa, fc, fb = hess32(Lf, f32(1.0 / D))
    hxx, hyy, hxy = O.hessian_int(Lp)
    ex = [h[2:-2, 2:-2].astype(np.float64) / D for h in (hxx, hyy, hxy)]
    delta = 448 * U * window_max(Lf.astype(np.float64)) / D
    for got, ref in zip((fa, fc, fb), ex):
        err = np.abs(got.astype(np.float64) - ref)
        assert np.all(err <= delta), float((err / np.maximum(delta, 1e-300)).max())


@pytest.mark.parametrize("k", range(6))
def test_gradient_bound(k):
    img = list(frames())[k]
    Lp, Ssum = O.smooth_int(img, 2.0)
    D = 128.0 * Ssum * Ssum
    Lf = Lp.astype(np.float32)
    gx, gy = grad32(Lf, f32(1.0 / D))
    ex, ey = O.gradient_int(Lp)
    delta = 576 * U * window_max(Lf.astype(np.float64)) / D
    for got, ref in ((gx, ex), (gy, ey)):
        err = np.abs(got.astype(np.float64) - ref[2:-2, 2:-2].astype(np.float64) / D)
        assert np.all(err <= delta), float((err / np.maximum(delta, 1e-300)).max())


@pytest.mark.parametrize("seed", [41, 42])
def test_float_frame_hessian_bound(seed):
    """Float frames (L of either sign), scaled by 1/64 exactly: delta = 512 u max|L| / 64."""
    rng = np.random.default_rng(seed)
    img = rng.normal(0.0, 1000.0, (96, 96)) + (rng.random() - 0.5) * 1e5
    g = S._taps_float(2.0)
    L = S._correlate1d(S._correlate1d(img, g, 1), g, 0)
    lxx, lyy, lxy = S.hessian_float(img, 2.0)
    fa, fc, fb = hess32(L.astype(np.float32), f32(1.0 / 64.0))
    delta = 512 * U * window_max(np.abs(L.astype(np.float32)).astype(np.float64)) / 64.0
    for got, ref in zip((fa, fc, fb), (lxx, lyy, lxy)):
        err = np.abs(got.astype(np.float64) - ref[2:-2, 2:-2])
        assert np.all(err <= delta), float((err / np.maximum(delta, 1e-300)).max())
