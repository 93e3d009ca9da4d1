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


def eig32(a, b, c, delta):
    """The stencil stage's FP32 eigen step in float32 (plain operations): k-,
    its bound, and the unit direction with its bound (nan where no bound is
    given)."""
    a, b, c = (np.asarray(v, np.float32) for v in (a, b, c))
    htr = (a + c) * f32(0.5)
    hdf = (a - c) * f32(0.5)
    rad = np.sqrt(hdf * hdf + b * b)
    k = htr - rad
    M = np.abs(a) + np.abs(b) + np.abs(c)
    ek = M * f32(16 * U) + f32(1e-30) + f32(3.0) * f32(delta)
    w = np.abs(hdf) + rad
    vx = np.where(hdf >= 0, b, -w)
    vy = np.where(hdf >= 0, -w, b)
    nrm = np.sqrt(vx * vx + vy * vy)
    ok = (nrm > f32(4.0) * f32(delta)) & (nrm > 0)
    with np.errstate(invalid="ignore", divide="ignore"):
        X, Y = vx / nrm, vy / nrm
        flip = (X < 0) | ((X == 0) & (Y < 0))
        X, Y = np.where(flip, -X, X), np.where(flip, -Y, Y)
        eX = (M * f32(16 * U)) / nrm + f32(4 * U) + f32(6.0) * f32(delta) / (nrm - f32(3.0) * f32(delta))
    return k, ek, X, Y, np.where(ok, eX, np.nan)


def test_eigen_bounds():
    """|k32 - k_def| <= ek and, where a bound is given and X_def is clear of
    the canonical-sign ambiguity (|X| > eX, the region the ridge test treats
    as undecided anyway), |X32 - X_def|, |Y32 - Y_def| <= eX; inputs exact
    in float32 (delta 0) and perturbed by up to delta."""
    rng = np.random.default_rng(7)
    n = 200000
    scale = 10.0 ** rng.uniform(-3, 3, n)
    a = (rng.normal(size=n) * scale).astype(np.float32)
    c = np.where(rng.random(n) < 0.2, a, (rng.normal(size=n) * scale).astype(np.float32))  # near-degenerate
    b = np.where(rng.random(n) < 0.2, (rng.normal(size=n) * scale * 1e-6).astype(np.float32),
                 (rng.normal(size=n) * scale).astype(np.float32))
    for rel in (0.0, 1e-5):
        delta = rel * (np.abs(a) + np.abs(b) + np.abs(c)).astype(np.float64)
        # the FP32 stage sees (a, b, c); the definition's values are within delta of them
        da = a.astype(np.float64) + rng.uniform(-1, 1, n) * delta
        db = b.astype(np.float64) + rng.uniform(-1, 1, n) * delta
        dc = c.astype(np.float64) + rng.uniform(-1, 1, n) * delta
        kd, Xd, Yd, deg = O.eigen(da, dc, db)
        k32, ek, X32, Y32, eX = eig32(a, b, c, delta.astype(np.float32))
        assert np.all(np.abs(k32.astype(np.float64) - kd) <= ek.astype(np.float64))
        sel = np.isfinite(eX) & ~deg & (np.abs(Xd) > eX)
        assert sel.mean() > 0.5
        assert np.all(np.abs(X32[sel].astype(np.float64) - Xd[sel]) <= eX[sel])
        assert np.all(np.abs(Y32[sel].astype(np.float64) - Yd[sel]) <= eX[sel])
