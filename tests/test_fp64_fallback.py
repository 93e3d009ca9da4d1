"""The FP64 fallback of the stencil stage (the exact test of pixels FP32 could
not decide) evaluates the definition's double operations in the oracle's
order, so its k-, X- and ridge verdicts equal the oracle's bit for bit.
Checked on CPU by replaying the kernel's sequence (each step one IEEE double
operation, as the kernel's round-to-nearest intrinsics do) on random,
near-degenerate, degenerate and exactly-axis Hessians of integer Sobel sums."""
import math

import numpy as np

from oracle import ringdet as O


def eigen64(hxx, hyy, hxy, D):
    a, c, b = hxx / D, hyy / D, hxy / D
    half_tr = (a + c) * 0.5
    half_df = (a - c) * 0.5
    rad = math.sqrt(half_df * half_df + b * b)
    k = half_tr - rad
    v1x, v1y = b, k - a
    v2x, v2y = k - c, b
    n1 = v1x * v1x + v1y * v1y
    n2 = v2x * v2x + v2y * v2y
    use1 = n1 >= n2
    vx, vy, n = (v1x, v1y, n1) if use1 else (v2x, v2y, n2)
    if n == 0.0:
        return k, 0.0, 0.0, True
    nrm = math.sqrt(n)
    X, Y = vx / nrm, vy / nrm
    if X < 0.0 or (X == 0.0 and Y < 0.0):
        X, Y = -X, -Y
    return k, X, Y, False


def bilinear64(fx, fy, k00, k01, k10, k11):
    gx, gy = 1.0 - fx, 1.0 - fy
    top = gx * k00 + fx * k01
    bot = gx * k10 + fx * k11
    return gy * top + fy * bot


def hessians(rng, n):
    out = []
    for _ in range(n):
        s = 10.0 ** rng.uniform(0, 17.5)                      # |H'| < 2^60 at 2^-19 taps
        out.append(tuple(int(v) for v in np.rint(rng.normal(0, s, 3))))
    for _ in range(n // 4):                                   # near-degenerate
        base = int(10.0 ** rng.uniform(3, 17.5))
        out.append((base + int(rng.integers(-2, 3)), base + int(rng.integers(-2, 3)), int(rng.integers(-2, 3))))
    out += [(5, 5, 0), (0, 0, 0), (-7, 3, 0), (3, -7, 0), (4, 4, 1), (1 << 51, -(1 << 51), 1 << 50),
            ((1 << 59) + 1, -(1 << 59) - 3, (1 << 58) + 1)]
    return out


def test_eigen_fallback_equals_oracle_bitwise():
    rng = np.random.default_rng(64)
    S = int(O.gaussian_taps(2.0).sum())
    D = float(64 * S * S)
    hs = hessians(rng, 20000)
    A = np.array([h[0] for h in hs], dtype=np.int64)
    C = np.array([h[1] for h in hs], dtype=np.int64)
    B = np.array([h[2] for h in hs], dtype=np.int64)
    k, X, Y, deg = O.eigen(A.astype(np.float64) / D, C.astype(np.float64) / D, B.astype(np.float64) / D)
    for i, (a, c, b) in enumerate(hs):
        kk, xx, yy, dd = eigen64(a, c, b, D)
        assert dd == bool(deg[i])
        assert kk == k[i] and xx == X[i] and yy == Y[i], (a, c, b)


def test_bilinear_fallback_equals_oracle_bitwise():
    """The fallback's bilinear sample against the oracle's ridge test on a
    random k- field: same verdict for every pixel, and the same sample value
    as the oracle's scalar bilinear."""
    rng = np.random.default_rng(65)
    H, W = 40, 50
    k = rng.normal(0, 1, (H, W))
    k[10:14, :] = 0.25                                       # plateaus: exact ties
    t = rng.uniform(0, np.pi, (H, W))
    X, Y = np.cos(t), np.sin(t)
    X[:, :5], Y[:, :5] = 1.0, 0.0                            # samples on grid points
    deg = np.zeros((H, W), bool)
    want = O.ridge_mask(k, X, Y, deg, 0.5)
    for y in range(H):
        for x in range(W):
            ok = k[y, x] < 0.5
            for s in (1, -1):
                qx, qy = x + s * X[y, x], y + s * Y[y, x]
                if not (0.0 <= qx <= W - 1 and 0.0 <= qy <= H - 1):
                    ok = False
                    break
                x0, y0 = math.floor(qx), math.floor(qy)
                fx, fy = qx - x0, qy - y0
                x1 = x0 if fx == 0.0 else min(x0 + 1, W - 1)   # the fallback skips a zero-weight corner
                y1 = y0 if fy == 0.0 else min(y0 + 1, H - 1)
                kt = bilinear64(fx, fy, k[y0, x0], k[y0, x1], k[y1, x0], k[y1, x1])
                assert kt == O.bilinear(k, qx, qy)
                ok = ok and (k[y, x] < kt if s == 1 else k[y, x] <= kt)
            assert ok == bool(want[y, x]), (y, x)
