"""The certified vote rounding of the voting stage, replayed on CPU.

The voting stage rounds s r X- in FP32 and keeps the result only when it is
certain to equal the double-precision definition (the vote bin
floor(p + s r X- + 1/2) of the oracle, or floor((p + s r X- + c/2) / c) in a
coarse parameter space).  This test replays, in NumPy float32 with every fused
multiply-add rounded once from the exact value, the three steps that decide:

* the direction stage's double-float X- from the exact integer Hessian, with
  its error bound eXr and the margins (kfast, kref) it stores per ridge pixel;
* the fast path (magic-constant rounding, margin r KF + 1e-10, KF = 1.72e-7,
  exact axes without a margin, pixels whose kfast exceeds KF always slow);
* the double-float refinement of undecided votes (vote_offset / vote_floor),
  which either decides or hands over to the FP64 definition.

On random Hessians over many magnitudes, near-degenerate ones, exact axes,
and Hessians built so that r X- falls within 1e-7 of a rounding boundary, every
vote that the fast path or the refinement decides must equal the oracle's bin,
and the double-float direction must lie within eXr of the definition's.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ringdet as O

f32 = np.float32
U32 = f32(2.0 ** -24)
KF_CONST = f32(1.72e-7)
MAGIC = f32(12582912.0)          # 1.5 * 2^23
SIGMA = 2.0


# ---------------------------------------------------------------- float32, one rounding per operation
def rn32(q: Fraction) -> float:
    """The float32 nearest to the rational q (ties to even), as a Python float."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    e = max(e, -126)                               # subnormal spacing below 2^-126
    scale = Fraction(2) ** (e - 23)
    m = q / scale
    n = m.numerator // m.denominator
    rem = m - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return float(sign * n * scale)


def fma(a, b, c):
    return f32(rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def ll2f(x: int):
    return f32(rn32(Fraction(int(x))))


def add(a, b):
    return f32(f32(a) + f32(b))


def sub(a, b):
    return f32(f32(a) - f32(b))


def mul(a, b):
    return f32(f32(a) * f32(b))


def div(a, b):
    return f32(f32(a) / f32(b))


# ---------------------------------------------------------------- double-float, as the direction stage runs it
def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def quick_two_sum(a, b):
    s = add(a, b)
    return s, sub(b, sub(s, a))


def two_prod(a, b):
    p = mul(a, b)
    return p, fma(a, b, -p)


def df_add(a, b):
    s = two_sum(a[0], b[0])
    t = two_sum(a[1], b[1])
    s = quick_two_sum(s[0], add(s[1], t[0]))
    return quick_two_sum(s[0], add(s[1], t[1]))


def df_mul(a, b):
    p, e = two_prod(a[0], b[0])
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    return quick_two_sum(p, e)


def df_sqrt(a):
    if a[0] <= 0:
        return f32(0), f32(0)
    s = f32(np.sqrt(f32(a[0])))
    s2 = two_prod(s, s)
    r = add(sub(sub(a[0], s2[0]), s2[1]), a[1])
    r = div(r, mul(2.0, s))
    return quick_two_sum(s, r)


def df_div(a, b):
    q1 = div(a[0], b[0])
    p = df_mul((q1, f32(0)), b)
    r = df_add(a, (-p[0], -p[1]))
    return quick_two_sum(q1, div(r[0], b[0]))


def df_from_ll(x: int):
    hi = ll2f(x)
    return hi, ll2f(x - int(hi))


def direction_stage(A: int, C: int, B: int):
    """X- of the exact Hessian (A, C, B) = D (Lxx, Lyy, Lxy) as double-float
    pairs with the canonical sign, its error bound eXr and the stored vote
    margins (kfast, kref)."""
    P, Bq = A - C, 2 * B
    dP, dB = df_from_ll(P), df_from_ll(Bq)
    Rr = df_sqrt(df_add(df_mul(dP, dP), df_mul(dB, dB)))
    aP = dP if P >= 0 else (-dP[0], -dP[1])
    Wc = df_add(aP, Rr)
    if P >= 0:
        vx, vy = dB, (-Wc[0], -Wc[1])
    else:
        vx, vy = (-Wc[0], -Wc[1]), dB
    nrm = df_sqrt(df_add(df_mul(vx, vx), df_mul(vy, vy)))
    X, Y = df_div(vx, nrm), df_div(vy, nrm)
    if X[0] < 0 or (X[0] == 0 and Y[0] < 0):
        X, Y = (-X[0], -X[1]), (-Y[0], -Y[1])
    M = add(add(abs(ll2f(A)), abs(ll2f(B))), abs(ll2f(C)))
    cond = div(mul(2.0, M), max(nrm[0], f32(1e-30)))
    eXr = fma(f32(3.5527137e-15), cond, f32(9.094947e-13))          # 2^-40 + 2^-48 cond
    lo = max(abs(X[1]), abs(Y[1]))
    kfast = fma(f32(1.25), add(add(lo, eXr), U32), U32)
    kref = fma(f32(1.25), eXr, f32(2.842171e-14))                      # + 2^-45
    return X, Y, eXr, kfast, kref


# ---------------------------------------------------------------- the refinement of undecided votes
INT_MIN = None


def refine(sr, r, xhi, xlo, kfast, kref, coarse):
    """vote_offset (coarse False: floor(t + 1/2)) or vote_floor (coarse True:
    floor(t)) of t = sr X, or None when the FP64 definition must decide."""
    t = mul(sr, xhi)
    if coarse:
        n = f32(math.floor(t))
        p = sub(t, n)
    else:
        n = f32(math.floor(add(t, 0.5)))
        p = sub(t, sub(n, 0.5))
    m = fma(r, kfast, f32(1e-10))
    if p > m and (p < 0.5 or sub(1.0, p) > m):
        return int(n)
    tp = two_prod(sr, xhi)
    e2 = fma(sr, xlo, tp[1])
    p2 = sub(tp[0], n) if coarse else sub(tp[0], sub(n, 0.5))
    q2 = sub(1.0, p2)
    mr = fma(r, kref, f32(1e-10))
    low_ok = p2 > sub(mr, e2)
    low_bad = p2 < sub(-mr, e2)
    up_ok = p2 < 0.5 or q2 > add(mr, e2)
    up_bad = p2 >= 0.5 and q2 < sub(e2, mr)
    if low_ok and up_ok:
        return int(n)
    if low_bad:
        return int(n) - 1
    if up_bad:
        return int(n) + 1
    return INT_MIN


# ---------------------------------------------------------------- one ridge pixel's votes
def kernel_offsets(A, C, B, radii, coarse):
    """{(r, s): (ox, oy, path)} for the decided votes; path 'fast', 'refine'
    (None: handed to the FP64 definition)."""
    X, Y, eXr, kfast, kref = direction_stage(A, C, B)
    axis = (X[0] == 0 and X[1] == 0) or (Y[0] == 0 and Y[1] == 0)
    ex = (f32(0) if X[0] == 0 else f32(1)) if axis else X[0]
    ey = (f32(1) - ex) if axis else Y[0]
    ill = (not axis) and kfast > KF_CONST
    kf = f32(-1.0) if axis else (f32(1e30) if ill else KF_CONST)
    out = {}
    for r in radii:
        rf = f32(r)
        m = fma(rf, kf, f32(1e-10))
        for s in (1, -1):
            sr = f32(s * r)
            tx, ty = mul(sr, ex), mul(sr, ey)
            fx, fy = add(tx, MAGIC), add(ty, MAGIC)
            dx, dy = sub(tx, sub(fx, MAGIC)), sub(ty, sub(fy, MAGIC))
            ox, oy = int(sub(fx, MAGIC)), int(sub(fy, MAGIC))
            if not coarse:
                sure = max(abs(dx), abs(dy)) < sub(0.5, m)
            else:
                sure = min(abs(dx), abs(dy)) > m
            if sure:
                if coarse:
                    ox -= 1 if dx < 0 else 0
                    oy -= 1 if dy < 0 else 0
                out[(r, s)] = (ox, oy, "fast")
                continue
            vx = refine(sr, rf, X[0], X[1], kfast, kref, coarse)
            vy = refine(sr, rf, Y[0], Y[1], kfast, kref, coarse)
            out[(r, s)] = (vx, vy, "refine") if vx is not None and vy is not None else None
    return out, (X, Y, eXr, kfast, axis, ill)


def definition_bins(A, C, B, D, p, r, c):
    """The oracle's two vote bins (x, y) of pixel p at radius r, as a sorted list."""
    k, X, Y, deg = O.eigen(np.array([A / D]), np.array([C / D]), np.array([B / D]))
    assert not deg[0]
    H = W = 1 << 17
    bx, by = O.cast_votes(np.array([p[0]]), np.array([p[1]]), X, Y, r, H, W, c)
    return sorted(zip(bx.tolist(), by.tolist())), (float(X[0]), float(Y[0]))


def kernel_bins(offs, p, c):
    """Bins from the kernel's offsets: p + o (c = 1) or (p + o + c/2) >> log2 c."""
    if c == 1:
        return [(p[0] + ox, p[1] + oy) for ox, oy in offs]
    return [((p[0] + ox + c // 2) // c, (p[1] + oy + c // 2) // c) for ox, oy in offs]


# ---------------------------------------------------------------- inputs
def hessian_D():
    S = int(O.gaussian_taps(SIGMA).sum())
    return 64 * S * S


def random_hessians(rng, n):
    out = []
    for _ in range(n):
        scale = 10.0 ** rng.uniform(2, 17.5)          # |H'| < 2^60 at 2^-19 taps
        A, C, B = (int(v) for v in np.rint(rng.normal(0, scale, 3)))
        out.append((A, C, B))
    return out


def near_degenerate(rng, n):
    """Eigenvalue gap a tiny fraction of the entries: large cond, ill records."""
    out = []
    for _ in range(n):
        base = int(10.0 ** rng.uniform(8, 17.5))
        A = base + int(rng.integers(-3, 4))
        C = base + int(rng.integers(-3, 4))
        B = int(rng.integers(-3, 4))
        out.append((A, C, B))
    return out


def axes(rng, n):
    out = []
    for _ in range(n):
        a, c = (int(v) for v in rng.integers(-10 ** 17, 10 ** 17, 2))
        if a != c:
            out.append((a, c, 0))
    return out


def near_boundary(rng, n, coarse):
    """Hessians whose X- makes r X- fall next to a rounding boundary (a
    half-integer, or an integer in a coarse space) for one radius."""
    out = []
    while len(out) < n:
        r = int(rng.integers(7, 98))
        k = int(rng.integers(-r + 1, r - 1))
        t = k + (0.0 if coarse else 0.5)
        xs = t / r
        if abs(xs) >= 1:
            continue
        ys = math.sqrt(1 - xs * xs) * (1 if rng.random() < 0.5 else -1)
        if rng.random() < 0.5:
            xs, ys = ys, xs                        # the boundary in y instead
        lam1 = -10.0 ** rng.uniform(9, 17)         # k-, the smaller eigenvalue
        lam2 = lam1 + abs(lam1) * 10.0 ** rng.uniform(-3, 0.5)
        v = np.array([xs, ys])
        w = np.array([-ys, xs])
        Hm = lam1 * np.outer(v, v) + lam2 * np.outer(w, w)
        out.append((int(round(Hm[0, 0])), int(round(Hm[1, 1])), int(round(Hm[0, 1])), r))
    return out


# ---------------------------------------------------------------- the checks
def check_pixel(A, C, B, D, radii, rng, coarse, counts):
    c = 2 if coarse else 1
    offs, (X, Y, eXr, kfast, axis, ill) = kernel_offsets(A, C, B, radii, coarse)
    _, (Xd, Yd) = definition_bins(A, C, B, D, (0, 0), radii[0], c)
    # the double-float direction is within eXr of the definition's (sign aligned)
    xdf = float(X[0]) + float(X[1])
    ydf = float(Y[0]) + float(Y[1])
    if xdf * Xd + ydf * Yd < 0:
        Xd, Yd = -Xd, -Yd
    if not ill:
        assert abs(xdf - Xd) <= float(eXr) and abs(ydf - Yd) <= float(eXr), (A, C, B, xdf - Xd, ydf - Yd, eXr)
    if axis:
        assert (Xd, Yd) in ((1.0, 0.0), (0.0, 1.0))
    counts["ill"] += int(ill)
    counts["axis"] += int(axis)
    for r in radii:
        p = (int(rng.integers(100, 65436)), int(rng.integers(100, 65436)))   # every vote inside the frame
        want, _ = definition_bins(A, C, B, D, p, r, c)
        got_pairs = [offs[(r, s)] for s in (1, -1)]
        if any(g is None for g in got_pairs):
            counts["fp64"] += 1
            continue
        for g in got_pairs:
            counts[g[2]] += 1
        got = sorted(kernel_bins([g[:2] for g in got_pairs], p, c))
        assert got == want, (A, C, B, r, p, got, want, got_pairs)


@pytest.mark.parametrize("coarse", [False, True])
def test_certified_vote_rounding(coarse):
    rng = np.random.default_rng(77 + int(coarse))
    D = hessian_D()
    counts = {"fast": 0, "refine": 0, "fp64": 0, "ill": 0, "axis": 0}
    radii = list(range(7, 98, 9))
    for A, C, B in random_hessians(rng, 120) + near_degenerate(rng, 30) + axes(rng, 20):
        if A == C and B == 0:
            continue
        check_pixel(A, C, B, D, radii, rng, coarse, counts)
    for A, C, B, r in near_boundary(rng, 250, coarse):
        if A == C and B == 0:
            continue
        check_pixel(A, C, B, D, [r], rng, coarse, counts)
    # every route was taken: certified FP32, the double-float refinement, the
    # FP64 definition, exact axes and ill-conditioned directions
    assert counts["fast"] > 1000 and counts["refine"] > 20 and counts["fp64"] > 0, counts
    assert counts["axis"] > 0 and counts["ill"] > 0, counts


def test_rn32_is_float32_rounding():
    """The exact rounding helper agrees with NumPy's float32 conversion where
    the latter is a single rounding (float64 inputs), including ties."""
    rng = np.random.default_rng(5)
    for v in list(rng.normal(0, 1e3, 500)) + [1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, -(2 + 2.0 ** -23), 1e-40]:
        assert rn32(Fraction(float(v))) == float(np.float32(v))
