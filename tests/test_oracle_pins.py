"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each check compares the oracle with a closed form, a library routine, brute
force on a tiny input, an invariant, or synthetic truth.  The checks are plain
functions returning bool so that ``test_oracle_mutations`` can show that a
planted mistake in the oracle makes one of them fail.
"""
import math

import numpy as np
import pytest

from oracle import ringdet as O
from paper_1310_1371_gb300 import synth


# ---------------------------------------------------------------- helpers
def gaussian_line_image(H, W, x0, amp=200.0, width=1.5, bg=20.0, vertical=True):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    d = (xx - x0) if vertical else (yy - x0)
    return np.rint(bg + amp * np.exp(-0.5 * (d / width) ** 2)).astype(np.uint16)


def ring_image(H, W, cx, cy, R, amp=120.0, width=1.5, bg=40.0, noise=0.0, seed=0):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    rho = np.hypot(xx - cx, yy - cy)
    img = bg + amp * np.exp(-0.5 * ((rho - R) / width) ** 2)
    if noise:
        img = img + np.random.default_rng(seed).normal(0, noise, img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def small_params(**kw):
    d = dict(sigma=2.0, r_min=5, r_max=20, ridge_thresh=-1.0, peak_frac=0.35,
             vote_thresh=3, annulus_w=2.0, sig_a=0.05, sig_b=0.25)
    d.update(kw)
    return O.Params.make(**d)


def reflect101(i, n):
    while i < 0 or i >= n:
        i = -i if i < 0 else 2 * (n - 1) - i
    return i


# ---------------------------------------------------------------- O1
def check_taps_are_gaussian(sigma):
    """Taps sum to 2^19 within rounding, are symmetric and peaked at 0, and
    the normalised discrete variance is sigma^2 (a sampled Gaussian's second
    moment; truncation at 4 sigma and 2^-19 quantisation change it by < 2e-3)."""
    Q = O.gaussian_taps(sigma)
    R = (len(Q) - 1) // 2
    i = np.arange(-R, R + 1)
    S = Q.sum()
    var = float((Q * i * i).sum()) / float(S)
    return (abs(int(S) - (1 << 19)) <= len(Q) and np.array_equal(Q, Q[::-1])
            and Q.argmax() == R and abs(var - sigma * sigma) < 2e-3 * max(1.0, sigma * sigma))


def check_smoothing_brute_force(seed=3):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 4096, size=(14, 13)).astype(np.uint16)
    Q = O.gaussian_taps(1.3)
    R = (len(Q) - 1) // 2
    H, W = img.shape
    ref = np.zeros((H, W), dtype=object)
    for y in range(H):
        for x in range(W):
            acc = 0
            for a in range(-R, R + 1):
                for b in range(-R, R + 1):
                    acc += int(Q[a + R]) * int(Q[b + R]) * int(img[reflect101(y + a, H), reflect101(x + b, W)])
            ref[y, x] = acc
    Lp, _ = O.smooth_int(img, 1.3)
    return np.array_equal(Lp.astype(object), ref)


def check_smoothing_vs_scipy(seed=4):
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=(40, 37)).astype(np.uint8)
    Q = O.gaussian_taps(2.0)
    ref = nd.correlate1d(img.astype(np.int64), Q, axis=1, mode="mirror")
    ref = nd.correlate1d(ref, Q, axis=0, mode="mirror")
    Lp, _ = O.smooth_int(img, 2.0)
    return np.array_equal(Lp, ref)


def check_constant_and_ramp():
    Q = O.gaussian_taps(2.0)
    S = int(Q.sum())
    c = np.full((30, 30), 77, dtype=np.uint8)
    Lp, _ = O.smooth_int(c, 2.0)
    ramp = np.tile(np.arange(60, dtype=np.uint16) * 3, (30, 1))
    Lr, _ = O.smooth_int(ramp, 2.0)
    interior = Lr[:, 9:-9]
    return bool((Lp == 77 * S * S).all() and (interior == ramp[:, 9:-9].astype(np.int64) * S * S).all())


# ---------------------------------------------------------------- O2
def check_quadratic_hessian(a=3, b=-2, c=5):
    """I = a x^2 + b x y + c y^2 + 7x - 4y + 900 gives exactly (2a, 2c, b)
    away from the borders (the smoothed image of a quadratic is a quadratic
    with the same second derivatives; the /64 Sobel is exact on quadratics)."""
    H = W = 40
    yy, xx = np.mgrid[0:H, 0:W].astype(np.int64)
    img = a * xx * xx + b * xx * yy + c * yy * yy + 7 * xx - 4 * yy + 900000
    Lxx, Lyy, Lxy = O.hessian(img, 2.0)
    s = np.s_[11:-11, 11:-11]
    return (np.all(Lxx[s] == 2 * a) and np.all(Lyy[s] == 2 * c) and np.all(Lxy[s] == b))


# ---------------------------------------------------------------- O3
def check_eigen_vs_eigh(seed=5, n=2000):
    rng = np.random.default_rng(seed)
    a, b, c = rng.normal(0, 10, size=(3, n))
    k, X, Y, deg = O.eigen(a, c, b)
    w, V = np.linalg.eigh(np.stack([np.stack([a, b], -1), np.stack([b, c], -1)], -2))
    kmin = w[:, 0]
    v = V[:, :, 0]
    dot = np.abs(v[:, 0] * X + v[:, 1] * Y)
    canon = (X > 0) | ((X == 0) & (Y > 0))
    return (np.allclose(k, kmin, rtol=1e-12, atol=1e-12) and np.all(dot > 1 - 1e-12)
            and np.all(canon) and not deg.any())


def check_eigen_special():
    k, X, Y, deg = O.eigen(np.array([-3.0, 2.0, 1.0]), np.array([1.0, -5.0, 1.0]), np.array([0.0, 0.0, 0.0]))
    return (list(k) == [-3.0, -5.0, 1.0] and (X[0], Y[0]) == (1.0, 0.0) and (X[1], Y[1]) == (0.0, 1.0)
            and list(deg) == [False, False, True])


# ---------------------------------------------------------------- O4
def check_line_ridge():
    """A vertical Gaussian line on an integer column is a ridge exactly on
    that column, with X along x; on a half-integer column exactly one of the
    two middle columns wins in every row."""
    img = gaussian_line_image(40, 41, 20.0)
    p = small_params()
    Lxx, Lyy, Lxy = O.hessian(img, p.sigma)
    k, X, Y, deg = O.eigen(Lxx, Lyy, Lxy)
    m = O.ridge_mask(k, X, Y, deg, p.ridge_thresh)
    rows = slice(12, 28)
    ok1 = np.all(m[rows, 20]) and m[rows].sum() == (rows.stop - rows.start) and np.allclose(X[rows, 20], 1.0)
    img2 = gaussian_line_image(40, 41, 20.5)
    Lxx, Lyy, Lxy = O.hessian(img2, p.sigma)
    k, X, Y, deg = O.eigen(Lxx, Lyy, Lxy)
    m2 = O.ridge_mask(k, X, Y, deg, p.ridge_thresh)
    ok2 = np.all(m2[rows].sum(axis=1) == 1) and np.all(m2[rows, 20] | m2[rows, 21])
    return bool(ok1 and ok2)


def check_ring_ridge_is_radial():
    img = ring_image(96, 96, 47.3, 48.6, 20.0)
    p = small_params()
    xy, Xv = O.directed_ridges(img, p)
    rho = np.hypot(xy[:, 0] - 47.3, xy[:, 1] - 48.6)
    radial = np.stack([xy[:, 0] - 47.3, xy[:, 1] - 48.6], 1) / rho[:, None]
    cosang = np.abs((radial * Xv).sum(1))
    return bool(len(xy) > 4 * 20 and np.all(np.abs(rho - 20.0) < 1.0) and np.all(cosang > 0.98))


# ---------------------------------------------------------------- O5
def full_cht_argmax(ridge_xy, H, W, rlo, rhi):
    """Undirected circle Hough (every ridge pixel votes for every centre at
    rounded distance r), normalised by 1/r; brute force."""
    best, arg = -1.0, None
    yy, xx = np.mgrid[0:H, 0:W]
    A = np.zeros((rhi + 1, H, W))
    for px, py in ridge_xy:
        d = np.floor(np.hypot(xx - px, yy - py) + 0.5).astype(int)
        for r in range(rlo, rhi + 1):
            A[r] += d == r
    for r in range(rlo, rhi + 1):
        s = A[r] / r
        i = np.unravel_index(np.argmax(s), s.shape)
        if s[i] > best:
            best, arg = s[i], (i[1], i[0], r)
    return arg


def check_directed_vs_full_cht():
    img = ring_image(48, 48, 23.4, 24.2, 11.3, noise=3.0, seed=1)
    p = small_params(r_min=6, r_max=16)
    res = O.detect(img, p)
    top = res.rings[np.argmax(res.rings["score"])]
    arg = full_cht_argmax(res.ridge_xy, 48, 48, p.r_min, p.r_max)
    return abs(int(top["ix"]) - arg[0]) <= 1 and abs(int(top["iy"]) - arg[1]) <= 1 and abs(int(top["ir"]) - arg[2]) <= 1


def check_votes_all_inside():
    img = ring_image(120, 120, 60.0, 60.0, 14.0)
    p = small_params(r_min=5, r_max=12)
    res = O.detect(img, p)
    return res.votes_in == res.votes_cast == 2 * len(res.ridge_xy) * (p.r_max - p.r_min + 3)


def check_sign_symmetry():
    img = ring_image(80, 80, 40.0, 39.0, 15.0, noise=4.0, seed=2)
    p = small_params()
    xy, Xv = O.directed_ridges(img, p)
    for r in (7, 15):
        a = O.accumulate(*O.cast_votes(xy[:, 0], xy[:, 1], Xv[:, 0], Xv[:, 1], r, 80, 80), 80, 80)
        b = O.accumulate(*O.cast_votes(xy[:, 0], xy[:, 1], -Xv[:, 0], -Xv[:, 1], r, 80, 80), 80, 80)
        if not np.array_equal(a, b):
            return False
    return True


def check_small_truth():
    f = synth.plain_small()
    res = O.detect(f.image, O.Params.make(**f.params))
    got = np.stack([res.rings["ix"], res.rings["iy"], res.rings["ir"]], 1).astype(float)
    if len(got) != len(f.rings):
        return False
    for cx, cy, R in f.rings:
        if not (np.abs(got - [cx, cy, R]).max(1) <= 1.0).any():
            return False
    return True


# ---------------------------------------------------------------- O6, O7
def check_spike_scores_two_pi():
    """A single voxel with round(2 pi r) votes scores S = round(2 pi r)/r
    (peak weight 1, normalisation 1/r)."""
    r = 30
    Q = O.smoothing_weights(r, np.float32(0.05), np.float32(0.25))
    A = np.zeros((64, 64), dtype=np.int64)
    n = int(round(2 * math.pi * r))
    A[20, 31] = n
    N = O.smooth_hot(A, Q, 3)
    S = N[20, 31] / (65536.0 * r)
    return N[20, 31] == 65536 * n and abs(S - 2 * math.pi) < 0.5 / r and N.sum() == N[20, 31]


def check_window_and_threshold():
    """sigma(r) = 0.05 r + 0.25: r = 20 gives sigma 1.25 and a 9x9 window;
    a hotspot at (+2, +1) from a spike sees the spike through the Gaussian
    weight exp(-5 / (2 sigma^2)); votes equal to the threshold are not hot."""
    sa, sb = float(np.float32(0.05)), float(np.float32(0.25))
    Q = O.smoothing_weights(20, sa, sb)
    sg = sa * 20 + sb
    A = np.zeros((40, 40), dtype=np.int64)
    A[10, 10] = 50
    A[11, 12] = 4
    A[30, 30] = 3
    N = O.smooth_hot(A, Q, 3)
    w = math.exp(-5.0 / (2 * sg * sg))
    return (Q.shape == (9, 9) and abs(N[11, 12] - (65536 * 4 + 50 * 65536 * w)) <= 50
            and N[30, 30] == 0)


def check_smooth_hot_brute_force(seed=11):
    """N(v) = sum over the window of Q(d) A(v + d), zero outside the frame,
    at every hotspot A(v) > T and 0 elsewhere: pure loops on a small random
    accumulator whose hotspots touch every border."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, 7, size=(9, 11)).astype(np.int64)
    Q = O.smoothing_weights(30, float(np.float32(0.05)), float(np.float32(0.25)))   # sigma 1.75, 13 x 13
    Rs = (Q.shape[0] - 1) // 2
    T = 3
    H, W = A.shape
    N = O.smooth_hot(A, Q, T)
    for y in range(H):
        for x in range(W):
            want = 0
            if A[y, x] > T:
                for dy in range(-Rs, Rs + 1):
                    for dx in range(-Rs, Rs + 1):
                        if 0 <= y + dy < H and 0 <= x + dx < W:
                            want += int(Q[dy + Rs, dx + Rs]) * int(A[y + dy, x + dx])
            if int(N[y, x]) != want:
                return False
    return bool((A > T).any() and (A <= T).any())


def check_peaks_brute_force(seed=12):
    """The 3 x 3 x 3 maximum with exact S = N / r comparisons and ties given
    to the first voxel in (r, y, x) order, by loops over Fractions on three
    small levels with many equal values; out-of-frame neighbours score 0."""
    from fractions import Fraction
    rng = np.random.default_rng(seed)
    r = 10
    levels = {dr: rng.choice([0, 400000, 500000], size=(6, 7)).astype(np.int64) for dr in (-1, 1)}
    levels[0] = rng.choice([0, 600000, 650000, 660000, 715000], size=(6, 7)).astype(np.int64)
    # exactly equal S across levels: the level below precedes (strict), the level above follows
    for (y, x), dr in (((2, 3), -1), ((4, 1), -1), ((1, 5), 1), ((3, 2), 1)):
        levels[dr][y, x] = levels[0][y, x] * (r + dr) // r
    p = small_params(peak_frac=0.15)
    got = sorted(O.find_peaks_level(levels[-1], levels[0], levels[1], r, p))
    thr = O.peak_threshold(p.peak_frac, r)
    H, W = levels[0].shape
    want = []
    for y in range(H):
        for x in range(W):
            n = int(levels[0][y, x])
            if not float(n) > thr:
                continue
            s = Fraction(n, r)
            ok = True
            for dr in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if (dr, dy, dx) == (0, 0, 0):
                            continue
                        yy, xx = y + dy, x + dx
                        sn = Fraction(int(levels[dr][yy, xx]), r + dr) if 0 <= yy < H and 0 <= xx < W else 0
                        first = (dr, dy, dx) < (0, 0, 0)
                        ok = ok and (s > sn if first else s >= sn)
            if ok:
                want.append((x, y, r, n))
    return got == sorted(want) and len(want) > 0


def check_fringes_suppressed_at_ring_scale():
    """Results: the thick outer ring admits scale selection; a Gaussian at
    about its scale suppresses the thinner inner rings.  A ring of R = 40
    with three inner fringes (period 4 px, amplitude halving) gives exactly
    one ring at sigma = 2; at sigma = 0.7 the fringes come out as extra
    concentric rings."""
    img = synth._render(160, 160, np.array([[80.3, 79.6, 40.0]]), synth._fringed_ring(600.0, 1.5, 3), 400.0)
    img = np.clip(np.rint(img), 0, 4095).astype(np.uint16)
    base = dict(synth.PLAIN_FULL_PARAMS, r_min=8, r_max=60)
    one = O.detect(img, O.Params.make(**base)).rings
    many = O.detect(img, O.Params.make(**dict(base, sigma=0.7))).rings
    return (len(one) == 1 and abs(float(one["r"][0]) - 40.0) < 0.1
            and abs(float(one["cx"][0]) - 80.3) < 0.1 and abs(float(one["cy"][0]) - 79.6) < 0.1
            and len(many) >= 2 and all(abs(float(a - b)) < 0.5 for a, b in zip(many["cx"], many["cx"][::-1])))


def check_clean_ring_score():
    img = ring_image(120, 120, 60.2, 59.7, 25.0)
    p = small_params(r_min=15, r_max=35)
    res = O.detect(img, p)
    return len(res.rings) == 1 and 5.0 < res.rings["score"][0] < 7.5 and int(res.rings["ir"][0]) in (24, 25, 26)


# ---------------------------------------------------------------- O8
def check_tie_break():
    p = small_params(r_min=5, r_max=7, peak_frac=0.0)
    H = W = 12
    Ns = {r: np.zeros((H, W), dtype=np.int64) for r in range(4, 9)}
    Ns[6][5, 5] = Ns[6][5, 6] = 6 * 1000      # equal S at the same level
    Ns[6][2, 2] = 6 * 500
    Ns[5][2, 3] = 5 * 500                      # equal S one level down, earlier in order
    peaks = []
    for r in (5, 6, 7):
        peaks += O.find_peaks_level(Ns[r - 1], Ns[r], Ns[r + 1], r, p)
    return sorted(peaks) == sorted([(5, 5, 6, 6000), (3, 2, 5, 2500)])


def check_peaks_only_in_range():
    p = small_params(r_min=5, r_max=7, peak_frac=0.0)
    Ns = {r: np.zeros((8, 8), dtype=np.int64) for r in range(4, 9)}
    Ns[4][3, 3] = 4 * 900           # global max below r_min
    Ns[5][3, 3] = 5 * 100
    Ns[8][0, 0] = 8 * 100           # above r_max
    Ns[7][0, 0] = 7 * 50            # corner voxel, neighbours out of image count as 0
    peaks = []
    for r in (5, 6, 7):
        peaks += O.find_peaks_level(Ns[r - 1], Ns[r], Ns[r + 1], r, p)
    return peaks == []


def check_corner_peak():
    p = small_params(r_min=5, r_max=7, peak_frac=0.0)
    Ns = {r: np.zeros((8, 8), dtype=np.int64) for r in range(4, 9)}
    Ns[6][0, 7] = 6 * 10
    peaks = []
    for r in (5, 6, 7):
        peaks += O.find_peaks_level(Ns[r - 1], Ns[r], Ns[r + 1], r, p)
    return peaks == [(7, 0, 6, 60)]


def ring_set(res):
    return sorted(zip(res.rings["ix"].tolist(), res.rings["iy"].tolist(), res.rings["ir"].tolist()))


def check_translation():
    f = synth.plain_small(seed=2001, H=160, W=160, n_rings=3)
    p = O.Params.make(**dict(f.params, r_max=30))
    big = np.full((200, 190), 40, dtype=np.uint8)
    big[:160, :160] = f.image
    a = O.detect(big, p)
    big2 = np.full((200, 190), 40, dtype=np.uint8)
    big2[17:177, 23:183] = f.image
    b = O.detect(big2, p)
    ra = [(x + 23, y + 17, r) for x, y, r in ring_set(a) if 45 <= x <= 120 and 45 <= y <= 120]
    rb = [(x, y, r) for x, y, r in ring_set(b) if 45 + 23 <= x <= 120 + 23 and 45 + 17 <= y <= 120 + 17]
    return len(ra) >= 1 and ra == rb


def check_rot90():
    f = synth.plain_small(seed=2002, H=128, W=128, n_rings=4)
    p = O.Params.make(**dict(f.params, r_max=30))
    a = O.detect(f.image, p)
    b = O.detect(np.ascontiguousarray(np.rot90(f.image)), p)
    # np.rot90 (counter-clockwise): new[y', x'] = old[x', W-1-y'] -> (x, y) maps to (y, W-1-x)
    W = f.image.shape[1]
    ra = sorted((y, W - 1 - x, r) for x, y, r in ring_set(a))
    return len(ra) >= 4 and ra == ring_set(b)


# ---------------------------------------------------------------- O9
def check_kasa_exact_circle():
    pts = []
    for u, v in [(3.5, 0.5), (0.5, 3.5), (2.5, 2.5)]:
        for su in (1, -1):
            for sv in (1, -1):
                pts.append((u * su + 0.5, v * sv + 0.5))
    pts = np.array(sorted(set(pts))) + np.array([100.0, 50.0])
    pts = pts.astype(np.int64)
    cx, cy, r, n, fl = O.kasa_fit(pts, 100, 50, 4)
    return fl == 0 and n == 12 and abs(cx - 100.5) < 1e-12 and abs(cy - 50.5) < 1e-12 and abs(r - math.sqrt(12.5)) < 1e-12


def check_kasa_failures():
    line = np.array([[i, 7] for i in range(10)], dtype=np.int64)
    few = np.array([[0, 5], [5, 0], [-5, 0], [0, -5]], dtype=np.int64)
    return O.kasa_fit(line, 0, 7, 3)[4] == O.FIT_FAIL and O.kasa_fit(few, 0, 0, 5)[4] == O.FIT_FAIL


def check_annulus_inclusive():
    pts = np.array([[0, 7], [0, 3], [0, 8], [0, 2], [0, 5]], dtype=np.int64)
    m = O.annulus_members(pts, 0, 0, 5, 2.0)
    return sorted(m[:, 1].tolist()) == [3, 5, 7]


# ---------------------------------------------------------------- coarse parameter space
def check_coarse_cell_is_nearest_centre():
    """In a coarse parameter space a vote at a goes to the cell whose centre
    c u is nearest, a cell covering [c u - c/2, c u + c/2) (so a tie goes to
    the upper cell), brute force over candidate cells; c = 1 is the pixel
    rule.  Radius 1 keeps s r X exact so that a is known exactly."""
    rng = np.random.default_rng(11)
    for c in (1, 2, 4):
        xs = rng.integers(0, 40, 400).astype(np.int64)
        X = np.concatenate([rng.integers(-8, 9, 200) / 8.0, rng.uniform(-1, 1, 200)])  # exact half-cells too
        ys = np.full_like(xs, 3)
        Y = np.zeros_like(X)
        bx, by = O.cast_votes(xs, ys, X, Y, 1, 64, 64, c)
        exp = []
        for s in (1, -1):
            for x0, dx in zip(xs, X):
                a = float(x0) + s * dx
                best = None
                for u in range(-3, 70):
                    lo, hi = c * u - c / 2.0, c * u + c / 2.0
                    if lo <= a < hi:
                        best = u
                if best is not None and 0 <= best < -(-64 // c):
                    exp.append(best)
        if sorted(bx.tolist()) != sorted(exp) or not np.all(by == (3 + c // 2) // c):
            return False
    return True


def check_coarse_weights_subsample_fine():
    """The coarse window is the same Gaussian measured in cells: Q^c(du, dv)
    = Q^1(c du, c dv) wherever both windows hold the tap, and its half-width
    is ceil(3 sigma(r) / c)."""
    a, b = np.float32(0.05), np.float32(0.25)
    for r in (8, 20, 41, 97):
        Q1 = O.smoothing_weights(r, a, b)
        R1 = (len(Q1) - 1) // 2
        for c in (2, 4):
            Qc = O.smoothing_weights(r, a, b, c)
            Rc = (len(Qc) - 1) // 2
            if Rc != math.ceil(3.0 * (0.05 * r + 0.25) / c - 1e-9):
                return False
            for du in range(-Rc, Rc + 1):
                for dv in range(-Rc, Rc + 1):
                    if abs(c * du) <= R1 and abs(c * dv) <= R1 and Qc[dv + Rc, du + Rc] != Q1[c * dv + R1, c * du + R1]:
                        return False
    return True


def check_coarse_spike_scores_two_pi():
    """An ideal ring's round(2 pi r) votes in one cell still score 2 pi: the
    coarse window also peaks at 2^16."""
    r = 30
    for c in (2, 4):
        Q = O.smoothing_weights(r, np.float32(0.05), np.float32(0.25), c)
        A = np.zeros((32, 32), dtype=np.int64)
        n = int(round(2 * math.pi * r))
        A[10, 15] = n
        N = O.smooth_hot(A, Q, 3)
        if not (N[10, 15] == 65536 * n and N.sum() == N[10, 15]):
            return False
    return True


def check_coarse_truth():
    """Cells of 2 px: every true ring of the small synthetic frame is found
    with its peak centre within one cell and its radius within 1 px, and the
    fit recovers the centre to a fraction of a pixel."""
    f = synth.plain_small()
    res = O.detect(f.image, O.Params.make(coarse=2, **f.params))
    got = np.stack([res.rings["ix"], res.rings["iy"], res.rings["ir"]], 1).astype(float)
    fit = np.stack([res.rings["cx"], res.rings["cy"]], 1)
    if len(got) != len(f.rings) or np.any(got[:, :2] % 2 != 0):
        return False
    for cx, cy, R in f.rings:
        m = (np.abs(got[:, :2] - [cx, cy]).max(1) <= 2.0) & (np.abs(got[:, 2] - R) <= 1.0)
        if not m.any() or np.abs(fit[m] - [cx, cy]).max() > 0.5:
            return False
    return True


PINS = {name[6:]: fn for name, fn in dict(globals()).items() if name.startswith("check_")}


@pytest.mark.parametrize("sigma", [1.0, 1.5, 2.0, 2.5])
def test_taps_are_gaussian(sigma):
    assert check_taps_are_gaussian(sigma)


@pytest.mark.parametrize("name", sorted(k for k in PINS if k != "taps_are_gaussian"))
def test_pin(name):
    assert PINS[name]()
