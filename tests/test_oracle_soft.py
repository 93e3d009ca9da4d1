"""Pins of the soft-score oracle (oracle/soft.py) against facts that do not
come from the oracle itself: the independently pinned integer Hessian, a
closed form, symmetry, translation invariance, central finite differences
and the location of the score's maximum on a clean synthetic ring."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ringdet as R
from oracle import soft as S
from paper_1310_1371_gb300 import synth

P = S.SoftParams.make(**synth.DIFF_PARAMS)


def ring_image(H, W, cx, cy, r, seed=0, noise=2.0):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = 40 + 120 * np.exp(-0.5 * ((np.hypot(xx - cx, yy - cy) - r) / 1.5) ** 2)
    return (img + rng.normal(0, noise, img.shape)).astype(np.float32)


def test_float_hessian_equals_integer_path():
    rng = np.random.default_rng(1)
    img = rng.integers(0, 4096, size=(40, 52)).astype(np.uint16)
    for sigma in (1.0, 2.0, 3.0):
        a = S.hessian_float(img.astype(np.float64), sigma)
        b = R.hessian(img, sigma)
        for u, v in zip(a, b):
            assert np.allclose(u, v, rtol=1e-11, atol=1e-11 * np.abs(v).max())


def twelve_points(c0=20.0):
    # the 12 integer points at distance 5 from (c0, c0), radial directions
    pts = [(5, 0), (-5, 0), (0, 5), (0, -5), (3, 4), (3, -4), (-3, 4), (-3, -4),
           (4, 3), (4, -3), (-4, 3), (-4, -3)]
    xs = np.array([c0 + a for a, b in pts], dtype=np.int64)
    ys = np.array([c0 + b for a, b in pts], dtype=np.int64)
    X = np.array([a / 5.0 for a, b in pts])
    Y = np.array([b / 5.0 for a, b in pts])
    flip = (X < 0) | ((X == 0) & (Y < 0))
    X, Y = np.where(flip, -X, X), np.where(flip, -Y, Y)
    k = np.full(len(pts), P.ridge_thresh - 60 * P.temperature)  # m = logistic(60) = 1 - 9e-27
    return S.Ridges(xs, ys, k, X, Y, np.ones(len(pts), bool))


def test_closed_form_twelve_points():
    rd = twelve_points()
    # every point votes exactly onto the centre with one sign (bil = 1, Gaussian = 1);
    # the other sign lands 10 px away: exp(-100 / (2 sigma(5)^2)) = exp(-200)
    sc = S.soft_score(rd, np.array([[20.0, 20.0, 5.0]]), P, 41, 41)
    assert abs(sc[0] - 12.0 / 5.0) < 1e-12


def test_symmetry_and_zero_gradient():
    rd = twelve_points()
    d = 0.137
    a = S.soft_score(rd, np.array([[20.0 + d, 20.0, 5.0], [20.0 - d, 20.0, 5.0],
                                   [20.0, 20.0 + d, 5.0], [20.0, 20.0 - d, 5.0]]), P, 41, 41)
    assert abs(a[0] - a[1]) < 1e-12 and abs(a[2] - a[3]) < 1e-12 and abs(a[0] - a[2]) < 1e-12
    assert a[0] < 12.0 / 5.0


def test_numpy_and_torch_forwards_agree():
    img = ring_image(64, 64, 31.3, 30.7, 15.2)
    rd = S.ridges_float(img, P)
    rings = np.array([[31.3, 30.7, 15.2], [30.0, 32.0, 14.0], [20.5, 40.2, 9.7]])
    a = S.soft_score(rd, rings, P, 64, 64)
    b = S.soft_score_torch(torch.tensor(img, dtype=torch.float64), torch.tensor(rings), rd, P).numpy()
    assert np.allclose(a, b, rtol=1e-12, atol=0)
    assert len(rd.xs) > 50 and a[0] > 4.0


def test_parameter_gradient_matches_central_differences():
    img = ring_image(64, 64, 31.3, 30.7, 15.2)
    rings = np.array([[31.1, 30.9, 15.0], [32.0, 29.5, 15.6]])
    sc, dimg, drg, rd = S.soft_grads(img, rings, P)
    h = 1e-5
    for i in range(len(rings)):
        for j in range(3):
            rp, rm = rings.copy(), rings.copy()
            rp[i, j] += h
            rm[i, j] -= h
            fd = (S.soft_score(rd, rp, P, 64, 64)[i] - S.soft_score(rd, rm, P, 64, 64)[i]) / (2 * h)
            assert abs(fd - drg[i, j]) <= 1e-6 * max(1.0, abs(drg[i, j])), (i, j, fd, drg[i, j])


def test_image_gradient_matches_central_differences():
    img = ring_image(48, 48, 23.4, 24.1, 10.3, noise=1.0)
    rings = np.array([[23.2, 24.0, 10.5]])
    sc, dimg, drg, rd = S.soft_grads(img, rings, P)
    base = torch.tensor(img, dtype=torch.float64)
    rg = torch.tensor(rings)
    big = np.argsort(-np.abs(dimg).ravel())[:4]
    h = 1e-4
    for flat in list(big) + [int(np.argmin(np.abs(dimg)))]:
        y, x = divmod(int(flat), 48)
        e = torch.zeros_like(base)
        e[y, x] = h
        fd = (S.soft_score_torch(base + e, rg, rd, P)[0] - S.soft_score_torch(base - e, rg, rd, P)[0]).item() / (2 * h)
        assert abs(fd - dimg[y, x]) <= 1e-6 * max(1e-3, abs(dimg).max()), (y, x, fd, dimg[y, x])
    assert np.abs(dimg).max() > 0


def test_translation_invariance():
    img = ring_image(64, 64, 31.3, 30.7, 12.2, seed=3)
    big = np.full((80, 90), 40.0, dtype=np.float32)
    big[9:73, 17:81] = img
    rd_a = S.ridges_float(img, P)
    rd_b = S.ridges_float(big, P)
    inner = (rd_b.xs >= 17 + 14) & (rd_b.xs < 81 - 14) & (rd_b.ys >= 9 + 14) & (rd_b.ys < 73 - 14)
    keep_a = (rd_a.xs >= 14) & (rd_a.xs < 50) & (rd_a.ys >= 14) & (rd_a.ys < 50)
    sub = lambda rd, k: S.Ridges(rd.xs[k], rd.ys[k], rd.k[k], rd.X[k], rd.Y[k], rd.use1[k])
    a = S.soft_score(sub(rd_a, keep_a), np.array([[31.3, 30.7, 12.2]]), P, 64, 64)
    b = S.soft_score(sub(rd_b, inner), np.array([[31.3 + 17, 30.7 + 9, 12.2]]), P, 80, 90)
    assert np.allclose(a, b, rtol=1e-10)


def test_maximum_near_truth():
    cx, cy, r = 31.37, 30.71, 15.23
    img = ring_image(64, 64, cx, cy, r, noise=0.5)
    rd = S.ridges_float(img, P)
    best, arg = -1.0, None
    for dx in np.linspace(-0.6, 0.6, 13):
        for dy in np.linspace(-0.6, 0.6, 13):
            for dr in np.linspace(-0.6, 0.6, 13):
                v = S.soft_score(rd, np.array([[cx + dx, cy + dy, r + dr]]), P, 64, 64)[0]
                if v > best:
                    best, arg = v, (dx, dy, dr)
    assert max(abs(arg[0]), abs(arg[1])) <= 0.2 and abs(arg[2]) <= 0.35, arg


def test_closed_form_offset_centre():
    """All twelve votes land exactly on (20, 20): the score at c = (20 + d, 20)
    is (1/5) exp(-d^2 / (2 sigma(5)^2)) times the sum of the twelve points'
    annulus weights exp(-(|p - c| - 5)^2 / 2), sigma(5) = 0.05 * 5 + 0.25 and
    the annulus's standard deviation w / 2 = 1 px; each point (5 cos t, 5 sin t)
    from (20, 20) lies sqrt(25 - 10 d cos t + d^2) from c."""
    rd = twelve_points()
    sig = P.sig_a * 5.0 + P.sig_b
    cosines = [1, -1, 0, 0, 0.6, 0.6, -0.6, -0.6, 0.8, 0.8, -0.8, -0.8]
    for d in (0.1, 0.3, 0.7):
        sc = S.soft_score(rd, np.array([[20.0 + d, 20.0, 5.0]]), P, 41, 41)[0]
        ann = sum(math.exp(-((math.sqrt(25 - 10 * d * ct + d * d) - 5.0) ** 2) / 2.0) for ct in cosines)
        assert ann < 12.0
        assert abs(sc - ann / 5.0 * math.exp(-d * d / (2 * sig * sig))) < 1e-12


def test_annulus_keeps_pixels_off_the_circle_out():
    """A ridge pixel 2 px outside the circle whose vote lands on the centre
    (a neighbouring ring's pixel pointing at c) counts with weight exp(-2)
    (2 standard deviations of the annulus); a pixel on the circle counts fully."""
    k = np.array([P.ridge_thresh - 60 * P.temperature] * 2)
    # (27, 20): 7 px from c = (20, 20) with rho = 5, X = (1, 0): its vote lands at (22, 20);
    # (25, 20): on the circle, its vote lands on c
    for x, want in ((27, math.exp(-2.0) * math.exp(-4.0 / (2 * (P.sig_a * 5 + P.sig_b) ** 2))), (25, 1.0)):
        rd = S.Ridges(np.array([x]), np.array([20]), k[:1], np.array([1.0]), np.array([0.0]), np.array([True]))
        sc = S.soft_score(rd, np.array([[20.0, 20.0, 5.0]]), P, 41, 41)[0]
        assert abs(sc * 5.0 - want) < 1e-12, (x, sc * 5.0, want)  # the other sign's vote is >= 10 px away


def test_closed_form_bilinear_split():
    """One ridge pixel at (10, 10) with X = (1, 0) votes at (12.5, 10) for
    rho = 2.5: half a vote on (12, 10) and half on (13, 10), each 0.5 px from
    c = (12.5, 10); the other sign lands 5 px away."""
    rd = S.Ridges(np.array([10]), np.array([10]), np.array([P.ridge_thresh - 60 * P.temperature]),
                  np.array([1.0]), np.array([0.0]), np.array([True]))
    sig = P.sig_a * 2.5 + P.sig_b
    sc = S.soft_score(rd, np.array([[12.5, 10.0, 2.5]]), P, 30, 30)[0]
    far = 0.5 * math.exp(-(5.5 ** 2) / (2 * sig * sig)) + 0.5 * math.exp(-(4.5 ** 2) / (2 * sig * sig))
    assert abs(sc - (math.exp(-0.25 / (2 * sig * sig)) + far) / 2.5) < 1e-14


def test_unnormalised_mass_is_stationary_at_the_true_radius():
    """For the symmetric twelve-point ring, rho * Score is even in rho - 5
    (the votes land at c0 -/+ (rho - 5) X for opposite directions) when the
    window width is fixed, so its rho-derivative vanishes at the true radius, while Score itself still
    decreases there: the 1/rho normalisation biases a refinement of rho.
    This is why refinement ascends rho * Score."""
    rd = twelve_points()
    h = 1e-5
    # sigma held at sigma(5) (sig_a = 0): a growing sigma(rho) would add mass
    # from the bilinear neighbours on one side only
    P0 = S.SoftParams(P.sigma, P.ridge_thresh, 0.0, P.sig_a * 5.0 + P.sig_b)
    mass = lambda rho: rho * S.soft_score(rd, np.array([[20.0, 20.0, rho]]), P0, 41, 41)[0]
    dm = (mass(5.0 + h) - mass(5.0 - h)) / (2 * h)
    ds = (mass(5.0 + h) / (5.0 + h) - mass(5.0 - h) / (5.0 - h)) / (2 * h)
    assert abs(dm) < 1e-8
    # d(T / rho)/drho = -T / rho^2 with T = 12; the votes sit h off the grid
    # point at rho = 5 +/- h, so T = 12 - O(h) on both sides
    assert abs(ds + 12.0 / 25.0) < 1e-4


def test_votes_beyond_nine_sigma_are_negligible():
    """The GPU leaves out votes farther than 9 sigma(rho) + 1.5 px from the
    centre, and ridge pixels farther than 9 annulus standard deviations from
    the circle.  On the synthetic soft-score frames their total contribution,
    computed term by term from the oracle's ridge set (without the annulus
    factor, an upper bound, for the first kind), is below 1e-12 of the score
    (the tolerances are 1e-5 for scores and 1e-4 for gradients)."""
    fr = synth.diff_frames(2, seed=2011, H=128, W=128, n_rings=4)
    sp = S.SoftParams.make(**synth.DIFF_PARAMS)
    for f in fr:
        rd = S.ridges_float(f.image.astype(np.float64), sp)
        m = S.logistic((sp.ridge_thresh - rd.k) / sp.temperature)
        H, W = f.image.shape
        full = S.soft_score(rd, f.rings, sp, H, W)
        for (cx, cy, rho), score in zip(f.rings, full):
            sig = sp.sig_a * rho + sp.sig_b
            cut = 9.0 * sig + 1.5
            left_out = 0.0
            for s in (1.0, -1.0):
                vx = rd.xs + s * rho * rd.X
                vy = rd.ys + s * rho * rd.Y
                far = (vx - cx) ** 2 + (vy - cy) ** 2 > cut * cut
                x0, y0 = np.floor(vx[far]), np.floor(vy[far])
                for ox in (0, 1):
                    for oy in (0, 1):
                        d2 = (x0 + ox - cx) ** 2 + (y0 + oy - cy) ** 2
                        left_out += float(np.sum(m[far] * np.exp(-d2 / (2 * sig * sig))))
            # pixels off the circle by more than 9 annulus standard deviations
            sa = sp.annulus_sigma
            dist = np.hypot(rd.xs - cx, rd.ys - cy)
            off = np.abs(dist - rho) > 9.0 * sa
            a_off = np.exp(-((dist[off] - rho) ** 2) / (2 * sa * sa))
            left_out += float(np.sum(2.0 * m[off] * a_off))   # every vote's weights sum to at most 1 per sign
            assert score > 0 and left_out / rho <= 1e-12 * score, (left_out, score)
