"""FP64 CPU oracle of the ridge-directed ring detector.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
definition of what the detector computes, written from the paper (Afik 2015,
"Robust and highly performant ring detection algorithm for 3d particle
tracking using 2d microscope imaging": Results, "Directed ridge detection &
votes collection", "Local maxima detection in a noisy parameter space",
"Ridge points classification & sub-pixel accuracy"; Methods, "Algorithm
implementation"; Supplementary "Detailed algorithm", steps 1-5 and
"Additional notes").  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path and imports nothing from the package.

Every step is dense and unoptimised: no vote sorting, no level recycling, no
undo lists (the paper's speed devices, which do not change the result).
Wherever the paper is silent the reading used is stated at the step.

Numerics.  Parameters arrive as float32 (the C struct holds floats) and are
widened to float64.  Smoothing and second derivatives of integer frames are
exact integer arithmetic (the Gaussian taps are quantised, step O1), so the
Hessian is known exactly and then divided once into float64.  Everything after
that is float64, evaluated in the order written below; each line is one
IEEE-754 operation so that the order is unambiguous.
"""
from __future__ import annotations

import dataclasses
import math
import numpy as np

GAUSS_BITS = 19          # O1: Gaussian taps are integers summing to ~2^19
SMOOTH_BITS = 16         # O7: level-smoothing weights are integers, peak 2^16
FIT_FAIL = 1             # ring flag: fewer than 5 annulus points or singular fit
MIN_FIT_POINTS = 5


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    sigma: float          # Gaussian scale (Results, scale selection)
    r_min: int            # radius search range (Results, voting)
    r_max: int
    ridge_thresh: float   # curvature threshold tau <= 0 (Detailed algorithm, step 2)
    peak_frac: float      # float threshold = peak_frac * 2 pi (step 4)
    vote_thresh: int      # integer hotspot threshold (step 4)
    annulus_w: float      # annulus half-width in px (step 5; not given in the paper)
    sig_a: float          # sigma(r) = sig_a * r + sig_b (Methods: 0.05, 0.25)
    sig_b: float
    features: str = "ridge"   # "ridge" (the method) or "edge" (Additional notes: directed edges)
    edge_thresh: float = 0.0  # gradient-magnitude threshold of the edge variant (intensity / px)
    coarse: int = 1           # accumulator cell edge in px: 1, 2 or 4 (Additional notes: a lower
                              # resolution of the circle parameter space)

    @staticmethod
    def make(**kw) -> "Params":
        f32 = lambda v: float(np.float32(v))
        return Params(sigma=f32(kw["sigma"]), r_min=int(kw["r_min"]), r_max=int(kw["r_max"]),
                      ridge_thresh=f32(kw["ridge_thresh"]), peak_frac=f32(kw["peak_frac"]),
                      vote_thresh=int(kw["vote_thresh"]), annulus_w=f32(kw.get("annulus_w", 2.0)),
                      sig_a=f32(kw.get("sig_a", 0.05)), sig_b=f32(kw.get("sig_b", 0.25)),
                      features=kw.get("features", "ridge"), edge_thresh=f32(kw.get("edge_thresh", 0.0)),
                      coarse=int(kw.get("coarse", 1) or 1))


# --------------------------------------------------------------------------
# O1  Gaussian smoothing (Results: scale selection suppresses the thin inner
#     rings; Methods: Gaussian convolution before the Sobel derivatives;
#     Detailed algorithm step 1)
# --------------------------------------------------------------------------
def gaussian_radius(sigma: float) -> int:
    """Kernel half-width R_g = ceil(4 sigma) (the paper gives no truncation)."""
    return int(math.ceil(4.0 * sigma))


def gaussian_taps(sigma: float) -> np.ndarray:
    """Integer taps Q_i = floor(2^19 g_i + 1/2), g_i = e_i / sum(e),
    e_i = exp(-i^2 / (2 sigma^2)), |i| <= R_g.  The smoothing operator is
    (1/S) sum_i Q_i f(x+i) with S = sum(Q): a normalised Gaussian quantised to
    multiples of 2^-19, which makes smoothing of integer frames exact.  The
    quantisation is fine enough that the rings equal those of the
    real-valued Gaussian (``detect_definition``), and coarse enough that the
    exact Hessian of a 16-bit frame fits int64 (|H'| < 2^60)."""
    R = gaussian_radius(sigma)
    i = np.arange(-R, R + 1, dtype=np.float64)
    den = 2.0 * sigma * sigma
    e = np.exp(-(i * i) / den)
    tot = 0.0
    for v in e:                      # left-to-right sum
        tot = tot + v
    g = e / tot
    return np.floor(g * float(1 << GAUSS_BITS) + 0.5).astype(np.int64)


def _correlate1d_int(f: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """Exact integer correlation along one axis with reflect-101 borders
    (index -1 maps to 1, W maps to W-2)."""
    R = (len(taps) - 1) // 2
    pad = [(0, 0), (0, 0)]
    pad[axis] = (R, R)
    fp = np.pad(f, pad, mode="reflect")          # numpy 'reflect' == reflect-101
    out = np.zeros(f.shape, dtype=np.int64)
    n = f.shape[axis]
    for j, t in enumerate(taps):
        if t == 0:
            continue
        sl = [slice(None), slice(None)]
        sl[axis] = slice(j, j + n)
        out += int(t) * fp[tuple(sl)]
    return out


def smooth_int(image: np.ndarray, sigma: float) -> tuple[np.ndarray, int]:
    """L' = sum_i sum_j Q_i Q_j I(y+i, x+j) exactly (int64).  The smoothed
    image is L = L' / S^2."""
    Q = gaussian_taps(sigma)
    I = image.astype(np.int64)
    Lp = _correlate1d_int(I, Q, axis=1)
    Lp = _correlate1d_int(Lp, Q, axis=0)
    S = int(Q.sum())
    return Lp, S


# --------------------------------------------------------------------------
# O2  5x5 second-order Sobel derivatives of the smoothed image (Methods;
#     Detailed algorithm step 1), scaled by 1/64 so that each is the true
#     second derivative on quadratics.
# --------------------------------------------------------------------------
SOBEL_S = np.array([1, 4, 6, 4, 1], dtype=np.int64)     # smoothing
SOBEL_D1 = np.array([-1, -2, 0, 2, 1], dtype=np.int64)  # first derivative
SOBEL_D2 = np.array([1, 0, -2, 0, 1], dtype=np.int64)   # second derivative


def hessian_int(Lp: np.ndarray):
    """Exact integer second-derivative stencils of L' with reflect-101
    borders: Hxx' = (d2_x (x) s_y) * L', Hyy' = (s_x (x) d2_y) * L',
    Hxy' = (d1_x (x) d1_y) * L'."""
    hxx = _correlate1d_int(_correlate1d_int(Lp, SOBEL_D2, 1), SOBEL_S, 0)
    hyy = _correlate1d_int(_correlate1d_int(Lp, SOBEL_S, 1), SOBEL_D2, 0)
    hxy = _correlate1d_int(_correlate1d_int(Lp, SOBEL_D1, 1), SOBEL_D1, 0)
    return hxx, hyy, hxy


def hessian_scale(S: int) -> float:
    """D = 64 S^2: Lxx = Hxx' / D (64 from the Sobel normalisation, S^2 from
    the two smoothing passes)."""
    return float(64 * S * S)


def hessian(image: np.ndarray, sigma: float):
    """Lxx, Lyy, Lxy in float64: each exact integer H' rounded to the
    nearest float64 (exact below 2^53), then one correctly rounded
    division by D."""
    Lp, S = smooth_int(image, sigma)
    hxx, hyy, hxy = hessian_int(Lp)
    D = hessian_scale(S)
    return hxx.astype(np.float64) / D, hyy.astype(np.float64) / D, hxy.astype(np.float64) / D


# --------------------------------------------------------------------------
# O3  Principal curvature k- (smaller Hessian eigenvalue) and its direction
#     X- (Results: ridge descriptor; Detailed algorithm steps 1-2).
# --------------------------------------------------------------------------
def eigen(a: np.ndarray, c: np.ndarray, b: np.ndarray):
    """Closed form for H = [[a, b], [b, c]] (a = Lxx, c = Lyy, b = Lxy).

    k = (a + c)/2 - sqrt(((a - c)/2)^2 + b^2).  Eigenvector candidates
    v1 = (b, k - a) and v2 = (k - c, b); the one with the larger squared norm
    (v1 on a tie) is normalised.  Sign: X > 0, or X == 0 and Y > 0.
    Returns k, X, Y and a mask of degenerate pixels (both candidates zero:
    b == 0 and a == c), which are never ridges."""
    half_tr = (a + c) * 0.5
    half_df = (a - c) * 0.5
    rad = np.sqrt(half_df * half_df + b * b)
    k = half_tr - rad
    v1x, v1y = b, k - a
    v2x, v2y = k - c, b
    n1 = v1x * v1x + v1y * v1y
    n2 = v2x * v2x + v2y * v2y
    use1 = n1 >= n2
    vx = np.where(use1, v1x, v2x)
    vy = np.where(use1, v1y, v2y)
    n = np.where(use1, n1, n2)
    degenerate = n == 0.0
    with np.errstate(invalid="ignore", divide="ignore"):
        nrm = np.sqrt(n)
        X = vx / nrm
        Y = vy / nrm
    flip = (X < 0.0) | ((X == 0.0) & (Y < 0.0))
    X = np.where(flip, -X, X)
    Y = np.where(flip, -Y, Y)
    X = np.where(degenerate, 0.0, X)
    Y = np.where(degenerate, 0.0, Y)
    return k, X, Y, degenerate


# --------------------------------------------------------------------------
# O4  Directed-ridge mask (Results: negative least principal curvature that
#     is a local minimum along its own direction; Detailed algorithm step 2).
# --------------------------------------------------------------------------
def bilinear(k: np.ndarray, qx: float, qy: float) -> float:
    """Bilinear sample of k at (qx, qy), 0 <= qx <= W-1, 0 <= qy <= H-1."""
    H, W = k.shape
    x0 = math.floor(qx)
    y0 = math.floor(qy)
    fx = qx - x0
    fy = qy - y0
    x1 = min(x0 + 1, W - 1)
    y1 = min(y0 + 1, H - 1)
    top = (1.0 - fx) * k[y0, x0] + fx * k[y0, x1]
    bot = (1.0 - fx) * k[y1, x0] + fx * k[y1, x1]
    return (1.0 - fy) * top + fy * bot


def ridge_mask(k, X, Y, degenerate, tau: float) -> np.ndarray:
    """ridge(p) <=> k(p) < tau and k(p) < k~(p + X) and k(p) <= k~(p - X),
    with k~ the bilinear sample at unit distance along X (the paper does not
    say how "local minimum along X" is sampled).  A sample outside
    [0, W-1] x [0, H-1] makes the pixel a non-ridge.  Strict on +X and
    non-strict on -X so that exactly one pixel of a two-pixel plateau wins.
    Vectorised over candidates; each element follows ``bilinear`` exactly."""
    H, W = k.shape
    out = np.zeros((H, W), dtype=bool)
    cy, cx = np.nonzero((k < tau) & ~degenerate)
    if len(cy) == 0:
        return out
    kp = k[cy, cx]
    ok = np.ones(len(cy), dtype=bool)
    fx0 = cx.astype(np.float64)
    fy0 = cy.astype(np.float64)
    for s in (1, -1):
        if s == 1:
            qx = fx0 + X[cy, cx]
            qy = fy0 + Y[cy, cx]
        else:
            qx = fx0 - X[cy, cx]
            qy = fy0 - Y[cy, cx]
        inb = (qx >= 0.0) & (qx <= W - 1) & (qy >= 0.0) & (qy <= H - 1)
        ok &= inb
        qx = np.where(inb, qx, 0.0)
        qy = np.where(inb, qy, 0.0)
        x0f = np.floor(qx)
        y0f = np.floor(qy)
        fx = qx - x0f
        fy = qy - y0f
        x0 = x0f.astype(np.int64)
        y0 = y0f.astype(np.int64)
        x1 = np.minimum(x0 + 1, W - 1)
        y1 = np.minimum(y0 + 1, H - 1)
        top = (1.0 - fx) * k[y0, x0] + fx * k[y0, x1]
        bot = (1.0 - fx) * k[y1, x0] + fx * k[y1, x1]
        kt = (1.0 - fy) * top + fy * bot
        ok &= (kp < kt) if s == 1 else (kp <= kt)
    out[cy, cx] = ok
    return out


# --------------------------------------------------------------------------
# O5  Ridge-directed circle Hough voting (Results: each directed ridge pixel
#     votes for (x, y) +/- r X- for every radius; Additional notes: votes over
#     [r_min - 1, r_max + 1], peaks only inside [r_min, r_max]).
# --------------------------------------------------------------------------
def radius_levels(r_min: int, r_max: int) -> np.ndarray:
    return np.arange(r_min - 1, r_max + 2, dtype=np.int64)


def cell_grid(H: int, W: int, c: int = 1) -> tuple[int, int]:
    """Accumulator cells of a coarse parameter space: ceil(H / c) x ceil(W / c)."""
    return -(-H // c), -(-W // c)


def cast_votes(xs, ys, X, Y, r: int, H: int, W: int, c: int = 1):
    """Both signs vote at every radius.  Vote bin = floor(p + s r X + 1/2)
    per coordinate, each product and sum one float64 operation; votes that
    fall outside the image are discarded.  Returns in-bounds (bx, by).

    Coarse parameter space (Additional notes: a lower resolution of the
    circle parameter space; the paper gives no form, this is the reading):
    cells of c x c px, c a power of two, cell u covering [c u - c/2, c u +
    c/2).  The bin is floor((a + c/2) / c) with a = p + s r X, the sum a +
    c/2 one float64 operation and the division exact; c = 1 is the rule
    above.  A cell is kept when it lies in the cell grid (cell_grid)."""
    Hc, Wc = cell_grid(H, W, c)
    bxs, bys = [], []
    for s in (1, -1):
        sr = float(s * r)
        ax = xs.astype(np.float64) + sr * X
        ay = ys.astype(np.float64) + sr * Y
        bx = np.floor((ax + 0.5 * c) / c).astype(np.int64)
        by = np.floor((ay + 0.5 * c) / c).astype(np.int64)
        keep = (bx >= 0) & (bx < Wc) & (by >= 0) & (by < Hc)
        bxs.append(bx[keep])
        bys.append(by[keep])
    return np.concatenate(bxs), np.concatenate(bys)


def accumulate(bx, by, H: int, W: int) -> np.ndarray:
    A = np.zeros((H, W), dtype=np.int64)
    np.add.at(A, (by, bx), 1)
    return A


# --------------------------------------------------------------------------
# O6, O7  Hotspots, radius-dependent smoothing and 1/r normalisation
#     (Results; Methods: sigma(r) = 0.05 r + 0.25, weights
#     exp{-1/2 (d / sigma)^2}; Detailed algorithm step 4).
# --------------------------------------------------------------------------
def level_sigma(r: int, sig_a: float, sig_b: float) -> float:
    return sig_a * r + sig_b


def smoothing_weights(r: int, sig_a: float, sig_b: float, c: int = 1) -> np.ndarray:
    """Q_r(dy, dx) = floor(2^16 exp(-(dx^2 + dy^2) / (2 sigma(r)^2)) + 1/2)
    on |dx|, |dy| <= R_s = ceil(3 sigma(r)).  Weights peak at 1 (2^16) and
    are not normalised, so that an ideal ring scores 2 pi after 1/r.  In a
    coarse parameter space (cells of c px) the window is the same Gaussian
    measured in cells: sigma(r) / c (exact: c is a power of two)."""
    sg = level_sigma(r, sig_a, sig_b) / c
    Rs = int(math.ceil(3.0 * sg))
    d = np.arange(-Rs, Rs + 1, dtype=np.float64)
    d2 = d[:, None] * d[:, None] + d[None, :] * d[None, :]
    den = 2.0 * sg * sg
    return np.floor(np.exp(-d2 / den) * float(1 << SMOOTH_BITS) + 0.5).astype(np.int64)


def smooth_hot(A: np.ndarray, Qr: np.ndarray, vote_thresh: int) -> np.ndarray:
    """N(v) = sum_d Q_r(d) A(v + d) at hotspots (A(v) > vote_thresh, the
    paper's "surpassed" read as strict), 0 elsewhere; A = 0 outside the
    image.  S = N / (2^16 r)."""
    H, W = A.shape
    Rs = (Qr.shape[0] - 1) // 2
    N = np.zeros((H, W), dtype=np.int64)
    hy, hx = np.nonzero(A > vote_thresh)
    if len(hy) == 0:
        return N
    Ap = np.pad(A, Rs, mode="constant")
    acc = np.zeros(len(hy), dtype=np.int64)
    for dy in range(-Rs, Rs + 1):
        for dx in range(-Rs, Rs + 1):
            q = int(Qr[dy + Rs, dx + Rs])
            if q:
                acc += q * Ap[hy + Rs + dy, hx + Rs + dx]
    N[hy, hx] = acc
    return N


# --------------------------------------------------------------------------
# O8  Float threshold and 3x3x3 local maximum (Results: nearest-neighbour
#     comparison; Detailed algorithm step 4; Additional notes: peaks only in
#     [r_min, r_max]).
# --------------------------------------------------------------------------
def peak_threshold(peak_frac: float, r: int) -> float:
    """S > f 2 pi  <=>  N > ((f * 2 pi) * 2^16) * r, evaluated in that order."""
    two_pi = 2.0 * math.pi
    return ((peak_frac * two_pi) * float(1 << SMOOTH_BITS)) * float(r)


NEIGHBOURS = [(dr, dy, dx) for dr in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
              if (dr, dy, dx) != (0, 0, 0)]


def find_peaks_level(N_lo: np.ndarray, N_mid: np.ndarray, N_hi: np.ndarray, r: int, p: Params) -> list:
    """Peaks at level r given N at levels r-1, r, r+1.  A voxel v = (r, y, x)
    is a peak iff N(v) > thr_r and, for each of its 26 neighbours n,
    S(v) > S(n) when n precedes v in (r, y, x) order and S(v) >= S(n)
    otherwise (ties go to the first voxel in that order).  S comparisons are
    exact: S(v) > S(n) <=> N(v) r_n > N(n) r_v.  Out-of-image neighbours
    have S = 0."""
    H, W = N_mid.shape
    thr = peak_threshold(p.peak_frac, r)
    cy, cx = np.nonzero(N_mid.astype(np.float64) > thr)
    if len(cy) == 0:
        return []
    nv = N_mid[cy, cx]
    ok = np.ones(len(cy), dtype=bool)
    lvl = {-1: N_lo, 0: N_mid, 1: N_hi}
    for dr, dy, dx in NEIGHBOURS:
        yy, xx = cy + dy, cx + dx
        inb = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        nn = np.where(inb, lvl[dr][np.clip(yy, 0, H - 1), np.clip(xx, 0, W - 1)], 0)
        lhs = nv * (r + dr)
        rhs = nn * r
        if (dr, dy, dx) < (0, 0, 0):
            ok &= lhs > rhs
        else:
            ok &= lhs >= rhs
    return [(int(x), int(y), int(r), int(n)) for x, y, n in zip(cx[ok], cy[ok], nv[ok])]


# --------------------------------------------------------------------------
# O9  Annulus classification and circle fit (Results: annulus masks and a
#     best-fit circle per peak; Detailed algorithm step 5).  The fit method
#     is not named in the paper: algebraic least squares (Kasa).
# --------------------------------------------------------------------------
def annulus_members(ridge_xy: np.ndarray, ix: int, iy: int, ir: int, w: float) -> np.ndarray:
    """Ridge pixels with |dist(p, c) - r0| <= w (inclusive; non-exclusive
    across rings)."""
    if len(ridge_xy) == 0:
        return ridge_xy
    u = ridge_xy[:, 0] - ix
    v = ridge_xy[:, 1] - iy
    dist = np.sqrt((u * u + v * v).astype(np.float64))
    keep = np.abs(dist - float(ir)) <= w
    return ridge_xy[keep]


def kasa_fit(pts: np.ndarray, ix: int, iy: int, ir: int):
    """Minimise sum (u^2 + v^2 + D u + E v + F)^2 over integer offsets
    (u, v) = p - c: 3x3 normal equations with exact integer moments, solved
    in float64.  Centre = c + (-D/2, -E/2), radius = sqrt(D^2/4 + E^2/4 - F).
    Fewer than 5 points or a singular system (exact integer determinant 0)
    returns the integer peak with FIT_FAIL."""
    n = len(pts)
    if n < MIN_FIT_POINTS:
        return float(ix), float(iy), float(ir), n, FIT_FAIL
    u = [int(a) - ix for a in pts[:, 0]]
    v = [int(b) - iy for b in pts[:, 1]]
    z = [a * a + b * b for a, b in zip(u, v)]
    Suu = sum(a * a for a in u); Svv = sum(b * b for b in v); Suv = sum(a * b for a, b in zip(u, v))
    Su = sum(u); Sv = sum(v)
    Suz = sum(a * c for a, c in zip(u, z)); Svz = sum(b * c for b, c in zip(v, z)); Sz = sum(z)
    M = [[Suu, Suv, Su], [Suv, Svv, Sv], [Su, Sv, n]]
    det = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
           - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
           + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))
    if det == 0:
        return float(ix), float(iy), float(ir), n, FIT_FAIL
    sol = np.linalg.solve(np.array(M, dtype=np.float64),
                          -np.array([Suz, Svz, Sz], dtype=np.float64))
    D, E, F = sol
    rr = D * D / 4.0 + E * E / 4.0 - F
    if not (rr > 0.0):
        return float(ix), float(iy), float(ir), n, FIT_FAIL
    return ix - D / 2.0, iy - E / 2.0, math.sqrt(rr), n, 0


# --------------------------------------------------------------------------
# the whole path
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Result:
    rings: np.ndarray            # structured: cx, cy, r, ix, iy, ir, score, n_fit, flags
    ridge_xy: np.ndarray         # [n, 2] int64 (x, y), row-major order
    ridge_X: np.ndarray          # [n, 2] float64 direction
    votes_in: int                # in-bounds votes over all levels
    votes_cast: int              # 2 * n_ridge * n_levels
    hotspots: int = 0            # voxels above the integer threshold over all levels
    smooth_macs: int = 0         # sum over hotspots of their smoothing window size
    A: dict | None = None        # level -> raw accumulator (when kept)
    N: dict | None = None        # level -> smoothed accumulator (when kept)


RING_DTYPE = np.dtype([("cx", "f8"), ("cy", "f8"), ("r", "f8"), ("ix", "i8"), ("iy", "i8"),
                       ("ir", "i8"), ("score", "f8"), ("n_fit", "i8"), ("flags", "i8")])


def directed_ridges(image: np.ndarray, p: Params):
    """Steps O1-O4: ridge pixel coordinates (row-major) and their X-."""
    Lxx, Lyy, Lxy = hessian(image, p.sigma)
    k, X, Y, deg = eigen(Lxx, Lyy, Lxy)
    mask = ridge_mask(k, X, Y, deg, p.ridge_thresh)
    ys, xs = np.nonzero(mask)
    return np.stack([xs, ys], axis=1).astype(np.int64), np.stack([X[ys, xs], Y[ys, xs]], axis=1)


# --------------------------------------------------------------------------
# Directed-edge variant (Additional notes: the Hessian is replaced by the
# gradient, whose magnitude, replacing k-, must be a local maximum along the
# gradient direction).  Readings: the gradient is the first-order 5x5 Sobel
# of L' (exact integers) scaled by 1/128 (Sum s = 16 times the first-order
# weight 8 of d1 on a unit ramp, so a linear ramp gives its slope exactly);
# an edge pixel has |grad| > edge_thresh, |grad| > its bilinear sample at
# p + X and >= its sample at p - X (strict/non-strict as for ridges), with
# X = grad / |grad| in the canonical sign; |grad| = 0 is never an edge.
# --------------------------------------------------------------------------
def gradient_int(Lp: np.ndarray):
    """Exact integer first-order Sobel of L': Gx' = (d1_x (x) s_y) * L',
    Gy' = (s_x (x) d1_y) * L', reflect-101 borders."""
    gx = _correlate1d_int(_correlate1d_int(Lp, SOBEL_D1, 1), SOBEL_S, 0)
    gy = _correlate1d_int(_correlate1d_int(Lp, SOBEL_S, 1), SOBEL_D1, 0)
    return gx, gy


def gradient(image: np.ndarray, sigma: float):
    """(Gx, Gy) = (Gx', Gy') / (128 S^2) in float64 (one division each)."""
    Lp, S = smooth_int(image, sigma)
    gx, gy = gradient_int(Lp)
    D = float(128 * S * S)
    return gx.astype(np.float64) / D, gy.astype(np.float64) / D


def edge_direction(gx: np.ndarray, gy: np.ndarray):
    """|grad| and its unit direction in the canonical sign (X > 0, or X == 0
    and Y > 0), one IEEE operation per step: g = sqrt(gx gx + gy gy),
    X = gx / g, Y = gy / g.  Degenerate where g == 0."""
    g = np.sqrt(gx * gx + gy * gy)
    degenerate = g == 0.0
    with np.errstate(invalid="ignore", divide="ignore"):
        X = gx / g
        Y = gy / g
    flip = (X < 0.0) | ((X == 0.0) & (Y < 0.0))
    X = np.where(flip, -X, X)
    Y = np.where(flip, -Y, Y)
    X = np.where(degenerate, 0.0, X)
    Y = np.where(degenerate, 0.0, Y)
    return g, X, Y, degenerate


def edge_mask(g, X, Y, degenerate, edge_thresh: float) -> np.ndarray:
    """edge(p) <=> g(p) > edge_thresh and g(p) > g~(p + X) and
    g(p) >= g~(p - X); bilinear samples as in ridge_mask (a maximum instead of
    a minimum); a sample outside the frame makes the pixel a non-edge."""
    # the ridge test of -g against the threshold -edge_thresh is the same test
    return ridge_mask(-g, X, Y, degenerate, -edge_thresh)


def directed_edges(image: np.ndarray, p: Params):
    """Edge pixel coordinates (row-major) and their gradient directions."""
    gx, gy = gradient(image, p.sigma)
    g, X, Y, deg = edge_direction(gx, gy)
    mask = edge_mask(g, X, Y, deg, p.edge_thresh)
    ys, xs = np.nonzero(mask)
    return np.stack([xs, ys], axis=1).astype(np.int64), np.stack([X[ys, xs], Y[ys, xs]], axis=1)


def hot_threshold(p: Params) -> int:
    """Integer hotspot threshold on a cell: T_int, times c^2 in a coarse
    parameter space (reading: the threshold is a vote density per pixel of
    the parameter space, and a cell covers c^2 pixels)."""
    return p.vote_thresh * p.coarse * p.coarse


def annulus_width(p: Params) -> float:
    """Annulus half-width of the fit: w, plus c - 1 px in a coarse parameter
    space (the peak's centre is then only known to within c / sqrt 2 px)."""
    return p.annulus_w + float(p.coarse - 1)


def detect(image: np.ndarray, p: Params, keep: bool = False) -> Result:
    """Frame -> rings, steps O1-O9 in order.  Levels are visited in
    increasing r; the peak test of level r runs once N of level r + 1 exists
    (a plain sliding window of three levels, kept only to bound memory).
    With p.coarse = c > 1 steps O5-O8 run on the c-px cell grid and a peak
    cell (u, v) is the centre (c u, c v) px of the fit."""
    if image.dtype.kind not in "ui":
        raise TypeError("the oracle's exact path takes integer frames")
    if p.coarse not in (1, 2, 4):
        raise ValueError("coarse must be 1, 2 or 4")
    H, W = image.shape
    c = p.coarse
    Hc, Wc = cell_grid(H, W, c)
    ridge_xy, ridge_X = directed_edges(image, p) if p.features == "edge" else directed_ridges(image, p)
    xs, ys = ridge_xy[:, 0], ridge_xy[:, 1]
    levels = radius_levels(p.r_min, p.r_max)
    Ns, As = {}, {}
    votes_in = 0
    hotspots = smooth_macs = 0
    peaks = []
    for r in levels:
        r = int(r)
        bx, by = cast_votes(xs, ys, ridge_X[:, 0], ridge_X[:, 1], r, H, W, c)
        votes_in += len(bx)
        A = accumulate(bx, by, Hc, Wc)
        Qr = smoothing_weights(r, p.sig_a, p.sig_b, c)
        Ns[r] = smooth_hot(A, Qr, hot_threshold(p))
        n_hot = int((A > hot_threshold(p)).sum())
        hotspots += n_hot
        smooth_macs += n_hot * Qr.size
        if keep:
            As[r] = A
        if r - 1 >= p.r_min:
            peaks += find_peaks_level(Ns[r - 2], Ns[r - 1], Ns[r], r - 1, p)
            if not keep:
                del Ns[r - 2]
    peaks = [(c * x, c * y, r, n) for x, y, r, n in peaks]
    peaks.sort(key=lambda t: (t[2], t[1], t[0]))
    rings = np.zeros(len(peaks), dtype=RING_DTYPE)
    w = annulus_width(p)
    for i, (ix, iy, ir, nv) in enumerate(peaks):
        pts = annulus_members(ridge_xy, ix, iy, ir, w)
        cx, cy, rr, nfit, flags = kasa_fit(pts, ix, iy, ir)
        rings[i] = (cx, cy, rr, ix, iy, ir, nv / (float(1 << SMOOTH_BITS) * ir), nfit, flags)
    return Result(rings, ridge_xy, ridge_X, votes_in, 2 * len(xs) * len(levels), hotspots, smooth_macs,
                  As if keep else None, Ns if keep else None)


# --------------------------------------------------------------------------
# Definition mode: steps O1-O9 with the Gaussian taps of O1 and the level
# weights of O7 as the paper defines them, real-valued, instead of quantised
# to multiples of 2^-19 and 2^-16.  The exact path above quantises both so
# that smoothing and scoring of integer frames become integer arithmetic; this
# mode exists so that the tests can show that the quantisation changes no
# ring.  Everything is float64, one IEEE operation per step; frames may be
# integer or float.  With ``quantised=True`` the same float64 code takes the
# quantised weights (Q_i / S and Q_r / 2^16), which ties this mode to the
# exact path.
# --------------------------------------------------------------------------
def gaussian_taps_fp64(sigma: float) -> np.ndarray:
    """g_i = e_i / sum(e), e_i = exp(-i^2 / (2 sigma^2)), |i| <= R_g: the
    normalised, truncated Gaussian of O1 without quantisation."""
    R = gaussian_radius(sigma)
    i = np.arange(-R, R + 1, dtype=np.float64)
    den = 2.0 * sigma * sigma
    e = np.exp(-(i * i) / den)
    tot = 0.0
    for v in e:                      # left-to-right sum
        tot = tot + v
    return e / tot


def _correlate1d_fp64(f: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """Float64 correlation along one axis with reflect-101 borders.  The
    taps of every stencil here are symmetric or antisymmetric, and the sum
    is taken in paired form, t_0 f(x) + sum_{i>0} t_i (f(x+i) +/- f(x-i)), so
    that the mirror identities of the exact sum hold exactly in float64 (at
    a reflect-101 border an antisymmetric stencil gives exactly 0)."""
    R = (len(taps) - 1) // 2
    t = np.asarray(taps, dtype=np.float64)
    if np.array_equal(t, t[::-1]):
        sgn = 1.0
    elif np.array_equal(t, -t[::-1]):
        sgn = -1.0
    else:
        raise ValueError("taps must be symmetric or antisymmetric")
    pad = [(0, 0), (0, 0)]
    pad[axis] = (R, R)
    fp = np.pad(f.astype(np.float64), pad, mode="reflect")
    n = f.shape[axis]

    def shifted(i):
        sl = [slice(None), slice(None)]
        sl[axis] = slice(R + i, R + i + n)
        return fp[tuple(sl)]

    out = t[R] * shifted(0)
    for i in range(1, R + 1):
        pair = shifted(i) + shifted(-i) if sgn > 0 else shifted(i) - shifted(-i)
        out = out + t[R + i] * pair
    return out


def hessian_fp64(image: np.ndarray, sigma: float, quantised: bool = False):
    """O1-O2 in float64: L = g_y * (g_x * I), then the 5x5 second-order
    Sobel stencils of L divided by 64 (reflect-101 borders throughout).
    g is the real Gaussian (``gaussian_taps_fp64``), or Q / S when
    ``quantised``."""
    if quantised:
        Q = gaussian_taps(sigma)
        g = Q.astype(np.float64) / float(Q.sum())
    else:
        g = gaussian_taps_fp64(sigma)
    L = _correlate1d_fp64(_correlate1d_fp64(image, g, 1), g, 0)
    s, d1, d2 = SOBEL_S, SOBEL_D1, SOBEL_D2
    lxx = _correlate1d_fp64(_correlate1d_fp64(L, d2, 1), s, 0) / 64.0
    lyy = _correlate1d_fp64(_correlate1d_fp64(L, s, 1), d2, 0) / 64.0
    lxy = _correlate1d_fp64(_correlate1d_fp64(L, d1, 1), d1, 0) / 64.0
    return lxx, lyy, lxy


def smoothing_weights_fp64(r: int, sig_a: float, sig_b: float, c: int = 1,
                           quantised: bool = False) -> np.ndarray:
    """w_r(dy, dx) = exp(-(dx^2 + dy^2) / (2 sigma(r)^2)) on the window
    |dx|, |dy| <= ceil(3 sigma(r)) (O7, peak 1, unnormalised), or
    Q_r / 2^16 when ``quantised``; sigma(r) in cells of c px."""
    if quantised:
        return smoothing_weights(r, sig_a, sig_b, c).astype(np.float64) / float(1 << SMOOTH_BITS)
    sg = level_sigma(r, sig_a, sig_b) / c
    Rs = int(math.ceil(3.0 * sg))
    d = np.arange(-Rs, Rs + 1, dtype=np.float64)
    d2 = d[:, None] * d[:, None] + d[None, :] * d[None, :]
    den = 2.0 * sg * sg
    return np.exp(-d2 / den)


def smooth_hot_fp64(A: np.ndarray, w: np.ndarray, hot: int, r: int) -> np.ndarray:
    """S(v) = (1/r) sum_d w(d) A(v + d) at hotspots (A(v) > hot), 0
    elsewhere; A = 0 outside the image (O6-O7 in float64)."""
    H, W = A.shape
    Rs = (w.shape[0] - 1) // 2
    S = np.zeros((H, W), dtype=np.float64)
    hy, hx = np.nonzero(A > hot)
    if len(hy) == 0:
        return S
    Ap = np.pad(A, Rs, mode="constant").astype(np.float64)
    acc = np.zeros(len(hy), dtype=np.float64)
    for dy in range(-Rs, Rs + 1):
        for dx in range(-Rs, Rs + 1):
            acc += w[dy + Rs, dx + Rs] * Ap[hy + Rs + dy, hx + Rs + dx]
    S[hy, hx] = acc / float(r)
    return S


def find_peaks_level_fp64(S_lo: np.ndarray, S_mid: np.ndarray, S_hi: np.ndarray, r: int,
                          p: Params) -> list:
    """O8 on float64 scores: S(v) > f 2 pi and, over the 26 neighbours,
    S(v) > S(n) when n precedes v in (r, y, x) order and S(v) >= S(n)
    otherwise; out-of-image neighbours score 0."""
    H, W = S_mid.shape
    thr = p.peak_frac * (2.0 * math.pi)
    cy, cx = np.nonzero(S_mid > thr)
    if len(cy) == 0:
        return []
    sv = S_mid[cy, cx]
    ok = np.ones(len(cy), dtype=bool)
    lvl = {-1: S_lo, 0: S_mid, 1: S_hi}
    for dr, dy, dx in NEIGHBOURS:
        yy, xx = cy + dy, cx + dx
        inb = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        sn = np.where(inb, lvl[dr][np.clip(yy, 0, H - 1), np.clip(xx, 0, W - 1)], 0.0)
        ok &= (sv > sn) if (dr, dy, dx) < (0, 0, 0) else (sv >= sn)
    return [(int(x), int(y), int(r), float(s)) for x, y, s in zip(cx[ok], cy[ok], sv[ok])]


def detect_definition(image: np.ndarray, p: Params, quantised: bool = False) -> Result:
    """Frame -> rings with real-valued Gaussian taps and level weights
    (``quantised=False``, the paper's definition) or their quantised
    versions evaluated in float64 (``quantised=True``).  Steps O3-O6 and O9
    are the functions of the exact path; ridges only (no edge variant).
    ``rings['score']`` is S at the integer peak."""
    if p.features != "ridge":
        raise ValueError("definition mode covers the ridge method only")
    H, W = image.shape
    c = p.coarse
    Hc, Wc = cell_grid(H, W, c)
    Lxx, Lyy, Lxy = hessian_fp64(image, p.sigma, quantised)
    k, X, Y, deg = eigen(Lxx, Lyy, Lxy)
    mask = ridge_mask(k, X, Y, deg, p.ridge_thresh)
    ys, xs = np.nonzero(mask)
    ridge_xy = np.stack([xs, ys], axis=1).astype(np.int64)
    ridge_X = np.stack([X[ys, xs], Y[ys, xs]], axis=1)
    levels = radius_levels(p.r_min, p.r_max)
    Ss = {}
    votes_in = 0
    peaks = []
    for r in levels:
        r = int(r)
        bx, by = cast_votes(xs, ys, ridge_X[:, 0], ridge_X[:, 1], r, H, W, c)
        votes_in += len(bx)
        A = accumulate(bx, by, Hc, Wc)
        Ss[r] = smooth_hot_fp64(A, smoothing_weights_fp64(r, p.sig_a, p.sig_b, c, quantised),
                                hot_threshold(p), r)
        if r - 1 >= p.r_min:
            peaks += find_peaks_level_fp64(Ss[r - 2], Ss[r - 1], Ss[r], r - 1, p)
            del Ss[r - 2]
    peaks = [(c * x, c * y, r, s) for x, y, r, s in peaks]
    peaks.sort(key=lambda t: (t[2], t[1], t[0]))
    rings = np.zeros(len(peaks), dtype=RING_DTYPE)
    w = annulus_width(p)
    for i, (ix, iy, ir, s) in enumerate(peaks):
        pts = annulus_members(ridge_xy, ix, iy, ir, w)
        cx, cy, rr, nfit, flags = kasa_fit(pts, ix, iy, ir)
        rings[i] = (cx, cy, rr, ix, iy, ir, s, nfit, flags)
    return Result(rings, ridge_xy, ridge_X, votes_in, 2 * len(xs) * len(levels))
