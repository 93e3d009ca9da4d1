"""FP64 CPU oracle of the differentiable (soft) ring score and its gradients.

TEST INFRASTRUCTURE ONLY (like ``oracle.ringdet``): only the test-suite and
``bench.py``'s CPU legs may import it.  It shares no code with the CUDA path.

The paper has no differentiable form of the method.  This module defines one
as a smooth extension of its voting and scoring steps (Results, "Directed
ridge detection & votes collection" and "Local maxima detection in a noisy
parameter space"), so that a ring's parameters can be refined by gradient
ascent and the score differentiated with respect to the image:

    Score(c, rho) = (1/rho) sum_{p in ridge} m(p) a(p) sum_{s = +1, -1}
                    sum_{q in corners(v)} bil(v, q) exp(-|q - c|^2 / (2 sigma(rho)^2)),
    v = p + s rho X(p),   m(p) = logistic((tau - k(p)) / T),   sigma(rho) = sig_a rho + sig_b,
    a(p) = exp(-(|p - c| - rho)^2 / (2 (w / 2)^2)).

* The ridge set is the hard directed-ridge mask of the frame (steps O1-O4 of
  ``oracle.ringdet`` on the float frame) and is held fixed: the score is not
  differentiated through the mask decision.
* k(p) and X(p) are the least principal curvature and its unit direction at
  p (step O3), computed from the Hessian of the float frame: the same
  quantised Gaussian taps (normalised, Q_i / S) and the same 5x5 second-order
  Sobel / 64 with reflect-101 borders as the integer path.
* A vote at the continuous position v is spread over the four grid points
  of its cell with bilinear weights bil(v, q) = (1 - |v_x - q_x|)(1 - |v_y - q_y|);
  grid points outside [0, W-1] x [0, H-1] receive nothing (votes are
  restricted to the image domain, as in step O5).  Each grid point
  contributes the unnormalised Gaussian of step O7 centred at the continuous
  centre c, and the sum is normalised by 1/rho as in O7.
* a(p) is the ring's soft annulus: the weight of a ridge pixel falls off as
  a Gaussian of its distance from the circle (c, rho), with standard
  deviation half the annulus half-width w of the classification step
  (Results, "Ridge points classification & sub-pixel accuracy": the ridge
  pixels within an annulus around each ring belong to it; w = 2 px).  It
  keeps the votes of neighbouring rings' pixels, which lie off the circle,
  out of a ring's score; without it a refined centre is worse than the
  detector's circle fit on crowded frames.
* Readings (the paper is silent): T = |tau| / 4 (with |tau| at least 1e-6);
  the annulus's standard deviation w / 2; the sum runs over all ridge pixels
  and both signs, with no window cut-off.

``soft_score`` is the definition written out with NumPy.  ``soft_score_torch``
is the same forward written with plain PyTorch CPU float64 ops; its autograd
gives the reference gradients with respect to the image and (cx, cy, rho).
"""
from __future__ import annotations

import dataclasses
import numpy as np

from oracle import ringdet as R


@dataclasses.dataclass
class SoftParams:
    sigma: float
    ridge_thresh: float
    sig_a: float
    sig_b: float
    annulus_w: float = 2.0

    @property
    def temperature(self) -> float:
        return max(abs(self.ridge_thresh), 1e-6) / 4.0

    @property
    def annulus_sigma(self) -> float:
        """Standard deviation of the soft annulus: half the half-width w."""
        return self.annulus_w * 0.5

    @staticmethod
    def make(**kw) -> "SoftParams":
        f32 = lambda v: float(np.float32(v))  # parameters arrive as float32
        return SoftParams(f32(kw["sigma"]), f32(kw["ridge_thresh"]), f32(kw.get("sig_a", 0.05)),
                          f32(kw.get("sig_b", 0.25)), f32(kw.get("annulus_w", 2.0)))


def annulus(xs, ys, cx, cy, rho, p: SoftParams):
    """a(p) = exp(-(|p - c| - rho)^2 / (2 (w/2)^2)) for ridge pixels (xs, ys)."""
    d = np.sqrt((xs - cx) * (xs - cx) + (ys - cy) * (ys - cy))
    sa = p.annulus_sigma
    return np.exp(-((d - rho) * (d - rho)) / (2.0 * sa * sa))


def _taps_float(sigma: float) -> np.ndarray:
    Q = R.gaussian_taps(sigma)
    return Q.astype(np.float64) / float(Q.sum())


def _correlate1d(f: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """Float64 correlation along one axis, reflect-101 borders."""
    r = (len(taps) - 1) // 2
    pad = [(0, 0), (0, 0)]
    pad[axis] = (r, r)
    fp = np.pad(f, pad, mode="reflect")
    out = np.zeros(f.shape, dtype=np.float64)
    n = f.shape[axis]
    for j, t in enumerate(taps):
        sl = [slice(None), slice(None)]
        sl[axis] = slice(j, j + n)
        out += t * fp[tuple(sl)]
    return out


def hessian_float(image: np.ndarray, sigma: float):
    """(Lxx, Lyy, Lxy) of a float frame: L = g_y * (g_x * I) with g = Q / S,
    then the second-order Sobel stencils / 64 (steps O1-O2)."""
    g = _taps_float(sigma)
    I = image.astype(np.float64)
    L = _correlate1d(_correlate1d(I, g, 1), g, 0)
    s, d1, d2 = (R.SOBEL_S.astype(np.float64), R.SOBEL_D1.astype(np.float64), R.SOBEL_D2.astype(np.float64))
    lxx = _correlate1d(_correlate1d(L, d2, 1), s, 0) / 64.0
    lyy = _correlate1d(_correlate1d(L, s, 1), d2, 0) / 64.0
    lxy = _correlate1d(_correlate1d(L, d1, 1), d1, 0) / 64.0
    return lxx, lyy, lxy


@dataclasses.dataclass
class Ridges:
    xs: np.ndarray   # int64 column
    ys: np.ndarray   # int64 row
    k: np.ndarray    # least principal curvature
    X: np.ndarray    # unit direction (canonical sign)
    Y: np.ndarray
    use1: np.ndarray  # which eigenvector candidate was normalised (O3)


def ridges_float(image: np.ndarray, p: SoftParams) -> Ridges:
    """The hard ridge set of a float frame with k and X at its pixels."""
    lxx, lyy, lxy = hessian_float(image, p.sigma)
    k, X, Y, deg = R.eigen(lxx, lyy, lxy)
    mask = R.ridge_mask(k, X, Y, deg, p.ridge_thresh)
    ys, xs = np.nonzero(mask)
    a, c, b = lxx[ys, xs], lyy[ys, xs], lxy[ys, xs]
    kk = k[ys, xs]
    n1 = b * b + (kk - a) * (kk - a)
    n2 = (kk - c) * (kk - c) + b * b
    return Ridges(xs.astype(np.int64), ys.astype(np.int64), kk, X[ys, xs], Y[ys, xs], n1 >= n2)


def logistic(z):
    return 1.0 / (1.0 + np.exp(-z))


def soft_score(rd: Ridges, rings: np.ndarray, p: SoftParams, H: int, W: int) -> np.ndarray:
    """Score(c, rho) for each ring (cx, cy, rho) of ``rings`` [n, 3]."""
    m = logistic((p.ridge_thresh - rd.k) / p.temperature)
    fx0 = rd.xs.astype(np.float64)
    fy0 = rd.ys.astype(np.float64)
    out = np.zeros(len(rings))
    for i, (cx, cy, rho) in enumerate(np.asarray(rings, dtype=np.float64)):
        sig = p.sig_a * rho + p.sig_b
        den = 2.0 * sig * sig
        ma = m * annulus(fx0, fy0, cx, cy, rho, p)
        total = 0.0
        for s in (1.0, -1.0):
            vx = fx0 + s * rho * rd.X
            vy = fy0 + s * rho * rd.Y
            x0 = np.floor(vx)
            y0 = np.floor(vy)
            fx = vx - x0
            fy = vy - y0
            for ox, oy, w in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)),
                              (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
                qx = x0 + ox
                qy = y0 + oy
                inside = (qx >= 0) & (qx <= W - 1) & (qy >= 0) & (qy <= H - 1)
                d2 = (qx - cx) ** 2 + (qy - cy) ** 2
                total += float(np.sum(np.where(inside, ma * w * np.exp(-d2 / den), 0.0)))
        out[i] = total / rho
    return out


def soft_score_torch(image, rings, rd: Ridges, p: SoftParams):
    """The same forward as ``soft_score`` on torch float64 CPU tensors:
    image [H, W] and rings [n, 3] may require grad; the ridge set ``rd`` (and
    its eigenvector branch and sign) is held fixed.  Returns scores [n]."""
    import torch
    import torch.nn.functional as F

    H, W = image.shape
    g = torch.tensor(_taps_float(p.sigma), dtype=torch.float64)

    def corr(f, taps, axis):
        rr = (len(taps) - 1) // 2
        x = f[None, None]
        if axis == 1:
            x = F.pad(x, (rr, rr, 0, 0), mode="reflect")
            return F.conv2d(x, taps.view(1, 1, 1, -1))[0, 0]
        x = F.pad(x, (0, 0, rr, rr), mode="reflect")
        return F.conv2d(x, taps.view(1, 1, -1, 1))[0, 0]

    L = corr(corr(image, g, 1), g, 0)
    s = torch.tensor([1., 4., 6., 4., 1.], dtype=torch.float64)
    d1 = torch.tensor([-1., -2., 0., 2., 1.], dtype=torch.float64)
    d2 = torch.tensor([1., 0., -2., 0., 1.], dtype=torch.float64)
    lxx = corr(corr(L, d2, 1), s, 0) / 64.0
    lyy = corr(corr(L, s, 1), d2, 0) / 64.0
    lxy = corr(corr(L, d1, 1), d1, 0) / 64.0
    ys = torch.as_tensor(rd.ys)
    xs = torch.as_tensor(rd.xs)
    a, c, b = lxx[ys, xs], lyy[ys, xs], lxy[ys, xs]
    k = (a + c) * 0.5 - torch.sqrt(((a - c) * 0.5) ** 2 + b * b)
    use1 = torch.as_tensor(rd.use1)
    vx = torch.where(use1, b, k - c)
    vy = torch.where(use1, k - a, b)
    nrm = torch.sqrt(vx * vx + vy * vy)
    X = vx / nrm
    Y = vy / nrm
    # canonical sign (X > 0, or X == 0 and Y > 0), held fixed like the branch
    Xd, Yd = X.detach().numpy(), Y.detach().numpy()
    sign = torch.as_tensor(np.where((Xd < 0) | ((Xd == 0) & (Yd < 0)), -1.0, 1.0))
    X = X * sign
    Y = Y * sign
    m = torch.sigmoid((p.ridge_thresh - k) / p.temperature)
    fx0 = xs.to(torch.float64)
    fy0 = ys.to(torch.float64)
    out = []
    sa = p.annulus_sigma
    for i in range(rings.shape[0]):
        cx, cy, rho = rings[i, 0], rings[i, 1], rings[i, 2]
        sig = p.sig_a * rho + p.sig_b
        den = 2.0 * sig * sig
        dist = torch.sqrt((fx0 - cx) * (fx0 - cx) + (fy0 - cy) * (fy0 - cy))
        ma = m * torch.exp(-((dist - rho) * (dist - rho)) / (2.0 * sa * sa))
        total = torch.zeros((), dtype=torch.float64)
        for sg in (1.0, -1.0):
            vx_ = fx0 + sg * rho * X
            vy_ = fy0 + sg * rho * Y
            x0 = torch.floor(vx_.detach())
            y0 = torch.floor(vy_.detach())
            fx = vx_ - x0
            fy = vy_ - y0
            for ox, oy, w in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)),
                              (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
                qx = x0 + ox
                qy = y0 + oy
                inside = (qx >= 0) & (qx <= W - 1) & (qy >= 0) & (qy <= H - 1)
                d2 = (qx - cx) ** 2 + (qy - cy) ** 2
                total = total + torch.sum(torch.where(inside, ma * w * torch.exp(-d2 / den), torch.zeros_like(w)))
        out.append(total / rho)
    return torch.stack(out)


def soft_grads(image: np.ndarray, rings: np.ndarray, p: SoftParams, dscore: np.ndarray | None = None):
    """Scores and the reference gradients of sum_i dscore_i Score_i with
    respect to the image [H, W] and to each ring's (cx, cy, rho) [n, 3]
    (dscore = 1 by default), by autograd of ``soft_score_torch``."""
    import torch
    rd = ridges_float(image, p)
    img = torch.tensor(image, dtype=torch.float64, requires_grad=True)
    rg = torch.tensor(np.asarray(rings, dtype=np.float64), requires_grad=True)
    sc = soft_score_torch(img, rg, rd, p)
    w = torch.ones_like(sc) if dscore is None else torch.tensor(np.asarray(dscore, dtype=np.float64))
    (sc * w).sum().backward()
    return sc.detach().numpy(), img.grad.numpy(), rg.grad.numpy(), rd
