"""Pins of the oracle's directed-edge variant (Additional notes: gradient in
place of the Hessian, magnitude a local maximum along the gradient)."""
import numpy as np

from oracle import ringdet as O
from paper_1310_1371_gb300 import synth


def disc_image(H, W, cx, cy, R, lo=60.0, hi=180.0, width=1.2, noise=0.0, seed=0):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    d = np.hypot(xx - cx, yy - cy) - R
    img = lo + (hi - lo) / (1.0 + np.exp(d / width))
    if noise:
        img = img + np.random.default_rng(seed).normal(0, noise, img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def test_linear_ramp_gives_its_slope_exactly():
    yy, xx = np.mgrid[0:48, 0:56]
    img = (3 * xx + 5 * yy + 10).astype(np.uint16)
    gx, gy = O.gradient(img, 2.0)
    inner = (slice(12, 36), slice(12, 44))
    assert np.all(gx[inner] == 3.0) and np.all(gy[inner] == 5.0)


def test_step_edge_single_column():
    img = np.full((40, 64), 100, dtype=np.uint8)
    img[:, 21:] = 200
    p = O.Params.make(**dict(synth.PLAIN_SMALL_PARAMS, features="edge", edge_thresh=1.0))
    xy, X = O.directed_edges(img, p)
    # |grad| is symmetric about x = 20.5: columns 20 and 21 tie, and the rule
    # (strict along +X, non-strict along -X) keeps exactly column 21
    assert len(xy) == 40 and np.all(xy[:, 0] == 21)
    assert np.allclose(X, [[1.0, 0.0]])


def test_disc_edges_on_the_circle_with_radial_directions():
    cx, cy, R = 32.4, 31.7, 15.3
    img = disc_image(64, 64, cx, cy, R)
    p = O.Params.make(**dict(synth.PLAIN_SMALL_PARAMS, features="edge", edge_thresh=2.0))
    xy, X = O.directed_edges(img, p)
    d = np.hypot(xy[:, 0] - cx, xy[:, 1] - cy)
    assert len(xy) > 60 and np.all(np.abs(d - R) < 1.0)
    radial = np.stack([xy[:, 0] - cx, xy[:, 1] - cy], 1) / d[:, None]
    assert np.all(np.abs(np.sum(radial * X, 1)) > 0.98)


def test_edge_detection_finds_the_disc():
    cx, cy, R = 40.3, 38.6, 17.4
    img = disc_image(80, 80, cx, cy, R, noise=3.0, seed=4)
    p = O.Params.make(**dict(synth.PLAIN_SMALL_PARAMS, features="edge", edge_thresh=4.0))
    res = O.detect(img, p)
    assert len(res.rings) >= 1
    best = res.rings[np.argmax(res.rings["score"])]
    assert abs(best["ix"] - cx) <= 1 and abs(best["iy"] - cy) <= 1 and abs(best["ir"] - R) <= 1
    assert abs(best["cx"] - cx) < 0.3 and abs(best["cy"] - cy) < 0.3 and abs(best["r"] - R) < 0.5


def test_edge_mode_rejects_flat_and_subthreshold():
    img = np.full((32, 32), 77, dtype=np.uint8)
    p = O.Params.make(**dict(synth.PLAIN_SMALL_PARAMS, features="edge", edge_thresh=0.5))
    assert len(O.directed_edges(img, p)[0]) == 0
    step = np.full((32, 32), 100, dtype=np.uint8)
    step[:, 16:] = 101  # |grad| at most 1/4 px^-1 after smoothing
    assert len(O.directed_edges(step, p)[0]) == 0


# ---- planted mistakes in the edge variant must make a pin fail -------------------
import pytest

_PINS = [test_linear_ramp_gives_its_slope_exactly, test_step_edge_single_column,
         test_disc_edges_on_the_circle_with_radial_directions, test_edge_detection_finds_the_disc]
_orig_gradient_int, _orig_edge_mask, _orig_gradient = O.gradient_int, O.edge_mask, O.gradient


def _transposed_gradient(Lp):
    gx, gy = _orig_gradient_int(Lp)
    return gy, gx


def _nonstrict_maximum(g, X, Y, deg, t):
    H, W = g.shape
    out = np.zeros((H, W), dtype=bool)
    for y, x in zip(*np.nonzero((g > t) & ~deg)):
        ok = True
        for s in (1, -1):
            qx, qy = x + s * X[y, x], y + s * Y[y, x]
            if not (0 <= qx <= W - 1 and 0 <= qy <= H - 1):
                ok = False
                break
            ok &= g[y, x] >= O.bilinear(g, qx, qy)
        out[y, x] = ok
    return out


def _half_scale(image, sigma):
    gx, gy = _orig_gradient(image, sigma)
    return 2.0 * gx, 2.0 * gy  # /64 instead of /128


@pytest.mark.parametrize("attr,fn", [("gradient_int", _transposed_gradient), ("edge_mask", _nonstrict_maximum),
                                     ("gradient", _half_scale)])
def test_edge_mutation_is_caught(attr, fn, monkeypatch):
    monkeypatch.setattr(O, attr, fn)
    failed = 0
    for pin in _PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1
