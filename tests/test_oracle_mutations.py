"""Planted mistakes in the oracle must make at least one pin fail (CPU only).

Each mutation replaces one step of ``oracle.ringdet`` for the duration of a
test (monkeypatch), runs every pin, and asserts that some pin now fails.  This
shows that the pins constrain each step, not just the whole pipeline.
"""
import numpy as np
import pytest

from oracle import ringdet as O
import tests.test_oracle_pins as P

_orig = {name: getattr(O, name) for name in
         ("eigen", "cast_votes", "smoothing_weights", "smooth_hot", "find_peaks_level",
          "kasa_fit", "ridge_mask", "hessian_int", "gaussian_taps")}


def _larger_eigen(a, c, b):
    k, X, Y, deg = _orig["eigen"](-a, -c, -b)
    return -k, X, Y, deg


def _one_sign_votes(xs, ys, X, Y, r, H, W, c=1):
    sr = float(r)
    bx = np.floor(xs + sr * X + 0.5).astype(np.int64)
    by = np.floor(ys + sr * Y + 0.5).astype(np.int64)
    keep = (bx >= 0) & (bx < W) & (by >= 0) & (by < H)
    return bx[keep], by[keep]


def _truncating_votes(xs, ys, X, Y, r, H, W, c=1):
    bxs, bys = [], []
    for s in (1, -1):
        bx = np.trunc(xs + s * r * X).astype(np.int64)
        by = np.trunc(ys + s * r * Y).astype(np.int64)
        keep = (bx >= 0) & (bx < W) & (by >= 0) & (by < H)
        bxs.append(bx[keep]); bys.append(by[keep])
    return np.concatenate(bxs), np.concatenate(bys)


def _normalised_weights(r, a, b, c=1):
    Q = _orig["smoothing_weights"](r, a, b, c)
    return np.floor(Q * 65536.0 / Q.sum() + 0.5).astype(np.int64)


def _geq_hot(A, Qr, t):
    return _orig["smooth_hot"](A, Qr, t - 1)


def _no_1_over_r_peaks(N_lo, N_mid, N_hi, r, p):
    return _orig["find_peaks_level"](N_lo * (r - 1), N_mid * r, N_hi * (r + 1), r, p)


def _strict_ties(N_lo, N_mid, N_hi, r, p):
    # ">=" against every neighbour: plateaus produce several peaks
    H, W = N_mid.shape
    thr = O.peak_threshold(p.peak_frac, r)
    out = []
    for y, x in zip(*np.nonzero(N_mid.astype(float) > thr)):
        nv = int(N_mid[y, x])
        ok = True
        for dr, dy, dx in O.NEIGHBOURS:
            yy, xx = y + dy, x + dx
            L = {-1: N_lo, 0: N_mid, 1: N_hi}[dr]
            nn = int(L[yy, xx]) if 0 <= yy < H and 0 <= xx < W else 0
            ok &= nv * (r + dr) >= nn * r
        if ok:
            out.append((int(x), int(y), int(r), nv))
    return out


def _kasa_sign(pts, ix, iy, ir):
    cx, cy, r, n, f = _orig["kasa_fit"](pts, ix, iy, ir)
    return 2 * ix - cx, 2 * iy - cy, r, n, f


def _both_nonstrict_ridge(k, X, Y, deg, tau):
    # "<=" on both sides: both pixels of a two-pixel plateau become ridges
    H, W = k.shape
    out = np.zeros((H, W), dtype=bool)
    for y, x in zip(*np.nonzero((k < tau) & ~deg)):
        ok = True
        for s in (1, -1):
            qx, qy = x + s * X[y, x], y + s * Y[y, x]
            if not (0 <= qx <= W - 1 and 0 <= qy <= H - 1):
                ok = False
                break
            ok &= k[y, x] <= O.bilinear(k, qx, qy)
        out[y, x] = ok
    return out


def _transposed_hessian(Lp):
    hxx, hyy, hxy = _orig["hessian_int"](Lp)
    return hyy, hxx, hxy


def _flipped_d1(Lp):
    hxx, hyy, hxy = _orig["hessian_int"](Lp)
    return hxx, hyy, -hxy


def _unnormalised_taps(sigma):
    Q = _orig["gaussian_taps"](sigma)
    Q = Q.copy()
    Q[len(Q) // 2] += 200
    return Q


def _coarse_floor_cells(xs, ys, X, Y, r, H, W, c=1):
    """Coarse cells by floor(a / c) instead of the nearest centre."""
    Hc, Wc = O.cell_grid(H, W, c)
    bxs, bys = [], []
    for s in (1, -1):
        ax = xs + float(s * r) * X
        ay = ys + float(s * r) * Y
        bx = (np.floor(ax / c) if c > 1 else np.floor(ax + 0.5)).astype(np.int64)
        by = (np.floor(ay / c) if c > 1 else np.floor(ay + 0.5)).astype(np.int64)
        keep = (bx >= 0) & (bx < Wc) & (by >= 0) & (by < Hc)
        bxs.append(bx[keep]); bys.append(by[keep])
    return np.concatenate(bxs), np.concatenate(bys)


def _coarse_sigma_unscaled(r, a, b, c=1):
    """The window left in pixel units on the cell grid."""
    return _orig["smoothing_weights"](r, a, b)


MUTATIONS = {
    "coarse_floor_cells": ("cast_votes", _coarse_floor_cells),
    "coarse_sigma_unscaled": ("smoothing_weights", _coarse_sigma_unscaled),
    "larger_eigenvalue": ("eigen", _larger_eigen),
    "one_sign_votes": ("cast_votes", _one_sign_votes),
    "truncating_votes": ("cast_votes", _truncating_votes),
    "normalised_level_weights": ("smoothing_weights", _normalised_weights),
    "hot_ge_threshold": ("smooth_hot", _geq_hot),
    "no_1_over_r": ("find_peaks_level", _no_1_over_r_peaks),
    "ties_not_broken": ("find_peaks_level", _strict_ties),
    "kasa_centre_sign": ("kasa_fit", _kasa_sign),
    "ridge_nonstrict_both": ("ridge_mask", _both_nonstrict_ridge),
    "hessian_transposed": ("hessian_int", _transposed_hessian),
    "hessian_xy_sign": ("hessian_int", _flipped_d1),
    "taps_unnormalised": ("gaussian_taps", _unnormalised_taps),
}


def _all_pins_pass():
    failed = []
    for name, fn in P.PINS.items():
        try:
            ok = fn(2.0) if name == "taps_are_gaussian" else fn()
        except Exception:
            ok = False
        if not ok:
            failed.append(name)
    return failed


@pytest.mark.parametrize("mut", sorted(MUTATIONS))
def test_mutation_is_caught(mut, monkeypatch):
    attr, fn = MUTATIONS[mut]
    monkeypatch.setattr(O, attr, fn)
    failed = _all_pins_pass()
    assert failed, f"planted mistake {mut!r} passed every pin"
