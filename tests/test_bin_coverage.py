"""The vote binning stage sends each (ridge pixel, slab, sign) segment to every
accumulator tile that one of its votes can reach, checked on CPU.

For an r-slab with peak levels lo..hi, the votes at r = lo - 1 .. hi + 1 lie
on the segment p + s r X- (Results: the votes p +- r X-).  The binning stage
bounds that segment by its end points in FP32, widens the box by one cell
(votes are rounded to the nearest pixel, or to a cell of c px), clips it to
the accumulator grid, and lists the tiles whose region, the tile plus its
smoothing halo h, meets the box.  This test replays that computation in
NumPy float32, both plain and with the end-point products contracted into
fused multiply-adds.  Every vote of the segment, binned as the definition
bins it, must fall only in listed tiles.  The test covers tiles of 64, 80,
96 and 128 cells, coarse cells of 1, 2 and 4 px, full and ragged frames,
pixels at the borders, and axis and diagonal directions.
"""
import numpy as np
import pytest

f32 = np.float32


def fma32(a, b, c):
    """a b + c rounded once to float32 (a b exact in float64; the float64 sum
    is within the 1-cell margin of the exact value, which is all this needs)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def tile_of(v, T):
    return np.floor_divide(v, T)


def seg_tiles(px, py, dx, dy, r0, r1, h, T, lc, Hc, Wc, contract, margin=1):
    """The binning stage's tile box [tx0, tx1] x [ty0, ty1] per pixel, or an
    empty box (tx0 > tx1) when the segment misses the grid."""
    inv_c = f32(1.0 / (1 << lc))
    if contract:
        ax0, ax1 = fma32(r0, dx, px) * inv_c, fma32(r1, dx, px) * inv_c
        ay0, ay1 = fma32(r0, dy, py) * inv_c, fma32(r1, dy, py) * inv_c
    else:
        ax0, ax1 = (px + f32(r0) * dx) * inv_c, (px + f32(r1) * dx) * inv_c
        ay0, ay1 = (py + f32(r0) * dy) * inv_c, (py + f32(r1) * dy) * inv_c
    bx0 = np.floor(np.minimum(ax0, ax1)).astype(np.int64) - margin
    bx1 = np.ceil(np.maximum(ax0, ax1)).astype(np.int64) + margin
    by0 = np.floor(np.minimum(ay0, ay1)).astype(np.int64) - margin
    by1 = np.ceil(np.maximum(ay0, ay1)).astype(np.int64) + margin
    bx0, by0 = np.maximum(bx0, 0), np.maximum(by0, 0)
    bx1, by1 = np.minimum(bx1, Wc - 1), np.minimum(by1, Hc - 1)
    n_atx, n_aty = -(-Wc // T), -(-Hc // T)
    tx0 = np.maximum(tile_of(bx0 - h, T), 0)
    tx1 = np.minimum(tile_of(bx1 + h, T), n_atx - 1)
    ty0 = np.maximum(tile_of(by0 - h, T), 0)
    ty1 = np.minimum(tile_of(by1 + h, T), n_aty - 1)
    empty = (bx0 > bx1) | (by0 > by1)
    tx1 = np.where(empty, tx0 - 1, tx1)
    return tx0, tx1, ty0, ty1


def vote_cells(px, py, X, Y, s, r, lc):
    """The definition's cell of the vote p + s r X (c = 2^lc; c = 1: the nearest pixel)."""
    c = 1 << lc
    ax = px.astype(np.float64) + float(s * r) * X.astype(np.float64)
    ay = py.astype(np.float64) + float(s * r) * Y.astype(np.float64)
    return np.floor((ax + 0.5 * c) / c).astype(np.int64), np.floor((ay + 0.5 * c) / c).astype(np.int64)


def directions(rng, n):
    t = rng.uniform(0, np.pi, n)
    X, Y = np.cos(t), np.sin(t)
    k = n // 8                                                     # exact axes and diagonals
    X[:k], Y[:k] = 1.0, 0.0
    X[k:2 * k], Y[k:2 * k] = 0.0, 1.0
    X[2 * k:3 * k] = Y[2 * k:3 * k] = np.sqrt(0.5)
    flip = (X < 0) | ((X == 0) & (Y < 0))
    X, Y = np.where(flip, -X, X), np.where(flip, -Y, Y)
    return X.astype(np.float32), Y.astype(np.float32)


def unlisted_votes(H, W, lc, T, contract, margin=1, halo_cut=0):
    """Number of (vote, tile) pairs where a vote lies in a tile's region but
    the segment's box does not list the tile."""
    rng = np.random.default_rng(1000 * T + 10 * lc + H)
    n = 3000
    px = rng.integers(0, W, n).astype(np.float32)
    py = rng.integers(0, H, n).astype(np.float32)
    px[:60], py[:60] = 0, rng.integers(0, H, 60)                   # pixels on the borders
    px[60:120], py[60:120] = W - 1, rng.integers(0, H, 60)
    py[120:180] = 0
    py[180:240] = H - 1
    X, Y = directions(rng, n)
    c = 1 << lc
    Hc, Wc = -(-H // c), -(-W // c)
    missed = 0
    for lo, hi in ((8, 39), (40, 71), (72, 96), (200, 231)):
        h = 1 + int(np.ceil(3.0 * (0.05 * (hi + 1) + 0.25) / c))  # 1 + the slab's largest window radius
        for s in (1, -1):
            tx0, tx1, ty0, ty1 = seg_tiles(px, py, f32(s) * X, f32(s) * Y, float(lo - 1), float(hi + 1),
                                           h - halo_cut, T, lc, Hc, Wc, contract, margin)
            for r in range(lo - 1, hi + 2):
                vx, vy = vote_cells(px, py, X, Y, s, r, lc)
                inside = (vx >= 0) & (vx < Wc) & (vy >= 0) & (vy < Hc)
                # every tile whose region [t T - h, t T + T + h) holds the vote
                for dtx in (-1, 0, 1):
                    for dty in (-1, 0, 1):
                        qx = tile_of(vx, T) + dtx
                        qy = tile_of(vy, T) + dty
                        touches = (inside & (qx >= 0) & (qx < -(-Wc // T)) & (qy >= 0) & (qy < -(-Hc // T))
                                   & (vx >= qx * T - h) & (vx < qx * T + T + h)
                                   & (vy >= qy * T - h) & (vy < qy * T + T + h))
                        listed = (qx >= tx0) & (qx <= tx1) & (qy >= ty0) & (qy <= ty1)
                        missed += int((touches & ~listed).sum())
    return missed


@pytest.mark.parametrize("contract", [False, True])
@pytest.mark.parametrize("T", [64, 80, 96, 128])
@pytest.mark.parametrize("lc", [0, 1, 2])
@pytest.mark.parametrize("H,W", [(1024, 1024), (77, 131)])
def test_segments_reach_every_tile_their_votes_touch(H, W, lc, T, contract):
    assert unlisted_votes(H, W, lc, T, contract) == 0


def test_planted_short_halo_is_caught():
    """The one-cell margin is slack on top of the rounding (floor and ceil of
    the end points already hold every rounded vote); a halo two cells short
    leaves votes unlisted."""
    assert unlisted_votes(1024, 1024, 0, 64, False, margin=0) == 0
    assert unlisted_votes(1024, 1024, 0, 64, False, halo_cut=2) > 0
    assert unlisted_votes(1024, 1024, 2, 128, False, margin=0, halo_cut=1) > 0
