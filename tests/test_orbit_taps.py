"""The sparse voting kernel smooths a hotspot with its window taps grouped in
rotation orbits, checked on CPU against the plain window sum.

The level weights Q_r(dx, dy) depend on dx^2 + dy^2 only (Methods: Gaussian
weights of width sigma(r)).  So the four taps (dx, dy), (-dy, dx), (-dx, -dy)
and (dy, -dx) share one weight.  The context stores one entry per orbit,
{o1, o2, Q}, for dx in 1..R and dy in 0..R, with o1 = dy RW + dx and
o2 = dx RW - dy the offsets in a shared-memory row of RW.  The kernel sums
Q (A[c + o1] + A[c - o1] + A[c + o2] + A[c - o2]) plus the centre.  This test
builds the table the same way for every level of several radius ranges and
cell sizes and checks three things:

* the orbits with the centre cover the (2R+1)^2 window exactly once;
* each orbit's four taps have the stored weight in the oracle's table;
* the orbit sum equals the oracle's smoothed value on random accumulators.
"""
import numpy as np
import pytest

from oracle import ringdet as O

SIG_A, SIG_B = float(np.float32(0.05)), float(np.float32(0.25))


def orbit_table(Q, RW):
    R = (Q.shape[0] - 1) // 2
    q = lambda dx, dy: int(Q[dy + R, dx + R])
    table = [(0, 0, q(0, 0))]
    for dx in range(1, R + 1):
        for dy in range(0, R + 1):
            w = q(dx, dy)
            assert q(-dy, dx) == w and q(-dx, -dy) == w and q(dy, -dx) == w
            table.append((dy * RW + dx, dx * RW - dy, w))
    return table


@pytest.mark.parametrize("c", [1, 2, 4])
def test_orbits_cover_the_window_once(c):
    for r in list(range(2, 98)) + [150, 251]:
        Q = O.smoothing_weights(r, SIG_A, SIG_B, c)
        R = (Q.shape[0] - 1) // 2
        RW = 128 + 2 * (R + 1)                       # a slab row: tile + halo on both sides
        table = orbit_table(Q, RW)
        offsets = [0] + [o for o1, o2, _ in table[1:] for o in (o1, -o1, o2, -o2)]
        window = sorted(dy * RW + dx for dy in range(-R, R + 1) for dx in range(-R, R + 1))
        assert sorted(offsets) == window, r
        weight = {dy * RW + dx: int(Q[dy + R, dx + R]) for dy in range(-R, R + 1) for dx in range(-R, R + 1)}
        assert weight[0] == table[0][2]
        for o1, o2, w in table[1:]:
            assert weight[o1] == weight[-o1] == weight[o2] == weight[-o2] == w


@pytest.mark.parametrize("r", [8, 31, 96])
def test_orbit_sum_equals_window_sum(r):
    rng = np.random.default_rng(r)
    Q = O.smoothing_weights(r, SIG_A, SIG_B)
    R = (Q.shape[0] - 1) // 2
    H = W = 48
    A = rng.integers(0, 9, size=(H, W)).astype(np.int64)
    T = 0
    N = O.smooth_hot(A, Q, T)
    RW = W + 2 * R                                    # zero-padded rows, as the slab holds its halo
    Ap = np.pad(A, R).ravel()
    table = orbit_table(Q, RW)
    for y in range(H):
        for x in range(W):
            if A[y, x] <= T:
                continue
            c = (y + R) * RW + (x + R)
            acc = table[0][2] * int(Ap[c])
            for o1, o2, w in table[1:]:
                acc += w * int(Ap[c + o1] + Ap[c - o1] + Ap[c + o2] + Ap[c - o2])
            assert acc == int(N[y, x]), (y, x)
