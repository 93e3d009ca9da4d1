"""The circle fit's solve (Results, "Ridge points classification & sub-pixel
accuracy"; the algebraic least-squares fit), checked on CPU against the exact
rational solution.

The fit kernel forms the Kasa normal equations from exact int64 moments of
the annulus points.  It solves them by Cramer's rule: exact int128
determinants, each converted to double as a high and a low 64-bit half, and
one double division per unknown.  The oracle solves the same integer system
with numpy.linalg.solve.  This test computes the exact solution with Python
integers and fractions, and checks the following:

* the oracle is within 1e-7 px of it, and the kernel's arithmetic (replayed
  with Python ints and floats) within 1e-9 px, on full rings, short arcs
  (ill-conditioned), tiny rings and the largest annuli;
* singular systems (collinear points) are detected by both, with the exact
  determinant 0;
* the int64 moments and int128 determinants keep at least 8 bits of headroom
  at the parameter limits (r_max = 250, annulus_w = 64, every pixel of the
  annulus a ridge pixel).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ringdet as O


def moments(pts, ix, iy):
    u = [int(x) - ix for x in pts[:, 0]]
    v = [int(y) - iy for y in pts[:, 1]]
    z = [a * a + b * b for a, b in zip(u, v)]
    S = dict(uu=sum(a * a for a in u), uv=sum(a * b for a, b in zip(u, v)), vv=sum(b * b for b in v),
             u=sum(u), v=sum(v), n=len(u), uz=sum(a * c for a, c in zip(u, z)),
             vz=sum(b * c for b, c in zip(v, z)), z=sum(z))
    M = [[S["uu"], S["uv"], S["u"]], [S["uv"], S["vv"], S["v"]], [S["u"], S["v"], S["n"]]]
    rhs = [-S["uz"], -S["vz"], -S["z"]]
    return S, M, rhs


def det3(m, largest=None):
    """The kernel's cofactor expansion; `largest` (a list) receives the
    largest magnitude of any product it forms."""
    p = [m[1][1] * m[2][2], m[1][2] * m[2][1], m[1][0] * m[2][2], m[1][2] * m[2][0], m[1][0] * m[2][1],
         m[1][1] * m[2][0]]
    a, b, c = p[0] - p[1], p[2] - p[3], p[4] - p[5]
    q = [m[0][0] * a, m[0][1] * b, m[0][2] * c]
    if largest is not None:
        largest.append(max(abs(t) for t in p + q))
    return q[0] - q[1] + q[2]


def with_column(M, rhs, c):
    return [[rhs[i] if j == c else M[i][j] for j in range(3)] for i in range(3)]


def exact_fit(pts, ix, iy):
    """Centre and radius^2 as exact fractions, or None for a singular system."""
    _, M, rhs = moments(pts, ix, iy)
    det = det3(M)
    if det == 0:
        return None
    D, E, F = (Fraction(det3(with_column(M, rhs, c)), det) for c in range(3))
    return ix - D / 2, iy - E / 2, D * D / 4 + E * E / 4 - F


def i128_to_double(x: int) -> float:
    """The kernel's conversion: |x| as two 64-bit halves, each converted to
    double, then hi 2^64 + lo in double."""
    neg = x < 0
    u = -x if neg else x
    hi, lo = float(u >> 64), float(u & ((1 << 64) - 1))
    d = hi * 18446744073709551616.0 + lo
    return -d if neg else d


def kernel_fit(pts, ix, iy):
    _, M, rhs = moments(pts, ix, iy)
    det = det3(M)
    if len(pts) < 5 or det == 0:
        return None
    sol = [i128_to_double(det3(with_column(M, rhs, c))) / i128_to_double(det) for c in range(3)]
    D, E, F = sol
    rr = D * D / 4.0 + E * E / 4.0 - F
    if not rr > 0.0:
        return None
    return ix - D / 2.0, iy - E / 2.0, math.sqrt(rr)


def ring_points(rng, cx, cy, r, arc_deg=360.0, a0=0.0, noise=0.6, n=None):
    n = n or max(12, int(2 * math.pi * r * arc_deg / 360.0))
    t = np.deg2rad(a0 + rng.uniform(0, arc_deg, n))
    rr = r + rng.uniform(-noise, noise, n)
    pts = np.stack([np.rint(cx + rr * np.cos(t)), np.rint(cy + rr * np.sin(t))], 1).astype(np.int64)
    return np.unique(pts, axis=0)


def cases():
    rng = np.random.default_rng(23)
    out = []
    for _ in range(20):                                      # full rings, r 8-96
        r = rng.uniform(8, 96)
        out.append(ring_points(rng, 300 + rng.uniform(-1, 1), 300 + rng.uniform(-1, 1), r))
    for arc in (10.0, 20.0, 45.0, 90.0):                     # short arcs: ill-conditioned
        for _ in range(4):
            out.append(ring_points(rng, 500.3, 480.7, rng.uniform(30, 240), arc, rng.uniform(0, 360)))
    for r in (2.5, 3.0, 4.2):                                # tiny rings
        out.append(ring_points(rng, 50.5, 60.25, r, noise=0.3, n=40))
    out.append(ring_points(rng, 1000.4, 1000.6, 249.6, noise=20.0, n=4000))   # the largest radius, wide annulus
    return out


CASES = cases()


@pytest.mark.parametrize("i", range(len(CASES)))
def test_fit_against_exact_solution(i):
    pts = CASES[i]
    c = np.rint(pts.mean(0)).astype(int)                        # any integer reference works
    ix, iy = int(c[0]), int(c[1])
    ex = exact_fit(pts, ix, iy)
    assert ex is not None
    ecx, ecy, err2 = ex
    er = math.sqrt(float(err2))
    ocx, ocy, orr, n, flags = O.kasa_fit(pts, ix, iy, 10)
    assert flags == 0 and n == len(pts)
    kcx, kcy, kr = kernel_fit(pts, ix, iy)
    for got, tol in (((ocx, ocy, orr), 1e-7), ((kcx, kcy, kr), 1e-9)):
        assert abs(got[0] - float(ecx)) < tol and abs(got[1] - float(ecy)) < tol and abs(got[2] - er) < tol, \
            (i, got, (float(ecx), float(ecy), er))


def test_singular_systems():
    """Collinear points: the exact determinant is 0 and both the oracle and
    the kernel report FIT_FAIL with the integer peak."""
    for pts in (np.array([[x, 7] for x in range(10, 20)]), np.array([[3 + k, 5 + 2 * k] for k in range(8)]),
                np.array([[x, 2 * x - 1] for x in range(-5, 5)])):
        _, M, _ = moments(pts, 4, 4)
        assert det3(M) == 0
        assert kernel_fit(pts, 4, 4) is None
        cx, cy, r, n, flags = O.kasa_fit(pts, 4, 4, 9)
        assert flags == O.FIT_FAIL and (cx, cy, r) == (4.0, 4.0, 9.0)


def test_integer_headroom_at_the_limits():
    """r_max = 250 and annulus_w = 64: every pixel with 185 <= |p - c| <= 315
    (the membership bounds ir - w - 1 .. ir + w + 1) is a ridge pixel; on a
    half and a quarter annulus (asymmetric moments) the int64 moments stay
    below 2^55, and the int128 determinants and every product formed on the
    way below 2^119."""
    R_in, R_out = 250 - 64 - 1, 250 + 64 + 1
    ys, xs = np.mgrid[-R_out:R_out + 1, -R_out:R_out + 1]
    d2 = xs * xs + ys * ys
    ring = (d2 >= R_in * R_in) & (d2 <= R_out * R_out)
    for keep in (ring, ring & (xs >= 0), ring & (xs >= 0) & (ys >= 0)):
        pts = np.stack([xs[keep], ys[keep]], 1)
        S, M, rhs = moments(pts, 0, 0)
        assert max(abs(v) for v in S.values()) < 2 ** 55
        largest = []
        dets = [abs(det3(M, largest))] + [abs(det3(with_column(M, rhs, c), largest)) for c in range(3)]
        assert max(dets + largest) < 2 ** 119, math.log2(max(dets + largest))
