"""The oracle against hand-worked examples (CPU only).

The fixtures under ``tests/golden/`` were worked out by hand from the
definitions they cite (eigen-decomposition of 2 x 2 Hessians, directed votes,
circles through lattice points, curvature fields whose bilinear samples are
exact); none was produced by running code.  Each fixture is also checked for
internal consistency (H v = k v, |v| = 1, points on their circle) so that a
typing slip in a fixture shows up as such.  Planted mistakes in the oracle that
these examples cover must make one of them fail.
"""
import math
import os

import numpy as np
import pytest

from oracle import ringdet as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line


def _pairs(text):
    return [tuple(int(v) for v in tok.split(",")) for tok in text.split()]


# --------------------------------------------------------------------------
# fixture readers
# --------------------------------------------------------------------------
def eigen_cases():
    return [tuple(float(v) for v in r.split()) for r in _rows("eigen_worked.txt")]


def vote_cases():
    out = []
    for r in _rows("votes_worked.txt"):
        head, kept = r.split("|")
        x, y, X, Y, rad, c, H, W = head.split()
        out.append((int(x), int(y), float(X), float(Y), int(rad), int(c), int(H), int(W), _pairs(kept)))
    return out


def kasa_cases():
    out = []
    for r in _rows("kasa_worked.txt"):
        peak, pts, want = r.split("|")
        ix, iy, ir = (int(v) for v in peak.split())
        cx, cy, rr, n, flags = want.split()
        out.append((ix, iy, ir, np.array(_pairs(pts), dtype=np.int64), float(cx), float(cy), float(rr), int(n),
                    int(flags)))
    return out


def ridge_cases():
    out = []
    for r in _rows("ridge_worked.txt"):
        head, pix = r.split("|")
        name, H, W, tau, X, Y = head.split()
        out.append((name, int(H), int(W), float(tau), float(X), float(Y), sorted(_pairs(pix))))
    return out


def edge_cases():
    return [tuple(float(v) for v in r.split()) for r in _rows("edge_worked.txt")]


def ridge_field(name, H, W):
    if name == "valley":
        ys, xs = np.mgrid[0:H, 0:W]
        return (-5.0 + np.abs(xs - 3) + np.abs(ys - 3)).astype(np.float64)
    prof = np.array([1.0, 0.0, -1.0, -1.0, 0.0, 1.0, 2.0])
    if name == "plateau":
        return np.tile(prof, (H, 1))
    if name == "plateau_t":
        return np.tile(prof[:, None], (1, W))
    raise ValueError(name)


# --------------------------------------------------------------------------
# the fixtures are consistent with themselves
# --------------------------------------------------------------------------
def test_fixtures_are_consistent():
    assert len(eigen_cases()) == 13 and len(vote_cases()) == 14 and len(kasa_cases()) == 4
    for a, c, b, k, X, Y, deg in eigen_cases():
        H = np.array([[a, b], [b, c]])
        assert k == pytest.approx(min(np.linalg.eigvalsh(H)), abs=1e-12)
        if not deg:
            v = np.array([X, Y])
            assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-15)
            assert np.allclose(H @ v, k * v, atol=1e-14)
            assert X > 0 or (X == 0 and Y > 0)
        else:
            assert b == 0 and a == c
    for ix, iy, ir, pts, cx, cy, rr, n, flags in kasa_cases():
        assert len(pts) == n and len(set(map(tuple, pts.tolist()))) == n
        if flags == 0:
            d = np.hypot(pts[:, 0] - cx, pts[:, 1] - cy)
            assert np.allclose(d, rr, atol=1e-12)
    for x, y, X, Y, r, c, H, W, kept in vote_cases():
        assert len(kept) <= 2
    for g0, g1, g, X, Y, deg in edge_cases():
        assert g == pytest.approx(math.hypot(g0, g1), abs=1e-15)
        if not deg:
            assert abs(X * g - g0) < 1e-14 or abs(X * g + g0) < 1e-14


# --------------------------------------------------------------------------
# the oracle reproduces them
# --------------------------------------------------------------------------
def check_eigen():
    rows = np.array(eigen_cases())
    k, X, Y, deg = O.eigen(rows[:, 0], rows[:, 1], rows[:, 2])
    assert np.array_equal(deg, rows[:, 6].astype(bool))
    assert np.allclose(k, rows[:, 3], rtol=0, atol=1e-14)
    assert np.allclose(X, rows[:, 4], rtol=0, atol=1e-15)
    assert np.allclose(Y, rows[:, 5], rtol=0, atol=1e-15)


def check_votes():
    for x, y, X, Y, r, c, H, W, kept in vote_cases():
        bx, by = O.cast_votes(np.array([x]), np.array([y]), np.array([X]), np.array([Y]), r, H, W, c)
        assert list(zip(bx.tolist(), by.tolist())) == kept, (x, y, X, Y, r, c)


def check_kasa():
    for ix, iy, ir, pts, cx, cy, rr, n, flags in kasa_cases():
        got = O.kasa_fit(pts, ix, iy, ir)
        assert got[3] == n and got[4] == flags
        assert np.allclose(got[:3], (cx, cy, rr), rtol=0, atol=1e-12), (got, cx, cy, rr)


def check_ridges():
    for name, H, W, tau, X, Y, want in ridge_cases():
        k = ridge_field(name, H, W)
        mask = O.ridge_mask(k, np.full((H, W), X), np.full((H, W), Y), np.zeros((H, W), bool), tau)
        ys, xs = np.nonzero(mask)
        assert sorted(zip(xs.tolist(), ys.tolist())) == want, name


def check_edges():
    rows = np.array(edge_cases())
    g, X, Y, deg = O.edge_direction(rows[:, 0], rows[:, 1])
    assert np.array_equal(deg, rows[:, 5].astype(bool))
    assert np.allclose(g, rows[:, 2], rtol=0, atol=1e-15)
    assert np.allclose(X, rows[:, 3], rtol=0, atol=1e-15)
    assert np.allclose(Y, rows[:, 4], rtol=0, atol=1e-15)


CHECKS = {"eigen": check_eigen, "votes": check_votes, "kasa": check_kasa, "ridges": check_ridges,
          "edges": check_edges}


@pytest.mark.parametrize("name", sorted(CHECKS))
def test_oracle_matches_worked_examples(name):
    CHECKS[name]()


def test_degenerate_pixels_are_never_ridges():
    """A degenerate flag removes a pixel that the valley example keeps."""
    k = ridge_field("valley", 7, 7)
    deg = np.zeros((7, 7), bool)
    deg[3, 3] = True
    mask = O.ridge_mask(k, np.full((7, 7), 0.6), np.full((7, 7), 0.8), deg, 0.0)
    ys, xs = np.nonzero(mask)
    assert sorted(zip(xs.tolist(), ys.tolist())) == [(1, 3), (2, 3), (4, 3), (5, 3)]


# planted mistakes (from the mutation suite) that a worked example covers
_CAUGHT = ["larger_eigenvalue", "one_sign_votes", "truncating_votes", "kasa_centre_sign",
           "ridge_nonstrict_both", "coarse_floor_cells"]


@pytest.mark.parametrize("mut", _CAUGHT)
def test_worked_examples_catch_planted_mistakes(mut, monkeypatch):
    from tests.test_oracle_mutations import MUTATIONS
    attr, fn = MUTATIONS[mut]
    monkeypatch.setattr(O, attr, fn)
    failed = []
    for name, check in CHECKS.items():
        try:
            check()
        except AssertionError:
            failed.append(name)
    assert failed, f"planted mistake {mut} passed every worked example"
