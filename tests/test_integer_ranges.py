"""The exact integer stages never overflow (CPU): for every sigma the
detector accepts, the ranges its kernels rely on hold on the worst input,
a frame of all 65535.

* A stencil tile whose inputs are at most narrow_max = floor((2^32 - 1) /
  (2 S)) keeps every horizontal Gaussian sum P = sum Q_i I below 2^31 and
  the pair P_j + P_{2R-j} that the vertical pass forms before its multiply
  below 2^32; narrow_max is at least 4095, so 8-bit and 12-bit frames are
  always narrow.
* A wider tile is smoothed once per byte of its inputs (high, then low):
  each part's horizontal sums stay below 2^28 and L' = 2^8 L'(high) +
  L'(low) below 2^54 (u64).
* The second-order Sobel sums H' = (stencil) * L' stay below 2^60 in
  magnitude (int64 with room); the first-order Sobel of the edge variant
  below 2^61.  Above 2^53 the oracle's and the kernels' conversion of H' to
  float64 rounds to nearest (ties to even) on both sides.
The oracle's taps are the kernels' (checked in the ABI tests)."""
import numpy as np
import pytest

from oracle import ringdet as O

SIGMAS = [0.05, 0.3, 0.5, 0.75, 1.0, 1.3, 1.5, 1.75, 2.0, 2.5, 3.0, 3.5, 3.9, 4.0]


@pytest.mark.parametrize("sigma", SIGMAS)
def test_worst_case_ranges(sigma):
    s32 = float(np.float32(sigma))
    Q = O.gaussian_taps(s32).astype(object)
    S = int(sum(Q))
    assert all(q >= 0 for q in Q)
    narrow_max = (2 ** 32 - 1) // (2 * S)
    assert narrow_max >= 4095                      # 8- and 12-bit frames take the u32 path
    P = narrow_max * S                             # largest horizontal sum of a narrow tile
    assert P < 2 ** 31 and 2 * P < 2 ** 32         # u32 sum, and the vertical pass's pair
    Pb = 255 * S                                   # one byte per part of a wide tile
    assert 2 * Pb < 2 ** 28
    Imax = 65535
    L = Imax * S * S
    assert (2 ** 8) * (255 * S * S) + 255 * S * S == L
    assert L < 2 ** 54                             # u64 with 10 bits to spare
    # second-order Sobel: |d2| x |s| has coefficient mass 4 x 16 = 64 (and 6 x 6 = 36 for Lxy)
    assert 64 * L < 2 ** 60
    # first-order Sobel of the edge variant: |d1| x |s| = 6 x 16 = 96
    assert 96 * L < 2 ** 61


def test_stencil_coefficients():
    """The Sobel stencils' absolute coefficient masses used above."""
    assert int(np.abs(O.SOBEL_D2).sum()) * int(np.abs(O.SOBEL_S).sum()) == 64
    assert int(np.abs(O.SOBEL_D1).sum()) ** 2 == 36
    assert int(np.abs(O.SOBEL_D1).sum()) * int(np.abs(O.SOBEL_S).sum()) == 96


def test_worst_case_frame_is_exact():
    """The oracle's own integer path on an all-65535 frame at sigma 4 (the
    widest taps): L' is exactly 65535 S^2 everywhere and H' is 0."""
    img = np.full((40, 40), 65535, dtype=np.uint16)
    Lp, S = O.smooth_int(img, 4.0)
    assert np.all(Lp == 65535 * S * S)
    for h in O.hessian_int(Lp):
        assert not h.any()


def _annulus_lattice_count(r, halfwidth):
    """Integer offsets p with r - halfwidth <= |p| <= r + halfwidth."""
    R = int(np.ceil(r + halfwidth)) + 1
    ys, xs = np.mgrid[-R:R + 1, -R:R + 1]
    d = np.hypot(xs, ys)
    return int(((d >= r - halfwidth) & (d <= r + halfwidth)).sum())


@pytest.mark.parametrize("c", [1, 2, 4])
def test_vote_counts_fit_u16(c):
    """The voting kernel keeps one level's counts as packed u16: no voxel may
    reach 65536 votes, or the carry would spill into its neighbour.  A pixel
    p votes into the voxel (cell) v at radius r only if p + s r X- rounds into
    v's cell, i.e. |p - centre(v)| is within r +- c / sqrt 2 (the cell's
    half-diagonal, plus 1/2 px rounding at c = 1), and it casts at most two
    votes per level.  Even with every pixel of that annulus a ridge pixel,
    at the largest voted radius (r_max + 1 = 251) the count stays far below
    2^16."""
    hw = c / np.sqrt(2.0) + 0.5
    worst = max(_annulus_lattice_count(r, hw) for r in (2, 10, 50, 100, 200, 251))
    assert 2 * worst < 65536, worst
