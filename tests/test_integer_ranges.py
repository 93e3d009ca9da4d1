"""The exact integer stages never overflow (CPU): for every sigma the
detector accepts, the ranges its kernels rely on hold on the worst input,
a frame of all 65535.

* horizontal Gaussian sums P = sum Q_i I fit u32, and so does the pair
  P_j + P_{2R-j} that the vertical pass forms before its multiply;
* L' = sum Q_j P fits well inside u64, and is exact in float64 (< 2^53);
* the second-order Sobel sums H' = (stencil) * L' stay below 2^52 in
  magnitude (int64 with room, and the FP32 path's bound takes |L'| < 2^53);
* the first-order Sobel of the edge variant likewise.
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
    Imax = 65535
    P = Imax * S                                   # every horizontal sum of the all-65535 frame
    assert P < 2 ** 31 and 2 * P < 2 ** 32         # u32 sum, and the vertical pass's pair
    L = P * S
    assert L < 2 ** 53                             # exact in float64; u64 with 11 bits to spare
    # second-order Sobel: |d2| x |s| has coefficient mass 4 x 16 = 64 (and 6 x 6 = 36 for Lxy)
    assert 64 * L < 2 ** 52
    # first-order Sobel of the edge variant: |d1| x |s| = 6 x 16 = 96
    assert 96 * L < 2 ** 53


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
