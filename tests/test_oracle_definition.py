"""The oracle's quantised weights against the paper's real-valued ones (CPU).

The exact oracle quantises two sets of weights so that both it and the
kernels compute in integers: the Gaussian taps of the smoothing step (Methods,
"Algorithm implementation": Gaussian smoothing before the Sobel derivatives)
to multiples of 2^-19, and the level-smoothing weights exp(-d^2 / (2
sigma(r)^2)), sigma(r) = 0.05 r + 0.25 (Results, "Local maxima detection in a
noisy parameter space"; Methods) to multiples of 2^-16.  ``detect_definition``
runs the same steps in float64 with the weights as the paper defines them.

* The definition mode's own plumbing is tied to the pinned oracle: with the
  quantised weights (``quantised=True``) it reproduces the exact oracle's
  ridge set, peaks and fits.
* On the workloads' frames (configs 1-4) the quantised and the real-valued
  weights give identical integer peak sets and fits within 0.01 px; at most
  two ridge pixels per frame may differ (near-ties of the definition within
  the taps' 2^-20 quantisation error).
* The paired float64 stencils keep the exact mirror identities of reflect-101
  borders (Lxy is exactly 0 on them), which the exact integer path has.
"""
import numpy as np
import pytest

from oracle import ringdet as O
from paper_1310_1371_gb300 import synth


def _peaks(res):
    return {(int(r["ix"]), int(r["iy"]), int(r["ir"])): r for r in res.rings}


def _ridges(res):
    return set(map(tuple, res.ridge_xy.tolist()))


def _compare(a, b, max_ridge_diff, fit_tol):
    pa, pb = _peaks(a), _peaks(b)
    assert set(pa) == set(pb), (sorted(set(pa) - set(pb)), sorted(set(pb) - set(pa)))
    assert len(_ridges(a) ^ _ridges(b)) <= max_ridge_diff, len(_ridges(a) ^ _ridges(b))
    for k in pa:
        d = max(abs(pa[k]["cx"] - pb[k]["cx"]), abs(pa[k]["cy"] - pb[k]["cy"]), abs(pa[k]["r"] - pb[k]["r"]))
        assert d <= fit_tol, (k, d)
        assert pa[k]["flags"] == pb[k]["flags"]
    return len(pa)


def test_definition_weights():
    """Real-valued taps sum to 1 and the quantised ones are within 2^-20 of
    them; real level weights peak at exactly 1 and the quantised ones are
    within 2^-17."""
    for sigma in (0.7, 1.3, 2.0, 3.5):
        s32 = float(np.float32(sigma))
        g = O.gaussian_taps_fp64(s32)
        assert abs(g.sum() - 1.0) < 1e-15 and np.array_equal(g, g[::-1]) and g.argmax() == len(g) // 2
        Q = O.gaussian_taps(s32)
        assert np.max(np.abs(Q / 2.0 ** 19 - g)) <= 2.0 ** -20
    for r in (5, 20, 96, 160):
        w = O.smoothing_weights_fp64(r, float(np.float32(0.05)), float(np.float32(0.25)))
        Rs = (w.shape[0] - 1) // 2
        assert w[Rs, Rs] == 1.0 and np.all(w > 0) and np.all(w <= 1)
        wq = O.smoothing_weights_fp64(r, float(np.float32(0.05)), float(np.float32(0.25)), quantised=True)
        assert wq.shape == w.shape and np.max(np.abs(wq - w)) <= 2.0 ** -17


def test_paired_stencils_keep_mirror_identities():
    """With reflect-101 borders the mixed derivative of any image is exactly
    0 on the first and last row and column (the stencil is antisymmetric
    about the mirror axis); the definition mode's float64 sums keep that, so
    border ridge pixels with an exactly axial X- are decided as in exact
    arithmetic."""
    rng = np.random.default_rng(5)
    img = rng.integers(0, 4096, size=(40, 52)).astype(np.uint16)
    lxx, lyy, lxy = O.hessian_fp64(img, 2.0)
    assert not lxy[:, 0].any() and not lxy[:, -1].any() and not lxy[0].any() and not lxy[-1].any()
    # the exact integer Hessian agrees (same identity, exact arithmetic)
    hxy = O.hessian_int(O.smooth_int(img, 2.0)[0])[2]
    assert not hxy[:, 0].any() and not hxy[0].any()
    # a constant frame: smoothing is exact and every second derivative is 0
    c = np.full((30, 30), 1234, dtype=np.uint16)
    for h in O.hessian_fp64(c, 2.0):
        assert not np.any(np.abs(h) > 1e-9)


def test_quantised_float_mode_reproduces_exact_oracle():
    """detect_definition(quantised=True) evaluates the exact oracle's
    quantised weights in float64: same ridge set, same peaks, same fits."""
    for img, params in ((synth.plain_small().image, synth.PLAIN_SMALL_PARAMS),
                        (np.ascontiguousarray(synth.plain_full().image[300:556, 200:456]), synth.PLAIN_FULL_PARAMS)):
        p = O.Params.make(**params)
        a = O.detect(img, p)
        b = O.detect_definition(img, p, quantised=True)
        assert _ridges(a) == _ridges(b)
        assert _compare(a, b, 0, 1e-9) > 0


def _cases():
    out = [(f"config1_seed{i}", lambda i=i: (synth.plain_small(seed=[1001, i]).image, synth.PLAIN_SMALL_PARAMS))
           for i in range(4)]
    out += [("config2_frame0", lambda: (synth.plain_full().image, synth.PLAIN_FULL_PARAMS)),
            ("config2_frame1", lambda: (synth.plain_full(seed=[1002, 1]).image, synth.PLAIN_FULL_PARAMS))]

    def video(i):
        tracks = synth.video_tracks(i + 1)
        return synth.video_frame(i, tracks[i]), synth.VIDEO_PARAMS
    out += [("config3_frame0", lambda: video(0)), ("config3_frame1", lambda: video(1))]
    out += [("config4_frame0", lambda: (synth.diff_frame(0).image, synth.DIFF_PARAMS))]
    return out


CASES = _cases()


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_quantisation_changes_no_ring(idx):
    """Quantised against real-valued Gaussian taps and level weights:
    identical integer peak sets, fits within 0.01 px, at most two ridge
    pixels apart.  Integer frames take the exact oracle; the float frames of
    config 4 take the float64 evaluation of the quantised weights."""
    name, make = CASES[idx]
    img, params = make()
    p = O.Params.make(**params)
    quant = O.detect(img, p) if img.dtype.kind in "ui" else O.detect_definition(img, p, quantised=True)
    real = O.detect_definition(img, p)
    n = _compare(quant, real, 2, 0.01)
    assert n >= 5, (name, n)
