"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300).

Gates (from the method's definition; integer work is exact):
* ridge pixels identical (as a set), with identical exact Hessians;
* raw accumulators bit-exact at every level, smoothed accumulators too;
* integer (x, y, r) peak sets identical;
* sub-pixel centre and radius within 0.01 px, scores within 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import ringdet as O
from paper_1310_1371_gb300 import synth

pytestmark = pytest.mark.gpu

SUBPX_TOL = 0.01


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def run(torch, frames, params, capture=False, max_hw=None, dense=False, bin_global=False):
    from paper_1310_1371_gb300 import rd
    frames = [np.ascontiguousarray(f) for f in frames]
    H, W = frames[0].shape
    mh, mw = max_hw or (H, W)
    det = rd.Detector(params, mh, mw, len(frames))
    if dense or bin_global:
        det.debug_route(dense, bin_global)
    t = torch.from_numpy(np.stack(frames)).cuda()
    acc = sm = None
    if capture:
        nl = params["r_max"] - params["r_min"] + 3
        acc = torch.zeros((nl, H, W), dtype=torch.int32, device="cuda")
        sm = torch.zeros((nl, H, W), dtype=torch.int32, device="cuda")
        det.debug_capture(acc, sm)
    rings, stats = det.detect(t)
    ridges = [det.debug_ridges(i) for i in range(len(frames))]
    out = dict(rings=rings, stats=stats, ridges=ridges)
    if capture:
        out["acc"] = acc.cpu().numpy()
        out["sm"] = sm.cpu().numpy().view(np.uint32)
    det.close()
    return out


def ring_keys(r):
    return list(zip(np.asarray(r["ix"]).tolist(), np.asarray(r["iy"]).tolist(), np.asarray(r["ir"]).tolist()))


def assert_rings_match(got, ref):
    assert ring_keys(got) == ring_keys(ref), "integer peak sets differ"
    if len(ref) == 0:
        return
    for k in ("cx", "cy", "r"):
        d = np.abs(got[k].astype(np.float64) - ref[k]).max()
        assert d <= SUBPX_TOL, (k, d)
    assert np.allclose(got["score"], ref["score"], rtol=1e-6, atol=0)
    assert np.array_equal(got["n_fit"], ref["n_fit"])
    assert np.array_equal(got["flags"], ref["flags"])


def assert_ridges_match(ridge, image, p):
    xy, d, h = ridge
    Lp, S = O.smooth_int(image, p.sigma)
    hxx, hyy, hxy = O.hessian_int(Lp)
    ref_xy, ref_X = O.directed_ridges(image, p)
    order = np.lexsort((xy[:, 0], xy[:, 1]))
    xy, d, h = xy[order], d[order], h[order]
    assert len(xy) == len(ref_xy), (len(xy), len(ref_xy))
    assert np.array_equal(xy, ref_xy), "ridge pixel sets differ"
    ys, xs = ref_xy[:, 1], ref_xy[:, 0]
    assert np.array_equal(h[:, 0], hxx[ys, xs]) and np.array_equal(h[:, 1], hyy[ys, xs])
    assert np.array_equal(h[:, 2], hxy[ys, xs])
    if len(xy) == 0:
        return
    # direction: same line (sign conventions agree except where X == 0 to
    # within rounding), within float32 rounding of the exact direction
    dot = np.abs((d.astype(np.float64) * ref_X).sum(1))
    assert np.all(dot > 1 - 1e-6)
    assert np.abs(np.abs(d) - np.abs(ref_X)).max() < 1.2e-7


def check_frame(torch, image, params, capture=False, dense=False):
    p = O.Params.make(**params)
    out = run(torch, [image], params, capture=capture, dense=dense)
    ref = O.detect(image, p, keep=capture)
    assert_ridges_match(out["ridges"][0], image, p)
    assert out["stats"].votes == ref.votes_in
    assert out["stats"].hotspots == ref.hotspots
    assert out["stats"].smooth_macs == ref.smooth_macs
    if capture:
        levels = O.radius_levels(p.r_min, p.r_max)
        for li, r in enumerate(levels):
            assert np.array_equal(out["acc"][li], ref.A[int(r)]), f"raw accumulator differs at r={r}"
            assert np.array_equal(out["sm"][li].astype(np.int64), ref.N[int(r)]), f"smoothed differs at r={r}"
    assert_rings_match(out["rings"][0], ref.rings)
    return out, ref


# ------------------------------------------------------------------ small frames
def test_plain_small_stagewise(torch):
    f = synth.plain_small()
    out, ref = check_frame(torch, f.image, f.params, capture=True)
    assert len(ref.rings) == 8


def test_plain_small_dense_route(torch):
    """The dense-storage voting kernel (the fallback for crowded tiles) on
    every tile gives the same accumulators and rings."""
    f = synth.plain_small(seed=14)
    check_frame(torch, f.image, f.params, capture=True, dense=True)


def test_plain_full_dense_route(torch):
    f = synth.plain_full(seed=[1002, 3])
    check_frame(torch, f.image, f.params, dense=True)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_plain_small_other_seeds(torch, seed):
    f = synth.plain_small(seed=seed)
    check_frame(torch, f.image, f.params, capture=True)


def test_ragged_frame_and_borders(torch):
    # odd size (partial stencil and accumulator tiles), rings cut by the border
    rng = np.random.default_rng(5)
    H, W = 77, 131
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    img = np.full((H, W), 40.0)
    for cx, cy, R in [(3.2, 5.1, 14.0), (128.5, 70.0, 20.3), (60.0, 38.0, 11.6), (100.0, 10.0, 25.0)]:
        img += 120 * np.exp(-0.5 * ((np.hypot(xx - cx, yy - cy) - R) / 1.5) ** 2)
    img = np.clip(np.rint(img + rng.normal(0, 8, img.shape)), 0, 255).astype(np.uint8)
    params = dict(synth.PLAIN_SMALL_PARAMS, r_max=30)
    check_frame(torch, img, params, capture=True)


def test_large_radius_range_small_tiles(torch):
    """Search radii up to 170: the dense voting kernel's per-tile storage for
    96-pixel accumulator tiles (window halo 28 px) no longer fits one SM, so
    the context works on 64-pixel tiles; both voting routes must still agree
    with the oracle, the largest ring (r = 140) included."""
    rng = np.random.default_rng(41)
    H = W = 320
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    img = np.full((H, W), 40.0)
    for cx, cy, R in [(160.3, 158.7, 140.0), (60.2, 70.5, 20.0), (250.0, 240.0, 35.5), (120.6, 200.2, 52.0)]:
        img += 120 * np.exp(-0.5 * ((np.hypot(xx - cx, yy - cy) - R) / 1.5) ** 2)
    img = np.clip(np.rint(img + rng.normal(0, 8, img.shape)), 0, 255).astype(np.uint8)
    params = dict(synth.PLAIN_SMALL_PARAMS, r_min=5, r_max=170)
    out, ref = check_frame(torch, img, params)
    assert len(ref.rings) == 4 and max(r[2] for r in ref.rings) > 139
    check_frame(torch, img, params, dense=True)


def test_flat_frame_has_nothing(torch):
    img = np.full((64, 64), 100, dtype=np.uint8)
    out, ref = check_frame(torch, img, synth.PLAIN_SMALL_PARAMS)
    assert out["stats"].ridge_pixels == 0 and len(out["rings"][0]) == 0


def test_minimum_frame(torch):
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, size=(12, 12)).astype(np.uint8)
    check_frame(torch, img, dict(synth.PLAIN_SMALL_PARAMS, r_min=2, r_max=6, ridge_thresh=-0.5), capture=True)


def test_axis_aligned_lines_exact_path(torch):
    # exactly axis-aligned directions and exact plateaus (ties everywhere)
    H, W = 48, 50
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    img = 20 + 200 * np.exp(-0.5 * ((xx - 20.5) / 1.5) ** 2) + 150 * np.exp(-0.5 * ((yy - 30.0) / 1.5) ** 2)
    img = np.rint(img).astype(np.uint16)
    check_frame(torch, img, dict(synth.PLAIN_SMALL_PARAMS, r_min=4, r_max=12), capture=True)


def test_full_range_u16(torch):
    # 16-bit extremes exercise the integer stencil's headroom
    rng = np.random.default_rng(3)
    H, W = 96, 96
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    img = 2000 + 60000 * np.exp(-0.5 * ((np.hypot(xx - 47.3, yy - 50.2) - 25.0) / 1.5) ** 2)
    img = np.clip(np.rint(img + rng.normal(0, 300, img.shape)), 0, 65535).astype(np.uint16)
    img[0, :] = 65535
    img[:, -1] = 0
    params = dict(synth.PLAIN_FULL_PARAMS, r_min=8, r_max=40, ridge_thresh=-50.0)
    check_frame(torch, img, params, capture=True)


def test_u8_equals_u16(torch):
    f = synth.plain_small(seed=21)
    a = run(torch, [f.image], f.params)
    b = run(torch, [f.image.astype(np.uint16)], f.params)
    for k in ("ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit"):
        assert np.array_equal(a["rings"][0][k], b["rings"][0][k])


def test_batch_equals_single(torch):
    frames = [synth.plain_small(seed=s).image for s in (31, 32, 33)]
    params = synth.PLAIN_SMALL_PARAMS
    batch = run(torch, frames, params)
    for i, img in enumerate(frames):
        one = run(torch, [img], params)
        g, s = batch["rings"][i], one["rings"][0]
        for k in ("ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit", "flags"):
            assert np.array_equal(g[k], s[k]), (i, k)
        assert np.all(g["frame"] == i) and np.all(s["frame"] == 0)


# ------------------------------------------------------------------ full size
def test_plain_full_frame(torch):
    f = synth.plain_full()
    out, ref = check_frame(torch, f.image, f.params)
    assert len(ref.rings) > 100


def test_plain_full_batch_sampled(torch):
    """The batched launch of the benchmark workload; frames 0 and 5 are
    compared in full with the oracle."""
    n = 8
    frames = [fr.image for fr in synth.plain_full_batch(n)]
    params = synth.PLAIN_FULL_PARAMS
    out = run(torch, frames, params)
    p = O.Params.make(**params)
    for i in (0, 5):
        ref = O.detect(frames[i], p)
        assert_rings_match(out["rings"][i], ref.rings)
        assert_ridges_match(out["ridges"][i], frames[i], p)


def test_global_bin_counters_equal_shared_ones(torch):
    """Binning with global atomic counters (the route of frames with more than
    8192 accumulator bins) gives the same rings and the same vote, hotspot and
    smoothing counts as the per-CTA shared-memory counters, on a batch of the
    benchmark workload and on small frames with many CTAs per frame."""
    cases = [([fr.image for fr in synth.plain_full_batch(4)], synth.PLAIN_FULL_PARAMS),
             ([synth.plain_small(seed=s).image for s in (41, 42)], synth.PLAIN_SMALL_PARAMS)]
    for frames, params in cases:
        a = run(torch, frames, params)
        b = run(torch, frames, params, bin_global=True)
        for i in range(len(frames)):
            for k in ("ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit", "flags"):
                assert np.array_equal(a["rings"][i][k], b["rings"][i][k]), (i, k)
        for k in ("ridge_pixels", "votes", "peaks", "hotspots", "smooth_macs", "overflow"):
            assert getattr(a["stats"], k) == getattr(b["stats"], k), k
        assert a["stats"].votes > 0


def test_crowded_bins_hand_off_to_dense(torch):
    """vote_thresh 0 makes every touched voxel a hotspot and peak_frac 0 lets
    most of them pass the float threshold, so tiles overflow the sparse
    kernel's hotspot and peak lists and are handed to the dense kernel mid-way
    (the sparse kernel's abort path) -- the result is still the oracle's."""
    f = synth.plain_small(seed=15)
    params = dict(f.params, vote_thresh=0, peak_frac=0.0, r_min=5, r_max=20)
    check_frame(torch, f.image, params, capture=True)
