"""The accumulator geometry (tile edge, slab depth) changes speed only:
every geometry gives the same rings, bit for bit, and the same counts; the
autotuner returns one of them and contexts created afterwards use it."""
import numpy as np
import pytest

from oracle import ringdet as O
from paper_1310_1371_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit", "flags")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def run(torch, frames, params, geometry=None):
    from paper_1310_1371_gb300 import rd
    H, W = frames[0].shape
    det = rd.Detector(params, H, W, len(frames), geometry=geometry)
    rings, stats = det.detect(torch.from_numpy(np.stack(frames)).cuda())
    geo = det.geometry()
    det.close()
    return rings, stats, geo


def same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        for k in FIELDS:
            assert np.array_equal(x[k], y[k]), k


@pytest.mark.parametrize("geometry", [(64, 8), (64, 4), (80, 12), (96, 12), (96, 16), (128, 16), (128, 8),
                                      (128, 32), (128, 64), (64, 40)])
def test_geometry_does_not_change_results(torch, geometry):
    frames = [synth.plain_small(seed=s).image for s in (51, 52)]
    params = synth.PLAIN_SMALL_PARAMS
    ref_rings, ref_stats, _ = run(torch, frames, params, (64, 8))
    rings, stats, geo = run(torch, frames, params, geometry)
    assert geo == geometry
    same(rings, ref_rings)
    for k in ("ridge_pixels", "votes", "hotspots", "smooth_macs", "peaks"):
        assert getattr(stats, k) == getattr(ref_stats, k), k
    # and against the oracle's integer peaks
    ref = O.detect(frames[0], O.Params.make(**params))
    key = lambda r: list(zip(np.asarray(r["ix"]).tolist(), np.asarray(r["iy"]).tolist(), np.asarray(r["ir"]).tolist()))
    assert key(rings[0]) == key(ref.rings)


def test_ragged_frame_every_geometry(torch):
    """A ragged frame (partial tiles on two sides) under each tile edge."""
    f = synth.plain_small(seed=53, H=203, W=341, n_rings=10)
    params = synth.PLAIN_SMALL_PARAMS
    base, bstats, _ = run(torch, [f.image], params, (96, 12))
    for geometry in [(64, 8), (80, 16), (64, 5), (128, 16)]:
        rings, stats, _ = run(torch, [f.image], params, geometry)
        same(rings, base)
        assert stats.votes == bstats.votes and stats.hotspots == bstats.hotspots


def test_autotune_choice_is_used(torch):
    from paper_1310_1371_gb300 import rd
    frames = [synth.plain_small(seed=s).image for s in (61, 62, 63, 64)]
    params = dict(synth.PLAIN_SMALL_PARAMS, r_max=39)  # a key no other test tunes
    t = torch.from_numpy(np.stack(frames)).cuda()
    best = rd.rd_autotune(params, t)
    assert best[0] in (64, 80, 96, 128) and best[1] in (8, 16, 24, 32)
    det = rd.Detector(params, 256, 256, 4)  # automatic geometry: the tuned one
    assert det.geometry() == best
    rings, _ = det.detect(t)
    det.close()
    ref, _, _ = run(torch, frames, params, (64, 8))
    same(rings, ref)
