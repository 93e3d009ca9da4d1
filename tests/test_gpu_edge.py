"""Directed-edge variant on the GPU against the oracle's edge mode: the same
edge pixels and directions, bit-exact vote and hotspot counts, identical
integer peaks, sub-pixel fits within 0.01 px."""
import numpy as np
import pytest

from oracle import ringdet as O
from paper_1310_1371_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def key(r):
    return list(zip(np.asarray(r["ix"]).tolist(), np.asarray(r["iy"]).tolist(), np.asarray(r["ir"]).tolist()))


def run_edge(torch, image, params, dense=False):
    from paper_1310_1371_gb300 import rd
    H, W = image.shape
    det = rd.Detector(params, H, W, 1)
    det.set_features("edge", params["edge_thresh"])
    if dense:
        det.debug_route(True)
    rings, stats = det.detect(torch.from_numpy(image[None].copy()).cuda())
    xy, d, _ = det.debug_ridges(0)
    det.close()
    return rings[0], stats, xy, d


def check(torch, image, params, dense=False):
    p = O.Params.make(**params)
    ref = O.detect(image, p)
    rings, stats, xy, d = run_edge(torch, image, params, dense)
    o = np.lexsort((xy[:, 0], xy[:, 1]))
    xy, d = xy[o], d[o]
    assert np.array_equal(xy, ref.ridge_xy), "edge pixel sets differ"
    assert np.abs(d - ref.ridge_X).max() < 1.2e-7
    assert stats.votes == ref.votes_in and stats.hotspots == ref.hotspots and stats.smooth_macs == ref.smooth_macs
    assert key(rings) == key(ref.rings), "integer peak sets differ"
    for a in ("cx", "cy", "r"):
        assert np.abs(np.asarray(rings[a], np.float64) - ref.rings[a]).max() <= 0.01
    return rings, ref


@pytest.mark.parametrize("seed", [3001, 3003])
def test_small_discs(torch, seed):
    f = synth.disc_small(seed=seed)
    rings, ref = check(torch, f.image, f.params)
    assert len(ref.rings) >= 6


def test_small_discs_dense_route(torch):
    f = synth.disc_small(seed=3004)
    check(torch, f.image, f.params, dense=True)


def test_full_size_discs(torch):
    f = synth.disc_full()
    rings, ref = check(torch, f.image, f.params)
    assert len(ref.rings) > 100


def test_back_to_ridges(torch):
    """Switching the feature stage back restores the method's results."""
    from paper_1310_1371_gb300 import rd
    f = synth.plain_small(seed=3005)
    t = torch.from_numpy(f.image[None].copy()).cuda()
    a = rd.Detector(f.params, 256, 256, 1)
    ra, sa = a.detect(t)
    b = rd.Detector(f.params, 256, 256, 1)
    b.set_features("edge", 4.0)
    b.detect(t)
    b.set_features("ridge")
    rb, sb = b.detect(t)
    assert key(rb[0]) == key(ra[0]) and sb.votes == sa.votes
    for k in ("cx", "cy", "r", "score", "n_fit"):
        assert np.array_equal(rb[0][k], ra[0][k])
    a.close()
    b.close()
