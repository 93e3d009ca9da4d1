"""Graph mode: rd_detect captured once into a CUDA graph and replayed gives
the eager results, follows new frame contents at the same address, and
refuses the legacy default stream."""
import numpy as np
import pytest

from paper_1310_1371_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("frame", "ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit", "flags")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        for k in FIELDS:
            assert np.array_equal(x[k], y[k]), k


def eager(torch, frames, params):
    from paper_1310_1371_gb300 import rd
    det = rd.Detector(params, 256, 256, len(frames))
    rings, stats = det.detect(torch.from_numpy(np.stack(frames)).cuda())
    det.close()
    return rings, stats


def test_graph_replay_matches_eager(torch):
    from paper_1310_1371_gb300 import rd
    params = synth.PLAIN_SMALL_PARAMS
    first = [synth.plain_small(seed=s).image for s in (71, 72, 73)]
    second = [synth.plain_small(seed=s).image for s in (74, 75, 76)]
    ref1, st1 = eager(torch, first, params)
    ref2, st2 = eager(torch, second, params)
    det = rd.Detector(params, 256, 256, 3)
    det.set_graph(True)
    stream = torch.cuda.Stream()
    t = torch.from_numpy(np.stack(first)).cuda()
    torch.cuda.synchronize()
    for _ in range(3):  # the first call captures, the others replay
        rings, stats = det.detect(t, stream=stream)
        same(rings, ref1)
        assert stats.votes == st1.votes and stats.hotspots == st1.hotspots
    with torch.cuda.stream(stream):
        t.copy_(torch.from_numpy(np.stack(second)).cuda())
    rings, stats = det.detect(t, stream=stream)  # same address, new contents
    same(rings, ref2)
    assert stats.votes == st2.votes
    with pytest.raises(rd.RdError) as ei:
        det.detect_async(t, stream=torch.cuda.default_stream())
    assert ei.value.status == rd.RD_E_INVAL
    det.set_graph(False)  # back to eager launches on the default stream
    rings, _ = det.detect(t)
    same(rings, ref2)
    det.close()
