"""Drifting-track video (1024x1024 u8, 20-300 rings per frame): the batched
path (autotuned geometry, persistent voting, CUDA-graph replay) gives, frame
by frame, exactly the rings of the plain per-frame path, and a video frame
matches the oracle."""
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


@pytest.fixture(scope="module")
def video():
    return synth.video(6, seed=1103)


def test_batched_graph_equals_per_frame(torch, video):
    from paper_1310_1371_gb300 import rd
    params = synth.VIDEO_PARAMS
    t = torch.from_numpy(np.stack([f.image for f in video])).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    geo = rd.rd_autotune(params, t, stream)
    batched = rd.Detector(params, 1024, 1024, len(video))
    assert batched.geometry() == geo
    batched.set_graph(True)
    for _ in range(2):  # capture, then replay
        rb, sb = batched.detect(t, stream)
    plain = rd.Detector(params, 1024, 1024, 1)
    votes = 0
    for i in range(len(video)):
        rp, sp = plain.detect(t[i:i + 1], stream)
        votes += sp.votes
        assert len(rp[0]) == len(rb[i])
        for k in FIELDS:
            assert np.array_equal(rp[0][k], rb[i][k]), (i, k)
    assert votes == sb.votes
    assert sum(len(r) for r in rb) > 0
    batched.close()
    plain.close()


def test_video_frame_matches_oracle(torch, video):
    from paper_1310_1371_gb300 import rd
    f = video[2]
    p = O.Params.make(**synth.VIDEO_PARAMS)
    ref = O.detect(f.image, p)
    det = rd.Detector(synth.VIDEO_PARAMS, 1024, 1024, 1)
    rings, stats = det.detect(torch.from_numpy(f.image[None].copy()).cuda())
    det.close()
    got = rings[0]
    key = lambda r: list(zip(np.asarray(r["ix"]).tolist(), np.asarray(r["iy"]).tolist(), np.asarray(r["ir"]).tolist()))
    assert key(got) == key(ref.rings)
    assert stats.votes == ref.votes_in and stats.hotspots == ref.hotspots
    for a in ("cx", "cy", "r"):
        assert np.abs(np.asarray(got[a], np.float64) - ref.rings[a]).max() <= 0.01
