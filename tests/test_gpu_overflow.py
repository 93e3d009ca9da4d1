"""Capacity overflow is reported, not hidden (host-side injection, no GPU
fault): a caller's ring buffer smaller than the rings found raises
RD_OVF_RINGS and RD_E_OVERFLOW, keeps the true per-frame counts, fills the
buffer with the first rings of the full result, and leaves the context
usable (the next call with room is clean)."""
import ctypes

import numpy as np
import pytest

from paper_1310_1371_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_ring_buffer_overflow(torch):
    from paper_1310_1371_gb300 import rd
    frames = torch.from_numpy(np.stack([synth.plain_small(seed=s).image for s in (91, 92)])).cuda()
    det = rd.Detector(synth.PLAIN_SMALL_PARAMS, 256, 256, max_batch=2)
    full, stats = det.detect(frames)
    counts = [len(r) for r in full]
    assert stats.overflow == 0 and counts[0] > 5
    cap = 5
    rings = torch.zeros(cap * 10, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    off = torch.zeros(2, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    st = det.lib.rd_detect(det.ctx, ctypes.c_void_p(frames.data_ptr()), 2, 256, 256, rd.RD_U8,
                           ctypes.c_void_p(s.cuda_stream), ctypes.c_void_p(rings.data_ptr()), cap,
                           ctypes.c_void_p(cnt.data_ptr()), ctypes.c_void_p(off.data_ptr()))
    assert st == rd.RD_OK                                   # enqueued; the overflow shows in the stats
    out = rd.rd_stats()
    assert det.lib.rd_get_stats(det.ctx, ctypes.byref(out)) == rd.RD_E_OVERFLOW
    assert out.overflow == rd.RD_OVF_RINGS
    assert cnt.cpu().tolist() == counts and off.cpu().tolist() == [0, counts[0]]
    got = rings.cpu().numpy().view(rd.RING_NP)
    for k in ("ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit", "flags"):
        assert np.array_equal(got[k], full[0][:cap][k]), k
    # the context stays usable: the next call with room reports no overflow
    again, stats2 = det.detect(frames)
    assert stats2.overflow == 0 and [len(r) for r in again] == counts
    det.close()
