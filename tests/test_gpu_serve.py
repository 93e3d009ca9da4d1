"""Continuous-batching server (rd_serve_*): every request's rings are the
ones rd_detect gives for that frame alone, whatever it was batched and
overlapped with; host-side faults (bad class, full queue, memory budget)
are reported without touching the data path."""
import time

import numpy as np
import pytest

from paper_1310_1371_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit", "flags")
SIZES = (256, 512, 1024)
BATCH = {256: 4, 512: 3, 1024: 2}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def frames():
    return {s: [synth.serve_frame(s, i, seed=2105).image for i in range(3)] for s in SIZES}


def classes(slots=2):
    return [dict(params=synth.SERVE_CLASSES[s], H=s, W=s, dtype="u16", max_batch=BATCH[s], slots=slots) for s in SIZES]


def alone(torch, frame, params):
    from paper_1310_1371_gb300 import rd
    det = rd.Detector(params, frame.shape[0], frame.shape[1], 1)
    rings, _ = det.detect(torch.from_numpy(frame[None].copy()).cuda())
    det.close()
    return rings[0]


def test_results_identical_alone_and_in_the_mix(torch, frames):
    from paper_1310_1371_gb300 import rd
    server = rd.Server(classes(), queue_cap=1024)
    rng = np.random.default_rng(5)
    plan = [(int(rng.integers(0, len(SIZES))), int(rng.integers(0, 3))) for _ in range(48)]
    for i, (c, k) in enumerate(plan):
        assert server.submit(c, frames[SIZES[c]][k], i) == rd.RD_OK
        if i % 8 == 7:
            time.sleep(0.003)  # bursts and gaps: batches of different sizes and mixes
    got = {}
    deadline = time.time() + 60
    while len(got) < len(plan) and time.time() < deadline:
        for rid, c, st, rings, lat in server.poll(wait_ms=50):
            assert st == rd.RD_OK and lat > 0
            got[rid] = (c, rings)
    assert len(got) == len(plan)
    stats = server.stats()
    assert stats["completed"] == len(plan) and stats["batches"] < len(plan)
    server.close()
    ref = {}
    for i, (c, k) in enumerate(plan):
        s = SIZES[c]
        if (c, k) not in ref:
            ref[(c, k)] = alone(torch, frames[s][k], synth.SERVE_CLASSES[s])
        r = ref[(c, k)]
        assert got[i][0] == c and len(got[i][1]) == len(r) > 0
        for f in FIELDS:
            assert np.array_equal(got[i][1][f], r[f]), (i, f)


def test_host_side_faults(torch, frames):
    from paper_1310_1371_gb300 import rd
    with pytest.raises(rd.RdError) as ei:
        rd.Server(classes(), mem_budget=1 << 20)
    assert ei.value.status == rd.RD_E_NOMEM
    server = rd.Server(classes(slots=1)[:1], queue_cap=1)
    import ctypes
    assert server.lib.rd_serve_submit(server.ptr, 5, ctypes.c_void_p(frames[256][0].ctypes.data), 0) == rd.RD_E_INVAL
    busy, ok = 0, 0
    for i in range(64):
        st = server.submit(0, frames[256][i % 3], i)
        ok += st == rd.RD_OK
        busy += st == rd.RD_E_BUSY
    assert busy > 0 and ok > 0
    n = 0
    deadline = time.time() + 30
    while n < ok and time.time() < deadline:
        n += len(server.poll(wait_ms=50))
    assert n == ok
    server.close()
