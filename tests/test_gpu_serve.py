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
SIZES = (256, 512, 1024, 2048)
BATCH = {256: 4, 512: 3, 1024: 2, 2048: 1}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def frames():
    return {s: [synth.serve_frame(s, i, seed=2105).image for i in range(3)] for s in SIZES}


def test_2048_class_matches_oracle(torch):
    """The largest serving class (2048 x 2048 u16, search r 8-160) through the
    server: its rings equal the FP64 oracle's (identical integer peaks, fits
    within 0.01 px)."""
    from oracle import ringdet as O
    from paper_1310_1371_gb300 import rd
    f = synth.serve_frame(2048, 1)
    server = rd.Server(classes()[3:], queue_cap=8)
    assert server.submit(0, f.image, 7) == rd.RD_OK
    got = []
    deadline = time.time() + 60
    while not got and time.time() < deadline:
        got = server.poll(wait_ms=100)
    server.close()
    assert len(got) == 1 and got[0][0] == 7 and got[0][2] == rd.RD_OK
    rings = got[0][3]
    ref = O.detect(f.image, O.Params.make(**f.params)).rings
    assert len(ref) >= 10
    assert list(zip(rings["ix"], rings["iy"], rings["ir"])) == list(zip(ref["ix"], ref["iy"], ref["ir"]))
    for k in ("cx", "cy", "r"):
        assert np.abs(rings[k].astype(np.float64) - ref[k]).max() <= 0.01, k


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


def _sizes(torch, sizes, slots):
    """Device bytes of one slot of each class (a server with no budget makes one per class)."""
    from paper_1310_1371_gb300 import rd
    out = []
    for s in sizes:
        server = rd.Server([dict(params=synth.SERVE_CLASSES[s], H=s, W=s, dtype="u16", max_batch=BATCH[s],
                                 slots=slots)], queue_cap=8)
        out.append(server.stats()["device_bytes"])
        server.close()
    return out


def _drain(server, n, timeout=90):
    got = {}
    deadline = time.time() + timeout
    while len(got) < n and time.time() < deadline:
        for rid, c, st, rings, lat in server.poll(wait_ms=50):
            got[rid] = (c, st, rings)
    return got


def test_memory_budget_admits_as_memory_frees(torch, frames):
    """A budget that holds one 2048 x 2048 slot and one 256 x 256 slot, never
    two large ones: six large requests submitted at once run one batch at a
    time (the scheduler waits for memory instead of making a second large
    slot), small requests keep running beside them, the slots never hold more
    than the budget, and every result equals the frame detected alone."""
    from paper_1310_1371_gb300 import rd
    big, small = _sizes(torch, (2048, 256), 1)
    budget = big + small + (1 << 20)
    assert 2 * big > budget
    cl = [dict(params=synth.SERVE_CLASSES[s], H=s, W=s, dtype="u16", max_batch=BATCH[s], slots=2)
          for s in (2048, 256)]
    server = rd.Server(cl, mem_budget=budget, queue_cap=64)
    plan = [(0, i % 3) for i in range(6)] + [(1, i % 3) for i in range(10)]
    for i, (c, k) in enumerate(plan):
        assert server.submit(c, frames[(2048, 256)[c]][k], i) == rd.RD_OK
    got = _drain(server, len(plan))
    stats = server.stats()
    server.close()
    assert len(got) == len(plan)
    assert stats["peak_device_bytes"] <= budget and stats["budget"] == budget
    assert stats["memory_waits"] > 0
    ref = {}
    for i, (c, k) in enumerate(plan):
        s = (2048, 256)[c]
        if (c, k) not in ref:
            ref[(c, k)] = alone(torch, frames[s][k], synth.SERVE_CLASSES[s])
        cls, st, rings = got[i]
        assert cls == c and st == rd.RD_OK and len(rings) == len(ref[(c, k)]) > 0
        for f in FIELDS:
            assert np.array_equal(rings[f], ref[(c, k)][f]), (i, f)


def test_host_allocation_failures_fail_requests_not_the_server(torch, frames):
    """Host allocation failures injected on the completion path fail exactly
    the requests they hit (RD_E_NOMEM, no rings); a class whose slot was
    destroyed and cannot be made again fails its queued requests; the
    server keeps serving correct results afterwards."""
    from paper_1310_1371_gb300 import rd
    ref = alone(torch, frames[256][0], synth.SERVE_CLASSES[256])
    server = rd.Server(classes(slots=1)[:1], queue_cap=16)
    server.inject("result", 2)
    for i in range(5):
        assert server.submit(0, frames[256][0], i) == rd.RD_OK
    got = _drain(server, 5)
    sts = [got[i][1] for i in range(5)]
    assert sts.count(rd.RD_E_NOMEM) == 2 and sts.count(rd.RD_OK) == 3
    for i in range(5):
        if got[i][1] == rd.RD_OK:
            assert np.array_equal(got[i][2]["ix"], ref["ix"]) and np.array_equal(got[i][2]["cx"], ref["cx"])
        else:
            assert len(got[i][2]) == 0
    assert server.stats()["failed"] == 2
    server.close()

    # a slot of class B destroyed to make room for class A; B's slot cannot be made again
    a, b = _sizes(torch, (1024, 256), 1)
    budget = 2 * a + b - 1
    cl = [dict(params=synth.SERVE_CLASSES[s], H=s, W=s, dtype="u16", max_batch=BATCH[s], slots=2 if s == 1024 else 1)
          for s in (1024, 256)]
    server = rd.Server(cl, mem_budget=budget, queue_cap=16)
    for i in range(6):
        assert server.submit(0, frames[1024][i % 3], i) == rd.RD_OK
    assert len(_drain(server, 6)) == 6
    st = server.stats()
    if st["slots_destroyed"] == 0:
        server.close()
        pytest.skip("the scheduler never needed a second large slot")
    server.inject("slot", 4)
    assert server.submit(1, frames[256][0], 100) == rd.RD_OK
    got = _drain(server, 1)
    assert got[100][1] == rd.RD_E_NOMEM
    server.inject("slot", 0)
    assert server.submit(1, frames[256][0], 101) == rd.RD_OK
    got = _drain(server, 1)
    assert got[101][1] == rd.RD_OK and np.array_equal(got[101][2]["ix"], ref["ix"])
    assert server.stats()["peak_device_bytes"] <= budget
    server.close()
