"""rd_ridges_static, the allocation-free entry point, against rd_detect.

rd_ridges_static keeps its scratch in a fixed device array inside the library
instead of allocating it, for callers that cannot allocate device memory at
the call site.  These tests call it through the C ABI twice in a row (the
second call on a smaller frame, with the array still holding the first call's
data) and compare each result with the ridge list rd_detect finds in the same
frame.  The file is named to run last, after every other test has used the
library on the same device; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

from paper_1310_1371_gb300 import synth

DIR_TOL = 1.2e-7   # the ridge-direction tolerance of the parity tests


@pytest.fixture(scope="module")
def rd():
    from paper_1310_1371_gb300 import rd as rd_mod
    rd_mod.load_library(build=True)
    return rd_mod


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def reference_ridges(rd, torch, img, params):
    """Ridge pixels and directions of rd_detect (context-allocated path)."""
    H, W = img.shape
    det = rd.Detector(params, H, W, 1)
    det.detect(torch.from_numpy(np.ascontiguousarray(img)[None]).cuda(), check=False)
    xy, d, _ = det.debug_ridges(0)
    det.close()
    return xy, d


def sort_by_position(x, y, *cols):
    o = np.lexsort((x, y))
    return (x[o], y[o]) + tuple(c[o] for c in cols)


def test_rejects_null_arguments(rd):
    lib = rd.load_library()
    p = rd.make_params(**synth.PLAIN_FULL_PARAMS)
    st = lib.rd_ridges_static(ctypes.byref(p), None, 64, 64, rd.RD_U16, None, None, None, 16, None)
    assert st == rd.RD_E_INVAL
    assert b"NULL" in lib.rd_static_last_error()


@pytest.mark.gpu
def test_two_calls_match_rd_detect(rd, torch):
    cases = [(synth.plain_full(seed=1002).image, synth.PLAIN_FULL_PARAMS),       # 1024 x 1024 u16: the maximum
             (synth.plain_small(seed=1001).image, synth.PLAIN_SMALL_PARAMS)]     # 256 x 256 u8
    cap = rd.RD_STATIC_MAX_RIDGE
    outs = []
    stream = torch.cuda.current_stream()
    for img, params in cases:   # two calls in a row on one stream, no sync between them
        frame = torch.from_numpy(np.ascontiguousarray(img)).cuda()
        xy = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        dirs = torch.full((cap, 4), float("nan"), dtype=torch.float32, device="cuda")
        count = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rd.rd_ridges_static(params, frame, xy, dirs, count, stream)
        outs.append((frame, xy, dirs, count))
    torch.cuda.synchronize()

    for (img, params), (_, xy, dirs, count) in zip(cases, outs):
        n = int(count.item())
        ref_xy, ref_d = reference_ridges(rd, torch, img, params)
        assert n == len(ref_xy) and 0 < n <= cap
        v = xy[:n].cpu().numpy().view(np.uint32)
        d = dirs[:n].cpu().numpy()
        gx, gy, gd = sort_by_position((v & 0xFFFF).astype(np.int64), (v >> 16).astype(np.int64), d)
        rx, ry, rdir = sort_by_position(ref_xy[:, 0].astype(np.int64), ref_xy[:, 1].astype(np.int64), ref_d)
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry), "ridge pixel sets differ"
        assert np.abs(gd[:, :2] - rdir).max() <= DIR_TOL
        # double-float directions: unit length, canonical sign
        X = gd[:, 0].astype(np.float64) + gd[:, 2]
        Y = gd[:, 1].astype(np.float64) + gd[:, 3]
        assert np.all(np.abs(np.hypot(X, Y) - 1.0) < 1e-6)
        assert np.all((X > 0) | ((X == 0) & (Y > 0)))


@pytest.mark.gpu
def test_overflow_keeps_true_count_and_first_records(rd, torch):
    """A capacity below the frame's ridge count: count_dev still holds the
    true count, the first cap records are valid ridge pixels of rd_detect's
    list (distinct, with its directions), and nothing is written past cap
    (the buffers extend 64 records beyond the capacity the call is given)."""
    cases = [(synth.plain_full(seed=1002).image, synth.PLAIN_FULL_PARAMS, 5000),
             (synth.plain_small(seed=1001).image, synth.PLAIN_SMALL_PARAMS, 300)]
    stream = torch.cuda.current_stream()
    for img, params, cap in cases:
        frame = torch.from_numpy(np.ascontiguousarray(img)).cuda()
        xy_all = torch.full((cap + 64,), -1, dtype=torch.int32, device="cuda")
        dirs_all = torch.full((cap + 64, 4), float("nan"), dtype=torch.float32, device="cuda")
        count = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rd.rd_ridges_static(params, frame, xy_all[:cap], dirs_all[:cap], count, stream)
        torch.cuda.synchronize()
        ref_xy, ref_d = reference_ridges(rd, torch, img, params)
        assert int(count.item()) == len(ref_xy) > cap
        v = xy_all[:cap].cpu().numpy().view(np.uint32)
        d = dirs_all[:cap].cpu().numpy()
        gx, gy = (v & 0xFFFF).astype(np.int64), (v >> 16).astype(np.int64)
        ref = {(int(x), int(y)): i for i, (x, y) in enumerate(ref_xy.tolist())}
        keys = list(zip(gx.tolist(), gy.tolist()))
        assert len(set(keys)) == cap, "records repeat"
        assert all(k in ref for k in keys), "a record is not a ridge pixel of rd_detect"
        idx = np.array([ref[k] for k in keys])
        assert np.abs(d[:, :2] - ref_d[idx]).max() <= DIR_TOL
        assert np.all(xy_all[cap:].cpu().numpy() == -1), "records written past cap"
        assert np.all(np.isnan(dirs_all[cap:].cpu().numpy())), "directions written past cap"


@pytest.mark.gpu
def test_rejects_sizes_beyond_the_limits(rd, torch):
    p = synth.PLAIN_FULL_PARAMS
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    big = torch.zeros((1024, 1025), dtype=torch.uint16, device="cuda")  # one column over 2^20 pixels
    xy = torch.zeros(16, dtype=torch.int32, device="cuda")
    dirs = torch.zeros((16, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(rd.RdError, match="RD_STATIC_MAX_PIXELS"):
        rd.rd_ridges_static(p, big, xy, dirs, count)
    frame = torch.zeros((64, 64), dtype=torch.uint16, device="cuda")
    xy = torch.zeros(rd.RD_STATIC_MAX_RIDGE + 1, dtype=torch.int32, device="cuda")
    dirs = torch.zeros((rd.RD_STATIC_MAX_RIDGE + 1, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(rd.RdError, match="RD_STATIC_MAX_RIDGE"):
        rd.rd_ridges_static(p, frame, xy, dirs, count)
    torch.cuda.synchronize()
    assert int(count.item()) == 0   # rejected calls enqueue nothing
