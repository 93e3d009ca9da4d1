"""rd_detect_host (host frames in, host rings out, copies inside the call)
against rd_detect on device buffers and against the oracle; two host threads,
each with its own context and stream, calling at the same time."""
import threading

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


def host_rings(rings, counts, offs):
    return [rings[o:o + c] for o, c in zip(offs.tolist(), counts.tolist())]


def same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert len(x) == len(y)
        for k in FIELDS:
            assert np.array_equal(x[k], y[k]), k


def test_host_equals_device_and_oracle(torch):
    from paper_1310_1371_gb300 import rd
    frames = np.stack([synth.plain_small(seed=s).image for s in (81, 82, 83)])
    params = synth.PLAIN_SMALL_PARAMS
    det = rd.Detector(params, 256, 256, len(frames))
    dev, _ = det.detect(torch.from_numpy(frames).cuda())
    rings, counts, offs, st = det.detect_host(np.ascontiguousarray(frames))
    torch.cuda.synchronize()
    det.close()
    assert st == rd.RD_OK
    got = host_rings(rings, counts, offs)
    same(got, dev)
    ref = O.detect(frames[0], O.Params.make(**params))
    assert list(zip(got[0]["ix"], got[0]["iy"], got[0]["ir"])) == list(zip(ref.rings["ix"], ref.rings["iy"], ref.rings["ir"]))


def test_two_host_threads(torch):
    """Each thread owns a context and a stream; results match one caller alone."""
    from paper_1310_1371_gb300 import rd
    params = synth.PLAIN_SMALL_PARAMS
    batches = [np.stack([synth.plain_small(seed=100 * t + s).image for s in range(4)]) for t in range(2)]
    ref = []
    for b in batches:
        det = rd.Detector(params, 256, 256, 4)
        ref.append(det.detect(torch.from_numpy(b).cuda())[0])
        det.close()
    out = [None, None]
    errs = []

    def work(t):
        try:
            det = rd.Detector(params, 256, 256, 4)
            s = torch.cuda.Stream()
            res = []
            for _ in range(5):
                rings, counts, offs, st = det.detect_host(np.ascontiguousarray(batches[t]), stream=s)
                assert st == rd.RD_OK
                res.append(host_rings(rings, counts, offs))
            s.synchronize()
            det.close()
            out[t] = res
        except Exception as e:  # reported by the main thread
            errs.append(e)

    ths = [threading.Thread(target=work, args=(t,)) for t in range(2)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert not errs, errs
    for t in range(2):
        for res in out[t]:
            same(res, ref[t])
