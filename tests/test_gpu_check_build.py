"""The bounds-checked debug build (librd_check.so, compiled with RD_CHECK).

compute-sanitizer is not available where these tests run, so the kernels
check their own data-dependent indices in a debug build: pixel lists of the
stencil stage, bin keys of the binning stage, vote slots and smoothing windows
of both voting kernels.  A failed check sets RD_OVF_CHECK and skips the
access, without trapping.  A child process loads the checked library
(RD_LIB_VARIANT=check) and runs the ridge method on small and full-size
frames through both voting routes, the coarse parameter space and the
directed-edge variant.  Every call must finish without RD_OVF_CHECK, with the
oracle's integer peaks.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np
import torch
from oracle import ringdet as O
from paper_1310_1371_gb300 import rd, synth

assert rd.load_library(build=True)._name.endswith("librd_check.so")
cases = [("small", synth.plain_small().image, synth.PLAIN_SMALL_PARAMS, None, False),
         ("small dense route", synth.plain_small().image, synth.PLAIN_SMALL_PARAMS, None, True),
         ("full", synth.plain_full().image, synth.PLAIN_FULL_PARAMS, None, False),
         ("coarse 2", synth.plain_small().image, dict(synth.PLAIN_SMALL_PARAMS, coarse=2), None, False),
         ("edges", synth.disc_small().image, synth.DISC_SMALL_PARAMS, "edge", False)]
for name, img, params, feat, dense in cases:
    det = rd.Detector(params, img.shape[0], img.shape[1], 1)
    if feat:
        det.set_features(feat, params["edge_thresh"])
    det.debug_route(dense)
    rings, stats = det.detect(torch.from_numpy(np.ascontiguousarray(img)[None]).cuda(), check=False)
    assert not (stats.overflow & rd.RD_OVF_CHECK), (name, stats.overflow)
    assert stats.overflow == 0, (name, stats.overflow)
    ref = O.detect(img, O.Params.make(**params)).rings
    got = rings[0]
    key = lambda r: list(zip(np.asarray(r["ix"]).tolist(), np.asarray(r["iy"]).tolist(), np.asarray(r["ir"]).tolist()))
    assert key(got) == key(ref) and len(ref) > 0, name
    det.close()
print("checked build ok")
"""


def test_checked_build_runs_clean_and_matches_oracle():
    env = dict(os.environ, RD_LIB_VARIANT="check", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    out = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                         timeout=1200)
    assert out.returncode == 0 and "checked build ok" in out.stdout, out.stdout[-3000:] + out.stderr[-3000:]
