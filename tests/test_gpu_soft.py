"""Soft (differentiable) ring score on the GPU against the FP64 oracle
(oracle/soft.py): scores, parameter gradients and image gradients within
1e-4 relative; central finite differences (step 1e-3 px) of the GPU score;
the torch.autograd wrapper; gradient-ascent refinement."""
import numpy as np
import pytest

from oracle import soft as S
from paper_1310_1371_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = synth.DIFF_PARAMS
SP = S.SoftParams.make(**PARAMS)


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def case(n=2, H=96, W=112, n_rings=3, seed=2004, jitter=0.3):
    fr = synth.diff_frames(n, seed=seed, H=H, W=W, n_rings=n_rings)
    imgs = np.stack([f.image for f in fr]).astype(np.float32)
    rng = np.random.default_rng(seed)
    params = [(f.rings + rng.uniform(-jitter, jitter, f.rings.shape)).astype(np.float32) for f in fr]
    return imgs, params, fr


def gpu_inputs(torch, rd, imgs, params):
    frames = torch.from_numpy(imgs).cuda()
    counts = torch.tensor([len(p) for p in params], dtype=torch.int32, device="cuda")
    flat = torch.from_numpy(np.concatenate(params)).cuda()
    return frames, counts, flat, rd.pack_rings(flat)


def test_scores_and_gradients_match_oracle(torch):
    from paper_1310_1371_gb300 import rd
    imgs, params, _ = case()
    n, H, W = imgs.shape
    det = rd.Detector(PARAMS, H, W, n)
    frames, counts, flat, rings = gpu_inputs(torch, rd, imgs, params)
    sc, dp = det.soft_score(frames, rings, counts, with_grad=True)
    w = np.random.default_rng(7).uniform(0.5, 2.0, size=flat.shape[0]).astype(np.float32)
    dimg, dpw = det.backward(frames, rings, counts, torch.from_numpy(w).cuda())
    sc, dp, dimg, dpw = (t.cpu().numpy() for t in (sc, dp, dimg, dpw))
    o = 0
    for f in range(n):
        pr = params[f].astype(np.float64)
        k = len(pr)
        s1, _, g1, _ = S.soft_grads(imgs[f], pr, SP)
        sw, gimg, gw, _ = S.soft_grads(imgs[f], pr, SP, dscore=w[o:o + k].astype(np.float64))
        assert np.allclose(sc[o:o + k], s1, rtol=1e-5, atol=1e-6), (sc[o:o + k], s1)
        scale = np.abs(g1).max()
        assert np.abs(dp[o:o + k] - g1).max() <= 1e-4 * scale
        assert np.abs(dpw[o:o + k] - gw).max() <= 1e-4 * np.abs(gw).max()
        assert np.abs(dimg[f] - gimg).max() <= 1e-4 * np.abs(gimg).max()
        assert np.abs(gimg).max() > 0
        o += k
    det.close()


def test_full_size_frame_matches_oracle(torch):
    """The differentiable workload at full size: one 512 x 512 f32 frame with
    64 rings (jittered by up to 0.3 px).  All 64 rings go through the GPU
    calls, so the tile-visit cut-off and the FP64 atomics of many
    overlapping rings run at scale; the FP64 autograd oracle covers 16 of
    them (every fourth).  Scores and ring gradients are compared for those
    16, and the image gradient of a backward whose dscore is 0 for the other
    48 rings is compared with the oracle's image gradient of the 16."""
    from paper_1310_1371_gb300 import rd
    fr = synth.diff_frame(0)
    img = fr.image[None].astype(np.float32)
    rng = np.random.default_rng(4004)
    params = (fr.rings + rng.uniform(-0.3, 0.3, fr.rings.shape)).astype(np.float32)
    n_r = len(params)
    assert img.shape == (1, 512, 512) and n_r == 64
    sel = np.arange(0, n_r, 4)
    w = np.zeros(n_r, np.float32)
    w[sel] = rng.uniform(0.5, 2.0, len(sel)).astype(np.float32)
    det = rd.Detector(PARAMS, 512, 512, 1)
    frames, counts, flat, rings = gpu_inputs(torch, rd, img, [params])
    sc, dp = det.soft_score(frames, rings, counts, with_grad=True)
    dimg, _ = det.backward(frames, rings, counts, torch.from_numpy(w).cuda())
    sc, dp, dimg = (t.cpu().numpy() for t in (sc, dp, dimg))
    pr = params[sel].astype(np.float64)
    s1, _, g1, _ = S.soft_grads(img[0], pr, SP)
    _, gimg, _, _ = S.soft_grads(img[0], pr, SP, dscore=w[sel].astype(np.float64))
    assert np.allclose(sc[sel], s1, rtol=1e-5, atol=1e-6), np.abs(sc[sel] - s1).max()
    assert np.abs(dp[sel] - g1).max() <= 1e-4 * np.abs(g1).max()
    assert np.abs(dimg[0] - gimg).max() <= 1e-4 * np.abs(gimg).max()
    assert np.abs(gimg).max() > 0 and np.all(s1 > 1.0)
    det.close()


def kink_free(rd_o, cx, cy, rho, h=1e-3, gmin=1e-8):
    """No vote with a non-negligible Gaussian factor lies within h of a grid line."""
    sig = SP.sig_a * rho + SP.sig_b
    for s in (1.0, -1.0):
        vx = rd_o.xs + s * rho * rd_o.X
        vy = rd_o.ys + s * rho * rd_o.Y
        near = np.exp(-((vx - cx) ** 2 + (vy - cy) ** 2) / (2 * (sig + 2) ** 2)) > gmin
        fx = np.abs(vx[near] - np.round(vx[near]))
        fy = np.abs(vy[near] - np.round(vy[near]))
        if np.any(fx < 2 * h) or np.any(fy < 2 * h):
            return False
    return True


def test_central_differences_on_gpu(torch):
    from paper_1310_1371_gb300 import rd
    imgs, params, _ = case(n=1, seed=2005)
    n, H, W = imgs.shape
    det = rd.Detector(PARAMS, H, W, n)
    rd_o = S.ridges_float(imgs[0], SP)
    frames = torch.from_numpy(imgs).cuda()
    counts = torch.tensor([1], dtype=torch.int32, device="cuda")
    h = 1e-3
    checked_r = 0
    for p0 in params[0]:
        p0 = p0.astype(np.float64)
        for j in range(3):
            if j == 2:  # the radius moves the votes: avoid bilinear kinks
                tries = 0
                while not kink_free(rd_o, p0[0], p0[1], p0[2]) and tries < 50:
                    p0[2] += 0.0137
                    tries += 1
                if tries == 50:
                    continue
                checked_r += 1
            base = torch.tensor(p0[None], dtype=torch.float32, device="cuda")
            _, g = det.soft_score(frames, rd.pack_rings(base), counts, with_grad=True)
            pp, pm = p0.copy(), p0.copy()
            pp[j] += h
            pm[j] -= h
            # score difference in double from the float scores of the two points
            sp, _ = det.soft_score(frames, rd.pack_rings(torch.tensor(pp[None], dtype=torch.float32, device="cuda")), counts)
            sm, _ = det.soft_score(frames, rd.pack_rings(torch.tensor(pm[None], dtype=torch.float32, device="cuda")), counts)
            dh = float(np.float32(pp[j])) - float(np.float32(pm[j]))
            fd = (float(sp[0]) - float(sm[0])) / dh
            gg = float(g[0, j])
            # float32 scores: add their rounding (2 ulp of the score over the step)
            tol = 1e-4 * max(abs(gg), 1e-3) + 2 * 6e-8 * abs(float(sp[0])) / dh
            assert abs(fd - gg) <= tol, (j, fd, gg)
    assert checked_r >= 1
    det.close()


def test_autograd_function(torch):
    from paper_1310_1371_gb300 import rd
    imgs, params, _ = case(seed=2006)
    n, H, W = imgs.shape
    det = rd.Detector(PARAMS, H, W, n)
    frames, counts, flat, rings = gpu_inputs(torch, rd, imgs, params)
    w = torch.linspace(0.5, 1.5, flat.shape[0], device="cuda")
    fr = frames.clone().requires_grad_(True)
    pr = flat.clone().requires_grad_(True)
    score = rd.soft_ring_score(det, fr, pr, counts)
    (score * w).sum().backward()
    dimg, dp = det.backward(frames, rings, counts, w.contiguous())
    assert torch.equal(fr.grad, dimg) and torch.equal(pr.grad, dp)
    det.close()


def test_refine_moves_rings_toward_truth(torch):
    from paper_1310_1371_gb300 import rd
    imgs, params, fr = case(n=2, H=192, W=192, n_rings=4, seed=2007, jitter=0.45)
    n, H, W = imgs.shape
    det = rd.Detector(PARAMS, H, W, n)
    frames, counts, flat, rings = gpu_inputs(torch, rd, imgs, params)
    truth = np.concatenate([f.rings for f in fr])
    before = np.abs(flat.cpu().numpy() - truth)
    det.refine(frames, rings, counts, iters=25, step=0.5)
    after = np.abs(rings[:, 1:4].cpu().numpy() - truth)
    # keep rings whose soft score is well defined (inside the frame, not merged with a neighbour)
    inside = (truth[:, 0] - truth[:, 2] > 6) & (truth[:, 0] + truth[:, 2] < W - 7) & \
             (truth[:, 1] - truth[:, 2] > 6) & (truth[:, 1] + truth[:, 2] < H - 7)
    assert inside.sum() >= 2
    assert np.median(after[inside]) < 0.5 * np.median(before[inside])
    assert np.median(after[inside]) < 0.15
    det.close()
