"""Seeded synthetic microscope frames shaped like the paper's ring video.

This module only draws random ring geometry and renders intensity images.
It holds none of the detector's arithmetic, so both the GPU path and the
CPU oracle can be fed from it without sharing any of the method.

Workloads (sizes and distributions follow the paper's experiment: frames of
out-of-focus tracer images with tens to hundreds of rings, overlapping and
nested, the outermost ring thicker than the inner fringes; Results section,
"Robustness assessment" and "Performance assessment"):

* ``plain_small``  256x256 u8, 8 non-overlapping rings, r in [8, 30].
* ``plain_full``   1024x1024 u16 (12-bit), 150 overlapping rings, r in
  [10, 80], each with 2-3 inner fringes, Poisson shot + Gaussian read noise.
* ``video``        1024x1024 u8 frames; 20-300 rings per frame drawn from a
  pool of drifting tracks (centre step N(0, 1.5^2), radius step U[-0.3, 0.3]).
* ``diff_frames``  512x512 f32 frames, 64 rings, r in [10, 50], sub-pixel
  centres and radii, no rounding or clipping.
* ``requests``     a Poisson arrival stream of frames of mixed sizes.

Seeds: workload k uses ``numpy.random.default_rng(1000 + k)``; frame i of a
multi-frame workload uses ``default_rng([1000 + k, i])``.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Detector settings used with each workload (the method's parameters; the
# values are the ones the workloads were specified with).
PLAIN_SMALL_PARAMS = dict(sigma=2.0, r_min=5, r_max=40, ridge_thresh=-1.0,
                          peak_frac=0.35, vote_thresh=3, annulus_w=2.0,
                          sig_a=0.05, sig_b=0.25)
PLAIN_FULL_PARAMS = dict(sigma=2.0, r_min=8, r_max=96, ridge_thresh=-2.0,
                         peak_frac=0.35, vote_thresh=3, annulus_w=2.0,
                         sig_a=0.05, sig_b=0.25)
VIDEO_PARAMS = dict(PLAIN_SMALL_PARAMS)
DIFF_PARAMS = dict(sigma=2.0, r_min=8, r_max=56, ridge_thresh=-1.0,
                   peak_frac=0.35, vote_thresh=3, annulus_w=2.0,
                   sig_a=0.05, sig_b=0.25)


@dataclasses.dataclass
class Frame:
    image: np.ndarray          # [H, W], u8 / u16 / f32
    rings: np.ndarray          # [n, 3] float64: cx, cy, R  (x = column, y = row)
    params: dict


def _render(H, W, rings, profile, background):
    """Sum ring profiles (functions of rho - R) on a flat background.
    ``profile`` is one function for all rings or a list with one per ring."""
    img = np.full((H, W), float(background))
    profiles = profile if isinstance(profile, (list, tuple)) else [profile] * len(rings)
    for (cx, cy, R), profile in zip(rings, profiles):
        ext = R + 12.0
        x0, x1 = max(0, int(np.floor(cx - ext))), min(W, int(np.ceil(cx + ext)) + 1)
        y0, y1 = max(0, int(np.floor(cy - ext))), min(H, int(np.ceil(cy + ext)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        rho = np.hypot(xx - cx, yy - cy)
        img[y0:y1, x0:x1] += profile(rho, R)
    return img


def _gauss_ring(amp, width):
    return lambda rho, R: amp * np.exp(-0.5 * ((rho - R) / width) ** 2)


def _fringed_ring(amp, width, n_fringes):
    """Main Gaussian ring plus inner fringes: a non-negative cosine of period
    4 px in radius, halving per fringe (fringe k peaks at R - 4k)."""
    def prof(rho, R):
        main = amp * np.exp(-0.5 * ((rho - R) / width) ** 2)
        d = R - rho
        k = np.floor((d + 2.0) / 4.0)
        inside = (d > 2.0) & (d <= 4.0 * n_fringes + 1.0) & (k >= 1)
        fr = amp * np.power(0.5, np.maximum(k, 1)) * np.maximum(0.0, np.cos(2 * np.pi * d / 4.0))
        return main + np.where(inside, fr, 0.0)
    return prof


def _nonoverlap(rng, n, lo, hi, rlo, rhi, gap, tries=10000):
    out = []
    t = 0
    while len(out) < n:
        t += 1
        if t > tries:
            raise RuntimeError("could not place non-overlapping rings")
        c = rng.uniform(lo, hi, size=2)
        R = rng.uniform(rlo, rhi)
        if all(np.hypot(c[0] - q[0], c[1] - q[1]) > R + q[2] + gap for q in out):
            out.append((c[0], c[1], R))
    return np.array(out, dtype=np.float64)


def plain_small(seed: int = 1001, H: int = 256, W: int = 256, n_rings: int = 8) -> Frame:
    """One 256x256 u8 frame: 8 non-overlapping rings, centres in a 40 px
    inner margin, R ~ U[8, 30], cross-section sigma 1.5, amplitude 120 on a
    background of 40, additive N(0, 8^2) noise, rounded and clipped."""
    rng = np.random.default_rng(seed)
    rings = _nonoverlap(rng, n_rings, 40.0, min(H, W) - 40.0, 8.0, 30.0, 6.0)
    img = _render(H, W, rings, _gauss_ring(120.0, 1.5), 40.0)
    img += rng.normal(0.0, 8.0, size=img.shape)
    img = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    return Frame(img, rings, dict(PLAIN_SMALL_PARAMS))


def plain_full(seed=1002, H: int = 1024, W: int = 1024, n_rings: int = 150) -> Frame:
    """One 1024x1024 u16 frame with 12-bit values: 150 rings (overlaps
    allowed), R ~ U[10, 80], main ring amplitude 600 (sigma 1.5) plus 2-3
    inner fringes; background 400, Poisson shot noise and N(0, 10^2) read
    noise, rounded and clipped to [0, 4095]."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, W, size=n_rings)
    cy = rng.uniform(0.0, H, size=n_rings)
    R = rng.uniform(10.0, 80.0, size=n_rings)
    K = rng.integers(2, 4, size=n_rings)
    rings = np.stack([cx, cy, R], axis=1)
    img = _render(H, W, rings, [_fringed_ring(600.0, 1.5, int(k)) for k in K], 400.0)
    img = rng.poisson(img).astype(np.float64) + rng.normal(0.0, 10.0, size=img.shape)
    img = np.clip(np.rint(img), 0, 4095).astype(np.uint16)
    return Frame(img, rings, dict(PLAIN_FULL_PARAMS))


def plain_full_batch(n: int, seed0: int = 1002, **kw) -> list[Frame]:
    """n independent full-size frames; frame i is seeded with [seed0, i]."""
    return [plain_full(seed=[seed0, i], **kw) for i in range(n)]


def video_tracks(n_frames: int, seed: int = 1003, H: int = 1024, W: int = 1024,
                 pool: int = 300, n_min: int = 20, n_max: int = 300) -> list[np.ndarray]:
    """Ring geometry of each frame of ``video``: frame i shows the first
    n_i ~ U{n_min..n_max} tracks of a drifting pool, as [n_i, 3] (cx, cy, R)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(40.0, np.array([W - 40.0, H - 40.0]), size=(pool, 2))
    R = rng.uniform(8.0, 30.0, size=pool)
    tracks = []
    for i in range(n_frames):
        n = int(np.random.default_rng([seed, i]).integers(n_min, n_max + 1))
        tracks.append(np.concatenate([c[:n], R[:n, None]], axis=1))
        c = c + rng.normal(0.0, 1.5, size=c.shape)
        c[:, 0] = np.clip(c[:, 0], 0.0, W - 1.0)
        c[:, 1] = np.clip(c[:, 1], 0.0, H - 1.0)
        R = np.clip(R + rng.uniform(-0.3, 0.3, size=R.shape), 8.0, 30.0)
    return tracks


def video_frame(i: int, rings: np.ndarray, seed: int = 1003, H: int = 1024, W: int = 1024,
                n_min: int = 20, n_max: int = 300) -> np.ndarray:
    """Frame i of ``video`` (u8) from its ring geometry."""
    fr = np.random.default_rng([seed, i])
    fr.integers(n_min, n_max + 1)  # the ring count drawn by video_tracks
    img = _render(H, W, rings, _gauss_ring(120.0, 1.5), 40.0)
    img += fr.normal(0.0, 8.0, size=img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def video(n_frames: int, seed: int = 1003, H: int = 1024, W: int = 1024,
          pool: int = 300, n_min: int = 20, n_max: int = 300) -> list[Frame]:
    """A drifting-track video of u8 frames rendered like ``plain_small``.
    Frame i shows the first n_i ~ U{n_min..n_max} tracks of the pool."""
    tracks = video_tracks(n_frames, seed, H, W, pool, n_min, n_max)
    return [Frame(video_frame(i, rings, seed, H, W, n_min, n_max), rings.copy(), dict(VIDEO_PARAMS))
            for i, rings in enumerate(tracks)]


def _video_frame_job(args):
    return video_frame(*args)


def video_images(n_frames: int, seed: int = 1003, H: int = 1024, W: int = 1024, workers: int = 0) -> np.ndarray:
    """The frames of ``video`` as one [n, H, W] u8 array, rendered by a pool
    of ``workers`` processes started with 'spawn' (0: all cores)."""
    import multiprocessing as mp
    import os
    tracks = video_tracks(n_frames, seed, H, W)
    jobs = [(i, rings, seed, H, W) for i, rings in enumerate(tracks)]
    out = np.empty((n_frames, H, W), dtype=np.uint8)
    workers = workers or (os.cpu_count() or 1)
    if workers <= 1:
        for i, j in enumerate(jobs):
            out[i] = _video_frame_job(j)
        return out
    with mp.get_context("spawn").Pool(workers) as pool:
        for i, img in enumerate(pool.imap(_video_frame_job, jobs, chunksize=4)):
            out[i] = img
    return out


def diff_frame(i: int, seed: int = 1004, H: int = 512, W: int = 512, n_rings: int = 64) -> Frame:
    """Frame i of ``diff_frames``."""
    rng = np.random.default_rng([seed, i])
    cx = rng.uniform(40.0, W - 40.0, size=n_rings)
    cy = rng.uniform(40.0, H - 40.0, size=n_rings)
    R = rng.uniform(10.0, 50.0, size=n_rings)
    rings = np.stack([cx, cy, R], axis=1)
    img = _render(H, W, rings, _gauss_ring(120.0, 1.5), 40.0)
    img += rng.normal(0.0, 8.0, size=img.shape)
    return Frame(img.astype(np.float32), rings, dict(DIFF_PARAMS))


def diff_frames(n: int, seed: int = 1004, H: int = 512, W: int = 512, n_rings: int = 64) -> list[Frame]:
    """f32 frames with sub-pixel centres and radii, no rounding or clipping."""
    return [diff_frame(i, seed, H, W, n_rings) for i in range(n)]


def _diff_frame_job(args):
    f = diff_frame(*args)
    return f.image, f.rings


def diff_images(n: int, seed: int = 1004, H: int = 512, W: int = 512, n_rings: int = 64, workers: int = 0):
    """The frames of ``diff_frames`` as ([n, H, W] f32, [n, n_rings, 3] truth),
    rendered by a pool of ``workers`` processes started with 'spawn' (0: all cores)."""
    import multiprocessing as mp
    import os
    jobs = [(i, seed, H, W, n_rings) for i in range(n)]
    imgs = np.empty((n, H, W), dtype=np.float32)
    truth = np.empty((n, n_rings, 3))
    workers = workers or (os.cpu_count() or 1)
    if workers <= 1:
        for i, j in enumerate(jobs):
            imgs[i], truth[i] = _diff_frame_job(j)
        return imgs, truth
    with mp.get_context("spawn").Pool(workers) as pool:
        for i, (img, rings) in enumerate(pool.imap(_diff_frame_job, jobs, chunksize=4)):
            imgs[i] = img
            truth[i] = rings
    return imgs, truth


# Serving workload: frame sizes and the detector settings of each size class
# (radius search range scaled with the frame size).
SERVE_CLASSES = {
    256: dict(PLAIN_FULL_PARAMS, r_min=5, r_max=20),
    512: dict(PLAIN_FULL_PARAMS, r_min=5, r_max=40),
    1024: dict(PLAIN_FULL_PARAMS, r_min=8, r_max=96),
    2048: dict(PLAIN_FULL_PARAMS, r_min=8, r_max=160),
}


def serve_frame(size: int, i: int, seed: int = 1005) -> Frame:
    """Frame i of the serving size class ``size`` (u16, rendered like
    ``plain_full``): 10-400 rings, radii uniform inside the class's search
    range (2 px in from each end)."""
    p = SERVE_CLASSES[size]
    rng = np.random.default_rng([seed, size, i])
    n = int(rng.integers(10, 401))
    cx = rng.uniform(0.0, size, size=n)
    cy = rng.uniform(0.0, size, size=n)
    R = rng.uniform(p["r_min"] + 2.0, p["r_max"] - 2.0, size=n)
    K = rng.integers(2, 4, size=n)
    rings = np.stack([cx, cy, R], axis=1)
    img = _render(size, size, rings, [_fringed_ring(600.0, 1.5, int(k)) for k in K], 400.0)
    img = rng.poisson(img).astype(np.float64) + rng.normal(0.0, 10.0, size=img.shape)
    img = np.clip(np.rint(img), 0, 4095).astype(np.uint16)
    return Frame(img, rings, dict(p))


def _serve_frame_job(args):
    return serve_frame(*args).image


def serve_images(per_class: int, seed: int = 1005, sizes=(256, 512, 1024, 2048), workers: int = 0) -> dict:
    """``per_class`` frames of each serving size class, {size: [frames]},
    rendered by a pool of processes started with 'spawn' (0: all cores)."""
    import multiprocessing as mp
    import os
    jobs = [(s, i, seed) for s in sizes for i in range(per_class)]
    workers = workers or (os.cpu_count() or 1)
    if workers <= 1:
        imgs = [_serve_frame_job(j) for j in jobs]
    else:
        with mp.get_context("spawn").Pool(workers) as pool:
            imgs = pool.map(_serve_frame_job, jobs, chunksize=1)
    out = {s: [] for s in sizes}
    for (s, i, _), img in zip(jobs, imgs):
        out[s].append(img)
    return out


# Filled discs for the directed-edge variant (features whose edges, not
# ridges, describe them): a logistic edge of width 1.2 px.
DISC_SMALL_PARAMS = dict(PLAIN_SMALL_PARAMS, features="edge", edge_thresh=4.0)
DISC_FULL_PARAMS = dict(PLAIN_FULL_PARAMS, features="edge", edge_thresh=20.0)


def _disc(amp, width):
    return lambda rho, R: amp / (1.0 + np.exp(np.clip((rho - R) / width, -50.0, 50.0)))


def disc_small(seed: int = 3001, H: int = 256, W: int = 256, n_discs: int = 8) -> Frame:
    """u8 frame with non-overlapping filled discs (R ~ U[8, 30], amplitude 120
    on 40, edge width 1.2 px) and N(0, 8^2) noise."""
    rng = np.random.default_rng(seed)
    discs = _nonoverlap(rng, n_discs, 40.0, min(H, W) - 40.0, 8.0, 30.0, 6.0)
    img = _render(H, W, discs, _disc(120.0, 1.2), 40.0)
    img += rng.normal(0.0, 8.0, size=img.shape)
    return Frame(np.clip(np.rint(img), 0, 255).astype(np.uint8), discs, dict(DISC_SMALL_PARAMS))


def disc_full(seed: int = 3002, H: int = 1024, W: int = 1024, n_discs: int = 150) -> Frame:
    """12-bit u16 frame with 150 overlapping filled discs (R ~ U[10, 80],
    amplitude 600 on 400), Poisson shot noise and N(0, 10^2) read noise."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, W, size=n_discs)
    cy = rng.uniform(0.0, H, size=n_discs)
    R = rng.uniform(10.0, 80.0, size=n_discs)
    discs = np.stack([cx, cy, R], axis=1)
    img = _render(H, W, discs, _disc(600.0, 1.2), 400.0)
    img = rng.poisson(img).astype(np.float64) + rng.normal(0.0, 10.0, size=img.shape)
    return Frame(np.clip(np.rint(img), 0, 4095).astype(np.uint16), discs, dict(DISC_FULL_PARAMS))
