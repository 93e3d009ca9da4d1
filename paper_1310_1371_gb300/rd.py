"""ctypes binding of librd.so (the C ABI in include/rd.h).

The functions below carry the C names and only marshal arguments: every step
of the detector runs in the library's CUDA kernels.  PyTorch is used for
device memory and streams.  There is no CPU fallback: if the library is
missing or has no GPU, the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_float, c_int, c_int32, c_int64, c_uint32, c_void_p

import numpy as np

from . import _build

RD_U8, RD_U16, RD_F32 = 0, 1, 2
RD_OK, RD_E_INVAL, RD_E_NOMEM, RD_E_CUDA, RD_E_OVERFLOW, RD_E_TIMEOUT, RD_E_BUSY, RD_E_HOST = range(8)
STATUS_NAMES = ["RD_OK", "RD_E_INVAL", "RD_E_NOMEM", "RD_E_CUDA", "RD_E_OVERFLOW", "RD_E_TIMEOUT", "RD_E_BUSY",
                "RD_E_HOST"]
# rd_stats.overflow bits (capacities that overflowed)
RD_OVF_RIDGE, RD_OVF_BINS, RD_OVF_PEAKS, RD_OVF_RINGS, RD_OVF_SCORE, RD_OVF_CHECK = 1, 2, 4, 8, 16, 32
RD_RING_FIT_FAIL = 1
RD_SERVE_FAIL_RESULT, RD_SERVE_FAIL_SLOT = 1, 2
PEAK_CAP = 4096   # per-frame peak capacity of a context


class rd_params(ctypes.Structure):
    _fields_ = [("sigma", c_float), ("r_min", c_int), ("r_max", c_int), ("ridge_thresh", c_float),
                ("peak_frac", c_float), ("vote_thresh", c_int), ("annulus_w", c_float),
                ("sig_a", c_float), ("sig_b", c_float), ("coarse", c_int)]


class rd_ring(ctypes.Structure):
    _fields_ = [("frame", c_int), ("cx", c_float), ("cy", c_float), ("r", c_float), ("ix", c_int),
                ("iy", c_int), ("ir", c_int), ("score", c_float), ("n_fit", c_int), ("flags", c_int)]


class rd_geometry(ctypes.Structure):
    _fields_ = [("tile", c_int), ("slab_levels", c_int)]


class rd_stats(ctypes.Structure):
    _fields_ = [("ridge_pixels", c_int64), ("votes", c_int64), ("peaks", c_int64),
                ("exact_fallbacks", c_int64), ("overflow", c_int32), ("n_frames", c_int32),
                ("hotspots", c_int64), ("smooth_macs", c_int64)]


RING_NP = np.dtype([("frame", "<i4"), ("cx", "<f4"), ("cy", "<f4"), ("r", "<f4"), ("ix", "<i4"),
                    ("iy", "<i4"), ("ir", "<i4"), ("score", "<f4"), ("n_fit", "<i4"), ("flags", "<i4")])
assert RING_NP.itemsize == ctypes.sizeof(rd_ring) == 40

_lib = None


def load_library(build: bool = False) -> ctypes.CDLL:
    """Load librd.so from the package (building it first when asked).  With
    RD_LIB_VARIANT=check in the environment the bounds-checked debug build
    librd_check.so is loaded instead."""
    global _lib
    if _lib is not None:
        return _lib
    variant = os.environ.get("RD_LIB_VARIANT") or None
    path = _build.build(variant=variant) if build else _build.lib_path(variant)
    if not os.path.exists(path):
        raise RuntimeError(f"librd.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = POINTER
    sig = {
        "rd_create": (c_int, [P(rd_params), c_int, c_int, c_int, P(c_void_p)]),
        "rd_create_ex": (c_int, [P(rd_params), c_int, c_int, c_int, P(rd_geometry), P(c_void_p)]),
        "rd_get_geometry": (c_int, [c_void_p, P(rd_geometry)]),
        "rd_autotune": (c_int, [P(rd_params), c_void_p, c_int, c_int, c_int, c_int, c_void_p, P(rd_geometry)]),
        "rd_detect": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_int,
                              c_void_p, c_void_p]),
        "rd_detect_host": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_int,
                                   c_void_p, c_void_p]),
        "rd_get_stats": (c_int, [c_void_p, P(rd_stats)]),
        "rd_get_device_bytes": (c_int, [c_void_p, P(ctypes.c_longlong)]),
        "rd_destroy": (c_int, [c_void_p]),
        "rd_last_error": (ctypes.c_char_p, [c_void_p]),
        "rd_gaussian_taps": (c_int, [c_float, P(c_int32), c_int]),
        "rd_level_weights": (c_int, [c_float, c_float, c_int, P(c_int32), c_int]),
        "rd_peak_threshold": (c_int64, [c_float, c_int]),
        "rd_debug_ridges": (c_int, [c_void_p, c_int, P(c_int32), P(c_float), P(c_int64), c_int]),
        "rd_debug_capture": (c_int, [c_void_p, c_void_p, c_void_p]),
        "rd_set_timing": (c_int, [c_void_p, c_int]),
        "rd_set_graph": (c_int, [c_void_p, c_int]),
        "rd_set_features": (c_int, [c_void_p, c_int, c_float]),
        "rd_soft_score": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p]),
        "rd_backward": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p]),
        "rd_refine": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_int,
                              c_float]),
        "rd_debug_route": (c_int, [c_void_p, c_int]),
        "rd_get_timing": (c_int, [c_void_p, P(c_float), c_int]),
        "rd_ridges_static": (c_int, [P(rd_params), c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                     c_int, c_void_p]),
        "rd_static_last_error": (ctypes.c_char_p, []),
        "rd_serve_create": (c_int, [c_void_p, c_int, ctypes.c_longlong, c_int, P(c_void_p)]),
        "rd_serve_submit": (c_int, [c_void_p, c_int, c_void_p, ctypes.c_longlong]),
        "rd_serve_poll": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                                  c_int, c_int]),
        "rd_serve_stats": (c_int, [c_void_p, c_void_p]),
        "rd_serve_stats_ex": (c_int, [c_void_p, c_void_p, c_int]),
        "rd_serve_debug_inject": (c_int, [c_void_p, c_int, c_int]),
        "rd_serve_destroy": (c_int, [c_void_p]),
        "rd_serve_last_error": (ctypes.c_char_p, []),
        "rd_probe_smem_atomics": (c_int, [c_int, c_int, c_int, c_void_p, P(ctypes.c_double), P(c_float)]),
        "rd_probe_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def make_params(**kw) -> rd_params:
    return rd_params(float(kw["sigma"]), int(kw["r_min"]), int(kw["r_max"]), float(kw["ridge_thresh"]),
                     float(kw["peak_frac"]), int(kw["vote_thresh"]), float(kw.get("annulus_w", 2.0)),
                     float(kw.get("sig_a", 0.05)), float(kw.get("sig_b", 0.25)), int(kw.get("coarse", 1) or 1))


# ---- host-only helpers -----------------------------------------------------------
def rd_gaussian_taps(sigma: float) -> np.ndarray:
    lib = load_library()
    buf = (c_int32 * 64)()
    n = lib.rd_gaussian_taps(sigma, buf, 64)
    if n < 0:
        raise RdError(RD_E_INVAL, "rd_gaussian_taps")
    return np.frombuffer(buf, dtype=np.int32, count=n).copy()


def rd_level_weights(sig_a: float, sig_b: float, r: int) -> np.ndarray:
    lib = load_library()
    buf = (c_int32 * (81 * 81))()
    n = lib.rd_level_weights(sig_a, sig_b, r, buf, 81 * 81)
    if n < 0:
        raise RdError(RD_E_INVAL, "rd_level_weights")
    w = int(round(n ** 0.5))
    return np.frombuffer(buf, dtype=np.int32, count=n).copy().reshape(w, w)


def rd_peak_threshold(peak_frac: float, r: int) -> int:
    return int(load_library().rd_peak_threshold(peak_frac, r))


def rd_autotune(params: dict, frames, stream=None) -> tuple[int, int]:
    """rd_autotune on device frames [n, H, W]: the fastest (tile, slab_levels),
    also cached in the library for contexts created afterwards."""
    import torch
    lib = load_library()
    if not frames.is_cuda or not frames.is_contiguous():
        raise ValueError("frames must be a contiguous CUDA tensor")
    n, H, W = frames.shape
    s = stream if stream is not None else torch.cuda.current_stream()
    p = make_params(**params)
    g = rd_geometry()
    st = lib.rd_autotune(ctypes.byref(p), c_void_p(frames.data_ptr()), n, H, W, Detector.dtype_code(frames.dtype),
                         c_void_p(s.cuda_stream), ctypes.byref(g))
    if st != RD_OK:
        raise RdError(st, lib.rd_last_error(None).decode())
    return g.tile, g.slab_levels


PROBE_PATTERNS = {0: "conflict-free u32", 1: "packed u16 pairs", 2: "random (vote stream)"}


def rd_probe_smem_atomics(pattern: int, ctas_per_sm: int = 4, iters: int = 4096, stream=None) -> tuple[float, float]:
    """Measured shared-memory atomic adds per second of the current GPU for an
    address pattern (0 conflict-free, 1 packed-u16 pairs, 2 random), and the
    timed launch's milliseconds."""
    import torch
    lib = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    rate, ms = ctypes.c_double(), c_float()
    st = lib.rd_probe_smem_atomics(pattern, ctas_per_sm, iters, c_void_p(s.cuda_stream), ctypes.byref(rate),
                                   ctypes.byref(ms))
    if st != RD_OK:
        raise RdError(st, lib.rd_probe_last_error().decode())
    return rate.value, ms.value


RD_STATIC_MAX_PIXELS = 1 << 20
RD_STATIC_MAX_RIDGE = 1 << 18


def rd_ridges_static(params: dict, frame, xy, dirs, count, stream=None) -> None:
    """rd_ridges_static: directed ridge pixels of one device frame [H, W]
    (uint8 / uint16) into caller-owned device tensors xy (int32 [cap]), dirs
    (float32 [cap, 4]) and count (int32 [1]).  Allocates no device memory, for
    callers that cannot; scratch is a fixed array inside the library, shared
    by every call on the device, so calls must be ordered on one stream."""
    import torch
    lib = load_library()
    for t in (frame, xy, dirs, count):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("arguments must be contiguous CUDA tensors")
    if xy.dtype != torch.int32 or dirs.dtype != torch.float32 or count.dtype != torch.int32:
        raise TypeError("xy and count must be int32, dirs float32")
    cap = xy.numel()
    if dirs.numel() < 4 * cap or count.numel() < 1:
        raise ValueError("dirs needs 4 * cap floats and count one int")
    H, W = frame.shape
    s = stream if stream is not None else torch.cuda.current_stream()
    p = make_params(**params)
    st = lib.rd_ridges_static(ctypes.byref(p), c_void_p(frame.data_ptr()), H, W, Detector.dtype_code(frame.dtype),
                              c_void_p(s.cuda_stream), c_void_p(xy.data_ptr()), c_void_p(dirs.data_ptr()), cap,
                              c_void_p(count.data_ptr()))
    if st != RD_OK:
        raise RdError(st, lib.rd_static_last_error().decode())


# ---- the detector ------------------------------------------------------------------
class Detector:
    """One rd_ctx: method parameters, maximum frame size and batch."""

    def __init__(self, params: dict, max_H: int, max_W: int, max_batch: int = 1, geometry=None):
        """geometry: None (automatic) or (tile, slab_levels) for rd_create_ex."""
        import torch  # device memory and streams
        self.torch = torch
        self.lib = load_library()
        self.params = dict(params)
        self.max_H, self.max_W, self.max_batch = max_H, max_W, max_batch
        ctx = c_void_p()
        p = make_params(**params)
        geo = rd_geometry(*geometry) if geometry is not None else None
        st = self.lib.rd_create_ex(ctypes.byref(p), max_H, max_W, max_batch,
                                   ctypes.byref(geo) if geo is not None else None, ctypes.byref(ctx))
        if st != RD_OK:
            raise RdError(st, self.lib.rd_last_error(None).decode())
        self.ctx = ctx
        dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.ring_cap = max_batch * PEAK_CAP
        self.rings = torch.empty(self.ring_cap * 10, dtype=torch.int32, device=dev)
        self.counts = torch.empty(max_batch, dtype=torch.int32, device=dev)
        self.offsets = torch.empty(max_batch, dtype=torch.int32, device=dev)

    def device_bytes(self) -> int:
        """rd_get_device_bytes: device memory the context holds."""
        b = ctypes.c_longlong()
        st = self.lib.rd_get_device_bytes(self.ctx, ctypes.byref(b))
        if st != RD_OK:
            raise RdError(st, "rd_get_device_bytes")
        return int(b.value)

    def geometry(self) -> tuple[int, int]:
        g = rd_geometry()
        st = self.lib.rd_get_geometry(self.ctx, ctypes.byref(g))
        if st != RD_OK:
            raise self._err(st)
        return g.tile, g.slab_levels

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.rd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _err(self, st):
        return RdError(st, self.lib.rd_last_error(self.ctx).decode())

    @staticmethod
    def dtype_code(t) -> int:
        import torch
        if t == torch.uint8:
            return RD_U8
        if t == torch.uint16:
            return RD_U16
        if t == torch.float32:
            return RD_F32
        raise TypeError(f"unsupported frame dtype {t}")

    # ---- differentiable soft score (rd_soft_score, rd_backward, rd_refine) ----
    def _soft_args(self, frames, rings, counts):
        torch = self.torch
        for t in (frames, rings, counts):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("frames, rings and counts must be contiguous CUDA tensors")
        if rings.dtype != torch.float32 or rings.dim() != 2 or rings.shape[1] != 10:
            raise TypeError("rings must be a float32 [n_rings, 10] tensor of rd_ring records (see pack_rings)")
        if counts.dtype != torch.int32:
            raise TypeError("counts must be int32")
        n, H, W = frames.shape
        return n, H, W

    def soft_score(self, frames, rings, counts, with_grad=False, stream=None):
        """rd_soft_score: per-ring scores [n_rings] (and d/d(cx, cy, r) [n_rings, 3])."""
        torch = self.torch
        n, H, W = self._soft_args(frames, rings, counts)
        s = stream if stream is not None else torch.cuda.current_stream()
        score = torch.empty(rings.shape[0], dtype=torch.float32, device=frames.device)
        dp = torch.empty((rings.shape[0], 3), dtype=torch.float32, device=frames.device) if with_grad else None
        st = self.lib.rd_soft_score(self.ctx, c_void_p(frames.data_ptr()), n, H, W, self.dtype_code(frames.dtype),
                                    c_void_p(s.cuda_stream), c_void_p(rings.data_ptr()), c_void_p(counts.data_ptr()),
                                    c_void_p(score.data_ptr()), c_void_p(dp.data_ptr() if dp is not None else 0))
        if st != RD_OK:
            raise self._err(st)
        return score, dp

    def backward(self, frames, rings, counts, dscore, stream=None):
        """rd_backward: (dimage [n, H, W], dparams [n_rings, 3]) for upstream dscore [n_rings]."""
        torch = self.torch
        n, H, W = self._soft_args(frames, rings, counts)
        if frames.dtype != torch.float32 or dscore.dtype != torch.float32 or not dscore.is_contiguous():
            raise TypeError("rd_backward takes float32 frames and a contiguous float32 dscore")
        s = stream if stream is not None else torch.cuda.current_stream()
        dimage = torch.empty_like(frames)
        dp = torch.empty((rings.shape[0], 3), dtype=torch.float32, device=frames.device)
        st = self.lib.rd_backward(self.ctx, c_void_p(frames.data_ptr()), n, H, W, c_void_p(s.cuda_stream),
                                  c_void_p(rings.data_ptr()), c_void_p(counts.data_ptr()), c_void_p(dscore.data_ptr()),
                                  c_void_p(dimage.data_ptr()), c_void_p(dp.data_ptr()))
        if st != RD_OK:
            raise self._err(st)
        return dimage, dp

    def refine(self, frames, rings, counts, iters=10, step=0.5, stream=None):
        """rd_refine: gradient ascent on the soft score, updating rings in place."""
        torch = self.torch
        n, H, W = self._soft_args(frames, rings, counts)
        s = stream if stream is not None else torch.cuda.current_stream()
        st = self.lib.rd_refine(self.ctx, c_void_p(frames.data_ptr()), n, H, W, self.dtype_code(frames.dtype),
                                c_void_p(s.cuda_stream), c_void_p(rings.data_ptr()), c_void_p(counts.data_ptr()),
                                int(iters), float(step))
        if st != RD_OK:
            raise self._err(st)

    def detect_async(self, frames, stream=None):
        """Enqueue rd_detect on device frames [n, H, W] (uint8 / uint16)."""
        torch = self.torch
        if not frames.is_cuda or not frames.is_contiguous():
            raise ValueError("frames must be a contiguous CUDA tensor")
        n, H, W = frames.shape
        s = stream if stream is not None else torch.cuda.current_stream()
        st = self.lib.rd_detect(self.ctx, c_void_p(frames.data_ptr()), n, H, W, self.dtype_code(frames.dtype),
                                c_void_p(s.cuda_stream), c_void_p(self.rings.data_ptr()), self.ring_cap,
                                c_void_p(self.counts.data_ptr()), c_void_p(self.offsets.data_ptr()))
        if st != RD_OK:
            raise self._err(st)
        return n

    def stats(self) -> rd_stats:
        out = rd_stats()
        st = self.lib.rd_get_stats(self.ctx, ctypes.byref(out))
        if st not in (RD_OK, RD_E_OVERFLOW):
            raise self._err(st)
        return out

    def detect(self, frames, stream=None, check=True):
        """rd_detect + sync; returns (list of per-frame ring arrays, stats)."""
        n = self.detect_async(frames, stream)
        stats = self.stats()
        if check and stats.overflow:
            raise RdError(RD_E_OVERFLOW, f"capacity overflow mask {stats.overflow}")
        counts = self.counts[:n].cpu().numpy()
        offs = self.offsets[:n].cpu().numpy()
        total = int(min(counts.sum(), self.ring_cap))
        rings = self.rings[: total * 10].cpu().numpy().view(RING_NP)
        return [rings[o:o + c] for o, c in zip(offs, counts)], stats

    def detect_host(self, frames_host: np.ndarray, stream=None):
        """rd_detect_host: host frames in, host rings out (copies inside)."""
        torch = self.torch
        n, H, W = frames_host.shape
        code = RD_U8 if frames_host.dtype == np.uint8 else RD_U16
        if frames_host.dtype not in (np.uint8, np.uint16) or not frames_host.flags.c_contiguous:
            raise TypeError("frames must be a C-contiguous uint8/uint16 array")
        rings = np.empty(self.ring_cap, dtype=RING_NP)
        counts = np.empty(n, dtype=np.int32)
        offs = np.empty(n, dtype=np.int32)
        s = stream if stream is not None else torch.cuda.current_stream()
        st = self.lib.rd_detect_host(self.ctx, c_void_p(frames_host.ctypes.data), n, H, W, code,
                                     c_void_p(s.cuda_stream), c_void_p(rings.ctypes.data), self.ring_cap,
                                     c_void_p(counts.ctypes.data), c_void_p(offs.ctypes.data))
        if st not in (RD_OK, RD_E_OVERFLOW):
            raise self._err(st)
        return rings, counts, offs, st

    def set_features(self, features: str = "ridge", edge_thresh: float = 0.0):
        """rd_set_features: 'ridge' (the method) or 'edge' (directed edges)."""
        code = {"ridge": 0, "edge": 1}[features]
        st = self.lib.rd_set_features(self.ctx, code, float(edge_thresh))
        if st != RD_OK:
            raise self._err(st)

    def set_graph(self, on: bool):
        """rd_set_graph: capture rd_detect into a CUDA graph and replay it."""
        st = self.lib.rd_set_graph(self.ctx, 1 if on else 0)
        if st != RD_OK:
            raise self._err(st)

    def set_timing(self, on: bool):
        st = self.lib.rd_set_timing(self.ctx, 1 if on else 0)
        if st != RD_OK:
            raise self._err(st)

    def timing(self) -> np.ndarray:
        """Stage durations (ms) of the last call: stencil, refine, bins, vote, fit."""
        buf = (c_float * 8)()
        n = self.lib.rd_get_timing(self.ctx, buf, 8)
        if n < 0:
            raise self._err(RD_E_INVAL)
        return np.frombuffer(buf, dtype=np.float32, count=n).copy()

    def debug_ridges(self, f: int = 0):
        """Ridge pixels of frame f of the last call: xy [n, 2], dir [n, 2], hess [n, 3]."""
        n = self.lib.rd_debug_ridges(self.ctx, f, None, None, None, 0)
        if n < 0:
            raise self._err(RD_E_INVAL)
        xy = np.empty((n, 2), dtype=np.int32)
        d = np.empty((n, 2), dtype=np.float32)
        h = np.empty((n, 3), dtype=np.int64)
        m = self.lib.rd_debug_ridges(self.ctx, f, xy.ctypes.data_as(POINTER(c_int32)),
                                     d.ctypes.data_as(POINTER(c_float)), h.ctypes.data_as(POINTER(c_int64)), n)
        return xy, d, h

    def debug_route(self, all_dense: bool, bin_global: bool = False):
        st = self.lib.rd_debug_route(self.ctx, (1 if all_dense else 0) | (2 if bin_global else 0))
        if st != RD_OK:
            raise self._err(st)

    def debug_capture(self, acc=None, sm=None):
        st = self.lib.rd_debug_capture(self.ctx, c_void_p(acc.data_ptr() if acc is not None else 0),
                                       c_void_p(sm.data_ptr() if sm is not None else 0))
        if st != RD_OK:
            raise self._err(st)


# ---- rd_ring records as a float32 [n, 10] tensor and the autograd wrapper ------------
def pack_rings(params):
    """rd_ring records (float32 [n, 10] view) whose cx, cy, r are params [n, 3];
    the integer fields are left zero (the soft entry points read only cx, cy, r)."""
    import torch
    rec = torch.zeros((params.shape[0], 10), dtype=torch.float32, device=params.device)
    rec[:, 1:4] = params
    return rec


def _soft_function():
    import torch

    class SoftRingScore(torch.autograd.Function):
        """Score of each ring [n_rings] of a batch of float32 frames [n, H, W];
        differentiable with respect to the frames and to params [n_rings, 3]
        (cx, cy, r); counts [n] int32 assigns consecutive rings to frames.
        Forward: rd_soft_score; backward: rd_backward."""

        @staticmethod
        def forward(ctx, frames, params, det, counts):
            rings = pack_rings(params.detach())
            score, _ = det.soft_score(frames.detach().contiguous(), rings, counts)
            ctx.save_for_backward(frames, params, counts)
            ctx.det = det
            return score

        @staticmethod
        def backward(ctx, dscore):
            frames, params, counts = ctx.saved_tensors
            dimage, dparams = ctx.det.backward(frames.detach().contiguous(), pack_rings(params.detach()), counts,
                                               dscore.contiguous().to(torch.float32))
            return dimage, dparams, None, None

    return SoftRingScore


_SOFT = None


def soft_ring_score(det: "Detector", frames, params, counts):
    """Differentiable soft ring score (torch.autograd) through rd_soft_score /
    rd_backward; see SoftRingScore."""
    global _SOFT
    if _SOFT is None:
        _SOFT = _soft_function()
    return _SOFT.apply(frames, params, det, counts)


# ---- continuous-batching server (rd_serve_*) ----------------------------------------
class rd_serve_class(ctypes.Structure):
    _fields_ = [("params", rd_params), ("H", c_int), ("W", c_int), ("dtype", c_int), ("max_batch", c_int),
                ("slots", c_int)]


class Server:
    """rd_serve_*: continuous-batching request server.  classes: list of dicts
    with params, H, W, dtype ('u8'/'u16'), max_batch, slots."""

    def __init__(self, classes, mem_budget=0, queue_cap=4096):
        import torch  # noqa: F401  (the CUDA context of the current device)
        self.lib = load_library()
        arr = (rd_serve_class * len(classes))()
        self.frame_shapes = []
        for i, c in enumerate(classes):
            arr[i] = rd_serve_class(make_params(**c["params"]), int(c["H"]), int(c["W"]),
                                    RD_U8 if c.get("dtype", "u16") == "u8" else RD_U16, int(c["max_batch"]),
                                    int(c["slots"]))
            self.frame_shapes.append((int(c["H"]), int(c["W"]), np.uint8 if c.get("dtype", "u16") == "u8" else np.uint16))
        self.ptr = c_void_p()
        st = self.lib.rd_serve_create(arr, len(classes), int(mem_budget), int(queue_cap), ctypes.byref(self.ptr))
        if st != RD_OK:
            raise RdError(st, self.lib.rd_serve_last_error().decode())

    def submit(self, cls: int, frame: np.ndarray, request_id: int) -> int:
        """Queue one frame; returns the status (RD_OK or RD_E_BUSY), raises on bad arguments."""
        H, W, dt = self.frame_shapes[cls]
        if frame.shape != (H, W) or frame.dtype != dt or not frame.flags.c_contiguous:
            raise ValueError(f"class {cls} takes C-contiguous {H}x{W} {np.dtype(dt).name} frames")
        st = self.lib.rd_serve_submit(self.ptr, cls, c_void_p(frame.ctypes.data), int(request_id))
        if st not in (RD_OK, RD_E_BUSY):
            raise RdError(st, self.lib.rd_serve_last_error().decode())
        return st

    def poll(self, max_results=256, rings_cap=1 << 20, wait_ms=0):
        """Completed requests: list of (id, class, status, rings array, latency_us)."""
        ids = np.empty(max_results, np.int64)
        cls = np.empty(max_results, np.int32)
        sts = np.empty(max_results, np.int32)
        nr = np.empty(max_results, np.int32)
        lat = np.empty(max_results, np.float64)
        rings = np.empty(rings_cap, dtype=RING_NP)
        k = self.lib.rd_serve_poll(self.ptr, ids.ctypes.data, cls.ctypes.data, sts.ctypes.data, nr.ctypes.data,
                                   rings.ctypes.data, rings_cap, lat.ctypes.data, max_results, int(wait_ms))
        if k < 0:
            raise RdError(RD_E_INVAL, "rd_serve_poll")
        out, o = [], 0
        for i in range(k):
            out.append((int(ids[i]), int(cls[i]), int(sts[i]), rings[o:o + nr[i]].copy(), float(lat[i])))
            o += int(nr[i])
        return out

    STATS_EX = ("submitted", "completed", "batches", "device_bytes", "peak_device_bytes", "slots_made",
                "slots_destroyed", "memory_waits", "failed", "budget")

    def stats(self):
        buf = np.zeros(len(self.STATS_EX), np.int64)
        n = self.lib.rd_serve_stats_ex(self.ptr, buf.ctypes.data, len(buf))
        if n != len(buf):
            raise RdError(RD_E_INVAL, "rd_serve_stats_ex")
        return {k: int(v) for k, v in zip(self.STATS_EX, buf)}

    def inject(self, kind: str, count: int):
        """Make the next `count` host allocations of a kind fail ('result' or 'slot')."""
        code = {"result": RD_SERVE_FAIL_RESULT, "slot": RD_SERVE_FAIL_SLOT}[kind]
        st = self.lib.rd_serve_debug_inject(self.ptr, code, int(count))
        if st != RD_OK:
            raise RdError(st, "rd_serve_debug_inject")

    def close(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            self.lib.rd_serve_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
