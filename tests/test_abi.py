"""The C ABI library builds, loads and exports every declared symbol; its
host-side weight tables equal the oracle's (CPU only, no GPU work)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import ringdet as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1310_1371_gb300 import rd
    return rd.load_library(build=True)


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(rd_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "rd_create" in names and "rd_detect" in names and "rd_detect_host" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("sigma", [0.7, 1.0, 1.5, 2.0, 2.5, 3.0, 3.3, 4.0])
def test_gaussian_taps_match_oracle(lib, sigma):
    from paper_1310_1371_gb300 import rd
    s32 = float(np.float32(sigma))
    assert np.array_equal(rd.rd_gaussian_taps(s32), O.gaussian_taps(s32))


@pytest.mark.parametrize("sig_a,sig_b", [(0.05, 0.25), (0.1, 0.5), (0.0, 1.0), (0.07, 0.13)])
def test_level_weights_match_oracle(lib, sig_a, sig_b):
    from paper_1310_1371_gb300 import rd
    a, b = float(np.float32(sig_a)), float(np.float32(sig_b))
    for r in range(1, 162):
        if np.ceil(3 * (a * r + b)) > 40:
            break
        assert np.array_equal(rd.rd_level_weights(a, b, r), O.smoothing_weights(r, a, b)), r


@pytest.mark.parametrize("frac", [0.0, 0.2, 0.35, 0.5, 0.91])
def test_peak_threshold_matches_oracle(lib, frac):
    from paper_1310_1371_gb300 import rd
    f = float(np.float32(frac))
    for r in range(1, 251):
        thr = O.peak_threshold(f, r)
        n = rd.rd_peak_threshold(f, r)
        # smallest integer N with N > thr
        assert n > thr and n - 1 <= thr, (r, n, thr)


def test_create_rejects_bad_params(lib):
    from paper_1310_1371_gb300 import rd
    good = dict(sigma=2.0, r_min=5, r_max=40, ridge_thresh=-1.0, peak_frac=0.35, vote_thresh=3)
    bad = [dict(good, sigma=0.0), dict(good, sigma=5.0), dict(good, r_min=1), dict(good, r_max=4),
           dict(good, ridge_thresh=0.5), dict(good, peak_frac=-1.0), dict(good, vote_thresh=-1),
           dict(good, r_max=600), dict(good, coarse=3), dict(good, coarse=8), dict(good, coarse=-2),
           dict(good, sigma=float("nan")), dict(good, sigma=float("inf")), dict(good, ridge_thresh=float("nan")),
           dict(good, peak_frac=float("inf")), dict(good, peak_frac=float("nan")), dict(good, annulus_w=float("nan")),
           dict(good, annulus_w=65.0), dict(good, sig_a=float("nan")), dict(good, sig_b=float("inf")),
           dict(good, sig_a=0.0, sig_b=-0.5), dict(good, sig_a=-0.01), dict(good, sig_a=2.0),
           dict(good, vote_thresh=65535), dict(good, coarse=4, vote_thresh=4096)]
    for kw in bad:
        p = rd.make_params(**kw)
        ctx = ctypes.c_void_p()
        st = lib.rd_create(ctypes.byref(p), 256, 256, 1, ctypes.byref(ctx))
        assert st == rd.RD_E_INVAL, kw
        assert ctx.value is None
        assert lib.rd_last_error(None)
    p = rd.make_params(**good)
    ctx = ctypes.c_void_p()
    assert lib.rd_create(ctypes.byref(p), 8, 256, 1, ctypes.byref(ctx)) == rd.RD_E_INVAL
    assert lib.rd_create(ctypes.byref(p), 256, 256, 0, ctypes.byref(ctx)) == rd.RD_E_INVAL


def test_null_context_calls_fail_cleanly(lib):
    from paper_1310_1371_gb300 import rd
    assert lib.rd_destroy(None) == rd.RD_E_INVAL
    assert lib.rd_detect(None, None, 1, 64, 64, 0, None, None, 0, None, None) == rd.RD_E_INVAL
    st = rd.rd_stats()
    assert lib.rd_get_stats(None, ctypes.byref(st)) == rd.RD_E_INVAL
    assert lib.rd_debug_ridges(None, 0, None, None, None, 0) == -1
    assert lib.rd_detect_host(None, None, 1, 64, 64, 0, None, None, 0, None, None) == rd.RD_E_INVAL
    assert lib.rd_set_graph(None, 1) == rd.RD_E_INVAL
    assert lib.rd_set_timing(None, 1) == rd.RD_E_INVAL
    assert lib.rd_set_features(None, 1, 1.0) == rd.RD_E_INVAL
    assert lib.rd_debug_route(None, 1) == rd.RD_E_INVAL
    assert lib.rd_debug_capture(None, None, None) == rd.RD_E_INVAL
    g = rd.rd_geometry()
    assert lib.rd_get_geometry(None, ctypes.byref(g)) == rd.RD_E_INVAL
    assert lib.rd_soft_score(None, None, 1, 64, 64, 0, None, None, None, None, None) == rd.RD_E_INVAL
    assert lib.rd_backward(None, None, 1, 64, 64, None, None, None, None, None, None) == rd.RD_E_INVAL
    assert lib.rd_refine(None, None, 1, 64, 64, 0, None, None, None, 1, 0.1) == rd.RD_E_INVAL
    ids = (ctypes.c_longlong * 4)()
    assert lib.rd_serve_submit(None, 0, None, 1) == rd.RD_E_INVAL
    assert lib.rd_serve_poll(None, ids, None, None, None, None, 0, None, 4, 0) == -1
    assert lib.rd_serve_stats(None, ids) == rd.RD_E_INVAL
    assert lib.rd_serve_destroy(None) == rd.RD_E_INVAL


@pytest.mark.parametrize("geo", [(72, 12), (96, 3), (96, 65), (0, 8), (64, 0)])
def test_bad_geometry_rejected(lib, geo):
    """rd_create_ex validates the accumulator geometry before touching the GPU."""
    from paper_1310_1371_gb300 import rd, synth
    p = rd.make_params(**synth.PLAIN_SMALL_PARAMS)
    g = rd.rd_geometry(*geo)
    ctx = ctypes.c_void_p()
    st = lib.rd_create_ex(ctypes.byref(p), 256, 256, 1, ctypes.byref(g), ctypes.byref(ctx))
    assert st == rd.RD_E_INVAL and not ctx.value
    assert b"geometry" in lib.rd_last_error(None)


def test_serve_create_validates_classes(lib):
    """rd_serve_create rejects bad class descriptions before touching the GPU."""
    from paper_1310_1371_gb300 import rd, synth
    good = rd.rd_serve_class(rd.make_params(**synth.PLAIN_SMALL_PARAMS), 256, 256, rd.RD_U8, 4, 1)
    for bad in (dict(slots=0), dict(slots=17), dict(max_batch=0), dict(max_batch=65536), dict(max_batch=1 << 30),
                dict(dtype=7)):
        c = rd.rd_serve_class(good.params, good.H, good.W, bad.get("dtype", good.dtype),
                              bad.get("max_batch", good.max_batch), bad.get("slots", good.slots))
        arr = (rd.rd_serve_class * 1)(c)
        out = ctypes.c_void_p()
        assert lib.rd_serve_create(arr, 1, 0, 16, ctypes.byref(out)) == rd.RD_E_INVAL and not out.value
    arr = (rd.rd_serve_class * 1)(good)
    out = ctypes.c_void_p()
    assert lib.rd_serve_create(arr, 0, 0, 16, ctypes.byref(out)) == rd.RD_E_INVAL
    assert lib.rd_serve_create(arr, 1, 0, 0, ctypes.byref(out)) == rd.RD_E_INVAL


def test_autotune_and_timing_reject_bad_sizes(lib):
    """rd_autotune bounds its batch before allocating; rd_get_timing rejects a
    negative capacity (both without GPU work)."""
    from paper_1310_1371_gb300 import rd, synth
    p = rd.make_params(**synth.PLAIN_SMALL_PARAMS)
    g = rd.rd_geometry()
    dummy = ctypes.c_void_p(16)                     # never dereferenced: the batch is checked first
    for n in (0, -1, 65536, 1 << 30):
        assert lib.rd_autotune(ctypes.byref(p), dummy, n, 256, 256, 0, None, ctypes.byref(g)) == rd.RD_E_INVAL
        assert b"rd_autotune" in lib.rd_last_error(None)
    ms = (ctypes.c_float * 8)()
    assert lib.rd_get_timing(None, ms, 8) == -1


def test_valid_create_without_a_device_releases_everything(lib):
    """With valid arguments and no CUDA device, rd_create and rd_serve_create
    stop at the device query: RD_E_CUDA, no handle, and the partly built
    context or server is released by its scope guard (the process stays
    usable for the next call)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: this checks the path without one")
    from paper_1310_1371_gb300 import rd, synth
    p = rd.make_params(**synth.PLAIN_SMALL_PARAMS)
    for _ in range(3):
        ctx = ctypes.c_void_p()
        assert lib.rd_create(ctypes.byref(p), 256, 256, 2, ctypes.byref(ctx)) == rd.RD_E_CUDA
        assert ctx.value is None and b"CUDA device" in lib.rd_last_error(None)
        arr = (rd.rd_serve_class * 1)(rd.rd_serve_class(p, 256, 256, rd.RD_U8, 4, 2))
        out = ctypes.c_void_p()
        assert lib.rd_serve_create(arr, 1, 0, 16, ctypes.byref(out)) == rd.RD_E_CUDA
        assert out.value is None and b"CUDA device" in lib.rd_serve_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without librd.so the binding raises: there is no fallback path."""
    from paper_1310_1371_gb300 import rd, _build
    monkeypatch.setattr(rd, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing" / "librd.so"))
    with pytest.raises(RuntimeError, match="not built"):
        rd.load_library()
    with pytest.raises(RuntimeError, match="not built"):
        rd.Detector({"sigma": 2.0, "r_min": 5, "r_max": 20, "ridge_thresh": -1.0}, 64, 64)


def test_static_entry_validates_before_device_work(lib):
    """rd_ridges_static rejects bad arguments with RD_E_INVAL and a message,
    before it touches a device (pointers below are never dereferenced)."""
    from paper_1310_1371_gb300 import rd, synth
    good = rd.make_params(**synth.PLAIN_SMALL_PARAMS)
    p16 = ctypes.c_void_p(16)                       # 16-byte aligned, never read
    cases = [
        (good, None, 256, 256, rd.RD_U8, p16, p16, 1024, p16, b"NULL"),
        (good, p16, 256, 256, rd.RD_U8, None, p16, 1024, p16, b"NULL"),
        (good, p16, 256, 256, 7, p16, p16, 1024, p16, b"dtype"),
        (good, p16, 8, 256, rd.RD_U8, p16, p16, 1024, p16, b"frame size"),
        (good, p16, 2048, 2048, rd.RD_U8, p16, p16, 1024, p16, b"pixels"),
        (good, p16, 256, 256, rd.RD_U8, p16, p16, -1, p16, b"cap"),
        (good, p16, 256, 256, rd.RD_U8, p16, p16, 1 << 20, p16, b"cap"),
        (good, p16, 256, 256, rd.RD_U8, p16, ctypes.c_void_p(20), 1024, p16, b"dir_dev must be 16-byte aligned"),
        (good, p16, 256, 256, rd.RD_U8, ctypes.c_void_p(18), p16, 1024, p16, b"xy_dev must be 4-byte aligned"),
        (good, p16, 256, 256, rd.RD_U8, p16, p16, 1024, ctypes.c_void_p(17), b"count_dev must be 4-byte aligned"),
        (good, ctypes.c_void_p(17), 256, 256, rd.RD_U16, p16, p16, 1024, p16, b"frame_dev must be 2-byte aligned"),
        (rd.make_params(**dict(synth.PLAIN_SMALL_PARAMS, sigma=0.0)), p16, 256, 256, rd.RD_U8, p16, p16, 1024, p16,
         b"sigma"),
        (rd.make_params(**dict(synth.PLAIN_SMALL_PARAMS, ridge_thresh=1.0)), p16, 256, 256, rd.RD_U8, p16, p16, 1024,
         p16, b"ridge_thresh"),
    ]
    for prm, frame, H, W, dt, xy, d, cap, cnt, msg in cases:
        st = lib.rd_ridges_static(ctypes.byref(prm), frame, H, W, dt, None, xy, d, cap, cnt)
        assert st == rd.RD_E_INVAL, msg
        assert msg in lib.rd_static_last_error(), (msg, lib.rd_static_last_error())


def test_status_codes_match_header():
    """The binding's status names are the header's rd_status enumerators, in order."""
    from paper_1310_1371_gb300 import rd
    txt = open(os.path.join(ROOT, "include", "rd.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} rd_status;", txt, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    pairs = re.findall(r"(RD_[A-Z_]+)\s*=\s*(\d+)", body)
    assert [n for n, _ in pairs] == rd.STATUS_NAMES
    assert [int(v) for _, v in pairs] == list(range(len(pairs)))
    assert all(getattr(rd, n) == i for i, n in enumerate(rd.STATUS_NAMES))
    ovf = dict((n, int(v)) for n, v in re.findall(r"#define (RD_OVF_[A-Z]+)\s+(\d+)", txt))
    assert ovf and all(getattr(rd, n) == v for n, v in ovf.items()), ovf


_STRUCTS = ("rd_params", "rd_ring", "rd_stats", "rd_geometry", "rd_serve_class")

_C_CALLER = r"""
#include <stddef.h>
#include <stdio.h>
#include "rd.h"
#define OFF(T, f) printf(#T " " #f " %d\n", (int)offsetof(T, f))
#define SIZE(T) printf(#T " sizeof %d\n", (int)sizeof(T))
int main(void) {
    int32_t taps[64];
    int i, n = rd_gaussian_taps(2.0f, taps, 64);
    rd_params p = {0};
    rd_ctx* ctx = NULL;
    rd_status st;
    printf("taps");
    for (i = 0; i < n; ++i) printf(" %d", (int)taps[i]);
    printf("\n");
    st = rd_create(&p, 64, 64, 1, &ctx);          /* sigma = 0: rejected before any device work */
    printf("create %d %d\n", (int)st, ctx == NULL);
@LAYOUT@
    return 0;
}
"""


def test_plain_c_caller(lib, tmp_path):
    """The header is plain C99 (no C++ in the declarations) and a C program
    links against the library; every struct the binding marshals has, in C,
    the binding's size and the binding's offset for each of its fields."""
    import shutil
    import subprocess
    from paper_1310_1371_gb300 import rd
    from paper_1310_1371_gb300 import _build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    layout = []
    for name in _STRUCTS:
        layout.append(f"    SIZE({name});")
        layout += [f"    OFF({name}, {f[0]});" for f in getattr(rd, name)._fields_]
    src = tmp_path / "caller.c"
    src.write_text(_C_CALLER.replace("@LAYOUT@", "\n".join(layout)))
    exe = tmp_path / "caller"
    libdir = os.path.dirname(_build.LIB)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-lrd", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    taps = [int(v) for v in out[0].split()[1:]]
    assert taps == O.gaussian_taps(2.0).tolist()
    assert out[1] == "create 1 1"                                     # RD_E_INVAL, no context
    seen = 0
    for line in out[2:]:
        name, field, value = line.split()
        cls = getattr(rd, name)
        want = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert int(value) == want, (name, field)
        seen += 1
    assert seen == sum(1 + len(getattr(rd, n)._fields_) for n in _STRUCTS)
