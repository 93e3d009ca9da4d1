#!/usr/bin/env python3
"""Throughput of the ring detector on one or more GPUs (one process per GPU).

Workload: batches of synthetic 1024x1024 uint16 microscope frames (12-bit,
150 overlapping rings with inner fringes, Poisson + read noise), detector
radius range 8-96 px, sigma 2.  One step = one rd_detect call over a batch of
B distinct frames resident in HBM (B = 96: 192 MiB of input, larger than L2,
so no flush is needed between steps).  Multi-GPU runs are independent
replicas (each rank its own frames; no data exchange).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload.  --workload video|diff|serve|discs|coarse
measures the batched path, the soft score, the server, directed edges and the
coarse parameter space on their own synthetic workloads.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s at 1024x1024 u16, r 8-96 (ridge-directed ring detection)"
WORKLOAD = "plain_full: 1024x1024 u16 frames, 150 rings r 10-80 with fringes, search r 8-96, sigma 2"
H = W = 1024
KERNELS_PER_CALL = 14   # stencil, refine, bin count, per-CTA bin scan, 3 scan, bin fill, queue, vote, vote (dense fallback), sort, offsets, fit
STAGES = ["stencil_ridge", "ridge_refine", "vote_bin", "vote_accumulate_peaks", "sort_fit"]


from paper_1310_1371_gb300.replicas import env_rank, frame_seeds, job_rate, max_over_ranks  # noqa: E402


def _one_frame(seed):
    from paper_1310_1371_gb300 import synth
    return synth.plain_full(seed=seed).image


def make_frames(n, rank):
    """n distinct seeded frames (seeds [1002 + 1000 rank, i]), rendered in a
    spawn-started process pool before any CUDA call."""
    import concurrent.futures as cf
    import multiprocessing as mp
    seeds = frame_seeds(rank, n)
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_one_frame, seeds))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = os.path.join(tempfile.gettempdir(), f"rd_clocks_{os.getpid()}.csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(gpu_index)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


# ------------------------------------------------------------------ CPU oracle
def _oracle_frame(job):
    """One frame through the FP64 oracle (a pool worker): its in-image votes."""
    from oracle import ringdet as O
    img, params = job
    return O.detect(img, O.Params.make(**params)).votes_in


def oracle_workers():
    return max(1, min(16, os.cpu_count() or 1))


def oracle_pool_run(frames, params, n_jobs, workers):
    """n_jobs frames (cycling over `frames`) through the oracle on a pool of
    `workers` spawn-started processes, frame-parallel as the paper's own CPU
    baseline ran; returns (frames/s, Mvotes/s, seconds)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_frame, [(frames[0], params)] * workers))  # start the workers, import numpy
        t0 = time.perf_counter()
        votes = sum(ex.map(_oracle_frame, [(frames[k % len(frames)], params) for k in range(n_jobs)]))
        dt = time.perf_counter() - t0
    return n_jobs / dt, votes / dt / 1e6, dt


def oracle_rate(frames, params, budget_s):
    """Frames/s and Mvotes/s of the FP64 oracle on a bounded sample: whole
    rounds of one frame per worker process (so that no worker idles), as
    many as fit in about budget_s seconds of wall time, at least two."""
    workers = oracle_workers()
    one = time.perf_counter()
    _oracle_frame((frames[0], params))
    per_frame = time.perf_counter() - one
    rounds = max(2, min(20, round(budget_s / max(per_frame, 1e-3))))
    fps, mv, dt = oracle_pool_run(frames, params, rounds * workers, workers)
    return fps, mv, rounds * workers, dt, workers


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return
    from paper_1310_1371_gb300 import synth
    frames = [f.image for f in synth.plain_full_batch(4)]
    params = synth.PLAIN_FULL_PARAMS
    workers = oracle_workers()
    # each step is one round: one frame per worker process, frame-parallel
    # (so that no worker idles in the timed region)
    oracle_pool_run(frames, params, args.warmup * workers, workers)
    value, mv, dt = oracle_pool_run(frames, params, args.steps * workers, workers)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD,
                                            "step": f"{workers} frames through the FP64 CPU oracle, one per worker",
                                            "workers": workers},
            "mvotes_per_s": mv,
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": workers, "kind": "oracle",
                             "sample": f"{args.steps * workers} frames of the workload (4 distinct, cycled), "
                                       f"{workers} per step, one per worker process"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU
def run_ours(args):
    import torch
    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_1310_1371_gb300 import rd, synth

    B = args.batch
    params = synth.PLAIN_FULL_PARAMS
    imgs = np.stack(make_frames(B, rank))
    video_imgs = serve_pool = None
    if rank == 0 and args.extras:   # inputs of the extra legs, rendered in spawn pools
        video_imgs = synth.video_images(args.extra_video_frames)
        serve_pool = synth.serve_images(args.extra_serve_pool)
    frames = torch.from_numpy(imgs).cuda()
    geo = (args.tile, args.slab) if args.tile else None  # None: the automatic geometry
    det = rd.Detector(params, H, W, B, geometry=geo)
    stream = torch.cuda.current_stream()

    # warm-up (also the parity smoke of this launch: overflow must not occur)
    for _ in range(args.warmup):
        det.detect_async(frames)
    st0 = det.stats()
    if st0.overflow:
        raise RuntimeError(f"capacity overflow in the benchmark workload: {st0.overflow}")

    # ---- device-resident throughput: K steps back to back, no host sync inside
    sampler = ClockSampler(local_rank) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        det.detect_async(frames)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    stats = det.stats()
    # ---- per-stage times (the library's CUDA events), a separate pass of the same steps
    det.set_timing(True)
    stage_ms = np.zeros(len(STAGES))
    for _ in range(args.steps):
        det.detect_async(frames)
        stage_ms += det.timing()
    det.set_timing(False)
    ms = max_over_ranks(ms, dist, "cuda")
    if dist:
        dist.barrier()
    value = job_rate(B * args.steps, world, ms / 1e3)
    votes_per_step = stats.votes

    # ---- end to end through rd_detect_host (pinned host frames in, host rings
    #      out): several callers, each with its own context, stream and pinned
    #      frames, so that one call's copies overlap another's kernels, as a
    #      client streaming batches would
    import threading
    nc = max(1, args.e2e_callers)
    dets = [det] + [rd.Detector(params, H, W, B, geometry=geo) for _ in range(nc - 1)]
    hosts = [torch.from_numpy(imgs).pin_memory().numpy() for _ in range(nc)]
    streams = [torch.cuda.Stream() for _ in range(nc)]
    for i in range(nc):
        dets[i].detect_host(hosts[i], streams[i])
    torch.cuda.synchronize()
    e2e_steps = max(2 * nc, args.steps // 4)
    e2e_steps -= e2e_steps % nc
    d2h_per = [0] * nc

    def caller(i):
        for _ in range(e2e_steps // nc):
            rings, counts, offs, stt = dets[i].detect_host(hosts[i], streams[i])
            d2h_per[i] = 8 * B + 40 * int(counts.sum())

    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    workers = [threading.Thread(target=caller, args=(i,)) for i in range(nc)]
    for w in workers:
        w.start()
    for w in workers:
        w.join()
    e2e_s = time.perf_counter() - t0
    d2h = max(d2h_per)
    for d in dets[1:]:
        d.close()
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = job_rate(B * e2e_steps, world, e2e_s)

    if rank == 0:
        # ---- roofline of the dominant stage (K4) and of the stencil stage (K1)
        per_launch = stage_ms / args.steps
        dom = int(np.argmax(per_launch))
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        ridge_per_step = stats.ridge_pixels
        # K1: frames read once, ridge records (x|y, exact Hessian) written once
        k1_bytes = B * H * W * 2 + ridge_per_step * (4 + 24)
        # K4: one increment per vote plus one multiply-add per smoothing-window tap at each hotspot
        k4_ops = stats.votes + stats.smooth_macs
        int_peak = 152 * 64 * sm_mhz * 1e6 / 1e9  # Gop/s: INT32 multiply-add issue rate, 64 lanes/SM/clk
        # a capture belongs to the kernel's source file and the shared headers it includes
        src_hash = {}
        for f in ("k_stencil.cu", "k_vote.cu"):
            h = hashlib.sha1()
            for part in (f, "rd_internal.cuh", "rd_cert.cuh"):
                h.update(open(os.path.join(ROOT, "paper_1310_1371_gb300", "csrc", part), "rb").read())
            src_hash[f] = h.hexdigest()[:12]
        traffic_db = {}
        tfile = os.path.join(ROOT, "profiles", "dram_traffic.json")
        if os.path.exists(tfile):
            traffic_db = json.load(open(tfile))

        def counter_for(stage, src, key):
            t = traffic_db.get(stage)
            if not t or t.get("source_sha1") != src_hash[src] or key not in t:
                return None          # no capture of the current kernel
            return t[key] * B

        def traffic_for(stage, src):
            return counter_for(stage, src, "bytes_per_frame")

        # instruction issue peak: 152 SMs x 4 schedulers x 32 lanes per clock
        issue_peak = 152 * 128 * sm_mhz * 1e6 / 1e9   # G thread-instructions/s
        k1 = {"kernel": "stencil_ridge", "bound": "hbm", "achieved": k1_bytes / (per_launch[0] / 1e3) / 1e9,
              "peak": hbm, "unit": "GB/s", "traffic": traffic_for("stencil_ridge", "k_stencil.cu"),
              "peak_source": hbm_src}
        k1["frac"] = k1["achieved"] / hbm
        k1_instr = counter_for("stencil_ridge", "k_stencil.cu", "thread_instructions_per_frame")
        k1["issue"] = None if k1_instr is None else {
            "achieved": k1_instr / (per_launch[0] / 1e3) / 1e9, "peak": issue_peak, "unit": "G thread-instr/s",
            "frac": k1_instr / (per_launch[0] / 1e3) / 1e9 / issue_peak,
            "instructions_per_pixel": k1_instr / (B * H * W),
            "source": "ncu smsp__thread_inst_executed.sum of the current kernel source (profiles/dram_traffic.json)",
            "peak_source": f"152 SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz"}
        k4 = {"kernel": "vote_accumulate_peaks", "bound": "alu", "achieved": k4_ops / (per_launch[3] / 1e3) / 1e9,
              "peak": int_peak, "unit": "Gop/s", "traffic": traffic_for("vote_accumulate_peaks", "k_vote.cu"),
              "ops_per_launch": int(k4_ops),
              "peak_source": f"152 SMs x 64 INT32 lanes x {sm_mhz:.0f} MHz (recipe unit counts and max clock)"}
        k4["frac"] = k4["achieved"] / int_peak
        # shared-memory atomic adds: the unit that accumulates the votes, peak measured now on this GPU
        probe = {}
        for pat, name in rd.PROBE_PATTERNS.items():
            rate, _ = rd.rd_probe_smem_atomics(pat, 4, 8192)
            probe[name] = rate / 1e9
        atom_peak = probe[rd.PROBE_PATTERNS[0]]
        k4_atom = {"kernel": "vote_accumulate_peaks", "bound": "smem_atomic",
                   "achieved": stats.votes / (per_launch[3] / 1e3) / 1e9, "peak": atom_peak,
                   "unit": "G atomic adds/s", "traffic": traffic_for("vote_accumulate_peaks", "k_vote.cu"),
                   "atomics_per_launch": int(stats.votes),
                   "peak_source": "measured in this run: rd_probe_smem_atomics, conflict-free u32 adds",
                   "measured_peaks": probe}
        k4_atom["frac"] = k4_atom["achieved"] / atom_peak
        k4_atom["frac_of_vote_stream_peak"] = k4_atom["achieved"] / probe[rd.PROBE_PATTERNS[2]]
        k4_instr = counter_for("vote_accumulate_peaks", "k_vote.cu", "thread_instructions_per_frame")
        k4_atom["issue"] = None if k4_instr is None else {
            "achieved": k4_instr / (per_launch[3] / 1e3) / 1e9, "peak": issue_peak, "unit": "G thread-instr/s",
            "frac": k4_instr / (per_launch[3] / 1e3) / 1e9 / issue_peak,
            "instructions_per_vote": k4_instr / max(1.0, float(stats.votes)),
            "source": "ncu smsp__thread_inst_executed.sum of the current kernel source (profiles/dram_traffic.json)",
            "peak_source": f"152 SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz"}
        if dom == 0:
            roofline, other = k1, k4_atom
        else:
            roofline, other = k4_atom, k1
        # ---- CPU baseline (oracle, bounded sample)
        cpu_fps, cpu_mv, ndone, cpu_dt, cpu_cores = oracle_rate(imgs[: max(1, args.cpu_frames)], params,
                                                               args.cpu_budget)
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch_frames": B, "frames_bytes": int(imgs.nbytes),
                       "l2": (f"inputs ({imgs.nbytes / 2**20:.0f} MiB) larger than L2; no flush" if imgs.nbytes > 129e6
                              else f"inputs ({imgs.nbytes / 2**20:.0f} MiB) fit in L2: L2-warm"),
                       "parallelism": f"replicas x{world}", "geometry": list(det.geometry())},
            "mvotes_per_s": votes_per_step * args.steps * world / (ms / 1e3) / 1e6,
            "votes_per_frame": votes_per_step / B, "ridge_pixels_per_frame": ridge_per_step / B,
            "rings_per_frame": stats.peaks / B, "exact_fallbacks_per_frame": stats.exact_fallbacks / B,
            "hotspots_per_frame": stats.hotspots / B, "smooth_macs_per_frame": stats.smooth_macs / B,
            "stage_ms_per_step": {s: round(float(v), 4) for s, v in zip(STAGES, per_launch)},
            "roofline": roofline,
            "roofline_other": other,
            "roofline_alu": k4,
            "cpu_baseline": {"value": cpu_fps, "unit": "frames/s", "cores": cpu_cores, "kind": "oracle",
                             "sample": f"{ndone} frames of the workload in {cpu_dt:.1f} s, one per worker process",
                             "mvotes_per_s": cpu_mv},
            "e2e": {"value": e2e_value, "unit": "frames/s", "h2d_bytes_per_step": int(imgs.nbytes),
                    "d2h_bytes_per_step": int(d2h), "api": "rd_detect_host", "steps": e2e_steps,
                    "callers": f"{nc} host threads, each its own context, stream and pinned frames"},
            "gpu_launches": KERNELS_PER_CALL * args.steps,
            "clocks": clocks,
        }
    det.close()
    if rank == 0:
        if args.extras:
            # the metric's other parts, bounded: batched vs plain on a video
            # subset, and a Poisson request stream through the server
            line["batched_vs_plain"] = measure_video(args.extra_video_frames, args.extra_video_batch, 3,
                                                     video_imgs)
            line["serve"] = measure_serve(args.extra_serve_requests, args.serve_rate, serve_pool,
                                          args.extra_serve_pool, args.serve_budget_gb)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ batched video (uneven frames)
VIDEO_METRIC = "frames/s, drifting-track video of 1024x1024 u8 frames (20-300 rings, r 5-40): batched graph path"


def measure_video(n, B, warmup, imgs=None):
    """The batched path (autotuned geometry, persistent voting) against the
    plain per-frame path (one rd_detect per frame) on the same resident
    n-frame video, with the results of both compared frame by frame
    (untimed).  With B = n the whole video is one rd_detect call captured in
    a CUDA graph: one persistent launch per kernel, one graph replay, no frame
    copies.  With B < n the batched path runs n / B calls on consecutive
    slices of the resident video (no graph).  Returns a dict."""
    from paper_1310_1371_gb300 import synth
    if n % B:
        raise SystemExit("video frames must be a multiple of the video batch")
    if imgs is None:
        imgs = synth.video_images(n)  # spawn pool
    import torch
    from paper_1310_1371_gb300 import rd
    params = synth.VIDEO_PARAMS
    vid = torch.from_numpy(imgs).cuda()
    stream = torch.cuda.Stream()
    geo = rd.rd_autotune(params, vid[:min(B, 100)], stream)
    batched = rd.Detector(params, H, W, B)  # automatic geometry: the tuned one
    graph = B == n
    batched.set_graph(graph)
    plain = rd.Detector(params, H, W, 1)
    dev_bytes = batched.device_bytes() + plain.device_bytes()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def batched_pass(collect=False):
        out, votes = [], 0
        for c in range(n // B):
            if collect:
                rings, st = batched.detect(vid[c * B:(c + 1) * B], stream)
                out += [r.copy() for r in rings]
                votes += st.votes
            else:
                batched.detect_async(vid[c * B:(c + 1) * B], stream)
        return out, votes

    def plain_pass(collect=False):
        out = []
        for i in range(n):
            if collect:
                rings, _ = plain.detect(vid[i:i + 1], stream)
                out.append(rings[0].copy())
            else:
                plain.detect_async(vid[i:i + 1], stream)
        return out

    for _ in range(warmup):  # the first pass captures the graph
        batched_pass()
    for i in range(max(3, warmup)):
        plain.detect_async(vid[i:i + 1], stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    time.sleep(0.3)
    ev0.record(stream)
    batched_pass()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_b = ev0.elapsed_time(ev1)
    ev0.record(stream)
    plain_pass()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_p = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    rb, votes = batched_pass(collect=True)
    rp = plain_pass(collect=True)
    fields = ("ix", "iy", "ir", "cx", "cy", "r", "score", "n_fit", "flags")
    identical = len(rb) == len(rp) == n and all(
        len(a) == len(b) and all(np.array_equal(a[k], b[k]) for k in fields) for a, b in zip(rb, rp))
    batched.close()
    plain.close()
    return {"batched_frames_per_s": n / (ms_b / 1e3), "plain_frames_per_s": n / (ms_p / 1e3),
            "ms_batched": ms_b, "ms_plain": ms_p, "speedup_vs_plain": ms_p / ms_b,
            "identical_results": bool(identical), "frames": n, "batch_frames": B, "geometry": list(geo),
            "graph": graph, "launches": "one rd_detect over the whole resident video, one graph replay" if graph
            else f"{n // B} rd_detect calls on slices of the resident video", "frame_copies": 0,
            "device_bytes": int(dev_bytes), "rings_total": int(sum(len(r) for r in rb)),
            "mvotes_per_s": votes / (ms_b / 1e3) / 1e6, "bytes": int(imgs.nbytes), "clocks": clocks}


def run_video(args):
    """--workload video: the whole drifting-track video, batched vs plain."""
    from paper_1310_1371_gb300 import synth
    n, B = args.video_frames, args.video_batch
    imgs = synth.video_images(n)  # spawn pool, before any CUDA call
    import torch
    torch.cuda.set_device(0)
    v = measure_video(n, B, args.warmup, imgs)
    line = {"metric": VIDEO_METRIC, "value": v["batched_frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": 1,
            "warmup": args.warmup, "ms_per_step": v["ms_batched"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"video: {n} frames 1024x1024 u8, 20-300 drifting rings r 8-30, search r 5-40",
                       "batch_frames": B, "geometry": v["geometry"], "graph": v["graph"], "launches": v["launches"],
                       "frame_copies": 0, "device_bytes": v["device_bytes"],
                       "l2": f"inputs ({v['bytes'] / 2**20:.0f} MiB) larger than L2; no flush"},
            "plain_per_frame": {"value": v["plain_frames_per_s"], "unit": "frames/s", "ms_total": v["ms_plain"]},
            "speedup_vs_plain": v["speedup_vs_plain"], "identical_results": v["identical_results"],
            "rings_total": v["rings_total"], "mvotes_per_s": v["mvotes_per_s"],
            "gpu_launches": (n // B) * KERNELS_PER_CALL, "clocks": v["clocks"]}
    print(json.dumps(line))


# ------------------------------------------------------------------ differentiable soft score
DIFF_METRIC = "frames/s, soft ring score + backward (image and ring gradients), 512x512 f32, 64 rings per frame"


def _match(truth, found, tol=3.0):
    """Index of the found ring nearest each true ring (centre within tol px), or -1."""
    out = np.full(len(truth), -1)
    if len(found) == 0:
        return out
    for i, (cx, cy, r) in enumerate(truth):
        d = np.hypot(found[:, 0] - cx, found[:, 1] - cy) + np.abs(found[:, 2] - r)
        j = int(np.argmin(d))
        if d[j] < tol:
            out[i] = j
    return out


def run_diff(args):
    """rd_soft_score (scores and ring gradients) and rd_backward (image and ring
    gradients) on 256 float frames with 64 rings each; rd_refine from the
    hard detector's rings, with the sub-pixel error against the true rings
    before and after; the FP64 oracle's forward + backward on a bounded sample."""
    from paper_1310_1371_gb300 import synth
    n, H, W = args.diff_frames, 512, 512
    imgs, truth = synth.diff_images(n)  # spawn pool, before any CUDA call
    import torch
    from paper_1310_1371_gb300 import rd
    torch.cuda.set_device(0)
    params = synth.DIFF_PARAMS
    det = rd.Detector(params, H, W, n)
    frames = torch.from_numpy(imgs).cuda()
    # starting rings: the hard detector on the frames rounded to u16
    f16 = torch.from_numpy(np.clip(np.rint(imgs), 0, 65535).astype(np.uint16)).cuda()
    found, _ = det.detect(f16)
    counts_l = [len(r) for r in found]
    flat = np.concatenate([np.stack([r["cx"], r["cy"], r["r"]], 1) for r in found]).astype(np.float32)
    counts = torch.tensor(counts_l, dtype=torch.int32, device="cuda")
    rings = rd.pack_rings(torch.from_numpy(flat).cuda())
    ones = torch.ones(len(flat), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(k):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / k

    sampler = ClockSampler(0)
    time.sleep(0.3)
    ms_fwd = timed(lambda: det.soft_score(frames, rings, counts, with_grad=True), args.steps)
    ms_step = timed(lambda: (det.soft_score(frames, rings, counts), det.backward(frames, rings, counts, ones)),
                    args.steps)
    refined = rings.clone()
    iters = 20
    ev0.record(stream)
    det.refine(frames, refined, counts, iters=iters, step=0.5)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_refine = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    # sub-pixel error of matched rings (centre distance, radius) before and after refinement
    ref = refined[:, 1:4].cpu().numpy()
    err_b, err_a = [], []
    o = 0
    for f in range(n):
        k = counts_l[f]
        m = _match(truth[f], flat[o:o + k])
        for i, j in enumerate(m):
            if j >= 0:
                t = truth[f, i]
                err_b.append((math.hypot(flat[o + j, 0] - t[0], flat[o + j, 1] - t[1]), abs(flat[o + j, 2] - t[2]),
                              abs(flat[o + j, 0] - t[0]), abs(flat[o + j, 1] - t[1])))
                err_a.append((math.hypot(ref[o + j, 0] - t[0], ref[o + j, 1] - t[1]), abs(ref[o + j, 2] - t[2]),
                              abs(ref[o + j, 0] - t[0]), abs(ref[o + j, 1] - t[1])))
        o += k
    err_b, err_a = np.array(err_b), np.array(err_a)
    # the FP64 oracle's forward + backward on a bounded sample of frames
    from oracle import soft as S
    sp = S.SoftParams.make(**params)
    t0, done, o = time.perf_counter(), 0, 0
    while done < n and (done == 0 or time.perf_counter() - t0 < args.cpu_budget):
        S.soft_grads(imgs[done], flat[o:o + counts_l[done]].astype(np.float64), sp)
        o += counts_l[done]
        done += 1
    cpu_s = time.perf_counter() - t0
    line = {"metric": DIFF_METRIC, "value": n / (ms_step / 1e3), "unit": "frames/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (f32 frames and outputs)", "data": "synthetic",
            "config": {"workload": f"diff: {n} frames 512x512 f32, 64 rings r 10-50 with sub-pixel truth, search r 8-56",
                       "rings": int(len(flat)), "l2": f"inputs ({imgs.nbytes / 2**20:.0f} MiB) larger than L2; no flush"},
            "score_and_ring_grads": {"value": n / (ms_fwd / 1e3), "unit": "frames/s"},
            "refine": {"iters": iters, "ms": ms_refine, "frames_per_s": n / (ms_refine / 1e3),
                       "matched_rings": int(len(err_b)),
                       "median_centre_err_px": [float(np.median(err_b[:, 0])), float(np.median(err_a[:, 0]))],
                       "median_radius_err_px": [float(np.median(err_b[:, 1])), float(np.median(err_a[:, 1]))],
                       "median_abs_cx_px": [float(np.median(err_b[:, 2])), float(np.median(err_a[:, 2]))],
                       "median_abs_cy_px": [float(np.median(err_b[:, 3])), float(np.median(err_a[:, 3]))],
                       "note": "[before (hard detector, Kasa fit on u16-rounded frames), after rd_refine]"},
            "cpu_baseline": {"value": done / cpu_s, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"{done} frames: FP64 soft score + autograd gradients in {cpu_s:.1f} s"},
            "gpu_launches": 14 * args.steps, "clocks": clocks}
    print(json.dumps(line))
    det.close()


# ------------------------------------------------------------------ serving (continuous batching)
SERVE_METRIC = "p50/p99 latency and frames/s, Poisson stream of single-frame requests (256^2-2048^2 u16)"


SERVE_SIZES = (256, 512, 1024, 2048)


def measure_serve(n, rate, pool, pool_per_class, budget_gb, slots=2):
    """A Poisson stream of n single-frame requests at `rate`/s (sizes uniform
    over 256^2 .. 2048^2, u16, 10-400 rings) through the continuous-batching
    server; latency from submission to results on the host.  `pool` holds
    the frames of each size class.  Returns a dict."""
    import threading
    from paper_1310_1371_gb300 import rd, synth
    import torch
    sizes = SERVE_SIZES
    batch = {256: 16, 512: 8, 1024: 4, 2048: 2}
    classes = [dict(params=synth.SERVE_CLASSES[s], H=s, W=s, dtype="u16", max_batch=batch[s], slots=slots) for s in sizes]
    server = rd.Server(classes, mem_budget=int(budget_gb * 2**30), queue_cap=8192)
    for c, s in enumerate(sizes):  # warm-up: one request per class
        server.submit(c, pool[s][0], -1 - c)
    got = 0
    while got < len(sizes):
        got += len(server.poll(wait_ms=100))
    rng = np.random.default_rng(1005)
    arrive = np.cumsum(rng.exponential(1.0 / rate, size=n))
    cls = rng.integers(0, len(sizes), size=n)
    idx = rng.integers(0, pool_per_class, size=n)
    lat = np.zeros(n)
    status = np.zeros(n, dtype=np.int32)
    t_done = [0.0]

    def collect():
        seen = 0
        while seen < n:
            for rid, c, st, rings, l in server.poll(wait_ms=20):
                lat[rid] = l
                status[rid] = st
                seen += 1
            t_done[0] = time.perf_counter()

    th = threading.Thread(target=collect)
    sampler = ClockSampler(torch.cuda.current_device())
    th.start()
    t0 = time.perf_counter()
    busy = 0
    for i in range(n):
        wait = t0 + arrive[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        while server.submit(int(cls[i]), pool[sizes[cls[i]]][idx[i]], i) == rd.RD_E_BUSY:
            busy += 1
            time.sleep(1e-4)
    th.join()
    clocks = sampler.stop()
    wall = t_done[0] - t0
    stats = server.stats()
    server.close()
    ms = lat / 1e3
    per = {f"{s}x{s}": {"requests": int((cls == c).sum()), "p50_ms": float(np.percentile(ms[cls == c], 50)),
                        "p99_ms": float(np.percentile(ms[cls == c], 99))} for c, s in enumerate(sizes)}
    return {"requests": n, "offered_per_s": rate, "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "frames_per_s": n / wall, "wall_s": wall, "per_class": per,
            "batches": stats["batches"] - len(sizes), "device_bytes": stats["device_bytes"],
            "errors": int((status != 0).sum()), "submit_retries_busy": busy, "max_batch": batch,
            "slots_per_class": slots, "mem_budget_gb": budget_gb, "frames_per_class_pool": pool_per_class,
            "clocks": clocks}


def run_serve(args):
    """--workload serve: the request stream, its latency percentiles."""
    from paper_1310_1371_gb300 import synth
    pool = synth.serve_images(args.serve_pool)  # spawn pool, before any CUDA call
    import torch
    torch.cuda.set_device(0)
    n, rate = args.serve_requests, args.serve_rate
    v = measure_serve(n, rate, pool, args.serve_pool, args.serve_budget_gb, args.serve_slots)
    line = {"metric": SERVE_METRIC, "value": v["p99_ms"], "unit": "ms (p99 latency)",
            "higher_is_better": False, "n_gpus": 1, "steps": n, "warmup": len(SERVE_SIZES),
            "ms_per_step": v["wall_s"] * 1e3 / n, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic",
            "config": {"workload": f"serve: {n} requests, Poisson {rate}/s, sizes uniform over 256..2048 squared, "
                                   f"10-400 rings, r ranges 5-20 / 5-40 / 8-96 / 8-160",
                       "frames_per_class_pool": args.serve_pool, "max_batch": v["max_batch"],
                       "slots_per_class": args.serve_slots,
                       "mem_budget_gb": args.serve_budget_gb},
            "p50_ms": v["p50_ms"], "p99_ms": v["p99_ms"], "frames_per_s": v["frames_per_s"], "offered_per_s": rate,
            "per_class": v["per_class"], "batches": v["batches"], "device_bytes": v["device_bytes"],
            "errors": v["errors"], "submit_retries_busy": v["submit_retries_busy"],
            "gpu_launches": KERNELS_PER_CALL * v["batches"], "clocks": v["clocks"]}
    print(json.dumps(line))


# ------------------------------------------------------------------ directed-edge variant
EDGE_METRIC = "frames/s at 1024x1024 u16 (directed-edge variant, filled discs r 10-80, search r 8-96)"


def run_discs(args):
    """The directed-edge variant on a batch of 96 disc frames resident in HBM
    (the same timing protocol as the default workload)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_1310_1371_gb300 import synth
    B = args.batch
    with cf.ProcessPoolExecutor(max(1, min(16, (os.cpu_count() or 2) - 1)), mp_context=mp.get_context("spawn")) as ex:
        imgs = np.stack([f.image for f in ex.map(synth.disc_full, [3100 + i for i in range(B)])])
    import torch
    from paper_1310_1371_gb300 import rd
    torch.cuda.set_device(0)
    params = synth.DISC_FULL_PARAMS
    det = rd.Detector(params, H, W, B)
    det.set_features("edge", params["edge_thresh"])
    frames = torch.from_numpy(imgs).cuda()
    for _ in range(args.warmup):
        det.detect_async(frames)
    st0 = det.stats()
    if st0.overflow:
        raise RuntimeError(f"capacity overflow: {st0.overflow}")
    sampler = ClockSampler(0)
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        det.detect_async(frames)
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    stats = det.stats()
    det.set_timing(True)
    stage_ms = np.zeros(len(STAGES))
    for _ in range(args.steps):
        det.detect_async(frames)
        stage_ms += det.timing()
    det.close()
    line = {"metric": EDGE_METRIC, "value": B * args.steps / (ms / 1e3), "unit": "frames/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": "discs: 1024x1024 u16, 150 overlapping filled discs r 10-80, directed edges, "
                                   "gradient threshold 20, search r 8-96",
                       "batch_frames": B, "l2": f"inputs ({imgs.nbytes / 2**20:.0f} MiB) larger than L2; no flush"},
            "edge_pixels_per_frame": stats.ridge_pixels / B, "votes_per_frame": stats.votes / B,
            "rings_per_frame": stats.peaks / B,
            "stage_ms_per_step": {k: float(v) for k, v in zip(["edge_stage", "(none)", "vote_bin",
                                                               "vote_accumulate_peaks", "sort_fit"],
                                                              np.round(stage_ms / args.steps, 4))},
            "gpu_launches": (KERNELS_PER_CALL + 2) * args.steps, "clocks": clocks}
    print(json.dumps(line))


def _one_frame_truth(seed):
    from paper_1310_1371_gb300 import synth
    f = synth.plain_full(seed=seed)
    return f.image, f.rings


def _accuracy(rings, truth):
    """Median |d cx|, |d cy|, |d r| of the fitted rings nearest to each true
    ring (within 3 px in centre and radius), and the fraction of true rings
    so matched."""
    got = np.stack([rings["cx"], rings["cy"], rings["r"]], 1).astype(np.float64)
    errs, hit = [], 0
    for t in truth:
        if len(got) == 0:
            continue
        d = np.abs(got - t)
        k = int(np.argmin(d.max(1)))
        if d[k].max() <= 3.0:
            errs.append(d[k])
            hit += 1
    e = np.median(np.array(errs), 0) if errs else np.full(3, np.nan)
    return {"median_abs_cx_px": float(e[0]), "median_abs_cy_px": float(e[1]), "median_abs_r_px": float(e[2]),
            "recall": hit / max(1, len(truth))}


def run_coarse(args):
    """A coarse circle parameter space (cells of c px) on the default
    workload's 96 frames: frames/s at c and at full resolution on the same
    resident frames (same timing protocol), and the fitted rings' accuracy
    against the synthetic truth for both."""
    import concurrent.futures as cf
    import multiprocessing as mp
    B = args.batch
    with cf.ProcessPoolExecutor(max(1, min(16, (os.cpu_count() or 2) - 1)), mp_context=mp.get_context("spawn")) as ex:
        got = list(ex.map(_one_frame_truth, frame_seeds(0, B)))
    imgs = np.stack([g[0] for g in got])
    truth = [g[1] for g in got]
    import torch
    from paper_1310_1371_gb300 import rd, synth
    torch.cuda.set_device(0)
    frames = torch.from_numpy(imgs).cuda()
    res = {}
    clocks = None
    for c in (1, args.coarse):
        params = dict(synth.PLAIN_FULL_PARAMS, coarse=c)
        geo = (args.tile, args.slab) if (c != 1 and args.tile) else None
        det = rd.Detector(params, H, W, B, geometry=geo)
        for _ in range(args.warmup):
            det.detect_async(frames)
        if det.stats().overflow:
            raise RuntimeError(f"capacity overflow: {det.stats().overflow}")
        sampler = ClockSampler(0) if c != 1 else None
        time.sleep(0.3)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            det.detect_async(frames)
        ev1.record()
        torch.cuda.synchronize()
        if sampler is not None:
            clocks = sampler.stop()
        ms = ev0.elapsed_time(ev1)
        rings, stats = det.detect(frames)
        acc = [_accuracy(rings[i], truth[i]) for i in range(B)]
        det.set_timing(True)
        stage_ms = np.zeros(len(STAGES))
        for _ in range(5):
            det.detect_async(frames)
            stage_ms += det.timing()
        res[c] = {"frames_per_s": B * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                  "geometry": list(det.geometry()),
                  "stage_ms_per_step": {k: float(v) for k, v in zip(STAGES, np.round(stage_ms / 5, 4))},
                  "rings_per_frame": stats.peaks / B, "votes_per_frame": stats.votes / B,
                  "hotspots_per_frame": stats.hotspots / B, "smooth_macs_per_frame": stats.smooth_macs / B,
                  "exact_fallbacks_per_frame": stats.exact_fallbacks / B,
                  "accuracy": {k: float(np.nanmedian([a[k] for a in acc])) for k in acc[0]}}
        det.close()
    c = args.coarse
    line = {"metric": METRIC + f", {c} px parameter-space cells", "value": res[c]["frames_per_s"], "unit": "frames/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[c]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": f"coarse: plain_full frames with a {c} px cell circle parameter space",
                       "batch_frames": B, "l2": f"inputs ({imgs.nbytes / 2**20:.0f} MiB) larger than L2; no flush"},
            "coarse": {str(k): v for k, v in res.items()},
            "gpu_launches": KERNELS_PER_CALL * args.steps, "clocks": clocks}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=96)
    ap.add_argument("--cpu-frames", type=int, default=4)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--workload", default="plain_full",
                    choices=["plain_full", "video", "diff", "serve", "discs", "coarse"])
    ap.add_argument("--coarse", type=int, default=2, choices=[2, 4])
    ap.add_argument("--e2e-callers", type=int, default=4, help="host threads of the end-to-end measurement")
    ap.add_argument("--tile", type=int, default=0,
                    help="accumulator tile (cells) of the default and coarse workloads; 0: automatic")
    ap.add_argument("--slab", type=int, default=16, help="slab levels with --tile")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=500.0)
    ap.add_argument("--serve-pool", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-slots", type=int, default=2, help="server slots (context, stream, staging) per size class")
    ap.add_argument("--diff-frames", type=int, default=256)
    ap.add_argument("--video-frames", type=int, default=2000)
    ap.add_argument("--video-batch", type=int, default=2000,
                    help="frames per rd_detect call of the batched path (the whole video: one graph replay)")
    ap.add_argument("--extras", type=int, default=1,
                    help="default workload: add the batched-vs-plain and serving legs to the line (rank 0)")
    ap.add_argument("--extra-video-frames", type=int, default=200)
    ap.add_argument("--extra-video-batch", type=int, default=200)
    ap.add_argument("--extra-serve-requests", type=int, default=1000)
    ap.add_argument("--extra-serve-pool", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "video":
        run_video(args)
    elif args.workload == "diff":
        run_diff(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "discs":
        run_discs(args)
    elif args.workload == "coarse":
        run_coarse(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
