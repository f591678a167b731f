#!/usr/bin/env python
"""Throughput of the FlowRoI hot path (flow -> RoI mask -> JPEG2000 front
end) on GB300, through the library's C ABI.

One step = one batch holding the next frame of every stream (16 streams of
2048x2048 12-bit frames by default), i.e. one pass of the whole hot path:
pyramid + expansion, coarse-to-fine displacement, saliency, exact quantile,
opening/closing, 9/7 DWT with quantisation and RoI up-shift.

Printed (one JSON line, rank 0):
  value      frames/s with inputs resident in HBM (CUDA events on the
             library's compute stream around K steps, max over ranks);
  e2e        the same through host buffers: every step copies its frames
             from pinned host memory and reads every mask and coefficient
             plane back to pinned host memory;
  plain_fps  the plain per-frame path (each frame launched alone, no graph);
  latency    p50/p99 submit -> result-ready of the e2e run;
  roofline   the dominant kernel (level-0 displacement) vs measured HBM
             bandwidth, from per-kernel CUDA events;
  cpu_baseline  the oracle, single-threaded, on a bounded crop sample;
  cpu_baseline_all_cores  the same with one oracle process per host core.
`--impl reference` times the oracle alone (rank 0) on crops of the same
workload and prints the same metric.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s (flow+mask+DWT) at 1 GB300 and p50/p99 frame latency vs plain per-frame path"

WORKLOADS = {
    # 16 streams (one per lens) x 32 frames of 2048^2 12-bit, 200 migrating
    # blobs, 5-level pyramid, 9/7 DWT 5 levels in float32.
    "batched_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                            dwt_levels=5, wavelet=97, precision=32, seed_base=3000),
    # same workload, pyramid and expansion fields stored in fp16
    "fp16_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                         dwt_levels=5, wavelet=97, precision=16, seed_base=3000),
    # same workload with the optional denoising of the flow input (median 3x3,
    # bilateral 5x5) on
    "denoise_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                            dwt_levels=5, wavelet=97, precision=32, seed_base=3000, denoise=1),
    # same workload with the small-component filter of the RoI mask on
    # (8-connected components under 500 pixels removed)
    "components_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                               dwt_levels=5, wavelet=97, precision=32, seed_base=3000, min_area=500),
    # same workload with each frame registered to its predecessor by phase
    # correlation of pyramid level 2 (512x512 FFTs)
    "register_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                             dwt_levels=5, wavelet=97, precision=32, seed_base=3000, register_frames=1, reg_level=2),
    # the batched workload, each step's 16 frames also coded into
    # rate-controlled containers of 1 bit per pixel of pass data (EBCOT tier-1,
    # rate control, container)
    "ebcot_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                          dwt_levels=5, wavelet=97, precision=32, seed_base=3000, codestream_bpp=1.0),
    # the same with the coder's contexts reset at every pass (code-block style
    # 0x02 with per-pass termination: no chain of context states through a
    # code-block, every pass's MQ states formed apart)
    "ebcot_reset_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                                dwt_levels=5, wavelet=97, precision=32, seed_base=3000, codestream_bpp=1.0,
                                codestream_reset=1),
    # the same with JPEG2000 Part 1 codestreams instead of containers
    "j2c_16x2048": dict(streams=16, frames=32, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                        dwt_levels=5, wavelet=97, precision=32, seed_base=3000, codestream_bpp=1.0, codestream_format=1),
    # four streams of it (small case for profiler captures of the coder)
    "ebcot_4x2048": dict(streams=4, frames=4, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                         dwt_levels=5, wavelet=97, precision=32, seed_base=3000, codestream_bpp=1.0),
    # four streams with fp16 storage (small case for profiler captures)
    "small_fp16_4x2048": dict(streams=4, frames=4, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                              dwt_levels=5, wavelet=97, precision=16, seed_base=3000),
    # four streams of the batched workload's frames (small case for profiler captures)
    "small_4x2048": dict(streams=4, frames=4, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                         dwt_levels=5, wavelet=97, precision=32, seed_base=3000),
    # serving: 64 streams (16 each of 512^2, 1024^2, 2048^2, 2048x1536, 12-bit)
    # through the scheduler thread; Poisson arrivals, then a burst replay
    "serving_64mixed": dict(streams=64, frames=4, h=2048, w=2048, blobs=200, bit_depth=12, pyr_levels=5,
                            dwt_levels=5, wavelet=97, precision=32, seed_base=5000,
                            sizes=[(512, 512), (1024, 1024), (2048, 2048), (1536, 2048)]),
    # one stream of 64 1024^2 12-bit frames, 5/3 DWT (plain method at full size)
    "stream_1024": dict(streams=1, frames=64, h=1024, w=1024, blobs=80, bit_depth=12, pyr_levels=4,
                        dwt_levels=5, wavelet=53, precision=32, seed_base=2000),
}

# Algorithmic bytes per level-0 pixel of one launch of the two displacement
# kernels (storage 32 = fp32 fields, 16 = fp16), (first iteration, later ones):
#   update: read the five expansion fields of the current frame and, at the
#           warped position, of the previous frame, plus the prior flow (the
#           coarse flow, a quarter of a pixel's 8 B, on the first iteration);
#           write the five G, h planes:   fp32 5*4+5*4+{2,8}+5*4 = {62, 68} B
#                                         fp16 5*2+5*2+{2,8}+5*2 = {32, 38} B
#   window: read the five G, h planes, write the flow: fp32 20+8 = 28 B,
#           fp16 10+8 = 18 B.
KERNEL_BYTES = {("update", 32): (62.0, 68.0), ("update", 16): (32.0, 38.0),
                ("window", 32): (28.0, 28.0), ("window", 16): (18.0, 18.0)}
# Algorithmic bytes per pixel of one launch of the other kernels with a
# roofline line (storage 32 / 16; `bpp` = bytes per raw sample):
#   expand level 0: read the raw frame, write the five expansion fields and
#           the next pyramid level (a quarter pixel): bpp + 5*4 + 4/4
#           (fp16: bpp + 5*2 + 2/4);
#   dwt level 1 (per frame pixel): read the raw sample and the RoI mask
#           byte, write the three high bands' int32 coefficients (3/4 of the
#           pixels) and the low-low band (a quarter: 4 B value + 1 B mask):
#           bpp + 1 + 3 + 1 + 0.25.
def other_bytes(name, storage, bpp):
    if name == "expand":
        return bpp + (5 * 4 + 1.0 if storage == 32 else 5 * 2 + 0.5)
    if name == "dwt":
        return bpp + 1 + 3 + 1 + 0.25
    raise KeyError(name)


# DRAM bytes (read + write) per level-0 pixel of one launch, measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on 4 frames of the same
# workload (traffic proportional to pixels; the fp32 update figure averages
# its three level-0 launches, the fp16 ones are single launches: update
# iteration 1, window, expansion), each
# with the source file the kernel was built from and its SHA-256 prefix at
# the time of the capture: a figure whose source has changed since is
# reported as null.
KERNEL_TRAFFIC_PER_PX = {("update", 32): (64.26, "k_flow.cu", "c9219d3d2d871711"),
                         ("window", 32): (26.06, "k_flow.cu", "c9219d3d2d871711"),
                         ("expand", 32): (19.16, "k_expand.cu", "83e2d4444934406d"),
                         ("dwt", 32): (4.03, "k_dwt.cu", "48cdef260a22e4fa"),
                         ("update", 16): (37.35, "k_flow.cu", "c9219d3d2d871711"),
                         ("window", 16): (15.25, "k_flow.cu", "c9219d3d2d871711"),
                         ("expand", 16): (8.91, "k_expand.cu", "83e2d4444934406d")}


def traffic_per_px(name, storage):
    import hashlib
    ent = KERNEL_TRAFFIC_PER_PX.get((name, storage))
    if not ent:
        return None
    per_px, src, sha = ent
    path = os.path.join(ROOT, "paper_2511_14419_gb300", "csrc", src)
    try:
        with open(path, "rb") as f:
            cur = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return per_px if cur == sha else None


# Tile table the contexts are created with (set in main: --tiles; by default
# the committed table for the workload's storage type, if there is one).
TILE_TABLE = None


def default_tiles(storage):
    path = os.path.join(ROOT, "paper_2511_14419_gb300", "tiles", f"gb300_fp{storage}.json")
    return path if os.path.exists(path) else None


def tile_kw():
    return {"tile_table": TILE_TABLE} if TILE_TABLE else {}


def tiles_desc():
    if not TILE_TABLE:
        return "built-in shapes"
    import hashlib
    with open(TILE_TABLE, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:12]
    return f"{os.path.relpath(TILE_TABLE, ROOT)} (sha256 {sha})"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def rank_streams(route, n_streams: int, ws: int, rank: int) -> list:
    """The stream ids this rank serves: the first n_streams ids (0, 1, 2,
    ...) that route(sid, ws) sends to this rank (the library's stream ->
    device routing), so every rank has n_streams streams and no stream is on
    two ranks."""
    out, sid = [], 0
    while len(out) < n_streams:
        if sid > 1000 * n_streams * ws:
            raise RuntimeError("stream routing sends too few streams to rank %d" % rank)
        if route(sid, ws) == rank:
            out.append(sid)
        sid += 1
    return out


def sid_of(wl, s: int) -> int:
    """Stream id of the workload's s-th stream on this rank."""
    return wl["sids"][s] if "sids" in wl else s


def make_frames(wl, device):
    import torch

    from synth import sequence_u16
    frames = []
    for s in range(wl["streams"]):
        frames.append(sequence_u16(wl["seed_base"] + sid_of(wl, s), wl["frames"], wl["h"], wl["w"], wl["blobs"],
                                   device=device))
    torch.cuda.synchronize()
    return frames


def max_over_ranks(x: float, ws: int, device) -> float:
    """Max of a per-rank float over all ranks (host reduction only)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank: int, ws: int, t_max: float) -> float:
    """Whole-job frames/s: every rank processed frames_per_rank frames; the
    job took as long as its slowest rank."""
    return frames_per_rank * ws / t_max


def frame_index(t, n):
    """Ping-pong through a sequence of n frames (0..n-1, n-2..0, ...)."""
    period = 2 * (n - 1)
    k = t % period
    return k if k < n else period - k


def submit(F, ctx, sid, data, idx, bd):
    while True:
        try:
            return F.flowroi_submit_frame(ctx, sid, data, idx, bd)
        except F.FlowRoIError as e:
            if e.code != F.EBUSY:
                raise
            time.sleep(50e-6)


def submit_all(F, ctx, items):
    """Submit (stream, data, frame_idx, bit_depth) items as one batch,
    retrying the tail while a stream's ring is still busy."""
    while items:
        k, st = F.flowroi_submit_frames(ctx, items)
        items = items[k:]
        if not items:
            return
        if st != F.EBUSY:
            raise F.FlowRoIError(st, F.flowroi_last_error(ctx))
        time.sleep(50e-6)


def run_device(F, wl, frames, steps, warmup, plain=False, profile_steps=0, sampler_device=None):
    """Device-resident run: returns dict(time_s, frames, launches, kernel_times, stats, clocks)."""
    import torch
    cfg = dict(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"],
               precision=wl["precision"], max_batch_frames=64, result_ring=8, denoise=wl.get("denoise", 0),
               min_area=wl.get("min_area", 0), register_frames=wl.get("register_frames", 0),
               reg_level=wl.get("reg_level", 2), flags=F.MANUAL | (F.PLAIN if plain else 0), device=torch.cuda.current_device())
    S, n, bd = wl["streams"], wl["frames"], wl["bit_depth"]
    res = {}
    with F.Context(**cfg, **tile_kw()) as ctx:
        stream = torch.cuda.ExternalStream(F.flowroi_compute_stream(ctx.h))
        t = 0

        def one_step():
            nonlocal t
            i = frame_index(t, n)
            submit_all(F, ctx.h, [(sid_of(wl, s), frames[s][i], t, bd) for s in range(S)])
            if plain:
                while F.flowroi_step(ctx.h) > 0:
                    pass
            else:
                F.flowroi_step(ctx.h)
            t += 1

        one_step()  # first frames: no predecessor
        for _ in range(warmup):
            one_step()
        F.flowroi_flush(ctx.h, -1)
        torch.cuda.synchronize()
        l0 = F.flowroi_get_stats(ctx.h)["kernel_launches"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(sampler_device) if sampler_device is not None else None
        if sampler:
            sampler.__enter__()
        gc.collect()
        gc.disable()  # no collector pauses in the timed host loop
        e0.record(stream)
        for _ in range(steps):
            one_step()
        e1.record(stream)
        gc.enable()
        F.flowroi_flush(ctx.h, -1)
        e1.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
            res["clocks"] = sampler.summary()
        res["time_s"] = e0.elapsed_time(e1) / 1e3
        res["frames"] = steps * S
        st = F.flowroi_get_stats(ctx.h)
        res["launches"] = st["kernel_launches"] - l0
        res["stats"] = st
        if profile_steps:
            F.flowroi_set_profiling(ctx.h, 2)
            for _ in range(profile_steps):
                one_step()
            F.flowroi_flush(ctx.h, -1)
            res["kernel_times"] = F.flowroi_get_kernel_times(ctx.h)
            F.flowroi_set_profiling(ctx.h, 0)
    return res


def run_e2e(F, wl, frames, steps, warmup):
    """Host-buffer run through the public API: pinned host frames in,
    pinned host masks and coefficients out, every step."""
    import torch
    S, n, bd = wl["streams"], wl["frames"], wl["bit_depth"]
    nh = min(n, 8)
    host = [[frames[s][i].cpu().pin_memory() for i in range(nh)] for s in range(S)]
    h, w = wl["h"], wl["w"]
    masks = [torch.empty((h, w), dtype=torch.uint8).pin_memory() for _ in range(S)]
    coefs = [torch.empty((h, w), dtype=torch.int32).pin_memory() for _ in range(S)]
    cfg = dict(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"],
               precision=wl["precision"], max_batch_frames=64, result_ring=8, denoise=wl.get("denoise", 0),
               min_area=wl.get("min_area", 0), register_frames=wl.get("register_frames", 0),
               reg_level=wl.get("reg_level", 2), flags=F.MANUAL,
               device=torch.cuda.current_device())
    res = {}
    with F.Context(**cfg, **tile_kw()) as ctx:
        t = 0

        def submit_step():
            nonlocal t
            i = frame_index(t, nh)
            submit_all(F, ctx.h, [(sid_of(wl, s), host[s][i], t, bd) for s in range(S)])
            F.flowroi_step(ctx.h)
            t += 1

        def fetch(step):
            # every stream's mask and coefficients of the step in one call
            # (the copies back to back, one wait)
            F.flowroi_get_results(ctx.h, [(sid_of(wl, s), step, masks[s], coefs[s]) for s in range(S)], -1)

        submit_step()
        fetch(0)
        for _ in range(warmup):
            submit_step()
            fetch(t - 1)
        torch.cuda.synchronize()
        gc.collect()
        gc.disable()  # no collector pauses in the timed host loop
        t0 = time.perf_counter()
        lag = 3  # steps in flight before a step's results are fetched (the result ring holds 8)
        for k in range(steps):
            submit_step()
            if k >= lag - 1:
                fetch(t - lag)
        for j in range(min(steps, lag - 1), 0, -1):
            fetch(t - j)
        dt = time.perf_counter() - t0
        gc.enable()
        st = F.flowroi_get_stats(ctx.h)
    res["time_s"] = dt
    res["frames"] = steps * S
    res["h2d"] = S * h * w * 2
    res["d2h"] = S * h * w * (1 + 4)
    res["stats"] = st
    return res


def run_codestream(F, wl, frames, steps, warmup, profile_steps=3):
    """Device-resident steps of the stream path with the JPEG2000 coder on
    (config.codestream_bpp): each batch's frames are coded into
    rate-controlled containers inside the batch's launches, and every
    frame's container is fetched (flowroi_get_codestream, device buffers).
    Returns the wall time of the timed steps, the containers' mean size and
    the per-kernel times of `profile_steps` further steps."""
    import torch
    cfg = dict(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"],
               precision=wl["precision"], max_batch_frames=64, result_ring=8, flags=F.MANUAL,
               codestream_bpp=wl["codestream_bpp"], codestream_format=wl.get("codestream_format", 0),
               codestream_reset=wl.get("codestream_reset", 0), device=torch.cuda.current_device())
    S, n, bd = wl["streams"], wl["frames"], wl["bit_depth"]
    H, W, L = wl["h"], wl["w"], wl["dwt_levels"]
    cap = F.flowroi_codestream_bound(W, H, L) // 4
    outs = [torch.empty(cap, dtype=torch.uint8, device="cuda") for _ in range(S)]
    res = {}
    with F.Context(**cfg, **tile_kw()) as ctx:
        t = 0
        lens = []

        def one_step(keep):
            nonlocal t
            i = frame_index(t, n)
            submit_all(F, ctx.h, [(sid_of(wl, s), frames[s][i], t, bd) for s in range(S)])
            F.flowroi_step(ctx.h)
            for s in range(S):
                k = F.flowroi_get_codestream(ctx.h, sid_of(wl, s), t, outs[s], -1)
                if keep:
                    lens.append(k)
            t += 1

        for _ in range(warmup + 1):
            one_step(False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            one_step(True)
        torch.cuda.synchronize()
        res["time_s"] = time.perf_counter() - t0
        F.flowroi_flush(ctx.h, -1)
        F.flowroi_set_profiling(ctx.h, 1)
        for _ in range(profile_steps):
            one_step(False)
        F.flowroi_flush(ctx.h, -1)
        kt = F.flowroi_get_kernel_times(ctx.h)
        F.flowroi_set_profiling(ctx.h, 0)
        launches = F.flowroi_get_stats(ctx.h)["kernel_launches"]
    res["frames"] = steps * S
    res["bpp"] = 8.0 * float(sum(lens)) / (len(lens) * H * W) if lens else None
    res["kernel_ms"] = {f"{k['name']}" + (f"[{k['level']}]" if k["level"] >= 0 else ""): round(k["total_ms"] / profile_steps, 4)
                        for k in kt}
    return res


def run_serving(F, wl, rate_fps: float, duration_s: float, burst_per_stream: int, seed: int = 7):
    """Serving through the public API with the scheduler thread: 64 streams
    of mixed resolution submit frames from pinned host memory, (1) as Poisson
    processes with `rate_fps` frames/s in aggregate for `duration_s`, then
    (2) as a burst: every stream submits `burst_per_stream` frames at once.
    Results are fetched as they complete.  Returns frames/s and latency
    percentiles (submit -> result ready) of each phase."""
    import numpy as np
    import torch

    from synth import sequence_u16
    rng = np.random.default_rng(seed)
    S, nf, bd = wl["streams"], wl["frames"], wl["bit_depth"]
    sizes = [wl["sizes"][s // (S // len(wl["sizes"]))] for s in range(S)]
    host = []
    for s in range(S):
        h, w = sizes[s]
        fr = sequence_u16(wl["seed_base"] + s, nf, h, w, max(8, wl["blobs"] * h * w // (2048 * 2048)), device="cuda")
        host.append([fr[i].cpu().pin_memory() for i in range(nf)])
    torch.cuda.synchronize()
    cfg = dict(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"],
               precision=wl["precision"], max_batch_frames=64, result_ring=8, device=torch.cuda.current_device())
    out = {}
    masks = {sz: torch.empty(sz, dtype=torch.uint8).pin_memory() for sz in set(sizes)}
    coefs = {sz: torch.empty(sz, dtype=torch.int32).pin_memory() for sz in set(sizes)}
    with F.Context(**cfg, **tile_kw()) as ctx:
        nxt = [0] * S
        pending = []  # (stream, frame index)

        def submit_one(s):
            i = nxt[s]
            submit(F, ctx.h, s, host[s][frame_index(i, nf)], i, bd)
            pending.append((s, i))
            nxt[s] += 1

        def drain(block: bool):
            keep = []
            for s, i in pending:
                sz = sizes[s]
                try:
                    F.flowroi_get_mask(ctx.h, s, i, masks[sz], -1 if block else 0)
                    F.flowroi_get_coeffs(ctx.h, s, i, coefs[sz], -1)
                except F.FlowRoIError as e:
                    if e.code != F.ETIMEDOUT:
                        raise
                    keep.append((s, i))
            pending[:] = keep

        for s in range(S):  # first frames (no predecessor), not measured
            submit_one(s)
        F.flowroi_flush(ctx.h, -1)
        drain(True)
        for phase in ("poisson", "burst"):
            st0 = F.flowroi_get_stats(ctx.h)
            n0 = st0["frames_done"]
            F.flowroi_reset_stats(ctx.h)
            t0 = time.perf_counter()
            if phase == "poisson":
                arrivals = np.sort(rng.uniform(0.0, duration_s, size=rng.poisson(rate_fps * duration_s)))
                who = rng.integers(0, S, size=arrivals.size)
                for ta, s in zip(arrivals, who):
                    while time.perf_counter() - t0 < ta:
                        drain(False)
                        time.sleep(0.0005)
                    submit_one(int(s))
            else:
                for _ in range(burst_per_stream):
                    for s in range(S):
                        submit_one(s)
            F.flowroi_flush(ctx.h, -1)
            dt = time.perf_counter() - t0
            drain(True)
            st = F.flowroi_get_stats(ctx.h)
            out[phase] = {"frames": st["frames_done"] - n0, "seconds": dt,
                          "frames_per_s": (st["frames_done"] - n0) / dt,
                          "p50_ms": st["lat_p50_ms"], "p99_ms": st["lat_p99_ms"], "batches": st["batches"]}
    return out


def cpu_sample(wl, frames_cpu, budget_s=12.0, crop=512):
    """The oracle (as it stands, single-threaded) on crop pairs of the
    workload (with the codestream workloads, each crop's coefficients also
    coded at the workload's rate); returns (frames/s scaled to full
    frames, seconds, crops)."""
    import numpy as np

    from oracle import oracle as O
    p = O.Params(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"])
    h, w = wl["h"], wl["w"]
    done, t0, k = 0, time.perf_counter(), 0
    while True:
        s = k % len(frames_cpu)
        a, b = frames_cpu[s]
        y0 = (k * 389) % (h - crop + 1) // 32 * 32
        x0 = (k * 613) % (w - crop + 1) // 32 * 32
        o = O.frame(np.ascontiguousarray(a[y0:y0 + crop, x0:x0 + crop]),
                    np.ascontiguousarray(b[y0:y0 + crop, x0:x0 + crop]), wl["bit_depth"], p)
        if "codestream_bpp" in wl:
            O.encode_frame(o["coeffs"], wl["dwt_levels"], wl["wavelet"], p.scale_shift, wl["bit_depth"],
                           int(wl["codestream_bpp"] * crop * crop / 8), reset=bool(wl.get("codestream_reset", 0)))
        done += 1
        k += 1
        el = time.perf_counter() - t0
        if el >= budget_s and done >= 2:
            break
    px_per_s = done * crop * crop / el
    return px_per_s / (h * w), el, done


def cpu_full_frames(wl, frames_cpu, n=1):
    """The oracle (single-threaded) on n whole frame pairs of the workload
    (no crop, no scaling); returns (frames/s, seconds)."""
    import numpy as np

    from oracle import oracle as O
    p = O.Params(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"])
    t0 = time.perf_counter()
    for k in range(n):
        a, b = frames_cpu[k % len(frames_cpu)]
        O.frame(np.ascontiguousarray(a), np.ascontiguousarray(b), wl["bit_depth"], p)
    el = time.perf_counter() - t0
    return n / el, el


def _cpu_worker(job):
    """One process of the all-cores oracle sample: the oracle on its crop
    pairs, round robin, for budget_s seconds (at least one crop)."""
    crops, wl, budget_s = job
    from oracle import oracle as O
    p = O.Params(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"])
    done, t0 = 0, time.perf_counter()
    while True:
        a, b = crops[done % len(crops)]
        o = O.frame(a, b, wl["bit_depth"], p)
        if "codestream_bpp" in wl:
            O.encode_frame(o["coeffs"], wl["dwt_levels"], wl["wavelet"], p.scale_shift, wl["bit_depth"],
                           int(wl["codestream_bpp"] * a.shape[0] * a.shape[1] / 8),
                           reset=bool(wl.get("codestream_reset", 0)))
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            return done, el


def _cpu_proc(i, job, q):
    try:
        q.put((i, _cpu_worker(job)))
    except Exception as e:  # reported to the parent, which gives up on the sample
        q.put((i, f"{type(e).__name__}: {e}"))


def cpu_sample_parallel(wl, frames_cpu, procs=None, budget_s=8.0, crop=512, per_proc=2):
    """The oracle (as it stands) on every host core: one process per core
    (spawned, never forked from a process that holds a CUDA context), each
    coding its own crop pairs of the workload one frame at a time.  Returns
    (frames/s scaled to full frames = the sum of the processes' rates,
    processes, crops done, seconds)."""
    import multiprocessing as mp
    import queue

    import numpy as np
    procs = procs or os.cpu_count() or 1
    h, w = wl["h"], wl["w"]
    jobs = []
    for pi in range(procs):
        crops = []
        for j in range(per_proc):
            k = pi * per_proc + j
            a, b = frames_cpu[k % len(frames_cpu)]
            y0 = (k * 389) % (h - crop + 1) // 32 * 32
            x0 = (k * 613) % (w - crop + 1) // 32 * 32
            crops.append((np.ascontiguousarray(a[y0:y0 + crop, x0:x0 + crop]),
                          np.ascontiguousarray(b[y0:y0 + crop, x0:x0 + crop])))
        jobs.append((crops, wl, budget_s))
    # plain processes and a queue: a worker that fails or dies ends the
    # sample with an exception, and none outlives the deadline
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_cpu_proc, args=(i, j, q), daemon=True) for i, j in enumerate(jobs)]
    for p in ps:
        p.start()
    out = {}
    deadline = time.monotonic() + 4 * budget_s + 120
    try:
        while len(out) < len(ps):
            try:
                i, r = q.get(timeout=1.0)
            except queue.Empty:
                dead = [k for k, p in enumerate(ps) if k not in out and p.exitcode not in (None, 0)]
                if dead:
                    raise RuntimeError(f"oracle process {dead[0]} exited with {ps[dead[0]].exitcode}")
                if time.monotonic() > deadline:
                    raise TimeoutError("oracle processes did not finish")
                continue
            if isinstance(r, str):
                raise RuntimeError(r)
            out[i] = r
    finally:
        for p in ps:
            p.join(timeout=5)
            if p.is_alive():
                p.terminate()
                p.join(timeout=5)
    res = [out[i] for i in range(len(ps))]
    px_per_s = sum(d * crop * crop / el for d, el in res)
    return px_per_s / (h * w), procs, sum(d for d, _ in res), max(el for _, el in res)


def cpu_parallel_line(wl, fc):
    fps, procs, n, el = cpu_sample_parallel(wl, fc)
    return {"value": fps, "unit": "frames/s", "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes, one per host core, each on its own 512x512 crop pairs of the workload's "
                      f"first frame pairs for {el:.1f} s ({n} crops in all); the sum of their rates, scaled to "
                      f"{wl['w']}x{wl['h']} frames by pixel count"}


def reference_arm(args, wl, ws, rank):
    """The oracle as the reference implementation (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    from oracle import oracle as O
    from synth import sequence_u16
    crop = 256
    seqs = [sequence_u16(wl["seed_base"] + s, 2, wl["h"], wl["w"], wl["blobs"], device="cpu")
            for s in range(min(2, wl["streams"]))]
    pairs = [(q[0].numpy().view(np.uint16), q[1].numpy().view(np.uint16)) for q in seqs]
    p = O.Params(pyr_levels=wl["pyr_levels"], dwt_levels=wl["dwt_levels"], wavelet=wl["wavelet"])

    def step(k):
        a, b = pairs[k % len(pairs)]
        y0 = (k * 389) % (wl["h"] - crop + 1) // 32 * 32
        x0 = (k * 613) % (wl["w"] - crop + 1) // 32 * 32
        O.frame(np.ascontiguousarray(a[y0:y0 + crop, x0:x0 + crop]), np.ascontiguousarray(b[y0:y0 + crop, x0:x0 + crop]),
                wl["bit_depth"], p)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    fps = args.steps * crop * crop / dt / (wl["h"] * wl["w"])
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args.workload, wl),
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} crops of {crop}x{crop} from the workload's frame pairs, "
                                       f"time scaled to {wl['w']}x{wl['h']} frames by pixel count"},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(name, wl):
    return {"workload": name, "streams": wl["streams"], "frame": f"{wl['w']}x{wl['h']} u16 ({wl['bit_depth']}-bit)",
            "frames_per_stream": wl["frames"], "blobs": wl["blobs"], "batch_frames": wl["streams"],
            "pyr_levels": wl["pyr_levels"], "dwt": f"{wl['wavelet'] // 10}/{wl['wavelet'] % 10} x{wl['dwt_levels']}",
            "storage": "fp16" if wl["precision"] == 16 else "fp32", "denoise": bool(wl.get("denoise", 0)),
            "min_area": wl.get("min_area", 0), "register": bool(wl.get("register_frames", 0)),
            "l2": "inputs larger than L2 (each step touches ~2.5 GB of frames and fields)", "tiles": tiles_desc()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="batched_16x2048", choices=sorted(WORKLOADS))
    ap.add_argument("--tiles", default="default",
                    help="tile table JSON for every context: a path, 'none' (built-in shapes) or 'default' "
                         "(the committed table for the workload's storage type, if any)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--serving-rate", type=float, default=8.0,
                    help="serving workload: aggregate Poisson arrival rate, frames/s (8 = 64 wells x 1 frame / 8 s)")
    ap.add_argument("--serving-seconds", type=float, default=20.0)
    ap.add_argument("--burst", type=int, default=4, help="serving workload: frames per stream in the burst replay")
    args = ap.parse_args()
    if not 1 <= args.burst <= 8:
        ap.error("--burst must be in [1, 8]: the serving context keeps 8 results per stream")
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]
    global TILE_TABLE
    if args.tiles == "default":
        TILE_TABLE = default_tiles(wl["precision"])
    elif args.tiles != "none":
        TILE_TABLE = os.path.abspath(args.tiles)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, wl, ws, rank)
        return

    import torch
    import torch.distributed as dist

    from paper_2511_14419_gb300 import build
    from paper_2511_14419_gb300 import flowroi as F
    build()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    # this rank's streams: stream -> device routing (one device per rank)
    wl = dict(wl, sids=rank_streams(F.flowroi_route, wl["streams"], ws, rank))
    if "sizes" in wl:
        # serving measurement: its own JSON line (rank 0), not the throughput line
        res = run_serving(F, wl, args.serving_rate, args.serving_seconds, args.burst)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "workload": args.workload, "n_gpus": ws, "data": "synthetic",
                              "streams": wl["streams"], "sizes": wl["sizes"],
                              "poisson_rate_fps": args.serving_rate, "poisson_seconds": args.serving_seconds,
                              "burst_frames_per_stream": args.burst, "tiles": tiles_desc(), "phases": res}), flush=True)
        return
    frames = make_frames(wl, f"cuda:{local}")
    if "codestream_bpp" in wl:
        # pipeline + codestream measurement: its own JSON line (rank 0)
        torch.cuda.synchronize()
        cr = run_codestream(F, wl, frames, args.steps, args.warmup)
        t_max = max_over_ranks(cr["time_s"], ws, "cpu")
        cpu = cpu_all = None
        if rank == 0 and ws == 1 and not args.no_cpu:
            import numpy as np
            fc = [(frames[s][0].cpu().numpy().view(np.uint16), frames[s][1].cpu().numpy().view(np.uint16))
                  for s in range(min(2, wl["streams"]))]
            fps_cpu, el, nc = cpu_sample(wl, fc)
            cpu = {"value": fps_cpu, "unit": "frames/s", "cores": 1, "kind": "oracle",
                   "sample": f"{nc} crops of 512x512 from the workload's first frame pairs, flow to codestream "
                             f"({el:.1f} s), time scaled to {wl['w']}x{wl['h']} frames by pixel count"}
            try:
                cpu_all = cpu_parallel_line(wl, fc)
            except Exception as e:  # the single-threaded figure stands on its own
                cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}
        if rank == 0:
            print(json.dumps({"metric": "frames/s (flow+mask+DWT+codestream) at 1 GB300", "workload": args.workload,
                              "value": job_throughput(cr["frames"], ws, t_max), "unit": "frames/s", "n_gpus": ws,
                              "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": 1e3 * t_max / args.steps,
                              "codestream_ms_per_step": cr["kernel_ms"].get("codestream"),
                              "codestream_target_bpp": wl["codestream_bpp"], "codestream_bpp": cr["bpp"],
                              "codestream_contexts": "reset at every pass" if wl.get("codestream_reset")
                              else "carried from pass to pass",
                              "kernel_avg_ms": cr["kernel_ms"],
                              "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
                              "config": config_of(args.workload, wl), "cpu_baseline": cpu,
                              "cpu_baseline_all_cores": cpu_all}), flush=True)
        return

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    dev_name = f"cuda:{local}" if ws > 1 and dist.get_backend() == "nccl" else "cpu"

    barrier()
    dev = run_device(F, wl, frames, args.steps, args.warmup, profile_steps=min(args.steps, 10), sampler_device=local)
    barrier()
    t_max = max_over_ranks(dev["time_s"], ws, dev_name)
    value = job_throughput(dev["frames"], ws, t_max)

    plain = None
    if not args.no_plain:
        ps = max(3, min(args.steps, 20))
        pr = run_device(F, wl, frames, ps, args.warmup, plain=True)
        barrier()
        plain = job_throughput(pr["frames"], ws, max_over_ranks(pr["time_s"], ws, dev_name))

    e2e = None
    if not args.no_e2e:
        es = max(3, min(args.steps, 200))
        er = run_e2e(F, wl, frames, es, args.warmup)
        barrier()
        e2e = {"value": job_throughput(er["frames"], ws, max_over_ranks(er["time_s"], ws, dev_name)), "unit": "frames/s",
               "h2d_bytes_per_step": er["h2d"], "d2h_bytes_per_step": er["d2h"]}
        latency = {"p50_ms": er["stats"]["lat_p50_ms"], "p99_ms": er["stats"]["lat_p99_ms"],
                   "source": "e2e run, submit -> result ready"}
    else:
        latency = None

    # roofline of the dominant kernel (by share of the step): the level-0
    # launches of the two displacement kernels
    peak, peak_kind = peaks()
    kt = dev.get("kernel_times") or []
    tot = sum(k["total_ms"] for k in kt) or 1.0
    px = wl["h"] * wl["w"] * wl["streams"]
    roofs = []
    for name in ("update", "window"):
        l0 = [k for k in kt if k["name"] == name and k["level"] == 0]
        if not l0:
            continue
        b_first, b_rest = KERNEL_BYTES[(name, wl["precision"])]
        byts = sum((b_first if k["iter"] == 0 else b_rest) * px * k["launches"] for k in l0)
        ms = sum(k["total_ms"] for k in l0)
        nl = sum(k["launches"] for k in l0)
        achieved = byts / (ms / 1e3) / 1e9
        tr = traffic_per_px(name, wl["precision"])
        roofs.append({"kernel": f"k_{name} level 0", "bound": "hbm", "achieved": achieved, "peak": peak,
                      "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"of {peak_kind}",
                      "traffic": (tr * px) if tr else None, "algorithmic_bytes_per_launch": byts / nl,
                      "avg_launch_ms": ms / nl, "share_of_step": ms / tot})
    for name, level, label in (("dwt", 1, "k_dwt level 1"), ("expand", 0, "k_expand level 0")):
        ks = [k for k in kt if k["name"] == name and k["level"] == level]
        if not ks:
            continue
        ms = sum(k["total_ms"] for k in ks)
        nl = sum(k["launches"] for k in ks)
        byts = other_bytes(name, wl["precision"], 2) * px
        achieved = byts / (ms / nl / 1e3) / 1e9
        tr = traffic_per_px(name, wl["precision"])
        roofs.append({"kernel": label, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                      "frac": achieved / peak, "peak_kind": f"of {peak_kind}", "traffic": (tr * px) if tr else None,
                      "algorithmic_bytes_per_launch": byts, "avg_launch_ms": ms / nl, "share_of_step": ms / tot})
    roofs.sort(key=lambda r: -r["share_of_step"])
    roof = roofs[0] if roofs else None
    kernels = {}
    for k in kt:
        key = k["name"] + ("" if k["level"] < 0 else f"[{k['level']}]")
        kernels[key] = round(kernels.get(key, 0.0) + k["total_ms"] / max(1, k["launches"]), 4)

    cpu = cpu_all = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import numpy as np
        fc = [(frames[s][0].cpu().numpy().view(np.uint16), frames[s][1].cpu().numpy().view(np.uint16))
              for s in range(min(2, wl["streams"]))]
        fps_cpu, el, nc = cpu_sample(wl, fc)
        cpu = {"value": fps_cpu, "unit": "frames/s", "cores": 1, "kind": "oracle",
               "sample": f"{nc} crops of 512x512 from the workload's first frame pairs ({el:.1f} s), "
                         f"time scaled to {wl['w']}x{wl['h']} frames by pixel count; host has {os.cpu_count()} cores"}
        try:
            cpu_all = cpu_parallel_line(wl, fc)
        except Exception as e:  # the single-threaded figure stands on its own
            cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}
        ff, fel = cpu_full_frames(wl, fc, 1)
        cpu_full = {"value": ff, "unit": "frames/s", "cores": 1, "kind": "oracle",
                    "sample": f"1 whole {wl['w']}x{wl['h']} frame pair of the workload ({fel:.1f} s), no crop, no scaling"}
    else:
        cpu_full = None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(args.workload, wl), "e2e": e2e, "gpu_launches": dev["launches"],
                "plain_fps": plain, "latency": latency, "clocks": dev.get("clocks"), "roofline": roof,
                "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "cpu_baseline_full_frame": cpu_full,
                "kernel_avg_ms": kernels,
                "roofline_other": roofs[1:]}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
