#!/usr/bin/env python
"""Throughput benchmark of the plain detector path on GB300.

One step = the whole hot path (pyramid, LBP+HOG cell histograms, block
normalisation + window scores, NMS) over one batch of 2048 synthetic 1242x375
frames (the paper's frame size; pyramid factor 1.05 -> 23 levels, 33,428
windows per frame), replayed as one CUDA graph; 20 steps take about 1.2 s.
Frames are resident in HBM when the timed region starts; L2 is flushed (256 MB
write) before every timed step and each step is timed with CUDA events on the
detector's stream. Secondary lines (other pipelines, kernels, pyramids, the
proposal, C1 latency, the C3 mixed batch) run their own batches.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. Under torchrun (N > 1) every rank runs an independent
replica on its own frames (frames are independent: weak scaling, no
collective on the data path); the step time is the max over ranks.
`--impl reference` times the CPU oracle (test infrastructure) on the host.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WIDTH, HEIGHT = 1242, 375
FACTOR = float(np.float32(1.05))
CFG_ID = 2                      # scene recipe of the 1242x375 workload
FLOP_PER_WINDOW = 2 * 15 * 7 * 95   # 9,975 FMA
# Algorithmic operations per pixel of a level's cell grid (HOG + LBP cells, Algorithms 1, 4, 5):
# LBP 18 (8 compares, 8 code shifts/ors, bin lookup, count), HOG 37 (gradient 2, magnitude 4,
# orientation 1 atan2 + 2, orientation interpolation 4, spatial weights 4, 8 weighted votes 16,
# vote weights 4).
OPS_PER_CELL_PIXEL = 55
# Tensor-core K4 MMA per block row of a strip: M 128 x N 112 x K 288 (bf16 high/low split)
TC_FLOP_PER_UNIT = 2 * 128 * 112 * 288
PAPER_FPS_1242x375 = 20.0       # Tegra X1, HOGLBP-SVM (context: another machine)
L2_FLUSH_BYTES = 256 << 20
METRIC = "frames/s (1242x375, HOG+LBP+SVM+NMS)"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--frames-per-step", type=int, default=2048)
    ap.add_argument("--side-frames", type=int, default=64,
                    help="frames per step of the secondary lines (other kernels, pipelines, pyramids)")
    ap.add_argument("--cpu-sample-frames", type=int, default=4,
                    help="frames the single-threaded CPU oracle times for cpu_baseline (bounded sample); "
                         "the all-cores figure times 2 frames per core")
    ap.add_argument("--c1-replays", type=int, default=200,
                    help="timed single-frame detects of the 320x240 latency config (0: skip)")
    ap.add_argument("--c3-steps", type=int, default=10,
                    help="timed steps of the 64-frame mixed batch (0: skip)")
    ap.add_argument("--proposal-steps", type=int, default=10,
                    help="timed steps of the 16x1920x1080 plain-vs-sparse comparison (0: skip)")
    ap.add_argument("--svm", default="tc", choices=["tc", "fp32"],
                    help="window-score kernel: tensor cores (default) or the FP32 CUDA-core kernel")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default tile costs of the FP32 kernel (profiler captures)")
    ap.add_argument("--proposal-4k", type=int, default=1,
                    help="also compare plain and sparse on the 4K mix (16 x 3840x2160 + 48 x 1242x375)")
    ap.add_argument("--proposal-frames", type=int, default=16,
                    help="frames of the proposal comparison (16 is the workload; fewer for profiler captures)")
    ap.add_argument("--scheme-reps", type=int, default=5,
                    help="timed calls per kernel scheme and size in the px/ns sweep (0: skip the sweep)")
    ap.add_argument("--pipeline-steps", type=int, default=10,
                    help="timed steps of the HOG-SVM and LBP-SVM pipelines on the same batch (0: skip)")
    ap.add_argument("--other-k4-steps", type=int, default=10,
                    help="timed steps of the same batch with the other window-score kernel (0: skip)")
    ap.add_argument("--upscale-steps", type=int, default=10,
                    help="timed steps of the same batch with 17 upsampled levels (40 levels per frame; 0: skip)")
    ap.add_argument("--hog-per-block", action="store_true",
                    help="main step with per-block HOG (Algorithm 5 read per 16x16 block; tensor-core K4 only)")
    args = ap.parse_args(argv)
    if args.hog_per_block and args.svm == "fp32":
        ap.error("--hog-per-block needs the tensor-core K4 (--svm tc)")
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_frame_indices(rank: int, frames_per_rank: int):
    """Frames of a rank's replica: disjoint seeded scenes per rank."""
    return list(range(rank * frames_per_rank, (rank + 1) * frames_per_rank))


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a per-rank scalar over all ranks (host logic; gloo or nccl)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _scene_worker(spec):
    import synth
    return synth.make_scene(*spec)


_ORACLE_T = None


def _oracle_init():
    global _ORACLE_T
    import oracle
    oracle.build()
    _ORACLE_T = load_template()


def _oracle_worker(img):
    import oracle
    w, b = _ORACLE_T
    oracle.detect(img, w, b, FACTOR)
    return 0


def make_pool(cores: int, oracle_workers: bool = False):
    """A process pool started with spawn (safe next to CUDA)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    return ctx.Pool(cores, initializer=_oracle_init if oracle_workers else None)


def time_oracle_parallel(pool, cores: int, frames) -> float:
    """Wall time of the oracle over `frames` on `cores` worker processes (one frame per task)."""
    pool.map(_oracle_worker, frames[:cores], chunksize=1)  # warm: library loaded in every worker
    t0 = time.perf_counter()
    pool.map(_oracle_worker, frames, chunksize=1)
    return time.perf_counter() - t0


def load_template():
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    return d["w"], float(d["b"])


def make_frames(indices, pool=None):
    specs = [(WIDTH, HEIGHT, CFG_ID, i) for i in indices]
    if pool is not None:
        return pool.map(_scene_worker, specs, chunksize=8)
    return [_scene_worker(sp) for sp in specs]


def svm_flag(args, pd) -> int:
    return pd.PD_FLAG_SVM_FP32 if args.svm == "fp32" else 0


def main_flags(args, pd) -> int:
    """Flags of the main step's detectors: the K4 kernel, and per-block HOG if asked for."""
    return svm_flag(args, pd) | (pd.PD_FLAG_HOG_PER_BLOCK if args.hog_per_block else 0)


def cells_per_frame() -> int:
    from paper_1611_01642_gb300 import pd_pyramid
    return sum((wk // 8) * (hk // 8) for wk, hk in pd_pyramid(WIDTH, HEIGHT, FACTOR))


def tc_units_per_frame() -> int:
    """Block rows the tensor-core K4 walks per frame: strips of 104 window columns, each cut into
    pieces of at most 64 window rows, each piece also walking the 14 block rows below it."""
    from paper_1611_01642_gb300 import pd_pyramid
    n = 0
    for wk, hk in pd_pyramid(WIDTH, HEIGHT, FACTOR):
        rows, cols = hk // 8 - 15, wk // 8 - 7
        if rows <= 0 or cols <= 0:
            continue
        pieces = -(-rows // 64)
        n += -(-cols // 104) * (rows + 14 * pieces)
    return n


def windows_per_frame(upscale: int = 0) -> int:
    from paper_1611_01642_gb300 import pd_pyramid
    return sum(max(hk // 8 - 15, 0) * max(wk // 8 - 7, 0)
               for wk, hk in pd_pyramid(WIDTH, HEIGHT, FACTOR, upscale_levels=upscale))


UPSCALE_LEVELS = 17     # 1242x375 at f = 1.05: 17 upsampled + 23 downsampled = 40 levels
# (with the upsampled levels a frame of this scene recipe has up to ~20,000 windows
# scoring above 0: the NMS takes up to 65,536 candidates per frame)


def run_upscaled(args, pd, torch, frames, flush, tile_costs, fp32_peak):
    """The same batch with the 17 upsampled levels in front of the 23 (40 levels per frame), under
    the main line's timing rules. A secondary figure: the headline line is the 23-level pyramid."""
    w, b = load_template()
    det = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=len(frames), max_width=WIDTH, max_height=HEIGHT,
                      upscale_levels=UPSCALE_LEVELS, max_candidates_per_frame=65536,
                      flags=pd.PD_FLAG_STAGE_TIMING | svm_flag(args, pd))
    pd.pd_set_tile_costs(det.h, tile_costs)
    ms, st = time_detector(det, frames, flush, args.upscale_steps, pd, torch)
    n_levels = len(det.levels(0))
    det.close()
    wpf = windows_per_frame(UPSCALE_LEVELS)
    k4 = len(frames) * wpf * FLOP_PER_WINDOW / (st[2] / 1e3) / 1e12
    return {"workload": f"{len(frames)} x {WIDTH}x{HEIGHT} u8 frames, pyramid factor 1.05 with "
                        f"{UPSCALE_LEVELS} upsampled levels ({n_levels} levels), plain HOG+LBP+SVM+NMS "
                        "(NMS candidate cap 65,536 per frame)",
            "frames_per_s": len(frames) / (ms / 1e3), "ms_per_step": ms, "levels_per_frame": n_levels,
            "windows_per_frame": wpf, "k4_algorithmic_tflops": k4,
            "stage_ms_per_step": dict(zip(["pyramid", "cells", "norm_svm", "nms"], map(float, st[:4]))),
            "steps": args.upscale_steps}


def time_detector(det, frames, flush, steps, pd, torch, warmup: int = 3):
    """Mean step time (CUDA events on the current stream, L2 flushed before every step) and mean
    per-stage times of `steps` detects of `frames` after `warmup` untimed ones."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.fill_(1)
        det.detect(frames)
        det.sync()
    tot, st = 0.0, np.zeros(5)
    for i in range(steps):
        flush.fill_(i & 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        det.detect(frames)
        e1.record(stream)
        if det.sync() != pd.PD_OK:
            raise RuntimeError(pd.pd_last_error(det.h))
        tot += e0.elapsed_time(e1)
        st += np.array(pd.pd_stage_times(det.h))
    return tot / steps, st / steps


def run_other_k4(args, pd, torch, frames, flush, w, b, fp32_peak, bf16_peak):
    """The same batch with the other window-score kernel (FP32 CUDA cores when the main line runs
    the tensor cores, and the reverse), so that one bench line carries both."""
    from paper_1611_01642_gb300 import autotune
    other = "fp32" if args.svm != "fp32" else "tc"
    flags = pd.PD_FLAG_STAGE_TIMING | (pd.PD_FLAG_SVM_FP32 if other == "fp32" else 0)
    det = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=len(frames), max_width=WIDTH, max_height=HEIGHT,
                      flags=flags)
    try:
        costs = (autotune.apply(det, frames[:16], w, b, FACTOR)
                 if other == "fp32" and not args.no_autotune else pd.pd_get_tile_costs(det.h))
        ms, st = time_detector(det, frames, flush, args.other_k4_steps, pd, torch)
    finally:
        det.close()
    k4 = len(frames) * windows_per_frame() * FLOP_PER_WINDOW / (st[2] / 1e3) / 1e12
    peak = fp32_peak if other == "fp32" else bf16_peak
    return {"kernel": "k_svm (FP32 CUDA cores, PD_FLAG_SVM_FP32)" if other == "fp32"
                      else "k_svm_tc (tensor cores)",
            "frames_per_s": len(frames) / (ms / 1e3), "ms_per_step": ms, "k4_ms": float(st[2]),
            "k4_algorithmic_tflops": k4, "k4_frac_of_peak": k4 / peak,
            "peak": peak, "tile_costs": [round(c, 4) for c in costs] if other == "fp32" else None,
            "steps": args.other_k4_steps}


def run_pipelines(args, pd, torch, frames, flush, w, b):
    """The paper's other two pipelines (Section 4.1) on the same batch: HOG-SVM and LBP-SVM (only
    that feature's cells computed; windows scored with that feature's weights); and HOGLBP-SVM with
    per-block HOG (Algorithm 5 read per 16x16 block: 36 HOG planes per cell, tensor-core K4)."""
    out = {}
    per_block = [("hoglbp_svm_per_block_hog", pd.PD_FLAG_HOG_PER_BLOCK)] if svm_flag(args, pd) == 0 else []
    for name, flag in [("hog_svm", pd.PD_FLAG_HOG_ONLY), ("lbp_svm", pd.PD_FLAG_LBP_ONLY)] + per_block:
        det = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=len(frames), max_width=WIDTH, max_height=HEIGHT,
                          flags=pd.PD_FLAG_STAGE_TIMING | flag | svm_flag(args, pd))
        try:
            ms, st = time_detector(det, frames, flush, args.pipeline_steps, pd, torch)
        finally:
            det.close()
        out[name] = {"frames_per_s": len(frames) / (ms / 1e3), "ms_per_step": ms,
                     "stage_ms_per_step": dict(zip(["pyramid", "cells", "norm_svm", "nms"], map(float, st[:4])))}
    out["steps"] = args.pipeline_steps
    return out


SCHEME_SIZES = [(320, 240), (640, 480), (1280, 720), (1920, 1080), (3840, 2160)]


def run_schemes(args, pd, torch, w, b):
    """px/ns of the paper's kernel schemes and of the fused kernels on single levels of growing size
    (Section 5.3's per-algorithm comparison): cells (LBP / HOG) from a level image, window scores
    from cell planes. Each figure: the median of `--scheme-reps` calls timed with CUDA events."""
    import synth
    stream = torch.cuda.current_stream()
    det = pd.Detector(w, b, max_frames=1, max_width=SCHEME_SIZES[-1][0], max_height=SCHEME_SIZES[-1][1],
                      flags=svm_flag(args, pd))

    def timed(fn):
        fn()
        ms = []
        for _ in range(args.scheme_reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    names = ["lbp_naive", "lbp_scalable", "hog_global", "hog_local", "hog_shared", "cells_fused",
             "svm_naive", "svm_warp", "svm_fused", "hog_block_global", "hog_block_local", "hog_block_shared",
             "cells_fused_per_block", "svm_fused_per_block"]
    out = {n: [] for n in names}
    det_pb = pd.Detector(w, b, max_frames=1, max_width=SCHEME_SIZES[-1][0], max_height=SCHEME_SIZES[-1][1],
                         flags=pd.PD_FLAG_HOG_PER_BLOCK)
    try:
        for W, H in SCHEME_SIZES:
            L = torch.from_numpy(synth.random_image(W, H, W + H, smooth=True)).cuda()
            Hc, Wc = H // 8, W // 8
            cp = max(16, -(-Wc // 16) * 16)
            plane = Hc * cp
            hog = torch.zeros((9 * plane,), dtype=torch.float32, device="cuda")
            lbp = torch.zeros((59 * plane,), dtype=torch.uint8, device="cuda")
            scores = torch.zeros((max((Hc - 15) * (Wc - 7), 1),), dtype=torch.float32, device="cuda")
            px = W * H
            for n, sch in (("lbp_naive", pd.PD_SCHEME_LBP_NAIVE), ("lbp_scalable", pd.PD_SCHEME_LBP_SCALABLE)):
                out[n].append(px / (timed(lambda: pd.pd_scheme_cells(det.h, sch, L, None, 0, lbp, plane, cp)) * 1e6))
            for n, sch in (("hog_global", pd.PD_SCHEME_HOG_GLOBAL), ("hog_local", pd.PD_SCHEME_HOG_LOCAL),
                           ("hog_shared", pd.PD_SCHEME_HOG_SHARED)):
                out[n].append(px / (timed(lambda: pd.pd_scheme_cells(det.h, sch, L, hog, plane, None, 0, cp)) * 1e6))
            out["cells_fused"].append(
                px / (timed(lambda: pd.pd_cell_features(det.h, L, hog, plane, lbp, plane, cp)) * 1e6))
            for n, sch in (("svm_naive", pd.PD_SCHEME_SVM_NAIVE), ("svm_warp", pd.PD_SCHEME_SVM_WARP)):
                out[n].append(px / (timed(lambda: pd.pd_scheme_window_scores(
                    det.h, sch, hog, plane, lbp, plane, cp, Wc, Hc, scores)) * 1e6))
            out["svm_fused"].append(px / (timed(lambda: pd.pd_window_scores(
                det.h, hog, plane, lbp, plane, cp, Wc, Hc, scores)) * 1e6))
            # per-block HOG (Algorithm 5 read per block): thread-per-block schemes, fused kernels
            hog36 = torch.zeros((36 * plane,), dtype=torch.float32, device="cuda")
            for n, sch in (("hog_block_global", pd.PD_SCHEME_HOG_GLOBAL), ("hog_block_local", pd.PD_SCHEME_HOG_LOCAL),
                           ("hog_block_shared", pd.PD_SCHEME_HOG_SHARED)):
                out[n].append(px / (timed(lambda: pd.pd_scheme_cells(det_pb.h, sch, L, hog36, plane, None, 0, cp))
                                    * 1e6))
            out["cells_fused_per_block"].append(
                px / (timed(lambda: pd.pd_cell_features(det_pb.h, L, hog36, plane, lbp, plane, cp)) * 1e6))
            out["svm_fused_per_block"].append(px / (timed(lambda: pd.pd_window_scores(
                det_pb.h, hog36, plane, lbp, plane, cp, Wc, Hc, scores)) * 1e6))
    finally:
        det.close()
        det_pb.close()
    return {"unit": "px/ns", "sizes": [f"{W}x{H}" for W, H in SCHEME_SIZES], "reps": args.scheme_reps,
            "note": "cells_fused computes LBP and HOG together; svm_fused is the K4 the line runs; "
                    "*_per_block: per-block HOG (36 HOG planes per cell; tensor-core K4)", **out}


def hbm_per_kernel(stage_ms, svm: str, frames: int):
    """Achieved HBM GB/s of each kernel of the step: the DRAM bytes of one launch recorded by ncu
    (committed summary of a 64-frame batch, scaled to `frames`; only for kernels whose source is
    unchanged since the capture) over the kernel's CUDA-event time in this run."""
    path = os.path.join(ROOT, "profiles", "dram_per_kernel_1242x375_b64.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            if line.startswith("@"):
                k, v = line[1:].split("=", 1)
                name, src, nbytes = v.split()
                rec[k.strip()] = (name, src, float(nbytes))
    peak = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    out = {}
    for kernel, t in zip(["k_resize", "k_cells", "k_svm_tc" if svm != "fp32" else "k_svm", "k_nms"], stage_ms):
        if kernel not in rec:
            continue
        name, src_hash, nbytes = rec[kernel]
        if _file_hash(os.path.join(ROOT, "paper_1611_01642_gb300", "csrc", name)) != src_hash:
            out[kernel] = None
            continue
        nbytes *= frames / 64.0
        gbs = nbytes / (t / 1e3) / 1e9
        out[kernel] = {"dram_bytes": nbytes, "achieved_gbs": gbs, "frac_of_peak": gbs / peak}
    return out


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples (200 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([float(r[1]) for r in rows])
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        loaded = sm[sm >= 0.5 * sm.max()]
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# ----------------------------------------------------------------------------- CPU oracle
def time_oracle(frames, w, b):
    """Single-threaded FP64 oracle over `frames` (the full plain path per frame)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for img in frames:
        oracle.detect(img, w, b, FACTOR)
    return time.perf_counter() - t0


def run_reference(args):
    """The oracle on the host's cores: each step is a bounded sample of the workload, one frame per
    core, detected in parallel by worker processes (one frame each)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    with make_pool(cores, oracle_workers=True) as pool:
        frames = make_frames(range((max(args.warmup, 0) + args.steps) * cores), pool)
        t_warm = time_oracle_parallel(pool, cores, frames[:max(args.warmup, 0) * cores]) if args.warmup > 0 else 0.0
        t = time_oracle_parallel(pool, cores, frames[max(args.warmup, 0) * cores:])
    del t_warm
    n = args.steps * cores
    fps = n / t
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": fps / PAPER_FPS_1242x375, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WIDTH}x{HEIGHT} u8 frames, pyramid factor 1.05 (23 levels), "
                               "plain HOG+LBP+SVM+NMS", "frames_per_step": cores},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "cpu": cpu_model(),
                         "sample": f"{args.steps} steps of {cores} seeded {WIDTH}x{HEIGHT} frames, one frame "
                                   f"per worker process ({cores} processes)"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU
def _file_hash(path: str) -> str:
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def recorded_traffic(profile: str, source: str, key: str = "dram_bytes_per_launch"):
    """DRAM bytes per launch (scaled to the bench's 64-frame batch), or another recorded figure
    (`key`), from a committed ncu summary, if the kernel's source is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", profile)
    src = os.path.join(ROOT, "paper_1611_01642_gb300", "csrc", source)
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            if "=" in line and line.startswith("@"):
                k, v = line[1:].split("=", 1)
                rec[k.strip()] = v.strip()
    if rec.get("source_sha256_16") != _file_hash(src):
        return None
    try:
        return float(rec[key])
    except (KeyError, ValueError):
        return None


def scaled(v, f):
    return None if v is None else v * f


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


PROPOSAL_CKPT = os.path.join(ROOT, "paper_1611_01642_gb300", "weights", "proposal_1920x1080.npz")


def run_proposal(args, pd, torch, flush, recipe: int = 4):
    """Plain vs sparse (learned proposal) path on a batch of synthetic frames: scene recipe 4
    (16 x 1920x1080) or 5 (16 x 3840x2160 + 48 x 1242x375).

    Both paths run the same frames with the same timing rules as the main line (L2 flushed before
    every step, CUDA events on the detector's stream). Recall and keep fraction are counted window
    by window over every level of the batch: recall = |scored on the sparse path and plain score > 0|
    / |plain score > 0|.
    """
    import synth
    from paper_1611_01642_gb300 import proposal as prop
    params, meta = prop.load_checkpoint(PROPOSAL_CKPT)
    tau = float(meta["keep_logit_threshold"])
    step = int(meta.get("level_step", 1))
    imgs = synth.make_frames(recipe, limit=args.proposal_frames if recipe == 4 else None)
    frames = [torch.from_numpy(im).cuda() for im in imgs]
    w, b = load_template()
    det = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=len(frames), max_width=max(im.shape[1] for im in imgs),
                      max_height=max(im.shape[0] for im in imgs), flags=pd.PD_FLAG_STAGE_TIMING | svm_flag(args, pd))
    pd.pd_cnn_set_params(det.h, params)
    stream = torch.cuda.current_stream()

    def timed(sparse: bool):
        det.set_proposal(sparse, tau, level_step=step)
        for _ in range(3):
            flush.fill_(1)
            det.detect(frames)
            det.sync()
        tot, st = 0.0, np.zeros(5)
        for i in range(args.proposal_steps):
            flush.fill_(i & 255)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            det.detect(frames)
            e1.record(stream)
            if det.sync() != pd.PD_OK:
                raise RuntimeError(pd.pd_last_error(det.h))
            tot += e0.elapsed_time(e1)
            st += np.array(pd.pd_stage_times(det.h))
        n = args.proposal_steps
        return tot / n, st / n

    ms_plain, st_plain = timed(False)
    plain_scores = torch.cat([m.reshape(-1) for f in range(len(frames)) for m in det.score_maps(f)]).clone()
    ms_sparse, st_sparse = timed(True)
    sparse_scores = torch.cat([m.reshape(-1) for f in range(len(frames)) for m in det.score_maps(f)])
    logits = torch.cat([m.reshape(-1) for f in range(len(frames)) for m in det.logit_maps(f)])
    scored = ~torch.isneginf(sparse_scores)
    pos = plain_scores > 0
    exact = bool(torch.equal(sparse_scores[scored], plain_scores[scored]))
    det.close()
    names = ["pyramid", "cells", "norm_svm", "nms", "proposal"]
    return {
        "workload": (f"{len(imgs)} x 1920x1080 u8 frames (scene recipe 4: Poisson(10) silhouettes, "
                     "48 px..0.8H), pyramid factor 1.05 (44 levels)") if recipe == 4 else
                    ("16 x 3840x2160 + 48 x 1242x375 u8 frames in one batch (scene recipe 5: Poisson(10) "
                     "silhouettes, 48..600 px), pyramid factor 1.05 (58 / 23 levels)"),
        "checkpoint": os.path.relpath(PROPOSAL_CKPT, ROOT), "keep_logit_threshold": tau,
        "level_step": step,
        "plain_frames_per_s": len(frames) / (ms_plain / 1e3),
        "sparse_frames_per_s": len(frames) / (ms_sparse / 1e3),
        "speedup": ms_plain / ms_sparse,
        "recall": float((pos & scored).sum().item() / max(pos.sum().item(), 1)),
        "keep_fraction": float(scored.float().mean().item()),
        "window_keep_fraction": float((logits > tau).float().mean().item()),
        "proposal_share": float(st_sparse[4] / ms_sparse),
        "scored_windows_equal_plain": exact,
        "stage_ms_plain": dict(zip(names, map(float, st_plain))),
        "stage_ms_sparse": dict(zip(names, map(float, st_sparse))),
        "steps": args.proposal_steps,
    }


def run_c1(args, pd, torch, w, b):
    """C1: one seeded 320x240 frame, pyramid factor 1.2 (4 levels), the latency configuration: the
    median of `--c1-replays` single-frame detects (graph replays), each timed with CUDA events."""
    import synth
    img = synth.make_scene(320, 240, 1, 0)
    f12 = float(np.float32(1.2))
    det = pd.Detector(w, b, pyr_factor=f12, max_frames=1, max_width=320, max_height=240)
    frame = [torch.from_numpy(img).cuda()]
    stream = torch.cuda.current_stream()
    try:
        # launch shapes for this workload (a single small frame: short tensor-core items cut the
        # score kernel's walk), measured by the autotuner like the main line's
        from paper_1611_01642_gb300 import autotune
        tuning = (pd.pd_get_tuning(det.h) if args.no_autotune else
                  autotune.apply_default(det, frame, w, b, f12))
        for _ in range(20):
            det.detect(frame)
            det.sync()
        ms = []
        for _ in range(args.c1_replays):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            det.detect(frame)
            e1.record(stream)
            if det.sync() != pd.PD_OK:
                raise RuntimeError(pd.pd_last_error(det.h))
            ms.append(e0.elapsed_time(e1))
        n_levels = len(det.levels(0))
        boxes = len(det.boxes(0))
    finally:
        det.close()
    med = float(np.median(ms))
    return {"workload": "1 x 320x240 u8 frame (scene recipe 1: 3 silhouettes of 64..128 px), pyramid factor 1.2 "
                        f"({n_levels} levels), plain HOG+LBP+SVM+NMS", "latency_ms_median": med,
            "latency_ms_p10": float(np.percentile(ms, 10)), "latency_ms_p90": float(np.percentile(ms, 90)),
            "frames_per_s": 1e3 / med, "boxes": boxes, "replays": args.c1_replays, "launch_shapes": tuning,
            "timing": "device-resident frame, graph replay, CUDA events per detect (L2 not flushed)"}


def run_c3(args, pd, torch, flush, w, b, pool):
    """C3: the 64-frame mixed batch (32 x 1242x375 + 16 x 640x480 + 16 x 1920x1080, scene recipe 3,
    Poisson(10) silhouettes), pyramid factor 1.05, one graph-replayed step per batch, timed like the
    main line's serial figure."""
    import synth
    imgs = pool.map(_scene_worker, synth.frame_specs(3), chunksize=1)
    frames = [torch.from_numpy(im).cuda() for im in imgs]
    det = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=len(frames), max_width=1920, max_height=1080,
                      flags=pd.PD_FLAG_STAGE_TIMING)
    try:
        # launch shapes picked by the autotuner on this batch (the configuration's "tiles picked
        # by the project's autotuner")
        from paper_1611_01642_gb300 import autotune
        tuning = (pd.pd_get_tuning(det.h) if args.no_autotune else
                  autotune.apply_default(det, frames, w, b, FACTOR))
        ms, st = time_detector(det, frames, flush, args.c3_steps, pd, torch)
        levels = sorted({len(det.levels(f)) for f in range(len(frames))})
    finally:
        det.close()
    px = sum(im.size for im in imgs)
    return {"workload": "64 mixed u8 frames in one batch: 32 x 1242x375 + 16 x 640x480 + 16 x 1920x1080 (scene "
                        f"recipe 3), pyramid factor 1.05 ({'/'.join(map(str, levels))} levels), plain "
                        "HOG+LBP+SVM+NMS",
            "frames_per_s": len(frames) / (ms / 1e3), "ms_per_step": ms, "px_per_ns": px / (ms * 1e6),
            "stage_ms_per_step": dict(zip(["pyramid", "cells", "norm_svm", "nms"], map(float, st[:4]))),
            "steps": args.c3_steps, "launch_shapes": tuning,
            "l2": "flushed (256 MB write) before every timed step"}


def run_gpu(args):
    rank, world, local = dist_env()
    # worker processes (spawn) for the synthetic frames and the CPU oracle, started before CUDA
    cores = host_cores()
    oracle_pool = rank == 0 and world == 1 and args.cpu_sample_frames > 0
    if oracle_pool:
        import oracle
        oracle.build()
    pool = make_pool(max(1, cores // world), oracle_workers=oracle_pool)
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1611_01642_gb300 import build as pkg_build
    pkg_build.build()
    import paper_1611_01642_gb300 as pd

    B = args.frames_per_step
    w, b = load_template()
    imgs = make_frames(rank_frame_indices(rank, B), pool)
    det = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=B, max_width=WIDTH, max_height=HEIGHT,
                      flags=pd.PD_FLAG_STAGE_TIMING | main_flags(args, pd))
    stream = torch.cuda.current_stream()
    frames = [torch.from_numpy(im).cuda() for im in imgs]
    pinned = [torch.from_numpy(im).pin_memory() for im in imgs]
    from paper_1611_01642_gb300 import autotune
    tile_costs = (pd.pd_get_tile_costs(det.h) if args.no_autotune or args.svm != "fp32"
                  else autotune.apply(det, frames[:16], w, b, FACTOR))
    # launch shapes of the default path (pyramid groups per warp task, score-kernel item rows),
    # timed on 64 of the step's frames, cached per GPU, library build and workload
    tuning = (pd.pd_get_tuning(det.h) if args.no_autotune else
              autotune.apply_default(det, frames[:64], w, b, FACTOR, flags=main_flags(args, pd)))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    wpf = windows_per_frame()

    def step():
        det.detect(frames)
        st = det.sync()
        if st != pd.PD_OK:
            raise RuntimeError(f"pd_sync: {pd.ERROR_NAMES.get(st, st)} {pd.pd_last_error(det.h)}")

    for _ in range(max(args.warmup, 0)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    total_ms, stage_ms = 0.0, np.zeros(5)
    launches = 0
    for i in range(args.steps):
        flush.fill_(i & 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        det.detect(frames)
        e1.record(stream)
        st = det.sync()
        if st != pd.PD_OK:
            raise RuntimeError(f"pd_sync: {pd.ERROR_NAMES.get(st, st)} {pd.pd_last_error(det.h)}")
        total_ms += e0.elapsed_time(e1)
        stage_ms += np.array(pd.pd_stage_times(det.h))
        launches += pd.pd_last_launch_count(det.h)
    torch.cuda.synchronize()
    serial_ms = reduce_max(total_ms, world, device="cuda")
    stage_step = stage_ms / args.steps

    # Pipelined: two handles alternate on two streams, so that step i+1's first
    # kernels run on the SMs that step i's last ones (NMS: one CTA per frame)
    # leave idle. K steps in all, timed from one event before the first to the
    # later of the two streams' events after the last; a handle is reused only
    # after its previous step has been synced (its arena holds the results).
    det_b = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=B, max_width=WIDTH, max_height=HEIGHT,
                        flags=pd.PD_FLAG_STAGE_TIMING | main_flags(args, pd))
    pd.pd_set_tile_costs(det_b.h, tile_costs)
    pd.pd_set_tuning(det_b.h, tuning["k1_groups"], tuning["tc_item_rows"])
    streams = [stream, torch.cuda.Stream()]
    pipe = [det, det_b]
    for _ in range(max(args.warmup, 0)):
        for d, s_ in zip(pipe, streams):
            d.detect(frames, stream=s_)
        for d in pipe:
            d.sync()
    barrier(world)
    torch.cuda.synchronize()
    e_start = torch.cuda.Event(enable_timing=True)
    e_start.record(streams[0])
    streams[1].wait_event(e_start)
    launches = 0
    for i in range(args.steps):
        d, s_ = pipe[i & 1], streams[i & 1]
        if i >= 2 and d.sync() != pd.PD_OK:
            raise RuntimeError(f"pd_sync: {pd.pd_last_error(d.h)}")
        with torch.cuda.stream(s_):
            flush.fill_(i & 255)
        d.detect(frames, stream=s_)
        launches += pd.pd_last_launch_count(d.h)
    e_end = [torch.cuda.Event(enable_timing=True) for _ in streams]
    for e, s_ in zip(e_end, streams):
        e.record(s_)
    for d in pipe:
        if d.sync() != pd.PD_OK:
            raise RuntimeError(f"pd_sync: {pd.pd_last_error(d.h)}")
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    pipe_ms = max(e_start.elapsed_time(e) for e in e_end)
    total_ms = reduce_max(pipe_ms, world, device="cuda")
    det_b.close()
    value = world * B * args.steps / (total_ms / 1e3)
    ms_step = total_ms / args.steps

    # end to end through the public API: host frames in, host boxes out. Two
    # handles alternate so that step i's results are read on the host while
    # step i+1 already runs (each step still copies its frames in and its
    # boxes out inside the timed region).
    det2 = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=B, max_width=WIDTH, max_height=HEIGHT,
                       flags=main_flags(args, pd))
    pd.pd_set_tile_costs(det2.h, tile_costs)
    pd.pd_set_tuning(det2.h, tuning["k1_groups"], tuning["tc_item_rows"])
    for _ in range(2):
        det2.detect_host(pinned, stream=streams[1])
        det2.sync()
    dets = [det, det2]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0

    def finish(d):
        st = d.sync()
        if st != pd.PD_OK:
            raise RuntimeError(f"pd_sync: {pd.ERROR_NAMES.get(st, st)}")
        return 8 * B + 4 + sum(32 * len(d.boxes(f)) for f in range(B))

    pending = None
    for i in range(args.steps):
        d = dets[i & 1]
        d.detect_host(pinned, stream=streams[i & 1])
        if pending is not None:
            d2h += finish(pending)
        pending = d
    if pending is not None:
        d2h += finish(pending)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, world, device="cuda")
    det2.close()
    e2e = {"value": world * B * args.steps / e2e_s, "unit": "frames/s",
           "h2d_bytes_per_step": int(sum(im.nbytes for im in imgs)),
           "d2h_bytes_per_step": int(d2h // max(args.steps, 1))}

    peaks, peak_kind = measured_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s (FMA = 2)
    lane_peak = sm_count * 128 * sm_mhz * 1e6 / 1e12       # T lane-ops/s
    # cells (K2 + K3): ALU bound; one op = one lane slot
    cells_ops = B * cells_per_frame() * 64 * OPS_PER_CELL_PIXEL
    cells_ach = cells_ops / (stage_step[1] / 1e3) / 1e12
    roof_cells = {"bound": "alu", "achieved": cells_ach, "peak": lane_peak, "unit": "Tops/s",
                  "frac": cells_ach / lane_peak,
                  "traffic": None if args.hog_per_block else scaled(
                      recorded_traffic("k_cells_warp_1242x375_b32.txt", "k_cells_warp.cu"), B / 64.0),
                  "kernel": "k_cells_warp (uniform LBP + soft-binned HOG cell histograms, a warp per strip)" + (
                      "; per-block HOG variant, ops still counted as for shared cells" if args.hog_per_block else ""),
                  "peak_basis": f"{sm_count} SMs x 128 lanes x {sm_mhz} MHz, one op per lane slot "
                                f"({OPS_PER_CELL_PIXEL} algorithmic ops per cell-grid pixel; max SM clock, "
                                f"{peak_kind})",
                  # ncu, same source: fraction of cycles the schedulers issued (the kernel runs ~1.9
                  # instructions per algorithmic op: addressing, shared-memory traffic, control)
                  "issue_active_frac": None if args.hog_per_block else recorded_traffic(
                      "k_cells_warp_1242x375_b32.txt", "k_cells_warp.cu", "issue_active_frac")}
    # window scores (K4)
    k4_s = stage_step[2] / 1e3
    if args.svm == "fp32":
        k4_ach = B * wpf * FLOP_PER_WINDOW / k4_s / 1e12
        roof_k4 = {"bound": "alu", "achieved": k4_ach, "peak": fp32_peak, "unit": "TFLOP/s",
                   "frac": k4_ach / fp32_peak, "traffic": None,
                   "kernel": "k_svm (block L2-Hys norm + window correlation, FP32 FMA)",
                   "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x {sm_mhz} MHz ({peak_kind})"}
    else:
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        k4_ach = B * wpf * FLOP_PER_WINDOW / k4_s / 1e12
        executed = B * tc_units_per_frame() * TC_FLOP_PER_UNIT / k4_s / 1e12
        roof_k4 = {"bound": "tensor", "achieved": k4_ach, "peak": bf16, "unit": "TFLOP/s",
                   "frac": k4_ach / bf16, "executed_tflops": executed, "executed_frac": executed / bf16,
                   "traffic": None if args.hog_per_block else scaled(recorded_traffic("k_svm_tc_1242x375_b64.txt",
                                                                                      "k_svm_tc.cu"), B / 64.0),
                   "tensor_active_frac": None if args.hog_per_block else recorded_traffic(
                       "k_svm_tc_1242x375_b64.txt", "k_svm_tc.cu", "tensor_active_frac"),
                   "kernel": "k_svm_tc (block norms + window scores as bf16-split tcgen05 GEMMs)",
                   "peak_basis": f"bf16 dense, cuBLAS burst ({peak_kind}); achieved counts the "
                                 f"definition's 19,950 flop per window, executed the MMAs issued "
                                 f"(3 bf16 terms, padding, strip halo)"}
    stage_names = ["k_resize", "k_cells", "k_svm_tc" if args.svm != "fp32" else "k_svm", "k_nms"]
    dominant = stage_names[int(np.argmax(stage_step[:4]))]
    # (the recorded DRAM bytes are those of the default shared-cell kernels)
    hbm = None if args.hog_per_block else hbm_per_kernel(stage_step[:4], args.svm, B)
    for name, roof in (("k_cells", roof_cells), (stage_names[2], roof_k4)):
        if roof["traffic"] is None and hbm and hbm.get(name):
            roof["traffic"] = hbm[name]["dram_bytes"]
    roofline = roof_cells if dominant == "k_cells" else roof_k4 if dominant.startswith("k_svm") else roof_cells

    side = frames[:args.side_frames]
    other_k4 = None
    if rank == 0 and args.other_k4_steps > 0:
        other_k4 = run_other_k4(args, pd, torch, side, flush, w, b, fp32_peak,
                                float(peaks.get("bf16_tflops", 1900.0)))

    schemes = None
    if rank == 0 and args.scheme_reps > 0:
        schemes = run_schemes(args, pd, torch, w, b)

    pipelines = None
    if rank == 0 and args.pipeline_steps > 0:
        pipelines = run_pipelines(args, pd, torch, side, flush, w, b)

    upscaled = None
    if rank == 0 and args.upscale_steps > 0:
        upscaled = run_upscaled(args, pd, torch, side, flush, tile_costs, fp32_peak)

    proposal = proposal_4k = None
    if rank == 0 and args.proposal_steps > 0 and os.path.exists(PROPOSAL_CKPT):
        proposal = run_proposal(args, pd, torch, flush)
        if args.proposal_4k:
            proposal_4k = run_proposal(args, pd, torch, flush, recipe=5)

    c1 = run_c1(args, pd, torch, w, b) if rank == 0 and args.c1_replays > 0 else None
    c3 = run_c3(args, pd, torch, flush, w, b, pool) if rank == 0 and args.c3_steps > 0 else None

    cpu = None
    if oracle_pool:
        n1 = min(args.cpu_sample_frames, B)
        t1 = time_oracle(imgs[:n1], w, b)
        nall = min(2 * cores, B)
        tall = time_oracle_parallel(pool, cores, imgs[:nall])
        cpu = {"value": nall / tall, "unit": "frames/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
               "sample": f"{nall} of the step's {B} frames through the whole plain path, FP64, one frame per "
                         f"worker process on all {cores} host cores",
               "single_thread": {"value": n1 / t1, "unit": "frames/s", "cores": 1,
                                 "sample": f"{n1} of the step's frames, one thread"}}
    pool.close()

    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_FPS_1242x375, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WIDTH}x{HEIGHT} u8 frames, pyramid factor 1.05 (23 levels), "
                               "plain HOG+LBP+SVM+NMS" + (", per-block HOG" if args.hog_per_block else ""),
                   "timing": "K steps on two detector handles alternating on two streams (step i+1 may "
                             "overlap step i); serial: the same K steps on one handle, each timed alone",
                   "frames_per_step": B * world, "frames_per_gpu": B, "windows_per_frame": wpf,
                   "l2": "flushed (256 MB write) before every timed step",
                   "k4_tile_costs": [round(c, 4) for c in tile_costs],
                   "launch_shapes": dict(tuning, source="autotuner (pyramid and score stage times on 64 "
                                         "of the step's frames)" if not args.no_autotune else "library defaults"),
                   "parallelism": f"{world} independent replicas"},
        "roofline": roofline,
        "roofline_k4": roof_k4,
        "hbm_per_kernel": hbm,
        "other_k4": other_k4,
        "pipelines": pipelines,
        "schemes": schemes,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "serial": {"value": world * B * args.steps / (serial_ms / 1e3), "ms_per_step": serial_ms / args.steps},
        "stage_ms_per_step": {"pyramid": stage_step[0], "cells": stage_step[1], "norm_svm": stage_step[2],
                              "nms": stage_step[3]},
        "upscaled_40_levels": upscaled,
        "proposal": proposal,
        "proposal_4k_mix": proposal_4k,
        "c1_latency_320x240": c1,
        "c3_mixed_64": c3,
        "px_per_ns": B * WIDTH * HEIGHT / (ms_step * 1e6),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    det.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
