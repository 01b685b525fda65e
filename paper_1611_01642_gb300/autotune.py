"""Autotuners of the launch shapes of the detector's kernels.

Default path (``tune_default_path`` / ``apply_default``): the pyramid kernel's
column groups per warp task (4, 8 or 16) and the tensor-core window-score
kernel's window rows per work item (16 .. 64), set with pd_set_tuning. Each is
chosen by timing its own stage (pd_stage_times, CUDA events) on the caller's
batch, median of a few detects, the pyramid first, then the score kernel.
Neither changes any result (the same sums in the same order). The choice is
cached per GPU, library build and workload (frame sizes, pyramid factor,
upsampled levels).

FP32 window-score kernel (K4 with PD_FLAG_SVM_FP32), below:

The planner picks, for every pyramid level, the K4 tile shape with the least
(number of tiles x cost[shape]). This module measures cost[shape] on the
running GPU: it forces each shape in turn on a synthetic batch, times the K4
stage with CUDA events (pd_stage_times) and divides by the number of tiles
that shape needs. Per-tile costs measured in isolation do not capture how
shapes behave mixed in one launch, so the measured table is then checked
against the library's default table on the whole batch, and the faster of
the two is kept. The result is cached as JSON, keyed by the GPU name, its SM
count and a hash of the library, under ``$XDG_CACHE_HOME`` (default
``~/.cache``)/paper_1611_01642_gb300/tile_costs.json.

Scores do not depend on the tiling beyond float rounding order (the same
sums in another tiling), so tuning never changes results by more than that.
"""
from __future__ import annotations

import hashlib
import json
import math
import os

import numpy as np

from . import (PD_FLAG_STAGE_TIMING, PD_FLAG_SVM_FP32, PD_OK, TILE_SHAPE_DIMS, TILE_SHAPES, Detector, library_path,
               pd_get_tile_costs, pd_get_tuning, pd_set_tile_costs, pd_set_tuning, pd_stage_times)

K1_GROUPS = (4, 8, 16)
TC_ITEM_ROWS = (8, 16, 24, 32, 48, 64)


def _cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "paper_1611_01642_gb300", "tile_costs.json")


def _key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    h = hashlib.sha256()
    with open(library_path(), "rb") as f:
        h.update(f.read())
    return f"{p.name}|{p.multi_processor_count}|{h.hexdigest()[:16]}"


def tiles_for(levels, shape: int) -> int:
    tw, th = TILE_SHAPE_DIMS[shape]
    return sum(math.ceil(lv["rows"] / th) * math.ceil(lv["cols"] / tw) for lv in levels if lv["rows"] > 0)


def measure(frames, svm_w, svm_b, factor: float, steps: int = 5, warmup: int = 2):
    """Per-tile K4 milliseconds of every shape on ``frames`` (device or host u8 arrays)."""
    import torch
    dev = [f if isinstance(f, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames]
    W = max(f.shape[1] for f in dev)
    H = max(f.shape[0] for f in dev)
    det = Detector(svm_w, svm_b, pyr_factor=factor, max_frames=len(dev), max_width=W, max_height=H,
                   flags=PD_FLAG_STAGE_TIMING | PD_FLAG_SVM_FP32)
    out = []
    try:
        for s in range(TILE_SHAPES):
            costs = [1e6] * TILE_SHAPES
            costs[s] = 1.0
            pd_set_tile_costs(det.h, costs)
            for _ in range(warmup):
                det.detect(dev)
                if det.sync() != PD_OK:
                    raise RuntimeError("detect failed while tuning")
            ms = 0.0
            for _ in range(steps):
                det.detect(dev)
                if det.sync() != PD_OK:
                    raise RuntimeError("detect failed while tuning")
                ms += pd_stage_times(det.h)[2]
            n = sum(tiles_for(det.levels(f), s) for f in range(len(dev)))
            out.append(ms / steps / max(n, 1))
    finally:
        det.close()
    return out


def plan_ms(frames, svm_w, svm_b, factor: float, cost, steps: int = 7, warmup: int = 2) -> float:
    """Median K4 milliseconds of the whole batch with the cost table ``cost``."""
    import torch
    dev = [f if isinstance(f, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames]
    det = Detector(svm_w, svm_b, pyr_factor=factor, max_frames=len(dev), max_width=max(f.shape[1] for f in dev),
                   max_height=max(f.shape[0] for f in dev), flags=PD_FLAG_STAGE_TIMING | PD_FLAG_SVM_FP32)
    try:
        pd_set_tile_costs(det.h, cost)
        ms = []
        for i in range(warmup + steps):
            det.detect(dev)
            if det.sync() != PD_OK:
                raise RuntimeError("detect failed while tuning")
            if i >= warmup:
                ms.append(pd_stage_times(det.h)[2])
        return float(np.median(ms))
    finally:
        det.close()


def tile_costs(frames, svm_w, svm_b, factor: float, refresh: bool = False):
    """Per-tile cost table for the planner, measured once per GPU and library build, then cached."""
    path = _cache_path()
    key = _key()
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not refresh and key in cache and len(cache[key].get("cost", [])) == TILE_SHAPES:
        return cache[key]["cost"]
    ms = measure(frames, svm_w, svm_b, factor)
    measured = [m / ms[0] for m in ms]
    default = default_costs(svm_w, svm_b)
    t_default = plan_ms(frames, svm_w, svm_b, factor, default)
    t_measured = plan_ms(frames, svm_w, svm_b, factor, measured)
    cost = measured if t_measured < t_default else default
    cache[key] = {"cost": cost, "ms_per_tile": ms, "measured": measured, "default": default,
                  "k4_ms_default": t_default, "k4_ms_measured": t_measured}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # read-only home: the costs still apply to this process
    return cost


def default_costs(svm_w, svm_b):
    """The library's built-in cost table (read from a fresh handle)."""
    det = Detector(svm_w, svm_b, max_frames=1, max_width=64, max_height=128)
    try:
        return [float(c) for c in pd_get_tile_costs(det.h)]
    finally:
        det.close()


def apply(det: Detector, frames, svm_w, svm_b, factor: float, refresh: bool = False):
    """Measures (or loads) the tile costs and sets them on ``det``; returns them."""
    cost = tile_costs(frames, svm_w, svm_b, factor, refresh)
    pd_set_tile_costs(det.h, cost)
    return cost


# ----------------------------------------------------------------------------- default path
def _load_cache(path):
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return {}


def _store_cache(path, cache):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # read-only home: the choice still applies to this process


def _workload_key(frames, factor: float, upscale: int) -> str:
    sizes = {}
    for f in frames:
        sizes[(int(f.shape[1]), int(f.shape[0]))] = sizes.get((int(f.shape[1]), int(f.shape[0])), 0) + 1
    return json.dumps([sorted([list(k) + [v] for k, v in sizes.items()]), round(float(factor), 6), int(upscale)])


def _stage_ms(det, dev, stage: int, steps: int, warmup: int) -> float:
    for _ in range(warmup):
        det.detect(dev)
        if det.sync() != PD_OK:
            raise RuntimeError("detect failed while tuning")
    ms = []
    for _ in range(steps):
        det.detect(dev)
        if det.sync() != PD_OK:
            raise RuntimeError("detect failed while tuning")
        ms.append(pd_stage_times(det.h)[stage])
    return float(np.median(ms))


def tune_default_path(frames, svm_w, svm_b, factor: float, upscale: int = 0, flags: int = 0,
                      steps: int = 5, warmup: int = 2, refresh: bool = False):
    """{k1_groups, tc_item_rows} for this GPU, library build and workload, measured once and cached."""
    import torch
    path = _cache_path().replace("tile_costs.json", "default_path.json")
    key = _key() + "|" + _workload_key(frames, factor, upscale) + f"|{flags}"
    cache = _load_cache(path)
    if not refresh and key in cache:
        return cache[key]["tuning"]
    dev = [f if isinstance(f, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames]
    det = Detector(svm_w, svm_b, pyr_factor=factor, max_frames=len(dev), max_width=max(f.shape[1] for f in dev),
                   max_height=max(f.shape[0] for f in dev), upscale_levels=upscale,
                   flags=PD_FLAG_STAGE_TIMING | flags)
    try:
        best = pd_get_tuning(det.h)
        k1_ms, tc_ms = {}, {}
        for g in K1_GROUPS:
            pd_set_tuning(det.h, g, best["tc_item_rows"])
            k1_ms[g] = _stage_ms(det, dev, 0, steps, warmup)
        best["k1_groups"] = min(k1_ms, key=k1_ms.get)
        if not flags & PD_FLAG_SVM_FP32:
            for r in TC_ITEM_ROWS:
                pd_set_tuning(det.h, best["k1_groups"], r)
                tc_ms[r] = _stage_ms(det, dev, 2, steps, warmup)
            best["tc_item_rows"] = min(tc_ms, key=tc_ms.get)
    finally:
        det.close()
    cache[key] = {"tuning": best, "pyramid_ms": {str(k): v for k, v in k1_ms.items()},
                  "scores_ms": {str(k): v for k, v in tc_ms.items()}}
    _store_cache(path, cache)
    return best


def apply_default(det: Detector, frames, svm_w, svm_b, factor: float, upscale: int = 0, flags: int = 0,
                  refresh: bool = False):
    """Measures (or loads) the default path's launch shapes and sets them on ``det``; returns them."""
    t = tune_default_path(frames, svm_w, svm_b, factor, upscale, flags, refresh=refresh)
    pd_set_tuning(det.h, t["k1_groups"], t["tc_item_rows"])
    return t
