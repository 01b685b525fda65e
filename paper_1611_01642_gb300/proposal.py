"""Training, calibration and checkpoints of the learned window proposal.

The proposal network (a small CNN, defined in the header of the library) is
not part of the paper: it predicts, for every sliding window of every pyramid
level, whether the window's SVM score (the linear classifier of Sec. 3 over
the HOG+LBP block features) exceeds the detection threshold, so that the
sparse path computes cells and scores only near such windows.

Labels are the detector's own scores: a window is positive iff its score on
the plain path is above ``label_threshold``. Every training step runs on the
GPU (pd_cnn_train_step: forward, mean binary cross-entropy with a positive
weight, backward, Adam, all in the library's kernels); this module only
orders the batches and keeps the bookkeeping.

Checkpoint format: one ``.npz`` with ``params`` (float32[14210], the flat
order w1 b1 w2 b2 w3 b3 wh bh v bv) and ``meta`` (a JSON string: training
recipe, keep threshold, measured recall and keep fraction).
"""
from __future__ import annotations

import json
import math
import time
from dataclasses import asdict, dataclass, field

import numpy as np

from . import (CNN_PARAMS, Detector, PD_EOVERFLOW, PD_OK, pd_cnn_get_params, pd_cnn_set_params,
               pd_cnn_train_loss, pd_cnn_train_step)


@dataclass
class TrainConfig:
    lr: float = 1e-3                 # Adam step size
    label_threshold: float = 0.0     # positive iff plain score > this
    pos_weight: float = 0.0          # 0: neg/pos of the first batch
    steps_per_batch: int = 4         # Adam steps on each detected batch
    init_seed: int = 0               # He initialisation seed
    total_batches: int = 0           # > 0: cosine decay of lr to 0 over this many batches
    extra: dict = field(default_factory=dict)


def init_params(seed: int) -> np.ndarray:
    """He-style initial parameters (flat float32), drawn from PCG64(SeedSequence([23, seed]))."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([23, seed])))
    parts = [rng.standard_normal(16 * 9) * np.sqrt(2.0 / 9), np.zeros(16),
             rng.standard_normal(32 * 16 * 9) * np.sqrt(2.0 / (16 * 9)), np.zeros(32),
             rng.standard_normal(32 * 32 * 9) * np.sqrt(2.0 / (32 * 9)), np.zeros(32),
             rng.standard_normal(32) * np.sqrt(1.0 / 32), np.zeros(1),
             rng.standard_normal(128) * np.sqrt(1.0 / 128), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == CNN_PARAMS
    return p


def _to_device(frames):
    import torch
    return [f if isinstance(f, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(f)).cuda()
            for f in frames]


def _flat_scores(det: Detector, n_frames: int, logits: bool = False) -> np.ndarray:
    maps = []
    for f in range(n_frames):
        src = det.logit_maps(f) if logits else det.score_maps(f)
        maps += [m.reshape(-1) for m in src]
    import torch
    return torch.cat(maps).cpu().numpy() if maps else np.zeros(0, np.float32)


def train(det: Detector, batches, cfg: TrainConfig, params: np.ndarray | None = None, log=print):
    """Trains the proposal on ``batches`` (an iterable of frame lists) and returns the flat parameters.

    Each batch is detected once on the plain path (labels), then ``steps_per_batch`` Adam steps run on
    all windows of all its levels. ``det`` must have been created with room for the largest batch.
    """
    det.set_proposal(False)
    pd_cnn_set_params(det.h, init_params(cfg.init_seed) if params is None else params)
    pos_weight = cfg.pos_weight
    history = []
    t0 = time.time()
    for b, frames in enumerate(batches):
        det.detect(_to_device(frames))
        # labels come from the score maps, which a frame with more NMS candidates
        # than the cap (PD_EOVERFLOW: no boxes for it) still has in full
        if det.sync() not in (PD_OK, PD_EOVERFLOW):
            raise RuntimeError("detect failed while labelling")
        if pos_weight <= 0:
            s = _flat_scores(det, len(frames))
            pos = int((s > cfg.label_threshold).sum())
            pos_weight = float(max(s.size - pos, 1) / max(pos, 1))
            log(f"pos_weight = neg/pos = {pos_weight:.2f} ({pos} of {s.size} windows positive)")
        lr = cfg.lr
        if cfg.total_batches > 0:
            lr = 0.5 * cfg.lr * (1.0 + math.cos(math.pi * min(b, cfg.total_batches) / cfg.total_batches))
        for _ in range(cfg.steps_per_batch):
            pd_cnn_train_step(det.h, pos_weight, cfg.label_threshold, lr)
        loss = pd_cnn_train_loss(det.h)
        history.append(loss)
        if b % 10 == 0:
            log(f"batch {b:4d}  loss {loss:.4f}  {time.time() - t0:.1f}s")
    cfg.pos_weight = pos_weight
    params, _ = pd_cnn_get_params(det.h)
    return params, history


def window_stats(det: Detector, batches, threshold: float = 0.0):
    """(scores, logits) of all windows of ``batches``: plain-path scores and the proposal's keep-logits."""
    S, Z = [], []
    for frames in batches:
        dev = _to_device(frames)
        det.set_proposal(False)
        det.detect(dev)
        if det.sync() not in (PD_OK, PD_EOVERFLOW):  # (scores only: an NMS overflow is fine)
            raise RuntimeError("detect failed")
        S.append(_flat_scores(det, len(frames)))
        det.set_proposal(True, float("-inf"))
        det.detect(dev)
        if det.sync() not in (PD_OK, PD_EOVERFLOW):  # (scores only: an NMS overflow is fine)
            raise RuntimeError("detect failed")
        Z.append(_flat_scores(det, len(frames), logits=True))
    det.set_proposal(False)
    return np.concatenate(S), np.concatenate(Z)


def calibrate(scores: np.ndarray, logits: np.ndarray, recall: float = 0.99, threshold: float = 0.0) -> float:
    """Largest keep threshold tau with |{z > tau} & {s > threshold}| >= recall * |{s > threshold}|."""
    z = np.sort(logits[scores > threshold].astype(np.float64))
    if z.size == 0:
        return float("-inf")
    m = int(np.floor((1.0 - recall) * z.size))     # windows that may be dropped
    m = min(m, z.size - 1)
    return float(np.nextafter(np.float32(z[m]), np.float32(-np.inf)))


def calibrate_sparse(det: Detector, batches, recall: float = 0.99, threshold: float = 0.0, lo: float | None = None,
                     iters: int = 12):
    """Largest keep threshold whose sparse path (tile-level keeping) still scores >= recall of the positives.

    A tile is scored if any of its windows is kept, so the sparse path's recall at a given tau is at
    least the window-level recall; this searches tau directly on the path's own recall (bisection
    between the window-level threshold ``lo`` and the largest keep-logit of the batches).
    """
    batches = list(batches)
    if lo is None:
        s, z = window_stats(det, batches, threshold)
        lo = calibrate(s, z, recall, threshold)
        hi = float(z.max()) if z.size else lo
    else:
        hi = lo + 16.0
    if sparse_metrics(det, batches, hi, threshold)["recall"] >= recall:
        return hi
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if sparse_metrics(det, batches, mid, threshold)["recall"] >= recall:
            lo = mid
        else:
            hi = mid
    return lo


def sparse_metrics(det: Detector, batches, tau: float, threshold: float = 0.0):
    """Recall and keep fraction of the sparse path against the plain path, window by window.

    recall = |scored on the sparse path and score > threshold| / |score > threshold on the plain path|;
    keep = fraction of windows the sparse path scored (tile-level decision); window_keep = fraction
    of windows whose own keep-logit is above tau.
    """
    pos = hit = kept = total = zkept = 0
    for frames in batches:
        dev = _to_device(frames)
        det.set_proposal(False)
        det.detect(dev)
        if det.sync() not in (PD_OK, PD_EOVERFLOW):  # (scores only: an NMS overflow is fine)
            raise RuntimeError("detect failed")
        s = _flat_scores(det, len(frames))
        det.set_proposal(True, tau)
        det.detect(dev)
        if det.sync() not in (PD_OK, PD_EOVERFLOW):  # (scores only: an NMS overflow is fine)
            raise RuntimeError("detect failed")
        sp = _flat_scores(det, len(frames))
        zkept += int((_flat_scores(det, len(frames), logits=True) > tau).sum())
        scored = ~np.isneginf(sp)
        if not np.array_equal(sp[scored], s[scored]):
            raise AssertionError("sparse scores differ from the plain path on scored windows")
        p = s > threshold
        pos += int(p.sum())
        hit += int((p & scored).sum())
        kept += int(scored.sum())
        total += s.size
    det.set_proposal(False)
    return dict(recall=hit / max(pos, 1), keep_fraction=kept / max(total, 1),
                window_keep_fraction=zkept / max(total, 1), positives=pos, windows=total)


def save_checkpoint(path: str, params: np.ndarray, meta: dict) -> None:
    np.savez(path, params=np.asarray(params, np.float32), meta=np.array(json.dumps(meta, sort_keys=True)))


def load_checkpoint(path: str):
    d = np.load(path, allow_pickle=False)
    params = np.asarray(d["params"], np.float32)
    if params.size != CNN_PARAMS:
        raise ValueError(f"{path}: {params.size} parameters, expected {CNN_PARAMS}")
    return params, json.loads(str(d["meta"]))


def _scene_batches(width, height, key, first, count, batch):
    """Synthetic frames (seeded by SeedSequence([key, i])) in batches, generated lazily."""
    import synth
    for i0 in range(first, first + count, batch):
        yield [synth.make_scene(width, height, key, i, n_sil=("poisson", 10.0), heights=(48, "0.8H"))
               for i in range(i0, min(i0 + batch, first + count))]


def recalibrate(path: str, out: str, calib_frames: int = 16, val_frames: int = 16, recall: float = 0.99,
                width: int = 1920, height: int = 1080, factor: float = 1.05, batch: int = 8,
                level_step: int | None = None):
    """Re-derives the keep threshold of a checkpoint on the sparse path's own recall; writes ``out``.
    level_step: the network runs on every level_step-th level (None: the checkpoint's, else 1)."""
    import os
    params, meta = load_checkpoint(path)
    svm = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                       "svm_template_seed0.npz")
    d = np.load(svm)
    det = Detector(d["w"], float(d["b"]), max_frames=batch, max_width=width, max_height=height,
                   pyr_factor=float(np.float32(factor)))
    try:
        pd_cnn_set_params(det.h, params)
        step = int(level_step if level_step is not None else meta.get("level_step", 1))
        det.set_proposal(False, 0.0, level_step=step)
        calib = list(_scene_batches(width, height, 101, 0, calib_frames, batch))
        s, z = window_stats(det, calib)
        tau_window = calibrate(s, z, recall)
        tau = calibrate_sparse(det, calib, recall)
        val = list(_scene_batches(width, height, 101, calib_frames, val_frames, batch))
        meta = dict(meta, keep_logit_threshold=tau, window_level_threshold=tau_window, level_step=step,
                    calibration=dict(kind="path", frames=calib_frames, recall=recall),
                    validation=sparse_metrics(det, val, tau))
        save_checkpoint(out, params, meta)
        return meta
    finally:
        det.close()


def _scene_worker(args):
    import synth
    width, height, key, i = args
    return synth.make_scene(width, height, key, i, n_sil=("poisson", 10.0), heights=(48, "0.8H"))


def _scene_pool(width, height, key, count, workers=0):
    """Frames i < count of scenes [key, i] (as _scene_batches), generated by spawned worker processes."""
    import multiprocessing as mp
    import os
    n = workers or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_scene_worker, [(width, height, key, i) for i in range(count)], chunksize=4)


def _curve(det: Detector, a, sizes):
    """Keep fraction at the calibrated recall against the training-set size: one model per size, all
    from the same initial parameters and for the same number of batches (a small set is visited more
    times), so that only the amount of training data differs."""
    pool = _scene_pool(a.width, a.height, 100, max(sizes), a.workers)
    calib = list(_scene_batches(a.width, a.height, 101, 0, a.calib_frames, a.batch))
    val = list(_scene_batches(a.width, a.height, 101, a.calib_frames, a.val_frames, a.batch))
    for n in sizes:
        order_rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([102, n])))

        def batches():
            done = 0
            while done < a.curve_batches:
                idx = order_rng.permutation(n)
                for i0 in range(0, n, a.batch):
                    if done == a.curve_batches:
                        return
                    yield [pool[i] for i in idx[i0:i0 + a.batch]]
                    done += 1
        cfg = TrainConfig(lr=a.lr, steps_per_batch=a.steps_per_batch, total_batches=a.curve_batches if a.cosine else 0)
        t0 = time.time()
        params, hist = train(det, batches(), cfg, log=lambda *x: None)
        train_s = time.time() - t0
        pd_cnn_set_params(det.h, params)
        det.set_proposal(False, 0.0, level_step=a.level_step)
        tau = calibrate_sparse(det, calib, a.recall)
        m = sparse_metrics(det, val, tau)
        print(json.dumps(dict(train_frames=n, batches=a.curve_batches, steps=a.curve_batches * a.steps_per_batch,
                              level_step=a.level_step, final_loss=hist[-1], keep_logit_threshold=tau,
                              train_seconds=train_s, **m)), flush=True)


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="Train and calibrate the window proposal on synthetic scenes.")
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--factor", type=float, default=1.05)
    ap.add_argument("--train-frames", type=int, default=256)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--steps-per-batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--cosine", type=int, default=1, help="cosine decay of the step size over the run")
    ap.add_argument("--calib-frames", type=int, default=32)
    ap.add_argument("--val-frames", type=int, default=32)
    ap.add_argument("--recall", type=float, default=0.99)
    ap.add_argument("--calibrate", choices=["window", "path"], default="path",
                    help="keep threshold from window-level recall, or from the sparse path's own recall")
    ap.add_argument("--svm", default=None, help="npz with w, b (default: the seed-0 template)")
    ap.add_argument("--level-step", type=int, default=1,
                    help="the network runs on every level_step-th level when calibrating (stored in the meta)")
    ap.add_argument("--curve", default=None,
                    help="comma-separated training-set sizes: train one model per size (same start, "
                         "--curve-batches batches each) and print its calibrated keep fraction; no checkpoint")
    ap.add_argument("--curve-batches", type=int, default=192)
    ap.add_argument("--workers", type=int, default=0, help="processes generating the scenes (0: all cores)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if a.curve is None and a.out is None:
        ap.error("--out is required (or --curve)")
    import os
    import torch  # noqa: F401  (CUDA context for the frames)
    from . import build as bld
    bld.build()
    svm = a.svm or os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "tests", "golden", "svm_template_seed0.npz")
    d = np.load(svm)
    w, b = d["w"], float(d["b"])
    det = Detector(w, b, max_frames=a.batch, max_width=a.width, max_height=a.height,
                   pyr_factor=float(np.float32(a.factor)))
    try:
        if a.curve is not None:
            _curve(det, a, [int(v) for v in a.curve.split(",")])
            return
        # training frames: a fixed pool, visited once per epoch in a seeded order
        pool = _scene_pool(a.width, a.height, 100, a.train_frames, a.workers)
        order_rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([102])))

        def epochs():
            for _ in range(a.epochs):
                idx = order_rng.permutation(len(pool))
                for i0 in range(0, len(idx), a.batch):
                    yield [pool[i] for i in idx[i0:i0 + a.batch]]
        cfg = TrainConfig(lr=a.lr, steps_per_batch=a.steps_per_batch,
                          total_batches=a.epochs * ((a.train_frames + a.batch - 1) // a.batch) if a.cosine else 0)
        t0 = time.time()
        params, hist = train(det, epochs(), cfg)
        train_s = time.time() - t0
        pd_cnn_set_params(det.h, params)
        det.set_proposal(False, 0.0, level_step=a.level_step)
        calib = list(_scene_batches(a.width, a.height, 101, 0, a.calib_frames, a.batch))
        s, z = window_stats(det, calib)
        tau_window = calibrate(s, z, a.recall)
        tau = calibrate_sparse(det, calib, a.recall) if a.calibrate == "path" else tau_window
        val = list(_scene_batches(a.width, a.height, 101, a.calib_frames, a.val_frames, a.batch))
        m = sparse_metrics(det, val, tau)
        meta = dict(recipe=vars(a), train=asdict(cfg), train_seconds=train_s, final_loss=hist[-1],
                    first_loss=hist[0], keep_logit_threshold=tau, window_level_threshold=tau_window,
                    level_step=a.level_step,
                    calib_window_recall=float(np.mean(z[s > 0] > tau)) if (s > 0).any() else 1.0,
                    validation=m)
        save_checkpoint(a.out, params, meta)
        print(json.dumps(meta, sort_keys=True))
    finally:
        det.close()


if __name__ == "__main__":
    main()
