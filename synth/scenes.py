"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *generates inputs*: grayscale frames, training crops, random
weights and random score maps. It contains none of the detector's arithmetic
(no pyramid, no LBP/HOG, no SVM, no NMS), so that the oracle and the CUDA path
stay independent while being fed the same bytes.

Scene recipe (the paper's video sequence is not available; these frames stand
in for its 1242x375 size and for the larger sizes of the batched workloads):

* background: i.i.d. U{0..255} noise from numpy's PCG64 seeded with
  ``SeedSequence([cfg_id, frame_idx])``, smoothed by a separable Gaussian
  (sigma 2, radius 6, half-sample symmetric borders) in float64, rounded half
  to even and clipped to u8;
* pedestrians: a silhouette of height ``h`` and box width ``h/2`` made of an
  elliptic head, a rectangular torso and two rectangular legs; every covered
  pixel gets ``clip(pixel + c)`` with ``c = +40`` or ``-40`` (fair coin);
  silhouettes are pasted one after another and clipped at the frame border.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "SCENE_CONFIGS",
    "make_scene",
    "make_frames",
    "make_training_crops",
    "random_image",
    "random_svm",
    "random_score_maps",
    "frame_specs",
    "uniform_noise_image",
]

# Workload recipes (sizes, pyramid factor, pedestrian statistics).
#   frames: list of (width, height, count)
#   n_sil:  ("uniform", lo, hi) integer count or ("poisson", lam)
#   heights: (lo, hi) pixel range; hi may be the string "0.8H"
SCENE_CONFIGS = {
    1: dict(name="320x240 single frame", frames=[(320, 240, 1)], factor=1.2,
            n_sil=("fixed", 3), heights=(64, 128)),
    2: dict(name="1242x375 single frame", frames=[(1242, 375, 1)], factor=1.05,
            n_sil=("uniform", 8, 20), heights=(48, 300)),
    3: dict(name="64 mixed frames", frames=[(1242, 375, 32), (640, 480, 16), (1920, 1080, 16)],
            factor=1.05, n_sil=("poisson", 10.0), heights=(48, "0.8H")),
    4: dict(name="16x1920x1080", frames=[(1920, 1080, 16)], factor=1.05,
            n_sil=("poisson", 10.0), heights=(48, "0.8H")),
    5: dict(name="16x3840x2160 + 48x1242x375", frames=[(3840, 2160, 16), (1242, 375, 48)],
            factor=1.05, n_sil=("poisson", 10.0), heights=(48, 600)),
}

_SIGMA = 2.0
_RADIUS = 6


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def _gauss_kernel() -> np.ndarray:
    i = np.arange(-_RADIUS, _RADIUS + 1, dtype=np.float64)
    k = np.exp(-(i * i) / (2.0 * _SIGMA * _SIGMA))
    return k / k.sum()


def _smooth(noise: np.ndarray) -> np.ndarray:
    """Separable Gaussian blur in float64 with half-sample symmetric borders."""
    k = _gauss_kernel()
    a = noise.astype(np.float64)
    p = np.pad(a, ((0, 0), (_RADIUS, _RADIUS)), mode="symmetric")
    h = np.zeros_like(a)
    for d in range(2 * _RADIUS + 1):
        h += k[d] * p[:, d:d + a.shape[1]]
    p = np.pad(h, ((_RADIUS, _RADIUS), (0, 0)), mode="symmetric")
    v = np.zeros_like(a)
    for d in range(2 * _RADIUS + 1):
        v += k[d] * p[d:d + a.shape[0], :]
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def _background(rng: np.random.Generator, width: int, height: int) -> np.ndarray:
    noise = rng.integers(0, 256, size=(height, width), dtype=np.int64)
    return _smooth(noise)


def _silhouette_mask(h: float, x0: float, y0: float, width: int, height: int):
    """Boolean mask of one silhouette (box of h/2 x h with top-left (x0, y0))."""
    ws = 0.5 * h
    xa = int(max(0, np.floor(x0)))
    xb = int(min(width, np.ceil(x0 + ws) + 1))
    ya = int(max(0, np.floor(y0)))
    yb = int(min(height, np.ceil(y0 + h) + 1))
    if xa >= xb or ya >= yb:
        return None
    yy, xx = np.mgrid[ya:yb, xa:xb].astype(np.float64)
    u = xx + 0.5 - x0 - 0.5 * ws          # horizontal offset from the axis
    v = yy + 0.5 - y0                     # vertical offset from the top
    head = (u / (0.07 * h)) ** 2 + ((v - 0.09 * h) / (0.09 * h)) ** 2 <= 1.0
    torso = (np.abs(u) <= 0.15 * h) & (v >= 0.18 * h) & (v < 0.58 * h)
    legs = ((np.abs(u) >= 0.02 * h) & (np.abs(u) <= 0.13 * h)
            & (v >= 0.58 * h) & (v < h))
    return (ya, yb, xa, xb), head | torso | legs


def _paste(img: np.ndarray, h: float, x0: float, y0: float, contrast: int) -> None:
    r = _silhouette_mask(h, x0, y0, img.shape[1], img.shape[0])
    if r is None:
        return
    (ya, yb, xa, xb), m = r
    sub = img[ya:yb, xa:xb].astype(np.int32)
    sub = np.where(m, np.clip(sub + contrast, 0, 255), sub)
    img[ya:yb, xa:xb] = sub.astype(np.uint8)


def make_scene(width: int, height: int, cfg_id: int, frame_idx: int,
               n_sil=None, heights=None) -> np.ndarray:
    """One seeded synthetic frame, u8[height][width] (row-major, pitch = width)."""
    cfg = SCENE_CONFIGS.get(cfg_id, SCENE_CONFIGS[2])
    n_sil = cfg["n_sil"] if n_sil is None else n_sil
    heights = cfg["heights"] if heights is None else heights
    rng = _rng(cfg_id, frame_idx)
    img = _background(rng, width, height)
    kind = n_sil[0]
    if kind == "fixed":
        n = int(n_sil[1])
    elif kind == "uniform":
        n = int(rng.integers(n_sil[1], n_sil[2] + 1))
    else:
        n = int(rng.poisson(n_sil[1]))
    lo, hi = heights
    if hi == "0.8H":
        hi = 0.8 * height
    hi = max(float(lo), float(hi))
    for _ in range(n):
        h = float(rng.uniform(lo, hi))
        ws = 0.5 * h
        x0 = float(rng.uniform(-0.25 * ws, width - 0.75 * ws))
        y0 = float(rng.uniform(-0.25 * h, height - 0.75 * h))
        c = 40 if rng.integers(0, 2) else -40
        _paste(img, h, x0, y0, c)
    return img


def frame_specs(cfg_id: int, first_frame: int = 0, limit: int | None = None):
    """(width, height, cfg_id, frame_idx) of the frames of workload ``cfg_id``, in order."""
    cfg = SCENE_CONFIGS[cfg_id]
    out = []
    idx = 0
    for (w, h, count) in cfg["frames"]:
        for _ in range(count):
            if idx >= first_frame and (limit is None or len(out) < limit):
                out.append((w, h, cfg_id, idx))
            idx += 1
    return out


def make_frames(cfg_id: int, first_frame: int = 0, limit: int | None = None):
    """Frames of workload ``cfg_id`` in order: list of u8 arrays."""
    return [make_scene(*spec) for spec in frame_specs(cfg_id, first_frame, limit)]


def make_training_crops(seed: int = 0, n_pos: int = 1000, n_neg: int = 1000):
    """64x128 crops for the mean-difference SVM template.

    Positives: a silhouette of height 96 +- 8 px centred in a smoothed-noise
    crop. Negatives: smoothed noise and, with probability 1/2, a silhouette
    shifted at least 32 px off the crop centre (a partial pedestrian).
    Returns (pos u8[n_pos][128][64], neg u8[n_neg][128][64]).
    """
    rng = _rng(seed)
    pos = np.empty((n_pos, 128, 64), np.uint8)
    neg = np.empty((n_neg, 128, 64), np.uint8)
    for n in range(n_pos):
        img = _background(rng, 64, 128)
        h = float(rng.uniform(88.0, 104.0))
        c = 40 if rng.integers(0, 2) else -40
        _paste(img, h, 32.0 - 0.25 * h, 64.0 - 0.5 * h, c)
        pos[n] = img
    for n in range(n_neg):
        img = _background(rng, 64, 128)
        if rng.integers(0, 2):
            h = float(rng.uniform(88.0, 104.0))
            c = 40 if rng.integers(0, 2) else -40
            if rng.integers(0, 2):
                dx = float(rng.uniform(32.0, 56.0)) * (1 if rng.integers(0, 2) else -1)
                dy = float(rng.uniform(-8.0, 8.0))
            else:
                dx = float(rng.uniform(-8.0, 8.0))
                dy = float(rng.uniform(32.0, 80.0)) * (1 if rng.integers(0, 2) else -1)
            _paste(img, h, 32.0 - 0.25 * h + dx, 64.0 - 0.5 * h + dy, c)
        neg[n] = img
    return pos, neg


def uniform_noise_image(width: int, height: int, seed: int) -> np.ndarray:
    """Unsmoothed U{0..255} noise (worst case for histogram contention)."""
    return _rng(7, seed).integers(0, 256, size=(height, width), dtype=np.uint8)


def random_image(width: int, height: int, seed: int, smooth: bool = True) -> np.ndarray:
    """Seeded test image: smoothed noise plus a few silhouettes."""
    rng = _rng(11, seed)
    img = _background(rng, width, height) if smooth else rng.integers(
        0, 256, size=(height, width), dtype=np.uint8)
    for _ in range(int(rng.integers(0, 4))):
        h = float(rng.uniform(32, max(33.0, 1.2 * height)))
        _paste(img, h, float(rng.uniform(-0.3 * h, width)), float(rng.uniform(-0.3 * h, height)),
               40 if rng.integers(0, 2) else -40)
    return img


def random_svm(seed: int, scale: float = 0.05):
    """Seeded Gaussian template w[15][7][95] (float32) and bias (float)."""
    rng = _rng(13, seed)
    w = (rng.standard_normal((15, 7, 95)) * scale).astype(np.float32)
    b = float(np.float32(rng.standard_normal() * scale))
    return w, b


def random_score_maps(dims, seed: int, n_distinct: int = 64, pos_frac: float = 0.3):
    """Seeded score maps for NMS tests: list of float32[rows][cols].

    Values are drawn from a small set of distinct levels so that equal scores
    (ties) are common; about ``pos_frac`` of them are above 0.
    """
    rng = _rng(17, seed)
    levels = np.sort(rng.uniform(0.01, 1.0, n_distinct)).astype(np.float32)
    out = []
    for (rows, cols) in dims:
        v = levels[rng.integers(0, n_distinct, size=(rows, cols))]
        neg = rng.uniform(size=(rows, cols)) >= pos_frac
        out.append(np.where(neg, -v, v).astype(np.float32))
    return out
