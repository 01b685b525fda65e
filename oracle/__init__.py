"""Plain FP64 CPU oracle of the HOG+LBP sliding-window SVM detector (arXiv 1611.01642).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline may import this package; the product path never does. It shares no
code with the CUDA library (``paper_1611_01642_gb300``) and neither imports
the other. The numerics live in ``pd_oracle.c`` (double precision, built with
``-ffp-contract=off``); this module compiles it with gcc on first use and
wraps it with ctypes/numpy.

Every function below is a thin marshalling wrapper; see the C source for the
definitions and their paper citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpd_oracle.so")
_lock = threading.Lock()
_lib = None

HOG_BINS = 9
HOG_DIM = 36
LBP_BINS = 59
FEAT = 95
WIN_BW = 7
WIN_BH = 15
CLIP = 0.2


class Box(ctypes.Structure):
    _fields_ = [("x", ctypes.c_float), ("y", ctypes.c_float), ("w", ctypes.c_float),
                ("h", ctypes.c_float), ("score", ctypes.c_float), ("level", ctypes.c_int32),
                ("wx", ctypes.c_int32), ("wy", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile pd_oracle.c into oracle/_build/libpd_oracle.so (gcc, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i, d, f = ctypes.c_int, ctypes.c_double, ctypes.c_float
            lib.pdo_pyramid.argtypes = [i, i, d, i, P, P]
            lib.pdo_pyramid.restype = i
            lib.pdo_pyramid_up.argtypes = [i, i, d, i, i, P, P]
            lib.pdo_pyramid_up.restype = i
            lib.pdo_resize.argtypes = [P, i, i, i, P, i, i, i]
            lib.pdo_lbp_code.argtypes = [P, i, i, i, i, i]
            lib.pdo_lbp_code.restype = i
            lib.pdo_lbp_transitions.argtypes = [i]
            lib.pdo_lbp_bin.argtypes = [i]
            lib.pdo_lbp_cells.argtypes = [P, i, i, i, P]
            lib.pdo_gradient.argtypes = [P, i, i, i, i, i, P, P]
            lib.pdo_orientation_vote.argtypes = [d, P, P, P, P]
            lib.pdo_spatial_vote.argtypes = [i, i, P, P, P, P]
            lib.pdo_hog_cells.argtypes = [P, i, i, i, P]
            lib.pdo_block_spatial_vote.argtypes = [i, P, P, P, P]
            lib.pdo_hog_blocks.argtypes = [P, i, i, i, P]
            lib.pdo_block_features_pb.argtypes = [P, P, i, i, d, P]
            lib.pdo_l2hys.argtypes = [P, i, d]
            lib.pdo_block_features.argtypes = [P, P, i, i, d, P]
            lib.pdo_scores.argtypes = [P, i, i, P, d, P]
            lib.pdo_level_scores.argtypes = [P, i, i, i, P, d, d, P, P, P, P]
            lib.pdo_level_scores_ex.argtypes = [P, i, i, i, P, d, d, i, P, P, P, P]
            lib.pdo_window_descriptor_bruteforce.argtypes = [P, i, i, i, i, i, d, P]
            lib.pdo_window_box.argtypes = [i, i, i, i, i, i, P, P, P, P]
            lib.pdo_iou.argtypes = [P, P]
            lib.pdo_iou.restype = d
            lib.pdo_nms.argtypes = [P, i, P, P, P, P, i, i, f, d, i, P, P]
            lib.pdo_nms.restype = i
            lib.pdo_detect.argtypes = [P, i, i, i, d, P, d, d, f, d, i, i, P, P, P, P, P, P]
            lib.pdo_detect.restype = i
            lib.pdo_detect_up.argtypes = [P, i, i, i, d, i, P, d, d, f, d, i, i, P, P, P, P, P, P]
            lib.pdo_detect_up.restype = i
            lib.pdo_detect_ex.argtypes = [P, i, i, i, d, i, i, P, d, d, f, d, i, i, P, P, P, P, P, P]
            lib.pdo_detect_ex.restype = i
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _img(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    assert img.ndim == 2
    return img


# ----------------------------------------------------------------------------- pyramid
def pyramid(W: int, H: int, factor: float, max_levels: int = 1024, upscale: int = 0):
    """Level sizes [(Wk, Hk), ...] (Section 4.4; read of the stop rule), the
    `upscale` upsampled levels (most upsampled first) before the others."""
    lib = _load()
    wk = np.zeros(max_levels, np.int32)
    hk = np.zeros(max_levels, np.int32)
    n = lib.pdo_pyramid_up(W, H, float(factor), int(upscale), max_levels, _p(wk), _p(hk))
    if n < 0:
        raise ValueError("pyramid factor must be > 1")
    return [(int(wk[k]), int(hk[k])) for k in range(n)]


def resize(img: np.ndarray, Wk: int, Hk: int) -> np.ndarray:
    """Q11 fixed-point bilinear level straight from the frame (u8[Hk][Wk])."""
    lib = _load()
    img = _img(img)
    out = np.zeros((Hk, Wk), np.uint8)
    lib.pdo_resize(_p(img), img.shape[1], img.shape[0], img.shape[1], _p(out), Wk, Hk, Wk)
    return out


def pyramid_levels(img: np.ndarray, factor: float):
    img = _img(img)
    return [resize(img, wk, hk) for (wk, hk) in pyramid(img.shape[1], img.shape[0], factor)]


# ----------------------------------------------------------------------------- LBP
def lbp_code(L: np.ndarray, x: int, y: int) -> int:
    lib = _load()
    L = _img(L)
    return lib.pdo_lbp_code(_p(L), L.shape[1], L.shape[0], L.shape[1], x, y)


def lbp_codes(L: np.ndarray) -> np.ndarray:
    """LBP map (Algorithm 1) of a whole image, pixel by pixel."""
    L = _img(L)
    out = np.zeros(L.shape, np.uint8)
    for y in range(L.shape[0]):
        for x in range(L.shape[1]):
            out[y, x] = lbp_code(L, x, y)
    return out


def lbp_transitions(code: int) -> int:
    return _load().pdo_lbp_transitions(code)


def lbp_bin(code: int) -> int:
    return _load().pdo_lbp_bin(code)


def lbp_cells(L: np.ndarray) -> np.ndarray:
    """u8[Hc][Wc][59] cell counts (Algorithm 2)."""
    lib = _load()
    L = _img(L)
    Hc, Wc = L.shape[0] // 8, L.shape[1] // 8
    out = np.zeros((Hc, Wc, LBP_BINS), np.uint8)
    lib.pdo_lbp_cells(_p(L), L.shape[1], L.shape[0], L.shape[1], _p(out))
    return out


# ----------------------------------------------------------------------------- HOG
def gradient(L: np.ndarray, x: int, y: int):
    lib = _load()
    L = _img(L)
    m = np.zeros(1, np.float64)
    t = np.zeros(1, np.float64)
    lib.pdo_gradient(_p(L), L.shape[1], L.shape[0], L.shape[1], x, y, _p(m), _p(t))
    return float(m[0]), float(t[0])


def orientation_vote(theta_deg: float):
    lib = _load()
    b = np.zeros(2, np.int32)
    w = np.zeros(2, np.float64)
    lib.pdo_orientation_vote(float(theta_deg), _p(b[0:1]), _p(b[1:2]), _p(w[0:1]), _p(w[1:2]))
    return (int(b[0]), float(w[0])), (int(b[1]), float(w[1]))


def spatial_vote(p: int, n: int):
    lib = _load()
    c = np.zeros(2, np.int32)
    w = np.zeros(2, np.float64)
    lib.pdo_spatial_vote(p, n, _p(c[0:1]), _p(c[1:2]), _p(w[0:1]), _p(w[1:2]))
    return (int(c[0]), float(w[0])), (int(c[1]), float(w[1]))


def hog_cells(L: np.ndarray) -> np.ndarray:
    """f64[Hc][Wc][9] soft-binned cell histograms (Algorithms 4-5)."""
    lib = _load()
    L = _img(L)
    Hc, Wc = L.shape[0] // 8, L.shape[1] // 8
    out = np.zeros((Hc, Wc, HOG_BINS), np.float64)
    lib.pdo_hog_cells(_p(L), L.shape[1], L.shape[0], L.shape[1], _p(out))
    return out


def block_spatial_vote(l: int):
    """(c0, c1, w0, w1) of local coordinate l inside a 16-pixel block (cells -1 and 2 are outside it)."""
    lib = _load()
    c = np.zeros(2, np.int32)
    w = np.zeros(2, np.float64)
    lib.pdo_block_spatial_vote(l, _p(c[0:1]), _p(c[1:2]), _p(w[0:1]), _p(w[1:2]))
    return int(c[0]), int(c[1]), float(w[0]), float(w[1])


def hog_blocks(L: np.ndarray) -> np.ndarray:
    """f64[Hb][Wb][36] per-block HOG histograms (Algorithm 5, each block from its own pixels)."""
    lib = _load()
    L = _img(L)
    Hb, Wb = L.shape[0] // 8 - 1, L.shape[1] // 8 - 1
    out = np.zeros((max(Hb, 0), max(Wb, 0), HOG_DIM), np.float64)
    if Hb > 0 and Wb > 0:
        lib.pdo_hog_blocks(_p(L), L.shape[1], L.shape[0], L.shape[1], _p(out))
    return out


def l2hys(v: np.ndarray, clip: float = CLIP) -> np.ndarray:
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    lib.pdo_l2hys(_p(v), v.size, float(clip))
    return v


def block_features(hog: np.ndarray, lbp: np.ndarray, clip: float = CLIP) -> np.ndarray:
    """f64[Hb][Wb][95]: L2-Hys HOG block (36) then L1-sqrt LBP block (59)."""
    lib = _load()
    hog = np.ascontiguousarray(hog, dtype=np.float64)
    lbp = np.ascontiguousarray(lbp, dtype=np.uint8)
    Hc, Wc = hog.shape[:2]
    out = np.zeros((max(Hc - 1, 0), max(Wc - 1, 0), FEAT), np.float64)
    if Hc >= 2 and Wc >= 2:
        lib.pdo_block_features(_p(hog), _p(lbp), Hc, Wc, float(clip), _p(out))
    return out


def block_features_pb(hogb: np.ndarray, lbp: np.ndarray, clip: float = CLIP) -> np.ndarray:
    """f64[Hb][Wb][95] from per-block HOG histograms (hog_blocks) and LBP cell counts."""
    lib = _load()
    hogb = np.ascontiguousarray(hogb, dtype=np.float64)
    lbp = np.ascontiguousarray(lbp, dtype=np.uint8)
    Hc, Wc = lbp.shape[:2]
    assert hogb.shape == (Hc - 1, Wc - 1, HOG_DIM)
    out = np.zeros((Hc - 1, Wc - 1, FEAT), np.float64)
    lib.pdo_block_features_pb(_p(hogb), _p(lbp), Hc, Wc, float(clip), _p(out))
    return out


def scores(feat: np.ndarray, w: np.ndarray, bias: float) -> np.ndarray:
    """f64[Hb-14][Wb-6] window scores (Algorithm 6)."""
    lib = _load()
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(WIN_BH, WIN_BW, FEAT)
    Hb, Wb = feat.shape[:2]
    rows, cols = Hb - WIN_BH + 1, Wb - WIN_BW + 1
    if rows <= 0 or cols <= 0:
        return np.zeros((max(rows, 0), max(cols, 0)), np.float64)
    out = np.zeros((rows, cols), np.float64)
    lib.pdo_scores(_p(feat), Hb, Wb, _p(w), float(bias), _p(out))
    return out


def level_all(L: np.ndarray, w: np.ndarray, bias: float, clip: float = CLIP, per_block: bool = False):
    """(hog cells, lbp cells, block features, scores) of one level image; with
    per_block the first item is the per-block HOG histograms (hog_blocks)."""
    lbp = lbp_cells(L)
    if per_block:
        hog = hog_blocks(L)
        feat = block_features_pb(hog, lbp, clip)
    else:
        hog = hog_cells(L)
        feat = block_features(hog, lbp, clip)
    return hog, lbp, feat, scores(feat, w, bias)


def level_scores(L: np.ndarray, w: np.ndarray, bias: float, clip: float = CLIP) -> np.ndarray:
    return level_all(L, w, bias, clip)[3]


def window_descriptor_bruteforce(L: np.ndarray, wx: int, wy: int, clip: float = CLIP) -> np.ndarray:
    """f64[15][7][95] descriptor of one window straight from its pixels."""
    lib = _load()
    L = _img(L)
    out = np.zeros((WIN_BH, WIN_BW, FEAT), np.float64)
    lib.pdo_window_descriptor_bruteforce(_p(L), L.shape[1], L.shape[0], L.shape[1], wx, wy,
                                         float(clip), _p(out))
    return out


def window_descriptor(feat: np.ndarray, wx: int, wy: int) -> np.ndarray:
    return feat[wy:wy + WIN_BH, wx:wx + WIN_BW, :]


# ----------------------------------------------------------------------------- NMS / detect
def window_box(W, H, Wk, Hk, wx, wy):
    lib = _load()
    v = np.zeros(4, np.float32)
    lib.pdo_window_box(W, H, Wk, Hk, wx, wy, _p(v[0:1]), _p(v[1:2]), _p(v[2:3]), _p(v[3:4]))
    return tuple(float(t) for t in v)


def iou(a, b) -> float:
    lib = _load()
    A = Box(*a[:4], 0.0, 0, 0, 0)
    B = Box(*b[:4], 0.0, 0, 0, 0)
    return lib.pdo_iou(ctypes.byref(A), ctypes.byref(B))


def nms(score_maps, level_dims, W: int, H: int, threshold: float = 0.0, iou_thr: float = 0.5,
        max_boxes: int = 4096):
    """Greedy NMS over float32 score maps. Returns (boxes structured array, n_candidates)."""
    lib = _load()
    nl = len(score_maps)
    rows = np.array([m.shape[0] for m in score_maps], np.int32)
    cols = np.array([m.shape[1] for m in score_maps], np.int32)
    wk = np.array([d[0] for d in level_dims], np.int32)
    hk = np.array([d[1] for d in level_dims], np.int32)
    flat = np.concatenate([np.ascontiguousarray(m, np.float32).ravel() for m in score_maps]) \
        if nl else np.zeros(1, np.float32)
    flat = np.ascontiguousarray(flat, np.float32)
    out = (Box * max(max_boxes, 1))()
    ncand = ctypes.c_int(0)
    k = lib.pdo_nms(_p(flat), nl, _p(rows), _p(cols), _p(wk), _p(hk), W, H, float(threshold),
                    float(iou_thr), max_boxes, out, ctypes.byref(ncand))
    if k < 0:
        raise MemoryError("oracle nms")
    return boxes_to_array(out, k), ncand.value


BOX_DTYPE = np.dtype([("x", np.float32), ("y", np.float32), ("w", np.float32), ("h", np.float32),
                      ("score", np.float32), ("level", np.int32), ("wx", np.int32), ("wy", np.int32)])


def boxes_to_array(arr, k: int) -> np.ndarray:
    raw = np.frombuffer(bytes(memoryview(arr))[:k * ctypes.sizeof(Box)], dtype=BOX_DTYPE)
    return raw.copy()


def detect(img: np.ndarray, w: np.ndarray, bias: float, factor: float, threshold: float = 0.0,
           iou_thr: float = 0.5, max_boxes: int = 4096, clip: float = CLIP, upscale: int = 0,
           per_block: bool = False):
    """Whole plain path for one frame. Returns dict(levels, scores (list of f64 maps), boxes, n_candidates)."""
    lib = _load()
    img = _img(img)
    H, W = img.shape
    dims = pyramid(W, H, factor, upscale=upscale)
    total = sum(max(hk // 8 - WIN_BH, 0) * max(wk // 8 - WIN_BW, 0) for wk, hk in dims)
    sc = np.zeros(max(total, 1), np.float64)
    wk = np.zeros(1024, np.int32)
    hk = np.zeros(1024, np.int32)
    nl = ctypes.c_int(0)
    ncand = ctypes.c_int(0)
    out = (Box * max(max_boxes, 1))()
    w64 = np.ascontiguousarray(w, np.float64).reshape(-1)
    k = lib.pdo_detect_ex(_p(img), W, H, W, float(factor), int(upscale), int(per_block), _p(w64), float(bias),
                          float(clip),
                          float(threshold), float(iou_thr), max_boxes, 1024, ctypes.byref(nl), _p(wk),
                          _p(hk), _p(sc), out, ctypes.byref(ncand))
    if k < 0:
        raise MemoryError("oracle detect")
    maps = []
    off = 0
    for (a, b) in dims:
        r, c = b // 8 - WIN_BH, a // 8 - WIN_BW
        maps.append(sc[off:off + r * c].reshape(r, c))
        off += r * c
    return dict(levels=dims, scores=maps, boxes=boxes_to_array(out, k), n_candidates=ncand.value)
