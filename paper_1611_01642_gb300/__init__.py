"""GB300 (sm_103a) HOG+LBP sliding-window SVM pedestrian detector (arXiv 1611.01642).

Python binding of the C ABI in ``include/pd.h``: the functions below carry
the C names and only marshal arguments (torch tensors -> device pointers,
numpy arrays -> host pointers, the current torch stream -> cudaStream_t).
Every step of the detector runs in the CUDA kernels of ``libpd.so``; there is
no Python or CPU fallback, and importing the binding fails loudly when the
library has not been built (``python -m paper_1611_01642_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

PD_OK = 0
PD_EINVAL = -1
PD_ENOMEM = -2
PD_ECUDA = -3
PD_ETIMEOUT = -4
PD_EBOUNDS = -5
PD_ESTATE = -6
PD_EOVERFLOW = -7
ERROR_NAMES = {0: "PD_OK", -1: "PD_EINVAL", -2: "PD_ENOMEM", -3: "PD_ECUDA", -4: "PD_ETIMEOUT",
               -5: "PD_EBOUNDS", -6: "PD_ESTATE", -7: "PD_EOVERFLOW"}
HOG_BINS, LBP_BINS, FEAT, WIN_BW, WIN_BH = 9, 59, 95, 7, 15
MAX_LEVELS = 96
PD_FLAG_STAGE_TIMING = 1
PD_FLAG_SVM_FP32 = 2
PD_FLAG_HOG_ONLY = 4
PD_FLAG_LBP_ONLY = 8
PD_FLAG_HOG_PER_BLOCK = 16
TILE_SHAPES = 7
TILE_SHAPE_DIMS = [(32, 16), (64, 8), (32, 8), (64, 4), (64, 2), (32, 12), (32, 4)]  # windows per K4 tile (x, y)

EXPORTED = ["pd_params_default", "pd_pyramid", "pd_create", "pd_destroy", "pd_last_error",
            "pd_detect", "pd_detect_host", "pd_sync", "pd_frame_candidates", "pd_frame_levels", "pd_scores", "pd_boxes",
            "pd_last_launch_count", "pd_stage_times", "pd_set_tile_costs", "pd_get_tile_costs", "pd_resize_levels", "pd_cell_features", "pd_window_scores",
            "pd_nms_maps", "pd_nms_noalloc", "pd_cnn_set_params", "pd_cnn_get_params", "pd_cnn_forward",
            "pd_cnn_train_step", "pd_cnn_train_loss", "pd_set_proposal", "pd_set_proposal_levels",
            "pd_set_tuning", "pd_get_tuning",
            "pd_logits", "pd_pyramid_ex",
            "pd_scheme_cells", "pd_scheme_window_scores"]


class pd_params(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("pyr_factor", ctypes.c_float),
                ("l2hys_clip", ctypes.c_float), ("threshold", ctypes.c_float),
                ("nms_iou", ctypes.c_float), ("max_boxes_per_frame", ctypes.c_int32),
                ("max_candidates_per_frame", ctypes.c_int32), ("max_frames", ctypes.c_int32),
                ("max_width", ctypes.c_int32), ("max_height", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("use_proposal", ctypes.c_int32),
                ("keep_logit_threshold", ctypes.c_float), ("upscale_levels", ctypes.c_int32),
                ("proposal_level_step", ctypes.c_int32)]


class pd_tuning(ctypes.Structure):
    _fields_ = [("k1_groups", ctypes.c_int32), ("tc_item_rows", ctypes.c_int32)]


class pd_box(ctypes.Structure):
    _fields_ = [("x", ctypes.c_float), ("y", ctypes.c_float), ("w", ctypes.c_float),
                ("h", ctypes.c_float), ("score", ctypes.c_float), ("level", ctypes.c_int32),
                ("wx", ctypes.c_int32), ("wy", ctypes.c_int32)]


class pd_level_info(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("cells_x", ctypes.c_int32),
                ("cells_y", ctypes.c_int32), ("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
                ("score_offset", ctypes.c_int64)]


BOX_DTYPE = np.dtype([("x", np.float32), ("y", np.float32), ("w", np.float32), ("h", np.float32),
                      ("score", np.float32), ("level", np.int32), ("wx", np.int32), ("wy", np.int32)])


class PDError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load(path: str | None = None):
    """Loads libpd.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libpd.so not built at {path}; run `python -m paper_1611_01642_gb300.build`")
    lib = ctypes.CDLL(path)
    P, i, f, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_int64
    sig = {
        "pd_params_default": ([P], i),
        "pd_pyramid": ([i, i, f, i, P, P], i),
        "pd_pyramid_ex": ([i, i, f, i, i, P, P], i),
        "pd_create": ([P, P, f, P], i),
        "pd_destroy": ([P], None),
        "pd_last_error": ([P], ctypes.c_char_p),
        "pd_detect": ([P, P, i, P, P, P, P], i),
        "pd_detect_host": ([P, P, i, P, P, P, P], i),
        "pd_sync": ([P], i),
        "pd_frame_candidates": ([P, i, P], i),
        "pd_frame_levels": ([P, i, P, P], i),
        "pd_scores": ([P, P, P], i),
        "pd_boxes": ([P, i, P, i, P], i),
        "pd_last_launch_count": ([P], i),
        "pd_stage_times": ([P, P], i),
        "pd_set_tile_costs": ([P, P], i),
        "pd_get_tile_costs": ([P, P], i),
        "pd_resize_levels": ([P, P, P, i, i, i, i, P, P, P, P, P], i),
        "pd_cell_features": ([P, P, P, i, i, i, P, i64, P, i64, i], i),
        "pd_window_scores": ([P, P, P, i64, P, i64, i, i, i, P], i),
        "pd_scheme_cells": ([P, P, i, P, i, i, i, P, i64, P, i64, i], i),
        "pd_scheme_window_scores": ([P, P, i, P, i64, P, i64, i, i, i, P], i),
        "pd_nms_maps": ([P, P, P, i, P, P, P, P, i, i, P, i, P], i),
        "pd_nms_noalloc": ([P, P, i, P, P, P, P, i, i, f, f, i, P, i, P], i),
        "pd_cnn_set_params": ([P, P, i], i),
        "pd_cnn_get_params": ([P, P, P, i], i),
        "pd_cnn_forward": ([P, P, P, i, i, i, P, i, P], i),
        "pd_cnn_train_step": ([P, P, f, f, f], i),
        "pd_cnn_train_loss": ([P, P, P], i),
        "pd_set_proposal": ([P, i, f], i),
        "pd_set_proposal_levels": ([P, i], i),
        "pd_set_tuning": ([P, P], i),
        "pd_get_tuning": ([P, P], i),
        "pd_logits": ([P, P, P], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(t) -> int:
    return int(t.data_ptr())


def _np(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream=None) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return int(getattr(stream, "cuda_stream", stream))


def _check(code, handle=None):
    if code != PD_OK:
        msg = load().pd_last_error(handle).decode() if handle else ""
        raise PDError(code, msg)
    return code


# ----------------------------------------------------------------------------- C-named wrappers
def pd_params_default(**overrides) -> pd_params:
    p = pd_params()
    _check(load().pd_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def pd_pyramid(W: int, H: int, factor: float, max_levels: int = MAX_LEVELS, upscale_levels: int = 0):
    wk = np.zeros(max_levels, np.int32)
    hk = np.zeros(max_levels, np.int32)
    n = load().pd_pyramid_ex(W, H, float(factor), int(upscale_levels), max_levels,
                             wk.ctypes.data_as(ctypes.c_void_p), hk.ctypes.data_as(ctypes.c_void_p))
    if n < 0:
        raise PDError(n, "pd_pyramid")
    return [(int(wk[k]), int(hk[k])) for k in range(n)]


def pd_create(params: pd_params, svm_w: np.ndarray, svm_b: float):
    w, wp = _np(svm_w, np.float32)
    assert w.size == WIN_BH * WIN_BW * FEAT
    h = ctypes.c_void_p()
    _check(load().pd_create(ctypes.byref(params), wp, float(svm_b), ctypes.byref(h)))
    return h


def pd_destroy(h) -> None:
    load().pd_destroy(h)


def pd_last_error(h) -> str:
    return load().pd_last_error(h).decode()


def pd_detect(h, frames, stream=None) -> None:
    """frames: list of 2-D uint8 CUDA tensors (row stride = pitch)."""
    n = len(frames)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[_ptr(f) for f in frames])
    w, wp = _np([f.shape[1] for f in frames], np.int32)
    hh, hp = _np([f.shape[0] for f in frames], np.int32)
    pi, pp = _np([f.stride(0) for f in frames], np.int32)
    _check(load().pd_detect(h, _stream(stream), n, ptrs, wp, hp, pp), h)


def pd_detect_host(h, frames, stream=None) -> None:
    """frames: list of 2-D uint8 host arrays (numpy, or pinned CPU tensors)."""
    n = len(frames)
    addrs, keep = [], []
    ws, hs, ps = [], [], []
    for f in frames:
        if isinstance(f, np.ndarray):
            a = np.ascontiguousarray(f, np.uint8)
            keep.append(a)
            addrs.append(a.ctypes.data)
            ws.append(a.shape[1]); hs.append(a.shape[0]); ps.append(a.strides[0])
        else:
            addrs.append(_ptr(f))
            ws.append(f.shape[1]); hs.append(f.shape[0]); ps.append(f.stride(0))
    ptrs = (ctypes.c_void_p * max(n, 1))(*addrs)
    w, wp = _np(ws, np.int32)
    hh, hp = _np(hs, np.int32)
    pi, pp = _np(ps, np.int32)
    _check(load().pd_detect_host(h, _stream(stream), n, ptrs, wp, hp, pp), h)


def pd_sync(h) -> int:
    """Waits for the last detect; returns the status code (PD_OK or a PD_E* code)."""
    return load().pd_sync(h)


def pd_frame_candidates(h, frame: int) -> int:
    n = ctypes.c_int(0)
    _check(load().pd_frame_candidates(h, frame, ctypes.byref(n)), h)
    return n.value


def pd_frame_levels(h, frame: int):
    info = (pd_level_info * MAX_LEVELS)()
    n = ctypes.c_int(0)
    _check(load().pd_frame_levels(h, frame, ctypes.byref(n), info), h)
    return [dict(width=info[k].width, height=info[k].height, cells_x=info[k].cells_x,
                 cells_y=info[k].cells_y, rows=info[k].rows, cols=info[k].cols,
                 score_offset=info[k].score_offset) for k in range(n.value)]


def pd_scores(h):
    """(device pointer, number of floats) of the score buffer."""
    p = ctypes.c_void_p()
    total = ctypes.c_int64()
    _check(load().pd_scores(h, ctypes.byref(p), ctypes.byref(total)), h)
    return p.value or 0, total.value


def pd_boxes(h, frame: int, cap: int = 4096) -> np.ndarray:
    """Kept boxes of one frame as a BOX_DTYPE array (at most cap of them)."""
    count = ctypes.c_int(0)
    lib = load()
    _check(lib.pd_boxes(h, frame, None, 0, ctypes.byref(count)), h)
    out = np.empty(min(count.value, cap), dtype=BOX_DTYPE)
    if out.size:
        _check(lib.pd_boxes(h, frame, out.ctypes.data_as(ctypes.c_void_p), out.size, ctypes.byref(count)), h)
    return out


def pd_last_launch_count(h) -> int:
    return load().pd_last_launch_count(h)


def pd_stage_times(h):
    """[K1, K2/K3, K4, K5, proposal] device milliseconds of the last detect (needs PD_FLAG_STAGE_TIMING)."""
    ms = np.zeros(5, np.float32)
    _check(load().pd_stage_times(h, ms.ctypes.data_as(ctypes.c_void_p)), h)
    return [float(v) for v in ms]


def pd_set_tile_costs(h, costs) -> None:
    c, cp = _np(costs, np.float32)
    assert c.size == TILE_SHAPES
    _check(load().pd_set_tile_costs(h, cp), h)


def pd_get_tile_costs(h):
    c = np.zeros(TILE_SHAPES, np.float32)
    _check(load().pd_get_tile_costs(h, c.ctypes.data_as(ctypes.c_void_p)), h)
    return [float(v) for v in c]


def pd_resize_levels(h, frame, level_dims, out, offsets, pitches, stream=None) -> None:
    """frame: 2-D uint8 CUDA tensor; out: uint8 CUDA buffer; offsets/pitches per level."""
    n = len(level_dims)
    wk, wkp = _np([d[0] for d in level_dims], np.int32)
    hk, hkp = _np([d[1] for d in level_dims], np.int32)
    of, ofp = _np(offsets, np.int64)
    pi, pip = _np(pitches, np.int32)
    _check(load().pd_resize_levels(h, _stream(stream), _ptr(frame), frame.shape[1], frame.shape[0],
                                   frame.stride(0), n, wkp, hkp, _ptr(out), ofp, pip), h)


def pd_cell_features(h, level, hog, hog_plane: int, lbp, lbp_plane: int, cell_pitch: int,
                     stream=None) -> None:
    _check(load().pd_cell_features(h, _stream(stream), _ptr(level), level.shape[1], level.shape[0],
                                   level.stride(0), _ptr(hog), hog_plane, _ptr(lbp), lbp_plane,
                                   cell_pitch), h)


def pd_window_scores(h, hog, hog_plane: int, lbp, lbp_plane: int, cell_pitch: int, cells_x: int,
                     cells_y: int, scores, stream=None) -> None:
    _check(load().pd_window_scores(h, _stream(stream), _ptr(hog), hog_plane, _ptr(lbp), lbp_plane,
                                   cell_pitch, cells_x, cells_y, _ptr(scores)), h)


# The paper's kernel schemes (comparison with the fused kernels; see include/pd.h).
PD_SCHEME_LBP_NAIVE, PD_SCHEME_LBP_SCALABLE = 1, 2
PD_SCHEME_HOG_GLOBAL, PD_SCHEME_HOG_LOCAL, PD_SCHEME_HOG_SHARED = 3, 4, 5
PD_SCHEME_SVM_NAIVE, PD_SCHEME_SVM_WARP = 6, 7


def pd_scheme_cells(h, scheme: int, level, hog, hog_plane: int, lbp, lbp_plane: int, cell_pitch: int,
                    stream=None) -> None:
    _check(load().pd_scheme_cells(h, _stream(stream), scheme, _ptr(level), level.shape[1], level.shape[0],
                                  level.stride(0), _ptr(hog) if hog is not None else None, hog_plane,
                                  _ptr(lbp) if lbp is not None else None, lbp_plane, cell_pitch), h)


def pd_scheme_window_scores(h, scheme: int, hog, hog_plane: int, lbp, lbp_plane: int, cell_pitch: int,
                            cells_x: int, cells_y: int, scores, stream=None) -> None:
    _check(load().pd_scheme_window_scores(h, _stream(stream), scheme, _ptr(hog), hog_plane, _ptr(lbp), lbp_plane,
                                          cell_pitch, cells_x, cells_y, _ptr(scores)), h)


def pd_nms_maps(h, scores, rows, cols, level_dims, W: int, H: int, boxes, max_boxes: int, counts,
                stream=None) -> None:
    n = len(rows)
    r, rp = _np(rows, np.int32)
    c, cp = _np(cols, np.int32)
    wk, wkp = _np([d[0] for d in level_dims], np.int32)
    hk, hkp = _np([d[1] for d in level_dims], np.int32)
    _check(load().pd_nms_maps(h, _stream(stream), _ptr(scores), n, rp, cp, wkp, hkp, W, H, _ptr(boxes),
                              max_boxes, _ptr(counts)), h)


def pd_nms_noalloc(scores, rows, cols, level_dims, W: int, H: int, threshold: float, nms_iou: float,
                   max_candidates: int, boxes, max_boxes: int, counts, stream=None) -> None:
    """NMS with no handle and no device allocation (scratch inside the library)."""
    n = len(rows)
    r, rp = _np(rows, np.int32)
    c, cp = _np(cols, np.int32)
    wk, wkp = _np([d[0] for d in level_dims], np.int32)
    hk, hkp = _np([d[1] for d in level_dims], np.int32)
    _check(load().pd_nms_noalloc(_stream(stream), _ptr(scores), n, rp, cp, wkp, hkp, W, H,
                                 float(threshold), float(nms_iou), max_candidates, _ptr(boxes),
                                 max_boxes, _ptr(counts)))


CNN_PARAMS = 14210


def pd_cnn_set_params(h, params) -> None:
    p, pp = _np(params, np.float32)
    assert p.size == CNN_PARAMS
    _check(load().pd_cnn_set_params(h, pp, CNN_PARAMS), h)


def pd_cnn_get_params(h):
    """(master parameters, gradient of the last training step) as float32 arrays."""
    p = np.zeros(CNN_PARAMS, np.float32)
    g = np.zeros(CNN_PARAMS, np.float32)
    _check(load().pd_cnn_get_params(h, p.ctypes.data_as(ctypes.c_void_p), g.ctypes.data_as(ctypes.c_void_p),
                                    CNN_PARAMS), h)
    return p, g


def pd_cnn_forward(h, level, hmap, h_pitch: int, logits, stream=None) -> None:
    _check(load().pd_cnn_forward(h, _stream(stream), _ptr(level), level.shape[1], level.shape[0], level.stride(0),
                                 _ptr(hmap), h_pitch, _ptr(logits)), h)


def pd_cnn_train_step(h, pos_weight: float, label_threshold: float, lr: float, stream=None) -> None:
    _check(load().pd_cnn_train_step(h, _stream(stream), float(pos_weight), float(label_threshold), float(lr)), h)


def pd_cnn_train_loss(h, stream=None) -> float:
    v = ctypes.c_float(0)
    _check(load().pd_cnn_train_loss(h, _stream(stream), ctypes.byref(v)), h)
    return float(v.value)


def pd_set_proposal(h, enable: bool, keep_logit_threshold: float) -> None:
    _check(load().pd_set_proposal(h, 1 if enable else 0, float(keep_logit_threshold)), h)


def pd_set_tuning(h, k1_groups: int, tc_item_rows: int) -> None:
    """Launch shapes of the default path (pyramid column groups per warp task, tensor-core score
    kernel window rows per item); results do not depend on them."""
    t = pd_tuning(int(k1_groups), int(tc_item_rows))
    _check(load().pd_set_tuning(h, ctypes.byref(t)), h)


def pd_get_tuning(h) -> dict:
    t = pd_tuning()
    _check(load().pd_get_tuning(h, ctypes.byref(t)), h)
    return {"k1_groups": t.k1_groups, "tc_item_rows": t.tc_item_rows}


def pd_set_proposal_levels(h, level_step: int) -> None:
    """The proposal network runs on every level_step-th level; the others read its head map."""
    _check(load().pd_set_proposal_levels(h, int(level_step)), h)


def pd_logits(h):
    p = ctypes.c_void_p()
    total = ctypes.c_int64()
    _check(load().pd_logits(h, ctypes.byref(p), ctypes.byref(total)), h)
    return p.value or 0, total.value


# ----------------------------------------------------------------------------- convenience
class Detector:
    """Owns a pd_handle: ``Detector(w, b, max_frames=..., max_width=..., ...)``.

    Keyword arguments are pd_params fields (pyr_factor, upscale_levels, threshold,
    nms_iou, max_boxes_per_frame, max_candidates_per_frame, flags, ...). flags
    selects the pipeline (PD_FLAG_HOG_ONLY, PD_FLAG_LBP_ONLY), per-block HOG
    (PD_FLAG_HOG_PER_BLOCK), the FP32 window-score kernel (PD_FLAG_SVM_FP32)
    and per-stage timing (PD_FLAG_STAGE_TIMING)."""

    def __init__(self, svm_w, svm_b, **params):
        self.params = pd_params_default(**params)
        self.h = pd_create(self.params, svm_w, svm_b)

    def close(self):
        if self.h:
            pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def detect(self, frames, stream=None):
        pd_detect(self.h, frames, stream)

    def set_proposal(self, enable: bool, keep_logit_threshold: float = 0.0, level_step: int | None = None):
        """Sparse path on/off (needs proposal parameters set with pd_cnn_set_params); level_step:
        the network runs on every level_step-th level of a frame (None: unchanged)."""
        if level_step is not None:
            pd_set_proposal_levels(self.h, level_step)
        pd_set_proposal(self.h, enable, keep_logit_threshold)

    def detect_host(self, frames, stream=None):
        pd_detect_host(self.h, frames, stream)

    def sync(self) -> int:
        return pd_sync(self.h)

    def levels(self, frame: int):
        return pd_frame_levels(self.h, frame)

    def boxes(self, frame: int) -> np.ndarray:
        return pd_boxes(self.h, frame, self.params.max_boxes_per_frame)

    def logit_maps(self, frame: int):
        """Keep-logit maps of the last detect with the proposal on (views, like score_maps)."""
        return self._maps(frame, *pd_logits(self.h))

    def score_maps(self, frame: int):
        """List of float32 CUDA tensors (views into the handle's score buffer)."""
        return self._maps(frame, *pd_scores(self.h))

    def _maps(self, frame: int, ptr: int, total: int):
        import torch
        if total == 0:
            return [torch.zeros((lv["rows"], lv["cols"]), dtype=torch.float32, device="cuda")
                    for lv in self.levels(frame)]
        buf = _device_view(ptr, total)
        return [buf[lv["score_offset"]:lv["score_offset"] + lv["rows"] * lv["cols"]].view(
            lv["rows"], lv["cols"]) for lv in self.levels(frame)]


def _device_view(ptr: int, n_floats: int):
    """A float32 torch view of library-owned device memory (no copy)."""
    import torch

    class _Arr:
        __cuda_array_interface__ = {"shape": (n_floats,), "typestr": "<f4", "data": (ptr, False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Arr(), device="cuda")
