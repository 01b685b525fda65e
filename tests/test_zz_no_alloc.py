"""The allocation-free NMS entry point against the handle-based one and the oracle.

pd_nms_noalloc serves callers that may not allocate device memory at run
time (a real-time frame loop that forbids allocation after start-up, a
plugin whose host framework owns all GPU memory): it keeps its scratch in a
static array inside the library instead of a pd_handle's arena. Its result
must be the result of pd_nms_maps on the same score maps and of the oracle's
greedy NMS with the same threshold, IoU and caps, and since every call reuses
the same array, two calls in a row must both be right.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_1611_01642_gb300")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _maps(seed, W, H):
    levels = oracle.pyramid(W, H, float(np.float32(1.05)))[:10]
    dims = [(hk // 8 - 15, wk // 8 - 7) for wk, hk in levels]
    maps = synth.random_score_maps(dims, seed, n_distinct=32, pos_frac=0.1)
    flat = np.concatenate([m.ravel() for m in maps]).astype(np.float32)
    return levels, dims, torch.from_numpy(flat).cuda()


def _boxes(t, n):
    return np.frombuffer(t.cpu().numpy().tobytes(), dtype=pd.BOX_DTYPE)[:n]


def test_noalloc_matches_handle_nms_twice():
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    det = pd.Detector(d["w"], float(d["b"]), max_frames=1, max_width=1242, max_height=375)
    try:
        for seed, (W, H) in [(11, (1242, 375)), (12, (900, 300))]:
            levels, dims, scores = _maps(seed, W, H)
            rows, cols = [r for r, _ in dims], [c for _, c in dims]
            ref_b = torch.zeros((4096, 8), dtype=torch.int32, device="cuda")
            ref_c = torch.zeros(2, dtype=torch.int32, device="cuda")
            pd.pd_nms_maps(det.h, scores, rows, cols, levels, W, H, ref_b, 4096, ref_c)
            got_b = torch.zeros((4096, 8), dtype=torch.int32, device="cuda")
            got_c = torch.zeros(2, dtype=torch.int32, device="cuda")
            pd.pd_nms_noalloc(scores, rows, cols, levels, W, H, 0.0, 0.5, 16384, got_b, 4096, got_c)
            torch.cuda.synchronize()
            rc, gc = ref_c.cpu().numpy().tolist(), got_c.cpu().numpy().tolist()
            assert gc == rc and rc[1] > 0 and rc[0] > 0
            assert np.array_equal(_boxes(got_b, gc[0]), _boxes(ref_b, rc[0]))
    finally:
        det.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    levels, dims, scores = _maps(13, 640, 480)
    b = torch.zeros((16, 8), dtype=torch.int32, device="cuda")
    c = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(pd.PDError) as e:
        pd.pd_nms_noalloc(scores, [r for r, _ in dims], [c_ for _, c_ in dims], levels, 640, 480,
                          0.0, 0.5, 16385, b, 16, c)
    assert e.value.code == pd.PD_EINVAL


def _oracle_boxes(levels, dims, scores, W, H, thr, iou, max_boxes):
    flat = scores.cpu().numpy()
    maps, off = [], 0
    for r, c in dims:
        maps.append(flat[off:off + r * c].reshape(r, c))
        off += r * c
    return oracle.nms(maps, levels, W, H, threshold=thr, iou_thr=iou, max_boxes=max_boxes)


def _same_boxes(got, ref):
    assert len(got) == len(ref)
    for name in ("x", "y", "w", "h", "score", "level", "wx", "wy"):
        assert np.array_equal(got[name], ref[name]), name


def test_noalloc_matches_oracle_nms_with_its_arguments_twice():
    """Non-default threshold and IoU, and a box cap that cuts the kept list: each call's result is
    the oracle's (Section 3's greedy suppression on the same float32 maps)."""
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    for seed, (W, H), thr, iou, cap in [(21, (1242, 375), 0.25, 0.3, 4096), (22, (700, 400), -0.1, 0.65, 4096),
                                        (23, (1242, 375), 0.0, 0.5, 7)]:
        levels, dims, scores = _maps(seed, W, H)
        rows, cols = [r for r, _ in dims], [c for _, c in dims]
        got_b = torch.zeros((4096, 8), dtype=torch.int32, device="cuda")
        got_c = torch.zeros(2, dtype=torch.int32, device="cuda")
        pd.pd_nms_noalloc(scores, rows, cols, levels, W, H, thr, iou, 16384, got_b, cap, got_c)
        torch.cuda.synchronize()
        ref, ncand = _oracle_boxes(levels, dims, scores, W, H, thr, iou, cap)
        gc = got_c.cpu().numpy().tolist()
        assert gc[1] == ncand and gc[0] == len(ref) and len(ref) > 0
        _same_boxes(_boxes(got_b, gc[0]), ref)


def test_noalloc_candidate_overflow_and_no_levels():
    """More candidates than max_candidates: counts (0, -candidates) and no boxes; zero levels:
    counts (0, 0). Each followed by a normal call on the same array."""
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    levels, dims, scores = _maps(31, 1242, 375)
    rows, cols = [r for r, _ in dims], [c for _, c in dims]
    _, ncand = _oracle_boxes(levels, dims, scores, 1242, 375, 0.0, 0.5, 4096)
    assert ncand > 8
    b = torch.zeros((64, 8), dtype=torch.int32, device="cuda")
    c = torch.full((2,), 7, dtype=torch.int32, device="cuda")
    pd.pd_nms_noalloc(scores, rows, cols, levels, 1242, 375, 0.0, 0.5, ncand - 1, b, 64, c)
    torch.cuda.synchronize()
    assert c.cpu().numpy().tolist() == [0, -ncand]
    pd.pd_nms_noalloc(scores, [], [], [], 1242, 375, 0.0, 0.5, 16384, b, 64, c)
    torch.cuda.synchronize()
    assert c.cpu().numpy().tolist() == [0, 0]
    pd.pd_nms_noalloc(scores, rows, cols, levels, 1242, 375, 0.0, 0.5, 16384, b, 64, c)
    torch.cuda.synchronize()
    ref, n2 = _oracle_boxes(levels, dims, scores, 1242, 375, 0.0, 0.5, 64)
    gc = c.cpu().numpy().tolist()
    assert gc == [len(ref), n2]
    _same_boxes(_boxes(b, gc[0]), ref)
