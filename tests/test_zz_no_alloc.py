"""The allocation-free NMS entry point against the handle-based one.

pd_nms_noalloc serves callers that may not allocate device memory at run
time (a real-time frame loop that forbids allocation after start-up, a
plugin whose host framework owns all GPU memory): it keeps its scratch in a
static array inside the library instead of a pd_handle's arena. Its result
must be the result of pd_nms_maps on the same score maps, and since every
call reuses the same array, two calls in a row must both be right.
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
