"""GPU parity of per-block HOG (Algorithm 5 read per 16x16 block, Section 4.3)
against the oracle: the cells kernel's 36 block-restricted histogram planes
assembled into blocks (within 1e-4 of the block's mass), the tensor-core K4
fed per-block planes (scores within 1e-4 of the dot-product scale), and the
whole detector with PD_FLAG_HOG_PER_BLOCK (score maps and boxes), for the
HOGLBP-SVM and HOG-SVM pipelines.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_1611_01642_gb300")

from test_gpu_parity import F12, _check_boxes, _check_scores  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOG_TOL = 1e-4
SCORE_TOL = 1e-4


@pytest.fixture(scope="module")
def template():
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    return d["w"], float(d["b"])


@pytest.fixture(scope="module")
def det(template):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    h = pd.Detector(w, b, max_frames=1, max_width=64, max_height=128, flags=pd.PD_FLAG_HOG_PER_BLOCK)
    yield h, w, b
    h.close()


def _planes(Hc, Wc):
    cp = max(16, ((Wc + 15) // 16) * 16)
    return cp, max(Hc, 1) * cp


def _assemble(q, Hc, Wc):
    """Blocks [Hb][Wb][36] from the 36 planes [36][Hc][Wc] of the cells kernel."""
    q = q.reshape(4, 9, Hc, Wc)
    return np.concatenate([q[0, :, :-1, :-1], q[1, :, :-1, 1:], q[2, :, 1:, :-1], q[3, :, 1:, 1:]],
                          axis=0).transpose(1, 2, 0)


def _scatter(hb):
    """The inverse of _assemble: planes [36][Hc][Wc] holding the oracle's blocks (unused places 0)."""
    Hb, Wb = hb.shape[:2]
    q = np.zeros((4, 9, Hb + 1, Wb + 1), np.float32)
    t = hb.transpose(2, 0, 1).reshape(4, 9, Hb, Wb)
    q[0, :, :-1, :-1] = t[0]
    q[1, :, :-1, 1:] = t[1]
    q[2, :, 1:, :-1] = t[2]
    q[3, :, 1:, 1:] = t[3]
    return q.reshape(36, Hb + 1, Wb + 1)


@pytest.mark.parametrize("W,H", [(16, 16), (23, 17), (130, 200), (640, 480), (1242, 375), (1000, 70)])
def test_cells_kernel_per_block_histograms(det, W, H):
    h, _, _ = det
    L = synth.random_image(W, H, 5 * W + H, smooth=W > 100)
    Hc, Wc = H // 8, W // 8
    cp, plane = _planes(Hc, Wc)
    hog = torch.full((36 * plane,), float("nan"), dtype=torch.float32, device="cuda")
    lbp = torch.full((59 * plane,), 255, dtype=torch.uint8, device="cuda")
    pd.pd_cell_features(h.h, torch.from_numpy(L).cuda(), hog, plane, lbp, plane, cp)
    torch.cuda.synchronize()
    q = hog.cpu().numpy().reshape(36, max(Hc, 1), cp)[:, :Hc, :Wc]
    got = _assemble(q, Hc, Wc)
    ref = oracle.hog_blocks(L)
    assert got.shape == ref.shape
    tol = HOG_TOL * ref.sum(axis=2, keepdims=True) + 1e-6
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) - tol))
    lg = lbp.cpu().numpy().reshape(59, max(Hc, 1), cp)[:, :Hc, :Wc].transpose(1, 2, 0)
    assert np.array_equal(lg, oracle.lbp_cells(L))


@pytest.mark.parametrize("W,H", [(64, 128), (900, 700), (1242, 375)])
def test_tensor_core_k4_on_per_block_planes(det, W, H):
    h, w, b = det
    L = synth.random_image(W, H, 9 * W + H, smooth=True)
    hb = oracle.hog_blocks(L)
    lbp = oracle.lbp_cells(L)
    feat = oracle.block_features_pb(hb.astype(np.float32).astype(np.float64), lbp)
    ref = oracle.scores(feat, w, b)
    Hc, Wc = lbp.shape[:2]
    cp, plane = _planes(Hc, Wc)
    hp = np.zeros((36, Hc, cp), np.float32)
    hp[:, :, :Wc] = _scatter(hb)
    lp = np.zeros((59, Hc, cp), np.uint8)
    lp[:, :, :Wc] = lbp.transpose(2, 0, 1)
    rows, cols = ref.shape
    out = torch.full((rows * cols,), float("nan"), dtype=torch.float32, device="cuda")
    pd.pd_window_scores(h.h, torch.from_numpy(hp.ravel()).cuda(), plane, torch.from_numpy(lp.ravel()).cuda(),
                        plane, cp, Wc, Hc, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(rows, cols).astype(np.float64)
    wabs = np.abs(w.astype(np.float64))
    step = max(rows // 8, 1)
    scale = abs(b) + np.array([[np.sum(np.abs(feat[y:y + 15, x:x + 7]) * wabs) for x in range(cols)]
                               for y in range(0, rows, step)])
    assert np.all(np.abs(got[::step] - ref[::step]) <= SCORE_TOL * scale)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= SCORE_TOL * (abs(b) + wabs.sum())


@pytest.mark.parametrize("hog_only", [False, True])
def test_detector_per_block_matches_oracle(template, hog_only):
    w, b = template
    W, H = 640, 480
    img = synth.make_scene(W, H, 3, 71)
    wm = w.copy()
    flags = pd.PD_FLAG_HOG_PER_BLOCK
    if hog_only:
        wm[:, :, 36:] = 0.0
        flags |= pd.PD_FLAG_HOG_ONLY
    d = pd.Detector(w, b, max_frames=1, max_width=W, max_height=H, pyr_factor=F12, flags=flags)
    try:
        d.detect([torch.from_numpy(img).cuda()])
        assert d.sync() == pd.PD_OK
        dims = [(lv["width"], lv["height"]) for lv in d.levels(0)]
        assert dims == oracle.pyramid(W, H, F12)
        ref = oracle.detect(img, wm, b, F12, per_block=True)
        feats = []
        for k, ((wk, hk), g) in enumerate(zip(dims, d.score_maps(0))):
            L = oracle.resize(img, wk, hk)
            _, _, feat, sc = oracle.level_all(L, wm, b, per_block=True)
            feats.append(feat)
            _check_scores(g.cpu().numpy(), feat, wm, b, sc, f"per-block level {k}")
        _check_boxes(d.boxes(0), ref["scores"], feats, dims, wm, b, W, H)
    finally:
        d.close()


def test_per_block_scores_differ_from_shared_cells(template):
    # the two readings of Algorithm 5 give different features, so different scores
    w, b = template
    img = synth.make_scene(320, 240, 2, 72)
    maps = []
    for flags in [0, pd.PD_FLAG_HOG_PER_BLOCK]:
        d = pd.Detector(w, b, max_frames=1, max_width=320, max_height=240, pyr_factor=F12, flags=flags)
        try:
            d.detect([torch.from_numpy(img).cuda()])
            assert d.sync() == pd.PD_OK
            maps.append(d.score_maps(0)[0].cpu().numpy().copy())
        finally:
            d.close()
    assert maps[0].shape == maps[1].shape
    assert np.abs(maps[0] - maps[1]).max() > 1e-3
