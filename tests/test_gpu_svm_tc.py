"""GPU tests of the tensor-core window-score kernel (K4 default) against the
oracle, the FP32 kernel and itself.

The tensor-core kernel computes every score as b plus the 105 template
position partial sums in a fixed order, so a frame's scores must not depend
on the batch it is in or on how the levels are cut into work items. A
one-hot template picks out a single feature (layout pin); a zero template
gives the bias exactly.
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
F105 = float(np.float32(1.05))


@pytest.fixture(scope="module")
def template():
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    return d["w"], float(d["b"])


def _planes(hog, lbp):
    Hc, Wc = hog.shape[:2]
    cp = max(16, ((Wc + 15) // 16) * 16)
    hp = np.zeros((9, Hc, cp), np.float32)
    hp[:, :, :Wc] = hog.transpose(2, 0, 1)
    lp = np.zeros((59, Hc, cp), np.uint8)
    lp[:, :, :Wc] = lbp.transpose(2, 0, 1)
    return hp, lp, cp, Hc * cp


def _window_scores(d, hog, lbp):
    Hc, Wc = hog.shape[:2]
    hp, lp, cp, plane = _planes(hog, lbp)
    rows, cols = Hc - 15, Wc - 7
    out = torch.full((rows * cols,), float("nan"), dtype=torch.float32, device="cuda")
    pd.pd_window_scores(d.h, torch.from_numpy(hp.ravel()).cuda(), plane, torch.from_numpy(lp.ravel()).cuda(),
                        plane, cp, Wc, Hc, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(rows, cols)


def _level(W, H, seed):
    L = synth.random_image(W, H, seed, smooth=True)
    hog = oracle.hog_cells(L).astype(np.float32)
    lbp = oracle.lbp_cells(L)
    feat = oracle.block_features(hog.astype(np.float64), lbp)
    return hog, lbp, feat


def test_one_hot_template_picks_one_feature():
    # template 1 at (i, j, t): score(wy, wx) = b + f[wy+i][wx+j][t]; strips of 104 windows and
    # items of at most 64 window rows are crossed (cols 105, rows 72)
    hog, lbp, feat = _level(900, 700, 11)
    for (i, j, t) in [(0, 0, 0), (14, 6, 94), (7, 3, 35), (3, 5, 36), (9, 1, 70)]:
        w = np.zeros((15, 7, 95), np.float32)
        w[i, j, t] = 1.0
        d = pd.Detector(w, 0.25, max_frames=1, max_width=64, max_height=128)
        try:
            got = _window_scores(d, hog, lbp).astype(np.float64)
        finally:
            d.close()
        rows, cols = got.shape
        ref = 0.25 + feat[i:i + rows, j:j + cols, t]
        assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref - 0.25) + 1e-6), (i, j, t)


def test_zero_template_gives_the_bias_exactly():
    hog, lbp, _ = _level(300, 260, 12)
    d = pd.Detector(np.zeros((15, 7, 95), np.float32), -1.5, max_frames=1, max_width=64, max_height=128)
    try:
        got = _window_scores(d, hog, lbp)
    finally:
        d.close()
    assert np.all(got == np.float32(-1.5))


@pytest.mark.parametrize("W,H", [(1242, 375), (1680, 200), (520, 900)])
def test_tensor_core_and_fp32_kernels_agree_with_the_oracle(template, W, H):
    w, b = template
    hog, lbp, feat = _level(W, H, 13 + W)
    ref = oracle.scores(feat, w, b)
    wabs = np.abs(w.astype(np.float64))
    rows, cols = ref.shape
    scale = abs(b) + np.array([[np.sum(np.abs(feat[y:y + 15, x:x + 7]) * wabs) for x in range(cols)]
                               for y in range(0, rows, max(rows // 6, 1))])
    got = {}
    for name, flags in [("tc", 0), ("fp32", pd.PD_FLAG_SVM_FP32)]:
        d = pd.Detector(w, b, max_frames=1, max_width=64, max_height=128, flags=flags)
        try:
            got[name] = _window_scores(d, hog, lbp).astype(np.float64)
        finally:
            d.close()
        sel = got[name][::max(rows // 6, 1)]
        err = np.abs(sel - ref[::max(rows // 6, 1)])
        assert np.all(err <= 1e-4 * scale), (name, float((err / scale).max()))
        full_err = np.abs(got[name] - ref) / (abs(b) + np.sum(wabs) * 1.0)
        assert np.isfinite(got[name]).all() and full_err.max() < 1e-4, name
    print(f"{W}x{H}: max |tc - fp32| {np.abs(got['tc'] - got['fp32']).max():.3g}, "
          f"max |tc - ref| {np.abs(got['tc'] - ref).max():.3g}")


def test_scores_do_not_depend_on_the_batch(template):
    w, b = template
    frames = [synth.make_scene(1242, 375, 2, 50), synth.make_scene(640, 480, 3, 51),
              synth.make_scene(1920, 1080, 3, 52)]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    d = pd.Detector(w, b, pyr_factor=F105, max_frames=3, max_width=1920, max_height=1080)
    try:
        d.detect(dev)
        assert d.sync() == pd.PD_OK
        batch = [torch.cat([m.reshape(-1) for m in d.score_maps(f)]).clone() for f in range(3)]
        for f in range(3):
            d.detect([dev[f]])
            assert d.sync() == pd.PD_OK
            alone = torch.cat([m.reshape(-1) for m in d.score_maps(0)])
            assert torch.equal(alone, batch[f]), f
    finally:
        d.close()
