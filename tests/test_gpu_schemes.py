"""GPU parity of the paper's kernel schemes (LBP Naive / Scalable, HOG Global /
Local / Shared, Naive and Warp-level SVM) re-expressed over the same readings
as the fused kernels: the same oracle and the same bars (LBP bit-exact, HOG
cells within 1e-4 of the cell's mass, window scores within 1e-4 of the
dot-product scale), at sizes that span several CTAs and ragged edges.
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
HOG_TOL = 1e-4
SCORE_TOL = 1e-4


@pytest.fixture(scope="module")
def det():
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    h = pd.Detector(d["w"], float(d["b"]), max_frames=1, max_width=64, max_height=128)
    yield h, d["w"], float(d["b"])
    h.close()


def _planes(Hc, Wc):
    cp = max(16, ((Wc + 15) // 16) * 16)
    plane = max(Hc, 1) * cp
    return cp, plane


@pytest.mark.parametrize("scheme", [pd.PD_SCHEME_LBP_NAIVE, pd.PD_SCHEME_LBP_SCALABLE])
@pytest.mark.parametrize("W,H", [(8, 8), (127, 129), (640, 480), (1242, 375)])
def test_lbp_schemes_bit_exact(det, scheme, W, H):
    h, _, _ = det
    L = synth.random_image(W, H, 7 * W + H, smooth=W > 100)
    Hc, Wc = H // 8, W // 8
    cp, plane = _planes(Hc, Wc)
    lbp = torch.full((59 * plane,), 255, dtype=torch.uint8, device="cuda")
    pd.pd_scheme_cells(h.h, scheme, torch.from_numpy(L).cuda(), None, 0, lbp, plane, cp)
    torch.cuda.synchronize()
    got = lbp.cpu().numpy().reshape(59, max(Hc, 1), cp)[:, :Hc, :Wc].transpose(1, 2, 0)
    assert np.array_equal(got, oracle.lbp_cells(L))


@pytest.mark.parametrize("scheme", [pd.PD_SCHEME_HOG_GLOBAL, pd.PD_SCHEME_HOG_LOCAL, pd.PD_SCHEME_HOG_SHARED])
@pytest.mark.parametrize("W,H", [(8, 8), (23, 17), (130, 200), (640, 480)])
def test_hog_schemes_within_tolerance(det, scheme, W, H):
    h, _, _ = det
    L = synth.random_image(W, H, 3 * W + H, smooth=W > 100)
    Hc, Wc = H // 8, W // 8
    cp, plane = _planes(Hc, Wc)
    hog = torch.full((9 * plane,), float("nan"), dtype=torch.float32, device="cuda")
    pd.pd_scheme_cells(h.h, scheme, torch.from_numpy(L).cuda(), hog, plane, None, 0, cp)
    torch.cuda.synchronize()
    got = hog.cpu().numpy().reshape(9, max(Hc, 1), cp)[:, :Hc, :Wc].transpose(1, 2, 0)
    ref = oracle.hog_cells(L)
    tol = HOG_TOL * ref.sum(axis=2, keepdims=True) + 1e-6
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) - tol))


@pytest.mark.parametrize("scheme", [pd.PD_SCHEME_SVM_NAIVE, pd.PD_SCHEME_SVM_WARP])
@pytest.mark.parametrize("W,H", [(64, 128), (300, 260), (1242, 375)])
def test_svm_schemes_within_tolerance(det, scheme, W, H):
    h, w, b = det
    L = synth.random_image(W, H, 11 * W + H, smooth=True)
    hog = oracle.hog_cells(L).astype(np.float32)
    lbp = oracle.lbp_cells(L)
    feat = oracle.block_features(hog.astype(np.float64), lbp)
    ref = oracle.scores(feat, w, b)
    Hc, Wc = hog.shape[:2]
    cp, plane = _planes(Hc, Wc)
    hp = np.zeros((9, Hc, cp), np.float32)
    hp[:, :, :Wc] = hog.transpose(2, 0, 1)
    lp = np.zeros((59, Hc, cp), np.uint8)
    lp[:, :, :Wc] = lbp.transpose(2, 0, 1)
    rows, cols = ref.shape
    out = torch.full((rows * cols,), float("nan"), dtype=torch.float32, device="cuda")
    pd.pd_scheme_window_scores(h.h, scheme, torch.from_numpy(hp.ravel()).cuda(), plane,
                               torch.from_numpy(lp.ravel()).cuda(), plane, cp, Wc, Hc, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(rows, cols).astype(np.float64)
    wabs = np.abs(w.astype(np.float64))
    scale = np.abs(b) + np.array([[np.sum(np.abs(feat[y:y + 15, x:x + 7]) * wabs) for x in range(cols)]
                                  for y in range(rows)])
    assert np.all(np.abs(got - ref) <= SCORE_TOL * scale), float(np.max(np.abs(got - ref) / scale))


def test_scheme_arguments_are_checked(det):
    h, _, _ = det
    L = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    lbp = torch.zeros((59 * 32,), dtype=torch.uint8, device="cuda")
    with pytest.raises(pd.PDError) as e:
        pd.pd_scheme_cells(h.h, 99, L, None, 0, lbp, 32, 16)
    assert e.value.code == pd.PD_EINVAL
    with pytest.raises(pd.PDError):  # an LBP scheme without LBP planes
        pd.pd_scheme_cells(h.h, pd.PD_SCHEME_LBP_NAIVE, L, None, 0, None, 32, 16)


@pytest.fixture(scope="module")
def det_pb():
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    h = pd.Detector(d["w"], float(d["b"]), max_frames=1, max_width=64, max_height=128,
                    flags=pd.PD_FLAG_HOG_PER_BLOCK)
    yield h, d["w"], float(d["b"])
    h.close()


@pytest.mark.parametrize("scheme", [pd.PD_SCHEME_HOG_GLOBAL, pd.PD_SCHEME_HOG_LOCAL, pd.PD_SCHEME_HOG_SHARED])
@pytest.mark.parametrize("W,H", [(16, 16), (23, 17), (130, 200), (640, 480)])
def test_hog_block_schemes_within_tolerance(det_pb, scheme, W, H):
    # Algorithm 5 as the paper lays it out: one thread per block histogram
    h, _, _ = det_pb
    L = synth.random_image(W, H, 13 * W + H, smooth=W > 100)
    Hc, Wc = H // 8, W // 8
    cp, plane = _planes(Hc, Wc)
    hog = torch.full((36 * plane,), float("nan"), dtype=torch.float32, device="cuda")
    pd.pd_scheme_cells(h.h, scheme, torch.from_numpy(L).cuda(), hog, plane, None, 0, cp)
    torch.cuda.synchronize()
    q = hog.cpu().numpy().reshape(4, 9, max(Hc, 1), cp)[:, :, :Hc, :Wc]
    got = np.concatenate([q[0, :, :-1, :-1], q[1, :, :-1, 1:], q[2, :, 1:, :-1], q[3, :, 1:, 1:]],
                         axis=0).transpose(1, 2, 0)
    ref = oracle.hog_blocks(L)
    tol = HOG_TOL * ref.sum(axis=2, keepdims=True) + 1e-6
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) - tol))


@pytest.mark.parametrize("scheme", [pd.PD_SCHEME_SVM_NAIVE, pd.PD_SCHEME_SVM_WARP])
def test_svm_schemes_on_per_block_planes(det_pb, scheme):
    h, w, b = det_pb
    W, H = 300, 260
    L = synth.random_image(W, H, 17, smooth=True)
    hb = oracle.hog_blocks(L).astype(np.float32)
    lbp = oracle.lbp_cells(L)
    feat = oracle.block_features_pb(hb.astype(np.float64), lbp)
    ref = oracle.scores(feat, w, b)
    Hc, Wc = lbp.shape[:2]
    cp, plane = _planes(Hc, Wc)
    q = np.zeros((4, 9, Hc, cp), np.float32)
    t = hb.transpose(2, 0, 1).reshape(4, 9, Hc - 1, Wc - 1)
    q[0, :, :-1, :Wc - 1] = t[0]
    q[1, :, :-1, 1:Wc] = t[1]
    q[2, :, 1:, :Wc - 1] = t[2]
    q[3, :, 1:, 1:Wc] = t[3]
    lp = np.zeros((59, Hc, cp), np.uint8)
    lp[:, :, :Wc] = lbp.transpose(2, 0, 1)
    rows, cols = ref.shape
    out = torch.full((rows * cols,), float("nan"), dtype=torch.float32, device="cuda")
    pd.pd_scheme_window_scores(h.h, scheme, torch.from_numpy(q.ravel()).cuda(), plane,
                               torch.from_numpy(lp.ravel()).cuda(), plane, cp, Wc, Hc, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(rows, cols).astype(np.float64)
    wabs = np.abs(w.astype(np.float64))
    scale = np.abs(b) + np.array([[np.sum(np.abs(feat[y:y + 15, x:x + 7]) * wabs) for x in range(cols)]
                                  for y in range(rows)])
    assert np.all(np.abs(got - ref) <= SCORE_TOL * scale), float(np.max(np.abs(got - ref) / scale))
