"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (written here; each follows from the arithmetic of the step it checks):
  * resize, LBP codes/counts: bit-exact;
  * HOG cell histogram: |gpu - ref| <= 1e-4 * sum_bins |ref_cell| + 1e-6;
  * window score: |gpu - ref| <= 1e-4 * (|b| + sum_t |w_t x_t|), the scale of
    the dot product (every feature is >= 0, so that sum is the oracle's score
    of the template |w| with bias |b|);
  * NMS: exact (same kept boxes, same order) on identical float score maps.
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
F12 = float(np.float32(1.2))
SCORE_TOL = 1e-4
HOG_TOL = 1e-4


@pytest.fixture(scope="module")
def template():
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    return d["w"], float(d["b"])


@pytest.fixture(scope="module")
def det(template):
    from paper_1611_01642_gb300 import build as b
    b.build()
    w, bias = template
    d = pd.Detector(w, bias, max_frames=8, max_width=1242, max_height=480, pyr_factor=F105)
    yield d
    d.close()


def _score_scale(feat, w, b):
    return oracle.scores(feat, np.abs(w.astype(np.float64)), abs(b))


def _check_scores(got, feat, w, b, ref, what=""):
    got = np.asarray(got, np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    if ref.size == 0:
        return 0.0
    tol = SCORE_TOL * _score_scale(feat, w, b)
    err = np.abs(got - ref)
    assert np.all(err <= tol), (what, float(err.max()), float((err / tol).max()))
    return float((err / tol).max())


# ----------------------------------------------------------------------------- K1 resize
@pytest.mark.parametrize("W,H", [(64, 128), (200, 150), (321, 257), (1242, 375), (640, 480), (131, 977)])
def test_resize_pyramid_bit_exact(det, W, H):
    img = synth.random_image(W, H, W * 7 + H, smooth=(W % 2 == 0))
    levels = oracle.pyramid(W, H, F105) or [(W // 2 + 1, H // 3 + 1), (W, H)]
    pitches = [((wk + 15) // 16) * 16 + 16 for (wk, hk) in levels]
    offs, tot = [], 0
    for (wk, hk), p in zip(levels, pitches):
        offs.append(tot)
        tot += p * hk + 32
    out = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    frame = torch.from_numpy(img).cuda()
    pd.pd_resize_levels(det.h, frame, levels, out, offs, pitches)
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    for (wk, hk), o, p in zip(levels, offs, pitches):
        got = host[o:o + p * hk].reshape(hk, p)[:, :wk]
        assert np.array_equal(got, oracle.resize(img, wk, hk)), (wk, hk)


def test_resize_arbitrary_ratios_and_pitched_frame(det):
    img = synth.random_image(300, 200, 5, smooth=False)
    pitched = np.zeros((200, 333), np.uint8)
    pitched[:, :300] = img
    frame = torch.from_numpy(pitched).cuda()[:, :300]
    # downsampled, odd, degenerate and upsampled (up to 3x) levels
    levels = [(300, 200), (150, 100), (299, 199), (17, 3), (1, 1), (100, 200), (300, 7),
              (600, 400), (331, 213), (900, 250), (301, 600)]
    pitches = [wk + 5 for wk, _ in levels]
    offs = list(np.cumsum([0] + [p * hk for (wk, hk), p in zip(levels, pitches)])[:-1])
    out = torch.zeros(int(sum(p * hk for (wk, hk), p in zip(levels, pitches))), dtype=torch.uint8,
                      device="cuda")
    pd.pd_resize_levels(det.h, frame, levels, out, offs, pitches)
    host = out.cpu().numpy()
    for (wk, hk), o, p in zip(levels, offs, pitches):
        got = host[o:o + p * hk].reshape(hk, p)[:, :wk]
        assert np.array_equal(got, oracle.resize(img, wk, hk)), (wk, hk)


# ----------------------------------------------------------------------------- K2/K3 cells
def _cells_gpu(det, L):
    Hk, Wk = L.shape
    Hc, Wc = Hk // 8, Wk // 8
    cp = max(16, ((Wc + 15) // 16) * 16)
    plane = max(Hc, 1) * cp
    hog = torch.full((9 * plane,), float("nan"), dtype=torch.float32, device="cuda")
    lbp = torch.full((59 * plane,), 255, dtype=torch.uint8, device="cuda")
    lv = torch.from_numpy(L).cuda()
    pd.pd_cell_features(det.h, lv, hog, plane, lbp, plane, cp)
    torch.cuda.synchronize()
    h = hog.cpu().numpy().reshape(9, max(Hc, 1), cp)[:, :Hc, :Wc].transpose(1, 2, 0)
    l = lbp.cpu().numpy().reshape(59, max(Hc, 1), cp)[:, :Hc, :Wc].transpose(1, 2, 0)
    return h, l


@pytest.mark.parametrize("W,H,smooth", [(8, 8, False), (23, 17, False), (130, 200, True),
                                        (127, 129, False), (1242, 375, True), (256, 64, True)])
def test_cells_lbp_exact_hog_within_tolerance(det, W, H, smooth):
    L = synth.random_image(W, H, W + 3 * H, smooth=smooth)
    h, l = _cells_gpu(det, L)
    rh = oracle.hog_cells(L)
    rl = oracle.lbp_cells(L)
    assert np.array_equal(l, rl)
    tol = HOG_TOL * rh.sum(axis=2, keepdims=True) + 1e-6
    assert np.all(np.abs(h - rh) <= tol), float(np.max(np.abs(h - rh) - tol))


def test_cells_constant_and_extreme_images(det):
    for L in [np.zeros((48, 40), np.uint8), np.full((48, 40), 255, np.uint8),
              (np.indices((64, 64)).sum(0) % 2 * 255).astype(np.uint8)]:
        h, l = _cells_gpu(det, L)
        assert np.array_equal(l, oracle.lbp_cells(L))
        rh = oracle.hog_cells(L)
        assert np.all(np.abs(h - rh) <= HOG_TOL * rh.sum(axis=2, keepdims=True) + 1e-6)


# ----------------------------------------------------------------------------- K4 scores
def _scores_gpu_from_cells(det, hog, lbp):
    Hc, Wc = hog.shape[:2]
    cp = max(16, ((Wc + 15) // 16) * 16)
    plane = max(Hc, 1) * cp
    hp = np.zeros((9, max(Hc, 1), cp), np.float32)
    hp[:, :Hc, :Wc] = hog.transpose(2, 0, 1)
    lp = np.zeros((59, max(Hc, 1), cp), np.uint8)
    lp[:, :Hc, :Wc] = lbp.transpose(2, 0, 1)
    rows, cols = max(Hc - 15, 0), max(Wc - 7, 0)
    if rows == 0 or cols == 0:
        rows = cols = 0
    out = torch.full((max(rows * cols, 1),), float("nan"), dtype=torch.float32, device="cuda")
    pd.pd_window_scores(det.h, torch.from_numpy(hp.ravel()).cuda(), plane,
                        torch.from_numpy(lp.ravel()).cuda(), plane, cp, Wc, Hc, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()[:rows * cols].reshape(rows, cols)


@pytest.mark.parametrize("W,H", [(64, 128), (72, 136), (300, 260), (520, 410), (1242, 375), (900, 700),
                                 (300, 900), (896, 128)])
def test_window_scores_from_oracle_cells(det, template, W, H):
    w, b = template
    L = synth.random_image(W, H, 101 + W, smooth=True)
    hog = oracle.hog_cells(L).astype(np.float32)
    lbp = oracle.lbp_cells(L)
    feat = oracle.block_features(hog.astype(np.float64), lbp)
    ref = oracle.scores(feat, w, b)
    got = _scores_gpu_from_cells(det, hog, lbp)
    _check_scores(got, feat, w, b, ref, f"{W}x{H}")


def test_window_scores_random_template(template):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = synth.random_svm(9)
    d = pd.Detector(w, b, max_frames=1, max_width=600, max_height=600)
    try:
        L = synth.random_image(600, 600, 3, smooth=False)
        hog = oracle.hog_cells(L).astype(np.float32)
        lbp = oracle.lbp_cells(L)
        feat = oracle.block_features(hog.astype(np.float64), lbp)
        got = _scores_gpu_from_cells(d, hog, lbp)
        _check_scores(got, feat, w, b, oracle.scores(feat, w, b), "random template")
    finally:
        d.close()


# ----------------------------------------------------------------------------- K5 NMS
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_nms_exact_on_identical_maps(det, seed):
    W, H = 1242, 375
    levels = oracle.pyramid(W, H, F105)[:8]
    dims = [(hk // 8 - 15, wk // 8 - 7) for wk, hk in levels]
    maps = synth.random_score_maps(dims, seed, n_distinct=16 if seed % 2 else 256,
                                   pos_frac=0.05 * (seed + 1))
    flat = np.concatenate([m.ravel() for m in maps]).astype(np.float32)
    boxes = torch.zeros((4096, 8), dtype=torch.int32, device="cuda")
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    pd.pd_nms_maps(det.h, torch.from_numpy(flat).cuda(), [d[0] for d in dims], [d[1] for d in dims],
                   levels, W, H, boxes, 4096, counts)
    torch.cuda.synchronize()
    kept, ncand = counts.cpu().numpy().tolist()
    ref, rcand = oracle.nms(maps, levels, W, H, threshold=0.0, iou_thr=0.5, max_boxes=4096)
    assert ncand == rcand and kept == len(ref)
    got = np.frombuffer(boxes.cpu().numpy().tobytes(), dtype=pd.BOX_DTYPE)[:kept]
    for name in ["level", "wx", "wy", "x", "y", "w", "h", "score"]:
        assert np.array_equal(got[name], ref[name]), name


@pytest.mark.parametrize("seed", [0, 1])
def test_nms_exact_with_more_candidates_than_shared_memory_holds(template, seed):
    # caps above 16,384 candidates keep the sort keys in global memory
    W, H = 1242, 375
    levels = oracle.pyramid(W, H, F105)
    dims = [(hk // 8 - 15, wk // 8 - 7) for wk, hk in levels]
    maps = synth.random_score_maps(dims, 10 + seed, n_distinct=64 if seed else 4096, pos_frac=0.8)
    flat = np.concatenate([m.ravel() for m in maps]).astype(np.float32)
    w, b = template
    d = pd.Detector(w, b, max_frames=1, max_width=W, max_height=H, max_candidates_per_frame=40000,
                    max_boxes_per_frame=4096)
    try:
        boxes = torch.zeros((4096, 8), dtype=torch.int32, device="cuda")
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        pd.pd_nms_maps(d.h, torch.from_numpy(flat).cuda(), [q[0] for q in dims], [q[1] for q in dims],
                       levels, W, H, boxes, 4096, counts)
        torch.cuda.synchronize()
    finally:
        d.close()
    kept, ncand = counts.cpu().numpy().tolist()
    ref, rcand = oracle.nms(maps, levels, W, H, threshold=0.0, iou_thr=0.5, max_boxes=4096)
    assert rcand > 16384 and ncand == rcand and kept == len(ref)
    got = np.frombuffer(boxes.cpu().numpy().tobytes(), dtype=pd.BOX_DTYPE)[:kept]
    for name in ["level", "wx", "wy", "x", "y", "w", "h", "score"]:
        assert np.array_equal(got[name], ref[name]), name


def test_nms_overflow_is_reported(template):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    d = pd.Detector(w, b, max_frames=1, max_width=640, max_height=480, max_candidates_per_frame=64)
    try:
        m = np.ones((20, 40), np.float32)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        boxes = torch.zeros((64, 8), dtype=torch.int32, device="cuda")
        pd.pd_nms_maps(d.h, torch.from_numpy(m.ravel()).cuda(), [20], [40], [(376, 280)], 640, 480,
                       boxes, 64, counts)
        torch.cuda.synchronize()
        assert counts.cpu().numpy().tolist() == [0, -800]
    finally:
        d.close()


# ----------------------------------------------------------------------------- whole path
def _check_boxes(got, ref_maps, feats, levels, w, b, W, H, thr=0.0, iou=0.5):
    """GPU boxes against the oracle's own detections (oracle scores, oracle NMS).

    Where no two overlapping candidates and no candidate and the threshold
    are closer than the score tolerance, greedy NMS has a unique answer and
    the kept windows must be identical. Otherwise every kept GPU machine must
    still be a window the oracle scores above threshold - tolerance, the
    kept set must be pairwise non-overlapping (IoU <= 0.5) and its scores
    must match the oracle's within tolerance.
    """
    ref, _ = oracle.nms([m.astype(np.float32) for m in ref_maps], levels, W, H, threshold=thr,
                        iou_thr=iou)
    tols = [SCORE_TOL * _score_scale(f, w, b) for f in feats]
    cand = []
    for k, (m, t) in enumerate(zip(ref_maps, tols)):
        ys, xs = np.nonzero(m > thr - t)
        for y, x in zip(ys, xs):
            cand.append((k, int(x), int(y), float(m[y, x]), float(t[y, x])))
    ambiguous = any(abs(s - thr) <= t for (_, _, _, s, t) in cand)
    if not ambiguous:
        cand.sort(key=lambda c: -c[3])
        for i in range(1, len(cand)):
            if cand[i - 1][3] - cand[i][3] <= cand[i - 1][4] + cand[i][4]:
                ambiguous = True
                break
    for g in got:
        m, t = ref_maps[g["level"]], tols[g["level"]]
        assert m[g["wy"], g["wx"]] > thr - t[g["wy"], g["wx"]]
        assert abs(float(g["score"]) - m[g["wy"], g["wx"]]) <= t[g["wy"], g["wx"]]
    for i in range(len(got)):
        for j in range(i):
            assert oracle.iou(tuple(got[i])[:4], tuple(got[j])[:4]) <= iou
    if not ambiguous:
        for name in ["level", "wx", "wy", "x", "y", "w", "h"]:
            assert np.array_equal(got[name], ref[name]), name
    return ambiguous


def _oracle_level_data(img, w, b, factor):
    out = []
    for (wk, hk) in oracle.pyramid(img.shape[1], img.shape[0], factor):
        L = oracle.resize(img, wk, hk)
        hog, lbp, feat, sc = oracle.level_all(L, w, b)
        out.append((feat, sc))
    return out


@pytest.mark.parametrize("cfg,W,H,factor", [(1, 320, 240, F12), (2, 1242, 375, F105)])
def test_detect_scores_match_oracle(template, cfg, W, H, factor):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    img = synth.make_scene(W, H, cfg, 0)
    d = pd.Detector(w, b, max_frames=1, max_width=W, max_height=H, pyr_factor=factor)
    try:
        d.detect([torch.from_numpy(img).cuda()])
        assert d.sync() == pd.PD_OK
        maps = [m.cpu().numpy() for m in d.score_maps(0)]
        ref = _oracle_level_data(img, w, b, factor)
        assert len(maps) == len(ref)
        worst = 0.0
        for k, (g, (feat, sc)) in enumerate(zip(maps, ref)):
            worst = max(worst, _check_scores(g, feat, w, b, sc, f"level {k}"))
        levels = [(lv["width"], lv["height"]) for lv in d.levels(0)]
        _check_boxes(d.boxes(0), [sc for _, sc in ref], [feat for feat, _ in ref], levels, w, b, W, H)
        assert pd.pd_last_launch_count(d.h) == 4
    finally:
        d.close()


def test_detect_with_upscaled_levels_matches_oracle(template):
    # the pyramid's upsampled levels (before the frame's own level 0) through the whole path
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    W, H, up = 320, 240, 3
    img = synth.make_scene(W, H, 1, 3)
    d = pd.Detector(w, b, max_frames=1, max_width=W, max_height=H, pyr_factor=F12, upscale_levels=up)
    try:
        d.detect([torch.from_numpy(img).cuda()])
        assert d.sync() == pd.PD_OK
        dims = oracle.pyramid(W, H, F12, upscale=up)
        assert [(lv["width"], lv["height"]) for lv in d.levels(0)] == dims
        assert dims[0][0] > W
        ref = oracle.detect(img, w, b, F12, upscale=up)
        feats = []
        for k, ((wk, hk), g) in enumerate(zip(dims, d.score_maps(0))):
            L = oracle.resize(img, wk, hk)
            hog, lbp, feat, sc = oracle.level_all(L, w, b)
            feats.append(feat)
            _check_scores(g.cpu().numpy(), feat, w, b, sc, f"level {k}")
        _check_boxes(d.boxes(0), ref["scores"], feats, dims, w, b, W, H)
    finally:
        d.close()


@pytest.mark.parametrize("kernel", [0, pd.PD_FLAG_SVM_FP32])
@pytest.mark.parametrize("pipeline", ["hog", "lbp"])
def test_hog_only_and_lbp_only_pipelines_match_oracle(template, pipeline, kernel):
    # HOG-SVM / LBP-SVM (Section 4.1): only that feature's cells are computed and the
    # other features' weights count as zero, so the oracle is the full definition with
    # those weights zeroed
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    W, H = 640, 480
    img = synth.make_scene(W, H, 3, 61)
    flag = pd.PD_FLAG_HOG_ONLY if pipeline == "hog" else pd.PD_FLAG_LBP_ONLY
    wm = w.copy()
    if pipeline == "hog":
        wm[:, :, 36:] = 0.0
    else:
        wm[:, :, :36] = 0.0
    d = pd.Detector(w, b, max_frames=1, max_width=W, max_height=H, pyr_factor=F12, flags=flag | kernel)
    try:
        d.detect([torch.from_numpy(img).cuda()])
        assert d.sync() == pd.PD_OK
        dims = [(lv["width"], lv["height"]) for lv in d.levels(0)]
        assert dims == oracle.pyramid(W, H, F12)
        ref = oracle.detect(img, wm, b, F12)
        feats = []
        for k, ((wk, hk), g) in enumerate(zip(dims, d.score_maps(0))):
            L = oracle.resize(img, wk, hk)
            _, _, feat, sc = oracle.level_all(L, wm, b)
            feats.append(feat)
            _check_scores(g.cpu().numpy(), feat, wm, b, sc, f"{pipeline} level {k}")
        _check_boxes(d.boxes(0), ref["scores"], feats, dims, wm, b, W, H)
    finally:
        d.close()


def test_batched_equals_single_frames(template):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    sizes = [(1242, 375), (640, 480), (200, 300), (63, 200), (64, 128), (333, 129)]
    imgs = [synth.make_scene(W, H, 3, i) for i, (W, H) in enumerate(sizes)]
    d = pd.Detector(w, b, max_frames=len(sizes), max_width=1242, max_height=480)
    try:
        frames = [torch.from_numpy(im).cuda() for im in imgs]
        d.detect(frames)
        assert d.sync() == pd.PD_OK
        batched = [[m.clone() for m in d.score_maps(i)] for i in range(len(sizes))]
        bboxes = [d.boxes(i) for i in range(len(sizes))]
        for i, f in enumerate(frames):
            d.detect([f])
            assert d.sync() == pd.PD_OK
            single = d.score_maps(0)
            assert len(single) == len(batched[i])
            for a, s in zip(batched[i], single):
                assert torch.equal(a, s)
            assert np.array_equal(d.boxes(0), bboxes[i])
        # a frame smaller than a window: no level, no box
        d.detect([frames[3]])
        assert d.sync() == pd.PD_OK and d.levels(0) == [] and len(d.boxes(0)) == 0
    finally:
        d.close()


def test_detect_host_equals_device(template):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    imgs = [synth.make_scene(1242, 375, 2, i) for i in range(3)]
    d = pd.Detector(w, b, max_frames=3, max_width=1242, max_height=375)
    try:
        d.detect([torch.from_numpy(im).cuda() for im in imgs])
        assert d.sync() == pd.PD_OK
        dev = [d.boxes(i) for i in range(3)]
        d.detect_host(imgs)  # pageable numpy frames: copied into the arena
        assert d.sync() == pd.PD_OK
        for i in range(3):
            assert np.array_equal(d.boxes(i), dev[i])
        pinned = [torch.from_numpy(im).pin_memory() for im in imgs]
        for _ in range(3):  # pinned frames: read in place (plan, capture, replay)
            d.detect_host(pinned)
            assert d.sync() == pd.PD_OK
            for i in range(3):
                assert np.array_equal(d.boxes(i), dev[i])
                assert pd.pd_frame_candidates(d.h, i) > 0
    finally:
        d.close()


def test_errors_are_reported(template):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    d = pd.Detector(w, b, max_frames=1, max_width=320, max_height=240)
    try:
        f = torch.zeros((240, 320), dtype=torch.uint8, device="cuda")
        with pytest.raises(pd.PDError) as e:
            d.detect([f, f])
        assert e.value.code == pd.PD_EINVAL
        big = torch.zeros((241, 320), dtype=torch.uint8, device="cuda")
        with pytest.raises(pd.PDError):
            d.detect([big])
        with pytest.raises(pd.PDError) as e:
            pd.pd_boxes(d.h, 0)
        assert e.value.code in (pd.PD_ESTATE, pd.PD_EINVAL)
    finally:
        d.close()


@pytest.mark.parametrize("shape", range(7))
def test_window_scores_every_tile_shape(template, shape):
    # force one tile shape of the FP32 K4 through the planner's cost table
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    d = pd.Detector(w, b, max_frames=1, max_width=700, max_height=600, flags=pd.PD_FLAG_SVM_FP32)
    try:
        costs = [1e6] * pd.TILE_SHAPES
        costs[shape] = 1.0
        pd.pd_set_tile_costs(d.h, costs)
        assert pd.pd_get_tile_costs(d.h) == costs
        for (W, H, seed) in [(520, 410, 1), (700, 600, 2), (64, 128, 3), (130, 300, 4)]:
            L = synth.random_image(W, H, 300 + seed, smooth=True)
            hog = oracle.hog_cells(L).astype(np.float32)
            lbp = oracle.lbp_cells(L)
            feat = oracle.block_features(hog.astype(np.float64), lbp)
            got = _scores_gpu_from_cells(d, hog, lbp)
            _check_scores(got, feat, w, b, oracle.scores(feat, w, b), f"shape {shape} {W}x{H}")
    finally:
        d.close()


def test_repeated_batch_shape_replays_graph_with_new_frames(template):
    # calls 1, 2, 3 with one batch shape: plan, capture, replay; each must
    # equal a fresh handle's result for the same frames
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    sizes = [(640, 480), (1242, 375), (333, 200)]
    batches = [[synth.make_scene(W, H, 3, 100 * k + i) for i, (W, H) in enumerate(sizes)]
               for k in range(3)]
    d = pd.Detector(w, b, max_frames=3, max_width=1242, max_height=480)
    try:
        got = []
        for imgs in batches:
            d.detect([torch.from_numpy(im).cuda() for im in imgs])
            assert d.sync() == pd.PD_OK
            got.append(([torch.cat([m.reshape(-1) for m in d.score_maps(i)]).clone() for i in range(3)],
                        [d.boxes(i) for i in range(3)]))
    finally:
        d.close()
    for imgs, (maps, boxes) in zip(batches, got):
        f = pd.Detector(w, b, max_frames=3, max_width=1242, max_height=480)
        try:
            f.detect([torch.from_numpy(im).cuda() for im in imgs])
            assert f.sync() == pd.PD_OK
            for i in range(3):
                assert torch.equal(torch.cat([m.reshape(-1) for m in f.score_maps(i)]), maps[i])
                assert np.array_equal(f.boxes(i), boxes[i])
        finally:
            f.close()


def test_results_do_not_depend_on_batch_size(template):
    """The batch size sets the launch shapes: the cells kernel's strip height
    (2 to 32 cell rows), the CTAs per frame of the NMS cluster (8, 4, 2, 1
    on a 152-SM GPU) and, with more frames than SMs, persistent NMS CTAs
    that take the frames most-candidates-first. Frame 0's score maps and
    boxes must not change, nor any frame's boxes between the last two batches."""
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    n_big = torch.cuda.get_device_properties(0).multi_processor_count + 8
    imgs = [synth.make_scene(1242, 375, 2, i) for i in range(n_big)]
    d = pd.Detector(w, b, pyr_factor=float(np.float32(1.05)), max_frames=n_big, max_width=1242, max_height=375)
    try:
        frames = [torch.from_numpy(im).cuda() for im in imgs]
        ref_maps = ref_boxes = None
        for n in (1, 20, 40, 128, n_big):
            d.detect(frames[:n])
            assert d.sync() == pd.PD_OK, pd.pd_last_error(d.h)
            maps = [m.clone() for m in d.score_maps(0)]
            boxes = d.boxes(0)
            if n == 128:
                all128 = [(d.boxes(i), pd.pd_frame_candidates(d.h, i)) for i in range(128)]
            if n == n_big:
                assert pd.pd_last_launch_count(d.h) == 6  # pyramid, cells, K4, count, order, NMS
                for i in range(128):
                    assert pd.pd_frame_candidates(d.h, i) == all128[i][1], i
                    assert np.array_equal(d.boxes(i), all128[i][0]), i
            if ref_maps is None:
                ref_maps, ref_boxes = maps, boxes
                assert len(ref_boxes) > 0
                continue
            assert len(maps) == len(ref_maps)
            for a, r in zip(maps, ref_maps):
                assert torch.equal(a, r), n
            assert np.array_equal(boxes, ref_boxes), n
    finally:
        d.close()


def test_batch_beyond_the_nms_frame_order(template):
    """16,400 frames of 64x128 (one window each; the seeded training crops,
    half of them positive): more frames than the NMS order kernel sorts
    (16,384), so the persistent NMS CTAs draw the frames in index order.
    Every frame's boxes and candidate count equal those of the same frame in
    a 100-frame batch (one CTA per frame)."""
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    n_big, n_small = 16400, 100
    pos, neg = synth.make_training_crops(seed=3, n_pos=64, n_neg=64)
    crops = [np.ascontiguousarray(c) for pair in zip(pos, neg) for c in pair]
    imgs = [crops[i % len(crops)] for i in range(n_big)]
    frames = [torch.from_numpy(im).cuda() for im in imgs]
    small = pd.Detector(w, b, pyr_factor=F105, max_frames=n_small, max_width=64, max_height=128,
                        max_candidates_per_frame=64)
    big = pd.Detector(w, b, pyr_factor=F105, max_frames=n_big, max_width=64, max_height=128,
                      max_candidates_per_frame=64)
    try:
        big.detect(frames)
        assert big.sync() == pd.PD_OK, pd.pd_last_error(big.h)
        assert pd.pd_last_launch_count(big.h) == 4  # pyramid, cells, K4, NMS (no count / order)
        n_boxes = 0
        for s0 in (0, 8200, n_big - n_small):
            small.detect(frames[s0:s0 + n_small])
            assert small.sync() == pd.PD_OK
            for i in range(n_small):
                assert pd.pd_frame_candidates(big.h, s0 + i) == pd.pd_frame_candidates(small.h, i), s0 + i
                bb = big.boxes(s0 + i)
                assert np.array_equal(bb, small.boxes(i)), s0 + i
                n_boxes += len(bb)
        assert n_boxes > 0
    finally:
        small.close()
        big.close()
