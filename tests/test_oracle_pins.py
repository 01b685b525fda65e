"""Pins of the CPU oracle to facts other than itself (CPU only).

Each test ties one oracle function to something the paper or mathematics
fixes: hand-worked values (tests/golden/), closed forms, invariants,
symmetries, special cases that reduce to a textbook routine, or brute force
on tiny inputs. They are chosen so that a dropped term, a wrong sign or
offset, or a transposed index in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _records(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [float(t) if "." in t else int(t) for t in line.split()]


# ----------------------------------------------------------------------------- pyramid (Section 4.4)
def test_pyramid_levels_hand_worked():
    for rec in _records("pyramid_levels.txt"):
        W, H, f, n = rec[:4]
        lv = oracle.pyramid(W, H, f)
        assert len(lv) == n, rec
        if n:
            assert lv[0] == (rec[4], rec[5]) and lv[-1] == (rec[6], rec[7]), (rec, lv)


def test_pyramid_monotone_and_min_window():
    for (W, H, f) in [(1920, 1080, 1.05), (640, 480, 1.1), (3840, 2160, 1.05)]:
        lv = oracle.pyramid(W, H, f)
        assert lv[0] == (W, H)
        for (a, b), (c, d) in zip(lv, lv[1:]):
            assert c <= a and d <= b
        assert lv[-1][0] >= 64 and lv[-1][1] >= 128
    with pytest.raises(ValueError):
        oracle.pyramid(100, 200, 1.0)


# ----------------------------------------------------------------------------- Q11 resize
def test_resize_level0_identity():
    img = synth.random_image(77, 53, 1)
    assert np.array_equal(oracle.resize(img, 77, 53), img)


def test_resize_constant_image():
    img = np.full((131, 97), 173, np.uint8)
    for (wk, hk) in [(97, 131), (80, 110), (41, 60), (13, 7), (1, 1)]:
        assert np.all(oracle.resize(img, wk, hk) == 173)


def test_resize_exact_half_is_rounded_2x2_mean():
    # W/Wk = 2 puts every source coordinate at x0 = 2x with weight 1024/2048,
    # so the output is (a + b + c + d + 2) >> 2 (closed form).
    img = synth.random_image(64, 48, 2, smooth=False).astype(np.int64)
    out = oracle.resize(img.astype(np.uint8), 32, 24).astype(np.int64)
    ref = (img[0::2, 0::2] + img[0::2, 1::2] + img[1::2, 0::2] + img[1::2, 1::2] + 2) >> 2
    assert np.array_equal(out, ref)


def _bilinear_f64(img, wk, hk):
    """Textbook bilinear with half-pixel centres and edge clamping, in float64."""
    H, W = img.shape
    out = np.zeros((hk, wk))
    for y in range(hk):
        sy = min(max((y + 0.5) * H / hk - 0.5, 0.0), H - 1.0)
        y0 = int(np.floor(sy)); y1 = min(y0 + 1, H - 1); fy = sy - y0
        for x in range(wk):
            sx = min(max((x + 0.5) * W / wk - 0.5, 0.0), W - 1.0)
            x0 = int(np.floor(sx)); x1 = min(x0 + 1, W - 1); fx = sx - x0
            top = (1 - fx) * img[y0, x0] + fx * img[y0, x1]
            bot = (1 - fx) * img[y1, x0] + fx * img[y1, x1]
            out[y, x] = (1 - fy) * top + fy * bot
    return out


@pytest.mark.parametrize("wk,hk", [(8, 8), (5, 7), (11, 3), (6, 6)])
def test_resize_close_to_float_bilinear_on_tiny_images(wk, hk):
    # Weights quantised to 1/2048 (coordinate rounding <= 0.5/2048 per axis)
    # plus the final rounding bound the error by 0.5 + 2*255*0.5/2048 < 0.63.
    for seed in range(6):
        img = synth.random_image(8, 8, seed, smooth=False)
        q = oracle.resize(img, wk, hk).astype(np.float64)
        ref = _bilinear_f64(img.astype(np.float64), wk, hk)
        assert np.max(np.abs(q - ref)) <= 0.5 + 2 * 255 * 0.5 / 2048 + 1e-9


def test_resize_within_source_2x2_range():
    img = synth.random_image(123, 77, 3, smooth=False)
    for (wk, hk) in [(100, 60), (61, 38), (117, 73)]:
        out = oracle.resize(img, wk, hk)
        ref = _bilinear_f64(img.astype(np.float64), wk, hk)
        # the fixed-point value stays inside the range of the 2x2 source block
        H, W = img.shape
        for y in range(0, hk, 7):
            sy = min(max((y + 0.5) * H / hk - 0.5, 0.0), H - 1.0)
            y0 = int(sy); y1 = min(y0 + 1, H - 1)
            for x in range(0, wk, 5):
                sx = min(max((x + 0.5) * W / wk - 0.5, 0.0), W - 1.0)
                x0 = int(sx); x1 = min(x0 + 1, W - 1)
                blk = img[[y0, y0, y1, y1], [x0, x1, x0, x1]]
                assert blk.min() <= out[y, x] <= blk.max()
        assert np.max(np.abs(out - ref)) < 0.63


# ----------------------------------------------------------------------------- LBP (Section 4.2)
def test_lbp_hand_worked_codes():
    for rec in _records("lbp_hand.txt"):
        patch = np.array(rec[:9], np.uint8).reshape(3, 3)
        code, trans, b = rec[9:]
        assert oracle.lbp_code(patch, 1, 1) == code, rec
        assert oracle.lbp_transitions(code) == trans, rec
        assert oracle.lbp_bin(code) == b, rec


def test_lbp_uniform_enumeration():
    # 8 neighbours: P(P-1)+2 = 58 uniform patterns, 59 bins in all.
    uni = [c for c in range(256) if oracle.lbp_transitions(c) <= 2]
    assert len(uni) == 58
    bins = [oracle.lbp_bin(c) for c in range(256)]
    assert sorted(set(bins)) == list(range(59))
    assert [oracle.lbp_bin(c) for c in uni] == list(range(58))
    assert all(oracle.lbp_bin(c) == 58 for c in range(256) if c not in uni)
    # rotation invariance of the transition count
    for c in range(256):
        r = ((c << 1) | (c >> 7)) & 255
        assert oracle.lbp_transitions(r) == oracle.lbp_transitions(c)


def test_lbp_cells_counts_and_borders():
    img = synth.random_image(75, 61, 4, smooth=False)
    cells = oracle.lbp_cells(img)
    assert cells.shape == (7, 9, 59)
    assert np.all(cells.sum(axis=2) == 64)
    # constant image: every code is 255 (bin 57), borders included (clamping)
    flat = oracle.lbp_cells(np.full((40, 24), 9, np.uint8))
    assert np.all(flat[:, :, 57] == 64) and flat.sum() == 64 * 15
    # the cell count equals a direct tally of the LBP map over the cell
    codes = oracle.lbp_codes(img)
    for (cy, cx) in [(0, 0), (3, 4), (6, 8)]:
        sub = codes[8 * cy:8 * cy + 8, 8 * cx:8 * cx + 8].ravel()
        tally = np.bincount([oracle.lbp_bin(int(c)) for c in sub], minlength=59)
        assert np.array_equal(tally, cells[cy, cx])


def test_lbp_block_l1_sqrt_unit_norm():
    img = synth.random_image(96, 80, 5)
    hog, lbp, feat, _ = oracle.level_all(img, np.zeros((15, 7, 95)), 0.0)
    f = feat[:, :, 36:]
    assert np.allclose((f * f).sum(axis=2), 1.0, atol=1e-12)
    # the LBP block is the reduction of its 4 cells (Algorithm 3)
    by, bx = 3, 5
    h = lbp[by:by + 2, bx:bx + 2].sum(axis=(0, 1)).astype(np.float64)
    assert h.sum() == 256
    assert np.allclose(f[by, bx], np.sqrt(h / 256.0), atol=0)


# ----------------------------------------------------------------------------- gradient / orientation
def test_gradient_vertical_step_goes_to_bins_8_and_0():
    img = np.zeros((16, 16), np.uint8)
    img[:, 8:] = 50
    m, th = oracle.gradient(img, 8, 5)
    assert m == 50.0 and th == 0.0
    (b0, w0), (b1, w1) = oracle.orientation_vote(th)
    assert {b0: w0, b1: w1} == {8: 0.5, 0: 0.5}
    # the opposite step has the same unsigned orientation
    m2, th2 = oracle.gradient(255 - img, 8, 5)
    assert m2 == 50.0 and th2 == 0.0


def test_gradient_horizontal_step_goes_to_bin_4():
    img = np.zeros((16, 16), np.uint8)
    img[8:, :] = 50
    m, th = oracle.gradient(img, 5, 8)
    assert m == 50.0 and abs(th - 90.0) < 1e-12
    (b0, w0), (b1, w1) = oracle.orientation_vote(th)
    assert b0 == 4 and abs(w0 - 1.0) < 1e-12 and abs(w1) < 1e-12


def test_gradient_45_degree_ramp_splits_bins_1_and_2():
    y, x = np.mgrid[0:16, 0:16]
    img = (10 + x + y).astype(np.uint8)
    m, th = oracle.gradient(img, 7, 7)
    assert abs(m - np.sqrt(8.0)) < 1e-12 and abs(th - 45.0) < 1e-12
    (b0, w0), (b1, w1) = oracle.orientation_vote(th)
    assert (b0, b1) == (1, 2) and abs(w0 - 0.25) < 1e-12 and abs(w1 - 0.75) < 1e-12


def test_gradient_clamped_border():
    img = np.zeros((10, 10), np.uint8)
    img[:, 0] = 40  # left edge brighter: at x=0, gx = L[1] - L[0] (clamped)
    m, th = oracle.gradient(img, 0, 4)
    assert m == 40.0 and th == 0.0  # atan2(0, -40) = 180 folds to 0


def test_orientation_vote_is_continuous_and_periodic():
    def dense(theta):
        v = np.zeros(9)
        for (b, w) in oracle.orientation_vote(theta):
            v[b] += w
        return v
    for th in np.linspace(0, 179.999, 361):
        v = dense(th)
        assert abs(v.sum() - 1.0) < 1e-12 and np.all(v >= 0)
        # the vote's centre of mass sits at theta on the 9-bin circle
        ang = 2 * np.pi * (np.arange(9) * 20 + 10) / 180
        z = (v * np.exp(1j * ang)).sum()
        # linear interpolation between neighbours keeps the argument between them
        assert abs(((np.angle(z) * 180 / (2 * np.pi)) - th + 90) % 180 - 90) < 10.0 + 1e-9
    assert np.allclose(dense(0.0), dense(179.9999999), atol=1e-8)
    assert np.allclose(dense(10.0), np.eye(9)[0]) and np.allclose(dense(170.0), np.eye(9)[8])


def test_spatial_vote_values_and_mirror_symmetry():
    cases = {0: {0: 1.0}, 3: {0: 1.0}, 4: {0: 0.9375, 1: 0.0625},
             7: {0: 0.5625, 1: 0.4375}, 11: {0: 0.0625, 1: 0.9375}, 12: {1: 0.9375, 2: 0.0625}}
    for p, want in cases.items():
        got = {}
        for (c, w) in oracle.spatial_vote(p, 5):
            got[c] = got.get(c, 0.0) + w
        got = {c: w for c, w in got.items() if w != 0.0}
        assert got == want, (p, got)
    n = 6
    for p in range(8 * n):
        a = {}
        for (c, w) in oracle.spatial_vote(p, n):
            a[c] = a.get(c, 0.0) + w
        b = {}
        for (c, w) in oracle.spatial_vote(8 * n - 1 - p, n):
            b[n - 1 - c] = b.get(n - 1 - c, 0.0) + w
        a = {c: w for c, w in a.items() if w}
        b = {c: w for c, w in b.items() if w}
        assert a == b, p


# ----------------------------------------------------------------------------- HOG cells
def _grid_mass(img):
    H, W = img.shape
    Hc, Wc = H // 8, W // 8
    tot = 0.0
    for y in range(8 * Hc):
        for x in range(8 * Wc):
            tot += oracle.gradient(img, x, y)[0]
    return tot


def test_hog_mass_is_grid_magnitude_sum():
    img = synth.random_image(44, 37, 6, smooth=False)
    hog = oracle.hog_cells(img)
    assert abs(hog.sum() - _grid_mass(img)) < 1e-9 * hog.sum()
    assert np.all(hog >= 0)


def test_hog_doubling_is_exact():
    img = synth.random_image(48, 40, 7) // 2
    h1 = oracle.hog_cells(img)
    h2 = oracle.hog_cells(img * 2)
    assert np.array_equal(h2, 2 * h1)


def test_hog_mirror_symmetry():
    # Flipping left-right maps theta -> 180 - theta (bin b -> 8 - b) and cell
    # cx -> Wc-1-cx; flipping up-down does the same for cy. Width and height
    # are multiples of 8 so the cell grid mirrors onto itself.
    img = synth.random_image(48, 40, 8, smooth=False)
    h = oracle.hog_cells(img)
    hl = oracle.hog_cells(img[:, ::-1].copy())
    hu = oracle.hog_cells(img[::-1, :].copy())
    assert np.allclose(hl, h[:, ::-1, ::-1], rtol=0, atol=1e-9)
    assert np.allclose(hu, h[::-1, :, ::-1], rtol=0, atol=1e-9)


def test_hog_single_impulse_closed_form():
    # One bright pixel at (11, 11) in a black 32x32 image: its 4 neighbours
    # carry magnitude 100; left/right ones have theta 0 (bins 8 and 0, half
    # each), upper/lower ones theta 90 (bin 4). Pixel 10 -> cells 0/1 with
    # weights 3/16, 13/16; pixel 11 -> 1/16, 15/16; pixel 12 -> cells 1/2 with
    # 15/16, 1/16 (cell centres at 8c+3.5).
    img = np.zeros((32, 32), np.uint8)
    img[11, 11] = 100
    h = oracle.hog_cells(img)
    wx = {10: {0: 3 / 16, 1: 13 / 16}, 11: {0: 1 / 16, 1: 15 / 16}, 12: {1: 15 / 16, 2: 1 / 16}}
    ref = np.zeros((4, 4, 9))
    for (px, py, bins) in [(10, 11, {8: 50, 0: 50}), (12, 11, {8: 50, 0: 50}),
                           (11, 10, {4: 100}), (11, 12, {4: 100})]:
        for cy, a in wx[py].items():
            for cx, b in wx[px].items():
                for o, m in bins.items():
                    ref[cy, cx, o] += m * a * b
    assert np.allclose(h, ref, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- L2-Hys
def test_l2hys_uniform_vector_closed_form():
    for a in [0.01, 0.3, 5.0, 1234.0]:
        v = oracle.l2hys(np.full(36, a))
        u = a / np.sqrt(36 * a * a + 1.0)
        want = u / np.sqrt(36 * u * u + 1e-6)
        assert np.allclose(v, want, rtol=1e-14, atol=0)
        assert abs(want - 1 / 6) < 1e-2 or a < 1


def test_l2hys_clip_and_norm():
    v = oracle.l2hys(np.array([1000.0] + [0.0] * 35))
    assert abs(v[0] - 0.2 / np.sqrt(0.04 + 1e-6)) < 1e-15 and np.all(v[1:] == 0)
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = rng.exponential(size=36) * rng.uniform(0.01, 500)
        y = oracle.l2hys(x)
        assert np.linalg.norm(y) <= 1.0 + 1e-12
        pre = x / np.sqrt((x * x).sum() + 1)
        assert np.all(y <= np.max(np.minimum(pre, 0.2)) / np.sqrt((np.minimum(pre, 0.2) ** 2).sum() + 1e-6) + 1e-15)
    assert np.all(oracle.l2hys(np.zeros(36)) == 0)


# ----------------------------------------------------------------------------- SVM scores (Algorithm 6)
@pytest.fixture(scope="module")
def level_data():
    img = synth.random_image(96, 152, 9)
    w, b = synth.random_svm(1)
    return img, w, b, oracle.level_all(img, w, b)


def test_scores_shape(level_data):
    img, w, b, (hog, lbp, feat, sc) = level_data
    assert hog.shape == (19, 12, 9) and lbp.shape == (19, 12, 59)
    assert feat.shape == (18, 11, 95) and sc.shape == (19 - 15, 12 - 7)


def test_scores_one_hot_template_picks_one_feature(level_data):
    img, _, _, (hog, lbp, feat, _) = level_data
    for (i, j, t) in [(0, 0, 0), (14, 6, 94), (3, 5, 36), (7, 2, 17)]:
        w = np.zeros((15, 7, 95))
        w[i, j, t] = 1.0
        sc = oracle.scores(feat, w, 0.25)
        for wy in range(sc.shape[0]):
            for wx in range(sc.shape[1]):
                assert sc[wy, wx] == feat[wy + i, wx + j, t] + 0.25


def test_scores_linear_in_template_and_ones(level_data):
    img, w, b, (hog, lbp, feat, sc) = level_data
    w2, _ = synth.random_svm(2)
    s1 = oracle.scores(feat, w, 0.0)
    s2 = oracle.scores(feat, w2, 0.0)
    s12 = oracle.scores(feat, w.astype(np.float64) + w2.astype(np.float64), 0.0)
    assert np.allclose(s12, s1 + s2, rtol=0, atol=1e-12)
    ones = oracle.scores(feat, np.ones((15, 7, 95)), 0.0)
    for wy in range(ones.shape[0]):
        for wx in range(ones.shape[1]):
            assert abs(ones[wy, wx] - feat[wy:wy + 15, wx:wx + 7].sum()) < 1e-10
    # numpy dot product over the window descriptor (template order [i][j][t])
    for wy in range(sc.shape[0]):
        for wx in range(sc.shape[1]):
            d = oracle.window_descriptor(feat, wx, wy).ravel()
            assert abs(sc[wy, wx] - (np.dot(d, w.astype(np.float64).ravel()) + b)) < 1e-10


def test_window_descriptor_bruteforce_matches_map(level_data):
    img, w, b, (hog, lbp, feat, sc) = level_data
    for (wx, wy) in [(0, 0), (4, 3), (2, 1), (4, 0)]:
        bf = oracle.window_descriptor_bruteforce(img, wx, wy)
        assert np.allclose(bf, oracle.window_descriptor(feat, wx, wy), rtol=0, atol=1e-12)


def test_translation_by_one_cell_shifts_score_map():
    base = synth.random_image(160, 176, 10)
    sh = base[:, 8:].copy()
    w, b = synth.random_svm(3)
    s0 = oracle.level_scores(base, w, b)
    s1 = oracle.level_scores(sh, w, b)
    # interior windows (away from the clamped borders of both images)
    assert np.array_equal(s1[1:-1, 1:-1], s0[1:-1, 2:s1.shape[1]])


# ----------------------------------------------------------------------------- boxes / NMS
def test_window_box_and_iou_closed_forms():
    assert oracle.window_box(1242, 375, 1242, 375, 3, 2) == (24.0, 16.0, 64.0, 128.0)
    x, y, w, h = oracle.window_box(1000, 500, 500, 250, 1, 1)
    assert (x, y, w, h) == (16.0, 16.0, 128.0, 256.0)
    assert oracle.iou((0, 0, 2, 1), (1, 0, 2, 1)) == pytest.approx(1 / 3, abs=1e-15)
    assert oracle.iou((0, 0, 2, 2), (0, 0, 2, 2)) == 1.0
    assert oracle.iou((0, 0, 1, 1), (1, 0, 1, 1)) == 0.0
    assert oracle.iou((0, 0, 4, 4), (1, 1, 2, 2)) == pytest.approx(4 / 16, abs=1e-15)


def test_nms_hand_examples():
    # level 0 of a 200x200 frame: boxes are 64x128 at (8wx, 8wy)
    dims = [(200, 200)]
    m = np.full((10, 18), -1.0, np.float32)
    m[0, 0] = 0.9      # box A
    m[0, 1] = 0.8      # shifted by 8 px: IoU 56/72 > 0.5 -> suppressed by A
    m[0, 12] = 0.7     # disjoint from A -> kept
    m[5, 12] = 0.7     # tie with previous; IoU = (64*88)/(2*64*128-64*88) ~ 0.52 -> suppressed
    m[9, 0] = 0.95     # overlaps A by 56 rows: IoU 56/200 -> kept, and it is first
    boxes, ncand = oracle.nms([m], dims, 200, 200)
    assert ncand == 5
    got = [(int(b["wy"]), int(b["wx"])) for b in boxes]
    assert got == [(9, 0), (0, 0), (0, 12)]
    # tie order is (level, wy, wx): a tie between (0,12) and (5,12) keeps (0,12)
    boxes2, _ = oracle.nms([m], dims, 200, 200, max_boxes=2)
    assert [(int(b["wy"]), int(b["wx"])) for b in boxes2] == [(9, 0), (0, 0)]
    # strict threshold
    boxes3, n3 = oracle.nms([m], dims, 200, 200, threshold=0.9)
    assert n3 == 1 and int(boxes3[0]["wy"]) == 9


def test_nms_keeps_no_pair_above_iou_and_is_deterministic():
    dims = [(400, 300), (350, 262), (300, 225)]
    maps = synth.random_score_maps([(300 // 8 - 15, 400 // 8 - 7), (262 // 8 - 15, 350 // 8 - 7),
                                    (225 // 8 - 15, 300 // 8 - 7)], seed=4)
    b1, n1 = oracle.nms(maps, dims, 400, 300)
    b2, n2 = oracle.nms(maps, dims, 400, 300)
    assert n1 == n2 and np.array_equal(b1, b2)
    for i in range(len(b1)):
        for j in range(i):
            assert oracle.iou(tuple(b1[i])[:4], tuple(b1[j])[:4]) <= 0.5
    assert np.all(np.diff(b1["score"]) <= 0)


# ----------------------------------------------------------------------------- whole path
def test_detect_matches_stagewise_composition():
    img = synth.make_scene(320, 240, 1, 0)
    w, b = synth.random_svm(5)
    r = oracle.detect(img, w, b, 1.2)
    assert len(r["levels"]) == 4
    for k, (wk, hk) in enumerate(r["levels"]):
        L = oracle.resize(img, wk, hk)
        assert np.array_equal(r["scores"][k], oracle.level_scores(L, w, b))


def test_tiny_frames_have_no_levels():
    w, b = synth.random_svm(6)
    for (W, H) in [(63, 200), (200, 127), (1, 1)]:
        r = oracle.detect(np.zeros((H, W), np.uint8), w, b, 1.05)
        assert r["levels"] == [] and len(r["boxes"]) == 0


def test_iou_separated_boxes_are_zero():
    # a gap on one axis (negative overlap) or on both must give 0, never a
    # positive product of two negative overlaps
    assert oracle.iou((0, 0, 1, 1), (3, 0, 1, 1)) == 0.0
    assert oracle.iou((0, 0, 1, 1), (0, 3, 1, 1)) == 0.0
    assert oracle.iou((0, 0, 1, 1), (3, 3, 1, 1)) == 0.0


def test_block_cell_order_tl_tr_bl_br():
    # One non-zero cell (cy, cx): the 4 blocks that contain it see it as their
    # top-left, top-right, bottom-left and bottom-right cell, in that order of
    # the 36-d HOG block vector.
    Hc, Wc, cy, cx = 5, 6, 2, 3
    hog = np.zeros((Hc, Wc, 9))
    hog[cy, cx, 4] = 10.0
    lbp = np.zeros((Hc, Wc, 59), np.uint8)
    lbp[:, :, 0] = 64
    f = oracle.block_features(hog, lbp)
    for (by, bx, q) in [(cy, cx, 0), (cy, cx - 1, 1), (cy - 1, cx, 2), (cy - 1, cx - 1, 3)]:
        v = f[by, bx, :36]
        assert np.count_nonzero(v) == 1 and v[q * 9 + 4] > 0.99, (by, bx, q)
    assert np.count_nonzero(f[:, :, :36]) == 4


# ----------------------------------------------------------------------------- upsampled levels
def test_upscaled_pyramid_adds_levels_before_the_frame():
    # 1242x375 at factor 1.05: 23 levels by the stop rule, plus 17 upsampled = 40
    f = float(np.float32(1.05))
    plain = oracle.pyramid(1242, 375, f)
    up = oracle.pyramid(1242, 375, f, upscale=17)
    assert len(plain) == 23 and len(up) == 40
    assert up[17:] == plain
    # hand arithmetic: 1242 x 1.05 = 1304.1, 375 x 1.05 = 393.75; x 1.1025: 1369.3, 413.4
    assert up[16] == (1304, 393) and up[15] == (1369, 413)
    widths = [wk for wk, _ in up]
    assert all(a > b for a, b in zip(widths, widths[1:]))


def test_resize_2x_upsampling_closed_form():
    # Wk = 2W: destination 2u reads source u-1, u with weights 1/4, 3/4 (u >= 1;
    # column 0 clamps to source 0), destination 2u+1 reads u, u+1 with 3/4, 1/4
    # (the last clamps to W-1); Q11 is exact for quarter weights, so the
    # level is (sum of the 4 weighted taps in 16ths + 8) // 16.
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, size=(8, 8)).astype(np.uint8)
    got = oracle.resize(img, 16, 16)

    def taps(n):
        t = []
        for x in range(2 * n):
            u = x // 2
            if x % 2 == 0:
                t.append([(0, 4)] if u == 0 else [(u - 1, 1), (u, 3)])
            else:
                t.append([(n - 1, 4)] if u == n - 1 else [(u, 3), (u + 1, 1)])
        return t
    tx, ty = taps(8), taps(8)
    ref = np.zeros((16, 16), np.int64)
    for y in range(16):
        for x in range(16):
            s = sum(wy * wx * int(img[sy, sx]) for sy, wy in ty[y] for sx, wx in tx[x])
            ref[y, x] = (s + 8) // 16
    assert np.array_equal(got.astype(np.int64), ref)


def test_detect_with_upscaled_levels_scores_each_level():
    w, b = synth.random_svm(3)
    f = float(np.float32(1.2))
    img = synth.make_scene(160, 200, 1, 5)
    ref = oracle.detect(img, w, b, f, upscale=2)
    assert ref["levels"] == oracle.pyramid(160, 200, f, upscale=2)
    assert ref["levels"][0][0] > 160 and len(ref["levels"]) == len(oracle.pyramid(160, 200, f)) + 2
    for (wk, hk), m in zip(ref["levels"], ref["scores"]):
        assert np.allclose(m, oracle.level_scores(oracle.resize(img, wk, hk), w, b), rtol=0, atol=1e-9)


# ----------------------------------------------------------------------------- HOG blocks (per-block reading)
def _tent_kept(l):
    """Weight of local coordinate l (0..15) kept inside a 16-pixel block, summed over its cells."""
    return min(1.0, (4.5 + l) / 8.0, (19.5 - l) / 8.0)


def test_block_spatial_vote_values_and_mirror():
    cases = {0: {0: 9 / 16}, 3: {0: 15 / 16}, 4: {0: 15 / 16, 1: 1 / 16}, 7: {0: 9 / 16, 1: 7 / 16},
             11: {0: 1 / 16, 1: 15 / 16}, 12: {1: 15 / 16}, 15: {1: 9 / 16}}
    for l, want in cases.items():
        c0, c1, w0, w1 = oracle.block_spatial_vote(l)
        got = {c: w for c, w in ((c0, w0), (c1, w1)) if 0 <= c <= 1 and w != 0.0}
        assert got == want, (l, got)
    for l in range(16):
        a = oracle.block_spatial_vote(l)
        b = oracle.block_spatial_vote(15 - l)
        ka = {c: w for c, w in ((a[0], a[2]), (a[1], a[3])) if 0 <= c <= 1}
        kb = {1 - c: w for c, w in ((b[0], b[2]), (b[1], b[3])) if 0 <= c <= 1}
        assert ka == kb and abs(sum(ka.values()) - _tent_kept(l)) < 1e-15, l


def test_hog_blocks_single_impulse_closed_form():
    # One bright pixel at (11, 11) of a black 32x32 image (the 4 gradient
    # pixels of the HOG cell pin above). Blocks (0,0), (0,1), (1,0), (1,1)
    # hold them; inside a block the cell centres are at local 3.5 and 11.5 and
    # votes leaving the block are dropped: local 2 -> cell 0 13/16; 3 -> cell 0
    # 15/16; 4 -> cells 0/1 15/16, 1/16; 10 -> 3/16, 13/16; 11 -> 1/16, 15/16;
    # 12 -> cell 1 15/16.
    img = np.zeros((32, 32), np.uint8)
    img[11, 11] = 100
    hb = oracle.hog_blocks(img)
    assert hb.shape == (3, 3, 36)
    w = {2: {0: 13 / 16}, 3: {0: 15 / 16}, 4: {0: 15 / 16, 1: 1 / 16},
         10: {0: 3 / 16, 1: 13 / 16}, 11: {0: 1 / 16, 1: 15 / 16}, 12: {1: 15 / 16}}
    ref = np.zeros((3, 3, 36))
    for (px, py, bins) in [(10, 11, {8: 50, 0: 50}), (12, 11, {8: 50, 0: 50}),
                           (11, 10, {4: 100}), (11, 12, {4: 100})]:
        for by in range(3):
            for bx in range(3):
                ly, lx = py - 8 * by, px - 8 * bx
                if not (0 <= ly < 16 and 0 <= lx < 16):
                    continue
                for a, wa in w[ly].items():
                    for b, wb in w[lx].items():
                        for o, m in bins.items():
                            ref[by, bx, (2 * a + b) * 9 + o] += m * wa * wb
    assert np.allclose(hb, ref, rtol=0, atol=1e-12)
    # a pixel lands in 2, 4 or 8 bins: in block (1, 1) the four gradient
    # pixels sit at local (2, 3), (4, 3), (3, 2), (3, 4) and fill bins 0, 4, 8
    # of cell 0, bins 0, 8 of cell 1 and bin 4 of cell 2 only
    assert np.count_nonzero(hb[1, 1]) == 6


def test_hog_blocks_ramp_closed_form():
    # I = 3x + 10 (64 x 48): interior gx = 6, gx = 3 on the two border columns,
    # gy = 0, theta = 0 -> bins 8 and 0 with 1/2 each. A cell of a block keeps
    # sum_l of its tent over the 16 block pixels = 7 per axis, so interior
    # blocks hold 0.5 * 6 * 7 * 7 = 147 in bins 0 and 8 of every cell (the
    # shared cell grid gives 0.5 * 6 * 8 * 8 = 192). Block column 0 loses
    # 3 * 9/16 on pixel column 0 of its left cells.
    x = np.arange(64)
    img = np.tile((3 * x + 10).astype(np.uint8), (48, 1))
    hb = oracle.hog_blocks(img).reshape(5, 7, 4, 9)
    ref = np.zeros((5, 7, 4, 9))
    ref[:, :, :, 0] = ref[:, :, :, 8] = 147.0
    left = 0.5 * 7 * (42 - 3 * 9 / 16)
    ref[:, 0, 0, [0, 8]] = ref[:, 0, 2, [0, 8]] = left
    ref[:, 6, 1, [0, 8]] = ref[:, 6, 3, [0, 8]] = left
    assert np.allclose(hb, ref, rtol=0, atol=1e-9)
    hc = oracle.hog_cells(img)
    assert np.allclose(hc[1:-1, 1:-1, 0], 192.0, rtol=0, atol=1e-9)
    # the same ramp along y: theta = 90 -> bin 4 only, 6 * 49 = 294
    hv = oracle.hog_blocks(img.T.copy()).reshape(7, 5, 4, 9)
    assert np.allclose(hv[1:-1, :, :, 4], 294.0, rtol=0, atol=1e-9)
    assert np.allclose(np.delete(hv, 4, axis=3), 0.0, rtol=0, atol=1e-12)


def test_hog_blocks_total_mass_closed_form():
    # summed over its 36 values a block holds sum_p |g(p)| T(lx) T(ly), T the
    # kept tent weight (9/16 .. 1 .. 9/16), with |g| from clamped central
    # differences computed here with numpy
    img = synth.random_image(56, 43, 21, smooth=False)
    hb = oracle.hog_blocks(img)
    Lp = np.pad(img.astype(np.float64), 1, mode="edge")
    gx = Lp[1:-1, 2:] - Lp[1:-1, :-2]
    gy = Lp[2:, 1:-1] - Lp[:-2, 1:-1]
    mag = np.hypot(gx, gy)
    T = np.array([_tent_kept(l) for l in range(16)])
    Hb, Wb = hb.shape[:2]
    for by in range(Hb):
        for bx in range(Wb):
            want = float(T @ mag[8 * by:8 * by + 16, 8 * bx:8 * bx + 16] @ T)
            assert abs(hb[by, bx].sum() - want) <= 1e-11 * max(want, 1.0), (by, bx)
    assert np.all(hb >= 0)


def test_hog_blocks_equal_cells_when_gradients_stay_in_the_block_centre():
    # A 6x6 random patch at rows/cols 8b+5 .. 8b+10 of a constant image: every
    # nonzero gradient lies in the central 8x8 of block b, where each vote
    # reaches the block's own 4 cells with the shared grid's weights, so the
    # block equals the 4 shared cells exactly (and the cells hold nothing
    # else).
    rng = np.random.default_rng(5)
    img = np.full((40, 48), 77, np.uint8)
    by, bx = 2, 3
    img[8 * by + 5:8 * by + 11, 8 * bx + 5:8 * bx + 11] = rng.integers(0, 256, (6, 6))
    hb = oracle.hog_blocks(img)
    hc = oracle.hog_cells(img)
    cells = np.concatenate([hc[by, bx], hc[by, bx + 1], hc[by + 1, bx], hc[by + 1, bx + 1]])
    assert cells.sum() > 0
    assert np.array_equal(hb[by, bx], cells)


def test_hog_blocks_are_local_and_cells_are_not():
    # a block reads only its 16x16 pixels and their 1-pixel gradient halo
    # (Section 4.3: block histograms cannot be assembled from shared cells)
    img = synth.random_image(64, 56, 22, smooth=False)
    by, bx = 2, 3
    other = img.copy()
    mask = np.ones_like(img, bool)
    mask[8 * by - 1:8 * by + 17, 8 * bx - 1:8 * bx + 17] = False
    other[mask] = 255 - other[mask]
    other[8 * by - 1:8 * by + 17, 8 * bx - 1] = img[8 * by - 1:8 * by + 17, 8 * bx - 1]  # halo kept
    a, b = oracle.hog_blocks(img), oracle.hog_blocks(other)
    assert np.array_equal(a[by, bx], b[by, bx])
    assert not np.array_equal(a[by, bx - 1], b[by, bx - 1])
    ca, cb = oracle.hog_cells(img), oracle.hog_cells(other)
    assert not np.array_equal(ca[by:by + 2, bx:bx + 2], cb[by:by + 2, bx:bx + 2])


def test_hog_blocks_mirror_symmetry():
    # left-right: block bx -> Wb-1-bx, cell column b -> 1-b, bin o -> 8-o;
    # up-down: block by -> Hb-1-by, cell row a -> 1-a, bin o -> 8-o
    img = synth.random_image(48, 40, 23, smooth=False)
    h = oracle.hog_blocks(img).reshape(4, 5, 2, 2, 9)
    hl = oracle.hog_blocks(img[:, ::-1].copy()).reshape(4, 5, 2, 2, 9)
    hu = oracle.hog_blocks(img[::-1, :].copy()).reshape(4, 5, 2, 2, 9)
    assert np.allclose(hl, h[:, ::-1, :, ::-1, ::-1], rtol=0, atol=1e-9)
    assert np.allclose(hu, h[::-1, :, ::-1, :, ::-1], rtol=0, atol=1e-9)


def test_block_features_pb_parts():
    img = synth.random_image(80, 72, 24, smooth=True)
    hb = oracle.hog_blocks(img)
    lbp = oracle.lbp_cells(img)
    f = oracle.block_features_pb(hb, lbp)
    g = oracle.block_features(oracle.hog_cells(img), lbp)
    assert np.array_equal(f[..., 36:], g[..., 36:])
    for by, bx in [(0, 0), (3, 5), (7, 8)]:
        assert np.allclose(f[by, bx, :36], oracle.l2hys(hb[by, bx]), rtol=0, atol=0)
    assert not np.allclose(f[..., :36], g[..., :36], atol=1e-3)


def test_detect_per_block_matches_stagewise_composition():
    w = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                             "svm_template_seed0.npz"))
    img = synth.make_scene(160, 300, 2, 25)
    F = float(np.float32(1.2))
    ref = oracle.detect(img, w["w"], float(w["b"]), F, per_block=True)
    for (wk, hk), sc in zip(ref["levels"], ref["scores"]):
        L = oracle.resize(img, wk, hk)
        assert np.array_equal(sc, oracle.level_all(L, w["w"], float(w["b"]), per_block=True)[3])


def test_hog_blocks_brute_force_tent_form_on_a_tiny_image():
    # the same histograms from a different form of the definition: each cell
    # of a block weighs a pixel by the tent max(0, 1 - |l - centre| / 8) on each
    # axis (centres at local 3.5 and 11.5), summed over the block's 256 pixels
    # only; orientation from the oracle's own pinned vote
    img = synth.random_image(32, 24, 26, smooth=False)
    hb = oracle.hog_blocks(img)
    Hb, Wb = hb.shape[:2]
    tent = lambda d: max(0.0, 1.0 - abs(d) / 8.0)
    for by in range(Hb):
        for bx in range(Wb):
            ref = np.zeros(36)
            for i in range(16):
                for j in range(16):
                    m, th = oracle.gradient(img, 8 * bx + j, 8 * by + i)
                    for (o, wo) in oracle.orientation_vote(th):
                        for a in range(2):
                            for b in range(2):
                                ref[(2 * a + b) * 9 + o] += m * wo * tent(i - (3.5 + 8 * a)) * tent(j - (3.5 + 8 * b))
            assert np.allclose(hb[by, bx], ref, rtol=0, atol=1e-9 * max(1.0, ref.sum())), (by, bx)
