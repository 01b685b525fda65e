"""GPU tests of the FP32 K4's tile-shape autotuner and of shape independence.

Every K4 tile shape accumulates a window's 15 x 7 x 95 products in the same
order (block rows, then columns, per channel; channels split over the 8
warps and summed in warp order), so the score maps are bit-identical for any
tiling; the autotuner may therefore change the plan but never the results.
"""
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_1611_01642_gb300")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FACTOR = float(np.float32(1.05))


@pytest.fixture(scope="module")
def template():
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    return d["w"], float(d["b"])


def _scores(d, dev):
    d.detect(dev)
    assert d.sync() == pd.PD_OK
    return [torch.cat([m.reshape(-1) for m in d.score_maps(f)]).cpu().numpy() for f in range(len(dev))]


def test_scores_identical_for_every_tiling(template):
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    frames = [synth.make_scene(1242, 375, 2, 7), synth.make_scene(640, 480, 3, 8)]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    d = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=2, max_width=1242, max_height=480,
                    flags=pd.PD_FLAG_SVM_FP32)
    try:
        ref = _scores(d, dev)
        for s in range(pd.TILE_SHAPES):
            costs = [1e6] * pd.TILE_SHAPES
            costs[s] = 1.0
            pd.pd_set_tile_costs(d.h, costs)
            got = _scores(d, dev)
            for a, g in zip(ref, got):
                assert np.array_equal(a, g), s
    finally:
        d.close()


def test_autotuner_measures_caches_and_applies(template, tmp_path, monkeypatch):
    from paper_1611_01642_gb300 import autotune
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    w, b = template
    frames = [synth.make_scene(1242, 375, 2, i) for i in range(4)]
    cost = autotune.tile_costs(frames, w, b, FACTOR)
    assert len(cost) == pd.TILE_SHAPES and all(c > 0 for c in cost)
    path = tmp_path / "paper_1611_01642_gb300" / "tile_costs.json"
    entry = next(iter(json.loads(path.read_text()).values()))
    assert entry["cost"] == cost
    assert cost in (entry["measured"], entry["default"])
    assert len(entry["ms_per_tile"]) == pd.TILE_SHAPES
    # cached: the second call returns the same table without measuring
    monkeypatch.setattr(autotune, "measure", lambda *a, **k: pytest.fail("measured again"))
    assert autotune.tile_costs(frames, w, b, FACTOR) == cost
    d = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=1, max_width=1242, max_height=375)
    try:
        autotune.apply(d, frames, w, b, FACTOR)
        assert np.allclose(pd.pd_get_tile_costs(d.h), cost)
    finally:
        d.close()


def _boxes(d, n):
    return [[tuple(r) for r in d.boxes(f).tolist()] for f in range(n)]


def test_default_path_results_identical_for_every_launch_shape(template):
    """The pyramid kernel's column groups per warp task and the tensor-core score kernel's window
    rows per item change the work split only: levels, score maps and boxes are bit-identical."""
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    w, b = template
    frames = [synth.make_scene(1242, 375, 2, 9), synth.make_scene(700, 500, 3, 10)]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    d = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=2, max_width=1242, max_height=500)
    try:
        assert pd.pd_get_tuning(d.h) == {"k1_groups": 8, "tc_item_rows": 64}
        ref, ref_b = _scores(d, dev), _boxes(d, 2)
        for g, r in [(4, 64), (16, 64), (8, 8), (8, 16), (4, 37), (16, 48)]:
            pd.pd_set_tuning(d.h, g, r)
            got = _scores(d, dev)
            for a, x in zip(ref, got):
                assert np.array_equal(a, x), (g, r)
            assert _boxes(d, 2) == ref_b, (g, r)
        for bad in [(2, 64), (8, 7), (8, 65)]:
            with pytest.raises(pd.PDError):
                pd.pd_set_tuning(d.h, *bad)
    finally:
        d.close()


def test_default_path_autotuner_picks_caches_and_applies(template, tmp_path, monkeypatch):
    from paper_1611_01642_gb300 import autotune
    from paper_1611_01642_gb300 import build as bld
    bld.build()
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    w, b = template
    frames = [synth.make_scene(1242, 375, 2, i) for i in range(8)]
    t = autotune.tune_default_path(frames, w, b, FACTOR)
    assert t["k1_groups"] in autotune.K1_GROUPS and t["tc_item_rows"] in autotune.TC_ITEM_ROWS
    path = tmp_path / "paper_1611_01642_gb300" / "default_path.json"
    entry = next(iter(json.loads(path.read_text()).values()))
    assert entry["tuning"] == t
    assert min(entry["pyramid_ms"], key=entry["pyramid_ms"].get) == str(t["k1_groups"])
    assert min(entry["scores_ms"], key=entry["scores_ms"].get) == str(t["tc_item_rows"])
    monkeypatch.setattr(autotune, "_stage_ms", lambda *a, **k: pytest.fail("measured again"))
    d = pd.Detector(w, b, pyr_factor=FACTOR, max_frames=8, max_width=1242, max_height=375)
    try:
        assert autotune.apply_default(d, frames, w, b, FACTOR) == t
        assert pd.pd_get_tuning(d.h) == t
    finally:
        d.close()
