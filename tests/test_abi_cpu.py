"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its host-only planning agrees with the pyramid rule."""
import os
import re

import numpy as np
import pytest

import paper_1611_01642_gb300 as pd
from paper_1611_01642_gb300 import build as pd_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pd_build.build()
    return pd.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "pd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z_]+)\s*\(", src)))


def test_header_declarations_are_all_exported(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(pd.EXPORTED) == [n for n in names if n in pd.EXPORTED]
    assert set(names) <= set(pd.EXPORTED)


def test_params_default(lib):
    p = pd.pd_params_default()
    assert p.struct_size == 60 and p.proposal_level_step == 1
    assert abs(p.pyr_factor - 1.05) < 1e-6 and abs(p.l2hys_clip - 0.2) < 1e-7
    assert p.threshold == 0.0 and p.nms_iou == 0.5 and p.max_candidates_per_frame == 16384


def test_pyramid_matches_oracle_rule(lib):
    import oracle
    for (W, H, f) in [(1242, 375, 1.05), (320, 240, 1.2), (1920, 1080, 1.05), (3840, 2160, 1.05),
                      (640, 480, 1.05), (64, 128, 1.1), (63, 500, 1.1)]:
        f32 = float(np.float32(f))
        assert pd.pd_pyramid(W, H, f32) == oracle.pyramid(W, H, f32)
        for up in [1, 17]:
            assert pd.pd_pyramid(W, H, f32, upscale_levels=up) == oracle.pyramid(W, H, f32, upscale=up)


def test_pyramid_rejects_bad_factor(lib):
    with pytest.raises(pd.PDError):
        pd.pd_pyramid(100, 200, 1.0)


def test_create_rejects_bad_params_without_gpu(lib):
    # argument checks happen before any CUDA call
    p = pd.pd_params_default(pyr_factor=0.9)
    with pytest.raises(pd.PDError) as e:
        pd.pd_create(p, np.zeros((15, 7, 95), np.float32), 0.0)
    assert e.value.code == pd.PD_EINVAL
    for bad in [dict(max_candidates_per_frame=65537), dict(upscale_levels=65),
                dict(flags=pd.PD_FLAG_HOG_ONLY | pd.PD_FLAG_LBP_ONLY),
                dict(flags=pd.PD_FLAG_HOG_PER_BLOCK | pd.PD_FLAG_SVM_FP32),
                dict(flags=pd.PD_FLAG_HOG_PER_BLOCK | pd.PD_FLAG_LBP_ONLY)]:
        p = pd.pd_params_default(**bad)
        with pytest.raises(pd.PDError) as e:
            pd.pd_create(p, np.zeros((15, 7, 95), np.float32), 0.0)
        assert e.value.code == pd.PD_EINVAL, bad
