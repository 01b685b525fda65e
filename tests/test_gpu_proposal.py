"""The learned proposal on its workload: recall against the plain path, and what the network gains.

Workload: the 16 seeded 1920x1080 frames of scene recipe 4 (the benchmark's proposal batch; held
out from training, seeds [100, i], and calibration, seeds [101, i]), pyramid factor 1.05 (44 levels),
with the committed checkpoint, its keep threshold and its level step. Checked:
  * recall = |scored on the sparse path and plain score > 0| / |plain score > 0| >= 0.99;
  * every scored window carries the plain path's score bit for bit;
  * what the network gains over the method without it (the plain path, which scores every window):
    the fraction of windows scored, and the step time, sparse against plain (CUDA events, same
    frames); the network on every level against its level groups is recorded too.
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
CKPT = os.path.join(ROOT, "paper_1611_01642_gb300", "weights", "proposal_1920x1080.npz")


def _timed(det, dev, reps=5):
    stream = torch.cuda.current_stream()
    for _ in range(2):
        det.detect(dev)
        assert det.sync() == pd.PD_OK
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        det.detect(dev)
        e1.record(stream)
        assert det.sync() == pd.PD_OK
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms))


def _all_scores(det, n):
    return torch.cat([m.reshape(-1) for f in range(n) for m in det.score_maps(f)]).clone()


def test_proposal_recall_and_gain_on_16_frames_1080p(record_property):
    from paper_1611_01642_gb300 import build as bld
    from paper_1611_01642_gb300 import proposal
    bld.build()
    params, meta = proposal.load_checkpoint(CKPT)
    tau, step = float(meta["keep_logit_threshold"]), int(meta.get("level_step", 1))
    d = np.load(os.path.join(ROOT, "tests", "golden", "svm_template_seed0.npz"))
    imgs = synth.make_frames(4)
    assert len(imgs) == 16
    det = pd.Detector(d["w"], float(d["b"]), pyr_factor=float(np.float32(1.05)), max_frames=16,
                      max_width=1920, max_height=1080)
    try:
        pd.pd_cnn_set_params(det.h, params)
        dev = [torch.from_numpy(im).cuda() for im in imgs]
        ms_plain = _timed(det, dev)
        plain = _all_scores(det, 16)
        pos = plain > 0
        out = {"level_step": step, "keep_logit_threshold": tau, "plain_ms": ms_plain,
               "positives": int(pos.sum().item()), "windows": int(plain.numel())}
        for name, m in (("groups", step), ("every_level", 1)):
            det.set_proposal(True, tau, level_step=m)
            ms = _timed(det, dev)
            sparse = _all_scores(det, 16)
            scored = ~torch.isneginf(sparse)
            assert torch.equal(sparse[scored], plain[scored])
            out[name] = {"sparse_ms": ms, "speedup": ms_plain / ms,
                         "recall": float((pos & scored).sum().item() / max(pos.sum().item(), 1)),
                         "scored_fraction": float(scored.float().mean().item())}
            det.set_proposal(False, tau)
        print(json.dumps(out))
        record_property("proposal", json.dumps(out))
        g = out["groups"]
        # the benchmark spec's bar, on held-out frames, with the checkpoint's own threshold and groups
        assert g["recall"] >= 0.99, out
        # the network's gain over the method without it: far fewer windows scored, a faster step
        assert g["scored_fraction"] < 0.5, out
        assert g["speedup"] > 1.0, out
    finally:
        det.close()
