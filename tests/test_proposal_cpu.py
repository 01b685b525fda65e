"""Host logic of the proposal module (no GPU): keep-threshold calibration,
checkpoints, initial parameters."""
import numpy as np
import pytest

pd = pytest.importorskip("paper_1611_01642_gb300")
from paper_1611_01642_gb300 import proposal  # noqa: E402


def test_calibrate_keeps_the_requested_fraction_of_positives():
    rng = np.random.default_rng(0)
    s = rng.normal(size=10000).astype(np.float32)
    z = (s + rng.normal(scale=0.5, size=s.size)).astype(np.float32)
    for recall in [0.9, 0.99, 0.999]:
        tau = proposal.calibrate(s, z, recall)
        pos = s > 0
        assert float(np.mean(z[pos] > tau)) >= recall
        # the largest such threshold: at the smallest kept positive logit the recall is lost
        z_min = float(np.min(z[pos][z[pos] > tau]))
        assert float(np.mean(z[pos] > z_min)) < recall


def test_calibrate_without_positives_keeps_everything():
    s = -np.ones(10, np.float32)
    assert proposal.calibrate(s, np.zeros(10, np.float32)) == float("-inf")


def test_checkpoint_round_trip(tmp_path):
    p = proposal.init_params(3)
    assert p.size == pd.CNN_PARAMS and p.dtype == np.float32
    meta = {"keep_logit_threshold": 0.25, "recipe": {"frames": 4}}
    path = tmp_path / "ck.npz"
    proposal.save_checkpoint(str(path), p, meta)
    q, m = proposal.load_checkpoint(str(path))
    assert np.array_equal(p, q) and m == meta


def test_checkpoint_rejects_wrong_size(tmp_path):
    path = tmp_path / "bad.npz"
    proposal.save_checkpoint(str(path), np.zeros(10, np.float32), {})
    with pytest.raises(ValueError):
        proposal.load_checkpoint(str(path))


def test_init_params_match_the_oracle_initialisation():
    from oracle import cnn as ocnn
    p = proposal.init_params(5)
    q = ocnn.flatten(ocnn.init_params(5)).astype(np.float32)
    assert np.array_equal(p, q)


def test_committed_checkpoint_is_loadable():
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    params, meta = proposal.load_checkpoint(
        os.path.join(root, "paper_1611_01642_gb300", "weights", "proposal_1920x1080.npz"))
    assert np.all(np.isfinite(params))
    assert np.isfinite(meta["keep_logit_threshold"])
    assert meta["validation"]["recall"] >= 0.99
