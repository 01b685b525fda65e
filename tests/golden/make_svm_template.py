"""Write tests/golden/svm_template_seed0.npz: the mean-difference linear SVM template.

The paper trains its SVM offline on a labelled pedestrian set (Section 4.4)
that is not available. Stand-in: from the seeded 64x128 crops of
``synth.make_training_crops(seed=0)`` (1000 positive, 1000 negative), the
oracle computes each crop's window descriptor phi (15x7 blocks x 95 features,
the crop being one pyramid level holding one window); the template is
w = mean(phi_pos) - mean(phi_neg) in float64, stored as float32, and the bias
b = -w . (mean(phi_pos) + mean(phi_neg)) / 2 puts the decision threshold 0
midway between the class means. Only the oracle and the input generator are
called.

    python tests/golden/make_svm_template.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def descriptor(crop):
    hog = oracle.hog_cells(crop)
    lbp = oracle.lbp_cells(crop)
    feat = oracle.block_features(hog, lbp)
    return oracle.window_descriptor(feat, 0, 0).astype(np.float64)


def main():
    pos, neg = synth.make_training_crops(seed=0)
    mp = np.mean([descriptor(c) for c in pos], axis=0)
    mn = np.mean([descriptor(c) for c in neg], axis=0)
    w = (mp - mn).astype(np.float32)
    b = np.float32(-np.sum(w.astype(np.float64) * (mp + mn)) / 2.0)
    out = os.path.join(HERE, "svm_template_seed0.npz")
    np.savez(out, w=w, b=np.array(b, np.float32))
    sp = np.array([np.sum(w * descriptor(c)) + b for c in pos[:200]])
    sn = np.array([np.sum(w * descriptor(c)) + b for c in neg[:200]])
    print(f"wrote {out}: |w|={np.linalg.norm(w):.4f} b={float(b):.4f} "
          f"pos>0 {np.mean(sp > 0):.3f} neg<=0 {np.mean(sn <= 0):.3f}")


if __name__ == "__main__":
    main()
