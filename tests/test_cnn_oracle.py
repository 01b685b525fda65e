"""Pins of the float64 proposal-network oracle (oracle/cnn.py), CPU only."""
import numpy as np
import pytest

from oracle import cnn


def _bf16_from_f32_bits(a):
    # independent route: round-to-nearest-even on the float32 bit pattern
    b = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_round_closed_forms_and_float32_route():
    assert cnn.bf16_round(1.0) == 1.0
    assert cnn.bf16_round(1 + 2 ** -8) == 1.0                 # tie -> even
    assert cnn.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6     # tie -> even (up)
    assert cnn.bf16_round(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7
    assert cnn.bf16_round(-0.3) == -cnn.bf16_round(0.3)
    vals = np.arange(256) / 255.0 - 0.5
    # exact on every value the input layer can see (float32-representable route)
    f32 = vals.astype(np.float32).astype(np.float64)
    assert np.array_equal(cnn.bf16_round(f32), _bf16_from_f32_bits(f32))
    rng = np.random.default_rng(0)
    x = rng.standard_normal(10000).astype(np.float32).astype(np.float64)
    assert np.array_equal(cnn.bf16_round(x), _bf16_from_f32_bits(x))


def test_conv_delta_kernel_is_strided_subsampling():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((3, 9, 12))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1] = 1.0
    out = cnn.conv3x3_s2(a, w, np.zeros(3))
    assert out.shape == (3, 5, 6)
    assert np.array_equal(out, a[:, ::2, ::2])
    # a corner tap reads the zero padding at the border
    w2 = np.zeros((1, 1, 3, 3))
    w2[0, 0, 0, 0] = 1.0
    o2 = cnn.conv3x3_s2(a[:1], w2, np.array([0.5]))
    assert o2[0, 0, 0] == 0.5 and o2[0, 1, 1] == a[0, 1, 1] + 0.5


def test_window_pool_one_hot_is_a_shift():
    rng = np.random.default_rng(2)
    h = rng.standard_normal((20, 12))
    v = np.zeros((16, 8))
    v[3, 5] = 2.0
    z = cnn.window_pool(h, v, 0.25, 5, 5)
    assert np.allclose(z, 2.0 * h[3:8, 5:10] + 0.25, atol=0)


def test_bce_closed_forms():
    loss, dz = cnn.bce_with_logits(np.zeros(4), np.array([1, 0, 1, 0.0]), 1.0)
    assert abs(loss - np.log(2)) < 1e-15
    assert np.allclose(dz, (0.5 - np.array([1, 0, 1, 0])) / 4)
    loss, _ = cnn.bce_with_logits(np.array([0.0]), np.array([1.0]), 3.0)
    assert abs(loss - 3 * np.log(2)) < 1e-15
    big, _ = cnn.bce_with_logits(np.array([800.0, -800.0]), np.array([1.0, 0.0]), 2.0)
    assert big == 0.0


def test_adam_first_step_closed_form():
    opt = cnn.Adam(lr=0.01)
    p = np.zeros(cnn.N_PARAMS)
    g = np.linspace(-1, 1, cnn.N_PARAMS)
    q = opt.step(p, g)
    assert np.allclose(q, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def _tiny_problem(seed):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 256, size=(136, 72)).astype(np.uint8)   # 17 x 9 cells -> 2 x 2 windows
    y = (rng.uniform(size=(2, 2)) > 0.5).astype(np.float64)
    return L, y


@pytest.mark.parametrize("name", cnn.ORDER)
def test_gradients_match_central_differences(name):
    L, y = _tiny_problem(3)
    q = cnn.rounded(cnn.init_params(1))
    for k in ["b1", "b2", "b3"]:
        q[k] = q[k] + 0.05  # keep most units active
    z, cache = cnn.forward_q(L, q)
    _, dz = cnn.bce_with_logits(z, y, 2.0)
    g = cnn.backward(cache, dz)
    rng = np.random.default_rng(4)
    flat = q[name].ravel()
    for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
        eps = 1e-6
        qp = {k: v.copy() for k, v in q.items()}
        qm = {k: v.copy() for k, v in q.items()}
        qp[name].ravel()[idx] += eps
        qm[name].ravel()[idx] -= eps
        lp, _ = cnn.bce_with_logits(cnn.forward_q(L, qp)[0], y, 2.0)
        lm, _ = cnn.bce_with_logits(cnn.forward_q(L, qm)[0], y, 2.0)
        fd = (lp - lm) / (2 * eps)
        an = g[name].ravel()[idx]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (name, idx, fd, an)


def test_training_reduces_loss_on_a_tiny_problem():
    L, y = _tiny_problem(5)
    p = cnn.flatten(cnn.init_params(2))
    opt = cnn.Adam(lr=3e-3)
    first = None
    for _ in range(40):
        loss, g = cnn.loss_and_grad([L], [y], cnn.unflatten(p), 1.0)
        first = loss if first is None else first
        p = opt.step(p, cnn.flatten(g))
    assert loss < 0.5 * first


# ----------------------------------------------------------------------------- level groups
def test_head_resample_identity_and_exact_half():
    rng = np.random.default_rng(7)
    h = rng.standard_normal((20, 30))
    assert np.array_equal(cnn.head_resample(h, (240, 160), (240, 160)), h)
    # a level exactly half the size: destination cell (cy, cx) reads source (2cy+1, 2cx+1)
    g = cnn.head_resample(h, (240, 160), (120, 80))
    assert g.shape == (10, 15)
    assert np.array_equal(g, h[1::2, 1::2])


def test_head_resample_reads_the_cell_holding_each_centre():
    """Brute force with exact rationals: the source cell read for destination cell c contains the
    destination cell's centre (8c + 4) mapped to source pixels, clamped to the source's cells."""
    from fractions import Fraction
    rng = np.random.default_rng(8)
    for (ws, hs), (wd, hd) in [((333, 257), (301, 233)), ((1242, 375), (1127, 340)), ((640, 480), (350, 262))]:
        h = rng.standard_normal((hs // 8, ws // 8))
        g = cnn.head_resample(h, (ws, hs), (wd, hd))
        assert g.shape == (hd // 8, wd // 8)
        idx = {v: (i, j) for (i, j), v in np.ndenumerate(h)}
        for cy in range(hd // 8):
            for cx in range(wd // 8):
                sy, sx = idx[g[cy, cx]]
                py = Fraction(8 * cy + 4) * hs / hd
                px = Fraction(8 * cx + 4) * ws / wd
                assert sy == min(int(py // 8), hs // 8 - 1)
                assert sx == min(int(px // 8), ws // 8 - 1)


def test_frame_logits_step_one_is_the_per_level_network():
    rng = np.random.default_rng(9)
    p = cnn.init_params(3)
    img = (rng.random((200, 300)) * 255).astype(np.uint8)
    levels = [img, img[:180, :270].copy(), img[:150, :200].copy()]
    z = cnn.frame_logits(levels, p, step=1)
    for L, zk in zip(levels, z):
        assert np.array_equal(zk, cnn.forward(L, p)[0])
    # with step 3 the first level is unchanged and the others pool resampled heads of level 0
    z3 = cnn.frame_logits(levels, p, step=3)
    assert np.array_equal(z3[0], z[0])
    h0 = cnn.forward(levels[0], p)[1]["h"]
    q = cnn.rounded(p)
    for k in (1, 2):
        Hk, Wk = levels[k].shape
        h = cnn.head_resample(h0, (300, 200), (Wk, Hk))
        ref = cnn.window_pool(h, q["v"], q["bv"][0], Hk // 8 - 15, Wk // 8 - 7)
        assert np.array_equal(z3[k], ref)
