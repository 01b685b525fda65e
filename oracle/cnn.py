"""Plain float64 oracle of the learned window proposal (test infrastructure only).

The paper has no learned component; the proposal network is an addition of
this project: a small CNN that predicts, per pyramid level, which windows can
score above the SVM threshold, so that the full HOG+LBP+SVM path only runs
where it matters. Definition (every layer evaluated in float64 on bfloat16
inputs and bfloat16 weights):

    x   = bf16(L / 255 - 0.5)                      level image L (u8)
    a1  = relu(conv3x3_s2_p1(x;  W1[16][1][3][3], b1[16]))
    a2  = relu(conv3x3_s2_p1(a1; W2[32][16][3][3], b2[32]))
    a3  = relu(conv3x3_s2_p1(a2; W3[32][32][3][3], b3[32]))   one vector per 8x8 cell
    h   = wh . a3 + bh                             1x1 head, one value per cell
    z[wy][wx] = bv + sum_{r<16, s<8} V[r][s] h[wy+r][wx+s]   one keep-logit per window

with conv3x3_s2_p1(a)[o][i][j] = b[o] + sum_{c,dy,dx} W[o][c][dy][dx]
a[c][2i+dy-1][2j+dx-1] (zero outside), output size ceil(n/2). The window
(wx, wy) covers cells wx..wx+7 x wy..wy+15, the same windows as the SVM score
map (Hc-15 x Wc-7).

Level groups (reading of this project): with a step m the network runs on
levels 0, m, 2m, ... of a frame, and level k pools the head map of level
j = m floor(k/m) read at the cell holding each of its cells' centres (cell
(cy, cx) of level k -> row min(floor((2cy+1) Hk_j / (2 Hk_k)), Hc_j - 1),
column likewise with the widths). m = 1 is the network on every level. Training minimises the mean binary cross-entropy with
logits and positive weight p, and steps with Adam.

Functions here are written for clarity: loops over layers, numpy einsum /
slicing for the sums that the definition states.
"""
from __future__ import annotations

import numpy as np

SHAPES = {"w1": (16, 1, 3, 3), "b1": (16,), "w2": (32, 16, 3, 3), "b2": (32,),
          "w3": (32, 32, 3, 3), "b3": (32,), "wh": (32,), "bh": (1,), "v": (16, 8), "bv": (1,)}
ORDER = ["w1", "b1", "w2", "b2", "w3", "b3", "wh", "bh", "v", "bv"]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())  # 14,210


def bf16_round(a) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps 8 significant bits: the float64 value is rounded to 8 bits
    of mantissa directly (no float32 step), with the usual exponent range.
    """
    a = np.asarray(a, np.float64)
    m, e = np.frexp(a)            # a = m * 2^e, 0.5 <= |m| < 1
    scaled = m * 256.0            # 8 significant bits above the binary point
    r = np.round(scaled)          # numpy rounds half to even
    return np.ldexp(r / 256.0, e)


def input_from_level(L: np.ndarray) -> np.ndarray:
    """x = bf16(L/255 - 0.5) as float64 [1][H][W]."""
    return bf16_round(np.asarray(L, np.float64) / 255.0 - 0.5)[None]


def init_params(seed: int = 0) -> dict:
    """He-style seeded initial weights (float64, not rounded)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([23, seed])))
    p = {}
    p["w1"] = rng.standard_normal(SHAPES["w1"]) * np.sqrt(2.0 / 9)
    p["w2"] = rng.standard_normal(SHAPES["w2"]) * np.sqrt(2.0 / (16 * 9))
    p["w3"] = rng.standard_normal(SHAPES["w3"]) * np.sqrt(2.0 / (32 * 9))
    p["wh"] = rng.standard_normal(SHAPES["wh"]) * np.sqrt(1.0 / 32)
    p["v"] = rng.standard_normal(SHAPES["v"]) * np.sqrt(1.0 / 128)
    for k in ["b1", "b2", "b3", "bh", "bv"]:
        p[k] = np.zeros(SHAPES[k])
    return p


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float64).ravel() for k in ORDER])


def unflatten(v: np.ndarray) -> dict:
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(v[o:o + n], np.float64).reshape(SHAPES[k])
        o += n
    return out


def rounded(p: dict) -> dict:
    """The bfloat16-rounded weights the forward pass uses (biases, head and pooling stay float)."""
    q = dict(p)
    for k in ["w1", "w2", "w3"]:
        q[k] = bf16_round(p[k])
    return q


def _pad(a):
    return np.pad(a, ((0, 0), (1, 1), (1, 1)))


def conv3x3_s2(a: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[o][i][j] = b[o] + sum_{c,dy,dx} w[o][c][dy][dx] a[c][2i+dy-1][2j+dx-1]."""
    C, H, W = a.shape
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    ap = _pad(a)
    out = np.zeros((w.shape[0], Ho, Wo)) + b[:, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = ap[:, dy:dy + 2 * Ho:2, dx:dx + 2 * Wo:2]   # [C][Ho][Wo]
            out += np.einsum("oc,cij->oij", w[:, :, dy, dx], patch)
    return out


def conv3x3_s2_backward(a: np.ndarray, w: np.ndarray, dout: np.ndarray):
    """Gradients of conv3x3_s2 w.r.t. its input, weights and bias."""
    C, H, W = a.shape
    Ho, Wo = dout.shape[1:]
    ap = _pad(a)
    dap = np.zeros_like(ap)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            patch = ap[:, dy:dy + 2 * Ho:2, dx:dx + 2 * Wo:2]
            dw[:, :, dy, dx] = np.einsum("oij,cij->oc", dout, patch)
            dap[:, dy:dy + 2 * Ho:2, dx:dx + 2 * Wo:2] += np.einsum("oc,oij->cij", w[:, :, dy, dx], dout)
    return dap[:, 1:H + 1, 1:W + 1], dw, dout.sum(axis=(1, 2))


def window_pool(h: np.ndarray, v: np.ndarray, bv: float, rows: int, cols: int) -> np.ndarray:
    """z[wy][wx] = bv + sum_{r,s} v[r][s] h[wy+r][wx+s]."""
    z = np.full((rows, cols), float(bv))
    for r in range(16):
        for s in range(8):
            z += v[r, s] * h[r:r + rows, s:s + cols]
    return z


def forward(L: np.ndarray, p: dict):
    """Keep-logits of one level image and the cached activations."""
    return forward_q(L, rounded(p))


def forward_q(L: np.ndarray, q: dict):
    """Same as forward with the weights taken as given (already rounded)."""
    x = input_from_level(L)
    z1 = conv3x3_s2(x, q["w1"], q["b1"]); a1 = np.maximum(z1, 0)
    z2 = conv3x3_s2(a1, q["w2"], q["b2"]); a2 = np.maximum(z2, 0)
    z3 = conv3x3_s2(a2, q["w3"], q["b3"]); a3 = np.maximum(z3, 0)
    h = np.einsum("c,cij->ij", q["wh"], a3) + q["bh"][0]
    Hc, Wc = L.shape[0] // 8, L.shape[1] // 8
    rows, cols = max(Hc - 15, 0), max(Wc - 7, 0)
    if rows == 0 or cols == 0:
        rows = cols = 0
    z = window_pool(h, q["v"], q["bv"][0], rows, cols)
    cache = dict(q=q, x=x, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, h=h)
    return z, cache


def head_resample(h_src: np.ndarray, src_size, dst_size) -> np.ndarray:
    """Head map of a level (dst_size = (Wk, Hk)) read from another level of its frame (src_size):
    destination cell (cy, cx) takes the source cell holding its centre, row
    min(floor((2cy+1) Hk_src / (2 Hk_dst)), Hc_src - 1), column likewise."""
    (ws, hs), (wd, hd) = src_size, dst_size
    ys = np.minimum(((2 * np.arange(hd // 8) + 1) * hs) // (2 * hd), hs // 8 - 1)
    xs = np.minimum(((2 * np.arange(wd // 8) + 1) * ws) // (2 * wd), ws // 8 - 1)
    return np.asarray(h_src)[np.ix_(ys, xs)]


def frame_logits(levels, p: dict, step: int = 1):
    """Keep-logits of every level of one frame (list of level images, largest first) when the
    network runs on levels 0, step, 2 step, ... and each level pools its group level's head map
    (head_resample; the identity for the group level itself)."""
    q = rounded(p)
    heads, out = {}, []
    for k, L in enumerate(levels):
        j = step * (k // step)
        if j not in heads:
            heads[j] = forward_q(levels[j], q)[1]["h"]
        Hk, Wk = L.shape
        src = (levels[j].shape[1], levels[j].shape[0])
        h = head_resample(heads[j], src, (Wk, Hk))
        rows, cols = max(Hk // 8 - 15, 0), max(Wk // 8 - 7, 0)
        if rows == 0 or cols == 0:
            rows = cols = 0
        out.append(window_pool(h, q["v"], q["bv"][0], rows, cols))
    return out


def bce_with_logits(z: np.ndarray, y: np.ndarray, pos_weight: float):
    """Mean of -[p y log s(z) + (1-y) log(1-s(z))] and its gradient w.r.t. z."""
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    if z.size == 0:
        return 0.0, np.zeros_like(z)
    log_s = -np.logaddexp(0.0, -z)        # log sigmoid(z)
    log_1ms = -np.logaddexp(0.0, z)       # log (1 - sigmoid(z))
    loss = -(pos_weight * y * log_s + (1 - y) * log_1ms)
    s = np.exp(log_s)
    dz = (pos_weight * y * (s - 1) + (1 - y) * s) / z.size
    return float(loss.mean()), dz


def backward(cache: dict, dz: np.ndarray) -> dict:
    """Gradients of all parameters (w.r.t. the rounded weights) given dL/dz."""
    q = cache["q"]
    h = cache["h"]
    rows, cols = dz.shape
    g = {k: np.zeros(SHAPES[k]) for k in ORDER}
    dh = np.zeros_like(h)
    g["bv"][0] = dz.sum()
    for r in range(16):
        for s in range(8):
            g["v"][r, s] = np.sum(dz * h[r:r + rows, s:s + cols])
            dh[r:r + rows, s:s + cols] += q["v"][r, s] * dz
    g["bh"][0] = dh.sum()
    g["wh"] = np.einsum("ij,cij->c", dh, cache["a3"])
    da3 = q["wh"][:, None, None] * dh[None]
    dz3 = da3 * (cache["z3"] > 0)
    da2, g["w3"], g["b3"] = conv3x3_s2_backward(cache["a2"], q["w3"], dz3)
    dz2 = da2 * (cache["z2"] > 0)
    da1, g["w2"], g["b2"] = conv3x3_s2_backward(cache["a1"], q["w2"], dz2)
    dz1 = da1 * (cache["z1"] > 0)
    _, g["w1"], g["b1"] = conv3x3_s2_backward(cache["x"], q["w1"], dz1)
    return g


def loss_and_grad(levels, labels, p: dict, pos_weight: float):
    """Mean over levels of the per-level mean BCE, and its gradient."""
    total, grads = 0.0, {k: np.zeros(SHAPES[k]) for k in ORDER}
    n = 0
    for L, y in zip(levels, labels):
        z, cache = forward(L, p)
        if z.size == 0:
            continue
        loss, dz = bce_with_logits(z, y, pos_weight)
        g = backward(cache, dz)
        total += loss
        for k in ORDER:
            grads[k] += g[k]
        n += 1
    n = max(n, 1)
    return total / n, {k: v / n for k, v in grads.items()}


class Adam:
    """m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr mhat / (sqrt(vhat) + eps)."""

    def __init__(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = np.zeros(N_PARAMS)
        self.v = np.zeros(N_PARAMS)
        self.t = 0

    def step(self, params: np.ndarray, grad: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mhat = self.m / (1 - self.b1 ** self.t)
        vhat = self.v / (1 - self.b2 ** self.t)
        return params - self.lr * mhat / (np.sqrt(vhat) + self.eps)
