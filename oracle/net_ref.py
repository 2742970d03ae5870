"""Plain FP64 CPU reference of the learned initial guess's network and field glue.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the test suite may use it.
The paper has no network; this file restates, in plain numpy, what the CUDA network
computes, so that its forward pass, its gradients and its AdamW step can be checked
element by element.  It is pinned (tests/test_net_ref.py) by central finite differences of
its own loss, by closed forms (a single-tap kernel is a shift, a ReLU network with positive
pre-activations is linear) and by the AdamW recurrence run by hand on scalars.

Layouts (the interface of both sides): images [B, H, W, C] (NHWC); a layer's weights
[9, co, ci] with tap t = 3 (dy + 1) + (dx + 1) multiplying the input pixel (h + dy, w + dx)
(zero outside the image), biases [co]; the flat parameter vector holds, layer by layer, the
weights then the biases, with channel counts padded: ci_0 = 16, 32 or 64 (the smallest that
holds cin), hidden elsewhere, co_3 = 16.

`quant=True` reproduces the BF16 rounding points of the tensor-core path: the input, every
weight, every hidden activation (after ReLU, through FP32) and every layer's output gradient
(through FP32) are rounded to BF16 (round to nearest even); all arithmetic between those
points is exact FP64.  `quant=False` is the plain FP64 network (used for the finite-difference
pins, since rounding is not differentiable).
"""
from __future__ import annotations

import numpy as np

LAYERS = 4


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), via FP32, returned as float64."""
    x32 = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def pad_in(c: int) -> int:
    return 16 if c <= 16 else (32 if c <= 32 else 64)


def shape(cin: int, hidden: int, cout: int):
    ci = [pad_in(cin), hidden, hidden, hidden]
    co = [hidden, hidden, hidden, 16]
    return ci, co


def n_params(cin, hidden, cout) -> int:
    ci, co = shape(cin, hidden, cout)
    return sum(9 * co[l] * ci[l] + co[l] for l in range(LAYERS))


def unpack(params, cin, hidden, cout):
    """Flat vector -> [(W_l [9, co, ci], b_l [co])]."""
    ci, co = shape(cin, hidden, cout)
    out, off = [], 0
    for l in range(LAYERS):
        nw = 9 * co[l] * ci[l]
        W = np.asarray(params[off:off + nw], dtype=np.float64).reshape(9, co[l], ci[l])
        off += nw
        b = np.asarray(params[off:off + co[l]], dtype=np.float64)
        off += co[l]
        out.append((W, b))
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def shift(x, dy, dx):
    """s[b, h, w] = x[b, h + dy, w + dx], zero outside the image."""
    B, H, W, C = x.shape
    p = np.zeros((B, H + 2, W + 2, C), dtype=x.dtype)
    p[:, 1:H + 1, 1:W + 1] = x
    return p[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]


def conv3x3(x, W):
    """out[p, co] = sum over taps t and channels ci of x[p + off_t, ci] W[t, co, ci]."""
    out = 0.0
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        out = out + shift(x, dy, dx) @ W[t].T
    return out


def conv3x3_transpose(g, W):
    """Adjoint of conv3x3 in its input: d[p, ci] = sum_t sum_co g[p - off_t, co] W[t, co, ci]."""
    out = 0.0
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        out = out + shift(g, -dy, -dx) @ W[t]
    return out


def forward(params, x, cin, hidden, cout, quant=True):
    """Returns (y [B, H, W, cout], cache of the layer inputs and pre-activations)."""
    q = bf16 if quant else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(params, cin, hidden, cout)
    ci, _ = shape(cin, hidden, cout)
    x = np.asarray(x, dtype=np.float64)
    a0 = np.zeros(x.shape[:3] + (ci[0],))
    a0[..., :cin] = x
    acts, pre = [q(a0)], []
    for l, (W, b) in enumerate(layers):
        z = conv3x3(acts[l], q(W)) + b
        pre.append(z)
        if l < LAYERS - 1:
            r = np.maximum(z, 0.0)
            acts.append(q(r) if quant else r)
    y = pre[-1][..., :cout]
    return y, {"acts": acts, "pre": pre, "layers": layers}


def loss_and_gradients(params, x, target, cin, hidden, cout, quant=True):
    """Mean squared error over the B*H*W*cout outputs and its gradient (flat layout)."""
    q = bf16 if quant else (lambda v: np.asarray(v, dtype=np.float64))
    y, cache = forward(params, x, cin, hidden, cout, quant)
    target = np.asarray(target, dtype=np.float64)
    n = y.size
    d = y - target
    loss = float(np.sum(d * d) / n)
    g = np.zeros(cache["pre"][-1].shape)
    g[..., :cout] = 2.0 * d / n
    if quant:
        g = np.asarray(g, dtype=np.float32).astype(np.float64)
    G = q(g)
    grads = [None] * LAYERS
    for l in range(LAYERS - 1, -1, -1):
        a = cache["acts"][l]
        W, _ = cache["layers"][l]
        dW = np.zeros_like(W)
        for t in range(9):
            dy, dx = t // 3 - 1, t % 3 - 1
            dW[t] = np.einsum("bhwo,bhwi->oi", G, shift(a, dy, dx))
        db = G.sum(axis=(0, 1, 2))
        grads[l] = (dW, db)
        if l == 0:
            break
        da = conv3x3_transpose(G, q(W))
        gl = da * (a > 0)
        if quant:
            gl = np.asarray(gl, dtype=np.float32).astype(np.float64)
        G = q(gl)
    return loss, pack(grads)


def adamw(params, grad, m, v, step, lr, wd, cin, hidden, cout, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step (bias-corrected moments, decoupled decay on weights only).
    Returns new (params, m, v)."""
    ci, co = shape(cin, hidden, cout)
    is_bias = np.zeros(len(params), dtype=bool)
    off = 0
    for l in range(LAYERS):
        off += 9 * co[l] * ci[l]
        is_bias[off:off + co[l]] = True
        off += co[l]
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = np.where(is_bias, params, params - lr * wd * params)
    p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


# ---------------------------------------------------------------- field glue
LEARN_IDX = [0, 1, 2, 4, 5, 6, 8, 10, 11, 12]   # rho, u1, u2, theta, s11, s12, s22, s33, q1, q2
LEARN_REST = [1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
FEATURE_SCALE, TARGET_SCALE = 10.0, 100.0


def interpolate(coarse):
    """Cell-centred bilinear interpolation to the grid twice as fine: a fine cell centre lies a
    quarter coarse cell from its parent's centre, so it takes 3/4 of the parent and 1/4 of the
    neighbour on that side, per axis; beyond the outermost centres the neighbour is the parent
    itself (constant extension)."""
    Hc, Wc, K = coarse.shape
    out = np.zeros((2 * Hc, 2 * Wc, K))
    for I in range(2 * Hc):
        i = I // 2
        i2 = min(i + 1, Hc - 1) if I % 2 else max(i - 1, 0)
        for J in range(2 * Wc):
            j = J // 2
            j2 = min(j + 1, Wc - 1) if J % 2 else max(j - 1, 0)
            out[I, J] = (0.75 * 0.75 * coarse[i, j] + 0.75 * 0.25 * coarse[i, j2] + 0.25 * 0.75 * coarse[i2, j]
                         + 0.25 * 0.25 * coarse[i2, j2])
    return out


def features(coarse, Kn, U, lx=1.0, ly=1.0):
    pro = interpolate(np.asarray(coarse, dtype=np.float64))
    H, W, _ = pro.shape
    x = np.zeros((H, W, 19))
    for k, (i, r) in enumerate(zip(LEARN_IDX, LEARN_REST)):
        x[..., k] = FEATURE_SCALE * (pro[..., i] - r) / U
    x[..., 10] = np.log10(Kn)
    x[..., 11] = np.log10(Kn * W / lx)
    x[..., 12] = U
    x[..., 13] = ((np.arange(W) + 0.5) / W)[None, :]
    x[..., 14] = ((np.arange(H) + 0.5) / H)[:, None]
    x[0, :, 15] = 1.0
    x[:, W - 1, 16] = 1.0
    x[H - 1, :, 17] = 1.0
    x[:, 0, 18] = 1.0
    return pro, x


def targets(pro, fine, U):
    return np.stack([TARGET_SCALE * (fine[..., i] - pro[..., i]) / U for i in LEARN_IDX], axis=-1)


def combine(pro, y, U):
    out = np.array(pro, dtype=np.float64)
    for k, i in enumerate(LEARN_IDX):
        out[..., i] += U / TARGET_SCALE * y[..., k]
    out[..., [3, 7, 9, 13]] = 0.0
    return out
