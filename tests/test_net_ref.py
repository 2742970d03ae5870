"""Pins of the CPU reference of the learned initial guess's network (oracle/net_ref.py).

The network is not in the paper, so the reference is pinned by mathematics that does not
depend on it: finite differences of its own loss, closed forms (a one-tap kernel is a shift,
the transpose is the adjoint, an identity network passes positive inputs through), the BF16
rounding of an independent library, the AdamW recurrence worked by hand, and the exactness of
bilinear interpolation on linear fields.
"""
import numpy as np
import pytest
import torch

from oracle import net_ref as R

CIN, HID, COUT = 3, 32, 2


def rand_params(rng, cin=CIN, hid=HID, cout=COUT, scale=0.3):
    ci, co = R.shape(cin, hid, cout)
    layers = []
    for l in range(R.LAYERS):
        W = np.zeros((9, co[l], ci[l]))
        rci = cin if l == 0 else hid
        rco = cout if l == R.LAYERS - 1 else hid
        W[:, :rco, :rci] = rng.standard_normal((9, rco, rci)) * scale / np.sqrt(9 * rci) * 2
        b = np.zeros(co[l])
        b[:rco] = rng.standard_normal(rco) * 0.1
        layers.append((W, b))
    return R.pack(layers)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.uniform(-20, 20, 5000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)]])
    ours = R.bf16(x)
    lib = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, lib)
    assert R.bf16(1 + 2 ** -8)[()] == 1.0                 # halfway, even neighbour is 1
    assert R.bf16(1 + 3 * 2 ** -8)[()] == 1 + 2 ** -6     # halfway, even neighbour is 1 + 2^-6


def test_one_tap_kernel_is_a_shift():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 7, 4))
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        W = np.zeros((9, 4, 4))
        W[t] = np.eye(4)
        y = R.conv3x3(x, W)
        for h in range(5):
            for w in range(7):
                src = (h + dy, w + dx)
                exp = x[:, src[0], src[1]] if 0 <= src[0] < 5 and 0 <= src[1] < 7 else 0.0
                assert np.array_equal(y[:, h, w], exp + 0 * y[:, h, w])


def test_transpose_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 5, 3))
    g = rng.standard_normal((2, 6, 5, 4))
    W = rng.standard_normal((9, 4, 3))
    lhs = np.sum(R.conv3x3(x, W) * g)
    rhs = np.sum(x * R.conv3x3_transpose(g, W))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_identity_network_passes_positive_inputs():
    cin, hid, cout = 3, 32, 2
    ci, co = R.shape(cin, hid, cout)
    layers = []
    for l in range(R.LAYERS):
        W = np.zeros((9, co[l], ci[l]))
        for c in range(min(co[l], ci[l])):
            W[4, c, c] = 1.0   # centre tap
        layers.append((W, np.zeros(co[l])))
    x = np.random.default_rng(3).uniform(0.1, 2.0, (1, 4, 5, cin))
    y, _ = R.forward(R.pack(layers), x, cin, hid, cout, quant=False)
    assert np.array_equal(y, x[..., :cout])


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    p = rand_params(rng)
    x = rng.standard_normal((2, 5, 6, CIN))
    t = rng.standard_normal((2, 5, 6, COUT)) * 0.1
    loss, g = R.loss_and_gradients(p, x, t, CIN, HID, COUT, quant=False)
    ci, co = R.shape(CIN, HID, COUT)
    # sample real weights and biases of every layer, plus padded entries (gradient zero)
    picks, off = [], 0
    for l in range(R.LAYERS):
        nw = 9 * co[l] * ci[l]
        rci = CIN if l == 0 else HID
        rco = COUT if l == R.LAYERS - 1 else HID
        for _ in range(8):
            tap, o, i = rng.integers(9), rng.integers(rco), rng.integers(rci)
            picks.append(off + (tap * co[l] + o) * ci[l] + i)
        picks.append(off + nw + int(rng.integers(rco)))
        off += nw + co[l]
    h = 1e-6
    for k in picks:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (R.loss_and_gradients(pp, x, t, CIN, HID, COUT, quant=False)[0]
              - R.loss_and_gradients(pm, x, t, CIN, HID, COUT, quant=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * abs(g[k]) + 1e-9, (k, fd, g[k])
    # padded input channels of layer 0 and padded outputs of layer 3 get exactly zero
    W0 = g[:9 * co[0] * ci[0]].reshape(9, co[0], ci[0])
    assert np.all(W0[:, :, CIN:] == 0.0)
    layers = R.unpack(g, CIN, HID, COUT)
    assert np.all(layers[3][0][:, COUT:, :] == 0.0) and np.all(layers[3][1][COUT:] == 0.0)


def test_quantized_gradient_is_close_to_exact():
    rng = np.random.default_rng(5)
    p = rand_params(rng)
    x = rng.standard_normal((1, 6, 6, CIN))
    t = rng.standard_normal((1, 6, 6, COUT)) * 0.1
    _, g0 = R.loss_and_gradients(p, x, t, CIN, HID, COUT, quant=False)
    _, g1 = R.loss_and_gradients(p, x, t, CIN, HID, COUT, quant=True)
    assert np.linalg.norm(g1 - g0) <= 0.05 * np.linalg.norm(g0)


def test_adamw_by_hand():
    cin, hid, cout = 3, 32, 2
    n = R.n_params(cin, hid, cout)
    rng = np.random.default_rng(6)
    p0 = rng.standard_normal(n)
    g = rng.standard_normal(n)
    lr, wd, eps = 1e-2, 0.1, 1e-8
    p1, m1, v1 = R.adamw(p0, g, np.zeros(n), np.zeros(n), 1, lr, wd, cin, hid, cout)
    # first step: m_hat = g, v_hat = g^2
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    ci, co = R.shape(cin, hid, cout)
    b0 = 9 * co[0] * ci[0]            # first bias of layer 0
    w = 0                             # first weight of layer 0
    assert p1[w] == pytest.approx(p0[w] * (1 - lr * wd) - lr * g[w] / (abs(g[w]) + eps), rel=1e-12)
    assert p1[b0] == pytest.approx(p0[b0] - lr * g[b0] / (abs(g[b0]) + eps), rel=1e-12)
    # second step with the same gradient: moments 0.19 g and 0.001999 g^2, bias corrections 0.19, 0.001999
    p2, _, _ = R.adamw(p1, g, m1, v1, 2, lr, wd, cin, hid, cout)
    assert p2[b0] == pytest.approx(p1[b0] - lr * g[b0] / (abs(g[b0]) + eps), rel=1e-9)


def test_interpolation_is_exact_on_linear_fields_inside():
    Hc, Wc = 6, 5
    yc = (np.arange(Hc) + 0.5) / Hc
    xc = (np.arange(Wc) + 0.5) / Wc
    a, bx, by = 0.7, -1.3, 2.1
    coarse = np.zeros((Hc, Wc, 14))
    coarse[..., 3] = a + bx * xc[None, :] + by * yc[:, None]
    fine = R.interpolate(coarse)
    yf = (np.arange(2 * Hc) + 0.5) / (2 * Hc)
    xf = (np.arange(2 * Wc) + 0.5) / (2 * Wc)
    exact = a + bx * xf[None, :] + by * yf[:, None]
    inner = fine[1:-1, 1:-1, 3] - exact[1:-1, 1:-1]
    assert np.max(np.abs(inner)) < 1e-14
    # constant extension beyond the outermost centres: the corner cell equals its parent
    assert fine[0, 0, 3] == pytest.approx(coarse[0, 0, 3], rel=1e-15)


def test_targets_and_combine_invert():
    rng = np.random.default_rng(7)
    coarse = rng.standard_normal((4, 3, 14))
    pro, x = R.features(coarse, 0.1, 0.3)
    fine = rng.standard_normal(pro.shape)
    t = R.targets(pro, fine, 0.3)
    back = R.combine(pro, t, 0.3)
    assert np.allclose(back[..., R.LEARN_IDX], fine[..., R.LEARN_IDX], rtol=0, atol=1e-14)
    assert x.shape == (8, 6, 19) and np.all(x[0, :, 15] == 1) and np.all(x[:, 0, 18] == 1)
