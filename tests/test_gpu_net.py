"""GPU parity of the learned initial guess: the tensor-core network (forward, gradients, AdamW)
against the FP64 CPU reference that reproduces its BF16 rounding points, the field glue
against its plain definition, the Grad state against the oracle's field formulas, and the
learned solve against the plain solve it must agree with."""
import math

import numpy as np
import pytest
import torch

from inputs import lid_cavity
from oracle import net_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_13164_gb300 import learned

    return learned


def rand_params(rng, cin, hid, cout, scale=1.0):
    ci, co = R.shape(cin, hid, cout)
    layers = []
    for l in range(R.LAYERS):
        W = np.zeros((9, co[l], ci[l]))
        rci = cin if l == 0 else hid
        rco = cout if l == R.LAYERS - 1 else hid
        W[:, :rco, :rci] = rng.uniform(-1, 1, (9, rco, rci)) * scale * math.sqrt(6.0 / (9 * rci))
        b = np.zeros(co[l])
        b[:rco] = rng.standard_normal(rco) * 0.05
        layers.append((W, b))
    return R.pack(layers).astype(np.float32)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


SHAPES = [(19, 64, 10, 2, 19, 40), (19, 64, 10, 1, 8, 32), (5, 32, 3, 3, 9, 17)]


@pytest.mark.parametrize("cin,hid,cout,B,H,W", SHAPES)
def test_forward_matches_reference(L, cin, hid, cout, B, H, W):
    rng = np.random.default_rng(10 + cin + H)
    p = rand_params(rng, cin, hid, cout)
    x = rng.standard_normal((B, H, W, cin)).astype(np.float32)
    net = L.Net(cin, hid, cout, max_pixels=B * H * W)
    net.set_params(torch.from_numpy(p))
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref, _ = R.forward(p.astype(np.float64), x.astype(np.float64), cin, hid, cout, quant=True)
    # FP32 accumulation against exact sums between the same BF16 rounding points: a few
    # activations may land one BF16 step apart, nothing more
    assert rel(y, ref) < 2e-3
    assert np.max(np.abs(y - ref)) < 2e-2 * np.max(np.abs(ref))
    # padding round trip of the parameters
    assert np.array_equal(net.get_params().cpu().numpy(), p)


@pytest.mark.parametrize("cin,hid,cout,B,H,W", SHAPES)
def test_gradients_match_reference(L, cin, hid, cout, B, H, W):
    rng = np.random.default_rng(20 + cin + H)
    p = rand_params(rng, cin, hid, cout)
    x = rng.standard_normal((B, H, W, cin)).astype(np.float32)
    t = (rng.standard_normal((B, H, W, cout)) * 0.5).astype(np.float32)
    net = L.Net(cin, hid, cout, max_pixels=B * H * W)
    net.set_params(torch.from_numpy(p))
    g, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = R.loss_and_gradients(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), cin, hid,
                                      cout, quant=True)
    assert loss == pytest.approx(lref, rel=1e-4)
    for l, ((Wg, bg), (Wr, br)) in enumerate(zip(R.unpack(g, cin, hid, cout), R.unpack(gref, cin, hid, cout))):
        assert rel(Wg, Wr) < 5e-3, l
        assert rel(bg, br) < 5e-3, l
    # and close to the exact FP64 gradient (BF16 rounding is the only approximation)
    _, gexact = R.loss_and_gradients(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), cin, hid, cout,
                                     quant=False)
    assert rel(g, gexact) < 5e-2
    # deterministic: the same call twice gives the same bits
    g2, _ = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    assert np.array_equal(g2.cpu().numpy().astype(np.float64), g)


def test_adamw_step_matches_reference(L):
    cin, hid, cout, B, H, W = 19, 64, 10, 2, 16, 32
    rng = np.random.default_rng(30)
    p = rand_params(rng, cin, hid, cout)
    x = torch.from_numpy(rng.standard_normal((B, H, W, cin)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, H, W, cout)).astype(np.float32)).cuda()
    net = L.Net(cin, hid, cout, max_pixels=B * H * W)
    net.set_params(torch.from_numpy(p))
    m = np.zeros(p.size)
    v = np.zeros(p.size)
    pr = p.astype(np.float64)
    lr, wd = 1e-3, 0.05
    for step in (1, 2, 3):
        g, _ = net.gradients(x, t)
        g = g.cpu().numpy().astype(np.float64)
        net.train_step(x, t, lr, wd)
        pr, m, v = R.adamw(pr, g, m, v, step, lr, wd, cin, hid, cout)
        got = net.get_params().cpu().numpy().astype(np.float64)
        assert np.allclose(got, pr, rtol=1e-5, atol=1e-6 * lr), step
        pr = got   # continue from the GPU's FP32 parameters
    assert np.all(got[R.n_params(cin, hid, cout) - 6:] == 0.0)   # padded output biases stay zero


def test_training_reduces_loss(L):
    cin, hid, cout, B, H, W = 19, 64, 10, 8, 32, 32
    rng = np.random.default_rng(40)
    teacher = L.Net(cin, hid, cout, max_pixels=B * H * W, seed=7)
    x = torch.from_numpy(rng.standard_normal((B, H, W, cin)).astype(np.float32)).cuda()
    t = teacher.forward(x)
    net = L.Net(cin, hid, cout, max_pixels=B * H * W, seed=8)
    l0 = net.train_step(x, t, 1e-3)
    for _ in range(300):
        l1 = net.train_step(x, t, 1e-3)
    assert math.isfinite(l1) and l1 < 0.2 * l0, (l0, l1)


def test_glue_matches_reference(L):
    rng = np.random.default_rng(50)
    Hc, Wc, Kn, U = 5, 7, 0.07, 0.23
    coarse = rng.standard_normal((Hc, Wc, 14))
    pro, x = L.features(torch.from_numpy(coarse).cuda(), Kn, U)
    pref, xref = R.features(coarse, Kn, U)
    assert np.allclose(pro.cpu().numpy(), pref, rtol=1e-14, atol=1e-14)
    assert np.allclose(x.cpu().numpy(), xref, rtol=1e-6, atol=1e-6)
    fine = rng.standard_normal(pref.shape)
    t = L.targets(pro, torch.from_numpy(fine).cuda(), U).cpu().numpy()
    assert np.allclose(t, R.targets(pref, fine, U), rtol=1e-6, atol=1e-6)
    y = rng.standard_normal((2 * Hc, 2 * Wc, 10)).astype(np.float32)
    out = L.combine(pro, torch.from_numpy(y).cuda(), U).cpu().numpy()
    assert np.allclose(out, R.combine(pref, y.astype(np.float64), U), rtol=1e-14, atol=1e-14)


def test_grad_state_reproduces_fields(L):
    """The Grad state built from fields gives those fields back (trace of the stress removed),
    by the library's field kernel and by the oracle's field formula on the returned state."""
    import oracle
    from paper_2206_13164_gb300 import from_problem

    rng = np.random.default_rng(60)
    prob = lid_cavity(16, 6, 0.1, 0.2, levels=2)
    s = from_problem(prob)
    nc = 16 * 16
    f = np.zeros((nc, 14))
    f[:, 0] = rng.uniform(0.8, 1.2, nc)
    f[:, 1:3] = rng.uniform(-0.2, 0.2, (nc, 2))
    f[:, 4] = rng.uniform(0.8, 1.3, nc)
    f[:, [5, 6, 8, 10]] = rng.standard_normal((nc, 4)) * 0.05
    f[:, [11, 12]] = rng.standard_normal((nc, 2)) * 0.05
    s.set_state_from_fields(torch.from_numpy(f).cuda())
    back = s.fields().reshape(nc, 14).cpu().numpy()
    exp = f.copy()
    tr = (f[:, 5] + f[:, 8] + f[:, 10]) / 3.0
    for k in (5, 8, 10):
        exp[:, k] -= tr
    assert np.allclose(back, exp, rtol=0, atol=1e-14)
    P, F = s.get_state()
    P, F = P.cpu().numpy(), F.cpu().numpy()
    for c in range(0, nc, 17):
        assert np.allclose(oracle.cell_fields(6, P[c], F[c]), exp[c], rtol=0, atol=1e-14)
    # only the 13-moment entries are nonzero
    al = oracle.alphas(6)
    deg = al.sum(1)
    assert np.all(F[:, deg >= 4] == 0.0)


@pytest.mark.parametrize("with_net", [False, True])
def test_learned_solve_reaches_the_plain_solution(L, with_net):
    """A network (here random, untrained) cannot change the answer: the candidates are chosen by
    the residual after the same FAS cycles and the final cycles stop at 1e-8 of the plain
    start's residual, so the fields equal those of the plain solve."""
    Kn, U, M = 0.1, 0.3, 5
    net = L.Net(max_pixels=32 * 32, seed=3) if with_net else None
    plain, rec = L.plain_solve(32, M, Kn, U)
    assert rec["status"] == 0
    ls = L.LearnedSolve(32, M, Kn, U, start=16, net=net)
    out = ls.run(tol=1e-8, coarse_tol=1e-6, polish=2, decide=2)
    assert out["status"] == 0 and out["rel_res"] <= 1e-8
    assert out["cycles"] < rec["cycles"]
    assert out["wasted_cycles"] == (2 if with_net else 0)
    a = plain.fields().cpu().numpy()
    b = ls.target.fields().cpu().numpy()
    scale = np.max(np.abs(a), axis=(0, 1))
    assert np.max(np.abs(a - b) / np.maximum(scale, 1e-3)) < 1e-6


def test_trained_network_gains_over_the_climb_without_it(L):
    """The committed network (trained on solver solutions at 64x64 and 128x128, M = 8) on a
    held-out cavity: fewer FAS cycles and less wall time to 1e-8 than the same climb without
    it, which in turn beats the plain start; all three reach the same fields."""
    import os

    if not os.path.exists(L.WEIGHTS):
        pytest.fail("trained weights missing: " + L.WEIGHTS)
    Kn, U, M, N = 0.03, 0.35, 8, 128
    net = L.Net.load(max_pixels=N * N)
    out = L.evaluate(N, M, Kn, U, net, start=32)
    plain, base, learned = out["plain"], out["no_net"], out["net"]
    for r in (plain, base, learned):
        assert r["status"] == 0 and r["rel_res"] <= 1e-8
    assert base["max_field_diff"] < 1e-6 and learned["max_field_diff"] < 1e-6
    assert [c["used"] for c in learned["climb"]] == ["net", "net"]
    assert learned["cycles"] < base["cycles"] < plain["cycles"]
    assert learned["t_total"] < plain["t_total"]
