"""The learned coarse-level correction (nrmg_fas_cycle_learned, nrmg_learned_correct): without a
network the cycle is the plain cycle of Algorithm 2 bit for bit; the correction increment moves
the ten fields as stated in nrmg_net.h; the network input holds the fields it is defined by;
with the committed network the cycle reaches the plain cycle's solution."""
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

LEARN_IDX = [0, 1, 2, 4, 5, 6, 8, 10, 11, 12]
REST = np.array([1.0, 0, 0, 1.0, 0, 0, 0, 0, 0, 0])


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_13164_gb300 import learned

    return learned


@pytest.mark.parametrize("order,slope,M", [(1, 0, 5), (2, 2, 6)])
def test_cycle_without_network_is_the_plain_cycle(L, order, slope, M):
    a = L.lid_solver(32, M, 0.1, 0.3, order=order, slope=slope, dtnu=0.0)
    b = L.lid_solver(32, M, 0.1, 0.3, order=order, slope=slope, dtnu=0.0)
    lc = L.LearnedCycle(b, 0.1, 0.3)
    for _ in range(3):
        ra = a.fas_cycle()
        rb, kept, sc = lc.cycle(None)
        assert ra == rb and not kept and sc > 0.0
    for lev in range(a.levels):
        Pa, Fa = a.get_state(lev)
        Pb, Fb = b.get_state(lev)
        assert torch.equal(Pa, Pb) and torch.equal(Fa, Fb)


def _fields(s):
    return s.fields().cpu().numpy().reshape(-1, 14)


@pytest.mark.parametrize("channel", [0, 1, 3, 5, 8])
def test_correction_increment_moves_its_field(L, channel):
    """One field's correction (rho, u1, theta, s12 or q1) of 3e-4: that field moves by it, the
    others stay put up to the second-order terms of the basis change."""
    U = 0.3
    s = L.lid_solver(16, 6, 0.1, U)
    for _ in range(3):
        s.fas_cycle()
    f0 = _fields(s)
    cells = f0.shape[0]
    y = torch.zeros((cells, 10), dtype=torch.float32, device="cuda")
    y[:, channel] = 0.01
    delta = U * 1.0 * 0.01 / 10.0
    L.learned_correct(s, y, 1.0, U)
    f1 = _fields(s)
    moved = LEARN_IDX[channel]
    assert np.allclose(f1[:, moved] - f0[:, moved], delta, rtol=1e-6, atol=1e-12)
    rho = f0[:, 0]
    for k, idx in enumerate(LEARN_IDX):
        if idx == moved:
            continue
        # a velocity change re-centres the stress and heat flux (terms of order rho delta^2 and
        # delta sigma); every other field is exact
        tol = 1e-12 + (10.0 * (rho.max() * delta ** 2 + delta * np.abs(f0[:, 5:]).max()) if channel == 1 and idx >= 5
                       else 0.0)
        assert np.max(np.abs(f1[:, idx] - f0[:, idx])) <= tol + 1e-10 * np.max(np.abs(f0[:, idx])), (channel, idx)


def test_network_input_channels(L):
    U, Kn, N = 0.3, 0.1, 32
    s = L.lid_solver(N, 6, Kn, U)
    lc = L.LearnedCycle(s, Kn, U)
    lc.cycle(None)
    x = torch.empty((N, N, L.CORR_CIN), dtype=torch.float32, device="cuda")
    fine = torch.empty((N, N, 14), dtype=torch.float64, device="cuda")
    _, _, sc = lc.cycle(None, x_out=x, fine_out=fine)
    x, fine = x.cpu().numpy().astype(np.float64), fine.cpu().numpy()
    assert sc > 0.0
    ref = (fine[..., LEARN_IDX] - REST) * 10.0 / U
    assert np.allclose(x[..., 10:20], ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
    # the interpolated coarse change is a convex combination of coarse values scaled by their
    # largest magnitude
    assert np.abs(x[..., :10]).max() <= 1.0 + 1e-6 and np.abs(x[..., :10]).max() >= 0.5
    I, J = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    assert np.allclose(x[..., 20], np.log10(Kn), atol=1e-6)
    assert np.allclose(x[..., 21], np.log10(Kn * N), atol=1e-6)
    assert np.allclose(x[..., 22], U, atol=1e-7)
    assert np.allclose(x[..., 23], (J + 0.5) / N, atol=1e-7) and np.allclose(x[..., 24], (I + 0.5) / N, atol=1e-7)
    assert np.array_equal(x[..., 25], (I == 0) * 1.0) and np.array_equal(x[..., 26], (J == N - 1) * 1.0)
    assert np.array_equal(x[..., 27], (I == N - 1) * 1.0) and np.array_equal(x[..., 28], (J == 0) * 1.0)


def test_rejected_correction_leaves_the_plain_update(L):
    """A network whose output is a huge constant: its candidate is non-physical or worse, so
    the cycle keeps the plain update and equals the plain cycle."""
    a = L.lid_solver(32, 6, 0.1, 0.3)
    b = L.lid_solver(32, 6, 0.1, 0.3)
    net = L.Net(L.CORR_CIN, 64, 10, max_pixels=32 * 32)
    p = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    p[-16:] = 1e4  # last layer's biases: y = 1e4 everywhere
    net.set_params(p)
    lc = L.LearnedCycle(b, 0.1, 0.3)
    for _ in range(2):
        ra = a.fas_cycle()
        rb, kept, _ = lc.cycle(net)
        assert not kept and ra == rb
    assert torch.equal(a.get_state()[1], b.get_state()[1])


@pytest.mark.skipif(not os.path.exists(os.path.join(os.path.dirname(__file__), "..", "paper_2206_13164_gb300",
                                                    "weights", "corr_net.npz")), reason="no trained weights")
def test_trained_correction_reaches_the_plain_solution(L):
    """Held-out cavity (128x128, M = 8, Kn 0.03, lid 0.35; training draws exclude it): the
    cycle with the committed network converges to the plain cycle's solution and needs no
    more cycles than the plain cycle (the acceptance test keeps it from doing worse)."""
    net = L.Net.load(L.CORR_WEIGHTS, max_pixels=128 * 128)
    ev = L.evaluate_correction(128, 8, 0.03, 0.35, net)
    assert ev["learned"]["rel_res"] <= 1e-8 and ev["plain"]["rel_res"] <= 1e-8
    assert max(ev["field_rel_err"].values()) <= 2e-6
    assert ev["learned"]["cycles"] <= ev["plain"]["cycles"] + 1, ev
