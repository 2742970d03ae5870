"""Parity of the exact-wavefront scheduler with the CPU oracle at full size, in the launch
configuration the benchmark times (the 256x256, M = 10, second-order van Albada level of the
lid-driven cavity, two FS steps in one persistent launch at 2 CTAs per SM, as in each
smoothing call of its V-cycle), and one whole V-cycle of the same cavity on 128x128 (five
levels).  The oracle takes about a minute for the two together on one host core."""
import numpy as np
import pytest
import torch

from conftest import oracle_solver
from inputs import config_c2, lid_cavity, random_state
from paper_2206_13164_gb300 import nrmg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("grid", [2])
def test_fs_steps_at_full_size_match_the_oracle(grid):
    """FS^2 on the finest level of the 256x256 M = 10 cavity: every cell of all eight sweeps in
    the serial order of Algorithm 1, while the persistent CTAs overlap sweeps and steps."""
    torch.cuda.set_device(0)
    prob = config_c2()
    top = prob.levels - 1
    rng = np.random.default_rng(200)
    P, F = random_state(rng, prob.ny, prob.nx, prob.M, amp=0.03)
    G = nrmg.from_problem(prob, device=DEV)
    G.set_grid(grid)
    G.set_state(_T(P), _T(F))
    G.smooth(top, 2)
    Pg, Fg = (t.cpu().numpy() for t in G.get_state())
    del G
    O = oracle_solver(prob)
    O.set_state(top, P, F)
    assert O.smooth(top, 2) == 0
    Po, Fo = O.get_state(top)
    assert _rel(Pg, Po) <= 1e-12 and _rel(Fg, Fo) <= 1e-12, (_rel(Pg, Po), _rel(Fg, Fo))


def test_v_cycle_at_128_matches_the_oracle():
    """One FAS V-cycle (five levels, 128x128 to 8x8) of the M = 10 van Albada lid cavity at
    the benchmark's grid of 2 CTAs per SM: state and relative residual."""
    torch.cuda.set_device(0)
    prob = lid_cavity(128, 10, 0.01, 0.5, order=2, slope=2, levels=5)
    top = prob.levels - 1
    rng = np.random.default_rng(201)
    P, F = random_state(rng, prob.ny, prob.nx, prob.M, amp=0.03)
    G = nrmg.from_problem(prob, device=DEV)
    G.set_grid(2)
    G.set_state(_T(P), _T(F))
    rg = G.fas_cycle()
    Pg, Fg = (t.cpu().numpy() for t in G.get_state())
    del G
    O = oracle_solver(prob)
    O.set_state(top, P, F)
    st, ro = O.fas_cycle()
    assert st == 0
    Po, Fo = O.get_state(top)
    assert _rel(Pg, Po) <= 1e-11 and _rel(Fg, Fo) <= 1e-11, (_rel(Pg, Po), _rel(Fg, Fo))
    assert abs(rg - ro) <= 1e-10 * ro
