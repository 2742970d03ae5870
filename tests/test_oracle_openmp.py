"""The oracle's OpenMP mode (used to time the CPU baseline on all host cores) gives the serial
oracle's results bit for bit: sweeps by anti-diagonals of the serial visiting order, residual,
restriction and coarse-grid update in parallel over cells (no GPU)."""
import numpy as np
import pytest

import oracle
from conftest import oracle_solver
from inputs import ESBGK, heated_cavity, lid_cavity, random_rhs, random_state


@pytest.mark.parametrize("prob", [
    heated_cavity(16, 4, 0.05, order=2, slope=2, levels=2),
    lid_cavity(12, 3, 0.1, 0.3, order=1).replace(ny=20),
    lid_cavity(16, 3, 0.1, 0.3, order=2, slope=1, levels=2, model=ESBGK, beta=2 / 3),
], ids=["heated_o2va", "lid_o1_ragged", "esbgk_o2central"])
def test_openmp_mode_is_bit_identical_to_serial(prob):
    rng = np.random.default_rng(60)
    top = prob.levels - 1
    P, F = random_state(rng, prob.ny, prob.nx, prob.M, amp=0.1)
    rP, rF = random_rhs(rng, prob.ny, prob.nx, prob.M)
    out = []
    for threads in (0, 4):
        S = oracle_solver(prob)
        S.set_threads(threads)
        S.set_state(top, P, F)
        S.set_rhs(top, rP, rF)
        for k in (1, 2, 3, 4):
            assert S.sweep(top, k) == oracle.OK
        R, norm = S.residual(top)
        S.set_rhs(top, None)
        cyc = [S.fas_cycle() for _ in range(2)]
        out.append((S.get_state(top), R, norm, cyc))
    (s0, R0, n0, c0), (s1, R1, n1, c1) = out
    assert np.array_equal(s0[0], s1[0]) and np.array_equal(s0[1], s1[1])
    assert np.array_equal(R0, R1) and n0 == n1 and c0 == c1
