import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def oracle_config(prob):
    """Problem -> oracle configuration struct."""
    import oracle

    c = oracle.OrConfig()
    c.nx, c.ny, c.lx, c.ly, c.levels = prob.nx, prob.ny, prob.lx, prob.ly, prob.levels
    c.M, c.Kn, c.model, c.Pr, c.omega, c.beta = prob.M, prob.Kn, prob.model, prob.Pr, prob.omega, prob.beta
    c.order, c.slope, c.cfl = prob.order, prob.slope, prob.cfl
    c.s1, c.s2, c.s3, c.gamma = prob.s1, prob.s2, prob.s3, prob.gamma
    c.dtnu = prob.dtnu
    if getattr(prob, "hx", None) is not None:
        import ctypes

        import numpy as np

        c._hx = np.ascontiguousarray(prob.hx, dtype=np.float64)  # kept alive with the struct
        c._hy = np.ascontiguousarray(prob.hy, dtype=np.float64)
        c.hx = c._hx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.hy = c._hy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for w in range(4):
        for d in range(3):
            c.wall_u[w][d] = prob.walls[w].u[d]
        c.wall_theta[w] = prob.walls[w].theta
        c.wall_chi[w] = prob.walls[w].chi
    return c


def oracle_solver(prob):
    import oracle

    return oracle.Solver(oracle_config(prob))
