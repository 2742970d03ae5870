"""Seeded synthetic inputs shared by the oracle tests and the CUDA parity tests.

This module holds no arithmetic of the method: it only describes cavity problems
(geometry, walls, gas, scheme options) and draws random but admissible states
(Grad form: f_0 = rho, f_{e_d} = 0, sum_d f_{2e_d} = 0, u_3 = 0 and zero
coefficients of odd alpha_3, the symmetry of a flow with d/dx_3 = 0).

Coefficient layout (the interface of both sides): multi-indices |alpha| <= M in graded
order -- |alpha| ascending, then alpha_1 descending, then alpha_2 descending.
Walls: 0 bottom (y=0), 1 right (x=lx), 2 top (y=ly), 3 left (x=0).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

BGK, SHAKHOV, ESBGK = 0, 1, 2


def multi_indices(M: int) -> np.ndarray:
    out = []
    for deg in range(M + 1):
        for a1 in range(deg, -1, -1):
            for a2 in range(deg - a1, -1, -1):
                out.append((a1, a2, deg - a1 - a2))
    return np.array(out, dtype=np.int64)


def nmom(M: int) -> int:
    return (M + 1) * (M + 2) * (M + 3) // 6


@dataclass
class Wall:
    u: tuple = (0.0, 0.0, 0.0)
    theta: float = 1.0
    chi: float = 1.0


@dataclass
class Problem:
    nx: int
    ny: int
    M: int
    Kn: float
    walls: list
    levels: int = 1
    lx: float = 1.0
    ly: float = 1.0
    model: int = BGK
    Pr: float = 2.0 / 3.0
    omega: float = 0.81
    beta: float = 1.0
    order: int = 1
    slope: int = 0
    cfl: float = 0.9
    s1: int = 2
    s2: int = 2
    s3: int = 4
    gamma: int = 1
    dtnu: float = 0.0  # > 0: local time step capped at dtnu / nu
    hx: tuple = None   # widths of the finest level's columns (None: uniform lx / nx)
    hy: tuple = None   # widths of the finest level's rows (None: uniform ly / ny)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def level_shape(self, level: int):
        sh = self.levels - 1 - level
        return self.ny >> sh, self.nx >> sh


def lid_cavity(N, M, Kn, U, order=1, slope=0, levels=1, model=BGK, Pr=2.0 / 3.0, **kw) -> Problem:
    walls = [Wall(), Wall(), Wall(u=(U, 0.0, 0.0)), Wall()]
    return Problem(nx=N, ny=N, M=M, Kn=Kn, walls=walls, levels=levels, order=order, slope=slope,
                   model=model, Pr=Pr, **kw)


def heated_cavity(N, M, Kn, theta_bottom=2.0, order=1, slope=0, levels=1, model=SHAKHOV, Pr=2.0 / 3.0, **kw):
    walls = [Wall(theta=theta_bottom), Wall(), Wall(), Wall()]
    return Problem(nx=N, ny=N, M=M, Kn=Kn, walls=walls, levels=levels, order=order, slope=slope,
                   model=model, Pr=Pr, **kw)


def levels_to_8(N: int) -> int:
    """Number of levels whose coarsest grid is 8x8 (the paper's choice)."""
    L, n = 1, N
    while n > 8:
        n //= 2
        L += 1
    return L


# the three single-instance cavity workloads, at full size
def config_c1() -> Problem:
    return lid_cavity(32, 5, 0.1, 0.1, order=1, levels=3)


def config_c2() -> Problem:
    return lid_cavity(256, 10, 0.01, 0.5, order=2, slope=2, levels=6)


def config_c3() -> Problem:
    return heated_cavity(512, 8, 0.05, theta_bottom=2.0, order=2, slope=2, levels=7, model=SHAKHOV)


def stretched_widths(n, length=1.0, ratio=1.5, pairs=True):
    """Cell widths of a grid refined towards both walls: a geometric progression of `ratio`
    between the wall cells and the middle ones, scaled to sum to `length`.  With pairs, the
    widths come in equal pairs (2k, 2k + 1) on the finest level, so every coarser level of the
    multigrid hierarchy is stretched the same way."""
    import numpy as np

    half = n // 2
    g = ratio ** (1.0 / max(half - 1, 1))
    w = np.array([g ** min(k, n - 1 - k) for k in range(n)], dtype=np.float64)
    if pairs:
        w = np.repeat(w.reshape(-1, 2).mean(1), 2) if n % 2 == 0 else w
    w *= length / w.sum()
    w[-1] = length - w[:-1].sum()
    return tuple(float(x) for x in w)


def maxwellian_state(ny, nx, M, rho=1.0, theta=1.0):
    n = nmom(M)
    P = np.zeros((ny * nx, 4))
    P[:, 3] = theta
    F = np.zeros((ny * nx, n))
    F[:, 0] = rho
    return P, F


def random_state(rng: np.random.Generator, ny: int, nx: int, M: int, amp: float = 0.05,
                 u: float = 0.2, rho=(0.8, 1.2), theta=(0.8, 1.25), decay: float = 0.5):
    """Admissible random cell states: params [cells,4] and coefficients [cells,N_M]."""
    al = multi_indices(M)
    deg = al.sum(1)
    nc = ny * nx
    P = np.zeros((nc, 4))
    P[:, 0] = rng.uniform(-u, u, nc)
    P[:, 1] = rng.uniform(-u, u, nc)
    P[:, 3] = rng.uniform(theta[0], theta[1], nc)
    r = rng.uniform(rho[0], rho[1], nc)
    F = rng.standard_normal((nc, len(al))) * amp * (decay ** np.maximum(deg - 2, 0))[None, :] * r[:, None]
    F[:, deg == 0] = r[:, None]
    F[:, deg == 1] = 0.0
    F[:, al[:, 2] % 2 == 1] = 0.0
    two = [int(np.where((al == e).all(1))[0][0]) for e in ([2, 0, 0], [0, 2, 0], [0, 0, 2])]
    F[:, two] -= F[:, two].mean(1, keepdims=True)
    return P, F


def random_rhs(rng: np.random.Generator, ny: int, nx: int, M: int, amp: float = 0.05):
    """Random right-hand side r with its own expansion bases (odd alpha_3 zero)."""
    al = multi_indices(M)
    deg = al.sum(1)
    nc = ny * nx
    P = np.zeros((nc, 4))
    P[:, 0] = rng.uniform(-0.2, 0.2, nc)
    P[:, 1] = rng.uniform(-0.2, 0.2, nc)
    P[:, 3] = rng.uniform(0.8, 1.25, nc)
    F = rng.standard_normal((nc, len(al))) * amp * (0.5 ** deg)[None, :]
    F[:, al[:, 2] % 2 == 1] = 0.0
    return P, F
