"""Plain FP64 CPU oracle of the regularized-moment FAS solver (Hu & Li, arXiv 2206.13164).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The oracle is plain serial C
(``nrmg_oracle.c``) compiled with gcc; this module builds it and wraps it with ctypes.
It shares no code with the CUDA library.

Readings whose parity with the paper is UNPINNED (the paper prints no formula): the
interior numerical flux (HLL reading), the Maxwell wall flux (half-range reading) and the mass
correction after each NMG step.  Each reading is itself pinned (tests/test_oracle_pins*.py):
the HLL flux by its consistency, upwind limits, conservation, intermediate-state form and
Rusanov special case; the wall flux by velocity-space quadrature; the van Albada slope (the
limiter reading; the paper prints the central slope) by its defining properties; the FAS
defect, restriction, coarse right-hand side and coarse-grid update by exact identities of the
cycle.  tests/test_oracle_mutants.py checks that planted mistakes in these parts fail them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrmg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

OK, ERR_ARG, ERR_NONPHYSICAL, ERR_NOT_CONVERGED = 0, 1, 4, 5
BGK, SHAKHOV, ESBGK = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree bit for bit)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrConfig(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int), ("lx", c_double), ("ly", c_double), ("levels", c_int),
        ("M", c_int), ("Kn", c_double), ("model", c_int), ("Pr", c_double), ("omega", c_double),
        ("beta", c_double), ("order", c_int), ("slope", c_int), ("cfl", c_double),
        ("s1", c_int), ("s2", c_int), ("s3", c_int), ("gamma", c_int),
        ("wall_u", (c_double * 3) * 4), ("wall_theta", c_double * 4), ("wall_chi", c_double * 4),
        ("dtnu", c_double),
        # widths of the finest level's columns [nx] and rows [ny] (NULL: uniform grid); read
        # by or_create only
        ("hx", POINTER(c_double)), ("hy", POINTER(c_double)),
    ]


_lib = None
_dp = POINTER(c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(build()))
    return _lib


def bind(L):
    """Declare the argument and result types of the oracle's C functions on a loaded library."""
    L.or_create.restype = c_void_p
    L.or_create.argtypes = [POINTER(OrConfig)]
    L.or_destroy.argtypes = [c_void_p]
    for name in ("or_level_nx", "or_level_ny"):
        getattr(L, name).restype = c_int
        getattr(L, name).argtypes = [c_void_p, c_int]
    L.or_c_m1.restype = c_double
    L.or_c_m1.argtypes = [c_void_p]
    L.or_nmom.restype = c_int
    L.or_nmom.argtypes = [c_int]
    L.or_alphas.argtypes = [c_int, POINTER(c_int)]
    L.or_hermite_max_root.restype = c_double
    L.or_hermite_max_root.argtypes = [c_int]
    L.or_transform.argtypes = [c_int, _dp, _dp, _dp, _dp]
    L.or_xi_mul.argtypes = [c_int, c_int, _dp, _dp, _dp]
    L.or_macros.argtypes = [c_int, _dp, _dp, _dp]
    L.or_cell_fields.argtypes = [c_int, _dp, _dp, _dp]
    L.or_halfrange.argtypes = [c_int, c_int, _dp]
    L.or_hll_flux.argtypes = [c_int, c_double, c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.or_wall_flux.argtypes = [c_int, _dp, c_double, c_double, c_int, _dp, _dp, _dp, _dp]
    L.or_collision.argtypes = [c_int, c_int, c_double, c_double, c_double, c_double, _dp, _dp, _dp]
    L.or_set_state.argtypes = [c_void_p, c_int, _dp, _dp]
    L.or_get_state.argtypes = [c_void_p, c_int, _dp, _dp]
    L.or_set_rhs.argtypes = [c_void_p, c_int, _dp, _dp]
    L.or_get_rhs.argtypes = [c_void_p, c_int, _dp, _dp]
    L.or_get_saved.argtypes = [c_void_p, c_int, _dp, _dp]
    L.or_mass.restype = c_double
    L.or_mass.argtypes = [c_void_p]
    L.or_res0.restype = c_double
    L.or_res0.argtypes = [c_void_p]
    L.or_sweep.restype = c_int
    L.or_sweep.argtypes = [c_void_p, c_int, c_int]
    L.or_smooth.restype = c_int
    L.or_smooth.argtypes = [c_void_p, c_int, c_int]
    L.or_euler.restype = c_int
    L.or_euler.argtypes = [c_void_p, c_int, c_int]
    L.or_cell_residual.argtypes = [c_void_p, c_int, c_int, c_int, _dp]
    L.or_residual.restype = c_double
    L.or_residual.argtypes = [c_void_p, c_int, _dp]
    L.or_mass_correct.argtypes = [c_void_p]
    L.or_fas_cycle.restype = c_int
    L.or_fas_cycle.argtypes = [c_void_p, _dp]
    L.or_solve.restype = c_int
    L.or_solve.argtypes = [c_void_p, c_double, c_int, POINTER(c_int), _dp]
    L.or_fields.argtypes = [c_void_p, _dp]
    L.or_two_grid_setup.restype = c_int
    L.or_two_grid_setup.argtypes = [c_void_p, c_int]
    L.or_two_grid_update.restype = c_int
    L.or_two_grid_update.argtypes = [c_void_p, c_int]
    L.or_set_threads.argtypes = [c_void_p, c_int]
    L.or_slope.restype = c_double
    L.or_slope.argtypes = [c_int, c_double, c_double, c_double, c_double]
    L.or_face_state.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_int, _dp, _dp]
    return L


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _arr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


# ---------------------------------------------------------------- building blocks
def nmom(M: int) -> int:
    return lib().or_nmom(M)


def alphas(M: int) -> np.ndarray:
    n = nmom(M)
    out = np.zeros(3 * n, dtype=np.int32)
    lib().or_alphas(M, out.ctypes.data_as(POINTER(c_int)))
    return out.reshape(n, 3)


def hermite_max_root(n: int) -> float:
    return lib().or_hermite_max_root(n)


def transform(M, src, dst, f):
    f = _arr(f)
    g = np.zeros_like(f)
    lib().or_transform(M, _p(_arr(src)), _p(_arr(dst)), _p(f), _p(g))
    return g


def xi_mul(M, d, p, f):
    f = _arr(f)
    g = np.zeros_like(f)
    lib().or_xi_mul(M, d, _p(_arr(p)), _p(f), _p(g))
    return g


def macros(M, p, f):
    out = np.zeros(5)
    lib().or_macros(M, _p(_arr(p)), _p(_arr(f)), _p(out))
    return out


def cell_fields(M, p, f):
    out = np.zeros(14)
    lib().or_cell_fields(M, _p(_arr(p)), _p(_arr(f)), _p(out))
    return out


def halfrange(K, s):
    J = np.zeros((K + 1) * (K + 1))
    lib().or_halfrange(K, s, _p(J))
    return J.reshape(K + 1, K + 1)


def hll_flux(M, C, ax, pc, pm, fm, pp, fp):
    F = np.zeros(nmom(M))
    lib().or_hll_flux(M, C, ax, _p(_arr(pc)), _p(_arr(pm)), _p(_arr(fm)), _p(_arr(pp)), _p(_arr(fp)), _p(F))
    return F


def wall_flux(M, uw, thw, chi, w, pc, pf, ff):
    F = np.zeros(nmom(M))
    lib().or_wall_flux(M, _p(_arr(uw)), thw, chi, w, _p(_arr(pc)), _p(_arr(pf)), _p(_arr(ff)), _p(F))
    return F


def slope(kind, qm, q0, qp, h):
    """Slope of one quantity from its values in three consecutive cells of width h along an
    axis (kind 1: central difference; kind 2: van Albada average)."""
    return lib().or_slope(kind, qm, q0, qp, h)


def collision(M, model, Kn, Pr, omega, beta, pc, f):
    Q = np.zeros(nmom(M))
    lib().or_collision(M, model, Kn, Pr, omega, beta, _p(_arr(pc)), _p(_arr(f)), _p(Q))
    return Q


# ---------------------------------------------------------------- solver
class Solver:
    """Multilevel solver state; levels are numbered as in Algorithm 2 (0 = coarsest)."""

    def __init__(self, cfg: OrConfig):
        self.cfg = cfg
        self.L = lib()
        self.h = self.L.or_create(ctypes.byref(cfg))
        if not self.h:
            raise ValueError("oracle: invalid configuration")
        self.n = nmom(cfg.M)
        self.top = cfg.levels - 1

    def __del__(self):
        if getattr(self, "h", None):
            self.L.or_destroy(self.h)
            self.h = None

    def shape(self, level):
        return self.L.or_level_ny(self.h, level), self.L.or_level_nx(self.h, level)

    @property
    def C(self):
        return self.L.or_c_m1(self.h)

    def set_state(self, level, P, F):
        ny, nx = self.shape(level)
        P, F = _arr(P).reshape(ny * nx, 4), _arr(F).reshape(ny * nx, self.n)
        self.L.or_set_state(self.h, level, _p(P), _p(F))

    def get_state(self, level=None):
        level = self.top if level is None else level
        ny, nx = self.shape(level)
        P, F = np.zeros((ny * nx, 4)), np.zeros((ny * nx, self.n))
        self.L.or_get_state(self.h, level, _p(P), _p(F))
        return P, F

    def set_rhs(self, level, rP=None, rF=None):
        if rP is None:
            self.L.or_set_rhs(self.h, level, None, None)
            return
        ny, nx = self.shape(level)
        rP, rF = _arr(rP).reshape(ny * nx, 4), _arr(rF).reshape(ny * nx, self.n)
        self.L.or_set_rhs(self.h, level, _p(rP), _p(rF))

    def get_rhs(self, level):
        ny, nx = self.shape(level)
        P, F = np.zeros((ny * nx, 4)), np.zeros((ny * nx, self.n))
        self.L.or_get_rhs(self.h, level, _p(P), _p(F))
        return P, F

    def get_saved(self, level):
        ny, nx = self.shape(level)
        P, F = np.zeros((ny * nx, 4)), np.zeros((ny * nx, self.n))
        self.L.or_get_saved(self.h, level, _p(P), _p(F))
        return P, F

    def set_threads(self, n):
        """n > 1: OpenMP mode with n threads (the same results bit for bit); 0 or 1: serial."""
        self.L.or_set_threads(self.h, int(n))

    def face_state(self, level, i, j, ax, sd):
        """Reconstructed state of cell (i, j) on its face sd (+1 east/north, -1 west/south) of
        axis ax (0 x, 1 y): params [4] and coefficients [N_M] in the face basis."""
        p, f = np.zeros(4), np.zeros(self.n)
        self.L.or_face_state(self.h, level, i, j, ax, sd, _p(p), _p(f))
        return p, f

    def sweep(self, level, k):
        return self.L.or_sweep(self.h, level, k)

    def smooth(self, level, steps):
        return self.L.or_smooth(self.h, level, steps)

    def euler(self, level, steps):
        """steps forward Euler steps (eq. euler-scheme, global step of eq. global-CFL)."""
        return self.L.or_euler(self.h, level, steps)

    def cell_residual(self, level, i, j):
        R = np.zeros(self.n)
        self.L.or_cell_residual(self.h, level, i, j, _p(R))
        return R

    def residual(self, level=None):
        level = self.top if level is None else level
        ny, nx = self.shape(level)
        R = np.zeros((ny * nx, self.n))
        norm = self.L.or_residual(self.h, level, _p(R))
        return R, norm

    def mass(self):
        return self.L.or_mass(self.h)

    def mass_correct(self):
        self.L.or_mass_correct(self.h)

    def fas_cycle(self):
        rel = c_double(0.0)
        st = self.L.or_fas_cycle(self.h, ctypes.byref(rel))
        return st, rel.value

    def solve(self, tol=1e-8, max_cycles=200):
        cyc, rel = c_int(0), c_double(0.0)
        st = self.L.or_solve(self.h, tol, max_cycles, ctypes.byref(cyc), ctypes.byref(rel))
        return st, cyc.value, rel.value

    def res0(self):
        return self.L.or_res0(self.h)

    def fields(self):
        ny, nx = self.shape(self.top)
        out = np.zeros((ny * nx, 14))
        self.L.or_fields(self.h, _p(out))
        return out.reshape(ny, nx, 14)

    def two_grid_setup(self, lf):
        return self.L.or_two_grid_setup(self.h, lf)

    def two_grid_update(self, lf):
        return self.L.or_two_grid_update(self.h, lf)
