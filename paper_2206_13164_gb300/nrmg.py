"""Thin Python binding of the C ABI in ``include/nrmg.h`` (argument marshalling only).

Every step of the solver runs in the CUDA kernels of ``libnrmg.so``; PyTorch provides the
device memory (the workspace and the state/result tensors) and the stream.  There is no
fallback: if the library is missing or CUDA is unavailable, construction raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_size_t, c_void_p

import torch

from . import build as _build

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NONPHYSICAL, ERR_NOT_CONVERGED, ERR_TIMEOUT = range(7)
BGK, SHAKHOV, ESBGK = 0, 1, 2


class NrmgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_status_name(status)} {detail}".strip())


class Grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("lx", c_double), ("ly", c_double), ("levels", c_int)]


class Wall(ctypes.Structure):
    _fields_ = [("u", c_double * 3), ("theta", c_double), ("chi", c_double)]


class Collision(ctypes.Structure):
    _fields_ = [("model", c_int), ("Pr", c_double), ("omega", c_double), ("beta", c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("order", c_int), ("slope", c_int), ("cfl", c_double), ("s1", c_int), ("s2", c_int),
                ("s3", c_int), ("gamma", c_int), ("precision", c_int), ("dtnu", c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libnrmg.so (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libnrmg.so missing at {path}")
        L = ctypes.CDLL(path)
        L.nrmg_workspace_bytes.restype = c_size_t
        L.nrmg_workspace_bytes.argtypes = [POINTER(Grid), c_int, POINTER(Opts)]
        L.nrmg_create.restype = c_int
        L.nrmg_create.argtypes = [POINTER(Grid), c_int, c_double, POINTER(Wall), POINTER(Collision), POINTER(Opts),
                                  c_void_p, c_size_t, c_void_p, POINTER(c_void_p)]
        L.nrmg_destroy.restype = c_int
        L.nrmg_destroy.argtypes = [c_void_p]
        for name in ("nrmg_set_state", "nrmg_get_state", "nrmg_set_rhs"):
            getattr(L, name).restype = c_int
            getattr(L, name).argtypes = [c_void_p, c_int, c_void_p, c_void_p]
        L.nrmg_smooth.restype = c_int
        L.nrmg_smooth.argtypes = [c_void_p, c_int, c_int]
        L.nrmg_residual.restype = c_int
        L.nrmg_residual.argtypes = [c_void_p, c_int, c_void_p, POINTER(c_double)]
        L.nrmg_fas_cycle.restype = c_int
        L.nrmg_fas_cycle.argtypes = [c_void_p, POINTER(c_double)]
        L.nrmg_solve.restype = c_int
        L.nrmg_solve.argtypes = [c_void_p, c_double, c_int, POINTER(c_int), POINTER(c_double)]
        L.nrmg_fields.restype = c_int
        L.nrmg_fields.argtypes = [c_void_p, c_void_p]
        L.nrmg_two_grid_setup.restype = c_int
        L.nrmg_two_grid_setup.argtypes = [c_void_p, c_int]
        L.nrmg_two_grid_update.restype = c_int
        L.nrmg_two_grid_update.argtypes = [c_void_p, c_int]
        L.nrmg_mass_correct.restype = c_int
        L.nrmg_mass_correct.argtypes = [c_void_p]
        L.nrmg_set_grid.restype = c_int
        L.nrmg_set_grid.argtypes = [c_void_p, c_int]
        L.nrmg_grid_limit.restype = c_int
        L.nrmg_grid_limit.argtypes = [c_void_p]
        L.nrmg_set_spacing.restype = c_int
        L.nrmg_set_spacing.argtypes = [c_void_p, c_void_p, c_void_p]
        L.nrmg_set_cluster.restype = c_int
        L.nrmg_set_cluster.argtypes = [c_void_p, c_int]
        L.nrmg_cluster_capacity.restype = c_int
        L.nrmg_cluster_capacity.argtypes = [c_void_p]
        L.nrmg_mixed_fallback.restype = c_int
        L.nrmg_mixed_fallback.argtypes = [c_void_p]
        L.nrmg_euler.restype = c_int
        L.nrmg_euler.argtypes = [c_void_p, c_int, c_int]
        L.nrmg_euler_solve.restype = c_int
        L.nrmg_euler_solve.argtypes = [c_void_p, c_double, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]
        L.nrmg_set_reference.restype = c_int
        L.nrmg_set_reference.argtypes = [c_void_p, c_double, c_double]
        L.nrmg_set_state_from_fields.restype = c_int
        L.nrmg_set_state_from_fields.argtypes = [c_void_p, c_void_p]
        L.nrmg_debug_stalled_sweep.restype = c_int
        L.nrmg_debug_stalled_sweep.argtypes = [c_void_p, c_int]
        L.nrmg_sync.restype = c_int
        L.nrmg_sync.argtypes = [c_void_p]
        L.nrmg_launch_count.restype = c_longlong
        L.nrmg_launch_count.argtypes = [c_void_p]
        L.nrmg_set_profiling.restype = c_int
        L.nrmg_set_profiling.argtypes = [c_void_p, c_int]
        L.nrmg_fs_profile.restype = c_int
        L.nrmg_fs_profile.argtypes = [c_void_p, POINTER(c_double), POINTER(c_longlong), POINTER(c_longlong),
                                      POINTER(c_longlong)]
        L.nrmg_residual_profile.restype = c_int
        L.nrmg_residual_profile.argtypes = [c_void_p, POINTER(c_double), POINTER(c_longlong), POINTER(c_longlong),
                                            POINTER(c_longlong)]
        for name in ("nrmg_set_state_host", "nrmg_get_state_host"):
            getattr(L, name).restype = c_int
            getattr(L, name).argtypes = [c_void_p, c_int, c_void_p, c_void_p]
        L.nrmg_fs_profile_levels.restype = c_int
        L.nrmg_fs_profile_levels.argtypes = [c_void_p, POINTER(c_double), POINTER(c_longlong)]
        L.nrmg_peak_fma.restype = c_int
        L.nrmg_peak_fma.argtypes = [c_int, c_int, c_void_p, POINTER(c_double)]
        L.nrmg_batch_workspace_bytes.restype = c_size_t
        L.nrmg_batch_workspace_bytes.argtypes = [POINTER(c_void_p), c_int]
        L.nrmg_batch_create.restype = c_int
        L.nrmg_batch_create.argtypes = [POINTER(c_void_p), c_int, c_void_p, c_size_t, POINTER(c_void_p)]
        L.nrmg_batch_destroy.restype = c_int
        L.nrmg_batch_destroy.argtypes = [c_void_p]
        L.nrmg_batch_fas_cycle.restype = c_int
        L.nrmg_batch_fas_cycle.argtypes = [c_void_p, POINTER(c_double)]
        L.nrmg_batch_solve.restype = c_int
        L.nrmg_batch_solve.argtypes = [c_void_p, c_double, c_int, POINTER(c_int), POINTER(c_double)]
        L.nrmg_batch_graph.restype = c_int
        L.nrmg_batch_graph.argtypes = [c_void_p]
        L.nrmg_batch_set_grid.restype = c_int
        L.nrmg_batch_set_grid.argtypes = [c_void_p, c_int]
        L.nrmg_batch_launch_count.restype = c_longlong
        L.nrmg_batch_launch_count.argtypes = [c_void_p]
        L.nrmg_status_str.restype = ctypes.c_char_p
        L.nrmg_status_str.argtypes = [c_int]
        L.nrmg_last_error.restype = ctypes.c_char_p
        L.nrmg_last_error.argtypes = [c_void_p]
        _lib = L
    return _lib


def _status_name(s: int) -> str:
    try:
        return lib().nrmg_status_str(s).decode()
    except Exception:  # pragma: no cover - only while reporting another failure
        return str(s)


def nmom(M: int) -> int:
    return (M + 1) * (M + 2) * (M + 3) // 6


def _host_ptr(t, cols):
    """Address of a host float64 array with `cols` columns (torch CPU tensor or numpy)."""
    if isinstance(t, torch.Tensor):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.shape[-1] != cols:
            raise ValueError(f"expected a contiguous float64 host tensor with {cols} columns")
        return c_void_p(t.data_ptr())
    import numpy as np

    if t.dtype != np.float64 or not t.flags["C_CONTIGUOUS"] or t.shape[-1] != cols:
        raise ValueError(f"expected a contiguous float64 host array with {cols} columns")
    return c_void_p(t.ctypes.data)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return c_void_p(t.data_ptr())


# ---------------------------------------------------------------- autotune cache
TUNE_CACHE = os.path.join(os.path.dirname(_build.LIB), "autotune.json")


def _tune_load(path):
    import json

    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _tune_store(path, key, best, times):
    """Record a tuning result (atomic replace, so concurrent writers never leave a torn file)."""
    import json

    data = _tune_load(path)
    data[key] = {"ctas_per_sm": int(best), "s_per_cycle": {str(k): v for k, v in times.items()}}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _device_tag(device):
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}/{p.multi_processor_count}sm"


def tune_key(device, shapes, opts, model):
    """Cache key of a sweep-grid tuning: the GPU, the (nx, ny, M, levels) of every problem
    (sorted), the scheme (order, slope) and precision, and the collision model."""
    sh = ";".join(f"{nx}x{ny}:M{M}:L{lv}" for nx, ny, M, lv in sorted(shapes))
    return f"{_device_tag(device)}|{sh}|order{opts.order}:slope{opts.slope}:prec{opts.precision}|model{model}"


# levels of at most this many cells sweep on two-CTA clusters unless set_cluster says otherwise
CLUSTER_CELLS_DEFAULT = 128 * 128


class Solver:
    """One cavity problem on the current CUDA device.

    walls: four (u, theta, chi) triples in the order bottom, right, top, left.
    Levels follow Algorithm 2: level 0 is the coarsest, ``levels-1`` the finest.
    """

    def __init__(self, nx, ny, M, Kn, walls, levels=1, lx=1.0, ly=1.0, model=BGK, Pr=2.0 / 3.0, omega=0.81,
                 beta=1.0, order=1, slope=0, cfl=0.9, s1=2, s2=2, s3=4, gamma=1, precision=0, dtnu=0.0,
                 device=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("nrmg needs a CUDA device")
        self.L = lib()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.M, self.N, self.levels = M, nmom(M), levels
        self.nx, self.ny = nx, ny
        self.grid = Grid(nx, ny, lx, ly, levels)
        self.opts = Opts(order, slope, cfl, s1, s2, s3, gamma, precision, dtnu)
        self.coll = Collision(model, Pr, omega, beta)
        wa = (Wall * 4)()
        for k, (u, th, chi) in enumerate(walls):
            wa[k].u = (c_double * 3)(*u)
            wa[k].theta = th
            wa[k].chi = chi
        self.walls = wa
        nbytes = self.L.nrmg_workspace_bytes(ctypes.byref(self.grid), M, ctypes.byref(self.opts))
        if nbytes == 0:
            raise NrmgError(ERR_ARG, "nrmg_workspace_bytes")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = c_void_p()
        st = self.L.nrmg_create(ctypes.byref(self.grid), M, Kn, wa, ctypes.byref(self.coll), ctypes.byref(self.opts),
                                c_void_p(self.workspace.data_ptr()), nbytes, c_void_p(self.stream.cuda_stream),
                                ctypes.byref(self.ctx))
        if st != OK:
            raise NrmgError(st, "nrmg_create")
        self.cluster_cells = CLUSTER_CELLS_DEFAULT  # the library's default (nrmg_set_cluster)
        self.cluster_times = {}

    # -- helpers
    def _check(self, st, where):
        if st != OK:
            raise NrmgError(st, where, self.L.nrmg_last_error(self.ctx).decode())

    def level_shape(self, level):
        sh = self.levels - 1 - level
        return self.ny >> sh, self.nx >> sh

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.L.nrmg_destroy(self.ctx)
            self.ctx = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state
    def set_state(self, params, coeffs, level=None):
        level = self.levels - 1 if level is None else level
        self._check(self.L.nrmg_set_state(self.ctx, level, _ptr(params), _ptr(coeffs)), "nrmg_set_state")

    def get_state(self, level=None):
        level = self.levels - 1 if level is None else level
        ny, nx = self.level_shape(level)
        P = torch.empty((ny * nx, 4), dtype=torch.float64, device=self.device)
        F = torch.empty((ny * nx, self.N), dtype=torch.float64, device=self.device)
        self._check(self.L.nrmg_get_state(self.ctx, level, _ptr(P), _ptr(F)), "nrmg_get_state")
        return P, F

    def set_state_host(self, params, coeffs, level=None):
        """State from host arrays (float64, contiguous, [cells,4] and [cells,N_M]; pinned
        memory gives asynchronous copies)."""
        level = self.levels - 1 if level is None else level
        self._check(self.L.nrmg_set_state_host(self.ctx, level, _host_ptr(params, 4), _host_ptr(coeffs, self.N)),
                    "nrmg_set_state_host")

    def get_state_host(self, params, coeffs, level=None):
        """Copy the state into host arrays (float64, contiguous); synchronizes."""
        level = self.levels - 1 if level is None else level
        self._check(self.L.nrmg_get_state_host(self.ctx, level, _host_ptr(params, 4), _host_ptr(coeffs, self.N)),
                    "nrmg_get_state_host")

    def set_rhs(self, level, rparams=None, rcoeffs=None):
        self._check(self.L.nrmg_set_rhs(self.ctx, level, _ptr(rparams), _ptr(rcoeffs)), "nrmg_set_rhs")

    # -- solver
    def smooth(self, level, steps):
        self._check(self.L.nrmg_smooth(self.ctx, level, steps), "nrmg_smooth")

    def residual(self, level=None, want_R=True):
        level = self.levels - 1 if level is None else level
        ny, nx = self.level_shape(level)
        R = torch.empty((ny * nx, self.N), dtype=torch.float64, device=self.device) if want_R else None
        norm = c_double(0.0)
        self._check(self.L.nrmg_residual(self.ctx, level, _ptr(R), ctypes.byref(norm)), "nrmg_residual")
        return R, norm.value

    def fas_cycle(self):
        rel = c_double(0.0)
        self._check(self.L.nrmg_fas_cycle(self.ctx, ctypes.byref(rel)), "nrmg_fas_cycle")
        return rel.value

    def solve(self, tol=1e-8, max_cycles=200, raise_on_fail=True):
        cyc, rel = c_int(0), c_double(0.0)
        st = self.L.nrmg_solve(self.ctx, tol, max_cycles, ctypes.byref(cyc), ctypes.byref(rel))
        if raise_on_fail and st not in (OK, ERR_NOT_CONVERGED):
            self._check(st, "nrmg_solve")
        return st, cyc.value, rel.value

    def euler(self, steps, level=None):
        """``steps`` forward Euler steps (eq. euler-scheme) on a level (default: the finest)."""
        level = self.levels - 1 if level is None else level
        self._check(self.L.nrmg_euler(self.ctx, level, steps), "nrmg_euler")

    def euler_solve(self, tol=1e-8, max_steps=100000, raise_on_fail=True):
        """Forward Euler on the finest level to relative residual tol: (status, steps, rel)."""
        n, rel = c_int(0), c_double(0.0)
        st = self.L.nrmg_euler_solve(self.ctx, tol, max_steps, ctypes.byref(n), ctypes.byref(rel))
        if raise_on_fail and st not in (OK, ERR_NOT_CONVERGED):
            self._check(st, "nrmg_euler_solve")
        return st, n.value, rel.value

    def mixed_fallback(self) -> bool:
        """True when the last solve of a mixed-precision solver stalled and finished with FP64
        smoothing (``nrmg_mixed_fallback``)."""
        return bool(self.L.nrmg_mixed_fallback(self.ctx))

    def fields(self):
        out = torch.empty((self.ny * self.nx, 14), dtype=torch.float64, device=self.device)
        self._check(self.L.nrmg_fields(self.ctx, _ptr(out)), "nrmg_fields")
        return out.view(self.ny, self.nx, 14)

    def two_grid_setup(self, lf):
        self._check(self.L.nrmg_two_grid_setup(self.ctx, lf), "nrmg_two_grid_setup")

    def two_grid_update(self, lf):
        self._check(self.L.nrmg_two_grid_update(self.ctx, lf), "nrmg_two_grid_update")

    def mass_correct(self):
        self._check(self.L.nrmg_mass_correct(self.ctx), "nrmg_mass_correct")

    def set_grid(self, ctas_per_sm: int):
        """Persistent CTAs per SM of the sweep launches (0: the kernel occupancy)."""
        self._check(self.L.nrmg_set_grid(self.ctx, ctas_per_sm), "nrmg_set_grid")
        self.tuned = ctas_per_sm

    def set_spacing(self, hx, hy):
        """Non-uniform grid: widths of the finest level's columns (nx) and rows (ny), adding up
        to lx and ly.  Resets every level to the global Maxwellian."""
        import numpy as np

        ax = np.ascontiguousarray(hx, dtype=np.float64)
        ay = np.ascontiguousarray(hy, dtype=np.float64)
        if ax.shape != (self.nx,) or ay.shape != (self.ny,):
            raise ValueError(f"expected {self.nx} column widths and {self.ny} row heights")
        self._check(self.L.nrmg_set_spacing(self.ctx, c_void_p(ax.ctypes.data), c_void_p(ay.ctypes.data)),
                    "nrmg_set_spacing")

    def set_cluster(self, max_cells: int):
        """FP64 sweeps of levels with at most max_cells cells split each cell update over a
        cluster of two CTAs (0: never)."""
        self._check(self.L.nrmg_set_cluster(self.ctx, int(max_cells)), "nrmg_set_cluster")
        self.cluster_cells = int(max_cells)

    @property
    def cluster_capacity(self) -> int:
        return int(self.L.nrmg_cluster_capacity(self.ctx))

    def tune_key(self):
        return tune_key(self.device, [(self.nx, self.ny, self.M, self.levels)], self.opts, self.coll.model)

    def autotune(self, candidates=None, reps=1, cache=None, clusters=()):
        """Time `reps` FAS cycles per candidate CTAs/SM of the sweep launches (the cycles advance
        the solution, not its fixed point) and keep the fastest.  Returns {candidate: s/cycle}.
        clusters: candidate level sizes (cells) up to which the FP64 sweeps use two-CTA
        clusters, timed after the grid (results in self.cluster_times).
        cache: a JSON file path (True: TUNE_CACHE) keyed by tune_key(); a cached entry is used
        without timing (the returned dict is then the cached timings), a new result is stored."""
        import time

        path = TUNE_CACHE if cache is True else cache
        if path:
            hit = _tune_load(path).get(self.tune_key())
            if hit:
                self.set_grid(hit["ctas_per_sm"])
                return {int(k): v for k, v in hit["s_per_cycle"].items()}
        limit = int(self.L.nrmg_grid_limit(self.ctx))
        cands = [c for c in (candidates or range(1, limit + 1)) if 1 <= c <= limit]
        times = {}
        self.cluster_times = {}
        for c in cands:
            self.set_grid(c)
            torch.cuda.synchronize(self.device)
            t0 = time.perf_counter()
            for _ in range(reps):
                self.fas_cycle()
            torch.cuda.synchronize(self.device)
            times[c] = (time.perf_counter() - t0) / reps
        best = min(times, key=times.get)
        self.set_grid(best)
        if clusters and self.cluster_capacity > 0:
            # then the largest level size whose sweeps run on two-CTA clusters
            for cells in clusters:
                self.set_cluster(cells)
                torch.cuda.synchronize(self.device)
                t0 = time.perf_counter()
                for _ in range(reps):
                    self.fas_cycle()
                torch.cuda.synchronize(self.device)
                self.cluster_times[cells] = (time.perf_counter() - t0) / reps
            self.set_cluster(min(self.cluster_times, key=self.cluster_times.get))
        if path:
            _tune_store(path, self.tune_key(), best, times)
        return times

    def set_reference(self, mass=0.0, res0=0.0):
        """Fix the reference mass of the correction and the residual norm that relative
        residuals divide by (0 keeps the current value)."""
        self._check(self.L.nrmg_set_reference(self.ctx, mass, res0), "nrmg_set_reference")

    def set_state_from_fields(self, fields):
        """Finest level := the 13-moment Grad state of fields ([cells, 14] float64 CUDA)."""
        f = fields.reshape(self.ny * self.nx, 14)
        self._check(self.L.nrmg_set_state_from_fields(self.ctx, _ptr(f)), "nrmg_set_state_from_fields")

    def debug_stalled_sweep(self, level=None) -> int:
        """Status of an FS launch whose dependency waits can never be satisfied (expected:
        ERR_TIMEOUT after the scheduler's time limit)."""
        level = self.levels - 1 if level is None else level
        return int(self.L.nrmg_debug_stalled_sweep(self.ctx, level))

    def sync(self):
        self._check(self.L.nrmg_sync(self.ctx), "nrmg_sync")

    @property
    def launches(self) -> int:
        return int(self.L.nrmg_launch_count(self.ctx))

    def set_profiling(self, on: bool):
        self._check(self.L.nrmg_set_profiling(self.ctx, 1 if on else 0), "nrmg_set_profiling")

    def fs_profile_levels(self):
        """Per level: (ms, cell updates) of the timed FS launches (does not reset the record)."""
        ms = (c_double * self.levels)()
        up = (c_longlong * self.levels)()
        self._check(self.L.nrmg_fs_profile_levels(self.ctx, ms, up), "nrmg_fs_profile_levels")
        return [(ms[l], up[l]) for l in range(self.levels)]

    def residual_profile(self):
        """(ms, launches, cells without r, cells with r) of the timed residual launches."""
        ms, n, c0, c1 = c_double(0.0), c_longlong(0), c_longlong(0), c_longlong(0)
        self._check(self.L.nrmg_residual_profile(self.ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(c0),
                                                 ctypes.byref(c1)), "nrmg_residual_profile")
        return ms.value, n.value, c0.value, c1.value

    def fs_profile(self):
        """(ms, launches, cell updates without r, cell updates with r) of the timed FS launches."""
        ms, n, u0, u1 = c_double(0.0), c_longlong(0), c_longlong(0), c_longlong(0)
        self._check(self.L.nrmg_fs_profile(self.ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(u0),
                                           ctypes.byref(u1)), "nrmg_fs_profile")
        return ms.value, n.value, u0.value, u1.value


def peak_fma(precision: int = 0, iters: int = 4096, stream=None) -> float:
    """Measured FMA rate (FLOP/s) of the current device: precision 0 FP64, 1 FP32."""
    out = c_double(0.0)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib().nrmg_peak_fma(precision, iters, c_void_p(s.cuda_stream), ctypes.byref(out))
    if st != 0:
        raise RuntimeError(f"nrmg_peak_fma failed ({st})")
    return out.value


class Batch:
    """Several Solvers (same scheme; grids, M, Kn, walls may differ) cycled in lockstep with
    one persistent FS launch per stage.  All work runs on the first solver's stream."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.L = lib()
        n = len(self.solvers)
        self._arr = (c_void_p * n)(*[s.ctx.value for s in self.solvers])
        nbytes = self.L.nrmg_batch_workspace_bytes(self._arr, n)
        if nbytes == 0:
            raise NrmgError(ERR_ARG, "nrmg_batch_workspace_bytes", "incompatible solvers")
        dev = self.solvers[0].device
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.h = c_void_p()
        st = self.L.nrmg_batch_create(self._arr, n, c_void_p(self.workspace.data_ptr()), nbytes, ctypes.byref(self.h))
        if st != OK:
            raise NrmgError(st, "nrmg_batch_create")

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.nrmg_batch_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fas_cycle(self):
        n = len(self.solvers)
        rel = (c_double * n)()
        st = self.L.nrmg_batch_fas_cycle(self.h, rel)
        if st != OK:
            raise NrmgError(st, "nrmg_batch_fas_cycle", self.L.nrmg_last_error(self.solvers[0].ctx).decode())
        return list(rel)

    def solve(self, tol=1e-8, max_cycles=200):
        n = len(self.solvers)
        cyc, rel = (c_int * n)(), (c_double * n)()
        st = self.L.nrmg_batch_solve(self.h, tol, max_cycles, cyc, rel)
        if st not in (OK, ERR_NOT_CONVERGED):
            raise NrmgError(st, "nrmg_batch_solve")
        return st, list(cyc), list(rel)

    @property
    def launches(self) -> int:
        return int(self.L.nrmg_batch_launch_count(self.h))

    @property
    def graph(self) -> bool:
        """True when the batched cycle replays a captured CUDA graph."""
        return bool(self.L.nrmg_batch_graph(self.h))

    def set_grid(self, ctas_per_sm: int):
        st = self.L.nrmg_batch_set_grid(self.h, ctas_per_sm)
        if st != OK:
            raise NrmgError(st, "nrmg_batch_set_grid")

    def tune_key(self):
        s0 = self.solvers[0]
        return tune_key(s0.device, [(s.nx, s.ny, s.M, s.levels) for s in self.solvers], s0.opts, s0.coll.model)

    def autotune(self, candidates=(1, 2, 3), reps=1, cache=None):
        """Time one batched cycle per candidate CTAs/SM (the cycles advance the solution) and
        keep the fastest.  Returns {candidate: seconds}.  cache: as Solver.autotune, keyed by
        the batch's problem shapes."""
        import time

        path = TUNE_CACHE if cache is True else cache
        if path:
            hit = _tune_load(path).get(self.tune_key())
            if hit:
                self.set_grid(hit["ctas_per_sm"])
                self.tuned = hit["ctas_per_sm"]
                return {int(k): v for k, v in hit["s_per_cycle"].items()}
        times = {}
        for c in candidates:
            try:
                self.set_grid(c)
            except NrmgError:
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                self.fas_cycle()
            torch.cuda.synchronize()
            times[c] = (time.perf_counter() - t0) / reps
        best = min(times, key=times.get)
        self.set_grid(best)
        self.tuned = best
        if path:
            _tune_store(path, self.tune_key(), best, times)
        return times


def from_problem(prob, **kw) -> Solver:
    """Build a Solver from any object with the fields of a cavity problem description (a
    non-uniform grid when it carries column widths hx and row heights hy)."""
    walls = [(tuple(w.u), w.theta, w.chi) for w in prob.walls]
    S = Solver(prob.nx, prob.ny, prob.M, prob.Kn, walls, levels=prob.levels, lx=prob.lx, ly=prob.ly,
               model=prob.model, Pr=prob.Pr, omega=prob.omega, beta=prob.beta, order=prob.order,
               slope=prob.slope, cfl=prob.cfl, s1=prob.s1, s2=prob.s2, s3=prob.s3, gamma=prob.gamma,
               dtnu=getattr(prob, "dtnu", 0.0), **kw)
    if getattr(prob, "hx", None) is not None:
        S.set_spacing(prob.hx, prob.hy)
    return S


def residual_noalloc(prob, params, coeffs, want_R=True, stream=None):
    """R(f) and its norm for one grid through ``nrmg_residual_noalloc`` (no workspace, no
    device allocation inside the library).  ``prob`` carries the cavity description (fields
    of a Solver's constructor); params/coeffs are float64 CUDA tensors [cells,4], [cells,N_M].
    Returns (R or None, norm)."""
    L = lib()
    if not getattr(L, "_noalloc_ready", False):
        L.nrmg_residual_noalloc.restype = c_int
        L.nrmg_residual_noalloc.argtypes = [POINTER(Grid), c_int, c_double, POINTER(Wall), POINTER(Collision),
                                            POINTER(Opts), c_void_p, c_void_p, c_void_p, POINTER(c_double),
                                            c_void_p]
        L._noalloc_ready = True
    grid = Grid(prob.nx, prob.ny, prob.lx, prob.ly, prob.levels)
    opts = Opts(prob.order, prob.slope, prob.cfl, prob.s1, prob.s2, prob.s3, prob.gamma, 0,
                getattr(prob, "dtnu", 0.0))
    coll = Collision(prob.model, prob.Pr, prob.omega, prob.beta)
    wa = (Wall * 4)()
    for k, w in enumerate(prob.walls):
        wa[k].u = (c_double * 3)(*w.u)
        wa[k].theta = w.theta
        wa[k].chi = w.chi
    ncell, n = prob.nx * prob.ny, nmom(prob.M)
    # the library reads params[ncell][4] and coeffs[ncell][N_M] blindly: check them here
    for name, t, cols in (("params", params, 4), ("coeffs", coeffs, n)):
        if tuple(t.shape) != (ncell, cols):
            raise ValueError(f"{name} must have shape ({ncell}, {cols}), got {tuple(t.shape)}")
    if params.device != coeffs.device or not coeffs.is_cuda:
        raise ValueError("params and coeffs must be on the same CUDA device")
    dev = coeffs.device
    R = torch.empty((ncell, n), dtype=torch.float64, device=dev) if want_R else None
    norm = c_double(0.0)
    # the library takes its scratch address and SM count from the current device
    with torch.cuda.device(dev):
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        st = L.nrmg_residual_noalloc(ctypes.byref(grid), prob.M, prob.Kn, wa, ctypes.byref(coll),
                                     ctypes.byref(opts), _ptr(params), _ptr(coeffs), _ptr(R), ctypes.byref(norm),
                                     c_void_p(s.cuda_stream))
    if st != OK:
        raise NrmgError(st, "nrmg_residual_noalloc")
    return R, norm.value
