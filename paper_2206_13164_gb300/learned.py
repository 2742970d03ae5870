"""The learned initial guess: binding of ``include/nrmg_net.h`` and the solve built on it.

The paper's solver starts every solve from the global Maxwellian.  This module adds a start
for the lid-driven cavity family: solve on a coarse grid, then go up one grid at a time,
predicting each finer solution from the coarser one with a small convolutional network (the
network corrects the bilinear interpolation of ten low-order fields, and the 13-moment Grad
state of the corrected fields becomes the finer grid's state), and finish with the plain FAS
cycles of Algorithm 2 on the target grid.  The network never decides the answer: at every
grid both starts, network and plain interpolation, run the same FAS cycles and the one with
the smaller residual norm (eq. relative-residual) after them continues, and the final solve
stops at the same 1e-8 of the plain start's residual as the plain solver
(``Solver.set_reference``).  By default the network is applied only on grids no finer than
the finest grid it was trained on; finer grids take the plain interpolation.

Everything numerical runs in ``libnrmg.so`` (network forward/backward/AdamW on the tensor
cores, the feature, target and Grad-state kernels, the solver); this file marshals arguments
and sequences the calls.  ``python -m paper_2206_13164_gb300.learned train`` regenerates the
training set with the solver and trains the network on the GPU.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import time
from ctypes import POINTER, c_double, c_float, c_int, c_longlong, c_size_t, c_ulonglong, c_void_p

import numpy as np
import torch

from . import nrmg
from .nrmg import Batch, NrmgError, Solver

CIN, COUT = 19, 10          # NRMG_LEARN_CIN, NRMG_LEARN_COUT
CORR_CIN = 29               # NRMG_CORR_CIN
ACCEPT_UPDATE, ACCEPT_SMOOTHED, ACCEPT_ALWAYS = 0, 1, 2  # NRMG_ACCEPT_*
HIDDEN = 64
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "lid_net.npz")
CORR_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "corr_net.npz")

_ready = False


def _lib():
    global _ready
    L = nrmg.lib()
    if not _ready:
        L.nrmg_net_workspace_bytes.restype = c_size_t
        L.nrmg_net_workspace_bytes.argtypes = [c_int, c_int, c_int, c_longlong]
        L.nrmg_net_create.restype = c_int
        L.nrmg_net_create.argtypes = [c_int, c_int, c_int, c_longlong, c_ulonglong, c_void_p, c_size_t, c_void_p,
                                      POINTER(c_void_p)]
        L.nrmg_net_destroy.restype = c_int
        L.nrmg_net_destroy.argtypes = [c_void_p]
        L.nrmg_net_param_count.restype = c_longlong
        L.nrmg_net_param_count.argtypes = [c_void_p]
        for name in ("nrmg_net_get_params", "nrmg_net_set_params"):
            getattr(L, name).restype = c_int
            getattr(L, name).argtypes = [c_void_p, c_void_p]
        L.nrmg_net_forward.restype = c_int
        L.nrmg_net_forward.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]
        L.nrmg_net_gradients.restype = c_int
        L.nrmg_net_gradients.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                         POINTER(c_double)]
        L.nrmg_net_train_step.restype = c_int
        L.nrmg_net_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_float, c_float,
                                          POINTER(c_double)]
        L.nrmg_learned_features.restype = c_int
        L.nrmg_learned_features.argtypes = [c_void_p, c_int, c_int, c_double, c_double, c_double, c_double, c_void_p,
                                            c_void_p, c_void_p]
        L.nrmg_learned_targets.restype = c_int
        L.nrmg_learned_targets.argtypes = [c_void_p, c_void_p, c_int, c_double, c_void_p, c_void_p]
        L.nrmg_learned_combine.restype = c_int
        L.nrmg_learned_combine.argtypes = [c_void_p, c_void_p, c_int, c_double, c_void_p, c_void_p]
        L.nrmg_learned_cycle_workspace_bytes.restype = c_size_t
        L.nrmg_learned_cycle_workspace_bytes.argtypes = [c_void_p]
        L.nrmg_fas_cycle_learned.restype = c_int
        L.nrmg_fas_cycle_learned.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_void_p,
                                             c_size_t, c_void_p, c_void_p, POINTER(c_double), POINTER(c_int),
                                             POINTER(c_double)]
        L.nrmg_learned_correct.restype = c_int
        L.nrmg_learned_correct.argtypes = [c_void_p, c_void_p, c_double, c_double]
        L.nrmg_learned_correction_targets.restype = c_int
        L.nrmg_learned_correction_targets.argtypes = [c_void_p, c_void_p, c_int, c_double, c_double, c_void_p,
                                                      c_void_p]
        _ready = True
    return L


def _p(t, dtype):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous {dtype} CUDA tensor")
    return c_void_p(t.data_ptr())


def _check(st, where):
    if st != nrmg.OK:
        raise NrmgError(st, where)


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


class Net:
    """The four-layer 3x3 convolutional network (BF16 tensor-core kernels, FP32 master weights)."""

    def __init__(self, cin=CIN, hidden=HIDDEN, cout=COUT, max_pixels=1 << 20, seed=0):
        if not torch.cuda.is_available():
            raise RuntimeError("the network kernels need a CUDA device")
        self.L = _lib()
        self.cin, self.hidden, self.cout, self.max_pixels = cin, hidden, cout, max_pixels
        nbytes = self.L.nrmg_net_workspace_bytes(cin, hidden, cout, max_pixels)
        if nbytes == 0:
            raise NrmgError(nrmg.ERR_ARG, "nrmg_net_workspace_bytes")
        self.stream = torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.h = c_void_p()
        _check(self.L.nrmg_net_create(cin, hidden, cout, max_pixels, seed, c_void_p(self.workspace.data_ptr()), nbytes,
                                      c_void_p(self.stream.cuda_stream), ctypes.byref(self.h)), "nrmg_net_create")
        self.n_params = int(self.L.nrmg_net_param_count(self.h))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.nrmg_net_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(self.L.nrmg_net_get_params(self.h, _p(out, torch.float32)), "nrmg_net_get_params")
        return out

    def set_params(self, params: torch.Tensor):
        params = params.to(device="cuda", dtype=torch.float32).contiguous()
        if params.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {params.numel()}")
        _check(self.L.nrmg_net_set_params(self.h, _p(params, torch.float32)), "nrmg_net_set_params")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x [B, H, W, cin] float32 CUDA -> [B, H, W, cout]."""
        B, H, W, _ = x.shape
        y = torch.empty((B, H, W, self.cout), dtype=torch.float32, device="cuda")
        _check(self.L.nrmg_net_forward(self.h, _p(x, torch.float32), B, H, W, _p(y, torch.float32)),
               "nrmg_net_forward")
        return y

    def gradients(self, x: torch.Tensor, t: torch.Tensor):
        """(gradient of the mean squared error in the flat parameter layout, loss)."""
        B, H, W, _ = x.shape
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = c_double(0.0)
        _check(self.L.nrmg_net_gradients(self.h, _p(x, torch.float32), _p(t, torch.float32), B, H, W,
                                         _p(g, torch.float32), ctypes.byref(loss)), "nrmg_net_gradients")
        return g, loss.value

    def train_step(self, x: torch.Tensor, t: torch.Tensor, lr: float, wd: float = 0.0, want_loss=True):
        B, H, W, _ = x.shape
        loss = c_double(0.0)
        _check(self.L.nrmg_net_train_step(self.h, _p(x, torch.float32), _p(t, torch.float32), B, H, W, lr, wd,
                                          ctypes.byref(loss) if want_loss else None), "nrmg_net_train_step")
        return loss.value if want_loss else None

    def save(self, path, **meta):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        np.savez(path, params=self.get_params().cpu().numpy(), cin=self.cin, hidden=self.hidden, cout=self.cout,
                 meta=json.dumps(meta))

    @classmethod
    def load(cls, path=WEIGHTS, max_pixels=1 << 20):
        z = np.load(path)
        net = cls(int(z["cin"]), int(z["hidden"]), int(z["cout"]), max_pixels=max_pixels)
        net.set_params(torch.from_numpy(z["params"]))
        net.meta = json.loads(str(z["meta"]))
        return net


# ---------------------------------------------------------------- field-level glue
def features(coarse_fields: torch.Tensor, Kn: float, U: float, lx=1.0, ly=1.0):
    """coarse fields [Hc, Wc, 14] float64 -> (interpolated fields [2Hc, 2Wc, 14], features [2Hc, 2Wc, 19])."""
    Hc, Wc, _ = coarse_fields.shape
    cf = coarse_fields.contiguous()
    pro = torch.empty((2 * Hc, 2 * Wc, 14), dtype=torch.float64, device="cuda")
    x = torch.empty((2 * Hc, 2 * Wc, CIN), dtype=torch.float32, device="cuda")
    _check(_lib().nrmg_learned_features(_p(cf, torch.float64), Hc, Wc, lx, ly, Kn, U, _p(pro, torch.float64),
                                        _p(x, torch.float32), _stream()), "nrmg_learned_features")
    return pro, x


def targets(prolonged: torch.Tensor, fine_fields: torch.Tensor, U: float) -> torch.Tensor:
    H, W, _ = prolonged.shape
    t = torch.empty((H, W, COUT), dtype=torch.float32, device="cuda")
    _check(_lib().nrmg_learned_targets(_p(prolonged, torch.float64), _p(fine_fields.contiguous(), torch.float64),
                                       H * W, U, _p(t, torch.float32), _stream()), "nrmg_learned_targets")
    return t


def combine(prolonged: torch.Tensor, y: torch.Tensor, U: float) -> torch.Tensor:
    H, W, _ = prolonged.shape
    out = torch.empty_like(prolonged)
    _check(_lib().nrmg_learned_combine(_p(prolonged, torch.float64), _p(y.contiguous(), torch.float32), H * W, U,
                                       _p(out, torch.float64), _stream()), "nrmg_learned_combine")
    return out


# ---------------------------------------------------------------- learned coarse-level correction
class LearnedCycle:
    """FAS cycles of one solver with the learned correction of the finest level's update
    (``nrmg_fas_cycle_learned``): the network's correction of the coarse change is kept only
    when it lowers the residual norm right after the update.  net=None runs the plain cycle
    (and still forms the network input, for training data)."""

    def __init__(self, solver: Solver, Kn: float, U: float, rule: int = ACCEPT_UPDATE):
        self.s, self.Kn, self.U, self.rule = solver, Kn, U, rule
        self.L = _lib()
        nbytes = self.L.nrmg_learned_cycle_workspace_bytes(solver.ctx)
        if nbytes == 0:
            raise NrmgError(nrmg.ERR_ARG, "nrmg_learned_cycle_workspace_bytes")
        self.nbytes = nbytes
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=solver.device)
        self.accepted = 0
        self.cycles = 0

    def cycle(self, net=None, x_out=None, fine_out=None, y=None, rule=None):
        """One cycle: (relative residual, correction kept, scale s of the coarse change).
        y: a given correction [H, W, 10] (network units) when net is None."""
        rel, acc, sc = c_double(0.0), c_int(0), c_double(0.0)
        rule = self.rule if rule is None else rule
        st = self.L.nrmg_fas_cycle_learned(self.s.ctx, net.h if net is not None else None,
                                           _p(y.contiguous(), torch.float32) if y is not None else None, rule,
                                           self.Kn, self.U, c_void_p(self.ws.data_ptr()), self.nbytes,
                                           _p(x_out, torch.float32) if x_out is not None else None,
                                           _p(fine_out, torch.float64) if fine_out is not None else None,
                                           ctypes.byref(sc), ctypes.byref(acc), ctypes.byref(rel))
        _check(st, "nrmg_fas_cycle_learned")
        self.cycles += 1
        self.accepted += acc.value
        return rel.value, bool(acc.value), sc.value

    def solve(self, net=None, tol=1e-8, max_cycles=400):
        """Cycles until the relative residual (of the solver's reference) is at most tol:
        (cycles, relative residual, corrections kept)."""
        rel, n0, a0 = 1.0, self.cycles, self.accepted
        while self.cycles - n0 < max_cycles:
            rel = self.cycle(net)[0]
            if rel <= tol:
                break
        return self.cycles - n0, rel, self.accepted - a0


def learned_correct(solver: Solver, y: torch.Tensor, scale: float, U: float):
    """The correction step alone on the solver's finest level (``nrmg_learned_correct``):
    y [cells, 10] float32 in network units."""
    _check(_lib().nrmg_learned_correct(solver.ctx, _p(y.contiguous(), torch.float32), scale, U),
           "nrmg_learned_correct")


def correction_targets(fine: torch.Tensor, converged: torch.Tensor, U: float, scale: float) -> torch.Tensor:
    """(converged - fine) of the ten learned fields in the units of the correction network."""
    H, W, _ = fine.shape
    t = torch.empty((H, W, COUT), dtype=torch.float32, device="cuda")
    _check(_lib().nrmg_learned_correction_targets(_p(fine.contiguous(), torch.float64),
                                                  _p(converged.contiguous(), torch.float64), H * W, U, scale,
                                                  _p(t, torch.float32), _stream()), "nrmg_learned_correction_targets")
    return t


def correction_pairs(problems, N, M, ref_tol=1e-10, stop=1e-7, max_cycles=60, log=print):
    """Training pairs of the correction network on the N x N cavity: for every (Kn, U), the
    converged solution (batched plain solve to ref_tol), then the plain cycles from the
    Maxwellian start; each cycle gives (network input, (converged - fine after the plain
    update) in network units) until the relative residual reaches `stop`."""
    t0 = time.perf_counter()
    sol = [lid_solver(N, M, kn, u) for kn, u in problems]
    b = Batch(sol)
    b.solve(ref_tol, 400)
    conv = [s.fields().clone() for s in sol]
    b.close()
    for s in sol:
        s.close()
    log(f"  {len(problems)} references on {N}x{N} in {time.perf_counter() - t0:.1f} s")
    xs, ts = [], []
    t0 = time.perf_counter()
    for (kn, u), F in zip(problems, conv):
        s = lid_solver(N, M, kn, u)
        lc = LearnedCycle(s, kn, u)
        for _ in range(max_cycles):
            x = torch.empty((N, N, CORR_CIN), dtype=torch.float32, device="cuda")
            fine = torch.empty((N, N, 14), dtype=torch.float64, device="cuda")
            rel, _, sc = lc.cycle(None, x_out=x, fine_out=fine)
            xs.append(x)
            ts.append(correction_targets(fine, F, u, sc))
            if rel <= stop:
                break
        s.close()
    log(f"  {len(xs)} pairs in {time.perf_counter() - t0:.1f} s")
    return torch.stack(xs), torch.stack(ts)


def evaluate_correction(N, M, Kn, U, net, tol=1e-8, max_cycles=400, grid=0, rules=(ACCEPT_UPDATE,)):
    """Cycles and wall time to tol from the Maxwellian start: the plain cycle and the cycle
    with the learned correction under each acceptance rule (\"learned\" for the first,
    \"learned_r<k>\" for the others), and each learned solution's largest field difference
    from the plain one."""
    out = {"N": N, "M": M, "Kn": Kn, "U": U}
    runs = {}
    names = [("plain", None, ACCEPT_UPDATE)] + [("learned" if k == 0 else f"learned_r{j}", net, j)
                                               for k, j in enumerate(rules)]
    for name, nn, j in names:
        s = lid_solver(N, M, Kn, U)
        s.set_grid(grid)
        lc = LearnedCycle(s, Kn, U, rule=j)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc, rel, acc = lc.solve(nn, tol, max_cycles)
        torch.cuda.synchronize()
        runs[name] = s
        out[name] = {"cycles": cyc, "rel_res": rel, "kept": acc, "rule": j, "seconds": time.perf_counter() - t0}
    fp = runs["plain"].fields()
    for name, s in runs.items():
        if name != "plain":
            out[name]["field_rel_err"] = field_rel_errors(s.fields(), fp)
    out["field_rel_err"] = out["learned"]["field_rel_err"]
    for s in runs.values():
        s.close()
    return out


# ---------------------------------------------------------------- the lid-driven cavity family
def lid_solver(N, M, Kn, U, order=2, slope=2, dtnu=1.0, coarsest=8, **kw) -> Solver:
    """N x N lid-driven cavity (BGK, diffuse walls at theta = 1, lid speed U along x), FAS
    levels down to a coarsest grid of `coarsest` cells."""
    levels = int(round(math.log2(N / coarsest))) + 1
    if coarsest << (levels - 1) != N:
        raise ValueError("N must be coarsest * 2^k")
    walls = [((0.0, 0.0, 0.0), 1.0, 1.0), ((0.0, 0.0, 0.0), 1.0, 1.0), ((U, 0.0, 0.0), 1.0, 1.0),
             ((0.0, 0.0, 0.0), 1.0, 1.0)]
    return Solver(N, N, M, Kn, walls, levels=levels, order=order, slope=slope, dtnu=dtnu, **kw)


def plain_res0(s: Solver) -> float:
    """Residual norm of the plain start (the global Maxwellian each context is created with)."""
    return s.residual(want_R=False)[1]


class LearnedSolve:
    """Contexts and sequence of one learned solve of the N x N lid-driven cavity.

    The first grid (`start` cells a side) is solved plainly; every finer grid up to N holds
    two contexts when a network is given: the interpolated start and the network's start.
    Both run the same FAS cycles (`polish` below the target, `decide` on the target) and the
    one with the smaller residual norm after them continues: the plain FAS cycle decides
    whether the network's start is used.  The final solve on the target stops at tol of the plain start's residual.
    Contexts are created here, outside the timed run."""

    def __init__(self, N, M, Kn, U, start=64, net=None, **kw):
        self.N, self.M, self.Kn, self.U, self.net = N, M, Kn, U, net
        self.coarse = lid_solver(start, M, Kn, U, **kw)
        self.grids = []
        n = start
        while n < N:
            n *= 2
            self.grids.append(n)
        if not self.grids or self.grids[-1] != N:
            raise ValueError("N must be start * 2^k with k >= 1")
        self.main = [lid_solver(n, M, Kn, U, **kw) for n in self.grids]
        self.twin = [lid_solver(n, M, Kn, U, **kw) for n in self.grids] if net is not None else None
        self.res0_grid = [plain_res0(s) for s in self.main]
        self.res0 = self.res0_grid[-1]

    def set_grid(self, ctas_per_sm: int):
        """Sweep grid (persistent CTAs per SM) of every context of the solve."""
        for s in [self.coarse] + self.main + (self.twin or []):
            s.set_grid(min(ctas_per_sm, int(s.L.nrmg_grid_limit(s.ctx))))

    def run(self, tol=1e-8, coarse_tol=1e-6, polish=2, decide=2, max_cycles=400, net_grids="trained",
            polish_tol=None):
        """net_grids: the grids on which the network's candidate is built: "trained" (default) =
        the grids no finer than the finest grid of the network's training data, None = all,
        or a list; polish_tol: below the target, after the deciding cycles, keep cycling the
        winner until its residual is polish_tol of that grid's plain start."""
        Kn, U = self.Kn, self.U
        if net_grids == "trained":
            sizes = (getattr(self.net, "meta", None) or {}).get("sizes")
            net_grids = [n for n in self.grids if n <= max(sizes)] if sizes else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, cyc_c, _ = self.coarse.solve(coarse_tol, max_cycles)
        fields = self.coarse.fields()
        t1 = time.perf_counter()
        log, wasted, decided = [], 0, 0
        target = None
        for k, n in enumerate(self.grids):
            last = k + 1 == len(self.grids)
            cyc = decide if last else polish
            pro, x = features(fields, Kn, U)
            cands = [self.main[k]]
            self.main[k].set_state_from_fields(pro)
            if self.net is not None and (net_grids is None or n in net_grids):
                y = self.net.forward(x[None])[0]
                try:
                    self.twin[k].set_state_from_fields(combine(pro, y, U))
                    cands.append(self.twin[k])
                except NrmgError:
                    pass
            res = []
            for c in cands:
                c.set_reference(mass=c.grid.lx * c.grid.ly)
                c.mass_correct()
                for _ in range(cyc):
                    c.fas_cycle()
                res.append(c.residual(want_R=False)[1])
            w = int(np.argmin(res))
            rec = {"N": n, "cycles": cyc, "res_interp": res[0], "used": ["interp", "net"][w]}
            if len(res) > 1:
                rec["res_net"] = res[1]
                wasted += cyc
            else:
                rec["net"] = "not applied"
            log.append(rec)
            if last:
                target = cands[w]
                decided = cyc
            else:
                if polish_tol is not None:
                    cands[w].set_reference(res0=self.res0_grid[k])
                    _, extra, _ = cands[w].solve(polish_tol, max_cycles)
                    rec["extra_cycles"] = extra
                fields = cands[w].fields()
        target.set_reference(mass=target.grid.lx * target.grid.ly, res0=self.res0)
        rel_start = target.residual(want_R=False)[1] / self.res0
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        st, cyc, rel = target.solve(tol, max_cycles)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        self.target = target
        return {"status": st, "cycles": decided + cyc, "final_cycles": cyc, "wasted_cycles": wasted,
                "rel_res": rel, "rel_res_after_climb": rel_start, "coarse_cycles": cyc_c, "t_coarse": t1 - t0,
                "t_climb": t2 - t1, "t_final": t3 - t2, "t_total": t3 - t0, "climb": log, "polish": polish,
                "decide": decide}


def plain_solve(N, M, Kn, U, tol=1e-8, max_cycles=400, grid=0, **kw):
    """The plain solve (global Maxwellian start) timed the same way: (solver, record)."""
    s = lid_solver(N, M, Kn, U, **kw)
    s.set_grid(grid)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, cyc, rel = s.solve(tol, max_cycles)
    torch.cuda.synchronize()
    return s, {"status": st, "cycles": cyc, "rel_res": rel, "t_total": time.perf_counter() - t0}


# ---------------------------------------------------------------- training data and training
def draw_problems(n, rng, holdout=None, kn_range=(0.01, 1.0), u_range=(0.05, 0.5), box=(0.08, 0.03)):
    """n (Kn, U) pairs: Kn log-uniform, U uniform, none within `box` (in log10 Kn, U) of holdout."""
    out = []
    while len(out) < n:
        kn = 10.0 ** rng.uniform(math.log10(kn_range[0]), math.log10(kn_range[1]))
        u = rng.uniform(*u_range)
        if holdout is not None and abs(math.log10(kn) - math.log10(holdout[0])) < box[0] and abs(u - holdout[1]) < box[1]:
            continue
        out.append((kn, u))
    return out


def solve_group(problems, sizes, M, tol, max_cycles=150, log=print):
    """Solve each (Kn, U) on every grid of `sizes` (ascending), the first plainly, each next one
    from the interpolated previous solution, all problems of one grid in one batch.  Returns
    per grid the fields [n, N, N, 14] and the cycle counts."""
    out = []
    prev = None
    for N in sizes:
        sol = [lid_solver(N, M, kn, u) for kn, u in problems]
        r0 = [plain_res0(s) for s in sol]
        if prev is not None:
            for s, f, r, (kn, u) in zip(sol, prev, r0, problems):
                pro, _ = features(f, kn, u)
                s.set_state_from_fields(pro)
                s.set_reference(mass=1.0, res0=r)
                s.mass_correct()
        b = Batch(sol)
        t0 = time.perf_counter()
        st, cyc, rel = b.solve(tol, max_cycles)
        torch.cuda.synchronize()
        log(f"  grid {N}: {len(sol)} problems, cycles max {max(cyc)} mean {np.mean(cyc):.1f}, "
            f"worst rel {max(rel):.2e}, {time.perf_counter() - t0:.1f} s")
        prev = [s.fields().clone() for s in sol]
        out.append((torch.stack(prev), cyc))
        b.close()
        for s in sol:
            s.close()
    return out


def make_pairs(problems, fields_by_size):
    """Training pairs (features, targets) for every consecutive pair of grids."""
    xs, ts = [], []
    for k in range(1, len(fields_by_size)):
        fc, ff = fields_by_size[k - 1], fields_by_size[k]
        X = torch.empty((len(problems),) + ff.shape[1:3] + (CIN,), dtype=torch.float32, device="cuda")
        T = torch.empty((len(problems),) + ff.shape[1:3] + (COUT,), dtype=torch.float32, device="cuda")
        for i, (kn, u) in enumerate(problems):
            pro, x = features(fc[i], kn, u)
            X[i] = x
            T[i] = targets(pro, ff[i], u)
        xs.append(X)
        ts.append(T)
    return xs, ts


def train(net, data, epochs, batch=16, lr=2e-3, lr_min=2e-5, wd=1e-4, seed=0, log=print):
    """AdamW over the pairs in `data` (a list of (X, T) tensors, one per image size) with a
    cosine learning-rate schedule.  Returns the per-epoch mean losses."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps_per_epoch = sum((X.shape[0] + batch - 1) // batch for X, _ in data)
    total = epochs * steps_per_epoch
    step, hist = 0, []
    for ep in range(epochs):
        order = []
        for k, (X, _) in enumerate(data):
            perm = torch.randperm(X.shape[0], generator=g)
            order += [(k, perm[i:i + batch]) for i in range(0, X.shape[0], batch)]
        idx = torch.randperm(len(order), generator=g).tolist()
        losses = []
        for j in idx:
            k, sel = order[j]
            X, T = data[k]
            sel = sel.to("cuda")
            cur = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * step / max(total, 1)))
            losses.append(net.train_step(X.index_select(0, sel).contiguous(), T.index_select(0, sel).contiguous(),
                                         cur, wd))
            step += 1
        hist.append(float(np.mean(losses)))
        log(f"  epoch {ep + 1}/{epochs}: loss {hist[-1]:.4e}")
    return hist


FIELD_NAMES = ("rho", "u1", "u2", "u3", "theta", "s11", "s12", "s13", "s22", "s23", "s33", "q1", "q2", "q3")


def field_rel_errors(f, ref):
    """Per field of nrmg_fields' [ny][nx][14] layout: max |f - ref| / max |ref| (fields whose
    reference vanishes, such as u3, are left out)."""
    dev = (f - ref).abs().amax(dim=(0, 1))
    scale = ref.abs().amax(dim=(0, 1))
    return {n: float(dev[k] / scale[k]) for k, n in enumerate(FIELD_NAMES) if float(scale[k]) > 1e-12}


def evaluate(N, M, Kn, U, net, start=64, polish=2, decide=2, tol=1e-8, grid=0, mixed=False):
    """Cycles and wall time to tol on one cavity: plain start, climb without the network, climb
    with it (and, with mixed, the plain start and the climb with the network on the
    mixed-precision smoother); the largest field difference of each against the plain
    solution.  grid: the sweep grid of every context (CTAs per SM, 0 = occupancy)."""
    plain, rp = plain_solve(N, M, Kn, U, tol, grid=grid)
    ref = plain.fields()
    out = {"N": N, "M": M, "Kn": Kn, "U": U, "start": start, "grid": grid, "plain": rp}
    if mixed:
        pm, rpm = plain_solve(N, M, Kn, U, tol, grid=grid, precision=1)
        fpm = pm.fields()
        rpm["max_field_diff"] = float((fpm - ref).abs().max())
        rpm["field_rel_err"] = field_rel_errors(fpm, ref)
        out["plain_mixed"] = rpm
        pm.close()
    runs = [("no_net", None, 0), ("net", net, 0)] + ([("net_mixed", net, 1)] if mixed else [])
    for name, nn, prec in runs:
        ls = LearnedSolve(N, M, Kn, U, start=start, net=nn, precision=prec)
        ls.set_grid(grid)
        r = ls.run(tol=tol, polish=polish, decide=decide)
        fl = ls.target.fields()
        r["max_field_diff"] = float((fl - ref).abs().max())
        r["field_rel_err"] = field_rel_errors(fl, ref)
        out[name] = r
        del ls
    plain.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="Generate solver solutions and train the learned initial guess.")
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--n64", type=int, default=1500, help="problems solved on 32x32 and 64x64")
    tr.add_argument("--n128", type=int, default=500, help="problems also solved on 128x128")
    tr.add_argument("--M", type=int, default=8)
    tr.add_argument("--tol", type=float, default=1e-6)
    tr.add_argument("--group", type=int, default=64)
    tr.add_argument("--epochs", type=int, default=60)
    tr.add_argument("--seed", type=int, default=2206)
    tr.add_argument("--holdout", type=float, nargs=2, default=(0.03, 0.35), metavar=("KN", "U"))
    tr.add_argument("--out", default=WEIGHTS)
    ev = sub.add_parser("eval")
    ev.add_argument("--N", type=int, default=512)
    ev.add_argument("--M", type=int, default=10)
    ev.add_argument("--Kn", type=float, default=0.03)
    ev.add_argument("--U", type=float, default=0.35)
    ev.add_argument("--start", type=int, default=64)
    ev.add_argument("--polish", type=int, default=2)
    ev.add_argument("--decide", type=int, default=2)
    ev.add_argument("--weights", default=WEIGHTS)
    tc = sub.add_parser("train-correction", help="generate cycle data and train the coarse-correction network")
    tc.add_argument("--n", type=int, default=64, help="training cavities")
    tc.add_argument("--N", type=int, default=64)
    tc.add_argument("--M", type=int, default=8)
    tc.add_argument("--epochs", type=int, default=40)
    tc.add_argument("--seed", type=int, default=2207)
    tc.add_argument("--holdout", type=float, nargs=2, default=(0.03, 0.35), metavar=("KN", "U"))
    tc.add_argument("--eval-N", type=int, default=128)
    tc.add_argument("--out", default=CORR_WEIGHTS)
    pr = sub.add_parser("profile", help="a few forward passes and training steps on one image (profiling case)")
    pr.add_argument("--N", type=int, default=512)
    pr.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    if a.cmd == "profile":
        net = Net(max_pixels=a.N * a.N, seed=0)
        x = torch.randn((1, a.N, a.N, CIN), dtype=torch.float32, device="cuda")
        t = torch.randn((1, a.N, a.N, COUT), dtype=torch.float32, device="cuda")
        for _ in range(a.reps):
            net.forward(x)
            net.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        print(f"profile case: {a.reps} forward passes and training steps on {a.N}x{a.N}", flush=True)
        return
    if a.cmd == "train-correction":
        rng = np.random.default_rng(a.seed)
        probs = draw_problems(a.n, rng, holdout=a.holdout)
        t0 = time.perf_counter()
        X, T = correction_pairs(probs, a.N, a.M)
        t_data = time.perf_counter() - t0
        net = Net(cin=CORR_CIN, cout=COUT, max_pixels=16 * a.N * a.N, seed=a.seed)
        t0 = time.perf_counter()
        hist = train(net, [(X, T)], a.epochs)
        t_train = time.perf_counter() - t0
        net.save(a.out, n_pairs=[int(X.shape[0])], sizes=[a.N], M=a.M, epochs=a.epochs, seed=a.seed,
                 holdout=list(a.holdout), loss_history=hist, t_data_s=t_data, t_train_s=t_train, problems=a.n)
        print(f"saved {a.out}: {X.shape[0]} pairs, final loss {hist[-1]:.4e}, data {t_data:.0f} s, "
              f"training {t_train:.0f} s", flush=True)
        del X, T
        ev = evaluate_correction(a.eval_N, a.M, a.holdout[0], a.holdout[1],
                                 Net.load(a.out, max_pixels=a.eval_N * a.eval_N),
                                 rules=(ACCEPT_UPDATE, ACCEPT_SMOOTHED, ACCEPT_ALWAYS))
        print(json.dumps(ev), flush=True)
        return
    if a.cmd == "eval":
        print(json.dumps(evaluate(a.N, a.M, a.Kn, a.U, Net.load(a.weights, max_pixels=a.N * a.N), start=a.start,
                                  polish=a.polish, decide=a.decide)), flush=True)
        return
    rng = np.random.default_rng(a.seed)
    t_start = time.perf_counter()
    probs = draw_problems(a.n64, rng, holdout=a.holdout)
    # the first n128 problems also get the 128 x 128 grid; within each part, groups of similar
    # Kn converge in similar cycle counts, so a batch rarely waits on one slow problem
    probs = sorted(probs[:a.n128]) + sorted(probs[a.n128:])
    data64, data128 = ([], []), ([], [])
    starts = list(range(0, a.n128, a.group)) + list(range(a.n128, a.n64, a.group))
    for g0 in starts:
        big = g0 < a.n128
        grp = probs[g0:min(g0 + a.group, a.n128 if big else a.n64)]
        print(f"group at {g0}: {len(grp)} problems, Kn {grp[0][0]:.3f}..{grp[-1][0]:.3f}, grids {'32/64/128' if big else '32/64'}", flush=True)
        res = solve_group(grp, [32, 64, 128] if big else [32, 64], a.M, a.tol)
        xs, ts = make_pairs(grp, [r[0] for r in res])
        data64[0].append(xs[0])
        data64[1].append(ts[0])
        if big:
            data128[0].append(xs[1])
            data128[1].append(ts[1])
        del res
    data = [(torch.cat(data64[0]), torch.cat(data64[1]))]
    if data128[0]:
        data.append((torch.cat(data128[0]), torch.cat(data128[1])))
    t_data = time.perf_counter() - t_start
    print(f"data: {sum(X.shape[0] for X, _ in data)} pairs in {t_data:.0f} s", flush=True)
    net = Net(max_pixels=16 * 128 * 128, seed=a.seed)
    t0 = time.perf_counter()
    hist = train(net, data, a.epochs)
    t_train = time.perf_counter() - t0
    net.save(a.out, n_pairs=[X.shape[0] for X, _ in data], sizes=[X.shape[1] for X, _ in data], M=a.M, tol=a.tol,
             epochs=a.epochs, seed=a.seed, holdout=list(a.holdout), loss_history=hist, t_data_s=t_data,
             t_train_s=t_train)
    print(f"saved {a.out}: final loss {hist[-1]:.4e}, data {t_data:.0f} s, training {t_train:.0f} s", flush=True)


if __name__ == "__main__":
    main()
