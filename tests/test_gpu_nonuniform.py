"""Non-uniform grids through the C ABI (nrmg_set_spacing) against the CPU oracle: residual,
sweeps (one-CTA and two-CTA cluster schedules), forward Euler, FAS cycles, the
mixed-precision smoother and the batched form on grids refined towards the walls."""
import numpy as np
import pytest
import torch

from conftest import oracle_solver
from inputs import ESBGK, SHAKHOV, heated_cavity, lid_cavity, random_rhs, random_state, stretched_widths
from paper_2206_13164_gb300 import nrmg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    return np.abs(a - b).max() / np.abs(b).max()


def stretched(prob, rx=2.5, ry=2.0):
    return prob.replace(hx=stretched_widths(prob.nx, prob.lx, rx), hy=stretched_widths(prob.ny, prob.ly, ry))


CASES = [
    ("lid_o1_M4_14x10", stretched(lid_cavity(14, 4, 0.1, 0.3).replace(ny=10))),
    ("lid_o2va_M6_16x12", stretched(lid_cavity(16, 6, 0.05, 0.4, order=2, slope=2).replace(ny=12), 3.0, 1.5)),
    ("lid_o2c_M5_12", stretched(lid_cavity(12, 5, 0.2, 0.3, order=2, slope=1))),
    ("heat_shak_o2va_M5_16", stretched(heated_cavity(16, 5, 0.3, order=2, slope=2, model=SHAKHOV))),
    ("lid_esbgk_o2va_M8_10x8", stretched(lid_cavity(10, 8, 0.1, 0.3, order=2, slope=2, model=ESBGK,
                                                    beta=2 / 3).replace(ny=8))),
]


def _pair(prob, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    P, F = random_state(rng, prob.ny, prob.nx, prob.M, amp=amp)
    G, O = nrmg.from_problem(prob, device=DEV), oracle_solver(prob)
    top = prob.levels - 1
    G.set_state(T(P), T(F))
    O.set_state(top, P, F)
    return G, O, rng


@pytest.mark.parametrize("name,prob", CASES, ids=[c[0] for c in CASES])
def test_residual_on_a_stretched_grid(name, prob):
    G, O, _ = _pair(prob, 300)
    Rg, ng = G.residual()
    Ro, no = O.residual()
    assert rel(Rg, Ro) <= 1e-12 and abs(ng - no) <= 1e-12 * no


@pytest.mark.parametrize("cluster", [False, True], ids=["one_cta", "two_cta_cluster"])
@pytest.mark.parametrize("name,prob", CASES, ids=[c[0] for c in CASES])
def test_fs_steps_on_a_stretched_grid(name, prob, cluster):
    G, O, rng = _pair(prob, 301)
    G.set_cluster((1 << 30) if cluster else 0)
    rP, rF = random_rhs(rng, prob.ny, prob.nx, prob.M, amp=0.02)
    G.set_rhs(0, T(rP), T(rF))
    O.set_rhs(0, rP, rF)
    G.smooth(0, 2)
    O.smooth(0, 2)
    Pg, Fg = G.get_state()
    Po, Fo = O.get_state(0)
    assert rel(Pg, Po) <= 1e-12 and rel(Fg, Fo) <= 1e-12


def test_euler_steps_on_a_stretched_grid():
    prob = CASES[1][1]
    G, O, _ = _pair(prob, 302)
    G.euler(3, 0)
    assert O.euler(0, 3) == 0
    Pg, Fg = G.get_state()
    Po, Fo = O.get_state(0)
    assert rel(Pg, Po) <= 1e-12 and rel(Fg, Fo) <= 1e-12


def test_fas_cycles_on_a_stretched_grid():
    """Three-level V-cycles: restriction with area weights, coarse right-hand sides, update
    and the area-weighted mass correction, against the oracle."""
    prob = stretched(lid_cavity(32, 5, 0.05, 0.3, order=2, slope=2, levels=3).replace(ny=16))
    G, O, _ = _pair(prob, 303, amp=0.03)
    m0 = O.mass()
    for _ in range(2):
        rg = G.fas_cycle()
        st, ro = O.fas_cycle()
        assert st == 0 and abs(rg - ro) <= 1e-10 * ro
    Pg, Fg = G.get_state()
    Po, Fo = O.get_state(2)
    assert rel(Pg, Po) <= 1e-11 and rel(Fg, Fo) <= 1e-11
    assert abs(O.mass() - m0) <= 1e-13


def test_explicit_uniform_widths_equal_the_uniform_grid():
    prob = lid_cavity(16, 5, 0.1, 0.3, order=2, slope=2, levels=2)
    rng = np.random.default_rng(304)
    P, F = random_state(rng, 16, 16, 5)
    A = nrmg.from_problem(prob, device=DEV)
    B = nrmg.from_problem(prob.replace(hx=tuple([1 / 16] * 16), hy=tuple([1 / 16] * 16)), device=DEV)
    for S in (A, B):
        S.set_state(T(P), T(F))
    ra, rb = A.fas_cycle(), B.fas_cycle()
    assert abs(ra - rb) <= 1e-12 * ra
    assert rel(B.get_state()[1], A.get_state()[1].cpu().numpy()) <= 1e-13


def test_solves_on_a_stretched_grid_fp64_mixed_and_batched():
    """To 1e-8 from the global Maxwellian: the FP64 cycle agrees with the oracle's solution
    (1e-10 per field) in the oracle's cycle count; the mixed-precision smoother and a batch
    reach the same solution (1e-6 and 1e-10)."""
    prob = stretched(lid_cavity(32, 4, 0.1, 0.2, order=2, slope=2, levels=3), 2.5, 2.5)
    O = oracle_solver(prob)
    sto, co, _ = O.solve(1e-8, 200)
    fo = O.fields()
    G = nrmg.from_problem(prob, device=DEV)
    st, cg, _ = G.solve(1e-8, 200)
    assert st == 0 and abs(cg - co) <= 1
    scale = np.abs(fo).reshape(-1, 14).max(0)
    keep = scale > 1e-12
    err = lambda f: (np.abs(f.cpu().numpy() - fo).reshape(-1, 14).max(0)[keep] / scale[keep]).max()  # noqa: E731
    assert err(G.fields()) <= 1e-10
    Xm = nrmg.Solver(prob.nx, prob.ny, prob.M, prob.Kn, [(tuple(w.u), w.theta, w.chi) for w in prob.walls],
                     levels=prob.levels, order=2, slope=2, precision=1, device=DEV)
    Xm.set_spacing(prob.hx, prob.hy)
    stm, cm, _ = Xm.solve(1e-8, 200)
    assert stm == 0 and err(Xm.fields()) <= 1e-6
    st2 = torch.cuda.Stream()
    with torch.cuda.stream(st2):
        bs = [nrmg.from_problem(prob, device=DEV, stream=st2)]
        B = nrmg.Batch(bs)
        stb, cb, _ = B.solve(1e-8, 200)
    assert stb == 0 and err(bs[0].fields()) <= 1e-10


def test_set_spacing_rejects_bad_widths():
    S = nrmg.from_problem(lid_cavity(8, 3, 0.1, 0.2), device=DEV)
    h = np.full(8, 1 / 8)
    bad = h.copy()
    bad[3] = -bad[3]
    for hx, hy in ((bad, h), (h * 1.01, h), (h, h[:7])):
        with pytest.raises((nrmg.NrmgError, ValueError)):
            S.set_spacing(hx, hy)
