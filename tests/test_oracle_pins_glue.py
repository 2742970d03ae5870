"""Pins of three oracle parts that the other pins leave open (no GPU):

* the limited slope of the second-order reconstruction (van Albada average; Sec. 2.3,
  eq. moments-recon prints the central slope, the limiter is this library's reading) and the
  face states built from it;
* the middle branch of the HLL flux (Sec. 2.3, eq. flux-force-expansion, with the HLL reading
  of the numerical flux);
* the glue of the FAS cycle: the defect, the restriction of the state and of the defect, the
  coarse right-hand side (Sec. 3.2.2-3.2.3, Algorithm 2, eq. coarse-grid-problem) and the
  coarse-grid update (eq. rewritten-update).

Each check compares the oracle with something other than itself: defining properties and
textbook special cases of the limiter, Taylor expansion, the HLL flux in its intermediate-state
form (Harten, Lax and van Leer 1983) and its Rusanov special case, and exact identities of the
FAS cycle that hold whatever the discrete operator is (a fine state that already solves its
problem is left unchanged; a coarse change is carried to the fine cells by the basis
transform).  The checks are plain functions so that ``test_oracle_mutants.py`` can run them on
copies of the oracle with planted mistakes.
"""
import math

import numpy as np
from numpy.polynomial import hermite_e as He

import oracle
from conftest import oracle_solver
from inputs import SHAKHOV, lid_cavity, multi_indices, random_rhs, random_state


def _close(x, y, rtol, atol=0.0, what=""):
    x, y = np.asarray(x, float), np.asarray(y, float)
    err = np.abs(x - y).max() if x.size else 0.0
    bound = atol + rtol * max(np.abs(y).max() if y.size else 0.0, 1e-300)
    assert err <= bound, f"{what}: max deviation {err:.3e} > {bound:.3e}"


def he_max_root(n):
    return float(np.real(He.hermeroots([0] * n + [1])).max())


# ------------------------------------------------------------------ limited slope
def check_central_slope_is_exact_on_quadratics():
    """kind 1 (the slope the paper prints): the central difference is exact for quadratics."""
    rng = np.random.default_rng(40)
    for _ in range(50):
        a2, a1, a0 = rng.normal(size=3)
        x0, h = rng.uniform(-1, 1), 10 ** rng.uniform(-3, -1)
        q = lambda x: (a2 * x + a1) * x + a0  # noqa: E731
        s = oracle.slope(1, q(x0 - h), q(x0), q(x0 + h), h)
        _close(s, 2 * a2 * x0 + a1, 1e-9, 1e-9, "central slope on a quadratic")


def check_van_albada_defining_properties():
    """van Albada average of the one-sided differences a = q0 - qm, b = qp - q0 (per unit h):
    equal differences give the central slope, opposite ones zero; symmetric in (a, b), odd
    under reversal of the axis; a convex combination of a and b that leans to the smaller one
    when they share a sign; zero where one side is flat (it limits at extrema)."""
    rng = np.random.default_rng(41)
    for _ in range(300):
        h = 10 ** rng.uniform(-3, 0)
        a, b = rng.choice([-1.0, 1.0], 2) * 10 ** rng.uniform(-2, 1, 2)  # |a|, |b| >> eps = 1e-6
        # equal and opposite differences (q0 = 0 makes the differences exact)
        _close(oracle.slope(2, -a, 0.0, a, h), a / h, 1e-14, 0.0, "a = b")
        assert abs(oracle.slope(2, -a, 0.0, -a, h)) <= 1e-15 * abs(a) / h, "a = -b"
        s = oracle.slope(2, -a, 0.0, b, h)
        _close(oracle.slope(2, -b, 0.0, a, h), s, 1e-14, 1e-300, "symmetry in (a, b)")
        _close(oracle.slope(2, b, 0.0, -a, h), -s, 1e-14, 1e-300, "reversal of the axis")
        sh = s * h
        assert abs(sh) <= max(abs(a), abs(b)) * (1 + 1e-14)
        if a * b > 0:
            small, large = (a, b) if abs(a) < abs(b) else (b, a)
            tol = 1e-14 * abs(large)
            assert min(a, b) - tol <= sh <= max(a, b) + tol, "convex combination"
            assert abs(sh - small) <= abs(sh - large) * (1 + 1e-12), "leans to the smaller difference"
        # one flat side: the slope vanishes (up to the smoothing constant)
        assert abs(oracle.slope(2, 0.0, 0.0, b, h) * h) <= 1e-6 * abs(b), "flat left side"
        assert abs(oracle.slope(2, -a, 0.0, 0.0, h) * h) <= 1e-6 * abs(a), "flat right side"
        # homogeneous of degree 1 in q up to the smoothing constant, inversely proportional to h
        _close(oracle.slope(2, -3 * a, 0.0, 3 * b, h), 3 * s, 1e-13 + 1e-11 / min(a * a, b * b), 1e-300,
               "scaling in q")
        _close(oracle.slope(2, -a, 0.0, b, 2 * h), s / 2, 1e-14, 1e-300, "scaling in h")


def check_van_albada_limiter_function():
    """For differences far above the smoothing constant the slope times h is b phi(a/b) with
    the van Albada limiter function phi(r) = (r^2 + r)/(r^2 + 1) in Sweby's (1984) form:
    phi(0) = 0, phi(1) = 1, phi(r) -> 1 for large r, phi(1/r) = phi(r)/r."""
    phi = lambda r: (r * r + r) / (r * r + 1)  # noqa: E731
    rng = np.random.default_rng(42)
    for r in list(rng.uniform(-5, 5, 40)) + [0.0, 1.0, 1e6, -1.0]:
        b = rng.choice([-1, 1]) * 10 ** rng.uniform(-1, 1)
        a = r * b
        _close(oracle.slope(2, -a, 0.0, b, 1.0), b * phi(r), 1e-9, 1e-12 * abs(b), f"phi({r})")
    assert abs(phi(1e6) - 1) < 1e-5 and abs(phi(3.0) * 3 - phi(1 / 3) * 9) < 1e-12


def check_van_albada_is_second_order_on_smooth_data():
    """On smooth data both slopes approximate q'(x) to O(h^2): halving h divides the error
    by about four."""
    q = lambda x: math.sin(2 * x) + 0.3 * x * x  # noqa: E731
    dq = lambda x: 2 * math.cos(2 * x) + 0.6 * x  # noqa: E731
    for kind in (1, 2):
        for x0 in (0.37, -0.8, 1.3):
            errs = []
            for h in (1 / 16, 1 / 32, 1 / 64, 1 / 128):
                errs.append(abs(oracle.slope(kind, q(x0 - h), q(x0), q(x0 + h), h) - dq(x0)))
            for e0, e1 in zip(errs, errs[1:]):
                assert 3.0 < e0 / e1 < 5.0, (kind, x0, errs)
            assert errs[-1] < 5e-3


# ------------------------------------------------------------------ face states
def _linear_level(N, M, rng):
    """Cell states whose params and coefficients are affine in the cell centre (x, y)."""
    al = multi_indices(M)
    xs = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(xs, xs)  # [j][i]
    P0, F0 = random_state(rng, 1, 1, M, amp=0.1)
    gP = rng.uniform(-0.05, 0.05, (2, 4))
    gP[:, 2] = 0.0
    gF = rng.normal(size=(2, len(al))) * 0.02
    gF[:, al.sum(1) == 1] = 0.0
    gF[:, al[:, 2] % 2 == 1] = 0.0
    P = P0 + X.reshape(-1, 1) * gP[0] + Y.reshape(-1, 1) * gP[1]
    F = F0 + X.reshape(-1, 1) * gF[0] + Y.reshape(-1, 1) * gF[1]
    return P, F, gP, gF


def check_face_states_of_linear_fields():
    """Second order: on data affine in (x, y) every limiter reproduces the data at the face
    centres exactly (a = b); cells next to a wall take zero slope along its normal (reading),
    and first order takes the cell state."""
    M, N = 4, 8
    rng = np.random.default_rng(43)
    P, F, gP, gF = _linear_level(N, M, rng)
    h = 1.0 / N
    for order, slope in ((2, 2), (2, 1), (1, 0)):
        S = oracle_solver(lid_cavity(N, M, 0.1, 0.2, order=order, slope=slope))
        S.set_state(0, P, F)
        for j in range(N):
            for i in range(N):
                c = j * N + i
                for ax in (0, 1):
                    pos = i if ax == 0 else j
                    for sd in (1, -1):
                        p, f = S.face_state(0, i, j, ax, sd)
                        if order == 1 or pos in (0, N - 1):
                            ep, ef = P[c], F[c]
                        else:
                            ep, ef = P[c] + sd * 0.5 * h * gP[ax], F[c] + sd * 0.5 * h * gF[ax]
                        _close(p, ep, 1e-13, 1e-15, f"params {order, slope, i, j, ax, sd}")
                        _close(f, ef, 1e-13, 1e-15, f"coefficients {order, slope, i, j, ax, sd}")


def check_face_states_take_the_slope_along_their_axis():
    """Generic data: the face state is the cell value plus or minus h/2 times the slope of the
    cell and its two neighbours along the face's axis."""
    M, N = 3, 6
    rng = np.random.default_rng(44)
    P, F = random_state(rng, N, N, M, amp=0.1)
    h = 1.0 / N
    S = oracle_solver(lid_cavity(N, M, 0.1, 0.2, order=2, slope=2))
    S.set_state(0, P, F)
    for j in range(1, N - 1):
        for i in range(1, N - 1):
            c = j * N + i
            for ax in (0, 1):
                cm, cp = (c - 1, c + 1) if ax == 0 else (c - N, c + N)
                for sd in (1, -1):
                    p, f = S.face_state(0, i, j, ax, sd)
                    ep = [P[c, q] + sd * 0.5 * h * oracle.slope(2, P[cm, q], P[c, q], P[cp, q], h) for q in range(4)]
                    ef = [F[c, o] + sd * 0.5 * h * oracle.slope(2, F[cm, o], F[c, o], F[cp, o], h)
                          for o in range(F.shape[1])]
                    _close(p, ep, 1e-15, 1e-16, "params")
                    _close(f, ef, 1e-15, 1e-16, "coefficients")


# ------------------------------------------------------------------ HLL middle branch
def check_hll_rusanov_special_case():
    """Equal face bases at rest along the normal give s_L = -s_R = -C sqrt(theta); the HLL
    flux is then the Rusanov (local Lax-Friedrichs) flux
    F = (Xi a- + Xi a+)/2 - s_R (a+ - a-)/2."""
    rng = np.random.default_rng(45)
    for M in (3, 5, 8):
        al = multi_indices(M)
        C = he_max_root(M + 1)
        for ax in (0, 1):
            pc, _ = random_state(rng, 1, 1, M, amp=0.1)
            p, fm = random_state(rng, 1, 1, M, amp=0.1)
            _, fp = random_state(rng, 1, 1, M, amp=0.1)
            pc, p, fm, fp = pc[0], p[0].copy(), fm[0], fp[0]
            p[ax] = 0.0
            F = oracle.hll_flux(M, C, ax, pc, p, fm, p, fp)
            am, ap = oracle.transform(M, p, pc, fm), oracle.transform(M, p, pc, fp)
            s = C * math.sqrt(p[3])
            ref = 0.5 * (oracle.xi_mul(M, ax, pc, am) + oracle.xi_mul(M, ax, pc, ap)) - 0.5 * s * (ap - am)
            _close(F, ref, 1e-13, 1e-15, f"Rusanov M={M} ax={ax}")
            assert len(F) == len(al)


def check_hll_intermediate_state_form():
    """General face states with s_L < 0 < s_R (Davis speed bounds from both states): the flux
    equals F_L + s_L (U* - U_L) = F_R + s_R (U* - U_R), U* the HLL intermediate state
    (s_R U_R - s_L U_L - (F_R - F_L)) / (s_R - s_L), with U the face states re-expanded in
    the cell basis and F = Xi U."""
    rng = np.random.default_rng(46)
    n_mid = 0
    for M in (3, 5, 8):
        C = he_max_root(M + 1)
        for ax in (0, 1):
            for _ in range(3):
                (pc, pm, pp), fs = zip(*[(a[0], b[0]) for a, b in
                                         (random_state(rng, 1, 1, M, amp=0.1, u=0.6) for _ in range(3))])
                fm, fp = fs[1], fs[2]
                sL = min(pm[ax] - C * math.sqrt(pm[3]), pp[ax] - C * math.sqrt(pp[3]))
                sR = max(pm[ax] + C * math.sqrt(pm[3]), pp[ax] + C * math.sqrt(pp[3]))
                assert sL < 0.0 < sR
                n_mid += 1
                UL, UR = oracle.transform(M, pm, pc, fm), oracle.transform(M, pp, pc, fp)
                FL, FR = oracle.xi_mul(M, ax, pc, UL), oracle.xi_mul(M, ax, pc, UR)
                Us = (sR * UR - sL * UL - (FR - FL)) / (sR - sL)
                F = oracle.hll_flux(M, C, ax, pc, pm, fm, pp, fp)
                _close(F, FL + sL * (Us - UL), 1e-12, 1e-15, "left form")
                _close(F, FR + sR * (Us - UR), 1e-12, 1e-15, "right form")
    assert n_mid == 18


# ------------------------------------------------------------------ FAS glue
def _two_level_problem(M=3, N=16):
    return lid_cavity(N, M, 0.1, 0.3, levels=2, order=2, slope=2, model=SHAKHOV)


def _coarse_residual(prob, P, F):
    """R_H of a coarse state, evaluated by a separate one-level oracle of the coarse grid
    (zero right-hand side)."""
    C = oracle_solver(prob.replace(nx=prob.nx // 2, ny=prob.ny // 2, levels=1))
    C.set_state(0, P, F)
    R, _ = C.residual(0)
    return R


def _children(N):
    """fine cells of each coarse cell, in the order (2I,2J), (2I+1,2J), (2I,2J+1), (2I+1,2J+1)"""
    n = N // 2
    out = np.zeros((n * n, 4), dtype=np.int64)
    for J in range(n):
        for I in range(n):
            out[J * n + I] = [(2 * J) * N + 2 * I, (2 * J) * N + 2 * I + 1, (2 * J + 1) * N + 2 * I,
                              (2 * J + 1) * N + 2 * I + 1]
    return out


def check_fas_leaves_a_solved_fine_state_unchanged():
    """r_h := R_h(f) makes f the solution of the fine problem: the defect vanishes, so the
    coarse right-hand side is exactly R_H(f_bar_H), the coarse smoother has nothing to do, and
    the coarse-grid update returns f."""
    prob = _two_level_problem()
    rng = np.random.default_rng(47)
    P, F = random_state(rng, prob.ny, prob.nx, prob.M, amp=0.1)
    S = oracle_solver(prob)
    S.set_state(1, P, F)
    R, _ = S.residual(1)
    S.set_rhs(1, P, R)
    S.two_grid_setup(1)
    Pb, Fb = S.get_saved(0)
    rP, rF = S.get_rhs(0)
    _close(rP, Pb, 0.0, 0.0, "basis of r_H")
    RH = _coarse_residual(prob, Pb, Fb)
    _close(rF, RH, 1e-12, 1e-15, "r_H = R_H(f_bar_H)")
    assert S.smooth(0, 4) == oracle.OK
    Pc, Fc = S.get_state(0)
    _close(Pc, Pb, 1e-13, 1e-15, "coarse params after smoothing")
    _close(Fc, Fb, 1e-12, 1e-15, "coarse coefficients after smoothing")
    assert S.two_grid_update(1) == oracle.OK
    Pn, Fn = S.get_state(1)
    _close(Pn, P, 1e-13, 1e-15, "fine params after the update")
    _close(Fn, F, 1e-12, 1e-15, "fine coefficients after the update")


def check_fas_restriction_and_coarse_rhs():
    """r_h = R_h(f) + d makes the defect r_h - R_h(f) = d.  Then (Sec. 3.2.2):
    (u_H, theta_H) conserve mass, momentum and energy of the four children; f_bar_H and
    R_bar_H are the means of the children's f and d re-expanded in that basis; and
    r_H = R_H(f_bar_H) + R_bar_H."""
    prob = _two_level_problem()
    M = prob.M
    rng = np.random.default_rng(48)
    P, F = random_state(rng, prob.ny, prob.nx, M, amp=0.1)
    S = oracle_solver(prob)
    S.set_state(1, P, F)
    R, _ = S.residual(1)
    _, d = random_rhs(rng, prob.ny, prob.nx, M, amp=0.05)
    S.set_rhs(1, P, R + d)
    S.two_grid_setup(1)
    Pb, Fb = S.get_saved(0)
    rP, rF = S.get_rhs(0)
    ch = _children(prob.nx)
    al = multi_indices(M)
    RH = _coarse_residual(prob, Pb, Fb)
    for C, kids in enumerate(ch):
        rho = F[kids, 0]
        m = rho.sum()
        u = (rho[:, None] * P[kids, :3]).sum(0) / m
        e = (rho * ((P[kids, :3] ** 2).sum(1) + 3 * P[kids, 3])).sum()
        th = (e - m * (u ** 2).sum()) / (3 * m)
        _close(Pb[C], [*u, th], 1e-14, 1e-16, f"coarse basis {C}")
        fH = np.mean([oracle.transform(M, P[k], Pb[C], F[k]) for k in kids], axis=0)
        fH[al.sum(1) == 1] = 0.0
        _close(Fb[C], fH, 1e-13, 1e-15, f"f_bar_H {C}")
        dH = np.mean([oracle.transform(M, P[k], Pb[C], d[k]) for k in kids], axis=0)
        _close(rF[C], RH[C] + dH, 1e-12, 1e-15, f"r_H {C}")
    _close(rP, Pb, 0.0, 0.0, "basis of r_H")


def check_fas_update_carries_the_coarse_change():
    """eq. rewritten-update: a coarse solution f~_H = T(H_bar -> H~)(f_bar_H + delta), in a
    basis H~ of its own, changes each fine cell by T(H_bar -> cell) delta (delta with zero
    moments of degree <= 2, so the fine basis stays put)."""
    prob = _two_level_problem(M=4)
    M = prob.M
    al = multi_indices(M)
    rng = np.random.default_rng(49)
    P, F = random_state(rng, prob.ny, prob.nx, M, amp=0.1)
    S = oracle_solver(prob)
    S.set_state(1, P, F)
    S.two_grid_setup(1)
    Pb, Fb = S.get_saved(0)
    nc = Pb.shape[0]
    delta = rng.normal(size=Fb.shape) * 0.01
    delta[:, al.sum(1) <= 2] = 0.0
    delta[:, al[:, 2] % 2 == 1] = 0.0
    Pt = Pb.copy()
    Pt[:, :2] += rng.uniform(-0.05, 0.05, (nc, 2))
    Pt[:, 3] *= rng.uniform(0.9, 1.1, nc)
    Ft = np.array([oracle.transform(M, Pb[C], Pt[C], Fb[C] + delta[C]) for C in range(nc)])
    S.set_state(0, Pt, Ft)
    assert S.two_grid_update(1) == oracle.OK
    Pn, Fn = S.get_state(1)
    ch = _children(prob.nx)
    expect = F.copy()
    for C, kids in enumerate(ch):
        for k in kids:
            expect[k] += oracle.transform(M, Pb[C], P[k], delta[C])
    _close(Pn, P, 1e-13, 1e-15, "fine params")
    _close(Fn, expect, 1e-12, 1e-15, "fine coefficients")
    assert np.abs(Fn - F).max() > 1e-4  # the change is there


CHECKS = [check_central_slope_is_exact_on_quadratics, check_van_albada_defining_properties,
          check_van_albada_limiter_function, check_van_albada_is_second_order_on_smooth_data,
          check_face_states_of_linear_fields, check_face_states_take_the_slope_along_their_axis,
          check_hll_rusanov_special_case, check_hll_intermediate_state_form,
          check_fas_leaves_a_solved_fine_state_unchanged, check_fas_restriction_and_coarse_rhs,
          check_fas_update_carries_the_coarse_change]


def test_central_slope_is_exact_on_quadratics():
    check_central_slope_is_exact_on_quadratics()


def test_van_albada_defining_properties():
    check_van_albada_defining_properties()


def test_van_albada_limiter_function():
    check_van_albada_limiter_function()


def test_van_albada_is_second_order_on_smooth_data():
    check_van_albada_is_second_order_on_smooth_data()


def test_face_states_of_linear_fields():
    check_face_states_of_linear_fields()


def test_face_states_take_the_slope_along_their_axis():
    check_face_states_take_the_slope_along_their_axis()


def test_hll_rusanov_special_case():
    check_hll_rusanov_special_case()


def test_hll_intermediate_state_form():
    check_hll_intermediate_state_form()


def test_fas_leaves_a_solved_fine_state_unchanged():
    check_fas_leaves_a_solved_fine_state_unchanged()


def test_fas_restriction_and_coarse_rhs():
    check_fas_restriction_and_coarse_rhs()


def test_fas_update_carries_the_coarse_change():
    check_fas_update_carries_the_coarse_change()
