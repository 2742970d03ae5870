"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: velocity-space
quadrature of the definitions in Sec. 2.1-2.2, numpy/scipy library routines, closed
forms, conservation laws, symmetries, and exact algebraic identities.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

import oracle
from conftest import oracle_solver
from hermite_quad import H_values, He_products, gauss_rule, half_line_rule, project
from inputs import (BGK, ESBGK, SHAKHOV, Wall, heated_cavity, lid_cavity, maxwellian_state, multi_indices,
                    random_rhs, random_state)


def rand_grad(rng, M, amp=0.1, u=0.3):
    P, F = random_state(rng, 1, 1, M, amp=amp, u=u)
    return P[0], F[0]


def rand_general(rng, M, amp=0.1):
    """A function of F_M^[w,t] with arbitrary (non-Grad) coefficients."""
    al = multi_indices(M)
    w = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-0.1, 0.1), rng.uniform(0.8, 1.3)])
    f = rng.standard_normal(len(al)) * amp * 0.5 ** al.sum(1)
    f[0] = rng.uniform(0.8, 1.2)
    return w, f


# ------------------------------------------------------------------ enumeration
@pytest.mark.parametrize("M", [3, 5, 8, 10])
def test_enumeration_matches_layout(M):
    al = oracle.alphas(M)
    assert len(al) == math.comb(M + 3, 3)
    np.testing.assert_array_equal(al, multi_indices(M))


def test_hermite_max_root_vs_numpy():
    for n in range(2, 22):
        roots = He.hermeroots([0] * n + [1])
        assert abs(oracle.hermite_max_root(n) - roots.max()) < 1e-12 * max(1, roots.max())
    # values quoted for the CFL condition at M = 5, 8, 10 (largest root of He_{M+1})
    assert abs(oracle.hermite_max_root(6) - 3.3242574335521193) < 1e-13
    assert abs(oracle.hermite_max_root(9) - 4.512745863399783) < 1e-13
    assert abs(oracle.hermite_max_root(11) - 5.188001224374871) < 1e-13


# ------------------------------------------------------------------ (i) quadrature of moments
@pytest.mark.parametrize("M", [3, 4])
def test_macros_general_basis_vs_quadrature(M):
    rng = np.random.default_rng(1)
    al = multi_indices(M)
    for _ in range(3):
        w, f = rand_general(rng, M)
        xi, W = gauss_rule(w[:3], w[3], 14)
        fv = H_values(al, w[:3], w[3], xi) @ f
        rho = (W * fv).sum()
        mom = (W[:, None] * xi * fv[:, None]).sum(0)
        en = (W * (xi ** 2).sum(1) * fv).sum()
        u = mom / rho
        theta = (en - rho * (u ** 2).sum()) / (3 * rho)
        mac = oracle.macros(M, w, f)
        np.testing.assert_allclose(mac, [rho, *u, theta], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("M", [3, 5])
def test_grad_fields_vs_quadrature(M):
    """sigma_ij and q_i of eq. (sigma-heat) against the Grad relations of eq. (moments-relation)."""
    rng = np.random.default_rng(2)
    al = multi_indices(M)
    for _ in range(3):
        p, f = rand_grad(rng, M, amp=0.2)
        xi, W = gauss_rule(p[:3], p[3], 16)
        fv = H_values(al, p[:3], p[3], xi) @ f
        rho = (W * fv).sum()
        c = xi - p[None, :3]
        sig = np.einsum("p,pi,pj,p->ij", W, c, c, fv) - rho * p[3] * np.eye(3)
        q = 0.5 * np.einsum("p,p,pi,p->i", W, (c ** 2).sum(1), c, fv)
        out = oracle.cell_fields(M, p, f)
        expect = [rho, *p[:3], p[3], sig[0, 0], sig[0, 1], sig[0, 2], sig[1, 1], sig[1, 2], sig[2, 2], *q]
        np.testing.assert_allclose(out, expect, rtol=1e-11, atol=1e-12)


# ------------------------------------------------------------------ (ii) basis transform
@pytest.mark.parametrize("M", [3, 5, 8])
def test_transform_vs_quadrature(M):
    rng = np.random.default_rng(3)
    al = multi_indices(M)
    for _ in range(2):
        src, f = rand_general(rng, M)
        dst = src + np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 0.0, rng.uniform(-0.25, 0.25)])
        xi, W = gauss_rule(src[:3], src[3], M + 3)
        fv = H_values(al, src[:3], src[3], xi) @ f
        g_quad = project(al, dst[:3], dst[3], fv, xi, W)
        g = oracle.transform(M, src, dst, f)
        np.testing.assert_allclose(g, g_quad, rtol=1e-11, atol=1e-12 * np.abs(g).max())


@pytest.mark.parametrize("M", [3, 6, 10])
def test_transform_round_trip_and_transitivity(M):
    rng = np.random.default_rng(4)
    for _ in range(3):
        A, f = rand_general(rng, M)
        B = A + np.array([0.2, -0.15, 0.0, 0.2])
        C = A + np.array([-0.1, 0.25, 0.0, -0.15])
        back = oracle.transform(M, B, A, oracle.transform(M, A, B, f))
        np.testing.assert_allclose(back, f, rtol=0, atol=1e-13 * np.abs(f).max())
        two = oracle.transform(M, B, C, oracle.transform(M, A, B, f))
        one = oracle.transform(M, A, C, f)
        np.testing.assert_allclose(two, one, rtol=0, atol=1e-13 * np.abs(one).max())


def test_transform_identity_is_exact():
    rng = np.random.default_rng(5)
    A, f = rand_general(rng, 6)
    assert np.array_equal(oracle.transform(6, A, A, f), f)


# ------------------------------------------------------------------ (iii) xi multiplication
@pytest.mark.parametrize("M", [3, 5])
def test_xi_mul_vs_quadrature(M):
    rng = np.random.default_rng(6)
    al = multi_indices(M)
    for d in range(3):
        p, f = rand_general(rng, M)
        xi, W = gauss_rule(p[:3], p[3], M + 4)
        fv = H_values(al, p[:3], p[3], xi) @ f
        g_quad = project(al, p[:3], p[3], xi[:, d] * fv, xi, W)
        np.testing.assert_allclose(oracle.xi_mul(M, d, p, f), g_quad, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("M", [3, 5, 8])
def test_regularized_xi_spectrum(M):
    """Eigenvalues of P_M xi_d P_M are w_d + sqrt(t) * roots of He_{L+1} over its index lines."""
    n = math.comb(M + 3, 3)
    p = np.array([0.3, -0.2, 0.0, 1.7])
    al = multi_indices(M)
    for d in range(3):
        A = np.stack([oracle.xi_mul(M, d, p, np.eye(n)[k]) for k in range(n)], 1)
        ev = np.sort(np.linalg.eigvals(A).real)
        expect = []
        perp = al.copy()
        perp[:, d] = 0
        for row in np.unique(perp, axis=0):
            L = M - row.sum()
            expect += list(p[d] + math.sqrt(p[3]) * He.hermeroots([0] * (L + 1) + [1]))
        np.testing.assert_allclose(ev, np.sort(expect), atol=1e-8)
        # hyperbolicity bound used by eq. (local-CFL)
        assert np.abs(ev - p[d]).max() <= oracle.hermite_max_root(M + 1) * math.sqrt(p[3]) + 1e-9


# ------------------------------------------------------------------ (iv) half-range integrals
def test_halfrange_vs_scipy_quad():
    from scipy.integrate import quad

    K = 10
    for s in (+1, -1):
        J = oracle.halfrange(K, s)
        for k in range(K + 1):
            for m in range(K + 1):
                ck = [0] * k + [1]
                cm = [0] * m + [1]
                fn = lambda v: v * He.hermeval(v, ck) * He.hermeval(v, cm) * math.exp(-v * v / 2) / math.sqrt(2 * math.pi)
                a, b = (0, np.inf) if s > 0 else (-np.inf, 0)
                val, _ = quad(fn, a, b, epsabs=1e-13, epsrel=1e-12, limit=200)
                assert abs(J[k, m] - val) <= 1e-10 * max(1.0, abs(val)), (s, k, m, J[k, m], val)


def test_halfrange_sum_is_full_range():
    K = 12
    Jp, Jm = oracle.halfrange(K, +1), oracle.halfrange(K, -1)
    full = np.zeros((K + 1, K + 1))
    for m in range(K + 1):
        if m + 1 <= K:
            full[m + 1, m] = math.factorial(m + 1)
        if m - 1 >= 0:
            full[m - 1, m] = math.factorial(m)
    np.testing.assert_allclose(Jp + Jm, full, atol=1e-9 * np.abs(full).max())


# ------------------------------------------------------------------ collision
@pytest.mark.parametrize("Pr", [2.0 / 3.0, 0.4])
def test_shakhov_equilibrium_vs_quadrature(Pr):
    """f^E of eq. (Shakhov-f^E) projected on the cell basis, via Q = nu (f^E - f)."""
    M = 5
    rng = np.random.default_rng(7)
    al = multi_indices(M)
    p, f = rand_grad(rng, M, amp=0.2)
    Kn, omega, beta = 0.3, 0.81, 1.0
    rho, u, th = f[0], p[:3], p[3]
    xi, W = gauss_rule(u, th, 12)
    fv = H_values(al, u, th, xi) @ f
    c = xi - u[None, :]
    q = 0.5 * ((c ** 2).sum(1)[:, None] * c * (W * fv)[:, None]).sum(0)
    maxw = rho / (2 * math.pi * th) ** 1.5 * np.exp(-(c ** 2).sum(1) / (2 * th))
    fE = (1 + (1 - Pr) * (c @ q) / (5 * rho * th ** 2) * ((c ** 2).sum(1) / th - 5)) * maxw
    fE_coef = project(al, u, th, fE, xi, W)
    nu = beta * math.sqrt(math.pi / 2) * rho * th ** (1 - omega) / Kn
    Q = oracle.collision(M, SHAKHOV, Kn, Pr, omega, beta, p, f)
    np.testing.assert_allclose(Q, nu * (fE_coef - f), rtol=1e-10, atol=1e-12 * nu)


def test_bgk_collision_vs_quadrature():
    M = 4
    rng = np.random.default_rng(8)
    al = multi_indices(M)
    p, f = rand_grad(rng, M, amp=0.2)
    xi, W = gauss_rule(p[:3], p[3], 10)
    c = xi - p[None, :3]
    maxw = f[0] / (2 * math.pi * p[3]) ** 1.5 * np.exp(-(c ** 2).sum(1) / (2 * p[3]))
    fE_coef = project(al, p[:3], p[3], maxw, xi, W)
    nu = math.sqrt(math.pi / 2) * f[0] * p[3] ** (1 - 0.81) / 0.1
    Q = oracle.collision(M, BGK, 0.1, 1.0, 0.81, 1.0, p, f)
    np.testing.assert_allclose(Q, nu * (fE_coef - f), rtol=1e-10, atol=1e-12 * nu)


def es_state(rng, M, Pr, amp=0.15):
    """A Grad state with all six stress components set (sigma_13, sigma_23 too, so the
    full 3x3 form of eq. ES-f^E is exercised), trace-free, with Lambda positive definite."""
    al = multi_indices(M)
    p = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-0.1, 0.1), rng.uniform(0.8, 1.3)])
    f = rng.standard_normal(len(al)) * 0.05 * 0.5 ** np.maximum(al.sum(1) - 2, 0)
    f[0] = rng.uniform(0.8, 1.2)
    f[al.sum(1) == 1] = 0.0
    S = rng.uniform(-amp, amp, (3, 3))
    S = 0.5 * (S + S.T)
    S -= np.trace(S) / 3 * np.eye(3)
    sigma = S * f[0] * p[3]
    for i in range(3):
        for j in range(i, 3):
            e = np.zeros(3, dtype=int)
            e[i] += 1
            e[j] += 1
            f[int(np.where((al == e).all(1))[0][0])] = sigma[i, j] / (2.0 if i == j else 1.0)
    Lam = p[3] * np.eye(3) + (1 - 1 / Pr) * sigma / f[0]
    assert np.linalg.eigvalsh(Lam).min() > 0.2 * p[3]
    return p, f, sigma, Lam


@pytest.mark.parametrize("Pr", [2.0 / 3.0, 0.5])
def test_esbgk_equilibrium_vs_quadrature(Pr):
    """f^E of eq. (ES-f^E) projected on the cell basis.  The Gaussian of covariance Lambda is
    integrated exactly by a tensor Gauss-Hermite rule in z, xi = u + chol(Lambda) z."""
    M = 6
    rng = np.random.default_rng(17)
    al = multi_indices(M)
    p, f, sigma, Lam = es_state(rng, M, Pr)
    rho, u, th = f[0], p[:3], p[3]
    x, wx = He.hermegauss(8)
    Z = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    Wz = (wx[:, None, None] * wx[None, :, None] * wx[None, None, :]).reshape(-1) / (2 * math.pi) ** 1.5
    xi = u[None, :] + Z @ np.linalg.cholesky(Lam).T
    P = He_products(al, u, th, xi)
    fact = np.array([math.factorial(a) * math.factorial(b) * math.factorial(c) for a, b, c in al], dtype=float)
    fE_coef = rho * (Wz[:, None] * P).sum(0) * th ** (al.sum(1) / 2.0) / fact
    Kn, omega, beta = 0.3, 0.81, Pr
    nu = beta * math.sqrt(math.pi / 2) * rho * th ** (1 - omega) / Kn
    Q = oracle.collision(M, ESBGK, Kn, Pr, omega, beta, p, f)
    np.testing.assert_allclose(Q, nu * (fE_coef - f), rtol=1e-10, atol=1e-12 * nu)


def test_esbgk_conservation_and_relaxation_rates():
    """Mass, momentum and energy are conserved; the stress relaxes at nu/Pr (the property
    that gives ES-BGK its Prandtl number) and the heat flux and other odd moments at nu."""
    M = 7
    Pr = 2.0 / 3.0
    rng = np.random.default_rng(18)
    al = multi_indices(M)
    deg = al.sum(1)
    p, f, sigma, Lam = es_state(rng, M, Pr)
    nu = Pr * math.sqrt(math.pi / 2) * f[0] * p[3] ** (1 - 0.81) / 0.2
    Q = oracle.collision(M, ESBGK, 0.2, Pr, 0.81, Pr, p, f)
    assert abs(Q[0]) <= 1e-14 * nu and np.abs(Q[deg == 1]).max() <= 1e-14 * nu
    two = [int(np.where((al == e).all(1))[0][0]) for e in ([2, 0, 0], [0, 2, 0], [0, 0, 2])]
    assert abs(Q[two].sum()) <= 1e-13 * nu
    np.testing.assert_allclose(Q[deg == 2], -(nu / Pr) * f[deg == 2], rtol=1e-13, atol=1e-16)
    odd = deg % 2 == 1
    np.testing.assert_allclose(Q[odd], -nu * f[odd], rtol=1e-13, atol=1e-16)
    # degree 4: the Gaussian's fourth cumulant vanishes, so f^E_alpha = rho [s^alpha] (s^T B s)^2 / 8
    B = (Lam - p[3] * np.eye(3))
    for o in np.where(deg == 4)[0]:
        a = al[o]
        c = 0.0  # coefficient of s^a in (s^T B s)^2 / 8 = (sum_ij B_ij s_i s_j)^2 / 8
        for i, j, k, l in np.ndindex(3, 3, 3, 3):
            e = np.zeros(3, dtype=int)
            for d in (i, j, k, l):
                e[d] += 1
            if (e == a).all():
                c += B[i, j] * B[k, l] / 8.0
        assert abs(Q[o] - nu * (f[0] * c - f[o])) <= 1e-12 * nu


def test_esbgk_pr1_equals_bgk():
    M = 5
    rng = np.random.default_rng(33)
    P, F = random_state(rng, 8, 8, M)
    out = []
    for model, Pr in ((BGK, 2 / 3), (ESBGK, 1.0)):
        S = oracle_solver(lid_cavity(8, M, 0.2, 0.2, order=2, slope=2, model=model, Pr=Pr))
        S.set_state(0, P, F)
        S.smooth(0, 1)
        out.append(S.get_state(0))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ------------------------------------------------------------------ forward Euler (comparison scheme)
def test_euler_step_is_jacobi_with_the_global_cfl_step():
    """eq. (euler-scheme) with eq. (global-CFL): every cell moves from the same old state by
    the smallest local step of eq. (local-CFL); rebuilt here from the residual of the old state,
    the largest He_{M+1} root from numpy, and the (separately pinned) macroscopics and basis
    transform."""
    M = 4
    prob = lid_cavity(8, M, 0.2, 0.3, order=2, slope=2).replace(ny=6)
    rng = np.random.default_rng(41)
    P, F = random_state(rng, prob.ny, prob.nx, M)
    O = oracle_solver(prob)
    O.set_state(0, P, F)
    R, _ = O.residual(0)
    C = He.hermeroots([0] * (M + 1) + [1]).real.max()
    dx, dy = 1.0 / prob.nx, 1.0 / prob.ny
    sq = np.sqrt(P[:, 3])
    dt = (prob.cfl / ((np.abs(P[:, 0]) + C * sq) / dx + (np.abs(P[:, 1]) + C * sq) / dy)).min()
    al = multi_indices(M)
    e1 = [int(np.where((al == e).all(1))[0][0]) for e in ([1, 0, 0], [0, 1, 0], [0, 0, 1])]
    e2 = [int(np.where((al == e).all(1))[0][0]) for e in ([2, 0, 0], [0, 2, 0], [0, 0, 2])]
    P1, F1 = np.zeros_like(P), np.zeros_like(F)
    for c in range(P.shape[0]):
        g = F[c] + dt * R[c]
        mac = oracle.macros(M, P[c], g)
        P1[c] = mac[1:]
        F1[c] = oracle.transform(M, P[c], P1[c], g)
        F1[c, e1] = 0.0
        F1[c, e2] -= F1[c, e2].mean()
    assert O.euler(0, 1) == 0
    Po, Fo = O.get_state(0)
    np.testing.assert_allclose(Po, P1, rtol=0, atol=1e-13)
    np.testing.assert_allclose(Fo, F1, rtol=0, atol=1e-13 * np.abs(F1).max())
    # mass: the fluxes cancel pairwise and the walls carry none
    assert abs(Fo[:, 0].sum() - F[:, 0].sum()) <= 1e-13 * F[:, 0].sum()


def test_euler_reaches_the_fs_fixed_point_more_slowly():
    """Forward Euler conserves the total mass exactly (Jacobi update, conservative fluxes, no
    wall mass flux), so it reaches the steady state of the initial mass, which the mass-corrected
    FAS solve also reaches; single-level FS needs several times fewer steps (the paper's
    Tables 1-9 show 6-9x)."""
    prob = lid_cavity(8, 3, 0.2, 0.3, order=1)
    S = oracle_solver(prob.replace(s3=1))
    st, n_fs, _ = S.solve(1e-9, 5000)
    assert st == 0
    ref = oracle_solver(prob.replace(levels=2))
    assert ref.solve(1e-11, 300)[0] == 0
    E = oracle_solver(prob)
    m0 = E.mass()
    r0 = E.residual(0)[1]
    n_eu = 0
    while E.residual(0)[1] > 1e-9 * r0:
        assert E.euler(0, 1) == 0
        n_eu += 1
        assert n_eu < 20000
    assert abs(E.mass() - m0) <= 1e-13 * m0
    fr, fe = ref.fields(), E.fields()
    for k in range(fr.shape[-1]):
        scale = max(np.abs(fr[..., k]).max(), 1e-3)
        assert np.abs(fe[..., k] - fr[..., k]).max() <= 1e-6 * scale, k
    assert n_eu >= 3 * n_fs, (n_eu, n_fs)


# ------------------------------------------------------------------ interior flux
def test_hll_consistency_equal_states():
    """Identical states on both sides: the flux is the exact projected flux P_M xi_n f."""
    M = 5
    rng = np.random.default_rng(9)
    pc, fc = rand_grad(rng, M)
    ps, fs = rand_grad(rng, M)
    C = oracle.hermite_max_root(M + 1)
    for ax in (0, 1):
        F = oracle.hll_flux(M, C, ax, pc, ps, fs, ps, fs)
        a = oracle.transform(M, ps, pc, fs)
        np.testing.assert_allclose(F, oracle.xi_mul(M, ax, pc, a), rtol=1e-12, atol=1e-14)


def test_hll_upwind_limits():
    M = 4
    rng = np.random.default_rng(10)
    pc, fc = rand_grad(rng, M)
    pm, fm = rand_grad(rng, M)
    pp, fp = rand_grad(rng, M)
    C = oracle.hermite_max_root(M + 1)
    pm2, pp2 = pm.copy(), pp.copy()
    pm2[0] = pp2[0] = C * 1.2 * math.sqrt(max(pm[3], pp[3]))  # all waves move right
    F = oracle.hll_flux(M, C, 0, pc, pm2, fm, pp2, fp)
    np.testing.assert_allclose(F, oracle.xi_mul(M, 0, pc, oracle.transform(M, pm2, pc, fm)), rtol=1e-13)
    pm2[0] = pp2[0] = -pm2[0]  # all waves move left
    F = oracle.hll_flux(M, C, 0, pc, pm2, fm, pp2, fp)
    np.testing.assert_allclose(F, oracle.xi_mul(M, 0, pc, oracle.transform(M, pp2, pc, fp)), rtol=1e-13)


@pytest.mark.parametrize("M", [3, 5, 8])
def test_hll_conservative_across_cell_bases(M):
    """Rows |alpha| <= 2 (mass, momentum, energy fluxes) agree between the two cells."""
    rng = np.random.default_rng(11)
    al = multi_indices(M)
    low = al.sum(1) <= 2
    C = oracle.hermite_max_root(M + 1)
    for ax in (0, 1):
        pL, fL = rand_grad(rng, M)
        pR, fR = rand_grad(rng, M)
        FL = oracle.hll_flux(M, C, ax, pL, pL, fL, pR, fR)
        FR = oracle.hll_flux(M, C, ax, pR, pL, fL, pR, fR)
        FL_in_R = oracle.transform(M, pL, pR, FL)
        np.testing.assert_allclose(FL_in_R[low], FR[low], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ wall flux
def _wall_flux_by_quadrature(M, uw, thw, chi, w, pf, ff):
    """The kinetic diffuse/specular wall flux, integrated directly in the wall basis."""
    axis, s = [1, 0, 1, 0][w], [-1, 1, 1, -1][w]
    al = multi_indices(M)
    # f_face truncated in the wall basis (exact projection by Gauss-Hermite in the face basis)
    xi, W = gauss_rule(pf[:3], pf[3], M + 4)
    fv = H_values(al, pf[:3], pf[3], xi) @ ff
    a = project(al, uw, thw, fv, xi, W)
    # grid in wall coordinates: Gauss-Hermite across, Gauss-Legendre along the normal half-lines
    xg, wg = He.hermegauss(M + 4)
    out = np.zeros(len(al))
    rho_w = None
    for part in ("out", "in"):
        sign = s if part == "out" else -s
        vn, wn = half_line_rule(sign)
        grids = []
        for d in range(3):
            if d == axis:
                grids.append((vn, wn * np.exp(-0.5 * vn ** 2)))
            else:
                grids.append((xg, wg))
        V = np.stack(np.meshgrid(grids[0][0], grids[1][0], grids[2][0], indexing="ij"), -1).reshape(-1, 3)
        Wt = (grids[0][1][:, None, None] * grids[1][1][None, :, None] * grids[2][1][None, None, :]).reshape(-1)
        Wt = Wt * np.exp(0.5 * (V ** 2).sum(1)) * thw ** 1.5
        Xi = np.asarray(uw)[None, :] + math.sqrt(thw) * V
        xin = Xi[:, axis]
        Hw = H_values(al, uw, thw, Xi)
        if part == "out":
            g_out = Hw @ a
            mass_out = (Wt * xin * g_out).sum()
            maxw = Hw[:, 0]
            out += project(al, uw, thw, xin * g_out, Xi, Wt)
        else:
            maxw = Hw[:, 0]
            Xr = Xi.copy()
            Xr[:, axis] = -Xr[:, axis]
            g_ref = H_values(al, uw, thw, Xr) @ a
            mass_in = (Wt * xin * maxw).sum()
            rho_w = -mass_out / mass_in
            out += project(al, uw, thw, xin * (chi * rho_w * maxw + (1 - chi) * g_ref), Xi, Wt)
    return out, rho_w


@pytest.mark.parametrize("w", [0, 1, 2, 3])
@pytest.mark.parametrize("chi", [1.0, 0.7])
def test_wall_flux_vs_quadrature(w, chi):
    M = 4
    rng = np.random.default_rng(20 + w)
    pc, fc = rand_grad(rng, M, amp=0.15)
    axis = [1, 0, 1, 0][w]
    uw = np.array([0.0, 0.0, 0.0])
    uw[1 - axis] = 0.3  # tangential wall motion
    thw = 1.4
    F = oracle.wall_flux(M, uw, thw, chi, w, pc, pc, fc)
    Gq, rho_w = _wall_flux_by_quadrature(M, uw, thw, chi, w, pc, fc)
    pw = np.array([*uw, thw])
    F_in_wall = oracle.transform(M, pc, pw, F)
    np.testing.assert_allclose(F_in_wall, Gq, rtol=1e-9, atol=1e-11)
    assert abs(F[0]) < 1e-14  # no mass crosses the wall


def test_wall_flux_of_wall_maxwellian_is_exact_flux():
    M = 6
    pw = np.array([0.25, 0.0, 0.0, 1.3])
    f = np.zeros(math.comb(M + 3, 3))
    f[0] = 0.9
    F = oracle.wall_flux(M, pw[:3], pw[3], 1.0, 0, pw, pw, f)
    np.testing.assert_allclose(F, oracle.xi_mul(M, 1, pw, f), atol=1e-14)


# ------------------------------------------------------------------ (v) Maxwellian fixed point
@pytest.mark.parametrize("order,slope", [(1, 0), (2, 1), (2, 2)])
@pytest.mark.parametrize("model", [BGK, SHAKHOV, ESBGK])
@pytest.mark.parametrize("M", [3, 5])
def test_maxwellian_is_fixed_point(order, slope, model, M):
    prob = lid_cavity(8, M, 0.1, 0.0, order=order, slope=slope, levels=2, model=model)
    S = oracle_solver(prob)
    for lev in (0, 1):
        R, norm = S.residual(lev)
        assert norm <= 1e-14 and np.abs(R).max() <= 1e-14


# ------------------------------------------------------------------ (vi) conservation
@pytest.mark.parametrize("model", [BGK, SHAKHOV, ESBGK])
@pytest.mark.parametrize("order,slope", [(1, 0), (2, 2)])
def test_residual_conserves_mass(order, slope, model):
    M = 4
    prob = lid_cavity(8, M, 0.1, 0.3, order=order, slope=slope, model=model)
    S = oracle_solver(prob)
    rng = np.random.default_rng(30)
    P, F = random_state(rng, 8, 8, M)
    S.set_state(0, P, F)
    R, _ = S.residual(0)
    assert abs(R[:, 0].sum()) <= 1e-13 * np.abs(R[:, 0]).max()


def test_restriction_conserves_mass_momentum_energy():
    M = 5
    prob = lid_cavity(8, M, 0.1, 0.3, levels=2)
    S = oracle_solver(prob)
    rng = np.random.default_rng(31)
    P, F = random_state(rng, 8, 8, M, amp=0.1)
    S.set_state(1, P, F)
    S.two_grid_setup(1)
    Pc, Fc = S.get_state(0)

    def totals(P, F, area):
        rho = F[:, 0]
        return np.array([rho.sum(), *(rho[:, None] * P[:, :3]).sum(0),
                         (rho * (P[:, :3] ** 2).sum(1) + 3 * rho * P[:, 3]).sum()]) * area

    np.testing.assert_allclose(totals(Pc, Fc, 1 / 16), totals(P, F, 1 / 64), rtol=1e-13, atol=1e-15)
    al = multi_indices(M)
    # coarse states are in Grad form
    assert np.abs(Fc[:, al.sum(1) == 1]).max() == 0.0
    assert np.abs(Fc[:, 4] + Fc[:, 7] + Fc[:, 9]).max() < 1e-15


# ------------------------------------------------------------------ (vii) Shakhov(Pr=1) == BGK
def test_shakhov_pr1_equals_bgk():
    M = 5
    rng = np.random.default_rng(32)
    P, F = random_state(rng, 8, 8, M)
    out = []
    for model, Pr in ((BGK, 2 / 3), (SHAKHOV, 1.0)):
        S = oracle_solver(lid_cavity(8, M, 0.2, 0.2, order=2, slope=2, model=model, Pr=Pr))
        S.set_state(0, P, F)
        S.smooth(0, 1)
        out.append(S.get_state(0))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ------------------------------------------------------------------ (viii) mirror symmetry
@pytest.mark.parametrize("model", [SHAKHOV, ESBGK])
@pytest.mark.parametrize("order,slope", [(1, 0), (2, 2)])
def test_residual_reflection_equivariance(order, slope, model):
    M = 5
    N = 8
    prob = heated_cavity(N, M, 0.3, order=order, slope=slope, model=model)
    S = oracle_solver(prob)
    rng = np.random.default_rng(33)
    P, F = random_state(rng, N, N, M)
    al = multi_indices(M)
    sgn = (-1.0) ** al[:, 0]

    def reflect(P, F):
        P2 = P.reshape(N, N, 4)[:, ::-1].reshape(-1, 4).copy()
        F2 = F.reshape(N, N, -1)[:, ::-1].reshape(-1, F.shape[1]).copy()
        P2[:, 0] *= -1
        return P2, F2 * sgn[None, :]

    S.set_state(0, P, F)
    R1, _ = S.residual(0)
    S.set_state(0, *reflect(P, F))
    R2, _ = S.residual(0)
    _, R1r = reflect(P, R1)
    np.testing.assert_allclose(R2, R1r, rtol=0, atol=1e-12 * np.abs(R1).max())


# ------------------------------------------------------------------ (ix) xi_3 parity
@pytest.mark.parametrize("model", [BGK, ESBGK])
def test_odd_alpha3_stays_zero(model):
    M = 5
    prob = lid_cavity(8, M, 0.1, 0.4, order=2, slope=2, levels=2, model=model)
    S = oracle_solver(prob)
    rng = np.random.default_rng(34)
    S.set_state(1, *random_state(rng, 8, 8, M))
    S.fas_cycle()
    P, F = S.get_state(1)
    al = multi_indices(M)
    assert np.all(P[:, 2] == 0.0)
    assert np.all(F[:, al[:, 2] % 2 == 1] == 0.0)


# ------------------------------------------------------------------ norm
def test_local_norm_is_weighted_L2_of_FM():
    """||R_ij||^2 = int R(xi)^2 / H_0(xi) d xi (weighted L2 norm of F_M), by quadrature."""
    M = 4
    prob = lid_cavity(1, M, 0.2, 0.3)
    S = oracle_solver(prob)
    rng = np.random.default_rng(35)
    P, F = random_state(rng, 1, 1, M, amp=0.2)
    S.set_state(0, P, F)
    R, norm = S.residual(0)
    al = multi_indices(M)
    p = P[0]
    xi, W = gauss_rule(p[:3], p[3], 2 * M + 4)
    Hv = H_values(al, p[:3], p[3], xi)
    rv = Hv @ R[0]
    integral = (W * rv ** 2 / Hv[:, 0]).sum()
    assert abs(norm ** 2 - integral) <= 1e-11 * integral


# ------------------------------------------------------------------ solver behaviour
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_sweep_is_algorithm1_in_order(k):
    """One directional sweep equals Algorithm 1 emulated cell by cell in the order of Dk:
    dt from eq. (local-CFL), f <- f + dt (R_ij(f) - r_ij) with the newest neighbours,
    then the two-step re-projection of Sec. 2.4."""
    M, N = 3, 4
    prob = lid_cavity(N, M, 0.1, 0.3, order=2, slope=1)
    rng = np.random.default_rng(36 + k)
    P, F = random_state(rng, N, N, M)
    rP, rF = random_rhs(rng, N, N, M)
    S = oracle_solver(prob)
    S.set_state(0, P, F)
    S.set_rhs(0, rP, rF)
    S.sweep(0, k)
    Pn, Fn = S.get_state(0)
    E = oracle_solver(prob)
    E.set_rhs(0, rP, rF)
    P, F = P.copy(), F.copy()
    C = oracle.hermite_max_root(M + 1)
    irange = range(N) if k in (1, 4) else range(N - 1, -1, -1)
    jrange = range(N) if k in (1, 2) else range(N - 1, -1, -1)
    al = multi_indices(M)
    for i in irange:
        for j in jrange:
            c = j * N + i
            E.set_state(0, P, F)
            Rr = E.cell_residual(0, i, j)  # R_ij(f) - r_ij in the cell basis
            sq = math.sqrt(P[c, 3])
            dt = 0.9 / ((abs(P[c, 0]) + C * sq) * N + (abs(P[c, 1]) + C * sq) * N)
            g = F[c] + dt * Rr
            mac = oracle.macros(M, P[c], g)
            pn = mac[1:]
            fn = oracle.transform(M, P[c], pn, g)
            fn[al.sum(1) == 1] = 0.0
            two = [4, 7, 9]
            fn[two] -= fn[two].sum() / 3.0
            P[c], F[c] = pn, fn
    np.testing.assert_allclose(Pn, P, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(Fn, F, rtol=1e-13, atol=1e-15)


def test_fas_converges_and_conserves_mass():
    prob = lid_cavity(16, 3, 0.1, 0.2, levels=2)
    S = oracle_solver(prob)
    m0 = S.mass()
    st, cyc, rel = S.solve(1e-8, 60)
    assert st == oracle.OK and rel <= 1e-8 and cyc < 40
    assert abs(S.mass() - m0) < 1e-14
    f = S.fields()
    assert np.all(f[..., 0] > 0) and np.all(f[..., 4] > 0)
    # the lid drags the gas: positive u_1 under the lid, negative near the bottom
    assert f[-1, :, 1].mean() > 0 > f[0, :, 1].mean()


def test_esbgk_fas_converges_with_the_gas_dragged_by_the_lid():
    """ES-BGK (beta = Pr = 2/3) through the whole FAS cycle: converges, keeps the mass, and the
    stress sigma_12 under the lid has the sign of a viscous stress, -mu du_1/dy < 0 (the gas
    above moves faster)."""
    prob = lid_cavity(16, 4, 0.1, 0.3, levels=2, order=2, slope=2, model=ESBGK, beta=2 / 3)
    S = oracle_solver(prob)
    m0 = S.mass()
    st, cyc, rel = S.solve(1e-8, 80)
    assert st == oracle.OK and rel <= 1e-8 and cyc < 40
    assert abs(S.mass() - m0) < 1e-13
    f = S.fields()  # rho, u (3), theta, sigma_11, sigma_12, ..., q (3)
    assert np.all(f[..., 0] > 0) and np.all(f[..., 4] > 0)
    assert f[-1, :, 1].mean() > 0 > f[0, :, 1].mean()
    assert f[-1, :, 6].mean() < 0


def test_multigrid_cycle_count_is_flat_fs_doubles():
    """Sec. 3.1/3.2 behaviour: FS iterations grow with the grid, NMG cycles stay nearly flat."""
    cyc = {}
    for N in (8, 16):
        prob = lid_cavity(N, 3, 0.1, 0.2, levels=N // 8)
        S = oracle_solver(prob)
        st, c, rel = S.solve(1e-6, 200)
        assert st == oracle.OK
        cyc[N] = c
    fs = {}
    for N in (8, 16):
        prob = lid_cavity(N, 3, 0.1, 0.2, levels=1, s3=1)
        S = oracle_solver(prob)
        st, c, rel = S.solve(1e-6, 2000)
        assert st == oracle.OK
        fs[N] = c
    assert fs[16] > 1.5 * fs[8]
    assert cyc[16] <= 1.5 * cyc[8] + 2
    assert cyc[16] < fs[16] / 3


def test_dt_cap_changes_the_step_not_the_fixed_point():
    """With dtnu > 0 the local step is min(CFL step, dtnu/nu): the first cell of sweep D1 moves
    by exactly that step, and the solved fields agree with the uncapped solve."""
    M, N = 3, 8
    base = lid_cavity(N, M, 0.02, 0.3, levels=1)
    capped = base.replace(dtnu=0.5)
    rng = np.random.default_rng(40)
    P, F = random_state(rng, N, N, M)
    S = oracle_solver(capped)
    S.set_state(0, P, F)
    R0 = S.cell_residual(0, 0, 0)
    S.sweep(0, 1)
    Pn, _ = S.get_state(0)
    C = oracle.hermite_max_root(M + 1)
    sq = math.sqrt(P[0, 3])
    dt = 0.9 / ((abs(P[0, 0]) + C * sq) * N + (abs(P[0, 1]) + C * sq) * N)
    nu = math.sqrt(math.pi / 2) * F[0, 0] * P[0, 3] ** 0.19 / 0.02
    dt = min(dt, 0.5 / nu)
    mac = oracle.macros(M, P[0], F[0] + dt * R0)
    np.testing.assert_allclose(Pn[0], mac[1:], rtol=1e-13, atol=1e-15)
    # at this Kn the explicit collision step of the uncapped sweep is unstable on 8x8 ...
    S2 = oracle_solver(base.replace(s3=1))
    st, c, rel = S2.solve(1e-10, 3000)
    assert st == oracle.ERR_NONPHYSICAL
    S3 = oracle_solver(capped.replace(s3=1))
    st, c, rel = S3.solve(1e-10, 3000)
    assert st == oracle.OK
    # ... and where both are stable, both reach the same fixed point
    fields = []
    for cap in (0.0, 0.5):
        S4 = oracle_solver(lid_cavity(N, M, 0.1, 0.3, levels=1, s3=1, dtnu=cap))
        st, c, rel = S4.solve(1e-11, 3000)
        assert st == 0
        fields.append(S4.fields())
    np.testing.assert_allclose(fields[0], fields[1], rtol=0, atol=1e-9)


def test_fas_iterations_match_the_papers_table():
    """Table 1 of the paper prints the NMG iteration counts of the Shakhov lid cavity
    (Kn = 0.1, M = 5, first order): 12 on 32x32 and 12 on 64x64.  The oracle's FAS cycle,
    with this repository's readings of the flux and the wall (which the paper defers to other
    work), needs within two cycles of them and is grid-independent like them."""
    from inputs import levels_to_8

    here = os.path.dirname(os.path.abspath(__file__))
    rows = [l.split() for l in open(os.path.join(here, "golden", "paper_iteration_counts.txt"))
            if l.strip() and not l.startswith("#")]
    paper = {int(r[6]): int(r[8]) for r in rows if r[0] == "Table1" and r[7] == "NMG"}
    U = 50.0 / math.sqrt(208.13 * 273.0)
    got = {}
    for N in (32, 64):
        O = oracle_solver(lid_cavity(N, 5, 0.1, U, order=1, levels=levels_to_8(N), model=SHAKHOV))
        st, cyc, rel = O.solve(1e-8, 60)
        assert st == 0 and rel <= 1e-8
        got[N] = cyc
        assert abs(cyc - paper[N]) <= 2, (N, cyc, paper[N])
    assert abs(got[64] - got[32]) <= 2
