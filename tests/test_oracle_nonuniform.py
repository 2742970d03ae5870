"""Pins of the oracle on non-uniform grids (no GPU).

The paper motivates its local time step (Sec. 2.4, eq. local-CFL) with non-uniform grids; the
cavity grids here are tensor products of column widths hx and row heights hy (refined towards
the walls), a coarse cell merging two columns and two rows of the next finer level.  The
residual divides each cell's flux differences by its own widths, the second-order slopes use
the distances between cell centres, the norm and the mass weigh each cell by its area, and the
restriction averages the four children with their areas.  Each check compares with what the
geometry fixes: a uniform grid given as explicit widths, the Maxwellian fixed point, mass
conservation, exact reconstruction of affine data, conservation by the restriction, and the
converged flow against the uniform grid's.
"""
import numpy as np

import oracle
from conftest import oracle_solver
from inputs import SHAKHOV, lid_cavity, multi_indices, random_rhs, random_state, stretched_widths


def _close(x, y, rtol, atol=0.0, what=""):
    x, y = np.asarray(x, float), np.asarray(y, float)
    err = np.abs(x - y).max()
    bound = atol + rtol * max(np.abs(y).max(), 1e-300)
    assert err <= bound, f"{what}: max deviation {err:.3e} > {bound:.3e}"


def stretched(prob, ratio=2.0):
    return prob.replace(hx=stretched_widths(prob.nx, prob.lx, ratio), hy=stretched_widths(prob.ny, prob.ly, ratio))


def check_explicit_uniform_widths_equal_the_uniform_grid():
    """Equal widths given explicitly take the non-uniform code paths (centre distances, area
    weights) and must reproduce the uniform grid to rounding."""
    prob = lid_cavity(16, 4, 0.1, 0.3, order=2, slope=2, levels=2, model=SHAKHOV)
    h = tuple([1.0 / 16] * 16)
    rng = np.random.default_rng(70)
    P, F = random_state(rng, 16, 16, 4, amp=0.1)
    rP, rF = random_rhs(rng, 16, 16, 4)
    out = []
    for p in (prob, prob.replace(hx=h, hy=h)):
        S = oracle_solver(p)
        S.set_state(1, P, F)
        S.set_rhs(1, rP, rF)
        R, n = S.residual(1)
        S.sweep(1, 2)
        S.set_rhs(1, None)
        st, rel = S.fas_cycle()
        out.append((R, n, S.get_state(1), rel))
    (R0, n0, s0, r0), (R1, n1, s1, r1) = out
    _close(R1, R0, 1e-13, 0, "residual")
    _close(s1[1], s0[1], 1e-13, 0, "state after a sweep and a cycle")
    assert abs(n1 - n0) <= 1e-13 * n0 and abs(r1 - r0) <= 1e-12 * r0


def check_maxwellian_is_a_fixed_point_on_a_stretched_grid():
    for order, slope in ((1, 0), (2, 1), (2, 2)):
        prob = stretched(lid_cavity(12, 4, 0.1, 0.0, order=order, slope=slope).replace(ny=10))
        S = oracle_solver(prob)
        _, norm = S.residual(0)
        assert norm <= 1e-14, (order, slope, norm)


def check_residual_conserves_mass_on_a_stretched_grid():
    """The mass rows of the interior fluxes cancel between neighbours only when each cell's
    flux difference is weighted with its own area: sum_ij R_ij,0 hx_i hy_j = 0."""
    prob = stretched(lid_cavity(12, 4, 0.1, 0.3, order=2, slope=2).replace(ny=10), ratio=3.0)
    S = oracle_solver(prob)
    rng = np.random.default_rng(71)
    P, F = random_state(rng, 10, 12, 4, amp=0.1)
    S.set_state(0, P, F)
    R, _ = S.residual(0)
    area = np.outer(prob.hy, prob.hx).ravel()
    total = (R[:, 0] * area).sum()
    assert abs(total) <= 1e-13 * (np.abs(R[:, 0]) * area).sum(), total


def check_face_states_of_affine_fields_on_a_stretched_grid():
    """Data affine in the cell-centre coordinates are reconstructed exactly at the face
    centres, x_i +- hx_i / 2, by both slopes (the van Albada average of equal scaled
    differences is their common value)."""
    M, nx, ny = 4, 10, 8
    hx, hy = stretched_widths(nx, 1.0, 3.0), stretched_widths(ny, 1.0, 2.0)
    xc = np.cumsum(hx) - 0.5 * np.array(hx)
    yc = np.cumsum(hy) - 0.5 * np.array(hy)
    X, Y = np.meshgrid(xc, yc)
    al = multi_indices(M)
    rng = np.random.default_rng(72)
    P0, F0 = random_state(rng, 1, 1, M, amp=0.1)
    gP = rng.uniform(-0.05, 0.05, (2, 4))
    gP[:, 2] = 0.0
    gF = rng.normal(size=(2, len(al))) * 0.02
    gF[:, al.sum(1) == 1] = 0.0
    gF[:, al[:, 2] % 2 == 1] = 0.0
    P = P0 + X.reshape(-1, 1) * gP[0] + Y.reshape(-1, 1) * gP[1]
    F = F0 + X.reshape(-1, 1) * gF[0] + Y.reshape(-1, 1) * gF[1]
    for slope in (1, 2):
        S = oracle_solver(lid_cavity(nx, M, 0.1, 0.2, order=2, slope=slope).replace(ny=ny, hx=hx, hy=hy))
        S.set_state(0, P, F)
        for j in range(1, ny - 1):
            for i in range(1, nx - 1):
                c = j * nx + i
                for ax, h in ((0, hx[i]), (1, hy[j])):
                    for sd in (1, -1):
                        p, f = S.face_state(0, i, j, ax, sd)
                        _close(p, P[c] + sd * 0.5 * h * gP[ax], 1e-13, 1e-15, f"params {slope, i, j, ax, sd}")
                        _close(f, F[c] + sd * 0.5 * h * gF[ax], 1e-13, 1e-15, f"coeffs {slope, i, j, ax, sd}")


def check_restriction_conserves_area_weighted_totals():
    prob = stretched(lid_cavity(16, 5, 0.1, 0.3, levels=2).replace(ny=12), ratio=3.0)
    S = oracle_solver(prob)
    rng = np.random.default_rng(73)
    P, F = random_state(rng, 12, 16, 5, amp=0.1)
    S.set_state(1, P, F)
    S.two_grid_setup(1)
    Pc, Fc = S.get_state(0)
    hx, hy = np.array(prob.hx), np.array(prob.hy)
    hxc, hyc = hx.reshape(-1, 2).sum(1), hy.reshape(-1, 2).sum(1)

    def totals(P, F, area):
        rho = F[:, 0] * area
        return np.array([rho.sum(), *(rho[:, None] * P[:, :3]).sum(0),
                         (rho * (P[:, :3] ** 2).sum(1) + 3 * rho * P[:, 3]).sum()])

    _close(totals(Pc, Fc, np.outer(hyc, hxc).ravel()), totals(P, F, np.outer(hy, hx).ravel()), 1e-13, 1e-15)


def check_stretched_grid_solution_matches_the_uniform_one():
    """The FAS cycle converges on a stretched grid, keeps the mass, and its flow agrees with the
    uniform grid's to the discretization error (vertical centre-line velocity, both grids
    interpolated to the same heights)."""
    base = lid_cavity(32, 4, 0.1, 0.2, levels=3)
    res = {}
    for name, prob in (("uniform", base), ("stretched", stretched(base, ratio=2.5))):
        S = oracle_solver(prob)
        m0 = S.mass()
        st, cyc, rel = S.solve(1e-8, 100)
        assert st == oracle.OK and rel <= 1e-8, (name, st, cyc, rel)
        assert abs(S.mass() - m0) <= 1e-13
        f = S.fields()
        hx = np.array(prob.hx) if prob.hx else np.full(32, 1 / 32)
        hy = np.array(prob.hy) if prob.hy else np.full(32, 1 / 32)
        xc, yc = np.cumsum(hx) - hx / 2, np.cumsum(hy) - hy / 2
        # u1 on the vertical line x = 1/2: linear in x between the two cells around it
        k = np.searchsorted(xc, 0.5)
        t = (0.5 - xc[k - 1]) / (xc[k] - xc[k - 1])
        u = (1 - t) * f[:, k - 1, 1] + t * f[:, k, 1]
        res[name] = np.interp(np.linspace(0.1, 0.9, 9), yc, u)
    assert np.abs(res["stretched"] - res["uniform"]).max() <= 0.02 * 0.2, res


CHECKS = [check_explicit_uniform_widths_equal_the_uniform_grid, check_maxwellian_is_a_fixed_point_on_a_stretched_grid,
          check_residual_conserves_mass_on_a_stretched_grid, check_face_states_of_affine_fields_on_a_stretched_grid,
          check_restriction_conserves_area_weighted_totals, check_stretched_grid_solution_matches_the_uniform_one]


def test_explicit_uniform_widths_equal_the_uniform_grid():
    check_explicit_uniform_widths_equal_the_uniform_grid()


def test_maxwellian_is_a_fixed_point_on_a_stretched_grid():
    check_maxwellian_is_a_fixed_point_on_a_stretched_grid()


def test_residual_conserves_mass_on_a_stretched_grid():
    check_residual_conserves_mass_on_a_stretched_grid()


def test_face_states_of_affine_fields_on_a_stretched_grid():
    check_face_states_of_affine_fields_on_a_stretched_grid()


def test_restriction_conserves_area_weighted_totals():
    check_restriction_conserves_area_weighted_totals()


def test_stretched_grid_solution_matches_the_uniform_one():
    check_stretched_grid_solution_matches_the_uniform_one()
