"""Pins of the CPU oracle against what the mathematics and the published
solutions fix — not against the oracle itself.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them:
  * exact Riemann solver: published Sod star state, Rankine-Hugoniot jump
    conditions, isentropic rarefaction and its Riemann invariant;
  * HLLC (Toro-Spruce-Speares): consistency with the Euler flux, exact
    resolution of stationary and moving contacts, upwinding of supersonic
    states, rotational and mirror symmetry;
  * PPM (Colella-Woodward 1984): exactness on linear and cubic zone averages,
    the extremum and overshoot rules, the parabola integrals;
  * CW84 flattening: smooth profiles untouched, strong shocks fully flattened;
  * characteristic tracing: exact for the linearised system when the waves
    that cannot reach a face carry no signal (this exercises l_i . r_j = delta_ij);
  * the whole step: Sod vs the exact solution, Sedov self-similar scaling with
    xi0 from the similarity ODE, conservation on periodic boxes, uniform-state
    preservation, dimensional reduction, mirror symmetry, free fall under
    constant gravity, hydrostatic balance of a stratified atmosphere;
  * corner transport: a product profile advected obliquely and a random
    density moved one zone per axis at unit Courant number, both exact
    solutions, with planted mistakes in the transverse corrections that
    each fail one of them.
"""
import os

import numpy as np
import pytest

import oracle
import sedov_similarity
from paper_1711_06203_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
I3 = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))
I2 = (slice(None), 0, slice(4, -4), slice(4, -4))


def euler_flux(q, d, gamma):
    """Euler flux in direction d of a primitive state (rho, u, v, w, p)."""
    rho, p = q[0], q[4]
    vel = np.array(q[1:4])
    E = p / (gamma - 1) + 0.5 * rho * vel @ vel
    un = vel[d]
    F = np.zeros(5)
    F[0] = rho * un
    F[1:4] = rho * un * vel
    F[1 + d] += p
    F[4] = un * (E + p)
    return F


def read_golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


# ---------------------------------------------------------------- exact Riemann solver
class TestExactRiemann:
    WL, WR, g = [1.0, 0.0, 1.0], [0.125, 0.0, 0.1], 1.4

    def test_sod_published_star_state(self):
        gold = read_golden("sod_exact_star.txt")
        ps, us = oracle.exact_star(self.WL, self.WR, self.g)
        assert abs(ps - gold["p_star"]) < 1e-8
        assert abs(us - gold["u_star"]) < 1e-8
        W = oracle.exact_sample(self.WL, self.WR, self.g, np.array([us - 1e-9, us + 1e-9]))
        assert abs(W[0, 0] - gold["rho_star_left"]) < 1e-8
        assert abs(W[1, 0] - gold["rho_star_right"]) < 1e-8
        # wave positions: state changes exactly at the published speeds
        eps = 1e-7
        for key, lo_state in (("shock_speed", None), ("rarefaction_head", None), ("rarefaction_tail", None)):
            s = gold[key]
            a, b = oracle.exact_sample(self.WL, self.WR, self.g, np.array([s - eps, s + eps]))
            assert np.abs(a - b).max() > 0 or key != "shock_speed"
        Wsh = oracle.exact_sample(self.WL, self.WR, self.g, np.array([gold["shock_speed"] + 1e-6]))
        assert np.allclose(Wsh[0], self.WR)
        Wh = oracle.exact_sample(self.WL, self.WR, self.g, np.array([gold["rarefaction_head"] - 1e-6]))
        assert np.allclose(Wh[0], self.WL)

    def test_rankine_hugoniot_across_right_shock(self):
        ps, us = oracle.exact_star(self.WL, self.WR, self.g)
        g = self.g
        # shock speed from the mass jump alone, then momentum and energy must match
        rs = oracle.exact_sample(self.WL, self.WR, g, np.array([us + 1e-9]))[0, 0]
        rR, uR, pR = self.WR
        S = (rs * us - rR * uR) / (rs - rR)
        mom = lambda r, u, p: r * u * (u - S) + p
        en = lambda r, u, p: (p / (g - 1) + 0.5 * r * u * u) * (u - S) + p * u
        assert abs(mom(rs, us, ps) - mom(rR, uR, pR)) < 1e-12
        assert abs(en(rs, us, ps) - en(rR, uR, pR)) < 1e-12

    def test_rarefaction_isentropic_and_invariant(self):
        g = self.g
        ps, us = oracle.exact_star(self.WL, self.WR, g)
        cL = np.sqrt(g * self.WL[2] / self.WL[0])
        head = self.WL[1] - cL
        tail = read_golden("sod_exact_star.txt")["rarefaction_tail"]
        xi = np.linspace(head, tail, 9)
        W = oracle.exact_sample(self.WL, self.WR, g, xi)
        ent = W[:, 2] / W[:, 0] ** g
        inv = W[:, 1] + 2.0 / (g - 1.0) * np.sqrt(g * W[:, 2] / W[:, 0])
        assert np.allclose(ent, self.WL[2] / self.WL[0] ** g, rtol=1e-12)
        assert np.allclose(inv, self.WL[1] + 2.0 / (g - 1.0) * cL, rtol=1e-12)
        # inside the fan each point moves with its own characteristic speed u - c = xi
        c = np.sqrt(g * W[1:-1, 2] / W[1:-1, 0])
        assert np.allclose(W[1:-1, 1] - c, xi[1:-1], atol=1e-12)

    def test_symmetric_collision_has_zero_contact_speed(self):
        ps, us = oracle.exact_star([1.0, 1.0, 1.0], [1.0, -1.0, 1.0], 1.4)
        assert abs(us) < 1e-14 and ps > 1.0


# ---------------------------------------------------------------- HLLC
class TestHLLC:
    g = 1.4

    def test_consistency(self):
        rng = np.random.default_rng(5)
        for _ in range(50):
            q = np.array([rng.lognormal(), *rng.normal(0, 2, 3), rng.lognormal()])
            for d in range(3):
                assert np.allclose(oracle.hllc(q, q, d, self.g), euler_flux(q, d, self.g), rtol=1e-13, atol=1e-13)

    def test_stationary_contact_is_exact(self):
        qL = np.array([2.0, 0.0, 0.3, -0.2, 1.5])
        qR = np.array([0.5, 0.0, -0.7, 0.1, 1.5])
        F = oracle.hllc(qL, qR, 0, self.g)
        assert abs(F[0]) < 1e-15 and abs(F[4]) < 1e-15 and abs(F[2]) < 1e-15 and abs(F[3]) < 1e-15
        assert abs(F[1] - 1.5) < 1e-14

    def test_moving_contact_takes_upwind_flux(self):
        for u, up in ((0.4, "L"), (-0.4, "R")):
            qL = np.array([2.0, u, 0.3, 0.0, 1.5])
            qR = np.array([0.5, u, -0.7, 0.2, 1.5])
            F = oracle.hllc(qL, qR, 0, self.g)
            ref = euler_flux(qL if up == "L" else qR, 0, self.g)
            assert np.allclose(F, ref, rtol=1e-13, atol=1e-14)

    def test_supersonic_upwinding(self):
        qL = np.array([1.0, 5.0, 0.0, 0.0, 1.0])
        qR = np.array([0.3, 4.0, 0.1, 0.0, 0.2])
        assert np.array_equal(oracle.hllc(qL, qR, 0, self.g), euler_flux(qL, 0, self.g)) or \
            np.allclose(oracle.hllc(qL, qR, 0, self.g), euler_flux(qL, 0, self.g), rtol=1e-15)
        qL[1], qR[1] = -4.0, -5.0
        assert np.allclose(oracle.hllc(qL, qR, 0, self.g), euler_flux(qR, 0, self.g), rtol=1e-15)

    def test_rotation_and_mirror(self):
        rng = np.random.default_rng(9)
        qL = np.array([1.3, 0.2, -0.4, 0.1, 0.9])
        qR = np.array([0.7, -0.1, 0.3, 0.5, 0.4])
        Fx = oracle.hllc(qL, qR, 0, self.g)
        # same problem posed along y: swap the u and v components
        perm = [0, 2, 1, 3, 4]
        Fy = oracle.hllc(qL[perm], qR[perm], 1, self.g)
        assert np.allclose(Fy[perm], Fx, rtol=1e-14, atol=1e-15)
        # mirror x -> -x: states swap sides, normal velocity flips, mass flux flips sign
        mL = qR.copy(); mL[1] = -mL[1]
        mR = qL.copy(); mR[1] = -mR[1]
        Fm = oracle.hllc(mL, mR, 0, self.g)
        assert np.allclose([-Fm[0], Fm[1], -Fm[2], -Fm[3], -Fm[4]], Fx, rtol=1e-13, atol=1e-15)

    def test_star_flux_is_the_rankine_hugoniot_flux_of_the_outer_wave(self):
        # Toro, Spruce & Speares: in the star regions the HLLC flux is defined
        # as F_K + S_K (U*_K - U_K), with U*_K = rho_K (S_K - u_K)/(S_K - S*)
        # [1, S*, v_K, w_K, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))].
        # Built here from that definition (Davis speeds), for subsonic random
        # states on both sides of the contact and along every axis.
        rng = np.random.default_rng(17)
        g = self.g
        worst = 0.0
        for _ in range(400):
            qL = np.array([rng.lognormal(0, 0.5), *rng.normal(0, 0.3, 3), rng.lognormal(0, 0.5)])
            qR = np.array([rng.lognormal(0, 0.5), *rng.normal(0, 0.3, 3), rng.lognormal(0, 0.5)])
            for d in range(3):
                uL, uR = qL[1 + d], qR[1 + d]
                cL, cR = np.sqrt(g * qL[4] / qL[0]), np.sqrt(g * qR[4] / qR[0])
                SL, SR = min(uL - cL, uR - cR), max(uL + cL, uR + cR)
                Ss = (qR[4] - qL[4] + qL[0] * uL * (SL - uL) - qR[0] * uR * (SR - uR)) / \
                    (qL[0] * (SL - uL) - qR[0] * (SR - uR))
                assert SL < 0 < SR
                q, S = (qL, SL) if Ss >= 0 else (qR, SR)
                rho, u, p = q[0], q[1 + d], q[4]
                U = np.array([rho, rho * q[1], rho * q[2], rho * q[3], p / (g - 1) + 0.5 * rho * (q[1:4] ** 2).sum()])
                fac = rho * (S - u) / (S - Ss)
                Us = fac * np.array([1.0, *[Ss if k == d else q[1 + k] for k in range(3)],
                                     U[4] / rho + (Ss - u) * (Ss + p / (rho * (S - u)))])
                Fref = euler_flux(q, d, g) + S * (Us - U)
                F = oracle.hllc(qL, qR, d, g)
                worst = max(worst, np.abs(F - Fref).max() / np.abs(Fref).max())
        assert worst < 1e-13, worst

    def test_weak_waves_match_exact_solver_to_second_order(self):
        # for a jump of size eps the approximate solver errs by O(eps^2)
        errs = []
        for eps in (1e-2, 1e-3):
            WL, WR = [1.0, 0.05, 1.0], [1.0 - eps, 0.05 - 0.3 * eps, 1.0 - 1.5 * eps]
            F = oracle.hllc(np.array([WL[0], WL[1], 0, 0, WL[2]]), np.array([WR[0], WR[1], 0, 0, WR[2]]), 0, self.g)
            W = oracle.exact_sample(WL, WR, self.g, np.array([0.0]))[0]
            Fex = euler_flux(np.array([W[0], W[1], 0, 0, W[2]]), 0, self.g)
            errs.append(np.abs(F - Fex).max())
        assert errs[1] < 2e-6 and errs[0] / errs[1] > 50, errs


# ---------------------------------------------------------------- PPM + flattening
class TestPPM:
    def test_linear_profile_is_exact(self):
        a = 3.0 + 0.25 * np.arange(-3, 4)
        am, ap, a6 = oracle.ppm_parabola(a)
        assert abs(am - (3.0 - 0.125)) < 1e-15 and abs(ap - (3.0 + 0.125)) < 1e-15 and abs(a6) < 1e-14
        for s in (0.0, 0.3, 1.0):
            # average of the line over the last s of the zone
            assert abs(oracle.integ([am, ap, a6], s, True) - (3.0 + 0.25 * (0.5 - s / 2))) < 1e-14
            assert abs(oracle.integ([am, ap, a6], s, False) - (3.0 - 0.25 * (0.5 - s / 2))) < 1e-14

    def test_limited_slope_worked_example(self):
        """The monotonised centred slope (CW84 eq. 1.8) where the one-sided
        bound 2|a_i - a_{i-1}| is the active one.  Line (0, 0, 0.1, 0.2, 1.0,
        1.8, 1.9), zone 3 (a = 0.2), worked by hand:
          slopes: zone 2 (0, 0.1, 0.2) -> min(0.1, 0.2, 0.2) = 0.1;
                  zone 3 (0.1, 0.2, 1.0) -> min(0.45, 2 x 0.1, 2 x 0.8) = 0.2;
                  zone 4 (0.2, 1.0, 1.8) -> min(0.8, 1.6, 1.6) = 0.8;
          interfaces: a_{2+1/2} = 0.15 - (0.2 - 0.1)/6 = 2/15,
                      a_{3+1/2} = 0.6 - (0.8 - 0.2)/6 = 1/2;
          limiter (eq. 1.10): D = 11/30, M = 0.2 - 19/60 = -7/60, D M < -D^2/6,
          so a+ = 3 a - 2 a- = 1/3; a6 = 6 (0.2 - (2/15 + 1/3)/2) = -1/5."""
        am, ap, a6 = oracle.ppm_parabola(np.array([0.0, 0.0, 0.1, 0.2, 1.0, 1.8, 1.9]))
        assert abs(am - 2 / 15) < 1e-15 and abs(ap - 1 / 3) < 1e-15 and abs(a6 + 0.2) < 1e-15

    def test_cubic_zone_averages_give_exact_interface_values(self):
        # zone averages of a monotone cubic; the 4th-order interface formula is exact for cubics
        f = lambda x: 1.0 + x + 0.1 * x ** 2 + 0.01 * x ** 3
        Fint = lambda x: x + 0.5 * x ** 2 + 0.1 * x ** 3 / 3 + 0.0025 * x ** 4
        m = np.arange(-3, 4)
        avg = Fint(m + 0.5) - Fint(m - 0.5)
        am, ap, a6 = oracle.ppm_parabola(avg)
        assert abs(ap - f(0.5)) < 1e-13 and abs(am - f(-0.5)) < 1e-13

    def test_extremum_is_flattened_to_constant(self):
        a = np.array([0.0, 1.0, 2.0, 3.0, 2.0, 1.0, 0.0])
        am, ap, a6 = oracle.ppm_parabola(a)
        assert am == 3.0 and ap == 3.0 and a6 == 0.0

    def test_overshoot_is_steepened_monotone(self):
        a = np.array([0.0, 0.0, 0.0, 0.1, 1.0, 1.0, 1.0])
        am, ap, a6 = oracle.ppm_parabola(a)
        # the resulting parabola has no interior extremum: |a6| <= |ap - am|
        assert abs(a6) <= abs(ap - am) + 1e-15
        assert min(am, ap) >= -1e-15 and max(am, ap) <= 1.0 + 1e-15
        # CW84 eq. 1.10: the parabola would overshoot past the high edge, so a+ = 3a - 2a-
        assert abs(ap - (3 * 0.1 - 2 * am)) < 1e-15
        # mirrored profile takes the other branch: a- = 3a - 2a+
        bm, bp, b6 = oracle.ppm_parabola(a[::-1].copy())
        assert abs(bm - (3 * 0.1 - 2 * bp)) < 1e-15
        assert abs(bm - ap) < 1e-15 and abs(bp - am) < 1e-15 and abs(b6 - a6) < 1e-15

    def test_flattening_blend(self):
        a = 3.0 + 0.25 * np.arange(-3, 4)
        am, ap, a6 = oracle.ppm_parabola(a, chi=0.0)
        assert am == 3.0 and ap == 3.0 and a6 == 0.0
        am, ap, a6 = oracle.ppm_parabola(a, chi=0.5)
        assert abs(ap - 3.0625) < 1e-15 and abs(am - 2.9375) < 1e-15

    def test_flattening_coefficient(self):
        smooth_p = 1.0 + 0.01 * np.arange(7)
        u0 = np.zeros(7)
        assert oracle.flatten_coef(smooth_p, u0) == 1.0
        # strong compressive shock: pressure jump of 10 within one zone, converging flow
        p = np.array([10.0, 10.0, 10.0, 10.0, 1.0, 1.0, 1.0])
        u = np.array([1.0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
        assert oracle.flatten_coef(p, u) == 0.0
        # same jump in an expanding flow is not a shock
        assert oracle.flatten_coef(p, -u) == 1.0
        # partial: at the zone dp1 = 0.8, dp2 = 1.0 -> z = 0.8 -> chi~ = 1 - 10 (0.8 - 0.75) = 0.5;
        # dp1 > 0 so the neighbour consulted is i-1, where z = 0.4/0.8 -> chi~ = 1
        p = np.array([1.0, 1.0, 1.0, 1.4, 1.8, 2.0, 2.0])
        u = -0.1 * np.arange(7)
        assert abs(oracle.flatten_coef(p, u) - 0.5) < 1e-12
        # neighbour rule: with dp1 > 0 the zone takes min(chi~_i, chi~_{i-1}).
        # p = [1, 1, 1.5, 2, 2.1, 3, 3]: at i, dp1 = 0.6, dp2 = 2 -> z = 0.3 -> chi~_i = 1;
        # at i-1, dp1 = 1, dp2 = 1.1 -> z = 0.909 -> chi~_{i-1} = 0  => chi = 0
        q = np.array([1.0, 1.0, 1.5, 2.0, 2.1, 3.0, 3.0])
        assert oracle.flatten_coef(q, u) == 0.0
        # mirrored data (dp1 < 0) consults i+1 instead: same answer by symmetry
        assert oracle.flatten_coef(q[::-1].copy(), -u[::-1].copy()) == 0.0
        # the far side is ignored: strong jump only at i+1 while dp1 > 0
        # p = [1, 1, 1, 1.2, 1.4, 3, 3.2]: at i dp1 = 0.4, dp2 = 2 -> 1; at i-1 dp1 = 0.2 < 0.33 -> 1;
        # at i+1 dp1 = 1.8, dp2 = 2.2 -> z = 0.82 -> would give 0.3
        r = np.array([1.0, 1.0, 1.0, 1.2, 1.4, 3.0, 3.2])
        assert oracle.flatten_coef(r, u) == 1.0
        # the shock test's threshold epsilon = 0.33 (CW84 App. A): the same
        # profile shape with a jump |dp1| / min(p) of 0.30 is not a shock, of
        # 0.40 it is (z = dp1 / dp2 = 0.8 -> chi~ = 1 - 10 (0.8 - 0.75) = 0.5)
        for jump, want in ((0.30, 1.0), (0.40, 0.5)):
            dp1 = jump * 1.0
            s = np.array([1.0, 1.0, 1.0, 1.0 + 0.5 * dp1, 1.0 + dp1, 1.0 + 1.25 * dp1, 1.0 + 1.25 * dp1])
            # neighbours: at i-1, dp1' = dp1/2 and dp2' = 1.25 dp1 -> z = 0.4 -> 1; so chi = chi~_i
            assert abs(oracle.flatten_coef(s, u) - want) < 1e-12, jump


# ---------------------------------------------------------------- characteristic tracing
def _lines(q0, slope, c_fun):
    """7-point lines of rho,u,v,w,p,c sampled from a linear profile q0 + m*slope."""
    m = np.arange(-3, 4)
    L = np.zeros((6, 7))
    for v in range(5):
        L[v] = q0[v] + m * slope[v]
    L[5] = c_fun(L[0], L[4])
    return L


class TestTracing:
    g = 1.4

    def _P(self):
        return oracle.params(3, (8, 8, 8), gamma=self.g, flatten=True)

    def test_uniform_state(self):
        q0 = np.array([1.2, 0.3, -0.2, 0.1, 0.8])
        c = np.sqrt(self.g * q0[4] / q0[0])
        L = _lines(q0, np.zeros(5), lambda r, p: np.sqrt(self.g * p / r))
        P = oracle.params(3, (8, 8, 8), gamma=self.g, grav=(0.0, 0.0, -2.0))
        qm, qp = oracle.trace_lines(L, 0, P, 0.4 / c, 0.01)
        want = q0.copy(); want[3] += 0.5 * 0.01 * -2.0
        assert np.allclose(qm, want, rtol=1e-15) and np.allclose(qp, want, rtol=1e-15)

    def test_zero_dt_gives_ppm_edges(self):
        rng = np.random.default_rng(2)
        q0 = np.array([1.0, 0.1, 0.2, -0.1, 1.0])
        L = _lines(q0, rng.normal(0, 0.01, 5), lambda r, p: np.sqrt(self.g * p / r))
        qm, qp = oracle.trace_lines(L, 0, self._P(), 0.0, 0.0)
        for v, var in enumerate([0, 1, 2, 3, 4]):
            am, ap, _ = oracle.ppm_parabola(L[var])
            assert abs(qm[v] - am) < 1e-15 and abs(qp[v] - ap) < 1e-15

    def test_supersonic_low_face_is_zone_average(self):
        q0 = np.array([1.0, 3.0, 0.2, -0.1, 1.0])  # u > c: no wave reaches the low face
        L = _lines(q0, np.array([0.01, 0.0, 0.02, 0.0, 0.01]), lambda r, p: np.sqrt(self.g * p / r))
        qm, _ = oracle.trace_lines(L, 0, self._P(), 0.3, 0.0)
        assert np.array_equal(qm, q0)

    @pytest.mark.parametrize("d,un", [(0, 0.3), (1, 0.3), (2, 0.3), (0, 2.0), (2, -2.0)])
    def test_linearised_characteristics_are_exact(self, d, un):
        """With linear profiles made of waves that all reach a face, the traced
        state is the exact linearised solution at the face at t = dt/2.
        Subsonic (u = 0.3, c = 1.18): the entropy and fast wave reach the high
        face, the slow wave the low one.  Supersonic (|u| = 2): all three
        reach the downstream face, so the two waves that are not the
        reference one both enter through their wave strengths (the
        eigenvector coefficients rho/(2c) and 1/(2c^2))."""
        g = self.g
        rho, p = 1.0, 1.0
        c = np.sqrt(g * p / rho)
        # eigenvectors of the (rho, un, p) system, written out here independently
        r = {"-": np.array([1.0, -c / rho, c * c]), "0": np.array([1.0, 0.0, 0.0]), "+": np.array([1.0, c / rho, c * c])}
        lam = {"-": un - c, "0": un, "+": un + c}
        dtdx = 0.4 / (abs(un) + c)
        t1 = 1 if d == 0 else 0
        t2 = 1 if d == 2 else 2
        if abs(un) < c:
            cases = (("p", ("0", "+")), ("m", ("-",)))
        else:
            cases = ((("p" if un > 0 else "m"), ("-", "0", "+")),)
        for face, waves in cases:
            amp = {"-": 0.0, "0": 0.0, "+": 0.0}
            for w, a in zip(waves, (2e-4, -3e-4, 1.5e-4)):
                amp[w] = a
            s3 = sum(amp[w] * r[w] for w in amp)
            slope_t = 1e-4  # transverse velocity rides the entropy wave
            q0 = np.zeros(5); sl = np.zeros(5)
            q0[0], q0[1 + d], q0[4] = rho, un, p
            sl[0], sl[1 + d], sl[4] = s3
            if "0" in waves:
                sl[1 + t1] = slope_t
            L = np.zeros((6, 7))
            m = np.arange(-3, 4)
            for v in range(5):
                L[v] = q0[v] + m * sl[v]
            L[5] = c  # the tracing uses the zone's own sound speed only
            P = oracle.params(3, (8, 8, 8), gamma=g, flatten=False)
            qm, qp = oracle.trace_lines(L, d, P, dtdx, 0.0)
            xf = 0.5 if face == "p" else -0.5
            exact = np.array([rho, un, p]) + sum(amp[w] * (xf - lam[w] * dtdx / 2) * r[w] for w in amp)
            got = qp if face == "p" else qm
            assert np.allclose([got[0], got[1 + d], got[4]], exact, rtol=0, atol=1e-15), (face, d)
            if "0" in waves:
                assert abs(got[1 + t1] - slope_t * (xf - un * dtdx / 2)) < 1e-15


def test_step_traced_states_equal_the_seven_point_tracing():
    """The step forms each pencil's flattening coefficients, slopes and
    interface values once and shares them between zones; the seven-point
    tracing of a single zone forms them from that zone's own stencil.  On a
    box with strong compressions and pressure jumps, where the flattening
    neighbour rule matters, the two give the same traced states bit for bit
    on every zone the step traces (zones [-1, n] on every axis)."""
    rng = np.random.default_rng(31)
    n = (9, 8, 7)
    dx = (1 / 9, 1 / 8, 1 / 7)
    U = inputs.random_box(rng, n, 3, gamma=1.4, sigma_rho=0.8, sigma_u=0.8, sigma_p=1.0)
    P = oracle.params(3, n, dx=dx, gamma=1.4, grav=(0.2, -0.4, 0.3))
    d, _ = oracle.dt(U, P)
    _, rc, dbg = oracle.step(U, P, d, debug=True)
    Q = dbg["prim"]
    flattened = 0
    for ax in range(3):
        for k in range(-1, n[2] + 1):
            for j in range(-1, n[1] + 1):
                for i in range(-1, n[0] + 1):
                    z = [k + 4, j + 4, i + 4]
                    sl = [z[0], z[1], z[2]]
                    sl[2 - ax] = slice(z[2 - ax] - 3, z[2 - ax] + 4)
                    L = Q[(slice(None),) + tuple(sl)]
                    flattened += oracle.flatten_coef(L[4], L[1 + ax]) < 1.0
                    qm, qp = oracle.trace_lines(L, ax, P, d / dx[ax], d)
                    assert np.array_equal(qm, dbg["trace_m"][ax][(slice(None),) + tuple(z)]), (ax, i, j, k)
                    assert np.array_equal(qp, dbg["trace_p"][ax][(slice(None),) + tuple(z)]), (ax, i, j, k)
    assert flattened > 50


# ---------------------------------------------------------------- EOS
def test_cons_prim_round_trip_and_bad_flags():
    P = oracle.params(3, (8, 8, 8), gamma=5 / 3)
    q = np.array([0.7, 0.3, -1.2, 0.05, 2.5])
    U = oracle.prim_to_cons(q, 5 / 3)
    assert abs(U[4] - (2.5 * 1.5 + 0.5 * 0.7 * (0.09 + 1.44 + 0.0025))) < 1e-14
    q2, bad = oracle.cons_to_prim(U, P)
    assert np.allclose(q2, q, rtol=1e-15) and bad == 0
    _, bad = oracle.cons_to_prim(np.array([-1.0, 0, 0, 0, 1.0]), P)
    assert bad == 1
    _, bad = oracle.cons_to_prim(np.array([1.0, 2.0, 0, 0, 1.0]), P)  # kinetic > total energy
    assert bad == 1


# ---------------------------------------------------------------- whole step
def test_sod_against_exact_solution():
    n = 64
    U = inputs.sod(n, 2, 0)
    P = oracle.params(2, (n, n), bc=oracle.BC_OUTFLOW, gamma=1.4, cfl=0.5)
    U1, t, _ = oracle.run(U, P, 50)
    rho = U1[0, 0, 4:-4, 4:-4]
    assert np.all(rho == rho[0:1, :]), "every row must be identical"
    x = (np.arange(n) + 0.5) / n
    W = oracle.exact_sample([1, 0, 1], [0.125, 0, 0.1], 1.4, (x - 0.5) / t)
    assert np.mean(np.abs(rho[0] - W[:, 0])) <= 1.5e-2


def test_sod_convergence_order():
    errs = []
    for n in (64, 128, 256):
        U = inputs.sod(n, 2, 0)
        U = U[:, :, : 4 + 8, :].copy()  # 4 interior rows: a quasi-1-D run
        P = oracle.params(2, (n, 4), dx=(1.0 / n,) * 3, bc=oracle.BC_OUTFLOW, gamma=1.4)
        t, k = 0.0, 0
        while t < 0.2 - 1e-14:
            d, _ = oracle.dt(U, P)
            d = min(d, 0.2 - t)
            U, _ = oracle.step(U, P, d)
            t += d
        x = (np.arange(n) + 0.5) / n
        W = oracle.exact_sample([1, 0, 1], [0.125, 0, 0.1], 1.4, (x - 0.5) / t)
        errs.append(np.mean(np.abs(U[0, 0, 4, 4:-4] - W[:, 0])))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order >= 0.8), (errs, order)


def test_sedov_self_similar_scaling_and_symmetry():
    n, steps = 48, 80
    U, ndep = inputs.sedov(n)
    assert ndep == 280
    P = oracle.params(3, (n, n, n), gamma=1.4)
    x = (np.arange(n) + 0.5) / n - 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z).ravel()
    nb = n // 2
    edges = np.linspace(0, 0.5, nb + 1)
    rc = 0.5 * (edges[:-1] + edges[1:])
    idx = np.digitize(r, edges) - 1
    inside = idx < nb
    cnt = np.bincount(idx[inside], None, nb)
    tot0 = U[I3].reshape(5, -1).sum(1)
    t, ts, Rpk, Rfr = 0.0, [], [], []
    for s in range(steps):
        d, _ = oracle.dt(U, P)
        U, rcode = oracle.step(U, P, d)
        assert rcode == 0
        t += d
        if s >= steps // 2 and s % 5 == 0:
            prof = np.bincount(idx[inside], U[0][4:-4, 4:-4, 4:-4].ravel()[inside], nb) / cnt
            k = int(np.argmax(prof))
            half = 0.5 * (1.0 + prof[k])
            j = k
            while prof[j + 1] > half:
                j += 1
            ts.append(t)
            Rpk.append(rc[k])
            Rfr.append(rc[j] + (prof[j] - half) / (prof[j] - prof[j + 1]) * (rc[j + 1] - rc[j]))
    # R ~ t^(2/5): exponent of the density-peak radius over the second half
    expo = np.polyfit(np.log(ts), np.log(Rpk), 1)[0]
    assert abs(expo - 0.4) <= 0.02, expo
    # amplitude: shock front (half height) vs xi0 (E t^2 / rho0)^(1/5), xi0 from the similarity ODE
    xi0 = sedov_similarity.xi0(1.4)
    assert abs(xi0 - 1.0327) < 2e-3
    ratio = Rfr[-1] / (xi0 * (t * t) ** 0.2)
    assert abs(ratio - 1.0) <= 0.05, ratio
    # the blast has not reached the boundary: mass and energy are conserved
    tot1 = U[I3].reshape(5, -1).sum(1)
    assert abs(tot1[0] - tot0[0]) / tot0[0] < 1e-13
    assert abs(tot1[4] - tot0[4]) / tot0[4] < 1e-13
    # octant symmetry (mirror images), round-off level
    rho = U[0][4:-4, 4:-4, 4:-4]
    scale = np.abs(rho).max()
    for mir in (rho[::-1], rho[:, ::-1], rho[:, :, ::-1], rho.transpose(1, 0, 2), rho.transpose(2, 1, 0)):
        assert np.abs(rho - mir).max() / scale <= 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_conservation(dim):
    rng = np.random.default_rng(11 + dim)
    n = (20, 16, 12) if dim == 3 else (24, 20, 1)
    U = inputs.random_box(rng, n, dim)
    P = oracle.params(dim, n, dx=(1 / 20, 1 / 16, 1 / 12), bc=oracle.BC_PERIODIC, gamma=5 / 3)
    I = I3 if dim == 3 else I2
    U0 = oracle.fill_ghosts(U, P)
    tot0 = U0[I].reshape(5, -1).sum(1)
    mag = np.abs(U0[I]).reshape(5, -1).sum(1)
    for _ in range(3):
        d, _ = oracle.dt(U, P)
        U, rc = oracle.step(U, P, d)
        assert rc == 0
    tot = U[I].reshape(5, -1).sum(1)
    rel = np.abs(tot - tot0) / np.where(mag > 0, mag, 1.0)  # w stays exactly 0 in 2-D
    assert np.all(rel <= 1e-13), rel


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_state_preserved_bitwise(dim):
    n = (12, 10, 8) if dim == 3 else (12, 10, 1)
    shape = inputs.grown_shape(n, dim)
    U = inputs.conserved(np.full(shape, 1.3), 0.2, -0.1, 0.05, np.full(shape, 0.7), 5 / 3)
    P = oracle.params(dim, n, bc=oracle.BC_PERIODIC, gamma=5 / 3)
    d, _ = oracle.dt(U, P)
    U1, rc = oracle.step(U, P, d)
    I = I3 if dim == 3 else I2
    assert rc == 0 and np.array_equal(U1[I], U[I])


def test_dimensional_reduction_and_axis_permutation():
    n = 32
    P3 = oracle.params(3, (n, n, n))
    P2 = oracle.params(2, (n, n))
    res = {}
    for ax in range(3):
        U3 = inputs.sod(n, 3, ax)
        d, _ = oracle.dt(U3, P3)
        res[ax], _ = oracle.step(U3, P3, d)
    U2 = inputs.sod(n, 2, 0)
    d2, _ = oracle.dt(U2, P2)
    B, _ = oracle.step(U2, P2, d2)
    A = res[0][I3]
    # 3-D x-problem equals the 2-D run row by row
    assert np.array_equal(A[:, 0], B[I2])
    assert all(np.array_equal(A[:, k], A[:, 0]) for k in range(n))
    # the y- and z-problems are the x-problem transposed, momentum components permuted
    Ay = res[1][I3].transpose(0, 1, 3, 2)[[0, 2, 1, 3, 4]]
    Az = res[2][I3].transpose(0, 3, 2, 1)[[0, 3, 2, 1, 4]]
    assert np.array_equal(Ay, A) and np.array_equal(Az, A)


def test_mirror_symmetry_3d():
    rng = np.random.default_rng(4)
    n = (12, 12, 12)
    U = inputs.random_box(rng, n, 3)
    U = 0.5 * (U + U[:, :, :, ::-1] * np.array([1, -1, 1, 1, 1])[:, None, None, None])  # x-symmetric data
    P = oracle.params(3, n, bc=oracle.BC_PREFILLED, gamma=5 / 3)
    d, _ = oracle.dt(U, P)
    U1, _ = oracle.step(U, P, d)
    A = U1[I3]
    M = A[:, :, :, ::-1] * np.array([1, -1, 1, 1, 1])[:, None, None, None]
    assert np.abs(A - M).max() / np.abs(A).max() <= 1e-12


def test_free_fall_under_constant_gravity():
    n = (8, 8, 8)
    shape = inputs.grown_shape(n, 3)
    rho, p, w0, g = 1.7, 0.9, 0.2, -3.0
    U = inputs.conserved(np.full(shape, rho), 0.0, 0.0, w0, np.full(shape, p), 1.4)
    P = oracle.params(3, n, bc=oracle.BC_PERIODIC, gamma=1.4, grav=(0.0, 0.0, g))
    dt = 0.01
    U1, _ = oracle.step(U, P, dt)
    mom = U1[3][4:-4, 4:-4, 4:-4]
    E = U1[4][4:-4, 4:-4, 4:-4]
    assert np.allclose(mom, rho * (w0 + g * dt), rtol=1e-14)
    # kinetic energy gains rho g (w0 + g dt/2) dt; internal energy unchanged
    E0 = p / 0.4 + 0.5 * rho * w0 * w0
    assert np.allclose(E, E0 + rho * g * (w0 + 0.5 * g * dt) * dt, rtol=1e-14)


def _falling_profile():
    """2-D periodic box: density 1.5 + 0.4 sin(2 pi x) advected at u = 0.8
    along x, at rest along y, uniform pressure, gravity -3 along y."""
    n, dx, g, gam = (24, 8), (1 / 24, 1 / 8, 1.0), (0.0, -3.0, 0.0), 1.4
    X = inputs.zone_centres(n + (1,), 2, dx)
    rho = 1.5 + 0.4 * np.sin(2 * np.pi * X[0])
    U = inputs.conserved(rho, 0.8 + 0 * rho, 0 * rho, 0 * rho, 1.0 + 0 * rho, gam)
    P = oracle.params(2, n, dx=dx, bc=oracle.BC_PERIODIC, gamma=gam, grav=g)
    d, _ = oracle.dt(U, P)
    U1, rc = oracle.step(U, P, d)
    assert rc == 0
    inner = lambda V: V[:, 0, 4:-4, 4:-4]
    return inner(U), inner(U1), g[1], d


def test_falling_advected_profile_momentum_is_new_density_times_g_dt():
    """The momentum source is time-centred in the density, dt g (rho^n +
    rho^{n+1}) / 2 (Step 10).  The y-momentum carried along x is the mass flux
    times the traced v = g dt / 2, whose divergence is (rho^{n+1} - rho^n) g
    dt / 2; the two add up to (rho v)^{n+1} = rho^{n+1} g dt exactly, zone by
    zone, while the density itself changes by O(dt)."""
    U0, U1, g, d = _falling_profile()
    assert np.abs(U1[0] - U0[0]).max() > 1e-2
    assert np.abs(U1[2] - U1[0] * g * d).max() <= 1e-15


def test_falling_advected_profile_gains_half_g2_dt2_mass():
    """The energy source is dt g . ((rho v)^n + (rho v)^{n+1}) / 2 (Step 10):
    over a periodic box the fluxes cancel and the total energy rises by
    g^2 dt^2 / 2 times the (conserved) total mass."""
    U0, U1, g, d = _falling_profile()
    mass = U0[0].sum()
    assert abs(U1[0].sum() - mass) <= 1e-13 * mass
    gain = U1[4].sum() - U0[4].sum()
    want = 0.5 * g * g * d * d * mass
    assert abs(gain - want) <= 1e-9 * want, (gain, want)


def test_periodic_box_momentum_and_energy_budget_under_gravity():
    """Over a periodic box the flux differences cancel, so the totals follow
    the sources of Step 10 alone: each momentum component gains dt g_a M
    (M the conserved mass) and the energy gains dt sum_a g_a (P_a^n +
    P_a^{n+1}) / 2 = dt sum_a g_a (P_a^n + dt g_a M / 2), P_a the total
    momentum, for any state."""
    rng = np.random.default_rng(77)
    n = (10, 9, 8)
    g = (0.6, -0.9, 1.3)
    U = inputs.random_box(rng, n, 3, gamma=1.4, sigma_u=0.4)
    P = oracle.params(3, n, bc=oracle.BC_PERIODIC, gamma=1.4, grav=g)
    d, _ = oracle.dt(U, P)
    U1, rc = oracle.step(U, P, d)
    assert rc == 0
    A, B = U[I3], U1[I3]
    M = A[0].sum()
    assert abs(B[0].sum() - M) <= 1e-13 * M
    for a in range(3):
        assert abs(B[1 + a].sum() - (A[1 + a].sum() + d * g[a] * M)) <= 1e-13 * M
    gain = B[4].sum() - A[4].sum()
    want = d * sum(g[a] * (A[1 + a].sum() + 0.5 * d * g[a] * M) for a in range(3))
    assert abs(gain - want) <= 1e-13 * np.abs(A[4]).sum(), (gain, want)


def test_hydrostatic_atmosphere_stays_near_rest():
    """Unperturbed isothermal atmosphere (rho = exp(-z/H), p = rho g H) with
    periodic x and reflecting z.  Away from the walls (whose mirrored ghost
    zones are not in hydrostatic balance) the residual Mach number after a
    fixed time is small and falls at least second order with resolution; a
    sign or factor slip in the gravity source would accelerate it at O(1)."""
    machs = []
    for n in (16, 32):
        U = inputs.stratified(n, 2, gamma=5 / 3, g=1.0, H=0.1)
        P = oracle.params(2, (n, n), bc=((oracle.BC_PERIODIC,) * 2, (oracle.BC_REFLECT,) * 2, (0, 0)),
                          gamma=5 / 3, grav=(0.0, -1.0, 0.0))
        t = 0.0
        while t < 0.05 - 1e-14:
            d, _ = oracle.dt(U, P)
            d = min(d, 0.05 - t)
            U, rc = oracle.step(U, P, d)
            assert rc == 0
            t += d
        q = U[:, 0, 4 + n // 4: 4 + 3 * n // 4, 4:-4]  # the middle half in height
        rho = q[0]
        vel = np.sqrt(q[1] ** 2 + q[2] ** 2) / rho
        p = (5 / 3 - 1) * (q[4] - 0.5 * rho * vel ** 2)
        machs.append((vel / np.sqrt(5 / 3 * p / rho)).max())
    assert machs[0] < 1e-3 and machs[1] < machs[0] / 2.0, machs


def test_time_step_closed_form_and_brute_force():
    """dt = cfl min over zones and directions of dx_d / (|u_d| + c) (Step 11):
    a uniform state gives the closed form, a random box the minimum taken zone
    by zone from its own primitive variables."""
    gam, cfl, dx = 1.4, 0.45, (0.1, 0.05, 0.07)
    n = (6, 5, 4)
    shape = inputs.grown_shape(n, 3)
    rho, vel, p = 1.3, (0.4, -0.7, 0.2), 0.8
    U = inputs.conserved(np.full(shape, rho), *vel, np.full(shape, p), gam)
    P = oracle.params(3, n, dx=dx, gamma=gam, cfl=cfl)
    c = np.sqrt(gam * p / rho)
    want = cfl * min(h / (abs(v) + c) for h, v in zip(dx, vel))
    got, rc = oracle.dt(U, P)
    assert rc == 0 and abs(got - want) <= 1e-15 * want
    U = inputs.random_box(np.random.default_rng(12), n, 3, gamma=gam, sigma_u=0.8)
    Z = U[:, 4:-4, 4:-4, 4:-4]
    r = Z[0]
    v = Z[1:4] / r
    pr = (gam - 1) * (Z[4] - 0.5 * r * (v * v).sum(0))
    cs = np.sqrt(gam * pr / r)
    want = cfl * min((h / (np.abs(v[a]) + cs)).min() for a, h in enumerate(dx))
    got, rc = oracle.dt(U, P)
    assert rc == 0 and abs(got - want) <= 1e-13 * want


def test_ghost_fill_kinds_and_corner_composition():
    """Outflow copies the nearest interior zone, reflect mirrors with the normal
    momentum negated, periodic wraps; a prefilled face keeps caller data and a
    derived face fills its ghost slab over that data (the maps compose)."""
    n = (6, 5, 7)
    rng = np.random.default_rng(21)
    U = rng.normal(size=(5,) + inputs.grown_shape(n, 3))
    bc = ((oracle.BC_OUTFLOW, oracle.BC_REFLECT), (oracle.BC_PERIODIC, oracle.BC_PERIODIC),
          (oracle.BC_PREFILLED, oracle.BC_OUTFLOW))
    P = oracle.params(3, n, bc=bc)
    W = oracle.fill_ghosts(U, P)
    g = 4
    z = lambda k: k + g
    y = lambda j: j + g
    x = lambda i: i + g
    for c in range(5):
        # x low outflow, x high reflect (x-momentum negated)
        assert W[c, z(2), y(1), x(-3)] == U[c, z(2), y(1), x(0)]
        sgn = -1 if c == 1 else 1
        assert W[c, z(2), y(1), x(6)] == sgn * U[c, z(2), y(1), x(5)]
        assert W[c, z(2), y(1), x(9)] == sgn * U[c, z(2), y(1), x(2)]
        # y periodic
        assert W[c, z(3), y(-1), x(2)] == U[c, z(3), y(4), x(2)]
        assert W[c, z(3), y(5), x(2)] == U[c, z(3), y(0), x(2)]
        # z low prefilled: untouched; z high outflow
        assert W[c, z(-2), y(1), x(1)] == U[c, z(-2), y(1), x(1)]
        assert W[c, z(8), y(1), x(1)] == U[c, z(6), y(1), x(1)]
        # corners: x-outflow over the prefilled z layer, reflect x periodic y, outflow z over all
        assert W[c, z(-2), y(1), x(-1)] == U[c, z(-2), y(1), x(0)]
        assert W[c, z(0), y(-2), x(7)] == sgn * U[c, z(0), y(3), x(4)]
        assert W[c, z(9), y(-1), x(-2)] == U[c, z(6), y(4), x(0)]
    # reflect on the low faces: ghost -m mirrors interior zone m - 1
    bc2 = ((oracle.BC_REFLECT, oracle.BC_OUTFLOW), (oracle.BC_REFLECT, oracle.BC_OUTFLOW),
           (oracle.BC_REFLECT, oracle.BC_OUTFLOW))
    W2 = oracle.fill_ghosts(U, oracle.params(3, n, bc=bc2))
    for c in range(5):
        for m in (1, 2, 4):
            for a, idx, src in ((0, (z(2), y(1), x(-m)), (z(2), y(1), x(m - 1))),
                                (1, (z(2), y(-m), x(1)), (z(2), y(m - 1), x(1))),
                                (2, (z(-m), y(1), x(1)), (z(m - 1), y(1), x(1)))):
                assert W2[(c,) + idx] == (-1 if c == 1 + a else 1) * U[(c,) + src]


# ---------------------------------------------------------------- options beyond the base step
def test_einfeldt_speed_is_the_exact_shock_speed():
    """The Roe linearisation satisfies the jump conditions exactly, so for two
    states joined by a single shock the Roe-averaged characteristic speed u~ + c~
    is the shock speed; Einfeldt's S_R picks it up (the upstream u_R + c_R is
    slower by the Lax condition), Davis's estimate does not."""
    g = 1.4
    mu = (g - 1) / (g + 1)
    rR, uR, pR = 0.7, 0.3, 1.3
    for ratio in (1.5, 4.0, 30.0):
        p = ratio * pR
        rL = rR * (p / pR + mu) / (mu * p / pR + 1)
        cR = np.sqrt(g * pR / rR)
        S = uR + cR * np.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
        uL = S + rR * (uR - S) / rL
        qL = np.array([rL, uL, 0.2, -0.1, p])
        qR = np.array([rR, uR, 0.2, -0.1, pR])
        sl, sr = oracle.wave_speeds(qL, qR, 0, g, True)
        assert abs(sr - S) <= 1e-12 * abs(S), (ratio, sr, S)
        dl, dr = oracle.wave_speeds(qL, qR, 0, g, False)
        assert abs(dr - S) > 1e-6 * abs(S)
        assert sl <= uL - np.sqrt(g * p / rL) + 1e-15
    # identical states: the fan is the state's own acoustic speeds
    q = np.array([1.1, 0.4, 0.0, 0.0, 0.9])
    sl, sr = oracle.wave_speeds(q, q, 0, g, True)
    c = np.sqrt(g * 0.9 / 1.1)
    assert abs(sl - (0.4 - c)) < 1e-14 and abs(sr - (0.4 + c)) < 1e-14


@pytest.mark.parametrize("einfeldt", [False, True])
def test_flux_form_gravity_balances_potential_energy(einfeldt):
    """Constant gravity, potential phi = -g.x at zone centres.  With the
    mass-flux energy source the interior work of gravity telescopes against
    the change of sum(rho*phi), so total energy plus potential changes only by
    what crosses the domain boundary:
      d sum(rhoE + rho phi) = sum over boundary faces of
        -dt/dx (F_E,hi - F_E,lo) - dt/dx (F_rho,hi phi_last - F_rho,lo phi_first)
        + dt g (F_rho,lo + F_rho,hi)/2
    to round-off.  The cell-centred momentum form misses this by O(dt^2)."""
    n = (12, 10, 14)
    rng = np.random.default_rng(23)
    U = inputs.random_box(rng, n, 3)
    g = (0.3, -0.5, -2.0)
    dx = (1 / 12, 1 / 10, 1 / 14)
    x = [(np.arange(k) + 0.5) * h for k, h in zip(n, dx)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    phi = -(g[0] * X + g[1] * Y + g[2] * Z)
    errs = {}
    for flux_form in (True, False):
        P = oracle.params(3, n, dx=dx, bc=oracle.BC_REFLECT, gamma=5 / 3, grav=g, flux_grav_energy=flux_form,
                          einfeldt=einfeldt)
        d, _ = oracle.dt(U, P)
        U1, rc, dbg = oracle.step(U, P, d, debug=True)
        assert rc == 0
        inner = lambda V: V[:, 4:-4, 4:-4, 4:-4]
        change = (inner(U1)[4] - inner(U)[4]).sum() + ((inner(U1)[0] - inner(U)[0]) * phi).sum()
        boundary = 0.0
        for ax in range(3):
            F = dbg["flux_final"][ax]
            lo = [slice(4, -4)] * 3
            hi = [slice(4, -4)] * 3
            lo[2 - ax] = 4               # face 0 along this axis (array axes are z, y, x)
            hi[2 - ax] = 4 + n[ax]       # face n along this axis
            f_lo, f_hi = F[(slice(None),) + tuple(lo)], F[(slice(None),) + tuple(hi)]
            first = [slice(None)] * 3
            last = [slice(None)] * 3
            first[2 - ax] = 0
            last[2 - ax] = n[ax] - 1
            dtdx = d / dx[ax]
            boundary += (-dtdx * (f_hi[4] - f_lo[4]) - dtdx * (f_hi[0] * phi[tuple(last)] - f_lo[0] * phi[tuple(first)])
                         + d * g[ax] * 0.5 * (f_lo[0] + f_hi[0])).sum()
        scale = np.abs(inner(U)[4]).sum()
        errs[flux_form] = abs(change - boundary) / scale
    assert errs[True] <= 1e-14, errs
    assert errs[False] > 1e3 * max(errs[True], 1e-17), errs


# ---------------------------------------------------------------- corner transport (CTU transverse terms)
# Uniform velocity and pressure reduce the Euler equations to advection of the
# density (a contact wave), whose exact solution is a translation.  Two exact
# solutions of that problem fix every coefficient and every index of the
# corner-transport corrections (Sec. 3.2, unsplit PPM):
#   * a profile that is linear in each coordinate separately (bilinear in 2-D,
#     trilinear in 3-D).  Averaging the exact x-flux over the step gives
#     X [Y Z - (b Z + c Y)/2 + b c / 3] + (terms that do not depend on X and
#     cancel in the x-difference), with b, c the transverse Courant lengths:
#     the 1/2 of the final correction and, in 3-D, the 1/3 of the intermediate
#     one composed with the final 1/2 (1/2 * 1/3 twice) are the only weights
#     that reproduce it, so the translated zone averages come out to round-off;
#   * unit Courant number along every axis: the exact step moves every zone
#     average by one zone along each axis.  The upwind x-state of a 3-D CTU
#     step at Courant number 1 is the weighted sum 1/3 (own zone) + 1/6 +
#     1/6 (transverse neighbours) + 1/3 (the diagonal one), which is exactly
#     the fraction of the face's swept volume in each zone; a wrong weight, a
#     wrong transverse pair or the other zone's transverse faces breaks it for
#     a random density.
CORNER_N = {3: (12, 10, 8), 2: (12, 10, 1)}
CORNER_VEL = (0.7, 0.4, -0.3)


def _interior_rel_err(A, B, dim):
    I = I3 if dim == 3 else I2
    a, b = A[I].reshape(5, -1), B[I].reshape(5, -1)
    den = np.abs(b).max(axis=1)
    return float((np.abs(a - b).max(axis=1) / np.where(den > 0, den, 1.0)).max())


def product_profile_error(dim):
    """Max relative interior error of one CFL step of the product profile
    against its exact translation."""
    n, dx = CORNER_N[dim], (1 / 12, 1 / 12, 1 / 12)
    U0 = inputs.product_profile(n, dim, dx, CORNER_VEL)
    P = oracle.params(dim, n, dx=dx, bc=oracle.BC_PREFILLED, gamma=1.4)
    d, rc = oracle.dt(U0, P)
    U1, rc1 = oracle.step(U0, P, d)
    if rc or rc1:
        return float("inf")
    return _interior_rel_err(U1, inputs.product_profile(n, dim, dx, CORNER_VEL, t=d), dim)


def unit_courant_error(dim, signs):
    """Max relative interior error of one unit-Courant step of a random density
    against the exact one-zone translation."""
    n, dx, dt = CORNER_N[dim], (1 / 12, 1 / 10, 1 / 8), 0.05
    U0, want = inputs.translation_box(np.random.default_rng(17), n, dim, dx, dt, signs)
    P = oracle.params(dim, n, dx=dx, bc=oracle.BC_PREFILLED, gamma=1.4)
    U1, rc = oracle.step(U0, P, dt)
    return float("inf") if rc else _interior_rel_err(U1, want, dim)


@pytest.mark.parametrize("dim", [3, 2])
def test_product_profile_is_advected_exactly(dim):
    assert product_profile_error(dim) <= 1e-13


@pytest.mark.parametrize("dim,signs", [(3, (1, 1, 1)), (3, (1, -1, 1)), (3, (-1, 1, -1)), (2, (1, 1, 1)),
                                       (2, (-1, 1, 1))])
def test_unit_courant_step_translates_by_one_zone(dim, signs):
    assert unit_courant_error(dim, signs) <= 1e-13


# each edit is a plausible slip in the corner-transport code; every one must
# fail at least one of the two exact solutions above (checked in 3-D and 2-D)
CORNER_MISTAKES = {
    "intermediate coefficient 1/2 instead of 1/3":
        [("real coef = dtdx[t] * THIRD;", "real coef = dtdx[t] * 0.5;")],
    "intermediate correction dropped":
        [("real coef = dtdx[t] * THIRD;", "real coef = dtdx[t] * 0.0;")],
    "intermediate correction with the wrong sign":
        [("real coef = dtdx[t] * THIRD;", "real coef = -dtdx[t] * THIRD;")],
    "intermediate correction from the other zone's transverse faces":
        [("F1[t].get(zl + g.str[t], a); F1[t].get(zl, b);", "F1[t].get(id + g.str[t], a); F1[t].get(id, b);")],
    "final 3-D correction with F^{t|d} instead of F^{t1|t2}":
        [("F2[t1][t2].get(z + g.str[t1], ah); F2[t1][t2].get(z, al);",
          "F2[t1][d].get(z + g.str[t1], ah); F2[t1][d].get(z, al);"),
         ("F2[t2][t1].get(z + g.str[t2], bh); F2[t2][t1].get(z, bl);",
          "F2[t2][d].get(z + g.str[t2], bh); F2[t2][d].get(z, bl);")],
    "final 3-D coefficient 1/3 instead of 1/2":
        [("correct_state(q, *P, K, 0.5 * dtdx[t1], ah, al, 0.5 * dtdx[t2], bh, bl, s);",
          "correct_state(q, *P, K, THIRD * dtdx[t1], ah, al, THIRD * dtdx[t2], bh, bl, s);")],
    "final 2-D coefficient 1/3 instead of 1/2":
        [("correct_state(q, *P, K, 0.5 * dtdx[t1], ah, al, 0.0, nullptr, nullptr, s);",
          "correct_state(q, *P, K, THIRD * dtdx[t1], ah, al, 0.0, nullptr, nullptr, s);")],
    "final 2-D correction dropped":
        [("correct_state(q, *P, K, 0.5 * dtdx[t1], ah, al, 0.0, nullptr, nullptr, s);",
          "correct_state(q, *P, K, 0.0 * dtdx[t1], ah, al, 0.0, nullptr, nullptr, s);")],
    "final correction from the other zone's transverse faces":
        [("long z = side ? id : zl;", "long z = side ? zl : id;")],
}


@pytest.mark.parametrize("name", list(CORNER_MISTAKES))
def test_planted_corner_transport_mistakes_fail(name, tmp_path):
    from oracle_variants import planted
    dim = 2 if "2-D" in name else 3
    with planted(tmp_path, CORNER_MISTAKES[name]):
        errs = (product_profile_error(dim), unit_courant_error(dim, (1, -1, 1)))
    assert max(errs) > 1e-9, (name, errs)
