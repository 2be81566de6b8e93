"""Pins of the CPU oracle against facts other than itself (no GPU needed).

Each test names the passage or textbook fact it checks.  The paper defines the chemistry step
as the integration of the reaction system (Sec. 2.2, Eq. 1) over one flow step (Eq. 2); the
kinetics and thermo forms are the textbook ones the paper's Cantera/CVODE stack uses.
"""
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from oracle.core import R_GAS, P0
from paper_2402_18858_gb300 import workload as w

from conftest import GOLDEN

P = 101325.0


def _z(st, i):
    return np.concatenate([st.Y[:, i], [st.T[i]]])


# --- NASA-7 (Sec. 2.1 "high-order temperature polynomials"): dh/dT = cp, ds/dT = cp/T --------
@pytest.mark.parametrize("kind", ["h2_9", "c_30"])
def test_nasa7_thermodynamic_identities(oracles, mechs, kind):
    o = oracles[kind]
    m, _ = mechs[kind]
    for T in (400.0, 800.0, 1500.0, 2500.0, 3500.0):
        dT = 1e-3
        cp, h, s = o.species_thermo(T)
        _, hp, sp = o.species_thermo(T + dT)
        _, hm, sm = o.species_thermo(T - dT)
        dh = (hp * (T + dT) - hm * (T - dT)) / (2 * dT)      # d(h/R)/dT
        ds = (sp - sm) / (2 * dT)                               # d(s/R)/dT
        assert np.allclose(dh, cp, rtol=1e-8, atol=0)
        assert np.allclose(ds, cp / T, rtol=1e-7, atol=0)
    # continuity of cp, h and s across T_mid
    a = o.species_thermo(m.T_mid * (1 - 1e-12))
    b = o.species_thermo(m.T_mid * (1 + 1e-12))
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-8, atol=1e-9)


# --- Arrhenius: d ln k / d ln T = b + Ea/(RT) (the Arrhenius-plot slope) ----------------------
def test_arrhenius_slope(oracles, mechs):
    o = oracles["h2_9"]
    m, _ = mechs["h2_9"]
    st = w.make_states(m, 1, 3)
    Y = st.Y[:, 0]
    for T in (600.0, 1500.0):
        e = 1e-5
        _, _, _, kp, _ = o.rates(T * math.exp(e), P, Y, with_rxn=True)
        _, _, _, km, _ = o.rates(T * math.exp(-e), P, Y, with_rxn=True)
        slope = (np.log(kp) - np.log(km)) / (2 * e)
        for j, r in enumerate(m.reactions):
            assert slope[j] == pytest.approx(r.b + r.Ea / (R_GAS * T), rel=1e-6, abs=1e-8)


# --- third body and Troe special cases ------------------------------------------------------
def test_troe_reduces_to_lindemann_and_thirdbody_total_concentration():
    o = Oracle(os.path.join(GOLDEN, "troe_lindemann.mech"))
    T = 1000.0
    Y = np.array([0.1, 0.2, 0.7])
    for p in (1.0, 1e3, P, 1e7, 1e12):
        M = p / (R_GAS * T)               # all efficiencies 1: [M] is the total concentration
        kinf, k0 = 1.0e3, 1.0e2
        Pr = k0 * M / kinf
        wd, hrr, q, kf, kr = o.rates(T, p, Y, with_rxn=True)
        assert kf[0] == pytest.approx(kinf * Pr / (1 + Pr), rel=1e-13)
        rho = p / (R_GAS * T) / (Y / o.W).sum()
        Cc = rho * Y / o.W
        q_noM = kf[1] * Cc[0] ** 2 - kr[1] * Cc[1]
        assert q[1] / q_noM == pytest.approx(M, rel=1e-12)
    # limits: high pressure -> k_inf, low pressure -> k0 [M]
    _, _, _, kf, _ = o.rates(T, 1e14, Y, with_rxn=True)
    assert kf[0] == pytest.approx(1.0e3, rel=1e-6)
    _, _, _, kf, _ = o.rates(T, 1e-3, Y, with_rxn=True)
    assert kf[0] == pytest.approx(1.0e2 * 1e-3 / (R_GAS * T), rel=1e-6)


def test_troe_center_point_gives_Fcent():
    o = Oracle(os.path.join(GOLDEN, "troe_general.mech"))
    Y = np.array([0.1, 0.2, 0.7])
    a, T3, T1, T2 = 0.6, 200.0, 1500.0, 4000.0
    for T in (500.0, 1200.0, 2400.0):
        Fc = (1 - a) * math.exp(-T / T3) + a * math.exp(-T / T1) + math.exp(-T2 / T)
        c = -0.4 - 0.67 * math.log10(Fc)
        Pr = 10.0 ** (-c)
        M = Pr * 3.0e4 / 2.0e3
        p = M * R_GAS * T
        _, _, _, kf, _ = o.rates(T, p, Y, with_rxn=True)
        assert kf[0] == pytest.approx(3.0e4 * Pr / (1 + Pr) * Fc, rel=1e-12)
        # away from the centre F differs from F_cent (the broadening is active)
        _, _, _, kf2, _ = o.rates(T, p * 100, Y, with_rxn=True)
        Pr2 = Pr * 100
        assert abs(kf2[0] / (3.0e4 * Pr2 / (1 + Pr2)) - Fc) > 1e-3


# --- RHS invariants of Eq. 1: mass, elements, enthalpy at constant p -------------------------
@pytest.mark.parametrize("kind", ["h2_9", "c_30", "c_53"])
def test_rhs_conservation(oracles, mechs, kind):
    o = oracles[kind]
    m, _ = mechs[kind]
    st = w.make_states(m, 16, 11)
    for i in range(16):
        z = _z(st, i)
        f = o.rhs(P, z)
        fY, fT = f[:-1], f[-1]
        gross = np.abs(fY).sum()
        assert abs(fY.sum()) <= 1e-13 * gross + 1e-300
        el = (o.comp.T * (fY / o.W)).sum(axis=1)
        elg = (np.abs(o.comp.T) * np.abs(fY / o.W)).sum(axis=1)
        assert (np.abs(el) <= 1e-13 * elg + 1e-300).all()
        cpR, hRT, _ = o.species_thermo(z[-1])
        hk = hRT * R_GAS * z[-1] / o.W             # J/kg of each species
        cp = (z[:-1] * cpR * R_GAS / o.W).sum()
        dh = (hk * fY).sum() + cp * fT
        assert abs(dh) <= 1e-12 * (np.abs(hk * fY).sum() + abs(cp * fT)) + 1e-300


# --- analytic Jacobian against central differences (Richardson-extrapolated) ------------------
@pytest.mark.parametrize("kind", ["h2_9", "c_30"])
def test_jacobian_finite_differences(oracles, mechs, kind):
    o = oracles[kind]
    m, _ = mechs[kind]
    st = w.make_states(m, 6, 12)
    for i in range(6):
        z = _z(st, i)
        J = o.jacobian(P, z)
        R1 = np.zeros_like(J)
        R2 = np.zeros_like(J)
        for j in range(o.n):
            hs = 1e-3 * max(abs(z[j]), 1e-12)

            def cd(hh):
                zp, zm = z.copy(), z.copy()
                zp[j] += hh
                zm[j] -= hh
                return (o.rhs(P, zp) - o.rhs(P, zm)) / (2 * hh)
            c1, c2, c3 = cd(hs), cd(hs / 2), cd(hs / 4)
            R1[:, j] = (4 * c2 - c1) / 3
            R2[:, j] = (4 * c3 - c2) / 3
        # the spread of two Richardson estimates bounds the finite-difference error; a wrong
        # analytic entry would sit far outside it
        scale = np.abs(J).max(axis=1, keepdims=True) + 1e-300
        bar = 10 * np.abs(R1 - R2) + 1e-7 * scale
        assert (np.abs(J - R2) <= bar).all()
        assert (np.abs(J - R2) <= 1e-6 * scale).mean() > 0.97


# --- dense LU with partial pivoting against LAPACK ------------------------------------------
def test_dense_solve_matches_lapack():
    rng = np.random.default_rng(0)
    for n in (1, 2, 10, 31, 54):
        A = rng.standard_normal((n, n))
        b = rng.standard_normal(n)
        assert np.allclose(Oracle.dense_solve(A, b), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    A = np.ones((3, 3))
    with pytest.raises(np.linalg.LinAlgError):
        Oracle.dense_solve(A, np.ones(3))


# --- integrator: closed form of a reversible first-order isomerisation -----------------------
def test_integrator_isomerisation_closed_form():
    o = Oracle(os.path.join(GOLDEN, "isomer.mech"))
    YA0, YB0, T0 = 0.6, 0.1, 1000.0
    for rtol, bar in ((1e-10, 1e-8), (1e-12, 1e-10)):
        for dt in (1e-7, 3e-6, 1e-5, 1e-3):
            z = np.array([YA0, YB0, 1 - YA0 - YB0, T0])
            zn, s, st = o.integrate(P, z, dt, rtol=rtol)
            assert s == 0
            YAeq = (YA0 + YB0) / 3.0
            exact = YAeq + (YA0 - YAeq) * math.exp(-(2e5 + 1e5) * dt)
            assert zn[0] == pytest.approx(exact, rel=bar)
            assert zn[3] == pytest.approx(T0, rel=1e-12)


# --- the oracle's method: three-stage Radau IIA (Hairer & Wanner II, Sec. IV.5) -----------
def test_radau_tableau_order_conditions():
    """Nodes are the zeros of d^2/dx^2 [x^2 (x-1)^3] (Radau right points); the weights satisfy
    B(5) (quadrature exact to degree 4, hence order 5), the coefficients C(3) (collocation:
    stage order 3), and the last row equals the weights (stiffly accurate)."""
    A, c = Oracle.radau_tableau()
    P = np.polynomial.Polynomial([0, 0, 1]) * np.polynomial.Polynomial([-1, 1]) ** 3
    assert np.allclose(np.sort(P.deriv(2).roots().real), c, rtol=0, atol=1e-14)
    b = A[2]
    for q in range(1, 6):
        assert (b * c ** (q - 1)).sum() == pytest.approx(1.0 / q, rel=1e-14)
    for q in range(1, 4):
        assert np.allclose(A @ c ** (q - 1), c ** q / q, rtol=1e-14, atol=1e-15)
    assert c[2] == 1.0


def test_radau_fixed_steps_converge_with_order_five():
    """On the closed-form isomerisation, halving the fixed step divides the global error by
    about 2^5 (a wrong coefficient drops the order)."""
    o = Oracle(os.path.join(GOLDEN, "isomer.mech"))
    YA0, YB0, T0, tend = 0.6, 0.1, 1000.0, 1e-5
    YAeq = (YA0 + YB0) / 3.0
    exact = YAeq + (YA0 - YAeq) * math.exp(-3e5 * tend)
    errs = []
    for N in (8, 16, 32):
        z = o.radau_fixed(P, np.array([YA0, YB0, 1 - YA0 - YB0, T0]), tend / N, N)
        errs.append(abs(z[0] - exact))
    for e1, e2 in zip(errs, errs[1:]):
        assert 4.6 < math.log2(e1 / e2) < 5.4, errs


@pytest.mark.parametrize("kind,n,dt", [("c_30", 4, 5e-6), ("c_53", 3, 1e-5)])
def test_integrator_rtol_refinement(oracles, mechs, kind, n, dt):
    """The oracle's default tolerance (rtol 1e-10) agrees with a 100x tighter run to 1e-9
    relative on T and on every mass fraction above 1e-10."""
    o = oracles[kind]
    m, _ = mechs[kind]
    st = w.make_states(m, n, 104)
    T1, Y1, s1, _ = o.integrate_batch(st.T, st.p, st.Y, dt)
    T2, Y2, s2, _ = o.integrate_batch(st.T, st.p, st.Y, dt, rtol=1e-12)
    assert (s1 == 0).all() and (s2 == 0).all()
    assert (np.abs(T1 - T2) <= 1e-9 * T2).all()
    big = Y2 > 1e-10
    assert (np.abs(Y1 - Y2)[big] <= 1e-9 * Y2[big]).all()


# --- integrator against brute-force fine-step RK4 ------------------------------------------
def test_integrator_against_rk4(oracles, mechs):
    o = oracles["h2_9"]
    m, _ = mechs["h2_9"]
    st = w.make_states(m, 64, 100)
    dt = 1e-6
    checked = 0
    for i in range(64):
        z = _z(st, i)
        J = o.jacobian(P, z)
        lam = np.abs(np.linalg.eigvals(J)).max()
        nsub = int(max(64, 4 * lam * dt))
        if nsub > 200000:
            continue           # too stiff for the explicit reference
        zb, s, _ = o.integrate(P, z, dt)
        assert s == 0
        za = o.rk4(P, z, dt, nsub)
        zb2 = o.rk4(P, z, dt, 2 * nsub)
        # the RK4 reference has converged (halving the step changes nothing that matters)
        big = np.abs(zb2) > 1e-10
        assert np.allclose(za[big], zb2[big], rtol=1e-9)
        assert np.allclose(zb[big], zb2[big], rtol=1e-8)
        checked += 1
        if checked >= 6:
            break
    assert checked >= 3


# --- integrator invariants after one step (Eq. 2): mass, elements, enthalpy -----------------
@pytest.mark.parametrize("kind,dt", [("h2_9", 1e-6), ("c_30", 5e-6)])
def test_integrator_invariants(oracles, mechs, kind, dt):
    o = oracles[kind]
    m, _ = mechs[kind]
    st = w.make_states(m, 24, 101)
    T, Y, status, steps = o.integrate_batch(st.T, st.p, st.Y, dt)
    assert (status == 0).all()
    assert np.allclose(Y.sum(0), 1.0, rtol=0, atol=1e-12)
    el0 = o.comp.T @ (st.Y / o.W[:, None])
    el1 = o.comp.T @ (Y / o.W[:, None])
    assert np.allclose(el1, el0, rtol=1e-11, atol=0)
    for i in range(24):
        h0 = o.thermo_props(st.T[i], st.Y[:, i])[1]
        h1 = o.thermo_props(T[i], Y[:, i])[1]
        assert h1 == pytest.approx(h0, rel=1e-8, abs=1e-3)


def test_integrator_tolerance_convergence(oracles, mechs):
    o = oracles["c_30"]
    m, _ = mechs["c_30"]
    st = w.make_states(m, 8, 102)
    ref = o.integrate_batch(st.T, st.p, st.Y, 5e-6, rtol=1e-12)
    prev = None
    for rtol in (1e-7, 1e-9, 1e-11):
        T, Y, s, _ = o.integrate_batch(st.T, st.p, st.Y, 5e-6, rtol=rtol)
        err = np.abs(T - ref[0]) / ref[0]
        e = err.max()
        if prev is not None:
            assert e < prev or e < 1e-12
        prev = e
    assert prev < 1e-9


# --- long-time limit is the Gibbs (HP) equilibrium; every net rate vanishes there ------------
@pytest.mark.parametrize("kind", ["h2_9", "c_30"])
def test_long_time_limit_is_gibbs_equilibrium(oracles, mechs, kind):
    """Kinetic equilibrium of the reverse rates (k_r = k_f/K_c) must be a Gibbs minimum.

    For each reaction, sum_k nu_kj (ln X_k + g_k/RT + ln p/p0) = 0 at equilibrium: a condition
    on thermodynamics alone, so a wrong K_c (sign, p0/RT factor, NASA-7 entropy) fails it.  Where
    the reactions span every composition change the elements allow, the state also satisfies
    the element-potential conditions of a constrained Gibbs minimum.
    """
    o = oracles[kind]
    m, _ = mechs[kind]
    nu = np.zeros((m.n_species, m.n_reactions))
    for j, r in enumerate(m.reactions):
        for k in r.reactants:
            nu[k, j] -= 1
        for k in r.products:
            nu[k, j] += 1
    full_rank = np.linalg.matrix_rank(nu) == m.n_species - np.linalg.matrix_rank(m.comp)
    st = w.make_states(m, 4, 103, T_range=(1500.0, 2000.0))
    for i in range(2):
        z = _z(st, i)
        h0 = o.thermo_props(z[-1], z[:-1])[1]
        ze, s, _ = o.integrate(P, z, 1e9, rtol=1e-11, atol_Y=1e-30, max_steps=10 ** 6)
        assert s == 0
        T, Y = ze[-1], ze[:-1]
        assert o.thermo_props(T, Y)[1] == pytest.approx(h0, rel=1e-8, abs=1e-3)
        X = (Y / o.W) / (Y / o.W).sum()
        cpR, hRT, sR = o.species_thermo(T)
        r = np.log(np.maximum(X, 1e-300)) + hRT - sR + math.log(P / P0)
        resolved = np.abs(nu[X < 1e-25]).sum(0) == 0        # reactions free of trace species
        assert resolved.sum() > 0.5 * m.n_reactions
        assert np.abs(nu.T @ r)[resolved].max() < 1e-9
        if full_rank:
            keep = X > 1e-12
            A = o.comp[keep].astype(float)
            lam, *_ = np.linalg.lstsq(A, r[keep], rcond=None)
            assert np.abs(A @ lam - r[keep]).max() < 1e-8
        # detailed balance: each net rate is negligible against its forward gross rate
        wd, hrr, q, kf, kr = o.rates(T, P, Y, with_rxn=True)
        rho = P / (R_GAS * T) / (Y / o.W).sum()
        Cc = rho * Y / o.W
        for j, rx in enumerate(m.reactions):
            if not resolved[j]:
                continue
            fwd = kf[j] * np.prod(Cc[rx.reactants])
            rev = kr[j] * np.prod(Cc[rx.products])
            assert abs(fwd - rev) <= 1e-8 * max(fwd, rev)


# --- mixture properties (Sec. 2.1): special cases of the mixing rules -----------------------
def test_thermo_props_special_cases(oracles, mechs):
    o = oracles["c_30"]
    m, _ = mechs["c_30"]
    for k in (0, 5, 13):
        Y = np.zeros(o.K)
        Y[k] = 1.0
        for T in (500.0, 1800.0):
            cp, h, mu, lam = o.thermo_props(T, Y)
            L = math.log(T)
            muk = math.exp(sum(m.mu_fit[k, i] * L ** i for i in range(4)))
            lamk = math.exp(sum(m.lam_fit[k, i] * L ** i for i in range(4)))
            assert mu == pytest.approx(muk, rel=1e-13)       # Wilke with one species
            assert lam == pytest.approx(lamk, rel=1e-13)     # combining rule, one species
    # two species with equal W and equal transport fits behave as one
    o2 = Oracle(os.path.join(GOLDEN, "isomer.mech"))
    Yi = np.array([0.3, 0.7, 0.0])
    Ya = np.array([1.0, 0.0, 0.0])
    for T in (400.0, 2000.0):
        a = o2.thermo_props(T, Yi)
        b = o2.thermo_props(T, Ya)
        assert a[2] == pytest.approx(b[2], rel=1e-14)
        assert a[3] == pytest.approx(b[3], rel=1e-14)
    # cp is the temperature derivative of h (mixture)
    st = w.make_states(m, 4, 5)
    for i in range(4):
        T = st.T[i]
        hp = o.thermo_props(T + 1e-3, st.Y[:, i])[1]
        hm = o.thermo_props(T - 1e-3, st.Y[:, i])[1]
        assert o.thermo_props(T, st.Y[:, i])[0] == pytest.approx((hp - hm) / 2e-3, rel=1e-7)
        # Newton T-from-h round trip
        h = o.thermo_props(T, st.Y[:, i])[1]
        assert o.T_from_h(h, st.Y[:, i], T0=1000.0) == pytest.approx(T, abs=1e-8)


def test_wilke_viscosity_textbook_example():
    """Wilke's rule on the worked example of Bird, Stewart & Lightfoot (Sec. 1.4): CO2/O2/N2 at
    mole fractions 0.133/0.039/0.828 give 1714e-7 g/(cm s) = 1.714e-5 Pa s (4 digits)."""
    o = Oracle(os.path.join(GOLDEN, "wilke_bsl.mech"))
    x = np.array([0.133, 0.039, 0.828])
    Y = x * o.W / (x * o.W).sum()
    mu = o.thermo_props(293.0, Y)[2]
    assert mu == pytest.approx(1.714e-5, abs=0.5e-8)        # half a unit of the 4th digit


def test_conductivity_combining_rule_binary():
    """Mixture-averaged conductivity (half the sum of the arithmetic and harmonic means over
    MOLE fractions): 0.25 CO2 (0.02 W/m/K) + 0.75 O2 (0.06) gives (0.05 + 0.04)/2 = 0.045."""
    o = Oracle(os.path.join(GOLDEN, "wilke_bsl.mech"))
    x = np.array([0.25, 0.75, 0.0])
    Y = x * o.W / (x * o.W).sum()
    assert o.thermo_props(800.0, Y)[3] == pytest.approx(0.045, rel=1e-13)


# --- loader rejects malformed input ----------------------------------------------------------
def test_mechanism_validation(tmp_path):
    with pytest.raises(ValueError, match="balanced"):
        Oracle(os.path.join(GOLDEN, "unbalanced.mech"))
    with pytest.raises(ValueError):
        Oracle(str(tmp_path / "missing.mech"))
    bad = tmp_path / "bad.mech"
    bad.write_text("mech x\nelements H\nspecies 1\nsp H 0.001 1\nbogus\n")
    with pytest.raises(ValueError):
        Oracle(str(bad))
