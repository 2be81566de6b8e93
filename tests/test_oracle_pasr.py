"""Pins of the PaSR source oracle (CPU): limits of the model, a hand-computed cell, and
conservation of the filtered source."""
import math

import numpy as np

from oracle.pasr import pasr_source


def _cell(Y0, Y1, rho=0.5, k=2.0, eps=1.0e3, nu=2.0e-5):
    Y0 = np.asarray(Y0, dtype=np.float64)[:, None]
    Y1 = np.asarray(Y1, dtype=np.float64)[:, None]
    f = lambda v: np.array([v], dtype=np.float64)  # noqa: E731
    return Y0, Y1, f(rho), f(k), f(eps), f(nu)


def test_hand_computed_two_species_cell():
    # A -> B over dt = 1e-6 s: B is formed (0.1 -> 0.3), A is consumed
    dt = 1e-6
    Y0, Y1, rho, k, eps, nu = _cell([0.9, 0.1], [0.7, 0.3])
    omega, kappa = pasr_source(rho, Y0, Y1, dt, k, eps, nu)
    tau_c = 0.3 / (0.2 / dt)                      # slowest (only) formation: B
    tau_mix = math.sqrt(math.sqrt(2e-5 / 1e3) * (2.0 / 1e3))
    kap = tau_c / (tau_c + tau_mix)
    assert kappa[0] == np.float64(kap) or abs(kappa[0] - kap) <= 1e-15 * kap
    np.testing.assert_allclose(omega[:, 0], kap * 0.5 * np.array([-0.2, 0.2]) / dt, rtol=1e-14)


def test_laminar_limit_gives_the_chemistry_rate():
    # no sub-grid turbulence (k = 0 or eps = 0): kappa = 1, omega = rho dY/dt
    dt = 5e-6
    rng = np.random.default_rng(3)
    Y0 = rng.dirichlet(np.ones(6), size=50).T
    Y1 = rng.dirichlet(np.ones(6), size=50).T
    rho = rng.uniform(0.1, 1.2, 50)
    k = np.where(np.arange(50) % 2 == 0, 0.0, 1.0)
    eps = np.where(np.arange(50) % 2 == 0, 1e3, 0.0)
    omega, kappa = pasr_source(rho, Y0, Y1, dt, k, eps, np.full(50, 1e-5))
    assert (kappa == 1.0).all()
    np.testing.assert_allclose(omega, rho * (Y1 - Y0) / dt, rtol=1e-15)


def test_fast_chemistry_limit():
    # tau_c << tau_mix: kappa -> tau_c / tau_mix (to first order in their ratio)
    dt = 1e-6
    Y0, Y1, rho, k, eps, nu = _cell([0.5, 0.5], [0.4, 0.6], k=1e4, eps=1e-2, nu=1e-4)
    _, kappa = pasr_source(rho, Y0, Y1, dt, k, eps, nu)
    tau_c = 0.6 / (0.1 / dt)
    tau_mix = math.sqrt(math.sqrt(1e-4 / 1e-2) * (1e4 / 1e-2))
    assert tau_c / tau_mix < 1e-6
    assert abs(kappa[0] - tau_c / tau_mix) <= 2 * (tau_c / tau_mix) ** 2


def test_trace_and_consumed_species_do_not_set_the_chemical_time():
    # species 0 is consumed, species 1 and 2 are formed, species 3 is a trace species (below
    # y_min) that grows very slowly: its formation time (~10 s) must not set tau_c
    dt = 1e-6
    Y0 = np.array([0.6, 0.2, 0.2 - 1e-12, 1e-12])[:, None]
    Y1 = np.array([0.0, 0.25, 0.2 - 1e-12 + 0.01, 1e-12 + 1e-19])[:, None]
    Y1[0, 0] = 1.0 - Y1[1:, 0].sum()
    omega, kappa = pasr_source(np.array([1.0]), Y0, Y1, dt, np.array([0.0]), np.array([0.0]), np.array([1e-5]))
    assert kappa[0] == 1.0
    tau_mix = math.sqrt(math.sqrt(1e-5 / 10.0) * (1.0 / 10.0))
    _, kappa = pasr_source(np.array([1.0]), Y0, Y1, dt, np.array([1.0]), np.array([10.0]), np.array([1e-5]))
    t1 = Y1[1, 0] / ((Y1[1, 0] - Y0[1, 0]) / dt)
    t2 = Y1[2, 0] / ((Y1[2, 0] - Y0[2, 0]) / dt)
    assert t2 > t1                      # species 2 is the slowest formed species above y_min
    assert abs(kappa[0] - t2 / (t2 + tau_mix)) <= 1e-15


def test_source_conserves_mass_and_elements():
    # omega is kappa rho dY/dt per cell: if the chemistry step conserves sum Y and the element
    # masses, so does the filtered source
    rng = np.random.default_rng(7)
    K, N, dt = 5, 200, 1e-6
    comp = rng.integers(0, 3, size=(3, K)).astype(np.float64)   # element counts
    W = comp.T @ np.array([1.0e-3, 12.0e-3, 16.0e-3]) + 1e-3
    Y0 = rng.dirichlet(np.ones(K), size=N).T
    # a step along the null space of [ones; comp / W]: conserves sum Y and elements
    A = np.vstack([np.ones(K), comp / W[None, :]])
    _, _, vt = np.linalg.svd(A)
    null = vt[A.shape[0]:]
    dY = (null.T @ rng.standard_normal((null.shape[0], N))) * 1e-4
    Y1 = Y0 + dY
    rho = rng.uniform(0.2, 1.0, N)
    omega, kappa = pasr_source(rho, Y0, Y1, dt, rng.uniform(0.1, 5.0, N), rng.uniform(10.0, 1e4, N),
                               rng.uniform(1e-5, 1e-4, N))
    # bound: the rounding of Y1 and of Y1 - Y0 (a few ulp of |Y|), scaled by kappa rho / dt
    ulp = 4 * np.finfo(np.float64).eps * (np.abs(Y0) + np.abs(Y1))
    bound = kappa * rho / dt * ulp.sum(axis=0)
    assert (np.abs(omega.sum(axis=0)) <= bound).all()
    cw = comp / W[None, :]
    assert (np.abs(cw @ omega) <= cw.max() * bound[None, :]).all()
