"""PaSR filtered reaction source from one chemistry step -- FP64 numpy oracle (test
infrastructure only: the tests, the package's smoke check and the benchmark's CPU-baseline leg
use it; it imports nothing from the GPU package).

The paper closes turbulence-chemistry interaction with the partially stirred reactor model
(Sec. 3, case set-up of the swirl flame): the learned step (or DI) supplies the reaction source
inside PaSR, the chemical time scale comes from the slowest species formation rate and the
mixing time from the geometric mean of the Taylor and Kolmogorov scales.  The paper gives no
formulas; the readings (stated here and in the design notes) are:

* reacting fraction (Chomiak's PaSR): kappa = tau_c / (tau_c + tau_mix);
* mixing time: tau_mix = sqrt(tau_K tau_t) with the Kolmogorov time tau_K = sqrt(nu / eps) and
  the sub-grid turbulence time tau_t = k / eps; k <= 0 or eps <= 0 (no sub-grid turbulence)
  gives tau_mix = 0, i.e. kappa = 1;
* chemical time: over the species formed during the step -- new mass fraction at least y_min
  and a gain Y_k(t+dt) - Y_k(t) above r_min Y_k(t+dt), so that rounding-level changes of
  species at rest do not count -- the largest formation time Y_k(t+dt) / (dY_k/dt), with
  dY_k/dt = (Y_k(t+dt) - Y_k(t)) / dt the step's mean rate; no such species gives tau_c = 0;
* filtered source: omega_k = kappa rho dY_k/dt (kg/m^3/s), rho the cell density.

Parity: pinned by tests/test_oracle_pasr.py (laminar limit kappa = 1, the fast-chemistry
limit kappa -> tau_c / tau_mix, a hand-computed two-species cell, species-sum and element
conservation of the source).
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

Y_MIN = 1e-10
R_MIN = 1e-9


def pasr_source(rho: np.ndarray, Y0: np.ndarray, Y1: np.ndarray, dt: float, k_sgs: np.ndarray,
                eps: np.ndarray, nu: np.ndarray, y_min: float = Y_MIN,
                r_min: float = R_MIN) -> Tuple[np.ndarray, np.ndarray]:
    """omega [K, N] (kg/m^3/s) and kappa [N] for N cells; Y0, Y1 species-major [K, N]."""
    rho = np.asarray(rho, dtype=np.float64)
    Y0 = np.asarray(Y0, dtype=np.float64)
    Y1 = np.asarray(Y1, dtype=np.float64)
    k_sgs = np.asarray(k_sgs, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    dY = Y1 - Y0
    rate = dY / dt
    # chemical time: the slowest formation among the species formed and present
    formed = (Y1 >= y_min) & (dY > r_min * Y1)
    tau_k = np.zeros_like(Y1)
    tau_k[formed] = Y1[formed] / rate[formed]
    tau_c = tau_k.max(axis=0) if tau_k.size else np.zeros(rho.shape)
    # mixing time: geometric mean of the Kolmogorov time and the sub-grid time k / eps
    turb = (k_sgs > 0.0) & (eps > 0.0)
    tau_mix = np.zeros_like(rho)
    tau_mix[turb] = np.sqrt(np.sqrt(nu[turb] / eps[turb]) * (k_sgs[turb] / eps[turb]))
    tot = tau_c + tau_mix
    kappa = np.ones_like(rho)
    pos = tot > 0.0
    kappa[pos] = tau_c[pos] / tot[pos]
    omega = kappa[None, :] * rho[None, :] * rate
    return omega, kappa
