"""Random augmentation of training states (the hybrid flamelet/random data method, Sec. 2.2,
Eqs. 3-6) -- FP64 numpy oracle, test infrastructure only (the tests, the package's smoke check
and the benchmark's CPU-baseline leg use it; it imports nothing from the GPU package).

For every base state (T, p, Y) and its uniform draws gamma in [-1, 1] (passed in, so that the
oracle and the GPU kernel see the same numbers):

* T' = T + alpha gamma_T (T_max - T_min)                    (Eq. 3)
* p' = p + beta gamma_p (p_max - p_min)                     (Eq. 4)
* Y'_N2 = Y_N2 + alpha gamma_N2 (Y_N2,max - Y_N2,min)       (Eq. 5)
* Y'_j = Y_j^(1 + theta gamma_j) for every other species    (Eq. 6)

with alpha = 0.125, beta = 10, theta = 0.1 and the ranges taken over the base data set.  The
constraints of the same passage then decide which augmented states are kept: the mass
fractions are renormalised to sum to one (reading: divide by their sum), and the molar
element ratios H/C and O/N and the equivalence ratio must lie in the stated ranges
(H/C in [2.65, 4.67], O/N in [0.254, 0.320], phi in [0.20, 1.15]).  Readings: gamma is drawn
independently for T, p, N2 and each species; the equivalence ratio is the element-based
phi = (2 n_C + n_H / 2) / n_O over all species; a mechanism without carbon skips the H/C
test; a state with T' <= 0, p' <= 0 or Y'_N2 < 0 is rejected.

Parity: pinned by tests/test_oracle_hfrd.py (gamma = 0 is the identity; Eq. 6 at gamma = +-1 is
y^1.1 and y^0.9; hand-computed ranges and ratios; constraint boundaries).
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np

ALPHA, BETA, THETA = 0.125, 10.0, 0.1
HC_RANGE = (2.65, 4.67)
ON_RANGE = (0.254, 0.320)
PHI_RANGE = (0.20, 1.15)


def data_ranges(T: np.ndarray, p: np.ndarray, Y_n2: np.ndarray) -> Dict[str, float]:
    """Extents of the base data set entering Eqs. 3-5."""
    return dict(dT=float(T.max() - T.min()), dp=float(p.max() - p.min()), dn2=float(Y_n2.max() - Y_n2.min()))


def element_moles(Y: np.ndarray, comp: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Moles of each element per kg of mixture: comp [E, K] (atoms per molecule), W [K]."""
    return comp @ (Y / W[:, None])


def augment(T: np.ndarray, p: np.ndarray, Y: np.ndarray, gamma: np.ndarray, i_n2: int,
            comp: np.ndarray, W: np.ndarray, elements: Sequence[str], ranges: Dict[str, float],
            alpha: float = ALPHA, beta: float = BETA, theta: float = THETA,
            hc=HC_RANGE, on=ON_RANGE, phi_range=PHI_RANGE) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """T', p', Y' [K, N] and the kept mask [N] for N states; gamma [3 + K, N] (rows: T, p, N2,
    then one per species, the N2 row of the per-species block unused)."""
    T = np.asarray(T, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    K = Y.shape[0]
    Tn = T + alpha * gamma[0] * ranges["dT"]
    pn = p + beta * gamma[1] * ranges["dp"]
    expo = 1.0 + theta * gamma[3:3 + K]
    Yn = np.where(Y > 0.0, np.power(np.maximum(Y, 0.0), expo), 0.0)
    Yn[i_n2] = Y[i_n2] + alpha * gamma[2] * ranges["dn2"]
    s = Yn.sum(axis=0)
    ok = (Tn > 0.0) & (pn > 0.0) & (Yn[i_n2] >= 0.0) & (s > 0.0)
    Yn = Yn / np.where(s > 0.0, s, 1.0)
    e = element_moles(Yn, comp, W)
    idx = {name: i for i, name in enumerate(elements)}
    nC = e[idx["C"]] if "C" in idx else None
    nH, nO, nN = e[idx["H"]], e[idx["O"]], e[idx["N"]]
    if nC is not None:
        with np.errstate(divide="ignore", invalid="ignore"):
            r = nH / nC
        ok &= (nC > 0.0) & (r >= hc[0]) & (r <= hc[1])
        num = 2.0 * nC + 0.5 * nH
    else:
        num = 0.5 * nH
    with np.errstate(divide="ignore", invalid="ignore"):
        on_r = nO / nN
        phi = num / nO
    ok &= (nN > 0.0) & (on_r >= on[0]) & (on_r <= on[1])
    ok &= (nO > 0.0) & (phi >= phi_range[0]) & (phi <= phi_range[1])
    return Tn, pn, Yn, ok
