"""Pins of the HFRD augmentation oracle (CPU): identity at gamma = 0, Eq. 6 at gamma = +-1,
Eqs. 3-5 by hand, element ratios of a hand-built methane-air state, constraint boundaries."""
import numpy as np

from oracle import hfrd

# a small C/H/O/N species set: CH4, O2, N2, H2O, CO2 (atoms per molecule, element order C H O N)
ELEMENTS = ["C", "H", "O", "N"]
COMP = np.array([[1, 0, 0, 0, 1],      # C
                 [4, 0, 0, 2, 0],      # H
                 [0, 2, 0, 1, 2],      # O
                 [0, 0, 2, 0, 0]], dtype=np.float64)   # N
W = np.array([16.043e-3, 31.998e-3, 28.014e-3, 18.015e-3, 44.009e-3])
I_N2 = 2


def _methane_air(phi):
    """Mass fractions of CH4 + (2/phi)(O2 + 3.76 N2)."""
    n = np.array([1.0, 2.0 / phi, 2.0 / phi * 3.76, 0.0, 0.0])
    m = n * W
    return m / m.sum()


def test_gamma_zero_is_the_identity_and_ratios_are_hand_computed():
    Y = np.stack([_methane_air(0.7), _methane_air(1.0), _methane_air(1.3)], axis=1)
    T = np.array([400.0, 800.0, 1200.0])
    p = np.full(3, 101325.0)
    rng = hfrd.data_ranges(T, p, Y[I_N2])
    assert rng["dT"] == 800.0 and rng["dp"] == 0.0
    Tn, pn, Yn, ok = hfrd.augment(T, p, Y, np.zeros((3 + 5, 3)), I_N2, COMP, W, ELEMENTS, rng)
    assert (Tn == T).all() and (pn == p).all()
    np.testing.assert_allclose(Yn, Y, rtol=1e-15)
    # element-based phi and ratios of CH4 + (2/phi)(O2 + 3.76 N2): H/C = 4, O/N = 1/3.76
    e = hfrd.element_moles(Yn, COMP, W)
    np.testing.assert_allclose(e[1] / e[0], 4.0, rtol=1e-13)
    np.testing.assert_allclose(e[2] / e[3], 1.0 / 3.76, rtol=1e-13)
    np.testing.assert_allclose((2 * e[0] + 0.5 * e[1]) / e[2], [0.7, 1.0, 1.3], rtol=1e-13)
    # H/C = 4 and O/N = 0.266 pass; phi = 1.3 is outside [0.20, 1.15]
    assert ok.tolist() == [True, True, False]


def test_equations_3_to_6_by_hand():
    T = np.array([500.0, 1500.0])
    p = np.array([1.0e5, 1.2e5])
    Y = np.stack([_methane_air(0.8), _methane_air(0.9)], axis=1)
    rng = hfrd.data_ranges(T, p, Y[I_N2])
    g = np.zeros((8, 2))
    g[0] = [1.0, -0.5]          # T
    g[1] = [0.25, 0.0]          # p
    g[2] = [0.0, 0.0]           # N2
    g[3:] = np.array([1.0, -1.0, 0.0, 0.0, 0.0])[:, None]   # CH4 ^ 1.1, O2 ^ 0.9
    Tn, pn, Yn, ok = hfrd.augment(T, p, Y, g, I_N2, COMP, W, ELEMENTS, rng)
    np.testing.assert_allclose(Tn, [500.0 + 0.125 * 1000.0, 1500.0 - 0.5 * 0.125 * 1000.0], rtol=1e-15)
    np.testing.assert_allclose(pn, [1.0e5 + 10.0 * 0.25 * 2.0e4, 1.2e5], rtol=1e-15)
    raw = Y.copy()
    raw[0] = Y[0] ** 1.1
    raw[1] = Y[1] ** 0.9
    np.testing.assert_allclose(Yn, raw / raw.sum(axis=0), rtol=1e-14)
    # N2 shift (Eq. 5) by alpha gamma (range) before the renormalisation
    g2 = np.zeros((8, 2))
    g2[2] = [1.0, 0.0]
    _, _, Yn2, _ = hfrd.augment(T, p, Y, g2, I_N2, COMP, W, ELEMENTS, rng)
    raw2 = Y.copy()
    raw2[I_N2, 0] += 0.125 * rng["dn2"]
    np.testing.assert_allclose(Yn2, raw2 / raw2.sum(axis=0), rtol=1e-14)


def test_constraint_boundaries():
    # a CH4/H2O/O2/N2 mixture whose H/C is moved across 4.67 by the water content
    def state(h2o):
        n = np.array([1.0, 2.0, 7.52, h2o, 0.0])
        m = n * W
        return m / m.sum()
    T = np.array([600.0, 600.0])
    p = np.full(2, 101325.0)
    # H/C = 4 + 2 n_H2O: 0.33 -> 4.66 (kept), 0.34 -> 4.68 (rejected)
    Y = np.stack([state(0.33), state(0.34)], axis=1)
    rng = hfrd.data_ranges(T, p, Y[I_N2])
    _, _, _, ok = hfrd.augment(T, p, Y, np.zeros((8, 2)), I_N2, COMP, W, ELEMENTS, rng)
    assert ok.tolist() == [True, False]
    # a negative N2 after Eq. 5 and a non-positive T after Eq. 3 are rejected
    Y = np.stack([_methane_air(1.0), _methane_air(0.5)], axis=1)
    T = np.array([300.0, 2300.0])
    rng = hfrd.data_ranges(T, p, Y[I_N2])
    g = np.zeros((8, 2))
    g[0, 0] = -1.0                                   # 300 - 0.125 * 2000 = 50 K > 0: kept
    g[2, 1] = -1.0                                   # N2 - 0.125 dN2 stays positive: kept
    _, _, _, ok = hfrd.augment(T, p, Y, g, I_N2, COMP, W, ELEMENTS, rng)
    assert ok.tolist() == [True, True]
    rng_big = dict(rng, dT=4000.0, dn2=100.0)
    _, _, _, ok = hfrd.augment(T, p, Y, g, I_N2, COMP, W, ELEMENTS, rng_big)
    assert ok.tolist() == [False, False]


def test_no_carbon_skips_the_hc_test():
    # H2/O2/N2/H2O only: the H/C test is skipped, O/N and phi still apply
    comp = np.array([[2, 0, 0, 2], [0, 2, 0, 1], [0, 0, 2, 0]], dtype=np.float64)   # H O N
    Wh = np.array([2.016e-3, 31.998e-3, 28.014e-3, 18.015e-3])
    n = np.array([1.4, 1.0, 3.76, 0.0])                        # phi = 0.7
    m = n * Wh
    Y = (m / m.sum())[:, None]
    _, _, _, ok = hfrd.augment(np.array([700.0]), np.array([101325.0]), Y, np.zeros((7, 1)), 2, comp, Wh,
                               ["H", "O", "N"], dict(dT=0.0, dp=0.0, dn2=0.0))
    assert ok.tolist() == [True]
