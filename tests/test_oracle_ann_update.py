"""Pins of the oracle's learned-step update (`oracle.mlp.ann_update`) against facts other than
itself: the paper's output definition (Sec. 2.2: the network predicts the change of the Box-Cox
transformed species, Eq. 7, over the flow step; T follows from the constant-pressure energy
balance) and the fallback rules (range, non-finite values, element conservation, temperature).
"""
import os

import numpy as np
import pytest

from oracle import Oracle, mlp
from paper_2402_18858_gb300 import workload as w

from conftest import GOLDEN

P = 101325.0


def test_identity_when_the_prediction_is_the_integrated_state(oracles, mechs):
    """A network output equal to the transformed change of an exact step (the oracle
    integrator's Eq. 2 result, which conserves mass, elements and enthalpy) is returned as
    that state: the renormalisation and the projection change nothing and T' from
    h(T', Y') = h(T, Y) is the integrator's temperature."""
    o = oracles["c_30"]
    m, _ = mechs["c_30"]
    st = w.make_states(m, 12, 31)
    T1, Y1, s, _ = o.integrate_batch(st.T, st.p, st.Y, 5e-6)
    assert (s == 0).all()
    Y1 = np.maximum(Y1, 0.0)          # the update's F clips at 0
    Y1 /= Y1.sum(axis=0)
    U = (mlp.bct(Y1) - mlp.bct(st.Y)).T
    K = m.n_species
    Tn, Yn, fl, _ = mlp.ann_update(o, st.T, st.Y, U, np.zeros(K), np.ones(K), elem_tol=1e-2,
                                   T_max=6000.0)
    assert (fl == 0).all()
    big = Y1 > 1e-12
    assert np.allclose(Yn[big], Y1[big], rtol=1e-9, atol=0)
    assert np.abs(Yn - Y1).max() < 1e-13
    assert np.allclose(Tn, T1, rtol=0, atol=1e-6)


def test_hand_computed_projection():
    """isomer.mech: A and B carry element X (same W, same enthalpy), N2 carries N.  From
    Y = (0.6, 0.1, 0.3) a prediction (0.5, 0.25, 0.25) has 7 % too much X and 17 % too little N;
    the weighted projection restores each element's mass in proportion to the prediction:
    A + B = 0.7 split 2:1 and N2 = 0.3.  T is unchanged: the X species' mass enthalpies are
    equal and N2 returns to its old fraction."""
    o = Oracle(os.path.join(GOLDEN, "isomer.mech"))
    Y = np.array([[0.6], [0.1], [0.3]])
    pred = np.array([0.5, 0.25, 0.25])
    U = (mlp.bct(pred) - mlp.bct(Y[:, 0]))[None, :]
    Tn, Yn, fl, info = mlp.ann_update(o, np.array([1200.0]), Y, U, np.zeros(3), np.ones(3),
                                      elem_tol=0.2)
    assert fl[0] == 0
    # largest relative change of element moles: X 0.05/0.7, N 0.05/0.3
    assert info["elem_residual"][0] == pytest.approx(0.05 / 0.3, rel=1e-12)
    assert np.allclose(Yn[:, 0], [0.7 * 2 / 3, 0.7 / 3, 0.3], rtol=1e-13, atol=0)
    assert Tn[0] == pytest.approx(1200.0, abs=1e-8)


def test_projection_conserves_elements_exactly(oracles, mechs):
    o = oracles["c_30"]
    m, _ = mechs["c_30"]
    n, K = 200, m.n_species
    st = w.make_states(m, n, 32)
    rng = np.random.default_rng(5)
    U = 0.05 * rng.standard_normal((n, K))
    Tn, Yn, fl, info = mlp.ann_update(o, st.T, st.Y, U, np.zeros(K), np.ones(K), elem_tol=0.5,
                                      T_max=6000.0)
    ok = fl == 0
    assert ok.mean() > 0.9
    Cm = o.comp / o.W[:, None]
    e0 = Cm.T @ st.Y[:, ok]
    e1 = Cm.T @ Yn[:, ok]
    assert np.allclose(e1, e0, rtol=1e-12, atol=0)
    assert np.allclose(Yn[:, ok].sum(axis=0), 1.0, rtol=0, atol=1e-12)
    assert (Yn >= 0).all()
    # the enthalpy of the new state equals the old one (adiabatic, constant p)
    for i in np.where(ok)[0][:20]:
        h0 = o.thermo_props(st.T[i], st.Y[:, i])[1]
        h1 = o.thermo_props(Tn[i], Yn[:, i])[1]
        assert h1 == pytest.approx(h0, rel=1e-10, abs=1e-4)


def test_flag_rules(oracles, mechs):
    o = oracles["c_30"]
    m, _ = mechs["c_30"]
    K = m.n_species
    st = w.make_states(m, 8, 33, T_range=(1200.0, 1300.0))
    T, Y = st.T, st.Y
    zero, one = np.zeros(K), np.ones(K)
    U = np.zeros((8, K))
    U[1, 3] = np.inf                       # non-finite output
    U[2, 4] = np.nan
    U[3, :] = 2.0                          # every species up: fine after renormalisation ...
    U[3, 0] = -30.0                        # ... but one species removed: element residual
    flags_in = np.zeros(8, np.int32)
    flags_in[4] = mlp.FLAG_RANGE
    # cell 5: the unchanged state but a temperature window that excludes it
    Tn, Yn, fl, info = mlp.ann_update(o, T, Y, U, zero, one, elem_tol=1e-2, flags_in=flags_in)
    assert fl[0] == 0 and fl[1] == mlp.FLAG_NONFINITE and fl[2] == mlp.FLAG_NONFINITE
    assert fl[3] & mlp.FLAG_ELEMENTS and fl[4] == mlp.FLAG_RANGE
    assert info["elem_residual"][0] < 1e-14        # zero output: the state itself
    assert Tn[0] == pytest.approx(T[0], abs=1e-8)
    for i in (1, 2, 3, 4):                         # flagged cells keep their state
        assert Tn[i] == T[i] and np.array_equal(Yn[:, i], Y[:, i])
    _, _, fl2, _ = mlp.ann_update(o, T, Y, np.zeros((8, K)), zero, one, T_min=250.0,
                                  T_max=1250.0)
    assert ((fl2 == mlp.FLAG_T_RANGE) == (T > 1250.0)).all()
    # a 100 K temperature change from a shifted enthalpy: changed composition, |dT| cap
    U5 = np.zeros((8, K))
    U5[:, 0] = 1.0
    _, _, _, inf5 = mlp.ann_update(o, T, Y, U5, zero, one, elem_tol=1.0)
    dT = np.abs(inf5["T_prime"] - T)
    cap = float(np.median(dT))
    _, _, fl5, _ = mlp.ann_update(o, T, Y, U5, zero, one, elem_tol=1.0, dT_max=cap)
    assert ((fl5 == mlp.FLAG_DT) == (dT > cap)).all()
    # the range flag of the inputs against the training limits
    rf, raw = mlp.range_flags(T, st.p, Y, np.concatenate([[1200, P], mlp.bct(Y).min(1)]),
                              np.concatenate([[1250, P], mlp.bct(Y).max(1)]), 0.0)
    assert ((rf == mlp.FLAG_RANGE) == (T > 1250)).all()
