"""Seeded input generators: determinism, element balance, state validity."""
import numpy as np
import pytest

from paper_2402_18858_gb300 import workload as w


@pytest.mark.parametrize("kind,seed,nr,ntb,ntroe", [("h2_9", 0, 24, 3, 0), ("c_30", 1, 180, 6, 8),
                                                    ("c_53", 5, 320, 10, 12)])
def test_mechanism_counts_and_balance(mechs, kind, seed, nr, ntb, ntroe):
    m, _ = mechs[kind]
    assert m.n_reactions == nr
    kinds = [r.kind for r in m.reactions]
    assert kinds.count(1) == ntb and kinds.count(2) == ntroe
    inert = m.index("N2")
    for r in m.reactions:
        assert (m.comp[r.reactants].sum(0) == m.comp[r.products].sum(0)).all()
        assert inert not in r.reactants + r.products
    # every non-inert species takes part in some reaction
    used = set()
    for r in m.reactions:
        used.update(r.reactants + r.products)
    assert used == set(range(m.n_species)) - {inert}
    assert abs(m.T_ad_stoich - 2300.0) < 1.0


def test_mechanism_seeded_determinism(tmp_path):
    a, b = tmp_path / "a.mech", tmp_path / "b.mech"
    w.write_mechanism(w.make_mechanism("c_30", 1), str(a))
    w.write_mechanism(w.make_mechanism("c_30", 1), str(b))
    assert a.read_text() == b.read_text()
    c = tmp_path / "c.mech"
    w.write_mechanism(w.make_mechanism("c_30", 2), str(c))
    assert a.read_text() != c.read_text()


def test_states(mechs):
    m, _ = mechs["c_30"]
    s = w.make_states(m, 1000, 7)
    assert s.Y.shape == (30, 1000)
    assert np.allclose(s.Y.sum(0), 1.0, rtol=0, atol=1e-14)
    assert (s.Y > 0).all()
    assert s.T.min() >= 300 and s.T.max() <= 2500
    s2 = w.make_states(m, 1000, 7)
    assert np.array_equal(s.Y, s2.Y) and np.array_equal(s.T, s2.T)


def test_unburnt_burnt_element_balance(mechs):
    # complete combustion conserves the elements of the fresh mixture
    m, _ = mechs["c_30"]
    phi = np.linspace(0.6, 1.0, 5)
    nu, nb = w.unburnt_and_burnt_moles(m, phi)
    assert np.allclose(m.comp.T @ nu, m.comp.T @ nb, rtol=1e-14)
    assert (nb >= -1e-15).all()
