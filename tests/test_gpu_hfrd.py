"""GPU parity of the HFRD augmentation (chem_hfrd_augment, Eqs. 3-6) against the FP64 oracle.

Inputs: seeded workload states and seeded uniform draws gamma in [-1, 1] (the same array for
both sides).  Tolerance: T' and p' are one FMA each (1e-15 relative); Y' = Y^(1 + theta
gamma) / sum uses the library pow on both sides (within 2 ulp each) and sums in different
orders, so 1e-13 relative.  The keep flags are compared exactly except for states whose
element ratios lie within 1e-9 (relative) of a bound, where the two sides' different
rounding orders (and the mechanism file's printed molar masses) may decide either way.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import hfrd  # noqa: E402
from paper_2402_18858_gb300 import workload as w  # noqa: E402


@pytest.fixture(scope="module")
def lc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem
    build.build()
    chem.lib()
    return chem


def _margin(lo_hi, x):
    lo, hi = lo_hi
    return np.minimum(np.abs(x - lo) / abs(lo), np.abs(x - hi) / abs(hi))


@pytest.mark.parametrize("kind,n", [("c_30", 20011), ("h2_9", 5003)])
def test_hfrd_parity(lc, mechs, kind, n):
    m, path = mechs[kind]
    gm = lc.chem_load_mech(path)
    st = w.make_states(m, n, 61)
    K = m.n_species
    gamma = np.random.default_rng(62).uniform(-1.0, 1.0, size=(3 + K, n))
    dev = torch.device("cuda")
    T, p, Y, g = (torch.as_tensor(a, device=dev) for a in (st.T, st.p, st.Y, gamma))
    To, po, Yo = torch.empty_like(T), torch.empty_like(p), torch.empty_like(Y)
    keep = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.empty(lc.chem_hfrd_workspace_bytes(), dtype=torch.uint8, device=dev)
    lc.chem_hfrd_augment(gm, T, p, Y, g, To, po, Yo, keep, ws)
    torch.cuda.synchronize()
    comp = np.asarray(m.comp, dtype=np.float64).T            # [E, K]
    W = np.asarray(m.W, dtype=np.float64)
    i_n2 = list(m.species).index("N2")
    rng = hfrd.data_ranges(st.T, st.p, st.Y[i_n2])
    Tr, pr, Yr, ok = hfrd.augment(st.T, st.p, st.Y, gamma, i_n2, comp, W, list(m.elements), rng)
    np.testing.assert_allclose(To.cpu().numpy(), Tr, rtol=1e-15)
    np.testing.assert_allclose(po.cpu().numpy(), pr, rtol=1e-15)
    np.testing.assert_allclose(Yo.cpu().numpy(), Yr, rtol=1e-13, atol=1e-300)
    kg = keep.cpu().numpy().astype(bool)
    e = hfrd.element_moles(Yr, comp, W)
    E = list(m.elements)
    nH, nO, nN = e[E.index("H")], e[E.index("O")], e[E.index("N")]
    near = _margin(hfrd.ON_RANGE, nO / nN) < 1e-9
    num = 0.5 * nH
    if "C" in E:
        nC = e[E.index("C")]
        near |= _margin(hfrd.HC_RANGE, nH / nC) < 1e-9
        num = num + 2.0 * nC
    near |= _margin(hfrd.PHI_RANGE, num / nO) < 1e-9
    assert (kg[~near] == ok[~near]).all()
    # both outcomes occur on this workload
    assert 0 < ok.sum() < n


def test_hfrd_in_place_and_options(lc, mechs):
    m, path = mechs["c_30"]
    gm = lc.chem_load_mech(path)
    n = 3001
    st = w.make_states(m, n, 63)
    K = m.n_species
    gamma = np.random.default_rng(64).uniform(-1.0, 1.0, size=(3 + K, n))
    dev = torch.device("cuda")
    T, p, Y, g = (torch.as_tensor(a, device=dev) for a in (st.T, st.p, st.Y, gamma))
    keep = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.empty(lc.chem_hfrd_workspace_bytes(), dtype=torch.uint8, device=dev)
    opts = dict(alpha=0.05, beta=0.0, theta=0.2, hc=(0.0, 1e9), on=(0.0, 1e9), phi=(0.0, 1e9))
    lc.chem_hfrd_augment(gm, T, p, Y, g, T, p, Y, keep, ws, opts=opts)   # outputs over the inputs
    torch.cuda.synchronize()
    comp = np.asarray(m.comp, dtype=np.float64).T
    i_n2 = list(m.species).index("N2")
    rng = hfrd.data_ranges(st.T, st.p, st.Y[i_n2])
    Tr, pr, Yr, ok = hfrd.augment(st.T, st.p, st.Y, gamma, i_n2, comp, np.asarray(m.W, dtype=np.float64),
                                  list(m.elements), rng, alpha=0.05, beta=0.0, theta=0.2,
                                  hc=(0.0, 1e9), on=(0.0, 1e9), phi_range=(0.0, 1e9))
    np.testing.assert_allclose(T.cpu().numpy(), Tr, rtol=1e-15)
    np.testing.assert_allclose(Y.cpu().numpy(), Yr, rtol=1e-13, atol=1e-300)
    assert (keep.cpu().numpy().astype(bool) == ok).all() and ok.all()
