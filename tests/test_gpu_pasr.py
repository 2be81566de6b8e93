"""GPU parity of the PaSR filtered source (chem_pasr_source) against the FP64 oracle.

Inputs: seeded states Y0 (the workload generator), Y1 = Y0 plus seeded changes of mixed sign
and size (exact zeros, rounding-level changes, trace species, large changes), and seeded
sub-grid fields with laminar cells.  No input or expected value comes from the CUDA path.

Tolerance: the mixing time is FP32 from correctly rounded inputs (a few FP32 ulp, < 1e-6
relative) and enters kappa = tau_c / (tau_c + tau_mix) with a factor below 1; the search for
the slowest formation compares FP32 cross products, so a near-tie (within 1e-6) may pick the
other species, whose formation time is then within 1e-6 -- so kappa within 2e-6 relative, and
omega = kappa rho dY / dt within 2e-6 relative per entry (the FP64 difference and product
add a few ulp).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.pasr import pasr_source  # noqa: E402
from paper_2402_18858_gb300 import workload as w  # noqa: E402

TOL = 2e-6


@pytest.fixture(scope="module")
def lc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem
    build.build()
    chem.lib()
    return chem


@pytest.fixture(scope="module")
def gmech(lc, mechs):
    return {k: lc.chem_load_mech(p) for k, (m, p) in mechs.items()}


def _step_like(Y0, seed):
    """Seeded 'after the step' states: relative changes of all sizes and both signs."""
    rng = np.random.default_rng(seed)
    K, N = Y0.shape
    mag = 10.0 ** rng.uniform(-17, -0.5, size=(K, N))            # rounding level .. large
    dY = np.sign(rng.standard_normal((K, N))) * mag * np.abs(Y0)
    dY[rng.random((K, N)) < 0.05] = 0.0                           # species at rest
    Y1 = np.maximum(Y0 + dY, 0.0)
    trace = rng.random((K, N)) < 0.02                            # trace species that grow
    Y1[trace] = 10.0 ** rng.uniform(-14, -11, trace.sum())
    Y0[trace] = 0.5 * Y1[trace]
    return Y0, Y1


def _run(lc, gm, Y0, Y1, tf, dt, n=None, ld_pad=0, with_kappa=True, y_min=-1.0, r_min=-1.0):
    K, N = Y0.shape
    ld = N + ld_pad
    dev = torch.device("cuda")

    def col(a):
        t = torch.zeros((K, ld), dtype=torch.float64, device=dev)
        t[:, :N] = torch.as_tensor(a, device=dev)
        return t
    y0, y1 = col(Y0), col(Y1)
    per = [torch.as_tensor(np.pad(a, (0, ld_pad)), device=dev) for a in (tf.rho, tf.k, tf.eps, tf.nu)]
    om = torch.full((K, ld), np.nan, dtype=torch.float64, device=dev)
    kap = torch.full((ld,), np.nan, dtype=torch.float64, device=dev) if with_kappa else None
    lc.chem_pasr_source(gm, dt, per[0], y0, y1, per[1], per[2], per[3], om, kap, y_min=y_min, r_min=r_min,
                        n=N if n is None else n)
    torch.cuda.synchronize()
    return om.cpu().numpy(), (kap.cpu().numpy() if kap is not None else None)


def _compare(om, kap, Y0, Y1, tf, dt, n, **kw):
    om_o, kap_o = pasr_source(tf.rho[:n], Y0[:, :n], Y1[:, :n], dt, tf.k[:n], tf.eps[:n], tf.nu[:n], **kw)
    if kap is not None:
        assert np.all(np.abs(kap[:n] - kap_o) <= TOL * kap_o + 1e-300), np.abs(kap[:n] - kap_o).max()
    tol = TOL * np.abs(om_o) + 1e-300
    assert np.all(np.abs(om[:, :n] - om_o) <= tol)
    return kap_o


@pytest.mark.parametrize("kind,n", [("h2_9", 4099), ("c_30", 3001), ("c_53", 1003)])
def test_pasr_parity(lc, gmech, mechs, kind, n):
    m, _ = mechs[kind]
    st = w.make_states(m, n, 41)
    Y0, Y1 = _step_like(st.Y.copy(), 42)
    tf = w.make_turbulence(n, 43)
    dt = 5e-6
    om, kap = _run(lc, gmech[kind], Y0, Y1, tf, dt)
    kap_o = _compare(om, kap, Y0, Y1, tf, dt, n)
    # the cases the model has: laminar cells (kappa = 1), turbulent cells with kappa in (0, 1)
    assert (kap_o[tf.k == 0.0] == 1.0).all()
    assert ((kap_o > 0) & (kap_o < 1)).sum() > n // 2


def test_pasr_edge_cases(lc, gmech, mechs):
    m, _ = mechs["c_30"]
    gm = gmech["c_30"]
    n, dt = 777, 1e-6
    st = w.make_states(m, n, 44)
    Y0, Y1 = _step_like(st.Y.copy(), 45)
    Y1[:, :5] = Y0[:, :5]                 # no change at all: tau_c = 0
    tf = w.make_turbulence(n, 46)
    # partial n with a padded leading dimension; entries past n stay untouched
    om, kap = _run(lc, gm, Y0, Y1, tf, dt, n=700, ld_pad=13)
    _compare(om, kap, Y0, Y1, tf, dt, 700)
    assert np.isnan(om[:, 700:]).all() and np.isnan(kap[700:]).all()
    assert (kap[:5][tf.k[:5] > 0] == 0.0).all()
    # kappa not requested; explicit thresholds
    om2, _ = _run(lc, gm, Y0, Y1, tf, dt, with_kappa=False, y_min=1e-6, r_min=1e-4)
    _compare(om2, None, Y0, Y1, tf, dt, n, y_min=1e-6, r_min=1e-4)
    # n = 0 is a no-op; bad dt is rejected
    om3, _ = _run(lc, gm, Y0, Y1, tf, dt, n=0)
    assert np.isnan(om3).all()
    with pytest.raises(lc.ChemError):
        _run(lc, gm, Y0, Y1, tf, 0.0)


def test_pasr_full_size_sampled(lc, gmech, mechs):
    """The 1,000,000-cell 30-species launch of the benchmark, checked on a seeded sample."""
    m, _ = mechs["c_30"]
    n, dt = 1_000_000, 5e-6
    st = w.make_states(m, n, 47)
    Y0, Y1 = _step_like(st.Y.copy(), 48)
    tf = w.make_turbulence(n, 49)
    om, kap = _run(lc, gmech["c_30"], Y0, Y1, tf, dt)
    idx = np.sort(np.random.default_rng(50).choice(n, 20_000, replace=False))
    sub = w.TurbulenceFields(rho=tf.rho[idx], k=tf.k[idx], eps=tf.eps[idx], nu=tf.nu[idx])
    _compare(om[:, idx], kap[idx], Y0[:, idx], Y1[:, idx], sub, dt, len(idx))
