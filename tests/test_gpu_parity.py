"""GPU parity: every libchem entry point against the CPU FP64 oracle on the same seeded inputs.

Tolerances (written here, derived in the design notes):
* rates, Jacobian: FP64 with a different summation order; compared against the gross rate
  scale sum_j |nu_kj q_j| (resp. the row's largest entry) at 1e-11 (resp. 1e-9);
* thermo properties: 1e-12 relative in FP64 mode, 2e-5 in the FP32-mixing mode;
* direct integration (Eq. 2): 1e-6 relative on T and on every Y_k the oracle puts above 1e-10.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2402_18858_gb300 import workload as w  # noqa: E402

DI_RTOL = 1e-6
Y_FLOOR = 1e-10


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


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def di_parity(T_g, Y_g, T_o, Y_o):
    """Per-cell pass mask of the 1e-6 relative criterion (T and Y_k > 1e-10)."""
    okT = np.abs(T_g - T_o) <= DI_RTOL * np.abs(T_o)
    big = Y_o > Y_FLOOR
    okY = np.where(big, np.abs(Y_g - Y_o) <= DI_RTOL * np.abs(Y_o), True).all(axis=0)
    return okT & okY


# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n", [("h2_9", 1000), ("c_30", 333), ("c_53", 130)])
def test_rates_parity(lc, gmech, mechs, oracles, kind, n):
    m, _ = mechs[kind]
    o = oracles[kind]
    st = w.make_states(m, n, 21)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    wdot = torch.empty_like(Y)
    hrr = torch.empty_like(T)
    lc.chem_rates(gmech[kind], T, p, Y, wdot, hrr)
    torch.cuda.synchronize()
    wd, hr = wdot.cpu().numpy(), hrr.cpu().numpy()
    nu = np.zeros((m.n_species, m.n_reactions))
    for j, r in enumerate(m.reactions):
        for k in r.reactants:
            nu[k, j] -= 1
        for k in r.products:
            nu[k, j] += 1
    for i in range(n):
        wo, ho, q, _, _ = o.rates(st.T[i], st.p[i], st.Y[:, i], with_rxn=True)
        gross = np.abs(nu) @ np.abs(q)
        assert (np.abs(wd[:, i] - wo) <= 1e-11 * gross + 1e-300).all(), i
        cpR, hRT, _ = o.species_thermo(st.T[i])
        hgross = (np.abs(hRT * 8.314462618 * st.T[i]) * gross).sum()
        assert abs(hr[i] - ho) <= 1e-11 * hgross


@pytest.mark.parametrize("kind,n", [("h2_9", 70), ("c_30", 40), ("c_53", 12)])
def test_jacobian_parity(lc, gmech, mechs, oracles, kind, n):
    m, _ = mechs[kind]
    o = oracles[kind]
    st = w.make_states(m, n, 22)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    nn = m.n_species + 1
    jac = torch.empty(n * nn * nn, dtype=torch.float64, device="cuda")
    lc.chem_jacobian(gmech[kind], T, p, Y, jac)
    torch.cuda.synchronize()
    J = jac.cpu().numpy().reshape(n, nn, nn)
    for i in range(n):
        Jo = o.jacobian(st.p[i], np.concatenate([st.Y[:, i], [st.T[i]]]))
        scale = np.abs(Jo).max(axis=1, keepdims=True) + 1e-300
        assert (np.abs(J[i] - Jo) <= 1e-9 * scale).all(), i


@pytest.mark.parametrize("kind,n", [("h2_9", 1000), ("c_30", 1000), ("c_53", 300)])
def test_thermo_props_parity(lc, gmech, mechs, oracles, kind, n):
    m, _ = mechs[kind]
    o = oracles[kind]
    st = w.make_states(m, n, 23)
    T, Y = _dev(st.T), _dev(st.Y)
    outs = {}
    for mixed in (False, True):
        cp, h, mu, kap = (torch.empty_like(T) for _ in range(4))
        lc.thermo_props(gmech[kind], T, Y, cp, h, mu, kap, mixed_precision=mixed)
        torch.cuda.synchronize()
        outs[mixed] = [x.cpu().numpy() for x in (cp, h, mu, kap)]
    for i in range(0, n, max(1, n // 200)):
        ref = o.thermo_props(st.T[i], st.Y[:, i])
        for mixed, tol in ((False, 1e-12), (True, 2e-5)):
            cp, h, mu, kap = (x[i] for x in outs[mixed])
            assert cp == pytest.approx(ref[0], rel=1e-12)
            assert h == pytest.approx(ref[1], rel=1e-12, abs=1e-6 * abs(ref[0]))
            assert mu == pytest.approx(ref[2], rel=tol)
            assert kap == pytest.approx(ref[3], rel=tol)


def test_thermo_T_from_h(lc, gmech, mechs, oracles):
    m, _ = mechs["c_30"]
    o = oracles["c_30"]
    st = w.make_states(m, 500, 24)
    hs = np.array([o.thermo_props(st.T[i], st.Y[:, i])[1] for i in range(500)])
    T0 = _dev(np.full(500, 1000.0))
    Tout = torch.empty_like(T0)
    cp = torch.empty_like(T0)
    lc.thermo_props(gmech["c_30"], T0, _dev(st.Y), cp=cp, h_in=_dev(hs), T_out=Tout)
    torch.cuda.synchronize()
    assert np.allclose(Tout.cpu().numpy(), st.T, rtol=0, atol=1e-8)


def test_thermo_props_full_size_sampled(lc, gmech, mechs, oracles):
    """The benchmark's launches: FP64 properties of 1,000,000 cells of the 30-species workload in
    one call (the step's mode) and the mixed mode beside it; 400 sampled cells (and the ragged
    last one) against the oracle."""
    m, _ = mechs["c_30"]
    o = oracles["c_30"]
    cfg = w.WORKLOADS["di_c_30sp_1m"]
    st = w.make_states(m, cfg["n"], cfg["state_seed"])
    T, Y = _dev(st.T), _dev(st.Y)
    pick = np.sort(np.random.default_rng(1).choice(cfg["n"], 400, replace=False))
    pick[-1] = cfg["n"] - 1
    for mixed, tol in ((False, 1e-12), (True, 2e-5)):
        cp, h, mu, kap = (torch.empty_like(T) for _ in range(4))
        lc.thermo_props(gmech["c_30"], T, Y, cp, h, mu, kap, mixed_precision=mixed)
        torch.cuda.synchronize()
        got = [x.cpu().numpy() for x in (cp, h, mu, kap)]
        for i in pick:
            ref = o.thermo_props(st.T[i], st.Y[:, i])
            assert got[0][i] == pytest.approx(ref[0], rel=1e-12)
            assert got[1][i] == pytest.approx(ref[1], rel=1e-12, abs=1e-6 * abs(ref[0]))
            assert got[2][i] == pytest.approx(ref[2], rel=tol)
            assert got[3][i] == pytest.approx(ref[3], rel=tol)


# ------------------------------------------------------------------------------------------
def _run_di(lc, gm, st, dt, idx=None, **kw):
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    n = st.T.size if idx is None else idx.numel()
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    stats = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    ws = torch.zeros(lc.chem_workspace_bytes(gm, n), dtype=torch.uint8, device="cuda")
    lc.chem_step_di(gm, dt, T, p, Y, status, idx=idx, stats=stats, workspace=ws, **kw)
    torch.cuda.synchronize()
    return (T.cpu().numpy(), Y.cpu().numpy(), status.cpu().numpy(),
            stats.cpu().numpy().reshape(4, n))


@pytest.mark.parametrize("kind,n,dt", [("h2_9", 4096, 1e-6), ("c_30", 515, 5e-6), ("c_53", 131, 1e-5)])
def test_di_parity(lc, gmech, mechs, oracles, kind, n, dt):
    """Eq. 2 on the GPU equals the oracle's solution within 1e-6 (T and Y_k > 1e-10)."""
    m, _ = mechs[kind]
    o = oracles[kind]
    st = w.make_states(m, n, 100)
    Tg, Yg, sg, stats = _run_di(lc, gmech[kind], st, dt)
    To, Yo, so, _ = o.integrate_batch(st.T, st.p, st.Y, dt)
    assert (so == 0).all()
    assert (sg == 0).all(), np.bincount(sg)
    ok = di_parity(Tg, Yg, To, Yo)
    bad = np.where(~ok)[0]
    assert ok.all(), f"{bad.size} cells outside 1e-6, first {bad[:5]}"
    assert (stats[0] > 0).all()


def test_di_full_size_sampled(lc, gmech, mechs, oracles):
    """1,000,000 cells of the 30-species workload in one launch; 48 sampled cells vs oracle."""
    m, _ = mechs["c_30"]
    o = oracles["c_30"]
    cfg = w.WORKLOADS["di_c_30sp_1m"]
    st = w.make_states(m, cfg["n"], cfg["state_seed"])
    Tg, Yg, sg, _ = _run_di(lc, gmech["c_30"], st, cfg["dt"])
    assert (sg == 0).all(), np.bincount(sg)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(cfg["n"], 48, replace=False))
    pick[-1] = cfg["n"] - 1          # the ragged tail
    To, Yo, so, _ = o.integrate_batch(st.T[pick], st.p[pick], st.Y[:, pick], cfg["dt"])
    assert di_parity(Tg[pick], Yg[:, pick], To, Yo).all()
    # invariants at every cell: mass and elements
    assert np.abs(Yg.sum(0) - 1.0).max() < 1e-11
    el0 = m.comp.T @ (st.Y / m.W[:, None])
    el1 = m.comp.T @ (Yg / m.W[:, None])
    assert np.abs(el1 - el0).max() <= 1e-11 * np.abs(el0).max()


def test_di_edge_cases(lc, gmech, mechs):
    gm = gmech["h2_9"]
    m, _ = mechs["h2_9"]
    st = w.make_states(m, 37, 5)
    # n = 0 is a no-op
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    status = torch.zeros(37, dtype=torch.int32, device="cuda")
    lc.chem_step_di(gm, 1e-6, T, p, Y, status, n=0, workspace=ws)
    # dt = 0 leaves the state untouched
    Tg, Yg, sg, _ = _run_di(lc, gm, st, 0.0)
    assert (sg == 0).all() and np.array_equal(Tg, st.T) and np.array_equal(Yg, st.Y)
    # non-finite and non-positive temperature inputs are flagged and left as they were
    bad = w.States(T=st.T.copy(), p=st.p.copy(), Y=st.Y.copy())
    bad.T[3] = np.nan
    bad.T[7] = -5.0
    bad.Y[2, 11] = np.inf
    Tg, Yg, sg, _ = _run_di(lc, gm, bad, 1e-6)
    assert sg[3] == 3 and sg[11] == 3 and sg[7] == 4
    assert np.isnan(Tg[3]) and Tg[7] == -5.0
    ok = np.ones(37, bool)
    ok[[3, 7, 11]] = False
    assert (sg[ok] == 0).all()
    # a step budget of one step reports "max steps" and keeps the input
    Tg, Yg, sg, _ = _run_di(lc, gm, st, 1e-6, max_steps=1)
    assert (sg == 1).any()
    assert np.array_equal(Tg[sg == 1], st.T[sg == 1])
    # a too-small workspace is an API error
    from paper_2402_18858_gb300.chem import ChemError
    with pytest.raises(ChemError):
        lc.chem_step_di(gm, 1e-6, T, p, Y, status, workspace=torch.zeros(8, dtype=torch.uint8, device="cuda"))


def test_di_subset_index_and_batch_invariance(lc, gmech, mechs):
    """A cell's result is bit-identical alone, in a batch, through an index list and on rerun."""
    gm = gmech["c_30"]
    m, _ = mechs["c_30"]
    st = w.make_states(m, 300, 77)
    Tg, Yg, sg, _ = _run_di(lc, gm, st, 5e-6)
    Tg2, Yg2, _, _ = _run_di(lc, gm, st, 5e-6)
    assert np.array_equal(Tg, Tg2) and np.array_equal(Yg, Yg2)
    idx = torch.tensor([299, 5, 17, 150], dtype=torch.int32, device="cuda")
    Ti, Yi, si, _ = _run_di(lc, gm, st, 5e-6, idx=idx)
    sel = idx.cpu().numpy()
    assert (si == 0).all()
    assert np.array_equal(Ti[sel], Tg[sel]) and np.array_equal(Yi[:, sel], Yg[:, sel])
    untouched = np.setdiff1d(np.arange(300), sel)
    assert np.array_equal(Ti[untouched], st.T[untouched])
    one = w.States(T=st.T[150:151].copy(), p=st.p[150:151].copy(), Y=st.Y[:, 150:151].copy())
    T1, Y1, s1, _ = _run_di(lc, gm, one, 5e-6)
    assert T1[0] == Tg[150] and np.array_equal(Y1[:, 0], Yg[:, 150])


def test_fp64_probe(lc):
    g = lc.chem_fp64_peak_gflops()
    assert 100.0 < g < 100000.0


def test_table_exp_against_cuda_exp(lc, gmech):
    """The kernels' table-driven FP64 exp stays within 2 ulp of CUDA's exp."""
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-708, 709.7, 200000), rng.uniform(-1, 1, 100000),
                        rng.uniform(-50, 50, 100000), [0.0, -0.0, 1e-300, -1e-300, 709.7, -708.0]])
    xd = _dev(x)
    y = torch.empty_like(xd)
    lc.chem_selftest_exp(gmech["h2_9"], xd, y)
    ref = torch.exp(xd)
    torch.cuda.synchronize()
    yy, rr = y.cpu().numpy(), ref.cpu().numpy()
    ulp = np.abs(yy - rr) / np.spacing(np.abs(rr))
    assert ulp.max() <= 2.0, (ulp.max(), x[np.argmax(ulp)])
    spec = _dev(np.array([np.nan, np.inf, -np.inf, -800.0, 800.0]))
    ys = torch.empty_like(spec)
    lc.chem_selftest_exp(gmech["h2_9"], spec, ys)
    torch.cuda.synchronize()
    v = ys.cpu().numpy()
    assert np.isnan(v[0]) and v[1] == np.inf and v[2] == 0.0 and v[3] == 0.0 and v[4] == np.inf


def test_scaled_exp_against_exp2(lc, gmech):
    """The kernels' FP64 exponential of pre-scaled arguments, 2^(x/256), stays within 2 ulp of
    exp2(x/256) over the range the rate and equilibrium constants use, and handles the ends."""
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-261485.0, 262143.9, 200000), rng.uniform(-300, 300, 100000),
                        rng.uniform(-20000, 20000, 100000), [0.0, -0.0, 1e-300, 256.0, -256.0, 262143.9]])
    xd = _dev(x)
    y = torch.empty_like(xd)
    lc.chem_selftest_exp256(gmech["h2_9"], xd, y)
    torch.cuda.synchronize()
    yy, rr = y.cpu().numpy(), np.exp2(x / 256.0)
    ulp = np.abs(yy - rr) / np.spacing(np.abs(rr))
    assert ulp.max() <= 2.0, (ulp.max(), x[np.argmax(ulp)])
    assert yy[x == 0.0][0] == 1.0 and yy[x == 256.0][0] == 2.0
    spec = _dev(np.array([np.nan, np.inf, -np.inf, -300000.0, 262144.0, 1e300]))
    ys = torch.empty_like(spec)
    lc.chem_selftest_exp256(gmech["h2_9"], spec, ys)
    torch.cuda.synchronize()
    v = ys.cpu().numpy()
    assert np.isnan(v[0]) and v[1] == np.inf and v[2] == 0.0 and v[3] == 0.0 and v[4] == np.inf and v[5] == np.inf


def test_reciprocal_against_division(lc):
    """The kernels' FP64 reciprocal (hardware estimate, one third-order step) stays within 1 ulp
    of the correctly rounded 1/x over the normal range, and gives NaN for 0 and inf."""
    rng = np.random.default_rng(6)
    x = np.concatenate([np.exp(rng.uniform(-700, 700, 300000)), rng.uniform(0.5, 2.0, 200000),
                        -np.exp(rng.uniform(-50, 50, 100000)), rng.uniform(200.0, 4000.0, 100000),
                        [1.0, 2.0, 3.0, 0.1, 1.0 - 2.0 ** -53, 1.0 + 2.0 ** -52]])
    xd = _dev(x)
    y = torch.empty_like(xd)
    lc.chem_selftest_rcp(xd, y)
    torch.cuda.synchronize()
    yy, rr = y.cpu().numpy(), 1.0 / x
    ulp = np.abs(yy - rr) / np.spacing(np.abs(rr))
    assert ulp.max() <= 1.0, (ulp.max(), x[np.argmax(ulp)])
    assert yy[x == 1.0][0] == 1.0 and yy[x == 2.0][0] == 0.5
    spec = _dev(np.array([0.0, np.inf, -np.inf]))
    ys = torch.empty_like(spec)
    lc.chem_selftest_rcp(spec, ys)
    torch.cuda.synchronize()
    assert np.isnan(ys.cpu().numpy()).all()


def test_table_log_against_cuda_log(lc, gmech):
    """The kernels' table-driven FP64 log stays within 3 ulp of CUDA's log, including near 1
    (its own error is about 2 ulp at most, CUDA's under 1)."""
    rng = np.random.default_rng(4)
    x = np.concatenate([np.exp(rng.uniform(-700, 700, 200000)), rng.uniform(200, 4000, 100000),
                        1.0 + rng.uniform(-0.05, 0.05, 100000), 1.0 + rng.uniform(-1e-6, 1e-6, 50000),
                        rng.uniform(0.5, 2.0, 100000),
                        [1.0, 2.0, 0.5, 0.75, 1.5, 1.4999999999999998, 2.2250738585072014e-308, 1.7976931348623157e308]])
    xd = _dev(x)
    y = torch.empty_like(xd)
    lc.chem_selftest_log(gmech["h2_9"], xd, y)
    ref = torch.log(xd)
    torch.cuda.synchronize()
    yy, rr = y.cpu().numpy(), ref.cpu().numpy()
    ulp = np.abs(yy - rr) / np.spacing(np.maximum(np.abs(rr), np.finfo(np.float64).tiny))
    assert ulp.max() <= 3.0, (ulp.max(), x[np.argmax(ulp)])
    assert yy[x == 1.0][0] == 0.0
    spec = _dev(np.array([0.0, -1.0, np.inf, np.nan, 5e-324]))
    ys = torch.empty_like(spec)
    lc.chem_selftest_log(gmech["h2_9"], spec, ys)
    torch.cuda.synchronize()
    v = ys.cpu().numpy()
    assert v[0] == -np.inf and np.isnan(v[1]) and v[2] == np.inf and np.isnan(v[3])
    assert abs(v[4] - np.log(5e-324)) < 1e-12 * abs(np.log(5e-324))
