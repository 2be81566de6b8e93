"""GPU parity of the learned step's update stage and of its fallback (Sec. 2.2 output
definition with Eq. 7; fallback rules: range, non-finite values, element conservation,
temperature range, |dT| cap).

* update: `chem_ann_update` (FP32 kernel) against `oracle.mlp.ann_update` (FP64), element by
  element, on network outputs of the committed network for 3,000 cells of the 30-species
  workload taken through a shuffled index list, with rows edited so that every flag occurs.
  Bounds, from the arithmetic of the kernel (FP32 up to the projection, which is FP64):
    - Y*_k: the inverse Box-Cox Y = t^10, t = 0.1 z + 1, amplifies the absolute FP32 error of
      z (a few units of eps32 times |z| <= ~10, so |dt| <~ 4 eps32) tenfold in relative terms:
      r_k = 64 eps32 / t_k (t = Y^0.1 of the oracle's result);
    - the projection onto element conservation is an orthogonal projection in the metric
      diag(1/Y*), hence non-expansive there: the projected states differ by at most
      sqrt(Y_k) sqrt(sum_j r_j^2 Y_j) besides each species' own r_k Y_k;
      |dY_k| <= r_k Y_k + sqrt(Y_k) sqrt(sum_j r_j^2 Y_j) + 1e-25; and the GPU's result
      conserves the elements to FP64 rounding;
    - T: the enthalpy sums h = sum_k Y_k h_k in FP32 carry about 8 eps32 sum_k |Y_k h_k| each
      (old and new state): |dT| <= 32 eps32 (sum |Y h_k(T)| + sum |Y' h_k(T')|) / c_p + 1e-3 K
      (the Newton stop at |dT| < 1e-4 T leaves well under 1e-3 K).
  Flags are decided in FP32 on the GPU and in FP64 in the oracle: a cell whose deciding
  quantity lies within the FP32 error of a threshold (element residual within 2e-5 of
  elem_tol, T' within 0.05 K of T_min, T_max or T +- dT_max) may go either way and is left out
  of the comparison; every other cell's flag word must match exactly.
* stages: chem_step_ann without fallback equals features -> forward -> update bit for bit.
* fallback (a12): every cell that chem_step_ann hands to DI (status 5) is bit-identical to
  chem_step_di on that cell with the same DI options, through an index list too.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp  # noqa: E402
from paper_2402_18858_gb300 import workload as w  # noqa: E402

CKPT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2402_18858_gb300",
                    "models", "ann_c30_seed1.ckpt")
EPS32 = float(np.finfo(np.float32).eps)
R = 8.314462618
N = 3000


@pytest.fixture(scope="module")
def env(mechs, oracles):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem
    build.build()
    m, path = mechs["c_30"]
    gm = chem.chem_load_mech(path)
    ann = chem.chem_ann_load(gm, CKPT)
    st = w.make_states(m, N, 61)
    st.T[:7] = 2900.0                      # outside the training range of T (300-2500 K)
    dev = torch.device("cuda")
    T = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y = torch.as_tensor(st.Y, device=dev)
    X = torch.empty((N, 64), dtype=torch.bfloat16, device=dev)
    flags = torch.empty(N, dtype=torch.int32, device=dev)
    chem.chem_ann_features(ann, T, p, Y, X, flags=flags, range_margin=0.0)
    U = torch.empty((N, ann.n_out_pad), dtype=torch.float32, device=dev)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ann, N), dtype=torch.uint8, device=dev)
    chem.chem_ann_forward(ann, X, U, ws)
    torch.cuda.synchronize()
    return chem, gm, ann, m, st, oracles["c_30"], flags.cpu().numpy(), U.cpu().numpy()


def test_range_flags_against_oracle(env):
    chem, gm, ann, m, st, o, flags, U = env
    norm = chem.chem_ann_get_norm(ann)
    n_in = ann.n_in
    mn, mx = norm[2 * n_in:3 * n_in].astype(np.float64), norm[3 * n_in:4 * n_in].astype(np.float64)
    rf, raw = mlp.range_flags(st.T, st.p, st.Y, mn, mx, 0.0)
    # FP32 features: a raw value within 1e-5 of a limit may go either way (features with a
    # zero range, like p here, sit exactly on both limits and are decided alike on both sides)
    live = (mx > mn)[:, None]
    near = (live & ((np.abs(raw - mn[:, None]) <= 1e-5 * (1 + np.abs(mn[:, None]))) |
                    (np.abs(raw - mx[:, None]) <= 1e-5 * (1 + np.abs(mx[:, None]))))).any(axis=0)
    assert (flags[:7] == 1).all()
    assert np.array_equal(flags[~near], rf[~near])
    assert near.mean() < 0.01


def _edit_rows(U, rng, K):
    """Network outputs with rows that exercise every flag."""
    U = U.copy()
    n = U.shape[0]
    rows = rng.permutation(n)
    U[rows[:10], 3] = np.inf
    U[rows[10:20], 5] = np.nan
    U[rows[20:30], 7] = -np.inf
    U[rows[30:130], :K] += rng.normal(0.0, 1.0, (100, K)).astype(np.float32)   # element residual
    U[rows[130:330], :K] += rng.normal(0.0, 0.05, (200, K)).astype(np.float32)  # small, projected
    return U


def _T_bound(o, T0, Y0, T1, Y1):
    """FP32 enthalpy-sum error bound of the kernel's T' (see the module docstring)."""
    _, h0, _ = o.species_thermo(T0)
    _, h1, _ = o.species_thermo(T1)
    E = (np.abs(Y0 * h0 * R * T0 / o.W).sum() + np.abs(Y1 * h1 * R * T1 / o.W).sum())
    cp = o.thermo_props(T1, Y1)[0]
    return 32 * EPS32 * E / cp + 1e-3


@pytest.mark.parametrize("case", ["defaults", "tight"])
def test_update_against_oracle(env, case):
    chem, gm, ann, m, st, o, flags_all, U_all = env
    K = m.n_species
    rng = np.random.default_rng(7)
    opts = dict(elem_tol=1e-2, T_min=250.0, T_max=3500.0, dT_max=0.0) if case == "defaults" else \
        dict(elem_tol=2e-3, T_min=600.0, T_max=2450.0, dT_max=40.0)
    idx = rng.permutation(N)[:2500].astype(np.int32)
    U = _edit_rows(U_all[idx], rng, K)
    fin = flags_all[idx].copy()
    dev = torch.device("cuda")
    T = torch.as_tensor(st.T, device=dev)
    Y = torch.as_tensor(st.Y, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    fl = torch.as_tensor(fin, device=dev)
    status = torch.full((idx.size,), -1, dtype=torch.int32, device=dev)
    chem.chem_ann_update(ann, T, p, Y, torch.as_tensor(U, device=dev), fl, status,
                         idx=torch.as_tensor(idx, device=dev), **opts)
    torch.cuda.synchronize()
    Tg, Yg, fg, sg = T.cpu().numpy(), Y.cpu().numpy(), fl.cpu().numpy(), status.cpu().numpy()

    norm = chem.chem_ann_get_norm(ann).astype(np.float64)
    om, osd = norm[4 * ann.n_in:4 * ann.n_in + K], norm[4 * ann.n_in + K:]
    To, Yo, fo, info = mlp.ann_update(o, st.T[idx], st.Y[:, idx], U.astype(np.float64), om, osd,
                                      flags_in=fin, **opts)
    # every flag occurs
    for bit in (mlp.FLAG_RANGE, mlp.FLAG_NONFINITE, mlp.FLAG_ELEMENTS):
        assert (fo & bit).any(), bit
    if case == "tight":
        assert (fo & mlp.FLAG_T_RANGE).any() and (fo & mlp.FLAG_DT).any()
    # cells with a deciding quantity at a threshold (within the FP32 error) may go either way
    res, Tp, T0 = info["elem_residual"], info["T_prime"], st.T[idx]
    near = np.abs(res - opts["elem_tol"]) <= 2e-5
    near |= np.abs(Tp - opts["T_min"]) <= 0.05
    near |= np.abs(Tp - opts["T_max"]) <= 0.05
    if opts["dT_max"] > 0:
        near |= np.abs(np.abs(Tp - T0) - opts["dT_max"]) <= 0.05
    assert near.mean() < 0.01
    cmp = ~near
    assert np.array_equal(fg[cmp], fo[cmp]), np.where(fg[cmp] != fo[cmp])
    assert np.array_equal(sg, np.where(fg != 0, 5, 0))
    # flagged cells keep their state bit for bit; untouched columns too
    cols_flag = idx[fg != 0]
    assert np.array_equal(Tg[cols_flag], st.T[cols_flag])
    assert np.array_equal(Yg[:, cols_flag], st.Y[:, cols_flag])
    rest = np.setdiff1d(np.arange(N), idx)
    assert np.array_equal(Tg[rest], st.T[rest]) and np.array_equal(Yg[:, rest], st.Y[:, rest])
    # accepted cells: values within the FP32 bounds
    acc = np.where(cmp & (fg == 0) & (fo == 0))[0]
    assert acc.size > 0.5 * idx.size
    Cm = o.comp / o.W[:, None]
    for s in acc:
        c = idx[s]
        yo, yg = Yo[:, s], Yg[:, c]
        r = 64 * EPS32 / np.maximum(yo, 1e-300) ** 0.1          # relative error of each Y*_k
        spread = np.sqrt((r * r * yo).sum())                     # its weighted norm
        bound = r * yo + np.sqrt(yo) * spread + 1e-25
        assert (np.abs(yg - yo) <= bound).all(), (s, np.abs(yg - yo).max())
        # the FP64 projection conserves the elements to FP64 rounding
        e0, e1 = Cm.T @ st.Y[:, c], Cm.T @ yg
        assert np.allclose(e1, e0, rtol=1e-12, atol=0), s
        assert abs(Tg[c] - To[s]) <= _T_bound(o, st.T[c], st.Y[:, c], To[s], yo), (s, Tg[c], To[s])


def test_step_ann_stages_compose(env):
    """chem_step_ann without fallback = features (range flags) -> forward -> update."""
    chem, gm, ann, m, st, o, _, _ = env
    dev = torch.device("cuda")
    kw = dict(elem_tol=1e-2, T_min=250.0, T_max=3500.0, dT_max=40.0)
    T1, Y1 = torch.as_tensor(st.T, device=dev), torch.as_tensor(st.Y, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    s1 = torch.empty(N, dtype=torch.int32, device=dev)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ann, N), dtype=torch.uint8, device=dev)
    chem.chem_step_ann(gm, ann, 5e-6, T1, p, Y1, s1, ws, range_margin=0.05, no_fallback=True, **kw)
    T2, Y2 = torch.as_tensor(st.T, device=dev), torch.as_tensor(st.Y, device=dev)
    X = torch.empty((N, 64), dtype=torch.bfloat16, device=dev)
    fl = torch.empty(N, dtype=torch.int32, device=dev)
    chem.chem_ann_features(ann, T2, p, Y2, X, flags=fl, range_margin=0.05)
    U = torch.empty((N, ann.n_out_pad), dtype=torch.float32, device=dev)
    chem.chem_ann_forward(ann, X, U, ws)
    s2 = torch.empty(N, dtype=torch.int32, device=dev)
    chem.chem_ann_update(ann, T2, p, Y2, U, fl, s2, **kw)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2) and torch.equal(T1, T2) and torch.equal(Y1, Y2)
    assert (s1 == 5).any() and (s1 == 0).any()


@pytest.mark.parametrize("with_idx", [False, True])
def test_fallback_cells_equal_direct_integration(env, with_idx):
    """a12: each status-5 cell of chem_step_ann carries exactly chem_step_di's result."""
    chem, gm, ann, m, st, o, _, _ = env
    dev = torch.device("cuda")
    di = dict(di_rtol=1e-7, di_atol_Y=1e-14)
    idx = None
    if with_idx:
        idx = torch.as_tensor(np.random.default_rng(3).permutation(N)[:2000].astype(np.int32), device=dev)
    n = N if idx is None else idx.numel()
    T, Y = torch.as_tensor(st.T, device=dev), torch.as_tensor(st.Y, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    status = torch.full((n,), -1, dtype=torch.int32, device=dev)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
    chem.chem_step_ann(gm, ann, 5e-6, T, p, Y, status, ws, idx=idx, dT_max=40.0, **di)
    torch.cuda.synchronize()
    sa = status.cpu().numpy()
    cols = np.arange(N) if idx is None else idx.cpu().numpy()
    fb = cols[sa == 5]
    assert fb.size >= 20 and (sa == 0).sum() > 0.5 * n
    assert set(np.unique(sa)) <= {0, 5}
    # the same cells by direct integration alone, with the same options
    Td, Yd = torch.as_tensor(st.T, device=dev), torch.as_tensor(st.Y, device=dev)
    sd = torch.full((fb.size,), -1, dtype=torch.int32, device=dev)
    wsd = torch.zeros(chem.chem_workspace_bytes(gm, fb.size), dtype=torch.uint8, device=dev)
    chem.chem_step_di(gm, 5e-6, Td, p, Yd, sd, idx=torch.as_tensor(fb.astype(np.int32), device=dev),
                      rtol=di["di_rtol"], atol_Y=di["di_atol_Y"], workspace=wsd)
    torch.cuda.synchronize()
    assert (sd.cpu().numpy() == 0).all()
    Ta, Ya, Tdd, Ydd = T.cpu().numpy(), Y.cpu().numpy(), Td.cpu().numpy(), Yd.cpu().numpy()
    assert np.array_equal(Ta[fb], Tdd[fb])
    assert np.array_equal(Ya[:, fb], Ydd[:, fb])
