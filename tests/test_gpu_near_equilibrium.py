"""GPU parity in the near-equilibrium regime, where the net rate of every reaction is a small
difference of large forward and reverse rates (the cancellation that keeps the rates, the
equilibrium constants and the Newton solve in FP64).

States come from the oracle's own long integrations (test-side use of the oracle), which reach
the Gibbs equilibrium: 9-species cells from 1400-2200 K run to 1e3 s, 30-species cells from
2200-2500 K run to 1e9 s.  On these states the
GPU's rates must match the oracle's within 1e-11 of the gross rate, and one direct-integration
step of dt must match the oracle's step within 1e-6 (T and every Y_k above 1e-10), as for the
workload's states.  The test also states how deep the cancellation is: the median over
reactions of |q_net| / max(q_f, q_r).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_18858_gb300 import workload as w  # noqa: E402

R = 8.314462618


@pytest.fixture(scope="module")
def lc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem
    build.build()
    chem.lib()
    return chem


def _relaxed(o, m, n, seed, T_range, t_relax):
    st = w.make_states(m, n, seed, T_range=T_range)
    T, Y, s, _ = o.integrate_batch(st.T, st.p, st.Y, t_relax, rtol=1e-11, atol_Y=1e-24, max_steps=10 ** 6)
    assert (s == 0).all()
    return w.States(T=T, p=st.p.copy(), Y=np.ascontiguousarray(np.maximum(Y, 0.0)))


def _cancellation(o, m, st):
    ratios = []
    for i in range(st.T.size):
        _, _, q, kf, kr = o.rates(st.T[i], st.p[i], st.Y[:, i], with_rxn=True)
        rho = st.p[i] / (R * st.T[i] * (st.Y[:, i] / o.W).sum())
        C = rho * st.Y[:, i] / o.W
        for j, rx in enumerate(m.reactions):
            f = kf[j] * np.prod(C[rx.reactants])
            r = kr[j] * np.prod(C[rx.products])
            g = max(f, r)
            if g > 0:
                ratios.append(abs(f - r) / g)
    return float(np.median(ratios))


@pytest.mark.parametrize("kind,n,T_range,t_relax,dt", [("h2_9", 48, (1400.0, 2200.0), 1e3, 1e-6),
                                                       ("c_30", 8, (2200.0, 2500.0), 1e9, 5e-6)])
def test_near_equilibrium_parity(lc, mechs, oracles, kind, n, T_range, t_relax, dt):
    m, path = mechs[kind]
    o = oracles[kind]
    gm = lc.chem_load_mech(path)
    st = _relaxed(o, m, n, 300, T_range, t_relax)
    med = _cancellation(o, m, st)
    print(f"{kind}: median |q_net| / max(q_f, q_r) = {med:.2e}")
    assert med < 1e-6
    dev = torch.device("cuda")
    T, p, Y = (torch.as_tensor(a, device=dev) for a in (st.T, st.p, st.Y))
    wdot = torch.empty_like(Y)
    lc.chem_rates(gm, T, p, Y, wdot)
    status = torch.full((n,), -1, dtype=torch.int32, device=dev)
    ws = torch.zeros(lc.chem_workspace_bytes(gm, n), dtype=torch.uint8, device=dev)
    lc.chem_step_di(gm, dt, T, p, Y, status, workspace=ws)
    torch.cuda.synchronize()
    wd = wdot.cpu().numpy()
    nu = np.zeros((m.n_species, m.n_reactions))
    for j, rx in enumerate(m.reactions):
        for k in rx.reactants:
            nu[k, j] -= 1
        for k in rx.products:
            nu[k, j] += 1
    for i in range(n):
        wo, _, q, kf, kr = o.rates(st.T[i], st.p[i], st.Y[:, i], with_rxn=True)
        rho = st.p[i] / (R * st.T[i] * (st.Y[:, i] / o.W).sum())
        C = rho * st.Y[:, i] / o.W
        gross = np.abs(nu) @ np.array([kf[j] * np.prod(C[rx.reactants]) + kr[j] * np.prod(C[rx.products])
                                       for j, rx in enumerate(m.reactions)])
        assert (np.abs(wd[:, i] - wo) <= 1e-11 * gross + 1e-300).all(), i
    To, Yo, so, _ = o.integrate_batch(st.T, st.p, st.Y, dt)
    Tg, Yg, sg = T.cpu().numpy(), Y.cpu().numpy(), status.cpu().numpy()
    assert (so == 0).all() and (sg == 0).all()
    assert (np.abs(Tg - To) <= 1e-6 * To).all()
    big = Yo > 1e-10
    assert np.all(np.where(big, np.abs(Yg - Yo) <= 1e-6 * Yo, True))
