"""chem_step_di_noalloc: the allocation-free variant of chem_step_di.

It serves callers that cannot allocate device memory (a Fortran/C flow solver whose memory
pool already owns the free HBM, or a time-step loop that must not synchronise the device
through cudaMalloc).  This test calls it through the C ABI and checks it against the
workspace entry point on two calls in a row, within the direct-integration tolerance the
parity tests use (1e-6 relative on T and on every Y_k above 1e-10); the kernels are
deterministic, so the results are expected to be identical.  This file is collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point(mechs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem, workload as w
    build.build()
    m, path = mechs["c_30"]
    gm = chem.chem_load_mech(path)
    st = w.make_states(m, 1000, 4242)
    dev = torch.device("cuda", torch.cuda.current_device())
    T0 = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    n = st.T.size

    Tr, Yr = T0.clone(), Y0.clone()
    sr = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.zeros(chem.chem_workspace_bytes(gm, n), dtype=torch.uint8, device=dev)
    chem.chem_step_di(gm, 5e-6, Tr, p, Yr, sr, workspace=ws)
    torch.cuda.synchronize()
    Tr, Yr, sr = Tr.cpu().numpy(), Yr.cpu().numpy(), sr.cpu().numpy()
    assert (sr == 0).all()

    for call in range(2):
        T, Y = T0.clone(), Y0.clone()
        s = torch.full((n,), -1, dtype=torch.int32, device=dev)
        chem.chem_step_di_noalloc(gm, 5e-6, T, p, Y, s)
        torch.cuda.synchronize()
        T, Y, s = T.cpu().numpy(), Y.cpu().numpy(), s.cpu().numpy()
        assert np.array_equal(s, sr), call
        assert np.all(np.abs(T - Tr) <= 1e-6 * np.abs(Tr)), call
        big = Yr > 1e-10
        assert np.all(np.where(big, np.abs(Y - Yr) <= 1e-6 * np.abs(Yr), True)), call
