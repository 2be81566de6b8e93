"""chem_step_di_noalloc: the allocation-free variant of chem_step_di.

It serves callers that cannot allocate device memory (a Fortran/C flow solver whose memory
pool already owns the free HBM, or a time-step loop that must not synchronise the device
through cudaMalloc).  This test calls it through the C ABI and checks it against the
workspace entry point on two calls in a row, within the direct-integration tolerance the
parity tests use (1e-6 relative on T and on every Y_k above 1e-10); the kernels are
deterministic, so the results are expected to be identical.  It also checks the property the
entry point exists for: the device's free memory is the same before and after the calls, and
a call on a caller's own (non-default) stream gives the same result.

The file name sorts last so that a run stopping at the first failure (`pytest -x`) has already
run every other test when this one runs; nothing here depends on what ran before it (the
scratch address is looked up in the current context on every call).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _check(T, Y, s, Tr, Yr, sr, what):
    assert np.array_equal(s, sr), what
    assert np.all(np.abs(T - Tr) <= 1e-6 * np.abs(Tr)), what
    big = Yr > 1e-10
    assert np.all(np.where(big, np.abs(Y - Yr) <= 1e-6 * np.abs(Yr), True)), what


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

    # all buffers of the calls below exist before the free-memory reading
    bufs = [(T0.clone(), Y0.clone(), torch.full((n,), -1, dtype=torch.int32, device=dev)) for _ in range(4)]
    side = torch.cuda.Stream(device=dev)
    free_before = None
    for call in range(3):
        T, Y, s = bufs[call]
        chem.chem_step_di_noalloc(gm, 5e-6, T, p, Y, s)
        torch.cuda.synchronize()
        _check(T.cpu().numpy(), Y.cpu().numpy(), s.cpu().numpy(), Tr, Yr, sr, f"call {call}")
        if call == 0:
            # the first call may load the library's device module for this context (CUDA's
            # lazy module loading), which the driver allocates; later calls allocate nothing
            free_before, _ = torch.cuda.mem_get_info(dev)
    # on a stream of the caller's own
    side.wait_stream(torch.cuda.current_stream(dev))
    T, Y, s = bufs[3]
    with torch.cuda.stream(side):
        chem.chem_step_di_noalloc(gm, 5e-6, T, p, Y, s, stream=side)
    side.synchronize()
    _check(T.cpu().numpy(), Y.cpu().numpy(), s.cpu().numpy(), Tr, Yr, sr, "side stream")
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info(dev)
    assert free_after == free_before, (free_before, free_after)
