"""GPU parity of the per-species networks (Sec. 2.2: one MLP per species) against the oracle.

* the grouped tensor-core GEMM (G GEMMs in one launch, each reading its own blocks of A and B
  and writing its own block of the output) against an FP64 reference of each group's GEMM,
  with the per-element bound of the one-GEMM test (FP32 accumulation over K, one BF16
  rounding for the BF16 epilogues); cases shaped like every per-species layer, with ragged M,
  N and K (a K slab that runs past a group's K, an N tile past a group's N);
* forward of K per-species networks against the oracle's K separate networks with BF16
  storage emulated (bound of the one-network forward test);
* gradients of one training step against the oracle's per-species backward with BF16
  storage emulated, element by element (|g - g_o| <= 2^-7 |dZ|^T |A|, tests/gradcheck.py);
* training, checkpoint and reload, and the learned step with fallback through the public API.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from scipy.special import erf  # noqa: E402

import gradcheck  # noqa: E402
from oracle import mlp  # noqa: E402
from paper_2402_18858_gb300 import workload as w  # noqa: E402


@pytest.fixture(scope="module")
def lc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem
    build.build()
    chem.lib()
    return chem


def _bf16(rng, shape, scale=1.0):
    return torch.as_tensor(rng.standard_normal(shape) * scale, dtype=torch.float32).to(torch.bfloat16)


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def _dgelu(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


# (name, epi, G, M, N, K): the per-species layers' GEMMs
#   fwd:   hidden layer forward, A [M, G K] column blocks, B [G N, K] row blocks, out [M, G N]
#   out:   output layer forward, N = 1 per group, out = column g of [M, 32]
#   wgrad: weight gradient, A [G N, K] row blocks (N rows per group), B [G K', K] row blocks
#   dgrad: data gradient with GELU', A [M, G K] column blocks, B [G N, K] row blocks
#   owgrad: output-layer weight gradient, one row per group
# (fwd 300 x 200 x 136 and wgrad 400 x 800 x 256 also run on CTA pairs)
CASES = [
    ("fwd", 0, 3, 300, 200, 136),
    ("fwd", 0, 4, 129, 800, 1600),
    ("fwd", 0, 2, 200, 400, 800),
    ("out", 1, 5, 260, 1, 48),
    ("out", 1, 30, 300, 1, 400),
    ("wgrad", 3, 4, 40, 72, 520),
    ("wgrad", 3, 3, 400, 800, 256),
    ("dgrad", 2, 3, 200, 72, 40),
    ("dgrad", 2, 2, 130, 800, 400),
    ("owgrad", 3, 6, 1, 48, 264),
    # at least 256 rows and 128+-wide tiles: CTA pairs
    ("fwd", 0, 3, 600, 800, 1600),
    ("dgrad", 2, 2, 520, 800, 400),
]


@pytest.mark.parametrize("name,epi,G,M,N,K", CASES)
def test_grouped_gemm(lc, name, epi, G, M, N, K):
    rng = np.random.default_rng(G * 1000 + M + N + K + epi)
    dev = torch.device("cuda")
    bias = z = None
    bias_goff = z_goff = ldz = 0
    if name in ("fwd", "dgrad"):
        A = _bf16(rng, (M, G * K))
        a_off, blkA = (0, K), [A[:, g * K:(g + 1) * K] for g in range(G)]
        B = _bf16(rng, (G * N, K), 1.0 / math.sqrt(K))
        b_off, blkB = (N, 0), [B[g * N:(g + 1) * N] for g in range(G)]
        ldo, out_goff = G * N, N
    elif name == "out":
        A = _bf16(rng, (M, G * K))
        a_off, blkA = (0, K), [A[:, g * K:(g + 1) * K] for g in range(G)]
        B = _bf16(rng, (G, K), 1.0 / math.sqrt(K))
        b_off, blkB = (1, 0), [B[g:g + 1] for g in range(G)]
        ldo, out_goff = 32, 1
    elif name == "wgrad":
        A = _bf16(rng, (G * M, K))
        a_off, blkA = (M, 0), [A[g * M:(g + 1) * M] for g in range(G)]
        B = _bf16(rng, (G * N, K), 1.0 / math.sqrt(K))
        b_off, blkB = (N, 0), [B[g * N:(g + 1) * N] for g in range(G)]
        ldo, out_goff = N, M * N
    else:  # owgrad: A has 32 rows (the padded output width), group g reads row g
        A = _bf16(rng, (32, K))
        a_off, blkA = (1, 0), [A[g:g + 1] for g in range(G)]
        B = _bf16(rng, (G * N, K), 1.0 / math.sqrt(K))
        b_off, blkB = (N, 0), [B[g * N:(g + 1) * N] for g in range(G)]
        ldo, out_goff = N, N
    if epi in (0, 1):
        bias = torch.as_tensor(rng.standard_normal(G * N) * 0.1, dtype=torch.float32)
        bias_goff = N
    if epi == 2:
        z = _bf16(rng, (M, G * N))
        ldz, z_goff = G * N, N
    out_rows = M if name in ("fwd", "out", "dgrad") else G * M
    dt = torch.bfloat16 if epi in (0, 2) else torch.float32
    out = torch.full((out_rows, ldo), float("nan"), dtype=dt, device=dev)
    err = lc.chem_selftest_gemm_grouped(epi, G, M, N, K, A.to(dev), a_off, B.to(dev), b_off, out, ldo, out_goff,
                                        bias=None if bias is None else bias.to(dev), bias_goff=bias_goff,
                                        z=None if z is None else z.to(dev), ldz=ldz, z_goff=z_goff)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got_all = out.double().cpu().numpy()
    written = np.zeros(got_all.shape, dtype=bool)
    for g in range(G):
        a, b = blkA[g].double().numpy(), blkB[g].double().numpy()
        acc = a @ b.T
        bound = 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-30
        if name == "wgrad" or name == "owgrad":
            rs, cs = slice(g * M, (g + 1) * M), slice(0, N)
        else:
            rs, cs = slice(0, M), slice(g * N, (g + 1) * N) if name != "out" else slice(g, g + 1)
        got = got_all[rs, cs]
        written[rs, cs] = True
        if epi == 3:
            assert (np.abs(got - acc) <= bound).all(), g
        elif epi == 1:
            ref = acc + bias.double().numpy()[g * N:(g + 1) * N][None, :]
            assert (np.abs(got - ref) <= bound + 1e-7 * np.abs(ref)).all(), g
        else:
            if epi == 0:
                pre = acc + bias.double().numpy()[g * N:(g + 1) * N][None, :]
                ref, slope = _gelu(pre), np.abs(_dgelu(pre))
            else:
                zz = z.double().numpy()[:, g * N:(g + 1) * N]
                ref, slope = acc * _dgelu(zz), np.abs(_dgelu(zz))
            tol = slope * bound + 2.0 ** -8 * np.abs(ref) + 1e-6 * np.abs(ref).max()
            assert (np.abs(got - ref) <= tol).all(), (g, np.abs(got - ref).max())
    # nothing outside the groups' output blocks is written
    assert np.isnan(got_all[~written]).all()


@pytest.fixture(scope="module")
def setup(lc, mechs):
    m, path = mechs["c_30"]
    gm = lc.chem_load_mech(path)
    st = w.make_states(m, 2048, 65)
    dev = torch.device("cuda")
    T = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    noise = torch.as_tensor(np.random.default_rng(2).standard_normal(st.Y.shape), device=dev)
    Y1 = (Y0 * (1.0 + 0.01 * noise)).contiguous()
    ann = lc.chem_ann_create_per_species(gm, [70, 44, 20], seed=11)
    lc.chem_ann_fit_norm(ann, T, p, Y0, Y1)
    X = torch.empty((2048, 64), dtype=torch.bfloat16, device=dev)
    bcty = torch.empty((2048, m.n_species), dtype=torch.float32, device=dev)
    lc.chem_ann_features(ann, T, p, Y0, X, bcty=bcty)
    U = torch.empty((2048, ann.n_out_pad), dtype=torch.float32, device=dev)
    lc.chem_ann_targets(ann, Y0, Y1, U)
    torch.cuda.synchronize()
    return gm, ann, st, X, bcty, U


def _forward(lc, ann, X):
    n = X.shape[0]
    Ug = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device="cuda")
    ws = torch.empty(lc.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device="cuda")
    lc.chem_ann_forward(ann, X, Ug, ws)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    return Ug


def test_layout(lc, setup, mechs):
    gm, ann, st, X, bcty, U = setup
    K = mechs["c_30"][0].n_species
    assert ann.groups == K and ann.n_out == K and ann.n_out_pad == 32
    # widths of one species' network, stored rounded up to multiples of 8
    assert ann.dims == [64, 72, 48, 24, 1]
    assert ann.n_params == K * (72 * 65 + 48 * 73 + 24 * 49 + 25)


def test_per_species_forward_parity(lc, setup):
    gm, ann, st, X, bcty, U = setup
    Ug = _forward(lc, ann, X)
    K = ann.n_out
    nets = mlp.unflatten_per_species(lc.chem_ann_get_params(ann), ann.dims, K)
    Uo, _ = mlp.forward_per_species(nets, X.float().cpu().numpy().astype(np.float64), bf16=True)
    d = Ug.cpu().numpy()[:, :K] - Uo
    assert np.abs(d).max() <= 2e-3 * np.abs(Uo).max() + 1e-3
    assert np.sqrt((d ** 2).mean()) <= 1e-3 * np.sqrt((Uo ** 2).mean())
    # the output padding columns read zero, as for the one network
    assert (Ug[:, K:] == 0).all()


def test_per_species_forward_parity_paper_widths(lc, setup):
    """Hidden widths 1600, 800, 400 per species (30 networks, 48,000 first-layer units)."""
    gm, ann0, st, X, bcty, U = setup
    ann = lc.chem_ann_create_per_species(gm, [1600, 800, 400], seed=12)
    lc.chem_ann_set_norm(ann, lc.chem_ann_get_norm(ann0))
    Xs = X[:300].contiguous()
    Ug = _forward(lc, ann, Xs)
    K = ann.n_out
    nets = mlp.unflatten_per_species(lc.chem_ann_get_params(ann), ann.dims, K)
    Uo, _ = mlp.forward_per_species(nets, Xs.float().cpu().numpy().astype(np.float64), bf16=True)
    d = Ug.cpu().numpy()[:, :K] - Uo
    assert np.abs(d).max() <= 2e-3 * np.abs(Uo).max() + 1e-3
    assert np.sqrt((d ** 2).mean()) <= 1e-3 * np.sqrt((Uo ** 2).mean())


def test_per_species_gradient_parity(lc, setup):
    gm, ann, st, X, bcty, U = setup
    B, K = 512, ann.n_out
    lc.chem_ann_train_step(ann, X[:B].contiguous(), U[:B].contiguous(), bcty[:B].contiguous(), apply=False)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    g_gpu = mlp.unflatten_per_species(lc.chem_ann_get_params(ann, which=1), ann.dims, K)
    nets = mlp.unflatten_per_species(lc.chem_ann_get_params(ann), ann.dims, K)
    norm = lc.chem_ann_get_norm(ann)
    om, osd = norm[4 * ann.n_in:4 * ann.n_in + K].astype(np.float64), norm[4 * ann.n_in + K:].astype(np.float64)
    Uo, caches = mlp.forward_per_species(nets, X[:B].float().cpu().numpy().astype(np.float64), bf16=True)
    _, _, _, dU = mlp.loss_and_grad(Uo, U[:B, :K].cpu().numpy().astype(np.float64), K,
                                    bcty[:B].cpu().numpy().astype(np.float64), om, osd, 1.0, 0.1)
    g_or, deltas = mlp.backward_per_species(nets, caches, dU, bf16=True, with_deltas=True)
    for l in range(ann.L):
        for k in range(K):
            gradcheck.check_layer(g_gpu[k][l][0], g_gpu[k][l][1], g_or[k][l][0], g_or[k][l][1],
                                  deltas[k][l], caches[k][0][l], f"species {k} layer {l}")
    # the padding units (70 -> 72, 44 -> 48, 20 -> 24) get no gradient
    for k in range(K):
        assert (g_gpu[k][0][0][70:] == 0).all() and (g_gpu[k][1][0][44:] == 0).all()
        assert (g_gpu[k][2][0][20:] == 0).all() and (g_gpu[k][3][0][:, 20:] == 0).all()


def test_per_species_training_checkpoint_and_step(lc, setup, tmp_path, mechs):
    gm, ann0, st, X, bcty, U = setup
    ann = lc.chem_ann_create_per_species(gm, [70, 44, 20], seed=13)
    lc.chem_ann_set_norm(ann, lc.chem_ann_get_norm(ann0))
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    B = 1024
    hist = []
    for it in range(30):
        s = (it * B) % 2048
        lc.chem_ann_train_step(ann, X[s:s + B].contiguous(), U[s:s + B].contiguous(), bcty[s:s + B].contiguous(),
                               lr=1e-3, loss_out=loss)
        hist.append(float(loss[0].item()))
    assert hist[-1] < 0.8 * hist[0]
    assert lc.chem_ann_error(ann) == 0
    path = str(tmp_path / "ann_ps.ckpt")
    lc.chem_ann_save(ann, path)
    ann2 = lc.chem_ann_load(gm, path)
    assert ann2.groups == ann.groups and ann2.dims == ann.dims
    assert np.array_equal(lc.chem_ann_get_params(ann), lc.chem_ann_get_params(ann2))
    assert torch.equal(_forward(lc, ann, X), _forward(lc, ann2, X))
    # the learned step with fallback through the public API
    m, _ = mechs["c_30"]
    n = 1500
    dev = torch.device("cuda")
    T = torch.as_tensor(st.T[:n].copy(), device=dev)
    p = torch.as_tensor(st.p[:n].copy(), device=dev)
    Y = torch.as_tensor(st.Y[:, :n].copy(), device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    ws = torch.empty(lc.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
    lc.chem_step_ann(gm, ann, 5e-6, T, p, Y, status, ws)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    s = status.cpu().numpy()
    assert np.isin(s, [0, 5]).all()
    Yh = Y.cpu().numpy()
    assert np.isfinite(Yh).all() and np.isfinite(T.cpu().numpy()).all()
    assert np.allclose(Yh.sum(axis=0), 1.0, atol=1e-9)


def test_per_species_53_species_multi_chunk(lc, mechs):
    """53 species (64-column output rows, 53 groups) over 40,000 rows: two inference chunks
    with a ragged second one; sampled rows against the oracle."""
    m, path = mechs["c_53"]
    gm = lc.chem_load_mech(path)
    n = 40_000
    st = w.make_states(m, n, 66)
    dev = torch.device("cuda")
    T = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    Y1 = (Y0 * (1.0 + 0.01 * torch.as_tensor(np.random.default_rng(3).standard_normal(st.Y.shape),
                                             device=dev))).contiguous()
    ann = lc.chem_ann_create_per_species(gm, [40, 24, 16], seed=14)
    assert ann.groups == 53 and ann.n_out_pad == 64
    lc.chem_ann_fit_norm(ann, T, p, Y0, Y1)
    X = torch.empty((n, 64), dtype=torch.bfloat16, device=dev)
    lc.chem_ann_features(ann, T, p, Y0, X)
    Ug = _forward(lc, ann, X)
    pick = np.sort(np.random.default_rng(67).choice(n, 300, replace=False))
    pick[-1] = n - 1
    nets = mlp.unflatten_per_species(lc.chem_ann_get_params(ann), ann.dims, 53)
    Xs = X[torch.as_tensor(pick, device=dev)].float().cpu().numpy().astype(np.float64)
    Uo, _ = mlp.forward_per_species(nets, Xs, bf16=True)
    d = Ug[torch.as_tensor(pick, device=dev)].cpu().numpy()[:, :53] - Uo
    assert np.abs(d).max() <= 2e-3 * np.abs(Uo).max() + 1e-3
    assert np.sqrt((d ** 2).mean()) <= 1e-3 * np.sqrt((Uo ** 2).mean())
    assert (Ug[:, 53:] == 0).all()
