"""GPU parity of the learned reaction step against the FP64 MLP oracle.

* forward: the BF16 tensor-core MLP against the oracle's forward with BF16 storage emulated
  (inputs, weights, hidden activations rounded to BF16): differences come only from FP32 vs
  FP64 accumulation and from activations that sit on a BF16 rounding boundary; bound
  max |dU| <= 2e-3 max|U| + 1e-3 and RMS(dU) <= 1e-3 RMS(U);
* gradients: GPU backward (BF16 GEMMs, BF16 dZ and pre-activations) against the FP64 backward
  with the same BF16 storage emulated, element by element: |g - g_o| <= 2^-7 (|dZ|^T |A|)
  (tests/gradcheck.py);
* Adam: two GPU steps against the oracle's Adam on the GPU's gradients, to FP32 rounding;
* training is deterministic: a checkpoint reloaded and trained on gives the same losses bit
  for bit as the original.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import gradcheck  # noqa: E402
from oracle import mlp  # noqa: E402
from paper_2402_18858_gb300 import workload as w  # noqa: E402

HIDDEN = [1600, 800, 400]


@pytest.fixture(scope="module")
def lc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem
    build.build()
    chem.lib()
    return chem


@pytest.fixture(scope="module")
def setup(lc, mechs):
    m, path = mechs["c_30"]
    gm = lc.chem_load_mech(path)
    ann = lc.chem_ann_create(gm, HIDDEN, seed=7)
    st = w.make_states(m, 2048, 55)
    dev = torch.device("cuda")
    T = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    # a perturbed copy stands in for Y(t + dt) when fitting the normalisation
    noise = torch.as_tensor(np.random.default_rng(1).standard_normal(st.Y.shape), device=dev)
    Y1 = (Y0 * (1.0 + 0.01 * noise)).contiguous()
    lc.chem_ann_fit_norm(ann, T, p, Y0, Y1)
    X = torch.empty((2048, 64), dtype=torch.bfloat16, device=dev)
    bcty = torch.empty((2048, m.n_species), dtype=torch.float32, device=dev)
    lc.chem_ann_features(ann, T, p, Y0, X, bcty=bcty)
    U = torch.empty((2048, ann.n_out_pad), dtype=torch.float32, device=dev)
    lc.chem_ann_targets(ann, Y0, Y1, U)
    torch.cuda.synchronize()
    return gm, ann, st, X, bcty, U


def test_features_and_targets(lc, setup, mechs):
    gm, ann, st, X, bcty, U = setup
    m, _ = mechs["c_30"]
    norm = lc.chem_ann_get_norm(ann)
    n_in = ann.n_in
    raw = np.concatenate([st.T[:, None], st.p[:, None], mlp.bct(st.Y).T], axis=1)
    ref = (raw - norm[:n_in]) / norm[n_in:2 * n_in]
    got = X.float().cpu().numpy()[:, :n_in]
    assert np.allclose(got, mlp.round_bf16(ref), rtol=2 ** -7, atol=2e-3)
    assert (X.float().cpu().numpy()[:, n_in:] == 0).all()
    assert np.allclose(bcty.cpu().numpy(), mlp.bct(st.Y).T, rtol=1e-5, atol=1e-5)


def test_forward_parity(lc, setup):
    gm, ann, st, X, bcty, U = setup
    n = X.shape[0]
    Ug = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device="cuda")
    ws = torch.empty(lc.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device="cuda")
    lc.chem_ann_forward(ann, X, Ug, ws)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    params = mlp.unflatten(lc.chem_ann_get_params(ann), ann.dims)
    Uo, _ = mlp.forward(params, X.float().cpu().numpy().astype(np.float64), bf16=True)
    d = Ug.cpu().numpy() - Uo
    assert np.abs(d).max() <= 2e-3 * np.abs(Uo).max() + 1e-3
    assert np.sqrt((d ** 2).mean()) <= 1e-3 * np.sqrt((Uo ** 2).mean())


def test_gradient_parity(lc, setup):
    gm, ann, st, X, bcty, U = setup
    B = 512
    lc.chem_ann_train_step(ann, X[:B].contiguous(), U[:B].contiguous(), bcty[:B].contiguous(), apply=False)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    g_gpu = mlp.unflatten(lc.chem_ann_get_params(ann, which=1), ann.dims)
    params = mlp.unflatten(lc.chem_ann_get_params(ann), ann.dims)
    norm = lc.chem_ann_get_norm(ann)
    K = ann.n_out
    om, osd = norm[4 * ann.n_in:4 * ann.n_in + K].astype(np.float64), norm[4 * ann.n_in + K:].astype(np.float64)
    Uo, cache = mlp.forward(params, X[:B].float().cpu().numpy().astype(np.float64), bf16=True)
    _, _, _, dU = mlp.loss_and_grad(Uo, U[:B].cpu().numpy().astype(np.float64), K,
                                    bcty[:B].cpu().numpy().astype(np.float64), om, osd, 1.0, 0.1)
    g_or, deltas = mlp.backward(params, cache, dU, bf16=True, with_deltas=True)
    for l, ((gw, gb), (ow, ob)) in enumerate(zip(g_gpu, g_or)):
        gradcheck.check_layer(gw, gb, ow, ob, deltas[l], cache[0][l], f"layer {l}")


def test_adam_steps_against_oracle(lc, setup):
    """Two Adam steps of the GPU (FP32 masters and moments) against oracle.mlp.adam_step fed
    the GPU's own gradients and the same FP32 hyper-parameters: equal to FP32 rounding (a few
    units in the last place of the weight and of its change, plus the rounding of the moments'
    sums carried through m / sqrt(v)); the BF16 weight copies the next forward reads follow
    the masters."""
    gm, ann0, st, X, bcty, U = setup
    ann = lc.chem_ann_create(gm, HIDDEN, seed=21)
    lc.chem_ann_set_norm(ann, lc.chem_ann_get_norm(ann0))
    f32 = lambda v: float(np.float32(v))
    lr, b1, b2, eps = f32(2e-3), f32(0.9), f32(0.999), f32(1e-8)
    B = 512
    p = lc.chem_ann_get_params(ann).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in (1, 2):
        s = (t - 1) * B
        lc.chem_ann_train_step(ann, X[s:s + B].contiguous(), U[s:s + B].contiguous(), bcty[s:s + B].contiguous(),
                               lr=lr, beta1=b1, beta2=b2, eps=eps)
        torch.cuda.synchronize()
        g = lc.chem_ann_get_params(ann, which=1).astype(np.float64)
        p_gpu = lc.chem_ann_get_params(ann).astype(np.float64)
        # FP32 error of the update: the moments' sums can cancel (m = b1 m + (1 - b1) g with
        # g of the opposite sign), so their error is eps32 times the terms' magnitudes
        e32 = float(np.finfo(np.float32).eps)
        bc1, bc2 = 1 - b1 ** t, 1 - b2 ** t
        Em = 4 * e32 * (np.abs(b1 * m) + np.abs((1 - b1) * g)) / bc1
        Ev = 4 * e32 * (b2 * v + (1 - b2) * g * g) / bc2
        p_or, m, v = mlp.adam_step(p, g, m, v, t, lr, b1, b2, eps)
        sv = np.sqrt(v / bc2)
        dupd = lr * (Em / (sv + eps) + np.abs(m / bc1) * Ev / (2 * np.maximum(sv, 1e-300) * (sv + eps) ** 2))
        ulp = np.spacing(np.abs(p_or).astype(np.float32)).astype(np.float64)
        bound = 4 * ulp + 8 * e32 * np.abs(p_or - p) + dupd
        assert (np.abs(p_gpu - p_or) <= bound).all(), (t, np.abs(p_gpu - p_or).max())
        assert (np.abs(p_or - p) > 0.5 * lr).mean() > 0.5          # the step moved the weights
        p = p_gpu
    params = mlp.unflatten(lc.chem_ann_get_params(ann), ann.dims)
    n = 512
    Ug = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device="cuda")
    ws = torch.empty(lc.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device="cuda")
    lc.chem_ann_forward(ann, X[:n].contiguous(), Ug, ws)
    torch.cuda.synchronize()
    Uo, _ = mlp.forward(params, X[:n].float().cpu().numpy().astype(np.float64), bf16=True)
    d = Ug.cpu().numpy() - Uo
    assert np.abs(d).max() <= 2e-3 * np.abs(Uo).max() + 1e-3


def test_training_is_deterministic_and_resumable(lc, setup, tmp_path, mechs):
    gm, ann0, st, X, bcty, U = setup
    ann = lc.chem_ann_create(gm, HIDDEN, seed=3)
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
    path = str(tmp_path / "ann.ckpt")
    lc.chem_ann_save(ann, path)
    ann2 = lc.chem_ann_load(gm, path)
    assert np.array_equal(lc.chem_ann_get_params(ann), lc.chem_ann_get_params(ann2))
    la, lb = [], []
    for it in range(5):
        s = (it * B) % 2048
        lc.chem_ann_train_step(ann, X[s:s + B].contiguous(), U[s:s + B].contiguous(), bcty[s:s + B].contiguous(),
                               lr=1e-3, loss_out=loss)
        la.append(float(loss[0].item()))
        lc.chem_ann_train_step(ann2, X[s:s + B].contiguous(), U[s:s + B].contiguous(), bcty[s:s + B].contiguous(),
                               lr=1e-3, loss_out=loss)
        lb.append(float(loss[0].item()))
    assert la == lb


def test_widths_that_are_not_multiples_of_8(lc, setup):
    """Hidden widths 20 and 12 are stored as 24 and 16; the padding units start at zero and stay
    exactly zero through training, so the network equals the 20-12 network of the oracle."""
    gm, ann0, st, X, bcty, U = setup
    ann = lc.chem_ann_create(gm, [20, 12], seed=5)
    assert list(ann.dims[1:3]) == [24, 16]
    lc.chem_ann_set_norm(ann, lc.chem_ann_get_norm(ann0))
    B = 1024
    for it in range(10):
        s = (it * B) % 2048
        lc.chem_ann_train_step(ann, X[s:s + B].contiguous(), U[s:s + B].contiguous(), bcty[s:s + B].contiguous(),
                               lr=1e-3)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    (W1, b1), (W2, b2), (W3, b3) = mlp.unflatten(lc.chem_ann_get_params(ann), ann.dims)
    assert (W1[20:] == 0).all() and (b1[20:] == 0).all()
    assert (W2[12:] == 0).all() and (W2[:, 20:] == 0).all() and (b2[12:] == 0).all()
    assert (W3[:, 12:] == 0).all()
    assert np.abs(W1[:20]).max() > 0 and np.abs(W2[:12, :20]).max() > 0
    n = X.shape[0]
    Ug = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device="cuda")
    ws = torch.empty(lc.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device="cuda")
    lc.chem_ann_forward(ann, X, Ug, ws)
    torch.cuda.synchronize()
    real = [(W1[:20], b1[:20]), (W2[:12, :20], b2[:12]), (W3[:, :12], b3)]
    Uo, _ = mlp.forward(real, X.float().cpu().numpy().astype(np.float64), bf16=True)
    d = Ug.cpu().numpy() - Uo
    assert np.abs(d).max() <= 2e-3 * np.abs(Uo).max() + 1e-3


def test_gradient_parity_with_heat_release_term(lc, setup):
    """Eq. 11 with W3 = 0.5: the GPU gradient of all three loss terms against the FP64 oracle."""
    gm, ann, st, X, bcty, U = setup
    B, K = 512, ann.n_out
    rng = np.random.default_rng(9)
    c = torch.as_tensor(rng.standard_normal((B, K)) * 0.3, dtype=torch.float32, device="cuda")
    r = torch.as_tensor(rng.standard_normal(B) * 0.2, dtype=torch.float32, device="cuda")
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    lc.chem_ann_train_step(ann, X[:B].contiguous(), U[:B].contiguous(), bcty[:B].contiguous(), apply=False,
                           hrr_c=c, hrr_r=r, w_hrr=0.5, loss_out=loss)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    g_gpu = mlp.unflatten(lc.chem_ann_get_params(ann, which=1), ann.dims)
    params = mlp.unflatten(lc.chem_ann_get_params(ann), ann.dims)
    norm = lc.chem_ann_get_norm(ann)
    om, osd = norm[4 * ann.n_in:4 * ann.n_in + K].astype(np.float64), norm[4 * ann.n_in + K:].astype(np.float64)
    Uo, cache = mlp.forward(params, X[:B].float().cpu().numpy().astype(np.float64), bf16=True)
    Lt, Ld, Lm, Lh, dU = mlp.loss_and_grad(Uo, U[:B].cpu().numpy().astype(np.float64), K,
                                           bcty[:B].cpu().numpy().astype(np.float64), om, osd, 1.0, 0.1,
                                           0.5, c.double().cpu().numpy(), r.double().cpu().numpy(), with_hrr=True)
    lg = loss.cpu().numpy()
    assert lg[3] == pytest.approx(Lh, rel=2e-2) and Lh > 0
    assert lg[0] == pytest.approx(Lt, rel=2e-2)
    g_or, deltas = mlp.backward(params, cache, dU, bf16=True, with_deltas=True)
    for l, ((gw, gb), (ow, ob)) in enumerate(zip(g_gpu, g_or)):
        gradcheck.check_layer(gw, gb, ow, ob, deltas[l], cache[0][l], f"layer {l}")


def test_heat_release_coefficients(lc, setup, mechs, oracles):
    """chem_ann_hrr_coeffs against the oracle's definition with its own NASA-7 enthalpies."""
    gm, ann, st, X, bcty, U = setup
    m, _ = mechs["c_30"]
    o = oracles["c_30"]
    n, K, dt, scale = 700, m.n_species, 5e-6, 3.0e9
    dev = torch.device("cuda")
    T0 = torch.as_tensor(st.T[:n], device=dev)
    p = torch.as_tensor(st.p[:n], device=dev)
    Y0 = torch.as_tensor(st.Y[:, :n].copy(), device=dev)
    dY = np.random.default_rng(10).standard_normal((K, n)) * 1e-3 * st.Y[:, :n]
    Y1 = torch.as_tensor(st.Y[:, :n] + dY, device=dev)
    c = torch.empty((n, K), dtype=torch.float32, device=dev)
    r = torch.empty(n, dtype=torch.float32, device=dev)
    lc.chem_ann_hrr_coeffs(ann, dt, scale, T0, p, Y0, Y1, c, r)
    torch.cuda.synchronize()
    h = np.stack([o.species_thermo(st.T[i])[1] * 8.314462618 * st.T[i] for i in range(n)], axis=1)
    c_o, r_o = mlp.hrr_coefficients(st.T[:n], st.p[:n], st.Y[:, :n], st.Y[:, :n] + dY, dt, np.asarray(m.W), h, scale)
    # FP64 arithmetic on both sides, FP32 results
    np.testing.assert_allclose(c.cpu().numpy(), c_o, rtol=2e-7, atol=1e-30)
    np.testing.assert_allclose(r.cpu().numpy(), r_o, rtol=2e-6, atol=1e-6 * np.abs(r_o).max())


def test_forward_full_size_sampled(lc, setup, mechs):
    """The benchmark's 2,000,000-row forward (61 chunks of 32,768 rows, ragged last chunk):
    512 sampled rows against the FP64 oracle with BF16 storage emulated."""
    gm, ann, st, X, bcty, U = setup
    m, _ = mechs["c_30"]
    n = 2_000_000
    big = w.make_states(m, n, 56)
    dev = torch.device("cuda")
    Xb = torch.empty((n, 64), dtype=torch.bfloat16, device=dev)
    lc.chem_ann_features(ann, torch.as_tensor(big.T, device=dev), torch.as_tensor(big.p, device=dev),
                         torch.as_tensor(big.Y, device=dev), Xb)
    Ug = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device=dev)
    ws = torch.empty(lc.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
    lc.chem_ann_forward(ann, Xb, Ug, ws)
    torch.cuda.synchronize()
    assert lc.chem_ann_error(ann) == 0
    pick = np.sort(np.random.default_rng(57).choice(n, 512, replace=False))
    pick[-1] = n - 1
    params = mlp.unflatten(lc.chem_ann_get_params(ann), ann.dims)
    Uo, _ = mlp.forward(params, Xb[torch.as_tensor(pick, device=dev)].float().cpu().numpy().astype(np.float64),
                        bf16=True)
    d = Ug[torch.as_tensor(pick, device=dev)].cpu().numpy() - Uo
    assert np.abs(d).max() <= 2e-3 * np.abs(Uo).max() + 1e-3
    assert np.sqrt((d ** 2).mean()) <= 1e-3 * np.sqrt((Uo ** 2).mean())


def test_train_epoch_is_the_shuffled_sequence_of_steps(lc, setup):
    """chem_ann_train_epoch: a seeded permutation per epoch (exact integer check), and the
    epoch equals the same minibatches taken through chem_ann_train_step with the cosine
    learning rate, bit for bit; its loss is the mean of the steps' losses."""
    import math
    gm, ann0, st, X, bcty, U = setup
    n, B = 2000, 256                     # 7 full minibatches; 208 rows not visited this epoch
    dev = torch.device("cuda")
    orders = {}
    for seed, ep in ((5, 0), (5, 1), (6, 0), (5, 0)):
        o = torch.empty(n, dtype=torch.int32, device=dev)
        lc.chem_selftest_epoch_order(n, seed, ep, o)
        torch.cuda.synchronize()
        a = o.cpu().numpy()
        assert np.array_equal(np.sort(a), np.arange(n))
        if (seed, ep) in orders:
            assert np.array_equal(orders[(seed, ep)], a)
        orders[(seed, ep)] = a
    assert not np.array_equal(orders[(5, 0)], orders[(5, 1)])
    assert not np.array_equal(orders[(5, 0)], orders[(6, 0)])
    assert not np.array_equal(orders[(5, 0)], np.arange(n))

    f32 = lambda v: float(np.float32(v))
    lr, lr_min, total, step0 = f32(1e-3), f32(1e-4), 20, 3
    a1 = lc.chem_ann_create(gm, [64, 32], seed=31)
    a2 = lc.chem_ann_create(gm, [64, 32], seed=31)
    for a in (a1, a2):
        lc.chem_ann_set_norm(a, lc.chem_ann_get_norm(ann0))
    Xs, Us, bs = X[:n].contiguous(), U[:n].contiguous(), bcty[:n].contiguous()
    loss = torch.zeros(4, dtype=torch.float32, device=dev)
    lc.chem_ann_train_epoch(a1, Xs, Us, bs, batch=B, lr=lr, lr_min=lr_min, total_steps=total, step0=step0,
                            seed=5, epoch=1, loss_out=loss)
    order = torch.as_tensor(orders[(5, 1)].astype(np.int64), device=dev)
    step_loss = torch.zeros(4, dtype=torch.float32, device=dev)
    losses = []
    for q in range(n // B):
        rows = order[q * B:(q + 1) * B]
        t = min(1.0, (step0 + q) / (total - 1))
        cur = f32(lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * t)))
        lc.chem_ann_train_step(a2, Xs[rows].contiguous(), Us[rows].contiguous(), bs[rows].contiguous(), lr=cur,
                               loss_out=step_loss)
        losses.append(step_loss.cpu().numpy().copy())
    torch.cuda.synchronize()
    assert lc.chem_ann_error(a1) == 0 and lc.chem_ann_error(a2) == 0
    assert np.array_equal(lc.chem_ann_get_params(a1), lc.chem_ann_get_params(a2))
    assert np.allclose(loss.cpu().numpy(), np.mean(losses, axis=0), rtol=1e-5, atol=0)
