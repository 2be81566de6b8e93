"""Pins of the FP64 MLP oracle (Sec. 2.2) against facts other than itself."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_box_cox_range_and_inverse():
    # Sec. 2.2: [0, 1] maps to [-1/lambda, 0] with lambda = 0.1
    assert mlp.bct(1.0) == 0.0
    assert mlp.bct(0.0) == pytest.approx(-10.0)
    x = np.logspace(-30, 0, 200)
    assert np.allclose(mlp.ibct(mlp.bct(x)), x, rtol=1e-10, atol=0)
    # lambda -> 0 limit is the logarithm (the second branch of Eq. 7)
    assert mlp.bct(0.37, lam=1e-9) == pytest.approx(math.log(0.37), rel=1e-7)


def test_gelu_special_values_and_derivative():
    assert mlp.gelu(0.0) == 0.0
    assert mlp.gelu(10.0) == pytest.approx(10.0, rel=1e-15)
    assert abs(mlp.gelu(-10.0)) < 1e-20
    # GELU(x) = x Phi(x): at x = 1, Phi(1) = 0.841344746068543 (standard normal table)
    assert mlp.gelu(1.0) == pytest.approx(0.841344746068543, rel=1e-12)
    x = np.linspace(-6, 6, 101)
    h = 1e-6
    assert np.allclose(mlp.dgelu(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-6, 6, 10000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.round_bf16(x), ref)


def _tiny(rng, dims):
    return [(rng.standard_normal((dims[l + 1], dims[l])) / math.sqrt(dims[l]),
             rng.standard_normal(dims[l + 1]) * 0.1) for l in range(len(dims) - 1)]


def test_backward_against_finite_differences():
    rng = np.random.default_rng(1)
    dims = [6, 7, 5, 4]
    params = _tiny(rng, dims)
    X = rng.standard_normal((9, 6))
    Ut = rng.standard_normal((9, 4))
    bcty = mlp.bct(rng.uniform(1e-6, 0.3, (9, 4)))
    om, osd = rng.standard_normal(4) * 0.1, rng.uniform(0.5, 2.0, 4)

    def L(flat):
        p = mlp.unflatten(flat, dims)
        U, _ = mlp.forward(p, X)
        return mlp.loss_and_grad(U, Ut, 4, bcty, om, osd, 1.0, 0.1)[0]

    U, cache = mlp.forward(params, X)
    _, _, _, dU = mlp.loss_and_grad(U, Ut, 4, bcty, om, osd, 1.0, 0.1)
    g = mlp.flatten(mlp.backward(params, cache, dU))
    flat = mlp.flatten(params)
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = 1e-6
        fd[i] = (L(flat + e) - L(flat - e)) / 2e-6
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9)


def test_adam_first_step_closed_form():
    # with zero moments, the bias-corrected first step is -lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_hrr_term_against_finite_differences_and_by_hand():
    rng = np.random.default_rng(2)
    dims = [6, 7, 5, 4]
    params = _tiny(rng, dims)
    X = rng.standard_normal((9, 6))
    Ut = rng.standard_normal((9, 4))
    bcty = mlp.bct(rng.uniform(1e-6, 0.3, (9, 4)))
    om, osd = rng.standard_normal(4) * 0.1, rng.uniform(0.5, 2.0, 4)
    c = rng.standard_normal((9, 4))
    r = rng.standard_normal(9) * 0.1

    def L(flat):
        p = mlp.unflatten(flat, dims)
        U, _ = mlp.forward(p, X)
        return mlp.loss_and_grad(U, Ut, 4, bcty, om, osd, 1.0, 0.1, 0.7, c, r)[0]

    U, cache = mlp.forward(params, X)
    Lt, Ld, Lm, Lh, dU = mlp.loss_and_grad(U, Ut, 4, bcty, om, osd, 1.0, 0.1, 0.7, c, r, with_hrr=True)
    # the term by hand: one sample's squared heat-release error
    Ys = mlp.ibct(bcty + U[:, :4] * osd + om)
    e0 = float(np.dot(c[0], Ys[0] - mlp.ibct(bcty[0])) - r[0])
    assert Lh == pytest.approx(np.mean([(np.dot(c[b], Ys[b] - mlp.ibct(bcty[b])) - r[b]) ** 2
                                         for b in range(9)]), rel=1e-13)
    assert Lt == pytest.approx(Ld + 0.1 * Lm + 0.7 * Lh, rel=1e-14) and e0 != 0.0
    g = mlp.flatten(mlp.backward(params, cache, dU))
    flat = mlp.flatten(params)
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = 1e-6
        fd[i] = (L(flat + e) - L(flat - e)) / 2e-6
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9)


def test_hrr_coefficients_by_hand():
    # two species with h = (-100, +50) kJ/mol, W = (0.02, 0.03) kg/mol: the step-mean heat
    # release of converting 1 % of the mass from species 2 to species 1
    T0, p, dt, scale = np.array([1000.0]), np.array([101325.0]), 1e-6, 2.0
    W = np.array([0.02, 0.03])
    h = np.array([[-1.0e5], [5.0e4]])
    Y0 = np.array([[0.5], [0.5]])
    Y1 = np.array([[0.51], [0.49]])
    c, r = mlp.hrr_coefficients(T0, p, Y0, Y1, dt, W, h, scale)
    rho = 101325.0 / (8.314462618 * 1000.0 * (0.5 / 0.02 + 0.5 / 0.03))
    hrr = -(rho / dt) * (-1.0e5 / 0.02 * 0.01 + 5.0e4 / 0.03 * (-0.01))
    assert r[0] == pytest.approx(hrr / scale, rel=1e-13)
    # coefficients relative to the cell's mean enthalpy hbar = 0.5 h_1 + 0.5 h_2
    hm = np.array([-1.0e5 / 0.02, 5.0e4 / 0.03])
    hbar = 0.5 * hm[0] + 0.5 * hm[1]
    np.testing.assert_allclose(c[0], -rho * (hm - hbar) / (dt * scale), rtol=1e-14)
    # a mass-sum error that rescales the mixture (dY = eps Y0, sum dY = eps) reads as no heat
    # release, while the same sizes in another direction do
    eps = 1e-3
    assert abs(np.dot(c[0], eps * Y0[:, 0])) <= 1e-12 * eps * np.abs(c[0]).sum()
    assert abs(np.dot(c[0], np.array([eps, 0.0]))) > 1e-3 * eps * np.abs(c[0]).sum()


def _block_diagonal(nets):
    """One network equal to the K per-species networks: the first layer stacks the species'
    units (shared input), later layers are block diagonal, the output row k reads species k's
    last hidden block only."""
    from scipy.linalg import block_diag
    layers = []
    for l in range(len(nets[0])):
        if l == 0:
            W = np.concatenate([net[0][0] for net in nets], axis=0)
        else:
            W = block_diag(*[net[l][0] for net in nets])
        b = np.concatenate([net[l][1] for net in nets])
        layers.append((W, b))
    return layers


def test_per_species_equals_block_diagonal_network():
    # Sec. 2.2 per-species networks written out as one network with zero off-diagonal weights;
    # the one-network forward and backward are pinned above by finite differences
    rng = np.random.default_rng(4)
    K, dims = 5, [6, 7, 5, 3, 1]
    nets = [_tiny(rng, dims) for _ in range(K)]
    X = rng.standard_normal((11, 6))
    big = _block_diagonal(nets)
    for bf16 in (False, True):
        U, caches = mlp.forward_per_species(nets, X, bf16=bf16)
        Ub, cache_b = mlp.forward(big, X, bf16=bf16)
        assert U.shape == (11, K)
        assert np.allclose(U, Ub, rtol=1e-13, atol=1e-13)
    dU = rng.standard_normal((11, K))
    U, caches = mlp.forward_per_species(nets, X)
    Ub, cache_b = mlp.forward(big, X)
    g = mlp.backward_per_species(nets, caches, dU)
    gb = mlp.backward(big, cache_b, dU)
    for l in range(len(dims) - 1):
        h, c = dims[l + 1], dims[l]
        for k in range(K):
            rows = slice(k * h, (k + 1) * h)
            cols = slice(None) if l == 0 else slice(k * c, (k + 1) * c)
            assert np.allclose(g[k][l][0], gb[l][0][rows, cols], rtol=1e-12, atol=1e-14)
            assert np.allclose(g[k][l][1], gb[l][1][rows], rtol=1e-12, atol=1e-14)


def test_per_species_outputs_are_independent_and_layout_round_trips():
    rng = np.random.default_rng(5)
    K, dims = 4, [6, 8, 8, 1]
    nets = [_tiny(rng, dims) for _ in range(K)]
    X = rng.standard_normal((7, 6))
    U0, _ = mlp.forward_per_species(nets, X)
    # changing species 2's network changes column 2 only
    nets2 = [list(net) for net in nets]
    W, b = nets2[2][1]
    nets2[2][1] = (W + 0.3, b)
    U1, _ = mlp.forward_per_species(nets2, X)
    changed = np.abs(U1 - U0).max(axis=0) > 0
    assert changed.tolist() == [False, False, True, False]
    # the stacked layout: species k's layer-l weights are rows k h .. (k + 1) h of the layer
    flat = mlp.flatten_per_species(nets)
    assert flat.size == K * sum(dims[l + 1] * (dims[l] + 1) for l in range(len(dims) - 1))
    back = mlp.unflatten_per_species(flat, dims, K)
    for k in range(K):
        for (W, b), (W2, b2) in zip(nets[k], back[k]):
            assert np.array_equal(W, W2) and np.array_equal(b, b2)
    assert np.array_equal(flat[dims[1] * dims[0]:2 * dims[1] * dims[0]], nets[1][0][0].ravel())


def test_per_species_backward_against_finite_differences():
    # the mass term of the loss couples the species' networks
    rng = np.random.default_rng(6)
    K, dims = 3, [5, 4, 3, 1]
    nets = [_tiny(rng, dims) for _ in range(K)]
    X = rng.standard_normal((6, 5))
    Ut = rng.standard_normal((6, K))
    bcty = mlp.bct(rng.uniform(1e-6, 0.4, (6, K)))
    om, osd = rng.standard_normal(K) * 0.1, rng.uniform(0.5, 2.0, K)

    def L(flat):
        U, _ = mlp.forward_per_species(mlp.unflatten_per_species(flat, dims, K), X)
        return mlp.loss_and_grad(U, Ut, K, bcty, om, osd, 1.0, 0.1)[0]

    U, caches = mlp.forward_per_species(nets, X)
    _, _, _, dU = mlp.loss_and_grad(U, Ut, K, bcty, om, osd, 1.0, 0.1)
    g = mlp.flatten_per_species(mlp.backward_per_species(nets, caches, dU))
    flat = mlp.flatten_per_species(nets)
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = 1e-6
        fd[i] = (L(flat + e) - L(flat - e)) / 2e-6
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9)


def test_bf16_emulated_backward_is_the_backward_within_rounding():
    """The BF16-storage emulation changes the gradients only by storage rounding: against the
    unemulated backward on the same (emulated) forward, each entry stays within 2^-7 of the
    sum of its terms' magnitudes per rounded layer passed."""
    rng = np.random.default_rng(4)
    dims = [9, 24, 16, 5]
    params = _tiny(rng, dims)
    X = rng.standard_normal((64, dims[0]))
    U, cache = mlp.forward(params, X, bf16=True)
    dU = rng.standard_normal(U.shape)
    g0, d0 = mlp.backward(params, cache, dU, with_deltas=True)
    g1, d1 = mlp.backward(params, cache, dU, bf16=True, with_deltas=True)
    acts = cache[0]
    for l in range(len(dims) - 1):
        depth = len(dims) - 1 - l                  # rounding stages above and at layer l
        bound = depth * 2 ** -7 * (np.abs(d0[l]).T @ np.abs(acts[l])) * 4
        assert (np.abs(g1[l][0] - g0[l][0]) <= bound + 1e-300).all(), l
        assert not np.array_equal(g1[l][0], g0[l][0])           # the emulation does something
