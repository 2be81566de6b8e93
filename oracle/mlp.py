"""FP64 oracle of the learned reaction step (Sec. 2.2) -- test infrastructure only.

* Box-Cox transform (Eq. 7; the printed equation is garbled, the stated range [0, 1] ->
  [-1/lambda, 0] fixes it as F(x) = (x^lambda - 1)/lambda), lambda = 0.1, and its inverse.
* MLP with GELU hidden layers (exact erf form, Hendrycks & Gimpel 2016) and a linear output,
  weights W_l [out, in], biases b_l; forward and a hand-written backward pass.
* Loss of Eq. 11 with L_data (Eq. 8, mean squared error in the normalised output space),
  L_mass (Eq. 9, mean over samples of |sum_k Y*_k - 1|) and L_HRR (Eq. 10, squared error of the
  step-mean heat release, in units of a scale; weight W3, 0 unless requested).
* Adam (Kingma & Ba 2015).
* Optional emulation of BF16 storage (round to nearest even) of inputs, weights and hidden
  activations, so that the GPU's BF16 tensor-core forward can be compared element by element.

* Per-species networks (Sec. 2.2: each species' transformed mass fraction is trained and
  predicted by its own MLP): K independent networks with one output each, evaluated one after
  the other on the same inputs; their parameters as one flat array stacked by species.

* The learned step's update of the cell state (`ann_update`): inverse Box-Cox of the predicted
  increments, renormalisation, the element-residual check, the weighted least-squares
  projection onto exact element conservation, T from enthalpy conservation, and the flags of
  the fallback rules (`range_flags` for the training-range check of the inputs).

Parity status: forward, backward, loss gradient (all three terms), the heat-release
coefficients and Adam are pinned by the tests in tests/test_oracle_mlp.py (finite differences,
closed forms, special values; the BF16-storage emulation of backward against the unemulated
pass within its rounding); the update by tests/test_oracle_ann_update.py (the identity on an
element-conserving integrated state, a hand-computed projection, exact element and enthalpy
conservation, each flag rule); the per-species networks by their equality with one network
of block-diagonal weights, by the independence of each output from the other species'
weights and by finite differences.  The loss weights W1, W2, W3 of Eq. 11 are unstated in the
paper: W1 = 1, W2 = 0.1 and W3 = 0 by default.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
from scipy.special import erf

LAMBDA = 0.1


def bct(x, lam: float = LAMBDA):
    """Box-Cox transform of mass fractions (x clipped at 0)."""
    x = np.maximum(np.asarray(x, dtype=np.float64), 0.0)
    return (np.power(x, lam) - 1.0) / lam


def ibct(z, lam: float = LAMBDA):
    """Inverse Box-Cox: (lam z + 1)^(1/lam), 0 where lam z + 1 <= 0."""
    t = np.maximum(lam * np.asarray(z, dtype=np.float64) + 1.0, 0.0)
    return np.power(t, 1.0 / lam)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def dgelu(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def round_bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    out = u.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


Params = List[Tuple[np.ndarray, np.ndarray]]


def unflatten(flat: np.ndarray, dims: List[int]) -> Params:
    """Flat [W_0, b_0, W_1, b_1, ...] (W_l of shape [dims[l+1], dims[l]]) -> list of (W, b)."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        nw = dims[l + 1] * dims[l]
        W = flat[o:o + nw].reshape(dims[l + 1], dims[l]).astype(np.float64)
        o += nw
        b = flat[o:o + dims[l + 1]].astype(np.float64)
        o += dims[l + 1]
        out.append((W, b))
    return out


def flatten(params: Params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def forward(params: Params, X: np.ndarray, bf16: bool = False):
    """U = MLP(X); returns (U, cache).  bf16=True rounds W, inputs and hidden activations."""
    A = round_bf16(X) if bf16 else np.asarray(X, dtype=np.float64)
    cache = [A]
    zs = []
    for l, (W, b) in enumerate(params):
        Wl = round_bf16(W) if bf16 else W
        Z = A @ Wl.T + b
        if l < len(params) - 1:
            zs.append(Z)
            A = gelu(Z)
            if bf16:
                A = round_bf16(A)
            cache.append(A)
        else:
            return Z, (cache, zs)
    raise AssertionError("empty network")


def backward(params: Params, cache, dU: np.ndarray, bf16: bool = False, with_deltas: bool = False):
    """Gradients of a scalar loss with dL/dU = dU: dW_l = delta_l^T A_l, db_l = sum_b delta_l,
    delta_{l-1} = (delta_l W_l) * GELU'(Z_{l-1}).

    bf16=True emulates BF16 storage where a BF16 training pass stores values: dU and every
    delta_l, the weights W_l and the pre-activations Z_l (GELU' is taken at the stored Z); the
    cache must come from forward(..., bf16=True).  with_deltas=True also returns the deltas
    (per layer, the sums' left operands), e.g. for element-wise error bounds."""
    acts, zs = cache
    grads = [None] * len(params)
    deltas = [None] * len(params)
    d = round_bf16(dU) if bf16 else dU
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        deltas[l] = d
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            if bf16:
                d = round_bf16((d @ round_bf16(W)) * dgelu(round_bf16(zs[l - 1])))
            else:
                d = (d @ W) * dgelu(zs[l - 1])
    return (grads, deltas) if with_deltas else grads


def unflatten_per_species(flat: np.ndarray, dims: List[int], K: int) -> List[Params]:
    """Flat parameters of K networks of widths dims (dims[-1] = 1), stored per layer as
    W [K dims[l+1], dims[l]] then b [K dims[l+1]] with species k in rows k dims[l+1] ...,
    -> one parameter list per species."""
    nets: List[Params] = [[] for _ in range(K)]
    o = 0
    for l in range(len(dims) - 1):
        h, c = dims[l + 1], dims[l]
        W = flat[o:o + K * h * c].reshape(K, h, c).astype(np.float64)
        o += K * h * c
        b = flat[o:o + K * h].reshape(K, h).astype(np.float64)
        o += K * h
        for k in range(K):
            nets[k].append((W[k], b[k]))
    return nets


def flatten_per_species(nets: List[Params]) -> np.ndarray:
    """Inverse of unflatten_per_species."""
    parts = []
    for l in range(len(nets[0])):
        parts.append(np.concatenate([net[l][0].ravel() for net in nets]))
        parts.append(np.concatenate([net[l][1] for net in nets]))
    return np.concatenate(parts)


def forward_per_species(nets: List[Params], X: np.ndarray, bf16: bool = False):
    """U[:, k] = MLP_k(X) for each species' own network; returns (U [n, K], caches)."""
    cols, caches = [], []
    for net in nets:
        U, cache = forward(net, X, bf16)
        cols.append(U[:, 0])
        caches.append(cache)
    return np.stack(cols, axis=1), caches


def backward_per_species(nets: List[Params], caches, dU: np.ndarray, bf16: bool = False,
                         with_deltas: bool = False):
    """Gradients of every species' network, given dL/dU [n, >= K] (options as backward)."""
    out = [backward(net, cache, dU[:, k:k + 1], bf16, with_deltas)
           for k, (net, cache) in enumerate(zip(nets, caches))]
    if with_deltas:
        return [g for g, _ in out], [d for _, d in out]
    return out


def loss_and_grad(U, Ut, K, bcty=None, out_mean=None, out_std=None, w_data=1.0, w_mass=0.1,
                  w_hrr=0.0, hrr_c=None, hrr_r=None, with_hrr=False):
    """Eq. 11 over the first K output columns; returns (L, L_data, L_mass, dU), or with
    with_hrr=True (L, L_data, L_mass, L_hrr, dU).

    L_hrr (Eq. 10): mean over samples of e_b^2, e_b = sum_k c_bk (Y*_bk - Y_bk(t)) - r_b, with
    Y* the predicted state, Y(t) = F^-1(bcty), c_bk the per-sample heat-release coefficients
    and r_b the DI target, both in units of a heat-release scale (see hrr_coefficients)."""
    U = np.asarray(U, dtype=np.float64)
    B = U.shape[0]
    d = U[:, :K] - Ut[:, :K]
    L_data = float((d * d).mean())
    dU = np.zeros_like(U)
    dU[:, :K] = w_data * 2.0 * d / (B * K)
    L_mass = 0.0
    L_hrr = 0.0
    need_y = bcty is not None and (w_mass != 0.0 or (w_hrr != 0.0 and hrr_c is not None))
    if need_y:
        Ys = ibct(bcty + U[:, :K] * out_std[None, :] + out_mean[None, :])
        dYs = np.power(np.maximum(Ys, 0.0), 1.0 - LAMBDA) * out_std[None, :]
    if bcty is not None and w_mass != 0.0:
        s = Ys.sum(axis=1)
        L_mass = float(np.abs(s - 1.0).mean())
        dU[:, :K] += w_mass / B * np.sign(s - 1.0)[:, None] * dYs
    if bcty is not None and w_hrr != 0.0 and hrr_c is not None:
        e = (hrr_c * (Ys - ibct(bcty))).sum(axis=1) - hrr_r
        L_hrr = float((e * e).mean())
        dU[:, :K] += w_hrr * 2.0 / B * e[:, None] * hrr_c * dYs
    L = w_data * L_data + w_mass * L_mass + w_hrr * L_hrr
    if with_hrr:
        return L, L_data, L_mass, L_hrr, dU
    return L, L_data, L_mass, dU


def hrr_coefficients(T0, p, Y0, Y1, dt, W, h_molar, scale):
    """Per-sample coefficients of the heat-release loss term (Eq. 10), read as the step-mean
    heat release HRR = -(rho / dt) sum_k h_k(T0) (Y_k(t + dt) - Y_k(t)) (W/m^3) with the mass
    enthalpies h_k = h_k,molar / W_k at the initial temperature and the initial density
    rho = p / (R T0 sum_k Y_k / W_k):  c_bk = -rho (h_k - hbar) / (dt scale) and the DI target
    r_b = sum_k c_bk (Y1_bk - Y0_bk).  hbar = sum_k Y0_k h_k, the cell's mean enthalpy: a
    common shift of the enthalpies leaves the heat release of a mass-conserving change
    unchanged, and removing the mean keeps a predicted change whose mass fractions do not sum
    to one (L_mass's concern) from reading as heat release.  h_molar [K, N] (J/mol) from the
    oracle's NASA-7; Y0, Y1 [K, N]; returns c [N, K], r [N]."""
    R = 8.314462618
    rho = p / (R * T0 * (Y0 / W[:, None]).sum(axis=0))
    h = h_molar / W[:, None]
    hbar = (Y0 * h).sum(axis=0)
    c = -(rho[None, :] * (h - hbar[None, :])) / (dt * scale)
    r = (c * (Y1 - Y0)).sum(axis=0)
    return c.T.copy(), r
def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------------------------------
# the learned step's update of the cell state (Sec. 2.2 output definition with Eq. 7, and the
# fallback rules, which the paper does not state: range, non-finite values, element
# conservation, temperature range and an optional cap on |dT|)
# ------------------------------------------------------------------------------------------
FLAG_RANGE, FLAG_NONFINITE, FLAG_ELEMENTS, FLAG_T_RANGE, FLAG_DT = 1, 2, 4, 8, 16


def range_flags(T, p, Y, in_min, in_max, margin):
    """Bit FLAG_RANGE per cell when a raw input feature x = [T, p, F(Y_1..Y_K)] lies outside
    [min - m (max - min), max + m (max - min)] of the training set.  Y [K, n]."""
    raw = np.concatenate([np.asarray(T, np.float64)[None, :], np.asarray(p, np.float64)[None, :],
                          bct(Y)], axis=0)
    span = (in_max - in_min)[:, None]
    out = (raw < in_min[:, None] - margin * span) | (raw > in_max[:, None] + margin * span)
    return np.where(out.any(axis=0), FLAG_RANGE, 0).astype(np.int32), raw


def ann_update(orc, T, Y, U, out_mean, out_std, elem_tol=1e-2, T_min=250.0, T_max=3500.0,
               dT_max=0.0, flags_in=None):
    """New cell states from the network output U [n, >= K] (z-scored Box-Cox increments), FP64.

    Per cell, in this order:
      1. z_k = F(Y_k) + sigma_k U_k + mu_k and Y*_k = F^-1(z_k) (0 where lambda z + 1 <= 0);
         a non-finite z_k, or a sum of the Y*_k that is not finite and positive, flags the cell
         FLAG_NONFINITE and nothing else is evaluated;
      2. Y* <- Y* / sum_k Y*_k (unit mass);
      3. element moles e_e = sum_k a_ke Y_k / W_k before (Y) and after (Y*); the residual
         max_e |e*_e - e_e| / e_e over the elements present before (e_e > 0) above elem_tol
         flags FLAG_ELEMENTS;
      4. if not flagged, Y* is projected onto exact element conservation: the change dY
         minimising sum_k dY_k^2 / Y*_k subject to sum_k a_ke (Y*_k + dY_k)/W_k = e_e is
         dY_k = Y*_k sum_e (a_ke/W_k) lambda_e with (C diag(Y*) C^T) lambda = e - C Y*
         (C_ek = a_ke/W_k; elements absent from both states form zero rows and are left
         out), then Y'_k = max(Y*_k + dY_k, 0);
      5. T' from enthalpy conservation at constant p, h(T', Y') = h(T, Y) (Newton, the oracle's
         NASA-7), with Y' the projected state, or Y* itself when FLAG_ELEMENTS is set;
      6. a non-finite T' flags FLAG_NONFINITE, else T' outside [T_min, T_max] FLAG_T_RANGE,
         else (dT_max > 0) |T' - T| > dT_max FLAG_DT.
    Cells with a non-zero flags_in (the range flag, bit FLAG_RANGE) are left as they are.
    Flagged cells keep (T, Y).  `orc` is the mechanism's Oracle (W, composition, h, T(h)).

    Returns (T_new, Y_new [K, n], flags, info) with info the per-cell element residual and the
    unchecked T' (nan where not reached), for comparisons near a decision threshold.
    """
    T = np.asarray(T, np.float64)
    Y = np.asarray(Y, np.float64)
    K, n = Y.shape
    U = np.asarray(U, np.float64)[:, :K]
    Cm = orc.comp.astype(np.float64) / orc.W[:, None]          # [K, E] element moles per kg
    flags = np.zeros(n, np.int32) if flags_in is None else np.array(flags_in, np.int32)
    T_new, Y_new = T.copy(), Y.copy()
    res_out = np.full(n, np.nan)
    Tp_out = np.full(n, np.nan)
    for i in range(n):
        if flags[i]:
            continue
        y = Y[:, i]
        with np.errstate(over="ignore", invalid="ignore"):
            z = bct(y) + U[i] * out_std + out_mean
            ys = ibct(z)
            s = ys.sum()
        if not np.isfinite(z).all() or not (np.isfinite(s) and s > 0):
            flags[i] = FLAG_NONFINITE
            continue
        ys = ys / s
        e_old = Cm.T @ y
        e_new = Cm.T @ ys
        present = e_old > 0
        res = np.max(np.abs(e_new[present] - e_old[present]) / e_old[present]) if present.any() else 0.0
        res_out[i] = res
        f = 0
        if not (res <= elem_tol):
            f = FLAG_ELEMENTS
        else:
            M = Cm.T @ (ys[:, None] * Cm)
            act = np.diag(M) > 0
            rhs = (e_old - e_new)[act]
            Ma = M[np.ix_(act, act)]
            try:
                lam = np.linalg.solve(Ma, rhs)
            except np.linalg.LinAlgError:
                lam = np.linalg.lstsq(Ma, rhs, rcond=None)[0]
            ys = np.maximum(ys * (1.0 + Cm[:, act] @ lam), 0.0)
        h0 = orc.thermo_props(T[i], y)[1]
        Tp = orc.T_from_h(h0, ys, T0=T[i])
        Tp_out[i] = Tp
        if not np.isfinite(Tp):
            f |= FLAG_NONFINITE
        elif Tp < T_min or Tp > T_max:
            f |= FLAG_T_RANGE
        elif dT_max > 0 and abs(Tp - T[i]) > dT_max:
            f |= FLAG_DT
        flags[i] = f
        if f == 0:
            Y_new[:, i] = ys
            T_new[i] = Tp
    return T_new, Y_new, flags, {"elem_residual": res_out, "T_prime": Tp_out}
