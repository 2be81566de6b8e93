"""Offline pipeline of the learned reaction step (Sec. 2.2, Fig. 2): generate states, integrate
them over dt with the GPU direct integration to get the targets (the paper uses CVODE), fit the
normalisation, train the MLP with the library's own kernels, and evaluate the learned step with
its DI fallback.  Every numerical step runs in libchem's kernels; this module only allocates
tensors and sequences the calls.

    python -m paper_2402_18858_gb300.train --train-cells 4000000 --epochs 40 --out ann.ckpt
"""
from __future__ import annotations

import argparse
import json
import math
import os
import tempfile
import time
from typing import Dict, Optional

import numpy as np
import torch

from . import build, chem, workload as wl

HIDDEN_30 = [1600, 800, 400]
HIDDEN_53 = [2000, 1000, 500]


def di_states(gm, m: wl.Mechanism, n: int, seed: int, dt: float, device="cuda", chunk: int = 1 << 20):
    """Seeded states and their DI results over dt (device tensors, SoA)."""
    st = wl.make_states(m, n, seed)
    dev = torch.device(device)
    T0 = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    T1, Y1 = T0.clone(), Y0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.zeros(chem.chem_workspace_bytes(gm, n), dtype=torch.uint8, device=dev)
    chem.chem_step_di(gm, dt, T1, p, Y1, status, workspace=ws)
    torch.cuda.synchronize()
    return dict(T0=T0, p=p, Y0=Y0, T1=T1, Y1=Y1, status=status, states=st)


def hfrd_states(gm, m: wl.Mechanism, n: int, seed: int, dt: float, device="cuda"):
    """Training states by the random augmentation of Eqs. 3-6 applied to seeded base states
    (chem_hfrd_augment), the kept ones integrated by DI over dt.  Draws base states until n are
    kept."""
    dev = torch.device(device)
    K = m.n_species
    parts, got, r = [], 0, 0
    while got < n:
        if r >= 8:
            raise RuntimeError(f"HFRD augmentation kept only {got} of {n} states after {r} rounds of draws")
        nb = max(2 * (n - got), 1024)
        st = wl.make_states(m, nb, seed + 1000 * r)
        g = torch.as_tensor(wl.uniform_draws(3 + K, nb, seed + 1000 * r + 1), device=dev)
        T = torch.as_tensor(st.T, device=dev)
        p = torch.as_tensor(st.p, device=dev)
        Y = torch.as_tensor(st.Y, device=dev)
        keep = torch.empty(nb, dtype=torch.int32, device=dev)
        ws = torch.empty(chem.chem_hfrd_workspace_bytes(), dtype=torch.uint8, device=dev)
        chem.chem_hfrd_augment(gm, T, p, Y, g, T, p, Y, keep, ws)
        sel = torch.nonzero(keep).flatten()[: n - got]
        parts.append((T[sel], p[sel], Y[:, sel]))
        got += sel.numel()
        r += 1
    T0 = torch.cat([a[0] for a in parts]).contiguous()
    p = torch.cat([a[1] for a in parts]).contiguous()
    Y0 = torch.cat([a[2] for a in parts], dim=1).contiguous()
    T1, Y1 = T0.clone(), Y0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.zeros(chem.chem_workspace_bytes(gm, n), dtype=torch.uint8, device=dev)
    chem.chem_step_di(gm, dt, T1, p, Y1, status, workspace=ws)
    torch.cuda.synchronize()
    return dict(T0=T0, p=p, Y0=Y0, T1=T1, Y1=Y1, status=status, states=None)


def hrr_terms(ann, T0, p, Y0, Y1, dt: float):
    """Coefficients and targets of the heat-release loss term (Eq. 10) in units of the training
    set's RMS step-mean heat release (first pass in W/m^3 to find that scale)."""
    n, K = T0.numel(), ann.n_out
    c = torch.empty((n, K), dtype=torch.float32, device=T0.device)
    r = torch.empty(n, dtype=torch.float32, device=T0.device)
    chem.chem_ann_hrr_coeffs(ann, dt, 1.0, T0, p, Y0, Y1, c, r)
    scale = float(torch.sqrt((r.double() ** 2).mean()).item()) or 1.0
    chem.chem_ann_hrr_coeffs(ann, dt, scale, T0, p, Y0, Y1, c, r)
    torch.cuda.synchronize()
    return c, r, scale


def prepare(ann, data, fit: bool = True, dt: Optional[float] = None):
    """Normalisation (if fit), BF16 features, raw Box-Cox inputs and normalised targets; with dt,
    also the heat-release loss terms (returned as a fourth item (c, r, scale))."""
    ok = data["status"] == 0
    T0, p, Y0, Y1 = data["T0"], data["p"], data["Y0"], data["Y1"]
    if not bool(ok.all()):
        keep = torch.nonzero(ok).flatten()
        T0, p = T0[keep].contiguous(), p[keep].contiguous()
        Y0, Y1 = Y0[:, keep].contiguous(), Y1[:, keep].contiguous()
    n = T0.numel()
    if fit:
        chem.chem_ann_fit_norm(ann, T0, p, Y0, Y1)
    X = torch.empty((n, 64), dtype=torch.bfloat16, device=T0.device)
    bcty = torch.empty((n, ann.n_out), dtype=torch.float32, device=T0.device)
    U = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device=T0.device)
    chem.chem_ann_features(ann, T0, p, Y0, X, bcty=bcty)
    chem.chem_ann_targets(ann, Y0, Y1, U)
    torch.cuda.synchronize()
    if dt is not None:
        return X, bcty, U, hrr_terms(ann, T0, p, Y0, Y1, dt)
    return X, bcty, U


def train(ann, X, bcty, U, epochs: int = 20, batch: int = 8192, lr: float = 1e-3, lr_min: float = 2e-5,
          w_data: float = 1.0, w_mass: float = 0.1, hrr=None, w_hrr: float = 0.0, seed: int = 0) -> Dict:
    """Adam over `epochs` calls of chem_ann_train_epoch (a seeded minibatch order per epoch,
    cosine learning rate over the whole run); the loss history holds each epoch's mean L_data."""
    n = X.shape[0]
    batch = min(batch, n) - min(batch, n) % 8
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    loss = torch.zeros(4, dtype=torch.float32, device=X.device)
    use_hrr = hrr is not None and w_hrr != 0.0
    hist = []
    t0 = time.perf_counter()
    for e in range(epochs):
        chem.chem_ann_train_epoch(ann, X, U, bcty, batch=batch, lr=lr, lr_min=lr_min, total_steps=total,
                                  step0=e * steps_per_epoch, seed=seed, epoch=e, w_data=w_data, w_mass=w_mass,
                                  hrr_c=hrr[0] if use_hrr else None, hrr_r=hrr[1] if use_hrr else None,
                                  w_hrr=w_hrr if use_hrr else 0.0, loss_out=loss)
        hist.append(((e + 1) * steps_per_epoch, float(loss[1].item())))
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    if chem.chem_ann_error(ann) != 0:
        raise RuntimeError("tensor-core pipeline timed out during training")
    return dict(steps=total, seconds=secs, loss_history=hist, samples_per_s=total * batch / secs)


def errors(T, Y, Tref, Yref, ok=None) -> Dict:
    """T error (max, p99) and per-species RMS normalised by the reference range (reading 13)."""
    T, Y, Tref, Yref = (x.cpu().numpy() if torch.is_tensor(x) else x for x in (T, Y, Tref, Yref))
    if ok is not None:
        T, Y, Tref, Yref = T[ok], Y[:, ok], Tref[ok], Yref[:, ok]
    dT = np.abs(T - Tref)
    rng = Yref.max(axis=1) - Yref.min(axis=1)
    rms = np.sqrt(((Y - Yref) ** 2).mean(axis=1)) / np.where(rng > 0, rng, 1.0)
    return dict(T_max_K=float(dT.max()) if dT.size else 0.0, T_p99_K=float(np.percentile(dT, 99)) if dT.size else 0.0,
                species_nrms_max=float(rms.max()) if rms.size else 0.0,
                species_nrms_mean=float(rms.mean()) if rms.size else 0.0)


def evaluate(gm, ann, data, dt: float, repeats: int = 3, **ann_opts) -> Dict:
    """ANN+fallback vs DI on the same cells: error (vs the DI result, itself within 1e-6 of
    the FP64 oracle) and throughput (CUDA events, best of `repeats`)."""
    T0, p, Y0, T1, Y1 = data["T0"], data["p"], data["Y0"], data["T1"], data["Y1"]
    n = T0.numel()
    dev = T0.device
    T, Y = T0.clone(), Y0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
    dws = torch.zeros(chem.chem_workspace_bytes(gm, n), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    best_ann, best_di = 1e30, 1e30
    for _ in range(repeats):
        T.copy_(T0)
        Y.copy_(Y0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        chem.chem_step_ann(gm, ann, dt, T, p, Y, status, ws, **ann_opts)
        e1.record(s)
        torch.cuda.synchronize()
        best_ann = min(best_ann, e0.elapsed_time(e1))
    st = status.cpu().numpy()
    Ta, Ya = T.clone(), Y.clone()
    for _ in range(max(1, repeats - 1)):
        T.copy_(T0)
        Y.copy_(Y0)
        st_di = torch.empty(n, dtype=torch.int32, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        chem.chem_step_di(gm, dt, T, p, Y, st_di, workspace=dws)
        e1.record(s)
        torch.cuda.synchronize()
        best_di = min(best_di, e0.elapsed_time(e1))
    ok_ref = data["status"].cpu().numpy() == 0
    learned = (st == 0) & ok_ref
    out = dict(cells=n, fallback_fraction=float((st != 0).mean()), ann_ms=best_ann, di_ms=best_di,
               ann_cells_per_s=n / (best_ann * 1e-3), di_cells_per_s=n / (best_di * 1e-3),
               speedup_vs_di=best_di / best_ann, failed=int(((st != 0) & (st != 5)).sum()))
    out["all_cells"] = errors(Ta, Ya, T1, Y1, ok_ref)
    out["learned_cells"] = errors(Ta, Ya, T1, Y1, learned)
    ident = errors(T0, Y0, T1, Y1, ok_ref)     # the state left unchanged, for scale
    out["identity_map"] = ident
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", default="c_30")
    ap.add_argument("--mech-seed", type=int, default=1)
    ap.add_argument("--train-cells", type=int, default=4_000_000)
    ap.add_argument("--eval-cells", type=int, default=2_000_000)
    ap.add_argument("--dt", type=float, default=5e-6)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--eval-seed", type=int, default=3)
    ap.add_argument("--out", default="")
    ap.add_argument("--with-moments", action="store_true", help="keep the Adam moments (resumable)")
    ap.add_argument("--repeats", type=int, default=3, help="timing repeats of the evaluation")
    ap.add_argument("--infer-cells", type=int, default=0,
                    help="> 0: also time the learned step with fallback on this many fresh cells")
    ap.add_argument("--elem-tol", type=float, default=1e-2)
    ap.add_argument("--w-hrr", type=float, default=0.0, help="weight W3 of the heat-release loss term (Eq. 10)")
    ap.add_argument("--hfrd", action="store_true",
                    help="train on states augmented by Eqs. 3-6 (random data method) instead of the plain draws")
    ap.add_argument("--per-species", action="store_true",
                    help="one 1600-800-400 network per species (Sec. 2.2) instead of one multi-output network")
    ap.add_argument("--dT-max", type=float, default=0.0, help="fallback cap on the predicted |dT| (0: none)")
    args = ap.parse_args()
    build.build()
    m = wl.make_mechanism(args.kind, args.mech_seed)
    path = wl.mechanism_file(args.kind, args.mech_seed, os.path.join(tempfile.gettempdir(), "chem_mech"))
    gm = chem.chem_load_mech(path)
    if args.per_species:
        ann = chem.chem_ann_create_per_species(gm, HIDDEN_30, seed=args.seed)
    else:
        ann = chem.chem_ann_create(gm, HIDDEN_30 if m.n_species <= 32 else HIDDEN_53, seed=args.seed)
    t0 = time.perf_counter()
    if args.hfrd:
        data = hfrd_states(gm, m, args.train_cells, args.seed, args.dt)
    else:
        data = di_states(gm, m, args.train_cells, args.seed, args.dt)
    gen_s = time.perf_counter() - t0
    hrr = None
    if args.w_hrr != 0.0:
        X, bcty, U, hrr = prepare(ann, data, dt=args.dt)
    else:
        X, bcty, U = prepare(ann, data)
    del data
    tr = train(ann, X, bcty, U, epochs=args.epochs, batch=args.batch, lr=args.lr,
               hrr=hrr, w_hrr=args.w_hrr)
    if args.out:
        chem.chem_ann_save(ann, args.out, with_moments=args.with_moments)
    del X, bcty, U
    ev = evaluate(gm, ann, di_states(gm, m, args.eval_cells, args.eval_seed, args.dt), args.dt,
                  repeats=args.repeats, elem_tol=args.elem_tol, dT_max=args.dT_max)
    out = dict(kind=args.kind, hidden=ann.dims, groups=ann.groups, hfrd=bool(args.hfrd), w_hrr=args.w_hrr,
               hrr_scale=hrr[2] if hrr is not None else None, data_generation_s=gen_s,
               di_generation_cells_per_s=args.train_cells / gen_s, train=tr, eval=ev)
    if args.infer_cells > 0:
        out["inference"] = time_inference(gm, m, ann, args.infer_cells, args.eval_seed + 1, args.dt,
                                          ev["di_cells_per_s"], elem_tol=args.elem_tol, dT_max=args.dT_max)
    hist = tr.pop("loss_history", None)
    out["loss_history"] = hist[-20:] if hist else None
    print(json.dumps(out))


def time_inference(gm, m: wl.Mechanism, ann, n: int, seed: int, dt: float, di_rate: float, repeats: int = 2,
                   **ann_opts) -> Dict:
    """Learned step with DI fallback on n fresh cells (best of `repeats`, CUDA events)."""
    st = wl.make_states(m, n, seed)
    dev = torch.device("cuda")
    T0 = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    del st
    T, Y = T0.clone(), Y0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    best = 1e30
    for _ in range(repeats):
        T.copy_(T0)
        Y.copy_(Y0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        chem.chem_step_ann(gm, ann, dt, T, p, Y, status, ws, **ann_opts)
        e1.record(s)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    fb = float((status != 0).float().mean().item())
    return dict(cells=n, ms=best, cells_per_s=n / (best * 1e-3), fallback_fraction=fb,
                speedup_vs_di=n / (best * 1e-3) / di_rate)


if __name__ == "__main__":
    main()
