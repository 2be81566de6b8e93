#!/usr/bin/env python3
"""Benchmark of the per-cell chemistry step on GB300.

One step = one pass of the hot path over one batch of synthetic cells resident in HBM:
direct integration of Eq. 2 for every cell (FP64 BDF, chem_step_di) followed by the mixture
property update (thermo_props, FP64).  Default workload: the 30-species / 180-reaction (8 Troe)
synthetic C/H/O/N mechanism, 1,000,000 cells, dt = 5e-6 s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--cells C]

Prints one JSON line (rank 0).  `--impl reference` times the CPU FP64 oracle on this host's
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_18858_gb300 import workload as wl  # noqa: E402

METRIC = "chem-step cells/s: GPU DI vs ANN+fallback at stated err; serve p50/p99 ms"
WORKLOAD = "di_c_30sp_1m"
DI_RTOL = 1e-9           # library defaults (rtol 1e-9, atol_Y 1e-18, Newton 0.2): what the parity tests validate
MECH_DIR = os.path.join(tempfile.gettempdir(), "chem_bench_mech")
# FP64 flops of one exponential and one logarithm, FMA = 2: those of the kernels' own routines --
# the table-driven exp (5 FMAs + 1 multiply + the 2 FMAs of the argument reduction: 13), its
# form for arguments kept in units of ln2/256 (rate constants, equilibrium-constant factors,
# falloff terms: 4 FMAs + 1 multiply + 1 subtraction: 10) and the log (8 FMAs + 4 others: 20)
EXP_FLOPS = 13
EXP_S_FLOPS = 10
LOG_FLOPS = 20
ORACLE_ERR_RTOL = 1e-8   # oracle tolerance for the learned step's error reference (far below its error)


def load_peaks() -> dict:
    """Roofline denominators: the measured figures of MEASURED_PEAKS.json, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "of measured (MEASURED_PEAKS.json)"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "of fallback"}


PEAKS = load_peaks()
# DRAM bytes of one di_kernel launch per cell, from an 8,202-cell ncu capture of the current
# kernel (dram__bytes_read.sum + dram__bytes_write.sum = 2,968,576 + 0 B; the written state
# stayed in L2 there), scaled to a launch by the cells processed
DI_DRAM_BYTES_PER_CELL = 2968576 / 8202


# ------------------------------------------------------------------------------------------
# algorithmic FP64 work model of the DI kernel (per call of each building block)
# ------------------------------------------------------------------------------------------
def di_flop_model(m: wl.Mechanism) -> dict:
    """FP64 flops of one RHS, one Jacobian, one LU and one Newton solve for this mechanism.

    Conventions: add/mul = 1, fma = 2, division = 1, exp = EXP_FLOPS or EXP_S_FLOPS (pre-scaled
    arguments), log = LOG_FLOPS (the FP64 operations of the kernels' own exp and log).  Counts
    follow the textbook formulas (NASA-7, Arrhenius, K_c, Troe, Eq. 1 and its analytic
    Jacobian)."""
    K, n = m.n_species, m.n_species + 1
    E = len(m.elements)
    nnz = 0
    rx = 0
    jx = 0
    for r in m.reactions:
        nr, npd = len(r.reactants), len(r.products)
        nnz += len(set(r.reactants) | set(r.products))
        c = 4 + EXP_S_FLOPS             # k_f = exp(ln A + b ln T - Ea/RT)
        c += (nr + npd) + 2             # 1/K_c from per-species exp(-g/RT) products, (p0/RT)^dnu
        c += (nr - 1) + (npd - 1) + 3   # concentration products, q
        if r.kind >= 1:
            c += 2 + 2 * len(r.eff)     # [M]
        if r.kind == 2:
            # Troe: k0/k_inf and F_cent's two or three exponentials, log10 F_cent and log10 P_r,
            # F = 10^(...), and the algebra (F_cent, P_r, c, n, x, the two divisions, k)
            n_exp = 1 + (len(r.troe) - 1)
            c += n_exp * (EXP_S_FLOPS + 2) + (EXP_FLOPS + 2) + 2 * (LOG_FLOPS + 1) + 40
        rx += c
        # Jacobian extras: dq/dC terms per species of the reaction, d/dT terms
        jx += 2 * (nr * nr + npd * npd) + 12 + (30 if r.kind == 2 else 0)
    # per species: NASA-7 c_p, h, s and dc_p/dT, g/RT, exp(-g/RT), concentration, element
    # terms; per cell: ln T and the scalars of the energy equation
    species = K * (8 + 10 + 10 + 1 + 2 + 4 + 2 * E + EXP_S_FLOPS + 1) + LOG_FLOPS + 10
    f_rhs = species + rx + 2 * nnz + 4 * K + 6
    f_jac = f_rhs + 2 * nnz * 3 + jx + 7 * K * K + 10 * K
    f_lu = 2 * n ** 3 / 3 + 2 * n * n
    f_solve = 2 * n * n + 6 * n
    return dict(rhs=f_rhs, jac=f_jac, lu=f_lu, solve=f_solve, step=30 * n)


def thermo_fp64_flops(K: int, mixed: bool) -> int:
    """FP64 flops per cell of the property kernel.  Both modes: sum Y_k/W_k (K FMAs), the six
    mixture coefficients A_i = sum_k Y_k a_ik/W_k (6K FMAs), c_p and h from them (~20).  FP64
    mode also: ln T and the reciprocals (~40); per species the mole fraction (2), the ln mu and
    ln lambda cubics (12), four exponentials (4 (EXP + 1)), the conductivity sums (4) and
    X/s, X/s^2 (2); Wilke's three sums (3 FMAs = 6 flops per species pair) and per species the
    denominator, the reciprocal and the sum (17).  The mixed mode's transport runs in FP32."""
    base = 2 * K + 2 * 6 * K + 20
    if mixed:
        return base
    return base + 40 + K * (2 + 12 + 4 * (EXP_FLOPS + 1) + 4 + 2 + 17) + 6 * K * K


def di_flops(stats: np.ndarray, fm: dict) -> float:
    steps, rhs, jac, lu = (stats[i].astype(np.float64) for i in range(4))
    solves = np.maximum(rhs - 2, 0)     # every RHS after the first two feeds one Newton solve
    return float((rhs * fm["rhs"] + jac * (fm["jac"] - fm["rhs"]) + lu * fm["lu"]
                  + solves * fm["solve"] + steps * fm["step"]).sum())


# ------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    def __init__(self, index: int = 0):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"chem_clocks_{os.getpid()}.csv")
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 4 + i and r[4 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
def cpu_baseline(m_path: str, m: wl.Mechanism, cfg: dict, cells: int, seed_offset: int = 0) -> dict:
    """The oracle on this host's cores over a bounded sample of the workload (cells/s)."""
    from oracle import Oracle
    o = Oracle(m_path)
    st = wl.make_states(m, cells, cfg["state_seed"] + 7919 * (1 + seed_offset))
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    _, _, status, _ = o.integrate_batch(st.T, st.p, st.Y, cfg["dt"], nthreads=threads)
    el = time.perf_counter() - t0
    return {"value": cells / el, "unit": "cells/s", "cores": threads, "kind": "oracle",
            "sample": f"{cells} cells of {WORKLOAD} (same mechanism, state distribution and dt), "
                      f"Radau IIA rtol 1e-10, OpenMP over cells", "seconds": el,
            "failed_cells": int((status != 0).sum())}


def run_reference(args, cfg, m, m_path):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cells = args.ref_cells
    for _ in range(args.warmup):
        cpu_baseline(m_path, m, cfg, max(cells // 8, 16))
    times = []
    for k in range(args.steps):
        r = cpu_baseline(m_path, m, cfg, cells, seed_offset=k)
        times.append(r["seconds"])
    value = cells * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "cells_per_step": cells, "dt": cfg["dt"]},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{cells} cells per step of {WORKLOAD}, Radau IIA rtol 1e-10"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# PaSR source assembly (the step after the chemistry step): HBM-bound, thread per cell
# ------------------------------------------------------------------------------------------
def run_pasr(gm, m, N, dt, Y0, Y1, seed, dev):
    import torch
    from paper_2402_18858_gb300 import chem
    tf = wl.make_turbulence(N, seed)
    rho, k, eps, nu = (torch.as_tensor(a, device=dev) for a in (tf.rho, tf.k, tf.eps, tf.nu))
    omega = torch.empty_like(Y0)
    kap = torch.empty_like(rho)
    s = torch.cuda.current_stream()
    times = []
    for r in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        chem.chem_pasr_source(gm, dt, rho, Y0, Y1, k, eps, nu, omega, kap)
        e1.record(s)
        torch.cuda.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    K = m.n_species
    bytes_cell = (3 * K + 5) * 8          # Y0, Y1, rho, k, eps, nu read; omega, kappa written
    gbs = N * bytes_cell / (ms * 1e-3) / 1e9
    kap_np = kap.cpu().numpy()
    return {"workload": f"{N} cells, {K} species, seeded sub-grid fields (5 % laminar)",
            "ms": ms, "cells_per_s": N / (ms * 1e-3), "bytes_per_cell": bytes_cell,
            "kappa_mean": float(kap_np.mean()), "kappa_laminar_or_1": float((kap_np == 1.0).mean()),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": PEAKS["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / PEAKS["hbm_gbs"], "kernel": "pasr_kernel",
                         "peak_source": "hbm_gbs " + PEAKS["source"]}}


# ------------------------------------------------------------------------------------------
# learned step (ANN + DI fallback): train on DI-generated states, then time inference
# ------------------------------------------------------------------------------------------
ANN_WORKLOAD = "ann_c_30sp_2m"
ANN_ELEM_TOL = 1e-2


def mlp_flops_per_cell(dims) -> int:
    return sum(2 * dims[l] * dims[l + 1] for l in range(len(dims) - 1))


ANN_CKPT = os.path.join(ROOT, "paper_2402_18858_gb300", "models", "ann_c30_seed1.ckpt")


def oracle_errors(m_path, T0, p, Y0, results, dt, pick):
    """T max / p99 and per-species RMS / range of learned-step results against the FP64 oracle
    (Radau IIA at ORACLE_ERR_RTOL) on the sampled cells `pick` (host arrays; several result
    sets: results = dict name -> (T [n], Y [K, n]))."""
    from oracle import Oracle
    from paper_2402_18858_gb300 import train as tr
    o = Oracle(m_path)
    t0 = time.perf_counter()
    To, Yo, so, _ = o.integrate_batch(T0[pick], p[pick], Y0[:, pick], dt, rtol=ORACLE_ERR_RTOL,
                                      nthreads=os.cpu_count() or 1)
    secs = time.perf_counter() - t0
    ok = so == 0
    out = {"reference": f"oracle (Radau IIA, rtol {ORACLE_ERR_RTOL:g}) on {pick.size} cells sampled "
                        f"from the timed batch ({secs:.1f} s on {os.cpu_count()} host cores)",
           "oracle_failed": int((~ok).sum())}
    for name, (T, Y) in results.items():
        e = tr.errors(T[pick], Y[:, pick], To, Yo, ok)
        rng = Yo[:, ok].max(axis=1) - Yo[:, ok].min(axis=1)
        nrms = np.sqrt(((Y[:, pick][:, ok] - Yo[:, ok]) ** 2).mean(axis=1)) / np.where(rng > 0, rng, 1.0)
        e["species_nrms"] = [round(float(v), 6) for v in nrms]
        out[name] = e
    return out


def run_ann(args, m, gm, di_rate, m_path):
    import torch
    from paper_2402_18858_gb300 import chem, train as tr
    dt = wl.WORKLOADS[WORKLOAD]["dt"]
    if os.path.exists(ANN_CKPT) and not args.ann_retrain:
        # trained offline by paper_2402_18858_gb300.train (16 M DI samples, 100 epochs, GPU)
        ann = chem.chem_ann_load(gm, ANN_CKPT)
        provenance = {"source": "paper_2402_18858_gb300/models/ann_c30_seed1.ckpt",
                      "train_cells": 16_000_000, "train_epochs": 100}
    else:
        t0 = time.perf_counter()
        data = tr.di_states(gm, m, args.ann_train_cells, 2, dt)
        gen_s = time.perf_counter() - t0
        ann = chem.chem_ann_create(gm, tr.HIDDEN_30, seed=2)
        X, bcty, U = tr.prepare(ann, data)
        del data
        trn = tr.train(ann, X, bcty, U, epochs=args.ann_epochs, batch=8192, lr=1e-3)
        del X, bcty, U
        provenance = {"source": "trained in this run", "train_cells": args.ann_train_cells,
                      "train_epochs": args.ann_epochs, "data_generation_s": gen_s, "train_s": trn["seconds"],
                      "train_samples_per_s": trn["samples_per_s"]}
    # three operating points of the learned step, all with a fallback DI at rtol 1e-5 (the
    # fallback's own error stays far below the network's): "fast" falls back on range and
    # element-residual checks only, "balanced" and "accurate" also on a predicted |dT| above
    # 100 K and 50 K.  The fallback cells are the hard (igniting) ones: a Jacobian re-evaluated
    # every 50 accepted steps and the Newton stop at 0.1 of the error test (CVODE's values)
    # serve them better than the library's defaults, which are tuned on the whole workload
    fb_di = dict(di_rtol=1e-5, di_atol_Y=1e-10, di_newton_tol=0.1, di_jac_max_age=50)
    points = {"fast": dict(elem_tol=ANN_ELEM_TOL, dT_max=0.0, **fb_di),
              "balanced": dict(elem_tol=ANN_ELEM_TOL, dT_max=100.0, **fb_di),
              "accurate": dict(elem_tol=ANN_ELEM_TOL, dT_max=50.0, **fb_di)}
    # accuracy against DI on held-out cells (DI is within 1e-6 of the FP64 oracle)
    ev_data = tr.di_states(gm, m, 100_000, 3, dt)
    errs = {k: tr.evaluate(gm, ann, ev_data, dt, repeats=1, **o) for k, o in points.items()}
    del ev_data
    # throughput of ANN + fallback on the full inference batch (2 M cells), and the MLP alone
    n = args.ann_cells
    st = wl.make_states(m, n, 3)
    dev = torch.device("cuda")
    T0 = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    T, Y = T0.clone(), Y0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    X = torch.empty((n, 64), dtype=torch.bfloat16, device=dev)
    Uo = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device=dev)
    chem.chem_ann_features(ann, T0, p, Y0, X)
    # DI at the fallback's own tolerance on the same cells: the like-for-like speed-up
    sd = torch.empty(n, dtype=torch.int32, device=dev)
    dws = torch.zeros(chem.chem_workspace_bytes(gm, n), dtype=torch.uint8, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    T.copy_(T0)
    Y.copy_(Y0)
    e0.record(s)
    chem.chem_step_di(gm, dt, T, p, Y, sd, rtol=fb_di["di_rtol"], atol_Y=fb_di["di_atol_Y"],
                      newton_tol=fb_di["di_newton_tol"], jac_max_age=fb_di["di_jac_max_age"], workspace=dws)
    e1.record(s)
    torch.cuda.synchronize()
    di_same_tol = n / (e0.elapsed_time(e1) * 1e-3)
    report = {"workload": f"{ANN_WORKLOAD}: MLP {ann.dims}, BF16 tcgen05, {n} cells, dt {dt}",
              "network": provenance, "points": {},
              "di_same_tol": {"options": fb_di, "cells_per_s": di_same_tol}}
    results = {}
    mlp_times = []
    for name, o in points.items():
        times = []
        for _ in range(3):
            T.copy_(T0)
            Y.copy_(Y0)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(s)
            chem.chem_step_ann(gm, ann, dt, T, p, Y, status, ws, **o)
            e1.record(s)
            chem.chem_ann_forward(ann, X, Uo, ws)
            e2.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            mlp_times.append(e1.elapsed_time(e2))
        best = float(np.median(times))       # the median of the repeats, like the DI figures
        results[name] = (T.cpu().numpy(), Y.cpu().numpy())
        fb = float((status != 0).float().mean().item())
        rate = n / (best * 1e-3)
        ev = errs[name]
        report["points"][name] = {"options": o, "cells_per_s": rate, "ms": best, "fallback_fraction": fb,
                                  "speedup_vs_di": rate / di_rate,
                                  "speedup_vs_di_same_tol": rate / di_same_tol,
                                  "error_vs_di_100k_heldout": {"fallback_fraction": ev["fallback_fraction"],
                                                               **ev["all_cells"]}}
    pick = np.sort(np.random.default_rng(11).choice(n, args.oracle_err_cells, replace=False))
    oe = oracle_errors(m_path, st.T, st.p, st.Y, results, dt, pick)
    for name in points:
        report["points"][name]["error_vs_oracle"] = oe.pop(name)
    report["error_vs_oracle_reference"] = oe
    best_mlp = float(np.median(mlp_times))
    mlp_tf = mlp_flops_per_cell(ann.dims) * n / (best_mlp * 1e-3) / 1e12
    acc = report["points"]["accurate"]
    report.update({"cells_per_s": acc["cells_per_s"], "speedup_vs_di": acc["speedup_vs_di"],
                   "speedup_vs_di_same_tol": acc["speedup_vs_di_same_tol"],
                   "fallback_fraction": acc["fallback_fraction"],
                   "error_vs_di_100k_heldout": acc["error_vs_di_100k_heldout"],
                   "mlp_ms": best_mlp, "mlp_tflops": mlp_tf, "mlp_cells_per_s": n / (best_mlp * 1e-3)})
    peak = PEAKS["bf16_tflops"]
    roof = {"bound": "tensor", "achieved": mlp_tf, "peak": peak, "unit": "TFLOP/s", "frac": mlp_tf / peak,
            "traffic": None, "kernel": "gemm_bf16_kernel (MLP forward, 2 M cells)",
            "peak_source": "bf16_tflops (burst) " + PEAKS["source"]}
    report["per_species_mlp"] = run_per_species_forward(gm, ann, X, Uo, mlp_tf)
    return {"report": report, "roofline": roof, "ann": ann}


def run_per_species_forward(gm, ann, X, Uo, multi_tflops):
    """Forward cost of one 1600-800-400 network per species (Sec. 2.2) on the same features:
    grouped tensor-core GEMMs, one launch per layer for all species (random weights: the cost
    does not depend on them; accuracy of trained per-species networks is measured offline)."""
    import torch
    from paper_2402_18858_gb300 import chem, train as tr
    ps = chem.chem_ann_create_per_species(gm, tr.HIDDEN_30, seed=2)
    chem.chem_ann_set_norm(ps, chem.chem_ann_get_norm(ann))
    n = min(X.shape[0], 262_144)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ps, n), dtype=torch.uint8, device=X.device)
    s = torch.cuda.current_stream()
    chem.chem_ann_forward(ps, X[:n], Uo[:n], ws)
    times = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        chem.chem_ann_forward(ps, X[:n], Uo[:n], ws)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    best = float(np.median(times))
    if chem.chem_ann_error(ps) != 0:
        raise RuntimeError("tensor-core pipeline timed out in the per-species forward")
    fpc = ps.groups * mlp_flops_per_cell(ps.dims)
    tf = fpc * n / (best * 1e-3) / 1e12
    multi = mlp_flops_per_cell(ann.dims)
    return {"workload": f"{ps.groups} networks {ps.dims}, BF16 tcgen05 grouped GEMMs, {n} cells",
            "cells": n, "ms": best, "cells_per_s": n / (best * 1e-3), "flops_per_cell": fpc,
            "flops_vs_multi_output": fpc / multi, "tflops": tf, "frac_of_bf16_peak": tf / PEAKS["bf16_tflops"],
            "time_vs_multi_output": (fpc / multi) * multi_tflops / tf}


# ------------------------------------------------------------------------------------------
# the other configurations of the metric: config 0 (9 species) and config 4 (53 species)
# ------------------------------------------------------------------------------------------
ANN_C53_CKPT = os.path.join(ROOT, "paper_2402_18858_gb300", "models", "ann_c53_seed5.ckpt")


def time_di(gm, m, st, dt, peak_gf, repeats):
    """GPU DI over the states `st` (resident; copies restored before each run): median time,
    cells/s and the FP64 roofline of the di_kernel launch."""
    import torch
    from paper_2402_18858_gb300 import chem
    dev = torch.device("cuda")
    n = st.T.size
    T0, p, Y0 = (torch.as_tensor(a, device=dev) for a in (st.T, st.p, st.Y))
    T, Y = T0.clone(), Y0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    stats = torch.empty(4 * n, dtype=torch.int32, device=dev)
    ws = torch.zeros(chem.chem_workspace_bytes(gm, n), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(repeats):
        T.copy_(T0)
        Y.copy_(Y0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        chem.chem_step_di(gm, dt, T, p, Y, status, rtol=DI_RTOL, stats=stats, workspace=ws)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    best = float(np.median(times))
    stn = stats.cpu().numpy().reshape(4, n)
    flops = di_flops(stn, di_flop_model(m))
    tf = flops / (best * 1e-3) / 1e12
    return {"ms": best, "cells_per_s": n / (best * 1e-3), "failed_cells": int((status != 0).sum().item()),
            "steps_per_cell": float(stn[0].mean()), "flops_per_cell": flops / n,
            "roofline": {"bound": "alu", "achieved": tf, "peak": peak_gf / 1e3, "unit": "TFLOP/s",
                         "frac": tf / (peak_gf / 1e3), "kernel": "di_kernel (FP64 DFMA pipe)"}}


def run_config0(peak_gf):
    """Config 0: 9-species H/O/N mechanism, 4,096 cells, dt = 1e-6 s, GPU DI."""
    from paper_2402_18858_gb300 import chem
    cfg = wl.WORKLOADS["di_h2_9sp_4k"]
    m = wl.make_mechanism(cfg["kind"], cfg["mech_seed"])
    gm = chem.chem_load_mech(wl.mechanism_file(cfg["kind"], cfg["mech_seed"], MECH_DIR))
    st = wl.make_states(m, cfg["n"], cfg["state_seed"])
    r = time_di(gm, m, st, cfg["dt"], peak_gf, repeats=7)
    r["workload"] = f"di_h2_9sp_4k: {m.n_species} species / {m.n_reactions} reactions, {cfg['n']} cells, dt {cfg['dt']}"
    return r


def run_config4(args, peak_gf):
    """Config 4: 53 species / 320 reactions (12 falloff), dt = 1e-5 s.  GPU DI on a seeded
    subsample of the 8,000,000-cell batch (per-cell cost is independent of the batch), the
    learned step with DI fallback on all 8,000,000 cells (committed 2000-1000-500 network), its
    speed-up and its error against the FP64 oracle on cells sampled from the timed batch."""
    import torch
    from paper_2402_18858_gb300 import chem
    cfg = wl.WORKLOADS["di_c_53sp_8m"]
    m = wl.make_mechanism(cfg["kind"], cfg["mech_seed"])
    m_path = wl.mechanism_file(cfg["kind"], cfg["mech_seed"], MECH_DIR)
    gm = chem.chem_load_mech(m_path)
    n, dt = cfg["n"] if not args.c53_cells else args.c53_cells, cfg["dt"]
    st = wl.make_states(m, n, cfg["state_seed"])
    nsub = min(args.c53_di_cells, n)
    sub = wl.States(T=st.T[:nsub].copy(), p=st.p[:nsub].copy(), Y=np.ascontiguousarray(st.Y[:, :nsub]))
    di = time_di(gm, m, sub, dt, peak_gf, repeats=2)
    out = {"workload": f"di_c_53sp_8m: {m.n_species} species / {m.n_reactions} reactions, {n} cells, dt {dt}",
           "di": {**di, "sample": f"first {nsub} cells of the batch (per-cell work does not depend on the batch)"}}
    if not os.path.exists(ANN_C53_CKPT):
        out["ann"] = None
        return out
    ann = chem.chem_ann_load(gm, ANN_C53_CKPT)
    dev = torch.device("cuda")
    T0, p, Y0 = (torch.as_tensor(a, device=dev) for a in (st.T, st.p, st.Y))
    T, Y = T0.clone(), Y0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
    o = dict(elem_tol=ANN_ELEM_TOL, dT_max=0.0, di_rtol=1e-5, di_atol_Y=1e-10, di_newton_tol=0.1, di_jac_max_age=50)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(2):
        T.copy_(T0)
        Y.copy_(Y0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        chem.chem_step_ann(gm, ann, dt, T, p, Y, status, ws, **o)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    best = float(np.median(times))
    rate = n / (best * 1e-3)
    pick = np.sort(np.random.default_rng(12).choice(n, args.oracle_err_cells_c53, replace=False))
    oe = oracle_errors(m_path, st.T, st.p, st.Y, {"ann": (T.cpu().numpy(), Y.cpu().numpy())}, dt, pick)
    out["ann"] = {"network": "paper_2402_18858_gb300/models/ann_c53_seed5.ckpt (4 M DI states, 40 epochs)",
                  "dims": ann.dims, "options": o, "ms": best, "cells_per_s": rate,
                  "fallback_fraction": float((status != 0).float().mean().item()),
                  "speedup_vs_di": rate / di["cells_per_s"], "error_vs_oracle": oe.pop("ann"),
                  "error_vs_oracle_reference": oe}
    return out


# ------------------------------------------------------------------------------------------
# serving: Poisson arrivals of mixed requests through continuous batching
# ------------------------------------------------------------------------------------------
def run_serve(args, m30, g30, ann_leg, di_rate30):
    """Config 3's request shape: cells log-uniform in [1e3, 2e6], 50/50 9-/30-species and
    DI/learned modes, Poisson arrivals at 70 % of the measured capacity.  The count is bounded
    (--serve-requests) so that the leg stays within about a minute of arrivals."""
    import torch
    from paper_2402_18858_gb300 import chem, train as tr
    m9 = wl.make_mechanism("h2_9", 0)
    g9 = chem.chem_load_mech(wl.mechanism_file("h2_9", 0, MECH_DIR))
    # 9-species classes: a small learned step trained the same way
    d9 = tr.di_states(g9, m9, 200_000, 12, 1e-6)
    a9 = chem.chem_ann_create(g9, [256, 128], seed=4)
    X, bcty, U = tr.prepare(a9, d9)
    tr.train(a9, X, bcty, U, epochs=10, batch=8192, lr=1e-3)
    del X, bcty, U
    ev9 = tr.evaluate(g9, a9, d9, 1e-6, repeats=1)
    di_rate9 = ev9["di_cells_per_s"]
    a30 = ann_leg["ann"] if ann_leg else None
    rate_ann30 = ann_leg["report"]["cells_per_s"] if ann_leg else di_rate30
    rng = np.random.default_rng(4)
    R = args.serve_requests
    lo, hi = 1e3, 2e6
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), R)).astype(int)
    kind = rng.random(R) < 0.5            # True: 30 species
    mode = (rng.random(R) < 0.5).astype(int)
    if a30 is None:
        mode[kind] = 0
    svc = np.where(kind, np.where(mode == 1, 1.0 / rate_ann30, 1.0 / di_rate30),
                   np.where(mode == 1, 1.0 / ev9["ann_cells_per_s"], 1.0 / di_rate9)) * sizes
    lam = 0.7 / svc.mean()                 # arrivals at 70 % of the measured capacity
    gaps = rng.exponential(1.0 / lam, R)
    # the requests' states, made before the clock starts, in pinned host memory: copies from
    # and to pageable memory would block the server's scheduler thread until they complete
    keep = []

    def pinned(a=None, shape=None, dtype=np.float64):
        if a is not None:
            shape, dtype = a.shape, a.dtype
        t = torch.empty(shape, dtype={np.float64: torch.float64, np.int32: torch.int32}[np.dtype(dtype).type],
                        pin_memory=True)
        keep.append(t)
        v = t.numpy()
        if a is not None:
            v[...] = a
        return v
    payload = []
    for i in range(R):
        mm = m30 if kind[i] else m9
        st = wl.make_states(mm, int(sizes[i]), 50_000 + i)
        payload.append(((pinned(st.T), pinned(st.p), pinned(st.Y)), pinned(shape=(sizes[i],)),
                        pinned(shape=(mm.n_species, sizes[i])), pinned(shape=(sizes[i],), dtype=np.int32)))
    sv = chem.chem_server_create(hbm_budget_bytes=16 << 30, n_streams=args.serve_streams, max_batch_cells=1 << 20,
                                 starvation_s=30.0, di_chunk_cells=args.serve_chunk)
    c30 = chem.chem_server_add_class(sv, g30, a30, capacity_cells=1 << 23)
    c9 = chem.chem_server_add_class(sv, g9, a9, capacity_cells=1 << 23)
    reqs = []
    t0 = time.perf_counter()
    for i in range(R):
        cls, dt = (c30, wl.WORKLOADS[WORKLOAD]["dt"]) if kind[i] else (c9, 1e-6)
        (T_in, p_in, Y_in), To, Yo, so = payload[i]
        target = t0 + gaps[:i + 1].sum()
        while time.perf_counter() < target:
            time.sleep(min(1e-3, max(0.0, target - time.perf_counter())))
        reqs.append(chem.chem_server_submit(sv, cls, int(mode[i]), dt, T_in, p_in, Y_in, To, Yo, so))
    for r in reqs:
        done, res = chem.chem_server_wait(sv, r, 900.0)
        if not done or res != 0:
            raise RuntimeError(f"serving request {r} did not complete ({done}, {res})")
    stt = chem.chem_server_stats(sv)
    lat = np.array([chem.chem_server_request_latency(sv, r) for r in reqs])
    del sv, payload, keep

    def pct(sel):
        v = lat[sel]
        return {"n": int(v.size), "p50_ms": float(np.percentile(v, 50)) if v.size else None,
                "p99_ms": float(np.percentile(v, 99)) if v.size else None}
    small = sizes < 30_000
    breakdown = {"cells_lt_3e4": pct(small), "cells_ge_3e4": pct(~small),
                 "di_30sp": pct(kind & (mode == 0)), "di_9sp": pct(~kind & (mode == 0)),
                 "ann_30sp": pct(kind & (mode == 1)), "ann_9sp": pct(~kind & (mode == 1))}
    return {"workload": f"{R} requests, cells log-uniform [{int(lo)}, {int(hi)}] (config 3's shape; count "
                        f"bounded), 50/50 9-/30-species, 50/50 DI/ANN, Poisson arrivals at 70 % of measured "
                        f"capacity ({lam:.3f}/s)",
            "p50_ms": stt["p50_ms"], "p99_ms": stt["p99_ms"], "mean_ms": stt["mean_ms"], "max_ms": stt["max_ms"],
            "cells_per_s": stt["cells_per_s"], "batches": stt["batches"],
            "mean_batch_requests": stt["mean_batch_requests"], "wall_s": stt["wall_s"],
            "failed": stt["failed"], "latency_by_kind": breakdown,
            "p99_cause": "the largest 30-species DI requests: their own GPU time (up to 2e6 cells at the DI "
                         f"rate) sets the tail; pieces of {args.serve_chunk} cells keep them from holding back "
                         "small requests",
            "host_buffers": "pinned",
            "scheduler": f"pieces of <= {args.serve_chunk} cells per DI request per launch, kind with the least "
                         f"work left first, 30 s starvation limit, {args.serve_streams} streams"}


# ------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=0, help="override the cell count (profiling)")
    ap.add_argument("--ref-cells", type=int, default=1024)
    ap.add_argument("--cpu-cells", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ann", action="store_true", help="skip the learned-step leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--ann-retrain", action="store_true", help="train the network in this run")
    ap.add_argument("--ann-train-cells", type=int, default=500_000)
    ap.add_argument("--ann-epochs", type=int, default=24)
    ap.add_argument("--ann-cells", type=int, default=2_000_000)
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--serve-streams", type=int, default=2)
    ap.add_argument("--serve-chunk", type=int, default=32768, help="cells of a DI request per launch")
    ap.add_argument("--oracle-err-cells", type=int, default=512,
                    help="cells of the timed learned-step batch compared with the FP64 oracle")
    ap.add_argument("--oracle-err-cells-c53", type=int, default=128)
    ap.add_argument("--no-config4", action="store_true", help="skip the 53-species legs")
    ap.add_argument("--c53-cells", type=int, default=0, help="override config 4's cell count")
    ap.add_argument("--c53-di-cells", type=int, default=65536, help="config 4 DI subsample")
    args = ap.parse_args()

    cfg = dict(wl.WORKLOADS[WORKLOAD])
    if args.cells:
        cfg["n"] = args.cells
    m = wl.make_mechanism(cfg["kind"], cfg["mech_seed"])
    m_path = wl.mechanism_file(cfg["kind"], cfg["mech_seed"], MECH_DIR)

    if args.impl == "reference":
        run_reference(args, cfg, m, m_path)
        return

    import torch
    from paper_2402_18858_gb300 import build, chem, sharding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    gm = chem.chem_load_mech(m_path)
    N = cfg["n"]
    # weak scaling: every rank owns its own batch of N cells (independent problems, no collective)
    st = wl.make_states(m, N, sharding.rank_state_seed(cfg["state_seed"], rank))
    dev = torch.device("cuda", local)
    T0 = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    T, Y = T0.clone(), Y0.clone()
    status = torch.empty(N, dtype=torch.int32, device=dev)
    stats = torch.empty(4 * N, dtype=torch.int32, device=dev)
    ws = torch.zeros(chem.chem_workspace_bytes(gm, N), dtype=torch.uint8, device=dev)
    cp, h, mu, kap = (torch.empty(N, dtype=torch.float64, device=dev) for _ in range(4))
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step(i=None):
        T.copy_(T0)
        Y.copy_(Y0)
        if i is not None:
            ev[i][0].record(stream)
        chem.chem_step_di(gm, cfg["dt"], T, p, Y, status, rtol=DI_RTOL, stats=stats, workspace=ws)
        if i is not None:
            ev[i][1].record(stream)
        chem.thermo_props(gm, T, Y, cp, h, mu, kap, mixed_precision=False)
        if i is not None:
            ev[i][2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            step(i)
        t1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = sharding.max_over_ranks(t0.elapsed_time(t1) / args.steps, device=dev)
    di_ms = float(np.mean([a.elapsed_time(b) for a, b, c in ev]))
    th_ms = float(np.mean([b.elapsed_time(c) for a, b, c in ev]))
    st_np = status.cpu().numpy()
    stats_np = stats.cpu().numpy().reshape(4, N)
    fm = di_flop_model(m)
    flops = di_flops(stats_np, fm)
    peak_gf = chem.chem_fp64_peak_gflops()
    hbm = PEAKS["hbm_gbs"]
    achieved_tf = flops / (di_ms * 1e-3) / 1e12
    th_bytes = N * (m.n_species + 1) * 8 + N * 4 * 8
    th_gbs = th_bytes / (th_ms * 1e-3) / 1e9
    th_flops_cell = thermo_fp64_flops(m.n_species, mixed=False)
    th_tf = th_flops_cell * N / (th_ms * 1e-3) / 1e12

    # the properties in the mixed mode (FP32 transport sums) beside the step's FP64 mode
    thm = []
    for r in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chem.thermo_props(gm, T, Y, cp, h, mu, kap, mixed_precision=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            thm.append(e0.elapsed_time(e1))
    thm_ms = float(np.median(thm))

    # PaSR filtered source from this step (Y0 -> Y after DI) with seeded sub-grid fields
    pasr = run_pasr(gm, m, N, cfg["dt"], Y0, Y, cfg["state_seed"] + 3, dev)

    # end to end through the public API from pinned host buffers (copies inside the timed region)
    hT = torch.as_tensor(st.T).pin_memory()
    hY = torch.as_tensor(st.Y).pin_memory()
    oT = torch.empty_like(hT).pin_memory()
    oY = torch.empty_like(hY).pin_memory()
    ost = torch.empty(N, dtype=torch.int32).pin_memory()

    def e2e_step():
        T.copy_(hT, non_blocking=True)
        Y.copy_(hY, non_blocking=True)
        chem.chem_step_di(gm, cfg["dt"], T, p, Y, status, rtol=DI_RTOL, workspace=ws)
        chem.thermo_props(gm, T, Y, cp, h, mu, kap, mixed_precision=False)
        oT.copy_(T, non_blocking=True)
        oY.copy_(Y, non_blocking=True)
        ost.copy_(status, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ke2e = max(1, min(args.steps, 2))
    e0.record(stream)
    for _ in range(ke2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = sharding.max_over_ranks(e0.elapsed_time(e1) / ke2e, device=dev)
    h2d = hT.numel() * 8 + hY.numel() * 8
    d2h = oT.numel() * 8 + oY.numel() * 8 + ost.numel() * 4

    di_rate = N / (di_ms * 1e-3)
    cfg0 = run_config0(peak_gf) if world == 1 else None
    cfg4 = run_config4(args, peak_gf) if (world == 1 and not args.no_config4) else None
    ann = None if args.no_ann else run_ann(args, m, gm, di_rate, m_path)
    serve = None if (args.no_serve or world > 1) else run_serve(args, m, gm, ann, di_rate)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(m_path, m, cfg, args.cpu_cells)
            cpu.pop("seconds", None)
        line = {
            "metric": METRIC, "value": sharding.job_throughput(N, world, ms * 1e-3), "unit": "cells/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": N, "species": m.n_species,
                       "reactions": m.n_reactions, "dt": cfg["dt"], "di_rtol": DI_RTOL,
                       "step": "chem_step_di (FP64 BDF) + thermo_props (FP64)",
                       "l2": f"inputs {N * (m.n_species + 1) * 8 / 1e6:.0f} MB > 129 MB L2",
                       "parallelism": f"dp{world} (independent cells, no collective)"},
            "di_cells_per_s": N / (di_ms * 1e-3), "di_ms": di_ms, "thermo_ms": th_ms,
            "thermo_gbs": th_gbs, "failed_cells": int((st_np != 0).sum()),
            "di_steps_per_cell": float(stats_np[0].mean()),
            "di_work_per_step": {"rhs": float(stats_np[1].sum() / max(stats_np[0].sum(), 1)),
                                 "jac": float(stats_np[2].sum() / max(stats_np[0].sum(), 1)),
                                 "lu": float(stats_np[3].sum() / max(stats_np[0].sum(), 1))},
            "di_flops_per_cell": flops / N,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_gf / 1e3,
                         "unit": "TFLOP/s", "frac": achieved_tf / (peak_gf / 1e3),
                         "traffic": DI_DRAM_BYTES_PER_CELL * N, "kernel": "di_kernel (FP64 DFMA pipe)",
                         "peak_source": "measured live: chem_fp64_peak_gflops DFMA probe"},
            "thermo_roofline": {"bound": "alu", "achieved": th_tf, "peak": peak_gf / 1e3, "unit": "TFLOP/s",
                                "frac": th_tf / (peak_gf / 1e3), "kernel": "thermo_kernel (FP64)",
                                "flops_per_cell": th_flops_cell,
                                "note": "FP64 Wilke sums (3 FMAs per species pair) bound it; HBM side: "
                                        f"{th_gbs:.0f} GB/s = {th_gbs / hbm:.3f} of {hbm:.0f} (hbm_gbs {PEAKS['source']})",
                                "hbm_gbs": th_gbs, "hbm_frac": th_gbs / hbm},
            "thermo_mixed": {"ms": thm_ms, "cells_per_s": N / (thm_ms * 1e-3),
                             "fp64_flops_per_cell": thermo_fp64_flops(m.n_species, mixed=True),
                             "note": "thermo_props with the O(K^2) transport sums in FP32 (c_p, h in FP64), "
                                     "same 1,000,000 cells; the step uses the FP64 mode"},
            "config0": cfg0,
            "config4": cfg4,
            "peaks": PEAKS,
            "e2e": {"value": sharding.job_throughput(N, world, e2e_ms * 1e-3), "unit": "cells/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * args.steps,  # di_kernel + thermo_kernel per step
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "ann": ann["report"] if ann else None,
            "tensor_roofline": ann["roofline"] if ann else None,
            "serve": serve,
            "pasr": pasr,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
