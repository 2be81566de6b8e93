"""One kernel case per invocation, for profilers (ncu) and quick timing.

    python -m paper_2402_18858_gb300.profile_cases di --cells 8192
    python -m paper_2402_18858_gb300.profile_cases di --kind c_53 --mech-seed 5 --dt 1e-5 --cells 16384
    python -m paper_2402_18858_gb300.profile_cases thermo --cells 1048576
    python -m paper_2402_18858_gb300.profile_cases thermo64 --cells 1048576
    python -m paper_2402_18858_gb300.profile_cases mlp --cells 65536
    python -m paper_2402_18858_gb300.profile_cases mlp_ps --cells 65536
    python -m paper_2402_18858_gb300.profile_cases ann --cells 2000000 --state-seed 3 --dt-cap 0
    python -m paper_2402_18858_gb300.profile_cases rates --cells 65536
    python -m paper_2402_18858_gb300.profile_cases jacobian --cells 8192
    python -m paper_2402_18858_gb300.profile_cases pasr --cells 1048576

Each case loads the 30-species workload mechanism (the DI case any mechanism kind and seed,
with its own dt), builds seeded inputs, runs the operation `--repeats` times (the first is the
warm-up) and prints the CUDA-event time of the last one.
"""
from __future__ import annotations

import argparse
import json
import os
import tempfile

import torch

from . import build, chem, workload as wl

MECH = ("c_30", 1)
CKPT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "models", "ann_c30_seed1.ckpt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["di", "thermo", "thermo64", "mlp", "mlp_ps", "ann", "rates", "jacobian", "pasr"])
    ap.add_argument("--cells", type=int, default=8192)
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--kind", default=MECH[0], help="mechanism kind (the DI case only; default c_30)")
    ap.add_argument("--mech-seed", type=int, default=MECH[1])
    ap.add_argument("--dt", type=float, default=5e-6, help="flow step of the DI case (s)")
    ap.add_argument("--state-seed", type=int, default=101, help="seed of the cell states")
    ap.add_argument("--dt-cap", type=float, default=0.0,
                    help="ann case: fallback when the predicted |dT| exceeds it (0: no cap)")
    a = ap.parse_args()
    if (a.kind, a.mech_seed) != MECH and a.case != "di":
        ap.error("--kind/--mech-seed apply to the di case only")
    build.build()
    mech = (a.kind, a.mech_seed)
    m = wl.make_mechanism(*mech)
    gm = chem.chem_load_mech(wl.mechanism_file(*mech, os.path.join(tempfile.gettempdir(), "chem_mech")))
    st = wl.make_states(m, a.cells, a.state_seed)
    dev = torch.device("cuda")
    T0 = torch.as_tensor(st.T, device=dev)
    p = torch.as_tensor(st.p, device=dev)
    Y0 = torch.as_tensor(st.Y, device=dev)
    n = a.cells
    if a.case == "di":
        status = torch.empty(n, dtype=torch.int32, device=dev)
        ws = torch.zeros(256, dtype=torch.uint8, device=dev)
        T, Y = T0.clone(), Y0.clone()
        stats = torch.zeros(4 * n, dtype=torch.int32, device=dev)

        def run():
            T.copy_(T0)
            Y.copy_(Y0)
            chem.chem_step_di(gm, a.dt, T, p, Y, status, workspace=ws, stats=stats)
    elif a.case == "rates":
        wdot = torch.empty_like(Y0)
        hrr = torch.empty_like(T0)

        def run():
            chem.chem_rates(gm, T0, p, Y0, wdot, hrr)
    elif a.case == "jacobian":
        nn = m.n_species + 1
        jac = torch.empty(n * nn * nn, dtype=torch.float64, device=dev)

        def run():
            chem.chem_jacobian(gm, T0, p, Y0, jac)
    elif a.case == "pasr":
        tf = wl.make_turbulence(n, 102)
        rho, k, eps, nu = (torch.as_tensor(x, device=dev) for x in (tf.rho, tf.k, tf.eps, tf.nu))
        Y1 = (Y0 * (1.0 + 1e-3 * torch.randn(Y0.shape, dtype=torch.float64, device=dev,
                                               generator=torch.Generator(device=dev).manual_seed(5)))).contiguous()
        omega = torch.empty_like(Y0)
        kap = torch.empty_like(T0)

        def run():
            chem.chem_pasr_source(gm, 5e-6, rho, Y0, Y1, k, eps, nu, omega, kap)
    elif a.case in ("thermo", "thermo64"):
        outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4)]
        mixed = a.case == "thermo"

        def run():
            chem.thermo_props(gm, T0, Y0, *outs, mixed_precision=mixed)
    elif a.case == "ann":
        # the learned step (features, MLP, update, fallback DI at rtol 1e-5) with the committed
        # network, in place on fresh copies of the states
        ann = chem.chem_ann_load(gm, CKPT)
        status = torch.empty(n, dtype=torch.int32, device=dev)
        ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)
        T, Y = T0.clone(), Y0.clone()

        def run():
            T.copy_(T0)
            Y.copy_(Y0)
            chem.chem_step_ann(gm, ann, a.dt, T, p, Y, status, ws, elem_tol=1e-2, dT_max=a.dt_cap,
                               di_rtol=1e-5, di_atol_Y=1e-10)
    elif a.case == "mlp_ps":
        # one 1600-800-400 network per species (grouped GEMMs), random weights
        ann0 = chem.chem_ann_load(gm, CKPT)
        ann = chem.chem_ann_create_per_species(gm, [1600, 800, 400], seed=2)
        chem.chem_ann_set_norm(ann, chem.chem_ann_get_norm(ann0))
        X = torch.empty((n, 64), dtype=torch.bfloat16, device=dev)
        chem.chem_ann_features(ann, T0, p, Y0, X)
        U = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device=dev)
        ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)

        def run():
            chem.chem_ann_forward(ann, X, U, ws)
    else:
        ann = chem.chem_ann_load(gm, CKPT)
        X = torch.empty((n, 64), dtype=torch.bfloat16, device=dev)
        chem.chem_ann_features(ann, T0, p, Y0, X)
        U = torch.empty((n, ann.n_out_pad), dtype=torch.float32, device=dev)
        ws = torch.empty(chem.chem_ann_workspace_bytes(ann, n), dtype=torch.uint8, device=dev)

        def run():
            chem.chem_ann_forward(ann, X, U, ws)
    ms = 0.0
    for _ in range(a.repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    out = {"case": a.case, "kind": a.kind, "cells": n, "ms": ms}
    if a.case == "di":
        # per-cell means of the kernel's counters: BDF steps, RHS, Jacobians, LU factorisations
        c = stats.view(4, n).double().mean(dim=1).tolist()
        out.update(steps=c[0], rhs=c[1], jac=c[2], lu=c[3], failed=int((status != 0).sum().item()))
    if a.case == "ann":
        out.update(fallback=int((status != 0).sum().item()))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
