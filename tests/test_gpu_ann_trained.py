"""What the trained network gains over direct integration, at the stated error.

The committed network (trained on the GPU by this package's kernels on 8 M DI-generated
states, 60 epochs) runs the learned step with DI fallback on 100,000 held-out states of the
30-species workload; errors are measured against the DI result (within 1e-6 of the FP64
oracle by the parity tests) and the learned step is timed against DI on the same cells.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_18858_gb300 import workload as w  # noqa: E402

CKPT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2402_18858_gb300",
                    "models", "ann_c30_seed1.ckpt")


def test_trained_network_gain_over_di(mechs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem, train as tr
    build.build()
    m, path = mechs["c_30"]
    gm = chem.chem_load_mech(path)
    ann = chem.chem_ann_load(gm, CKPT)
    data = tr.di_states(gm, m, 100_000, 3, 5e-6)
    ev = tr.evaluate(gm, ann, data, 5e-6, repeats=2)
    e = ev["all_cells"]
    # stated error and gain (measured on 200 k held-out states: 0.075 % fallback, NRMS 0.24 %,
    # T p99 1.9 K, 104x)
    assert ev["failed"] == 0
    assert ev["fallback_fraction"] < 0.03
    assert e["species_nrms_max"] < 0.01
    assert e["T_p99_K"] < 5.0
    assert ev["speedup_vs_di"] > 20.0
    # the network does far better than leaving the state unchanged
    assert e["T_p99_K"] < 0.05 * ev["identity_map"]["T_p99_K"]
