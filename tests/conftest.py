"""Shared fixtures.  GPU tests are marked `gpu`; everything else runs on a CPU-only host."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def mech_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("mech"))


@pytest.fixture(scope="session")
def mechs(mech_dir):
    """Generated mechanism objects and their files for the three mechanism kinds."""
    from paper_2402_18858_gb300 import workload as w
    out = {}
    for kind, seed in (("h2_9", 0), ("c_30", 1), ("c_53", 5)):
        m = w.make_mechanism(kind, seed)
        path = os.path.join(mech_dir, f"{kind}.mech")
        w.write_mechanism(m, path)
        out[kind] = (m, path)
    return out


@pytest.fixture(scope="session")
def oracles(mechs):
    from oracle import Oracle
    return {k: Oracle(p) for k, (m, p) in mechs.items()}
