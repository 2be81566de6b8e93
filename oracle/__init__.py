"""CPU FP64 oracle for the per-cell chemistry step (test infrastructure).

Only the tests, the package's smoke check and the benchmark's CPU-baseline leg use this
package.  It shares no code with the GPU library: the C file here has its own mechanism
parser and formulas, and nothing here imports the GPU package.

Parity status of each function is recorded in its docstring; every function here is pinned by
a `-m "not gpu"` test against a closed form, an invariant, a special case or brute force,
except the MLP loss weights of Eq. 11, which the paper leaves unstated (see `mlp.py`).
"""
from .core import Oracle, build_oracle  # noqa: F401
