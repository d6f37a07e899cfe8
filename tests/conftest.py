import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Per-result relative L2 errors recorded by the GPU parity tests (record_rel),
# appended as JSON lines to $HD_PARITY_REPORT when that is set.


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def rel_l2(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    return num / den if den > 0 else num


def record_rel(case, err, tol, n=None):
    """Keep one result's relative L2 error against the oracle for the report."""
    path = os.environ.get("HD_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"case": case, "relL2": float(err), "tol": float(tol), "outputs_checked": n}) + "\n")
    return err


@pytest.fixture
def rel():
    return rel_l2
