import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


# Parity results (relative final-cost error and per-vertex pose error against
# the oracle) collected by the GPU parity tests and printed at the end of the
# run, one line per result.
PARITY_RESULTS = []


@pytest.fixture
def parity_record():
    def rec(name, rel_cost, pose_err=None):
        import numpy as np
        row = {"case": name, "rel_cost": float(rel_cost)}
        if pose_err is not None and len(pose_err):
            pe = np.asarray(pose_err, dtype=float)
            row["pose_max"] = float(pe.max())
            row["pose_rms"] = float(np.sqrt(np.mean(pe * pe)))
        PARITY_RESULTS.append(row)
        return row
    return rec


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if not PARITY_RESULTS:
        return
    tr = terminalreporter
    tr.section("parity against the FP64 oracle (final cost; pose error |log(S_gpu S_oracle^-1)|)")
    for r in PARITY_RESULTS:
        pe = ""
        if "pose_max" in r:
            pe = f"  pose max {r['pose_max']:.2e} rms {r['pose_rms']:.2e}"
        tr.write_line(f"{r['case']:<44} rel cost {r['rel_cost']:.2e}{pe}")
