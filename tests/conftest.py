import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


# ---- oracle trajectories of the per-configuration parity report, computed in the background -----------------------
# When the report's tests are selected and a CUDA device is present, every case's oracle trajectory is queued at the
# end of collection in a pool of spawned worker processes, so that the oracle runs while the other GPU tests do; the
# report's tests then wait for their own case.
_PARITY_BATCH = None


def pytest_collection_finish(session):
    global _PARITY_BATCH
    if not any(it.nodeid.startswith("tests/test_gpu_parity_report.py") or "test_gpu_parity_report.py" in it.nodeid
               for it in session.items):
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except Exception:
        return
    import oracle_runs
    import parity_cases
    _PARITY_BATCH = oracle_runs.Batch()
    parity_cases.submit_all(_PARITY_BATCH)


def pytest_sessionfinish(session, exitstatus):
    global _PARITY_BATCH
    if _PARITY_BATCH is not None:
        _PARITY_BATCH.close()
        _PARITY_BATCH = None


@pytest.fixture(scope="session")
def parity_oracle():
    """result(key) -> (per-step oracle states, per-step stats) of a parity-report run (parity_cases.key)."""
    import oracle_runs
    import parity_cases

    class _Lazy:
        def result(self, name):
            global _PARITY_BATCH
            if _PARITY_BATCH is None:  # not queued at collection (e.g. run on its own): queue every case now
                _PARITY_BATCH = oracle_runs.Batch()
                parity_cases.submit_all(_PARITY_BATCH)
            return _PARITY_BATCH.result(name)

    return _Lazy()
