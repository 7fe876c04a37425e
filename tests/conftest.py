import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_finish(session):
    """Starts the long oracle runs of the selected GPU parity tests in a spawned
    process pool now, after selection and before any test touches the GPU, so
    they overlap the rest of the suite (tests/oracle_jobs.py)."""
    from tests import oracle_jobs
    names = []
    for it in session.items:
        base = it.name.split("[")[0]
        if base in oracle_jobs.JOB_OF_TEST and it.get_closest_marker("gpu") is not None:
            names.append(oracle_jobs.JOB_OF_TEST[base])
    if names:
        oracle_jobs.start(sorted(set(names)))


def pytest_sessionfinish(session, exitstatus):
    from tests import oracle_jobs
    oracle_jobs.shutdown()
