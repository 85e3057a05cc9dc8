import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

_POOL = {}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.hookimpl(trylast=True)
def pytest_collection_modifyitems(session, config, items):
    """Start the long oracle runs as soon as the session knows it will need
    them (a selected test uses the `oracle_jobs` fixture), so that they run in
    spawned workers while the other tests do."""
    if any("oracle_jobs" in getattr(it, "fixturenames", ()) for it in items):
        import tempfile
        import oracle_jobs
        d = tempfile.mkdtemp(prefix="ts_oracle_jobs_")
        _POOL["pool"] = oracle_jobs.Pool(d)
        _POOL["dir"] = d


@pytest.fixture(scope="session")
def oracle_jobs():
    pool = _POOL.get("pool")
    if pool is None:
        import tempfile
        import oracle_jobs as oj
        d = tempfile.mkdtemp(prefix="ts_oracle_jobs_")
        pool = _POOL["pool"] = oj.Pool(d)
        _POOL["dir"] = d
    return pool


def pytest_sessionfinish(session, exitstatus):
    pool = _POOL.pop("pool", None)
    if pool is not None:
        import shutil
        pool.close()
        shutil.rmtree(_POOL.pop("dir", ""), ignore_errors=True)
