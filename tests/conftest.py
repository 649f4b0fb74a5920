import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
SESSION_START = time.time()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


# The full-size precision test compares with a 5000-step FP64 oracle run of
# the 2048 x 1024 drop that takes 10-15 minutes on the host cores: start it
# in a background process as soon as the selection is known, so that it runs
# while the other GPU tests do.
LONG_REFERENCE_TEST = "test_precision_2048x1024_5000_steps"


def pytest_collection_finish(session):
    if not _cuda_available():
        return
    import long_reference
    for it in session.items:
        if it.originalname == LONG_REFERENCE_TEST and "gpu" in it.keywords:
            Ca = it.callspec.params.get("Ca") if hasattr(it, "callspec") else None
            skipped = any(m.name == "skip" or (m.name == "skipif" and m.args and m.args[0])
                          for m in it.iter_markers())
            if Ca is not None and not skipped:
                long_reference.start(Ca, 5000)


def pytest_sessionfinish(session, exitstatus):
    import long_reference
    long_reference.stop_all()
