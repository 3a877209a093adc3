import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workloads")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device; mark them skipped only when
    # selected explicitly on a machine without CUDA, so "-m gpu" on a box
    # with a GPU always runs them.
    try:
        import torch
        have = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have = False
    if have:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_sessionfinish(session, exitstatus):
    # the largest relative errors of every oracle comparison, per kind of
    # result, written where PARDTW_PARITY_LOG points (nothing otherwise)
    path = os.environ.get("PARDTW_PARITY_LOG")
    if not path:
        return
    from tests import _parity
    if not _parity.RECORD:
        return
    import json
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    with open(path, "w") as f:
        json.dump({"total_rel_bound": _parity.TOTAL_REL, "path_rel_bound": _parity.PATH_REL,
                   "near_zero": _parity.NEAR_ZERO, "results": _parity.RECORD}, f, indent=1)
