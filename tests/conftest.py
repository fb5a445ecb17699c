import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# achieved errors per output, written at the end of the session to the JSON
# file named by SG_PARITY_RECORD (nothing is written without it)
_RECORD = {}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and the built libsg.so")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture
def record_error(request):
    """record_error(output_name, **figures): keeps the achieved error figures
    of one compared output under the test's name."""
    def rec(name, **figures):
        clean = {k: (float(v) if hasattr(v, "__float__") else v) for k, v in figures.items()}
        _RECORD.setdefault(request.node.nodeid, {})[name] = clean
    return rec


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("SG_PARITY_RECORD")
    if path and _RECORD:
        with open(path, "w") as f:
            json.dump(_RECORD, f, indent=1, sort_keys=True)
