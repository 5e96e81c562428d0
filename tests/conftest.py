import os
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libpse.so")


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


@pytest.fixture(scope="session")
def record_error():
    """record_error(case, **numbers): appends one JSON line per measured error
    to the file named by the environment variable PSE_ERROR_LOG (if set), so
    that a GPU run leaves a table of the errors against the FP64 oracle."""
    import json

    path = os.environ.get("PSE_ERROR_LOG")

    def rec(case, **vals):
        if path:
            with open(path, "a") as f:
                f.write(json.dumps({"case": case, **{k: (float(v) if not isinstance(v, (str, int)) else v)
                                                     for k, v in vals.items()}}) + "\n")
    return rec
