import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size workload (minutes)")


def pytest_collection_modifyitems(config, items):
    # keep the file order stable: pytest collects files alphabetically, and the
    # no-allocation test file is named to come last
    pass


@pytest.fixture(autouse=True)
def _no_failed_bounds_checks(request):
    """Under HELM_LIBRARY=check (the bounds-checking build of the library) every GPU test
    must end without a failed check of a kernel's global access."""
    yield
    if os.environ.get("HELM_LIBRARY") != "check" or "gpu" not in request.keywords:
        return
    from paper_2209_10886_gb300 import helm
    if helm._lib is None:
        return
    rep = helm.check_bounds_report(reset=True)
    assert rep["checking_build"] and rep["violations"] == 0, f"failed bounds checks: {rep}"


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")
