import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer statistical test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


def pytest_sessionfinish(session, exitstatus):
    """With HSG_PARITY_REPORT set to a path, write what the parity checks
    measured (per check: sites compared, sites excluded by the rules,
    ill-conditioned sites, max errors) there as JSON."""
    path = os.environ.get("HSG_PARITY_REPORT")
    rules = sys.modules.get("parity_rules")
    if not path or rules is None:
        return
    import json

    with open(path, "w") as f:
        json.dump(rules.REPORT, f, indent=0)
