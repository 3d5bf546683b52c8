import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


def load_fig3():
    """Parse tests/golden/fig3.txt into a dict of sections."""
    path = os.path.join(ROOT, "tests", "golden", "fig3.txt")
    sec = {}
    cur = None
    for line in open(path):
        line = line.rstrip("\n")
        if not line or line.startswith("#"):
            continue
        if line.endswith(":") and " " not in line:
            cur = line[:-1]
            sec[cur] = []
            continue
        if line.startswith("euler:"):
            sec["euler"] = int(line.split(":")[1])
            continue
        sec[cur].append(line)
    return sec


@pytest.fixture(scope="session")
def fig3():
    return load_fig3()
