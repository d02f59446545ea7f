import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def golden(name):
    """Rows of a whitespace-separated fixture under tests/golden (comments skipped)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture
def scratch(request):
    """A fresh, git-ignored folder inside the tree for one test's files."""
    import pathlib
    import shutil
    d = pathlib.Path(ROOT, "tests", "_scratch", request.node.name.replace("[", "_").replace("]", ""))
    if d.exists():
        shutil.rmtree(d)
    d.mkdir(parents=True)
    return d
