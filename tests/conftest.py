import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_golden(name):
    """Parse a fixture under tests/golden: '# ...' comments, 'key: value' scalars,
    and 'key:' followed by rows of numbers."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, cur = {}, None
    import numpy as np
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if ":" in line:
                k, v = line.split(":", 1)
                v = v.strip()
                if v:
                    out[k] = float(v)
                    cur = None
                else:
                    cur = k
                    out[k] = []
                continue
            out[cur].append([float(x) for x in line.split()])
    return {k: (np.array(v) if isinstance(v, list) else v) for k, v in out.items()}


@pytest.fixture
def golden():
    return read_golden
