import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU case")


def read_golden(name):
    """Parse a tests/golden/*.txt fixture: '# comment' lines are skipped;
    returns a list of token lists (comments after '#' stripped)."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def golden_dict(name):
    return {r[0]: float(r[1]) for r in read_golden(name) if len(r) == 2}


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def oracle_table(oracle_mod):
    """The oracle's own 400 x 200 node table (0 <= D <= 30), cached on disk."""
    return oracle_mod.cached_table(400, 30.0, 200, oracle_mod.QUAD_TABLE)


@pytest.fixture(scope="session")
def oracle_spline(oracle_mod, oracle_table):
    return oracle_mod.Spline(oracle_table, 30.0)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
