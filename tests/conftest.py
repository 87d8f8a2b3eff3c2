import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built librexi.so")
    config.addinivalue_line("markers", "slow: longer CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """A fixture under tests/golden/: '# ' lines are comments, 'key value' lines give named
    scalars, every other line is a row of numbers."""
    import numpy as np
    keys, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if len(t) == 2 and t[0][0].isalpha():
                keys[t[0]] = float(t[1])
            else:
                rows.append([float(v) for v in t])
    return keys, np.array(rows)


def golden_rexi_step(name):
    """(parameters, U0, U1) of a stored REXI step: rows are field, index, U0 re/im, U1 re/im."""
    import numpy as np
    keys, rows = read_golden(name)
    nf, nlm = 3, int(rows[:, 1].max()) + 1
    U0 = np.zeros((nf, nlm), complex)
    U1 = np.zeros((nf, nlm), complex)
    f, i = rows[:, 0].astype(int), rows[:, 1].astype(int)
    U0[f, i] = rows[:, 2] + 1j * rows[:, 3]
    U1[f, i] = rows[:, 4] + 1j * rows[:, 5]
    return keys, U0, U1


@pytest.fixture
def golden():
    return read_golden


@pytest.fixture
def golden_step():
    return golden_rexi_step
