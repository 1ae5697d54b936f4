import json
import os
import sys
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def load_worked_example():
    """The 3-state IMDP of Sec. 3.1 as CSC arrays (0-based), plus exact bounds."""
    with open(os.path.join(TESTS, "golden", "worked_example.json")) as f:
        ex = json.load(f)
    n = ex["n_states"]
    stateptr = [0]
    colptr = [0]
    rowval, lower, upper, exact = [], [], [], []
    for s in range(n):
        for a in range(len(ex["actions"][s])):
            for d in range(n):
                lo = ex["lower"][s][a][d]
                up = ex["upper"][s][a][d]
                if up == 0.0 and lo == 0.0:
                    continue  # structural zero: not stored in CSC
                rowval.append(d)
                lower.append(lo)
                upper.append(up)
                exact.append((Fraction(ex["lower_decimal"][s][a][d]), Fraction(ex["upper_decimal"][s][a][d])))
            colptr.append(len(rowval))
        stateptr.append(len(colptr) - 1)
    return dict(
        n_states=n,
        stateptr=np.array(stateptr, np.int32),
        colptr=np.array(colptr, np.int32),
        rowval=np.array(rowval, np.int32),
        lower=np.array(lower, np.float64),
        upper=np.array(upper, np.float64),
        exact=exact,
        goal=np.array([g - 1 for g in ex["goal_1based"]], np.int32),
        horizon=ex["horizon"],
    )


@pytest.fixture(scope="session")
def worked_example():
    return load_worked_example()
