import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def tet_problem():
    from oracle import problem as P
    from synth import instances as I

    inst = I.tet()
    prob, d, allowed = P.make_problem(inst)
    return inst, prob


@pytest.fixture(scope="session")
def ico_problem():
    from oracle import problem as P
    from synth import instances as I

    inst = I.config1()
    prob, d, allowed = P.make_problem(inst)
    return inst, prob
