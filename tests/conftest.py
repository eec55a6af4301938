import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs of tens of seconds")


@pytest.fixture(scope="session")
def cfg1():
    import synth
    return synth.make_config(1)


@pytest.fixture(scope="session")
def cfg1_oracle(cfg1):
    import oracle
    mol, grid = cfg1
    return oracle.solve(mol, grid)


@pytest.fixture(scope="session")
def gwlib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1101_2065_gb300 as gw
    return gw


@pytest.fixture(scope="session")
def ctx(gwlib):
    c = gwlib.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="session")
def cfg2():
    import synth
    return synth.make_config(2)


@pytest.fixture(scope="session")
def cfg2_oracle(cfg2):
    import oracle
    mol, grid = cfg2
    return oracle.solve(mol, grid, keep_W_freqs=[1, 100, 400, 1023])
