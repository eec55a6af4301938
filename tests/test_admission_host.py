"""The serving engine's admission estimate (gw_server_job_bytes), a host-only
function of the C ABI: no GPU needed.  Its dominant term is the N_omega
complex packed triangles of chi0 and of the factors, so for a fixed grid it
grows as N_sub^2 and for a fixed molecule linearly in N_omega."""
import pytest

import synth
from synth import molecules as sm


@pytest.fixture(scope="module")
def gwlib():
    from paper_1101_2065_gb300 import build, gw
    gw.load(build.build())
    return gw


def _chain(atoms):
    return sm._uniform_molecule("chain", atoms, 1)


def test_estimate_follows_the_packed_triangles(gwlib):
    g1, g2 = synth.Grid(1024), synth.Grid(2048)
    m = _chain(40)
    b1 = gwlib.Server.job_bytes(m, g1, gwlib.GW_MIXED)
    b2 = gwlib.Server.job_bytes(m, g2, gwlib.GW_MIXED)
    n = m.n_sub
    tri = n * (n + 1) // 2
    # two complex binary32 triangles per frequency (chi0 or M, and the factors), with 1/8 slack
    per_omega = (b2 - b1) / 1024
    assert 2 * tri * 8 <= per_omega <= 1.25 * (2 * tri * 8 + (n + 32) * 32 * 8)
    # binary64 doubles the complex elements
    assert gwlib.Server.job_bytes(m, g1, gwlib.GW_FP64) > 1.8 * b1
    # N_sub^2 at a fixed grid: 40 -> 80 atoms is about 4x
    r = gwlib.Server.job_bytes(_chain(80), g1, gwlib.GW_MIXED) / b1
    assert 3.5 < r < 4.6


def test_estimate_grows_with_the_states(gwlib):
    g = synth.Grid(1024)
    m = _chain(40)
    assert gwlib.Server.job_bytes(m, g, gwlib.GW_MIXED, n_states=8) > gwlib.Server.job_bytes(m, g, gwlib.GW_MIXED)
