"""Device-side time limits (needs a GB300): a wait that runs out returns a status and leaves the simulation usable.

Every device wait of the library (the persistent PCG's grid barrier) gives up after a time limit, sets a flag and
returns; the host turns the flag into BDEM_E_TIMEOUT. The test runs a wait on a word that nothing writes with a
short limit: the call must return BDEM_E_TIMEOUT after about that long, without a fault, and the same simulation
must then step exactly like a fresh one.
"""
import time

import numpy as np
import pytest

import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()


@pytest.mark.parametrize("limit_ms", [0.0, 50.0])
def test_wait_that_runs_out_returns_timeout_and_the_sim_stays_usable(limit_ms):
    sc = scenes.cube_lattice(nx=3, z_bottom=0.006, k_ground=1e6)
    sim = pkg.Sim(sc, precision=pkg.BDEM_FP64)
    t0 = time.perf_counter()
    st = sim.bdem_debug_wait_timeout(limit_ms)
    dt = time.perf_counter() - t0
    assert st == pkg.BDEM_E_TIMEOUT
    assert limit_ms * 1e-3 <= dt < limit_ms * 1e-3 + 1.0
    assert sim.bdem_debug_wait_timeout(limit_ms) == pkg.BDEM_E_TIMEOUT  # and again: the flag was reset
    sim.step(3)
    got = sim.read_state()
    ref = pkg.Sim(sc, precision=pkg.BDEM_FP64)
    ref.step(3)
    want = ref.read_state()
    for k in ("pos", "quat", "vel", "quat_vel"):
        assert np.array_equal(got[k], want[k]), k
    sim.close()
    ref.close()
