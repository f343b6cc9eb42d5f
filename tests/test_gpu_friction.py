"""Post-step friction (Sec. 5.4, Friction) of the CUDA path against physics and the oracle (needs a GB300).

A sphere at its equilibrium penetration on the ground slides with Coulomb deceleration mu_s g per unit time and
stops exactly; the plate construction with sliding and rotation friction follows the oracle (positions: FP64 path
1e-9, mixed path 1e-4 of the scene size; velocities: the same over one time step).
"""
import math

import numpy as np
import pytest

import oracle
import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu
TOL = {pkg.BDEM_FP64: 1e-9, pkg.BDEM_MIXED: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()
    oracle.build()


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED])
def test_sliding_sphere_coulomb_deceleration(prec):
    r, rho, k, g, dt, mu, v0 = 0.005, 2500.0, 1e5, 9.81, 1e-3, 0.3, 0.05
    m = rho * 4.0 / 3.0 * math.pi * r ** 3
    cfg = scenes.default_config(dt=dt, k_ground=k, friction_slide=mu)
    sc = scenes._assemble(np.array([[0.0, 0.0, r - m * g / k]]), np.full(1, r), np.zeros(1, np.int32),
                          np.zeros(1, np.uint8), np.zeros((0, 2), np.int64), [scenes.Material(1e7, 0.3, rho)], cfg,
                          "sphere", vel=np.array([[v0, 0.0, 0.0]]))
    sim = pkg.Sim(sc, precision=prec)
    stop = math.ceil(v0 / (mu * g * dt))
    for n in range(1, stop + 3):
        sim.step(1)
        v = sim.read_state()["vel"][0]
        assert v[0] == pytest.approx(max(v0 - n * mu * g * dt, 0.0), abs=1e-9), n
    assert abs(v[0]) < 1e-15
    sim.close()


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED])
def test_plate_with_friction_matches_the_oracle(prec):
    sc = scenes.c2_plate_small(R=0.015)
    sc.config = dict(sc.config, friction_slide=0.5, friction_roll=0.05)
    o = oracle.OracleSim(sc)
    sim = pkg.Sim(sc, precision=prec)
    L = float(np.linalg.norm(sc.pos.max(0) - sc.pos.min(0)))
    vtol = TOL[prec] * L / sc.config["dt"]  # a position tolerance over one step
    for k in range(3):
        o.step(1)
        sim.step(1)
        st, ref = sim.read_state(), o.state()
        assert np.abs(st["pos"] - ref["pos"]).max() <= TOL[prec] * L, k
        assert np.abs(st["vel"] - ref["vel"]).max() <= vtol, k
        assert np.array_equal(st["broken"], ref["broken"]), k
    sim.close()
