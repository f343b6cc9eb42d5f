"""Stress fracture criterion (Sec. 3.2, Fracture Criteria) of the CUDA path against the oracle (needs a GB300).

The bond stresses sigma = |F_n|/S + |M_b| r0/I and tau = |F_s|/S + |M_t| r0/J are computed in FP64 in both
precisions, by the kernel the fracture test uses: they must match the oracle's (which differentiates the energy
parts by jets) to 1e-9 relative on a deformed lattice; a stress-driven tear must break the same bonds at the same
steps as the oracle's.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu
Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()
    oracle.build()


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED])
def test_bond_stresses_match_the_oracle(prec):
    """Every mode at once: a 4x4x4 lattice with random displacements and rotations of its particles."""
    sc = scenes.cube_lattice(nx=4, k_ground=0.0)
    rng = np.random.default_rng(11)
    p = sc.pos + rng.normal(size=sc.pos.shape) * 2e-4
    q = Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * 0.05).as_quat()
    sim = pkg.Sim(sc, precision=prec)
    sim.write_state(p, q, np.zeros((sc.n, 3)), np.zeros((sc.n, 4)))
    got = sim.bdem_debug_bond_stress()
    sim.close()
    o = oracle.OracleSim(sc)
    ref = o.bond_stresses(p, q)
    assert got.shape == ref.shape == (sc.nb, 2)
    scale = np.abs(ref).max(0)
    assert np.all(np.abs(got - ref) <= 1e-9 * np.abs(ref) + 1e-12 * scale)


def stress_textile(nx=12, steps=8):
    """The textile tear with the strain limit replaced by a tensile strength: sigma_c = 0.25 E."""
    sc = scenes.c3_textile(nx=nx, steps=steps)
    m = sc.materials[0]
    sc.materials = [dataclasses.replace(m, break_strain=math.inf, tensile_strength=0.25 * m.E)]
    return sc


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED])
def test_stress_driven_tear_breaks_the_same_bonds_as_the_oracle(prec):
    sc = stress_textile()
    cfg = dict(newton_rel_tol=1e-9)
    o = oracle.OracleSim(sc, cfg)
    sim = pkg.Sim(sc, precision=prec, config=cfg)
    total = 0
    for k in range(8):
        total += o.step(1)[0][0]["bonds_broken"]
        sim.step(1)
        st = sim.read_state()
        assert np.array_equal(st["broken"], o.broken), (k, np.nonzero(st["broken"] != o.broken))
    sim.close()
    assert total > 20  # the criterion is exercised inside the window
