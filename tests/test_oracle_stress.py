"""Pins of the oracle's stress fracture criterion (Sec. 3.2, Fracture Criteria) against closed forms.

sigma = |F_n|/S + |M_b| r0/I and tau = |F_s|/S + |M_t| r0/J with F_n, F_s the position gradients of the stretch
and shear potentials and K t the bend-twist moment. On a two-particle bond along x (rest length l0, r0 = r) each
single deformation mode has a closed form:
  axial extension d:          sigma = kn |d| / S = E |d| / l0,            tau = 0
  relative twist phi about x: sigma = 0,  tau = (GJ/l0) sin(phi/2) r0/J = G r0 sin(phi/2) / l0
  relative bend phi about y:  sigma = (EI/l0) sin(phi/2) r0/I = E r0 sin(phi/2) / l0,  tau = 0
  common rotation phi about z (shear angle phi): tau = kt s^2 phi / (l0 S) = G s^2 phi / l0^2,  sigma = 0
and for pure axial loading the stress criterion with sigma_c = E eps_c breaks the bond at the same step as the
strain criterion with limit eps_c.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_10459_gb300 import scenes

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

E, NU, R, L0, S_SCALE = 2e8, 0.25, 0.004, 0.01, 0.007
G = E / (2 * (1 + NU))


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def pair(sigma_c=math.inf, tau_c=math.inf, break_strain=math.inf, kinematic=(0, 0)):
    pos = np.array([[0.0, 0.0, 0.0], [L0, 0.0, 0.0]])
    cfg = scenes.default_config(dt=1e-3, gravity=(0.0, 0.0, 0.0))
    mat = scenes.Material(E, NU, 2500.0, break_strain, 1.0, S_SCALE, sigma_c, tau_c)
    return scenes._assemble(pos, np.full(2, R), np.zeros(2, np.int32), np.array(kinematic, np.uint8),
                            np.array([[0, 1]]), [mat], cfg, "pair")


def stress_at(pos, quat):
    o = oracle.OracleSim(pair())
    return o.bond_stress(0, pos, quat)


def q_of(axis, angle):
    return Rotation.from_rotvec(np.asarray(axis, float) * angle).as_quat()


IDENT = np.array([[0.0, 0.0, 0.0, 1.0], [0.0, 0.0, 0.0, 1.0]])


@pytest.mark.parametrize("d", [1e-5, -3e-5])
def test_axial_extension(d):
    s, t = stress_at(np.array([[0.0, 0.0, 0.0], [L0 + d, 0.0, 0.0]]), IDENT)
    assert s == pytest.approx(E * abs(d) / L0, rel=1e-10)
    assert abs(t) <= 1e-12 * E * abs(d) / L0


@pytest.mark.parametrize("phi", [0.01, 0.3])
def test_relative_twist(phi):
    pos = np.array([[0.0, 0.0, 0.0], [L0, 0.0, 0.0]])
    q = np.stack([q_of([1, 0, 0], phi / 2), q_of([1, 0, 0], -phi / 2)])
    s, t = stress_at(pos, q)
    assert t == pytest.approx(G * R * math.sin(phi / 2) / L0, rel=1e-10)
    assert abs(s) <= 1e-9 * t


@pytest.mark.parametrize("phi", [0.01, 0.3])
def test_relative_bend(phi):
    pos = np.array([[0.0, 0.0, 0.0], [L0, 0.0, 0.0]])
    q = np.stack([q_of([0, 1, 0], phi / 2), q_of([0, 1, 0], -phi / 2)])
    s, t = stress_at(pos, q)
    assert s == pytest.approx(E * R * math.sin(phi / 2) / L0, rel=1e-10)
    assert abs(t) <= 1e-9 * s


@pytest.mark.parametrize("phi", [0.01, 0.3])
def test_common_rotation_is_pure_shear(phi):
    pos = np.array([[0.0, 0.0, 0.0], [L0, 0.0, 0.0]])
    q = np.stack([q_of([0, 0, 1], phi), q_of([0, 0, 1], phi)])
    s, t = stress_at(pos, q)
    assert t == pytest.approx(G * S_SCALE ** 2 * phi / L0 ** 2, rel=1e-9)
    assert abs(s) <= 1e-9 * t


def test_endpoints_and_rigid_motion_leave_stresses_unchanged():
    """The stresses of a deformed pair do not change under a rigid rotation and translation of the pair."""
    rng = np.random.default_rng(3)
    pos = np.array([[0.0, 0.0, 0.0], [L0 + 2e-5, 3e-5, -1e-5]])
    q = np.stack([q_of(rng.normal(size=3), 0.05), q_of(rng.normal(size=3), 0.04)])
    base = stress_at(pos, q)
    Rg = Rotation.from_rotvec([0.3, -0.7, 0.2])
    pos2 = Rg.apply(pos) + np.array([1.0, -2.0, 0.5])
    q2 = (Rg * Rotation.from_quat(q)).as_quat()
    assert np.allclose(stress_at(pos2, q2), base, rtol=1e-9)


def test_stress_criterion_under_axial_pull_matches_the_strain_criterion():
    """Both particles kinematic, pulled apart at 0.5 m/s: the bond is in pure tension, sigma = E eps, so the
    stress criterion with sigma_c = E eps_c breaks it at the same step as the strain criterion with eps_c."""
    eps_c = 0.12
    steps = {}
    for name, sc in (("strain", pair(break_strain=eps_c, kinematic=(1, 1))),
                     ("stress", pair(sigma_c=E * eps_c, kinematic=(1, 1)))):
        sc.vel[0, 0], sc.vel[1, 0] = -0.25, 0.25
        o = oracle.OracleSim(sc)
        for n in range(1, 10):
            if o.step(1)[0][0]["bonds_broken"]:
                steps[name] = n
                break
    assert steps["strain"] == steps["stress"] == math.ceil(eps_c * L0 / (0.5 * 1e-3))


def test_shear_strength_breaks_a_sheared_bond_only_above_tau_c():
    """Both particles kinematic and at rest, turned together by phi about z after the bond was made: tau =
    G s^2 phi / l0^2; the bond breaks at the end of the step exactly when tau_c is below that value."""
    phi = 0.02
    tau = G * S_SCALE ** 2 * phi / L0 ** 2
    for tau_c, expect in ((0.9 * tau, 1), (1.1 * tau, 0)):
        o = oracle.OracleSim(pair(tau_c=tau_c, kinematic=(1, 1)))
        o.set_state(o.p.copy(), np.stack([q_of([0, 0, 1], phi)] * 2), np.zeros((2, 3)), np.zeros((2, 4)))
        o.step(1)
        assert int(o.broken[0]) == expect
