"""Pins of the oracle's post-step friction (Sec. 5.4, Friction; Alg. 3) against physics and symmetry.

A sphere resting on the ground at its equilibrium penetration carries |F_n| = m g, so the explicit correction
dv = -min(1, mu_s |F_n| dt / (m |v_t|)) v_t is Coulomb friction: a sliding sphere loses mu_s g dt of speed per step
and stops exactly; a spinning one loses mu_r |F_n| r^3 dt / I = 2.5 mu_r g r dt of angular speed per step. Two equal
spheres in contact sliding past each other slow down mirror-symmetrically and keep zero total momentum.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_10459_gb300 import scenes

R, RHO, K, G, DT = 0.005, 2500.0, 1e5, 9.81, 1e-3
M = RHO * 4.0 / 3.0 * math.pi * R ** 3


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def resting_sphere(vel=(0.0, 0.0, 0.0), mu_s=0.0, mu_r=0.0, kinematic=0):
    z0 = R - M * G / K  # equilibrium penetration: k |g| = m g
    cfg = scenes.default_config(dt=DT, k_ground=K, friction_slide=mu_s, friction_roll=mu_r)
    return scenes._assemble(np.array([[0.0, 0.0, z0]]), np.full(1, R), np.zeros(1, np.int32),
                            np.array([kinematic], np.uint8), np.zeros((0, 2), np.int64),
                            [scenes.Material(1e7, 0.3, RHO)], cfg, "sphere", vel=np.array([vel], float))


def omega(q, u):
    """World angular velocity w from q' = 1/2 (w, 0) q, computed with scipy-free quaternion algebra."""
    x, y, z, w = q
    qc = np.array([-x, -y, -z, w])
    a, b = u, qc
    prod = np.array([a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1],
                     a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0],
                     a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3],
                     a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2]])
    return 2.0 * prod[:3]


def test_sliding_sphere_decelerates_by_mu_g_dt_and_stops():
    mu, v0 = 0.3, 0.05
    o = oracle.OracleSim(resting_sphere(vel=(v0, 0.0, 0.0), mu_s=mu))
    stop = math.ceil(v0 / (mu * G * DT))
    for n in range(1, stop + 4):
        o.step(1)
        assert o.v[0, 0] == pytest.approx(max(v0 - n * mu * G * DT, 0.0), abs=1e-9)
        assert abs(o.v[0, 1]) < 1e-15 and abs(o.v[0, 2]) < 1e-9
    assert abs(o.v[0, 0]) < 1e-15  # at rest, not reversed


def test_spinning_sphere_loses_2p5_mu_r_g_r_dt_per_step():
    mu_r, w0 = 0.2, 3.0
    sc = resting_sphere(mu_r=mu_r)
    sc.quat_vel[0] = 0.5 * np.array([0.0, 0.0, w0, 0.0])  # q' = 1/2 (w, 0) q with q = identity
    sc_free = resting_sphere()
    sc_free.quat_vel[0] = sc.quat_vel[0]
    o, f = oracle.OracleSim(sc), oracle.OracleSim(sc_free)
    o.step(1)
    f.step(1)
    assert np.allclose(o.p, f.p, rtol=0, atol=0) and np.allclose(o.q, f.q, rtol=0, atol=0)
    w_fric, w_free = omega(o.q[0], o.u[0]), omega(f.q[0], f.u[0])
    drop = np.linalg.norm(w_free) - np.linalg.norm(w_fric)
    assert drop == pytest.approx(2.5 * mu_r * G * R * DT, rel=1e-6)
    assert np.allclose(np.cross(w_fric, w_free), 0.0, atol=1e-12)  # same axis


def test_zero_coefficients_change_nothing_and_kinematic_spheres_are_exempt():
    a = oracle.OracleSim(resting_sphere(vel=(0.05, 0.0, 0.0)))
    b = oracle.OracleSim(resting_sphere(vel=(0.05, 0.0, 0.0), mu_s=0.0, mu_r=0.0))
    a.step(3)
    b.step(3)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.u, b.u)
    k = oracle.OracleSim(resting_sphere(vel=(0.05, 0.0, 0.0), mu_s=0.5, kinematic=1))
    k.step(2)
    assert k.v[0, 0] == 0.05


def test_two_spheres_sliding_past_each_other_slow_down_symmetrically():
    u, mu = 0.2, 0.4
    pos = np.array([[0.0, 0.0, 0.0], [2 * R - 2e-5, 0.0, 0.0]])
    cfg = scenes.default_config(dt=DT, gravity=(0.0, 0.0, 0.0), k_self=K, contact_skin=R, friction_slide=mu)
    sc = scenes._assemble(pos, np.full(2, R), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.zeros((0, 2), np.int64),
                          [scenes.Material(1e7, 0.3, RHO)], cfg, "pair", vel=np.array([[0.0, u, 0.0], [0.0, -u, 0.0]]))
    free = scenes._assemble(pos, np.full(2, R), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.zeros((0, 2), np.int64),
                            [scenes.Material(1e7, 0.3, RHO)], dict(cfg, friction_slide=0.0), "pair",
                            vel=np.array([[0.0, u, 0.0], [0.0, -u, 0.0]]))
    o, f = oracle.OracleSim(sc), oracle.OracleSim(free)
    o.step(1)
    f.step(1)
    assert np.allclose(o.v[0], -o.v[1], atol=1e-14)           # mirror symmetry
    assert np.allclose(o.v.sum(0), 0.0, atol=1e-14)           # momentum
    assert abs(o.v[0, 1]) < abs(f.v[0, 1])                    # the tangential motion is slowed
    assert np.linalg.norm(o.v[0]) < np.linalg.norm(f.v[0])
