"""Pins of the oracle's bond model (Sec. 3.2) and its manifold derivatives (Sec. 4.1-4.2).

Closed forms are worked out from the paper's formulas for configurations where only one deformation
mode is present; derivatives are checked against central finite differences of the pullback
phi(xi) = V(R_x(xi)) through the exponential-map retraction (a second-order retraction, so the
pullback Hessian at 0 equals the Riemannian Hessian); invariances follow from the energy's form.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_10459_gb300 import scenes

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

L0, R, E, NU = 0.01, 0.005, 1e7, 0.3


def pair_scene(direction=(1.0, 0.0, 0.0), q_init=None, bts=1.0, shs=1.0):
    d = np.asarray(direction, float)
    d = d / np.linalg.norm(d)
    pos = np.stack([np.zeros(3), L0 * d])
    sc = scenes._assemble(pos, np.full(2, R), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.array([[0, 1]]),
                          [scenes.Material(E, NU, 2500.0, math.inf, bts, shs)], scenes.default_config(), "pair")
    if q_init is not None:
        sc.quat[:] = q_init
    return sc


def stiffness():
    r0 = R
    S, I, J = math.pi * r0 ** 2, math.pi * r0 ** 4 / 4, math.pi * r0 ** 4 / 2
    G = E / (2 * (1 + NU))
    return dict(kn=E * S / L0, kt=G * S / L0, kb=E * I / L0, ktw=G * J / L0)


def qrot(axis, ang):
    return Rotation.from_rotvec(np.asarray(axis, float) * ang).as_quat()


def test_rest_data():
    """l0, d0 = conj(q_c) (.) n0 and R0 d0 = e_x with R0 a rotation (readings of Sec. 3.2)."""
    rng = np.random.default_rng(0)
    for k in range(6):
        d = rng.normal(size=3)
        qc = qrot(rng.normal(size=3), 0.7) if k % 2 else np.array([0, 0, 0, 1.0])
        o = oracle.OracleSim(pair_scene(d, q_init=qc))
        n0 = d / np.linalg.norm(d)
        assert abs(o.l0[0] - L0) < 1e-16
        assert np.allclose(o.d0[0], Rotation.from_quat(qc).inv().apply(n0), atol=1e-15)
        R0 = o.R0[0].reshape(3, 3)
        assert np.allclose(R0 @ R0.T, np.eye(3), atol=1e-14) and abs(np.linalg.det(R0) - 1) < 1e-14
        assert np.allclose(R0 @ o.d0[0], [1, 0, 0], atol=1e-14)
    o = oracle.OracleSim(pair_scene((-1.0, 0.0, 0.0)))  # antiparallel: 180 degrees about e_z
    assert np.allclose(o.R0[0].reshape(3, 3) @ o.d0[0], [1, 0, 0], atol=1e-14)
    s = stiffness()
    assert np.isclose(o.kn[0], s["kn"]) and np.isclose(o.kt[0], s["kt"])
    assert np.allclose(o.kbt[0], [s["ktw"], s["kb"], s["kb"]])


@pytest.mark.parametrize("direction", [(1, 0, 0), (0.3, -0.5, 0.8)])
def test_static_energy_closed_forms(direction):
    """Single-mode closed forms (identity rest orientations, bond direction n0):
    stretch by delta -> 1/2 kn delta^2; twist by phi about n0 on one particle -> 1/2 (GJ/l0) sin^2(phi/2);
    opposite bends +-phi about an axis normal to n0 -> 1/2 (EI/l0) sin^2(phi); common rotation by phi about
    a normal axis with positions fixed -> shear 1/2 kt phi^2. Other parts vanish in each case."""
    n0 = np.asarray(direction, float)
    n0 /= np.linalg.norm(n0)
    e_perp = np.cross(n0, [0.0, 0.0, 1.0] if abs(n0[2]) < 0.9 else [1.0, 0.0, 0.0])
    e_perp /= np.linalg.norm(e_perp)
    o = oracle.OracleSim(pair_scene(n0))
    s = stiffness()
    pi, pj, I4 = np.zeros(3), L0 * n0, np.array([0, 0, 0, 1.0])
    delta = 3e-4
    parts = o.bond_energy_parts(0, pi, I4, pj + delta * n0, I4)
    assert np.allclose(parts, [0.5 * s["kn"] * delta ** 2, 0, 0], rtol=1e-12, atol=1e-20)
    for phi in (0.05, 0.4, 1.2):
        parts = o.bond_energy_parts(0, pi, qrot(n0, phi), pj, I4)
        assert np.allclose(parts, [0, 0, 0.5 * s["ktw"] * math.sin(phi / 2) ** 2], rtol=1e-12, atol=1e-18)
        parts = o.bond_energy_parts(0, pi, qrot(e_perp, phi), pj, qrot(e_perp, -phi))
        assert np.allclose(parts, [0, 0, 0.5 * s["kb"] * math.sin(phi) ** 2], rtol=1e-12, atol=1e-18)
        parts = o.bond_energy_parts(0, pi, qrot(e_perp, phi), pj, qrot(e_perp, phi))
        assert np.allclose(parts, [0, 0.5 * s["kt"] * phi ** 2, 0], rtol=1e-11, atol=1e-18)
    # shear_scale multiplies theta; bend_twist_scale multiplies K
    o2 = oracle.OracleSim(pair_scene(n0, bts=1e-3, shs=L0))
    phi = 0.3
    assert np.isclose(o2.bond_energy_parts(0, pi, qrot(e_perp, phi), pj, qrot(e_perp, phi))[1],
                      0.5 * s["kt"] * (L0 * phi) ** 2, rtol=1e-11)
    assert np.isclose(o2.bond_energy_parts(0, pi, qrot(n0, phi), pj, I4)[2],
                      1e-3 * 0.5 * s["ktw"] * math.sin(phi / 2) ** 2, rtol=1e-12)


def test_double_cover_and_symmetry():
    """The energy is unchanged by q_j -> -q_j (double cover reading of q_c) and by swapping endpoints."""
    rng = np.random.default_rng(1)
    o = oracle.OracleSim(pair_scene((0.2, 0.9, -0.3)))
    for _ in range(5):
        pi, pj = rng.normal(size=3) * 1e-3, L0 * np.array([0.2, 0.9, -0.3]) / np.linalg.norm([0.2, 0.9, -0.3])
        pj = pj + rng.normal(size=3) * 1e-4
        qi, qj = qrot(rng.normal(size=3), 0.2), qrot(rng.normal(size=3), 0.2)
        e = o.bond_energy_parts(0, pi, qi, pj, qj)
        assert np.allclose(o.bond_energy_parts(0, pi, qi, pj, -qj), e, rtol=1e-12)
        assert np.allclose(o.bond_energy_parts(0, pi, -qi, pj, qj), e, rtol=1e-12)


def rigid(p, q, rot, shift):
    r = Rotation.from_quat(rot)
    return r.apply(p) + shift, (r * Rotation.from_quat(q)).as_quat()


def test_rigid_invariance():
    """Zero energy and reduced gradient for a rigidly moved bond at rest; unchanged energy for a rigidly
    moved deformed bond."""
    rng = np.random.default_rng(2)
    o = oracle.OracleSim(pair_scene((0.4, 0.1, 0.9)))
    s = stiffness()
    n0 = np.array([0.4, 0.1, 0.9]) / np.linalg.norm([0.4, 0.1, 0.9])
    for _ in range(5):
        rot, shift = qrot(rng.normal(size=3), rng.uniform(0.1, 3.0)), rng.normal(size=3)
        pi, qi = rigid(np.zeros(3), np.array([0, 0, 0, 1.0]), rot, shift)
        pj, qj = rigid(L0 * n0, np.array([0, 0, 0, 1.0]), rot, shift)
        e, g, H, Hs = o.bond_terms(0, pi, qi, pj, qj)
        # scale: the stiffest mode's force per unit angle (the shear term, kt per radian, kt/l0 per metre);
        # the shifted positions carry rounding of eps |shift| relative to l0
        rel = 1e-13 * max(1.0, np.linalg.norm(shift) / L0)
        assert abs(e) < rel ** 2 * s["kt"]
        assert np.abs(g[[0, 1, 2, 6, 7, 8]]).max() < rel * s["kt"] / L0
        assert np.abs(g[[3, 4, 5, 9, 10, 11]]).max() < rel * s["kt"]
        # a deformed bond moved rigidly keeps its energy
        dpi, dqi = rng.normal(size=3) * 1e-4, qrot(rng.normal(size=3), 0.1)
        dpj, dqj = L0 * n0 + rng.normal(size=3) * 1e-4, qrot(rng.normal(size=3), 0.1)
        e0 = o.bond_energy_parts(0, dpi, dqi, dpj, dqj).sum()
        a, b = rigid(dpi, dqi, rot, shift), rigid(dpj, dqj, rot, shift)
        assert np.isclose(o.bond_energy_parts(0, a[0], a[1], b[0], b[1]).sum(), e0, rtol=1e-9)


def pullback(o, x, xi):
    pi, qi = oracle.retract(x[0], x[1], xi[:6])
    pj, qj = oracle.retract(x[2], x[3], xi[6:])
    return o.bond_energy_parts(0, pi, qi, pj, qj).sum()


def deformed_states(seed, n):
    rng = np.random.default_rng(seed)
    n0 = np.array([0.3, -0.2, 0.93])
    n0 /= np.linalg.norm(n0)
    out = []
    for k in range(n):
        pi = rng.normal(size=3) * 1e-3
        pj = pi + L0 * n0 * (1 + rng.uniform(-0.05, 0.05)) + rng.normal(size=3) * 5e-4
        qi, qj = qrot(rng.normal(size=3), rng.uniform(0.0, 0.5)), qrot(rng.normal(size=3), rng.uniform(0.0, 0.5))
        out.append((pi, qi, pj, qj))
    return n0, out


@pytest.mark.parametrize("shs", [1.0, L0])
def test_gradient_and_hessian_against_pullback_differences(shs):
    """Reduced gradient = d phi/d xi (0); reduced Riemannian Hessian (Eq. manifold-hessian-1..4 and the
    nullspace reduction) = d^2 phi/d xi^2 (0), by central differences in scaled coordinates."""
    n0, states = deformed_states(3, 4)
    o = oracle.OracleSim(pair_scene(n0, shs=shs))
    hs = np.array([1e-6] * 3 + [1e-4] * 3 + [1e-6] * 3 + [1e-4] * 3)
    for x in states:
        e, g, H, Hs = o.bond_terms(0, *x)
        assert np.isclose(e, pullback(o, x, np.zeros(12)), rtol=1e-13)
        # 4th-order central differences for the gradient
        gfd = np.zeros(12)
        for a in range(12):
            ea = np.zeros(12)
            ea[a] = hs[a]
            gfd[a] = (-pullback(o, x, 2 * ea) + 8 * pullback(o, x, ea) - 8 * pullback(o, x, -ea)
                      + pullback(o, x, -2 * ea)) / (12 * hs[a])
        sc = np.abs(g) + np.abs(gfd).max() * 1e-7
        assert np.all(np.abs(g - gfd) <= 1e-5 * sc + 1e-9 * np.abs(g).max()), (g, gfd)
        Hfd = np.zeros((12, 12))
        for a in range(12):
            for b in range(a, 12):
                ea, eb = np.zeros(12), np.zeros(12)
                ea[a], eb[b] = hs[a], hs[b]
                v = (pullback(o, x, ea + eb) - pullback(o, x, ea - eb) - pullback(o, x, -ea + eb)
                     + pullback(o, x, -ea - eb)) / (4 * hs[a] * hs[b])
                Hfd[a, b] = Hfd[b, a] = v
        d = np.sqrt(np.abs(np.outer(np.diag(H), np.diag(H)))) + 1e-12 * np.abs(H).max()
        assert np.all(np.abs(H - Hfd) <= 2e-5 * d + 1e-7 * np.abs(H).max()), np.abs(H - Hfd).max()
        # symmetric; translation null space; projection = eigen-clamp of the unprojected Hessian
        assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
        T = np.zeros(12)
        T[[0, 6]] = 1.0
        assert np.abs(H @ T).max() < 1e-9 * np.abs(H).max()
        lam, V = np.linalg.eigh(H)
        assert np.allclose(Hs, V @ np.diag(np.maximum(lam, 0)) @ V.T, atol=1e-11 * np.abs(H).max())


def test_shear_angle_small_and_exact_limits():
    """At the rest configuration the shear term has zero gradient; its Hessian is finite (series branch)."""
    o = oracle.OracleSim(pair_scene((1, 0, 0)))
    e, g, H, Hs = o.bond_terms(0, np.zeros(3), np.array([0, 0, 0, 1.0]), np.array([L0, 0, 0]), np.array([0, 0, 0, 1.0]))
    assert abs(e) == 0.0 and np.abs(g).max() == 0.0
    assert np.all(np.isfinite(H)) and np.linalg.eigvalsh(H).min() > -1e-9 * np.abs(H).max()
    s = stiffness()
    # transverse stiffness of the shear term at rest: d^2/dz^2 of 1/2 kt theta^2 with theta ~ z/l0
    assert np.isclose(H[8, 8], s["kt"] / L0 ** 2, rtol=1e-9)
    assert np.isclose(H[6, 6], s["kn"], rtol=1e-10)
