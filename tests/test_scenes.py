"""The synthetic input generators (host logic, no GPU): each construction has the sizes, structure and settings its
recipe states (the cube, the full-size plate, the full-size textile; the batched boxes and the slab impact at reduced
counts of the same generators)."""
import math

import numpy as np
import pytest

from paper_2308_10459_gb300 import scenes

cKDTree = pytest.importorskip("scipy.spatial").cKDTree


def bond_lengths(sc):
    return np.linalg.norm(sc.pos[sc.bond_j] - sc.pos[sc.bond_i], axis=1)


def degrees(sc):
    return np.bincount(np.concatenate([sc.bond_i, sc.bond_j]), minlength=sc.n)


def test_cube():
    sc = scenes.c1_cube()
    assert (sc.n, sc.nb, sc.n_scenes) == (1000, 2700, 1)
    assert np.allclose(bond_lengths(sc), 0.01, rtol=0, atol=1e-15)
    assert sc.pos[:, 2].min() == pytest.approx(0.2)
    assert np.all(sc.quat == np.array([0.0, 0.0, 0.0, 1.0]))
    assert sc.config["dt"] == 1e-3 and sc.config["k_ground"] == 1e6
    assert np.all(sc.radius == 0.005)
    assert np.all((sc.bond_i < sc.bond_j))


def test_full_size_plate():
    sc = scenes.c2_plate()
    assert (sc.n, sc.nb) == (219314, 1092558)
    r = 1e-3
    L = bond_lengths(sc)
    # bonds to neighbours within 1.05 * 2r on the unjittered lattice, then +-1e-5 m jitter per coordinate
    assert L.max() <= 2 * r + 2 * math.sqrt(3) * 1e-5 + 1e-12 and L.min() >= 2 * r - 2 * math.sqrt(3) * 1e-5 - 1e-12
    deg = degrees(sc)
    assert deg.max() == 12 and np.count_nonzero(deg == 12) > sc.n // 4  # interior particles of an HCP stack
    assert np.allclose(sc.vel, [0.0, 0.0, -3.0])
    # tilted 10 degrees about x, lowest sphere surface 1 mm above the ground plane
    assert (sc.pos[:, 2] - sc.radius).min() == pytest.approx(1e-3, abs=1e-9)
    assert sc.pos[:, 1].max() - sc.pos[:, 1].min() > 0.5  # R = 0.284 m
    m = sc.materials[0]
    assert (m.E, m.nu, m.density, m.break_strain) == (5e9, 0.3, 2500.0, 1e-3)
    assert sc.config["dt"] == 5e-4 and sc.config["k_ground"] == sc.config["k_self"] == pytest.approx(5e9 * r)
    assert sc.config["newton_rel_tol"] == 1e-6


def test_full_size_textile():
    sc = scenes.c3_textile()
    assert (sc.n, sc.nb) == (90000, 358202)
    L = bond_lengths(sc)
    assert np.all(np.isclose(L, 2e-3) | np.isclose(L, 2e-3 * math.sqrt(2)))
    kin = sc.kinematic.astype(bool)
    x = sc.pos[:, 0]
    assert np.array_equal(kin, np.isclose(x, x.min()) | np.isclose(x, x.max()))
    assert np.allclose(sc.vel[kin & np.isclose(x, x.min()), 0], -0.5)
    assert np.allclose(sc.vel[kin & np.isclose(x, x.max()), 0], 0.5)
    m = sc.materials[0]
    assert (m.E, m.density, m.break_strain, m.bend_twist_scale) == (1e9, 1500.0, 0.3, 1e-3)


def test_batched_boxes_at_reduced_counts():
    sc = scenes.c4_batched(n_scenes=6, n_min=200, n_max=900)
    r = 2e-3
    counts = np.diff(sc.scene_offsets)
    assert sc.n_scenes == 6 and np.all((counts >= 200) & (counts <= 900))
    for s in range(6):
        a, b = int(sc.scene_offsets[s]), int(sc.scene_offsets[s + 1])
        tree = cKDTree(sc.pos[a:b])
        assert not tree.query_pairs(2 * r * (1 - 1e-12))  # Poisson disk: no two spheres overlap
        sel = (sc.bond_i >= a) & (sc.bond_i < b)
        assert np.all((sc.bond_j[sel] >= a) & (sc.bond_j[sel] < b))  # bonds stay inside their scene
    assert bond_lengths(sc).max() < 1.1 * 2 * r
    assert sc.config["dt"] == 1e-3 and sc.materials[0].E == 1e8 and sc.materials[0].break_strain == 2e-3


def test_slab_impact_at_reduced_counts():
    sc = scenes.c5_impact(n_slab=4000, n_ball=300, footprint=0.06, ball_R=0.02)
    r = 2e-3
    ball = sc.material == 1
    # dart throwing stops when its rounds run out: the counts reach most of their targets, never more
    nb_, ns_ = np.count_nonzero(ball), np.count_nonzero(~ball)
    assert 150 <= nb_ <= 300 and 3800 <= ns_ <= 4000, (nb_, ns_)
    assert np.allclose(sc.vel[ball], [0.0, 0.0, -20.0]) and np.allclose(sc.vel[~ball], 0.0)
    assert sc.pos[ball, 2].min() > sc.pos[~ball, 2].max()  # the ball starts above the slab
    assert not cKDTree(sc.pos).query_pairs(2 * r * (1 - 1e-12))
    # the slab's bond cutoff is bisected for a mean of 12 neighbours (interior of a small slab: boundary lowers it)
    slab_bonds = (sc.bond_material == 0)
    deg = np.bincount(np.concatenate([sc.bond_i[slab_bonds], sc.bond_j[slab_bonds]]), minlength=sc.n)[~ball]
    assert 8.0 < deg.mean() <= 12.5
    assert sc.materials[1].E == 10 * sc.materials[0].E and math.isinf(sc.materials[1].break_strain)
    assert sc.config["dt"] == 2e-4
