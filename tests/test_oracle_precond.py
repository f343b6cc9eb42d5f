"""Pins of the oracle's block-Jacobi preconditioner (Sec. 5.3): z = D_i^-1 r_i per 6x6 diagonal block.

The preconditioner is checked against what fixes it independently of the oracle: numpy's dense solve of each block
(random SPD blocks over a wide range of conditioning and the assembled diagonal blocks of a deformed contact lattice),
the stated fallback for a block that is not positive definite, and the textbook property that PCG with an exact
block preconditioner solves a block-diagonal system in exactly one iteration (a wrong triangular solve takes more
and misses the dense solution).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2308_10459_gb300 import scenes
from test_oracle_step import deformed_small_system


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def random_spd(rng, cond):
    Q, _ = np.linalg.qr(rng.normal(size=(6, 6)))
    ev = np.geomspace(1.0, cond, 6)
    rng.shuffle(ev)
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("cond", [1.0, 1e3, 1e8])
def test_block_solve_matches_dense_solve(cond):
    rng = np.random.default_rng(int(np.log10(cond)) + 11)
    for _ in range(20):
        D = random_spd(rng, cond) * rng.uniform(1e-3, 1e6)
        r = rng.normal(size=6)
        z, ok = oracle.precond_apply(D, r)
        ref = np.linalg.solve(D, r)
        assert ok == 1
        # backward-stable Cholesky: error bounded by cond(D) times the rounding unit
        assert np.linalg.norm(z - ref) <= 50 * cond * 2.2e-16 * np.linalg.norm(ref)
        # and the residual of the solve is at rounding level of |D| |z|
        assert np.linalg.norm(D @ z - r) <= 1e-13 * np.linalg.norm(D, 2) * np.linalg.norm(z)


def test_assembled_blocks_of_a_contact_lattice():
    """The diagonal blocks the PCG preconditions with (inertia + bonds + ground + self contact, deformed state)."""
    o, p, q, phat, qhat = deformed_small_system()
    sysd = o.system(p, q, phat, qhat)
    rng = np.random.default_rng(5)
    dense_blocks = 0
    for D in sysd["diag"]:
        off = np.abs(D - np.diag(np.diag(D))).max()
        dense_blocks += off > 1e-6 * np.abs(D).max()
        r = rng.normal(size=6)
        z, ok = oracle.precond_apply(D, r)
        assert ok == 1
        ref = np.linalg.solve(D, r)
        assert np.allclose(z, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert dense_blocks == len(sysd["diag"])  # every block couples translation and rotation


def test_fallback_for_blocks_that_are_not_positive_definite():
    rng = np.random.default_rng(9)
    # symmetric, positive diagonal, indefinite: the Cholesky factorisation breaks down -> r_a / D_aa
    D = np.eye(6) * np.array([2.0, 3.0, 5.0, 7.0, 11.0, 13.0])
    D[0, 1] = D[1, 0] = 10.0
    assert np.linalg.eigvalsh(D).min() < 0
    r = rng.normal(size=6)
    z, ok = oracle.precond_apply(D, r)
    assert ok == 0
    assert np.array_equal(z, r / np.diag(D))
    # a non-positive diagonal entry leaves its component of r unchanged
    D2 = np.diag([4.0, 0.0, -1.0, 2.0, 8.0, 16.0])
    z2, ok2 = oracle.precond_apply(D2, r)
    assert ok2 == 0
    expect = r.copy()
    for a in (0, 3, 4, 5):
        expect[a] = r[a] / D2[a, a]
    assert np.array_equal(z2, expect)


def block_diagonal_system():
    """Free particles each bonded to a kinematic partner, pairs far apart: with the kinematic rows removed the
    Newton system is block diagonal with dense 6x6 blocks (inertia + the bond's own block)."""
    n_pairs = 6
    pos, pairs, kin = [], [], []
    for k in range(n_pairs):
        base = np.array([0.1 * k, 0.0, 0.5])
        pos += [base, base + np.array([0.01, 0.002 * k, 0.0])]
        pairs.append([2 * k, 2 * k + 1])
        kin += [0, 1]
    pos = np.array(pos)
    cfg = scenes.default_config(dt=1e-3, k_ground=0.0, k_self=0.0)
    sc = scenes._assemble(pos, np.full(len(pos), 0.005), np.zeros(len(pos), np.int32), np.array(kin, np.uint8),
                          np.array(pairs), [scenes.Material(1e8, 0.3, 2500.0, shear_scale=0.01)], cfg, "pairs")
    o = oracle.OracleSim(sc)
    rng = np.random.default_rng(2)
    p = pos + rng.normal(size=pos.shape) * 2e-4
    q = Rotation.from_rotvec(rng.normal(size=(len(pos), 3)) * 0.3).as_quat()
    phat = pos + rng.normal(size=pos.shape) * 1e-4
    qhat = q + rng.normal(size=q.shape) * 0.01
    return o, p, q, phat, qhat, np.array(kin, bool)


def test_pcg_on_a_block_diagonal_system_takes_one_iteration():
    o, p, q, phat, qhat, kin = block_diagonal_system()
    sysd = o.system(p, q, phat, qhat)
    b = np.random.default_rng(4).normal(size=(len(p), 6))
    b[kin] = 0.0
    x, it = o.pcg_solve(p, q, phat, qhat, b, 1e-12, 50)
    assert it == 1
    for i in np.flatnonzero(~kin):
        D = sysd["diag"][i]
        assert np.abs(D - np.diag(np.diag(D))).max() > 1e-3 * np.abs(D).max()  # dense block
        ref = np.linalg.solve(D, b[i])
        assert np.allclose(x[i], ref, rtol=1e-10, atol=1e-14 * np.abs(ref).max())
    assert np.abs(x[kin]).max() == 0.0
