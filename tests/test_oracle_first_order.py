"""Pins of the oracle's first-order manifold optimisation (Alg. 1) against closed forms and the second-order method.

Alg. 1 steps along -grad f with the same line search and stopping test as Alg. 2. A free particle falls to the
closed-form minimiser p = phat + g dt^2 with either method. On a bonded lattice the second-order method needs the
same few iterations at every stiffness while the first-order method slows down as the bonds stiffen (the shape of
the paper's convergence comparison of the two methods).
"""
import numpy as np
import pytest

import oracle
from paper_2308_10459_gb300 import scenes


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def test_free_particle_reaches_the_closed_form_minimiser():
    dt, g = 1e-3, np.array([0.0, 0.0, -9.81])
    for opt in (0, 1):
        cfg = scenes.default_config(dt=dt, optimizer=opt, newton_rel_tol=1e-12)
        sc = scenes._assemble(np.array([[0.1, -0.2, 0.5]]), np.full(1, 0.005), np.zeros(1, np.int32),
                              np.zeros(1, np.uint8), np.zeros((0, 2), np.int64), [scenes.Material(1e7, 0.3, 2500.0)],
                              cfg, "free", vel=np.array([[0.3, 0.0, -1.0]]))
        o = oracle.OracleSim(sc)
        st = o.step(1)[0][0]
        assert st["status"] == 0
        phat = np.array([0.1, -0.2, 0.5]) + dt * np.array([0.3, 0.0, -1.0])
        assert np.allclose(o.p[0], phat + g * dt * dt, rtol=0, atol=1e-15)
        assert st["pcg_iters"] == 0 if opt == 1 else st["pcg_iters"] > 0


def test_first_order_slows_with_stiffness_second_order_does_not():
    iters = {}
    for E in (1e5, 1e6, 1e7):
        for opt in (0, 1):
            sc = scenes.cube_lattice(nx=3, E=E, k_ground=0.0, optimizer=opt, newton_max_iter=300)
            st = oracle.OracleSim(sc).step(1)[0][0]
            iters[E, opt] = (st["newton_iters"], st["status"])
    assert len({iters[E, 0] for E in (1e5, 1e6, 1e7)}) == 1 and iters[1e5, 0][0] <= 6
    assert iters[1e5, 1][0] > 2 * iters[1e5, 0][0]
    assert iters[1e6, 1][0] > 4 * iters[1e5, 1][0]
    assert iters[1e7, 1] == (300, 4)  # the iteration cap
