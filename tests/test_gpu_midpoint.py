"""The variational midpoint integrator (Sec. 3.1; App. C) of the CUDA path against the oracle (needs a GB300).

- zhat = xhat - 1/2 M_s^{-1} dt^2 grad V((x_{n-1} + x_n)/2) of a moving, rotating, deformed lattice in contact with
  the ground and itself: FP64 on both paths, to rounding.
- The Newton system of Phi(x) = 1/(2 dt^2) (x - zhat)^T M_s (x - zhat) + V((x + x_n)/2) at an iterate x away from the
  start state x_n: reduced gradient, assembled diagonal blocks and per-bond 12x12 projected Hessians, with the
  tolerances of the implicit-Euler-like system's parity test.
- Trajectories: the spring pair (the trapezoidal recurrence), a cube bouncing off the ground and three Poisson-disk
  boxes landing with fracture; mixed to 1e-4 of the scene diagonal, identical break sets; FP64 to 1e-9 of the spring
  pair's size, and for the contact cases to twice the distance the oracle's own trajectory moves when its Newton
  tolerance is tightened 100x (tests/golden/newton_spread.json, "cube_mid" and "c4_mid": the stiff one-sided contact
  makes these trajectories sensitive to where each Newton solve stops); the step graph and the host-driven loop
  bit-identical.
The stiff plate and textile configurations are not run with this form: at their time steps (hundreds of contact
and bond periods) its Newton iteration stalls in the line search on the oracle too.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu
Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

PRECS = [(pkg.BDEM_FP64, "fp64"), (pkg.BDEM_MIXED, "mixed")]
TOL = {pkg.BDEM_FP64: 1e-9, pkg.BDEM_MIXED: 1e-4}
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "newton_spread.json")) as _f:
    SPREAD = json.load(_f)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()
    oracle.build()


def contact_lattice():
    return scenes.cube_lattice(nx=3, spacing=0.0098, r=0.005, k_ground=1e6, z_bottom=0.0045, k_self=1e5,
                               contact_skin=0.005, integrator=1)


def moving_state(sc, seed):
    rng = np.random.default_rng(seed)
    p = sc.pos + rng.normal(size=sc.pos.shape) * 3e-4
    q = Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * 0.15).as_quat()
    v = rng.normal(size=sc.pos.shape) * 0.1
    w = rng.normal(size=(sc.n, 3)) * 2.0
    u = 0.5 * np.stack([oracle.qmul(np.r_[w[i], 0.0], q[i]) for i in range(sc.n)])  # q' = 1/2 (w, 0) q
    return p, q, v, u


@pytest.mark.parametrize("prec,name", PRECS)
def test_zhat_matches_the_oracle(prec, name):
    sc = contact_lattice()
    p, q, v, u = moving_state(sc, 1)
    o = oracle.OracleSim(sc)
    o.set_state(p, q, v, u)
    ph, qh, _, _ = o.predict()
    zp_r, zq_r = o.zhat(ph, qh)
    sim = pkg.Sim(sc, precision=prec)
    sim.write_state(p, q, v, u)
    zp, zq = sim.bdem_debug_zhat()
    sim.close()
    sp, sq = np.abs(zp_r - ph).max(), np.abs(zq_r - qh).max()
    assert sp > 0 and sq > 0
    assert np.abs(zp - zp_r).max() <= 1e-10 * sp + 1e-15
    assert np.abs(zq - zq_r).max() <= 1e-10 * sq + 1e-15


@pytest.mark.parametrize("prec,name", PRECS)
def test_midpoint_newton_system_matches_the_oracle(prec, name):
    sc = contact_lattice()
    pn, qn, v, u = moving_state(sc, 2)
    rng = np.random.default_rng(3)
    p = pn + rng.normal(size=pn.shape) * 2e-4
    q = (Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * 0.1) * Rotation.from_quat(qn)).as_quat()
    phat = pn + rng.normal(size=pn.shape) * 1e-4
    qhat = q + rng.normal(size=q.shape) * 0.01
    o = oracle.OracleSim(sc)
    o.set_state(pn, qn, v, u)
    ref = o.system(p, q, phat, qhat)
    sim = pkg.Sim(sc, precision=prec)
    sim.write_state(pn, qn, v, u)
    got = sim.bdem_debug_system(phat, qhat, pos=p, quat=q)
    assert got["n_candidates"] == ref["n_candidates"]
    assert np.abs(got["g"] - ref["g"]).max() <= 1e-10 * np.abs(ref["g"]).max()
    htol, ftol = (1e-10, 1e-13) if prec == pkg.BDEM_FP64 else (2e-5, 1e-6)
    for i in range(sc.n):
        Dr, Dg = ref["diag"][i], got["diag"][i]
        s_ = np.sqrt(np.abs(np.outer(np.diag(Dr), np.diag(Dr))))
        assert np.all(np.abs(Dg - Dr) <= htol * s_ + ftol * np.abs(Dr).max()), (i, np.abs(Dg - Dr).max())
    for k, b in enumerate(ref["bond_ids"]):
        Hr, Hg = ref["bondH"][k], got["bondH"][b]
        s_ = np.sqrt(np.abs(np.outer(np.diag(Hr), np.diag(Hr))))
        assert np.all(np.abs(Hg - Hr) <= htol * s_ + ftol * np.abs(Hr).max()), (b, np.abs(Hg - Hr).max())
    sim.close()


def compare_run(sc, prec, steps, spread_key):
    o = oracle.OracleSim(sc)
    sim = pkg.Sim(sc, precision=prec)
    L = float(np.linalg.norm(sc.pos.max(0) - sc.pos.min(0)))
    sp = SPREAD[spread_key]
    ptol = max(TOL[prec], 2.0 * sp["pos"])
    qtol = max(TOL[prec], 2.0 * sp["quat"])
    for k in range(steps):
        o.step(1)
        sim.step(1)
        st = sim.read_state()
        assert np.abs(st["pos"] - o.p).max() <= ptol * L, (k, np.abs(st["pos"] - o.p).max() / L)
        qe = np.minimum(np.abs(st["quat"] - o.q).max(1), np.abs(st["quat"] + o.q).max(1)).max()
        assert qe <= qtol, (k, qe)
        assert np.array_equal(st["broken"], o.broken), k
    sim.close()


@pytest.mark.parametrize("prec,name", PRECS)
def test_spring_pair_trajectory(prec, name):
    pos = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0]])
    cfg = scenes.default_config(dt=2e-4, gravity=(0.0, 0.0, 0.0), newton_rel_tol=1e-12, integrator=1)
    sc = scenes._assemble(pos, np.full(2, 0.005), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.array([[0, 1]]),
                          [scenes.Material(1e7, 0.3, 2500.0)], cfg, "axial")
    o = oracle.OracleSim(sc)
    p = o.p.copy()
    p[1, 0] += 1e-5  # released stretched by 1e-5 m
    o.set_state(p, o.q.copy(), np.zeros((2, 3)), np.zeros((2, 4)))
    sim = pkg.Sim(sc, precision=prec)
    sim.write_state(p, o.q.copy(), np.zeros((2, 3)), np.zeros((2, 4)))
    for k in range(40):
        o.step(1)
        sim.step(1)
        got = sim.read_state()["pos"]
        # the extension, relative to the scene size 0.01 m
        assert abs((got[1, 0] - got[0, 0]) - (o.p[1, 0] - o.p[0, 0])) <= TOL[prec] * 0.01, k
    sim.close()


@pytest.mark.parametrize("prec,name", PRECS)
def test_cube_bounce_trajectory(prec, name):
    """A 4x4x4 cube released 5 mm above the ground: it lands at about step 32 and leaves again."""
    sc = scenes.cube_lattice(nx=4, z_bottom=0.01, k_ground=1e6, steps=50, integrator=1)
    compare_run(sc, prec, 50, "cube_mid")


def boxes():
    sc = scenes.c4_batched(n_scenes=3, n_min=150, n_max=400, heights=(0.0002, 0.001))
    sc.config = dict(sc.config, integrator=1)
    return sc


@pytest.mark.parametrize("prec,name", PRECS)
def test_boxes_landing_with_fracture(prec, name):
    compare_run(boxes(), prec, 25, "c4_mid")


def test_graph_and_host_loop_are_identical():
    sc = boxes()
    out = []
    for graph in (True, False):
        sim = pkg.Sim(sc, precision=pkg.BDEM_MIXED)
        sim.set_step_graph(graph)
        sim.step(4)
        out.append(sim.read_state())
        if graph:  # every step after the first (host-driven, under phase timing) goes through the graph
            assert sim.graph_steps() == 3, sim.graph_error()
        sim.close()
    for k in ("pos", "quat", "vel", "quat_vel", "broken"):
        assert np.array_equal(out[0][k], out[1][k]), k
