"""CUDA path vs the CPU oracle, element by element, through the C ABI (needs a GB300)."""
import math

import numpy as np
import pytest

import oracle
import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu
Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

PRECS = [(pkg.BDEM_FP64, "fp64"), (pkg.BDEM_MIXED, "mixed")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()


def deformed_state(sc, seed, dp=3e-4, ang=0.2, dv=0.1):
    rng = np.random.default_rng(seed)
    p = sc.pos + rng.normal(size=sc.pos.shape) * dp
    q = Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * ang).as_quat()
    v = rng.normal(size=sc.pos.shape) * dv
    u = rng.normal(size=(sc.n, 4)) * dv
    return p, q, v, u


def small_contact_scene():
    return scenes.cube_lattice(nx=3, spacing=0.0098, r=0.005, k_ground=1e6, z_bottom=0.0045, k_self=1e5,
                               contact_skin=0.005)


def scaled_close(a, b, scale, tol):
    return np.abs(a - b).max() <= tol * scale


@pytest.mark.parametrize("prec,name", PRECS)
def test_newton_system_parity(prec, name):
    """Reduced gradient (FP64 on both paths), assembled diagonal blocks and per-bond 12x12 projected Hessians."""
    sc = small_contact_scene()
    p, q, v, u = deformed_state(sc, 1)
    phat = sc.pos + np.random.default_rng(2).normal(size=sc.pos.shape) * 1e-4
    qhat = q + np.random.default_rng(3).normal(size=q.shape) * 0.01
    ref = oracle.OracleSim(sc).system(p, q, phat, qhat)
    sim = pkg.Sim(sc, precision=prec)
    sim.write_state(p, q, v, u)
    got = sim.bdem_debug_system(phat, qhat)
    assert got["n_candidates"] == ref["n_candidates"]
    gs = np.abs(ref["g"]).max()
    assert np.abs(got["g"] - ref["g"]).max() <= 1e-10 * gs
    # FP64: both sides to rounding; FP32 Hessians: entry error bounded by 2e-5 of sqrt(H_aa H_bb) plus 1e-6 of
    # the block's largest entry (FP32 eigen-clamp of a graded matrix)
    htol, ftol = (1e-10, 1e-13) if prec == pkg.BDEM_FP64 else (2e-5, 1e-6)
    for i in range(sc.n):
        Dr, Dg = ref["diag"][i], got["diag"][i]
        sc_ = np.sqrt(np.abs(np.outer(np.diag(Dr), np.diag(Dr))))
        assert np.all(np.abs(Dg - Dr) <= htol * sc_ + ftol * np.abs(Dr).max()), (i, np.abs(Dg - Dr).max())
    order = sim.bond_order()
    assert np.array_equal(order, np.stack([sc.bond_i, sc.bond_j], 1))
    for k, b in enumerate(ref["bond_ids"]):
        Hr, Hg = ref["bondH"][k], got["bondH"][b]
        sc_ = np.sqrt(np.abs(np.outer(np.diag(Hr), np.diag(Hr))))
        assert np.all(np.abs(Hg - Hr) <= htol * sc_ + ftol * np.abs(Hr).max()), (b, np.abs(Hg - Hr).max())
    sim.close()


@pytest.mark.parametrize("prec,name", PRECS)
def test_matvec_and_pcg_parity(prec, name):
    sc = small_contact_scene()
    p, q, v, u = deformed_state(sc, 4)
    phat, qhat = p + 1e-4, q + 0.01
    o = oracle.OracleSim(sc)
    sim = pkg.Sim(sc, precision=prec)
    sim.write_state(p, q, v, u)
    sim.bdem_debug_system(phat, qhat, want_bonds=False)
    x = np.random.default_rng(5).normal(size=(sc.n, 6))
    yr = o.matvec(p, q, phat, qhat, x)
    yg = sim.bdem_debug_matvec(x)
    tol = 1e-11 if prec == pkg.BDEM_FP64 else 1e-5
    assert np.abs(yg - yr).max() <= tol * np.abs(yr).max()
    b = np.random.default_rng(6).normal(size=(sc.n, 6))
    eps = 1e-12 if prec == pkg.BDEM_FP64 else 1e-6
    xr, itr = o.pcg_solve(p, q, phat, qhat, b, eps, 2000)
    xg, itg = sim.bdem_debug_pcg(b, eps, 2000)
    # mixed: the refined solve meets eps on the true residual of the stored FP32 system (FP64 product), so it differs
    # from the FP64 solution only by the FP32 rounding of the blocks, amplified by the system's conditioning
    tol = 1e-8 if prec == pkg.BDEM_FP64 else 1e-4
    assert np.abs(xg - xr).max() <= tol * np.abs(xr).max(), np.abs(xg - xr).max() / np.abs(xr).max()
    if prec == pkg.BDEM_FP64:
        assert abs(int(itg[0]) - itr) <= 2
    else:
        r = b - sim.bdem_debug_matvec(xg)
        assert np.linalg.norm(r) <= eps * np.linalg.norm(b) * (1.0 + 1e-3), np.linalg.norm(r) / np.linalg.norm(b)
    sim.close()


def bbox_diag(sc):
    return float(np.linalg.norm(sc.pos.max(0) - sc.pos.min(0)))


def quat_err(a, b):
    return np.minimum(np.abs(a - b).max(1), np.abs(a + b).max(1)).max()


def run_pair(sc, prec, steps, check_every=10, pos_tol=1e-9, quat_tol=1e-9):
    o = oracle.OracleSim(sc)
    sim = pkg.Sim(sc, precision=prec)
    L = bbox_diag(sc)
    worst = 0.0
    for k in range(steps):
        so = o.step(1)[0]
        sg = sim.step(1)
        if (k + 1) % check_every == 0 or k == steps - 1:
            st = sim.read_state()
            e = np.abs(st["pos"] - o.p).max() / L
            worst = max(worst, e)
            assert e <= pos_tol, (k, e)
            assert quat_err(st["quat"], o.q) <= quat_tol, k
            assert np.array_equal(st["broken"], o.broken), k
    sim.close()
    return worst


@pytest.mark.parametrize("prec,name", PRECS)
def test_trajectory_cube_ground_contact(prec, name):
    """4x4x4 cube released 1 mm above the ground with random velocities and spins, 100 steps."""
    sc = scenes.cube_lattice(nx=4, z_bottom=0.006, k_ground=1e6)
    rng = np.random.default_rng(7)
    sc.vel[:] = rng.normal(size=sc.vel.shape) * 0.05 + np.array([0.0, 0.0, -0.3])
    tol = 1e-9 if prec == pkg.BDEM_FP64 else 1e-4
    run_pair(sc, prec, 100, pos_tol=tol, quat_tol=tol)
