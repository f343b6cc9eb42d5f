"""The captured step graph (device-driven Newton and line-search loops) against the host-driven loop (needs a GB300).

Both run the same kernels on the same data, so the committed states, velocities and bond flags must be
bit-identical; the graph must actually be used (steps after the first), and a step whose contact candidates
outgrow the arrays must be repeated through the host-driven loop without being committed twice.
"""
import dataclasses

import numpy as np
import pytest

import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()


def run(sc, prec, steps, graph, config=None, pcg_blocks=None):
    sim = pkg.Sim(sc, precision=prec, config=config)
    if pcg_blocks is not None:
        sim.set_pcg_shape(2, pcg_blocks)
    sim.set_step_graph(graph)
    stats = [sim.step(1) for _ in range(steps)]
    st = sim.read_state()
    out = (st, stats, sim.graph_steps(), sim.graph_error())
    sim.close()
    return out


def assert_identical(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def implosion(n_side=6):
    """Unbonded particles (r = 1 mm) on an 8 mm lattice moving towards the centre (v = -(x - c) / 10 ms), self
    contact with a 5 mm skin: no candidates at first, then more than the 16 per particle the arrays start with."""
    sc = scenes.cube_lattice(nx=n_side, spacing=0.008, r=0.001, z_bottom=0.5, k_ground=0.0, k_self=1e4,
                             contact_skin=0.005, name="implosion")
    c = sc.pos.mean(0)
    empty = np.zeros(0, np.int32)
    return dataclasses.replace(sc, vel=-(sc.pos - c) / 0.01, bond_i=empty, bond_j=empty, bond_material=empty)


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED])
def test_graph_matches_host_loop_with_contact(prec):
    """Small plate (R = 15 mm): ground and self contact, several Newton iterations and line-search trials."""
    sc = scenes.c2_plate_small(R=0.015)
    a, sa, ga, ea = run(sc, prec, 4, True)
    b, sb, gb, eb = run(sc, prec, 4, False)
    assert ea == "", ea
    assert ga == 3 and gb == 0  # every step after the first went through the graph
    assert_identical(a, b)
    for x, y in zip(sa, sb):
        assert x[0]["newton_iters"] == y[0]["newton_iters"]
        assert x[0]["pcg_iters"] == y[0]["pcg_iters"]
        assert x[0]["ls_halvings"] == y[0]["ls_halvings"]
        assert x[0]["contact_entry_pcg_iters"] == y[0]["contact_entry_pcg_iters"]


def test_graph_matches_host_loop_with_fracture_and_kinematic_edges():
    sc = scenes.c3_textile(nx=12, steps=8)
    a, sa, ga, ea = run(sc, pkg.BDEM_MIXED, 8, True)
    b, sb, _, _ = run(sc, pkg.BDEM_MIXED, 8, False)
    assert ea == "" and ga == 7
    assert_identical(a, b)
    assert a["broken"].sum() > 50
    assert sum(s[0]["bonds_broken"] for s in sa) == int(a["broken"].sum())
    assert sa[-1][0]["intact_bonds"] == sc.nb - int(a["broken"].sum())


def test_graph_step_repeated_when_contact_candidates_outgrow_the_arrays():
    sc = implosion()
    a, sa, ga, ea = run(sc, pkg.BDEM_FP64, 8, True)
    b, sb, _, _ = run(sc, pkg.BDEM_FP64, 8, False)
    assert ea == ""
    cands = [s[0]["contact_candidates"] for s in sb]
    assert max(cands) > 16 * sc.n  # the arrays had to grow during the run
    assert 0 < ga < 7               # the outgrown steps were repeated through the host-driven loop
    assert_identical(a, b)
    assert [s[0]["contact_candidates"] for s in sa] == cands


def test_batched_uneven_scenes_through_the_graph():
    """Four scenes in one set of launches (a cube near the ground, an empty scene, a jittered cube, five free
    particles), self contact on: per-scene convergence decided inside the graph."""
    a = scenes.cube_lattice(nx=2, z_bottom=0.006, k_ground=1e6, vel=(0.1, 0.0, -0.5))
    b = scenes.cube_lattice(nx=3, z_bottom=0.02, k_ground=1e6, vel=(0.0, 0.2, -1.0), jitter=1e-4, seed=5)
    rng = np.random.default_rng(9)
    free = rng.uniform(0.0, 0.05, (5, 3)) + np.array([0.0, 0.0, 0.01])
    parts = [a.pos, np.zeros((0, 3)), b.pos, free]
    offs = np.cumsum([0] + [len(x) for x in parts])
    pos = np.concatenate(parts, 0)
    pairs = np.concatenate([np.stack([a.bond_i, a.bond_j], 1), np.stack([b.bond_i, b.bond_j], 1) + offs[2]], 0)
    vel = np.concatenate([a.vel, np.zeros((0, 3)), b.vel, rng.normal(size=(5, 3)) * 0.1], 0)
    n = pos.shape[0]
    cfg = scenes.default_config(dt=1e-3, k_ground=1e6, k_self=1e5, contact_skin=0.005)
    mats = [scenes.Material(1e7, 0.3, 2500.0, float("inf"), 1.0, 0.01)]
    sc = scenes._assemble(pos, np.full(n, 0.005), np.zeros(n, np.int32), np.zeros(n, np.uint8), pairs, mats, cfg,
                          "batched", vel=vel, offsets=offs)
    for prec in (pkg.BDEM_FP64, pkg.BDEM_MIXED):
        x, sx, ga, ea = run(sc, prec, 6, True)
        y, sy, _, _ = run(sc, prec, 6, False)
        assert ea == "" and ga == 5
        assert_identical(x, y)
        assert [[t["newton_iters"] for t in st] for st in sx] == [[t["newton_iters"] for t in st] for st in sy]


@pytest.mark.parametrize("blocks", [3, 64])
def test_many_scenes_through_the_graph(blocks):
    """65 scenes (64 Poisson boxes landing, an empty scene): with 64 PCG blocks the rows of the scenes still
    iterating are split evenly over the grid at every PCG iteration and every block takes every scene's decision;
    with 3 blocks a block spans more than 16 scenes and the last block to reach the barrier decides every scene.
    Either way the graph and the host-driven loop commit bit-identical states."""
    from parity_cases import c4_boxes64
    sc = c4_boxes64()
    for prec in (pkg.BDEM_FP64, pkg.BDEM_MIXED):
        x, sx, ga, ea = run(sc, prec, 4, True, pcg_blocks=blocks)
        y, sy, _, _ = run(sc, prec, 4, False, pcg_blocks=blocks)
        assert ea == "" and ga == 3
        assert_identical(x, y)
        assert [[t["newton_iters"] for t in st] for st in sx] == [[t["newton_iters"] for t in st] for st in sy]
        assert [[t["pcg_iters"] for t in st] for st in sx] == [[t["pcg_iters"] for t in st] for st in sy]


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED])
def test_graph_matches_host_loop_with_the_amg_preconditioner(prec):
    """With the AMG preconditioner the step graph holds the AMG-PCG iterations as a device-driven while loop inside
    the Newton loop; the host-driven step launches the same loop as a graph of its own: bit-identical results."""
    sc = scenes.c2_plate_small(R=0.015)
    cfg = dict(preconditioner=pkg.BDEM_PRECOND_AMG)
    a, sa, ga, ea = run(sc, prec, 4, True, cfg)
    b, sb, gb, eb = run(sc, prec, 4, False, cfg)
    assert ea == "", ea
    assert ga == 3 and gb == 0
    assert_identical(a, b)
    for x, y in zip(sa, sb):
        assert x[0]["newton_iters"] == y[0]["newton_iters"] and x[0]["pcg_iters"] == y[0]["pcg_iters"]
