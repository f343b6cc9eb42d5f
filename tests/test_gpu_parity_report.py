"""Error of both GPU paths against the FP64 oracle, per configuration (needs a GB300; run with -s to see the table).

Each configuration runs at a size the oracle finishes in seconds, built by the same generator as the full-size
workload: the 10x10x10 cube in free fall (100 steps) and dropped onto the ground (100 steps), the plate at R = 15 mm,
the 12x12 textile tear, three Poisson-disk boxes landing on their grounds, and a small slab hit by a ball. The
largest position error (relative to the scene's bounding-box diagonal), quaternion error and the bond-break sets are
compared step by step; the mixed path is held to 1e-4 and the break sets must be identical. The FP64 path is held to
1e-9 where the method pins the answer down that far, and otherwise to how far the oracle's own trajectory moves
when its Newton tolerance is tightened: for the slab impact and the landing boxes that spread is recorded in
tests/golden/newton_spread.json (written by the oracle-only script beside it); for the textile, whose tighter-
tolerance trajectories tear differently, positions are held to 1e-8 and orientations to 1e-7 (the oracle's spread
between tolerances 1e-9 and 1e-12 before the tear is 2.6e-9 and 5.2e-8).
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()
    oracle.build()


def qerr(a, b):
    return float(np.minimum(np.abs(a - b).max(1), np.abs(a + b).max(1)).max()) if len(a) else 0.0


with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "newton_spread.json")) as _f:
    SPREAD = json.load(_f)

# name: (scene, steps, config, FP64 position bound, FP64 quaternion bound)
CASES = {
    "c1 cube 10^3, free fall": (lambda: scenes.c1_cube(), 100, None, 1e-9, 1e-9),
    "c1b cube 10^3 on the ground": (lambda: scenes.c1b_cube_contact(steps=100), 100, None, 1e-9, 1e-9),
    "c2 plate R=15 mm": (lambda: scenes.c2_plate_small(R=0.015), 5, None, 1e-9, 1e-9),
    "c3 textile 12x12 (tear)": (lambda: scenes.c3_textile(nx=12, steps=8), 8, dict(newton_rel_tol=1e-9), 1e-8, 1e-7),
    "c4 3 Poisson boxes landing": (lambda: scenes.c4_batched(n_scenes=3, n_min=150, n_max=400,
                                                             heights=(0.0002, 0.001)), 25, None,
                                   max(1e-9, SPREAD["c4"]["pos"]), max(1e-9, SPREAD["c4"]["quat"])),
    "c5 slab 600 + ball 80 impact": (lambda: scenes.c5_impact(n_slab=600, n_ball=80, footprint=0.035,
                                                              ball_R=0.008), 3, None,
                                     max(1e-9, SPREAD["c5"]["pos"]), max(1e-9, SPREAD["c5"]["quat"])),
}


@pytest.mark.parametrize("name", list(CASES))
def test_error_against_the_oracle_per_configuration(name):
    make, steps, cfg, ptol64, qtol64 = CASES[name]
    sc = make()
    o = oracle.OracleSim(sc, cfg)
    ref = []
    for _ in range(steps):
        o.step(1)
        ref.append(o.state())
    L = float(np.linalg.norm(sc.pos.max(0) - sc.pos.min(0)))
    row = {}
    for prec, label in ((pkg.BDEM_FP64, "fp64"), (pkg.BDEM_MIXED, "mixed")):
        sim = pkg.Sim(sc, precision=prec, config=cfg)
        ep = eq = 0.0
        same = True
        for k in range(steps):
            sim.step(1)
            st = sim.read_state()
            ep = max(ep, float(np.abs(st["pos"] - ref[k]["pos"]).max()) / L)
            eq = max(eq, qerr(st["quat"], ref[k]["quat"]))
            same = same and bool(np.array_equal(st["broken"], ref[k]["broken"]))
        sim.close()
        row[label] = (ep, eq, same)
    print(f"\nPARITY | {name} | n={sc.n} bonds={sc.nb} steps={steps} | fp64 pos {row['fp64'][0]:.2e} quat "
          f"{row['fp64'][1]:.2e} breaks {'same' if row['fp64'][2] else 'DIFFER'} | mixed pos {row['mixed'][0]:.2e} "
          f"quat {row['mixed'][1]:.2e} breaks {'same' if row['mixed'][2] else 'DIFFER'} | broken {int(ref[-1]['broken'].sum())}"
          f" | fp64 bounds {ptol64:.1e} / {qtol64:.1e}")
    assert row["fp64"][0] <= ptol64 and row["fp64"][1] <= qtol64 and row["fp64"][2]
    assert row["mixed"][0] <= 1e-4 and row["mixed"][1] <= 1e-4 and row["mixed"][2]
