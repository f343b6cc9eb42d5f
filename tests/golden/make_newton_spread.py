"""Writes newton_spread.json: how far the oracle's own trajectory moves when its Newton tolerance is tightened 100x.

A Newton solve stopped at |g| <= tol |g_0| pins the state down only to the scene's sensitivity to that stopping
test; two correct solvers that round differently can land that far apart. For each case of the per-configuration
parity report whose FP64 agreement is limited by it, this runs the oracle (and nothing else) at the case's tolerance
and at 1/100 of it and records the
largest position difference (relative to the bounding-box diagonal) and quaternion difference over the steps.

    python tests/golden/make_newton_spread.py [case ...]   # all cases, or only the named ones (merged into the file)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402
from paper_2308_10459_gb300 import scenes  # noqa: E402

# the cases whose FP64 agreement with the oracle is limited by this spread rather than by rounding (the cube and
# plate cases agree to 1e-12, far inside the 1e-9 bound; the textile's bound is derived where it is tested, since
# tightening its tolerance changes its break set)
CASES = {
    "c4": (lambda: scenes.c4_batched(n_scenes=3, n_min=150, n_max=400, heights=(0.0002, 0.001)), 25, 1e-6),
    "c5": (lambda: scenes.c5_impact(n_slab=600, n_ball=80, footprint=0.035, ball_R=0.008), 3, 1e-6),
    # the plate at R = 50 mm (about 6,800 particles) of the PCG launch-shape test: two grids that round differently
    "plate50": (lambda: scenes.c2_plate_small(R=0.05), 2, 1e-6),
    # the variational midpoint form: the 4x4x4 cube bouncing off the ground and three Poisson-disk boxes landing
    "cube_mid": (lambda: scenes.cube_lattice(nx=4, z_bottom=0.01, k_ground=1e6, steps=50, integrator=1), 50, 1e-6),
    "c4_mid": (lambda: _with(scenes.c4_batched(n_scenes=3, n_min=150, n_max=400, heights=(0.0002, 0.001)),
                             integrator=1), 25, 1e-6),
}


def _with(sc, **cfg):
    sc.config = dict(sc.config, **cfg)
    return sc


def qerr(a, b):
    return float(np.minimum(np.abs(a - b).max(1), np.abs(a + b).max(1)).max()) if len(a) else 0.0


def spread(make, steps, tol):
    sc = make()
    L = float(np.linalg.norm(sc.pos.max(0) - sc.pos.min(0)))
    runs = []
    for t in (tol, tol / 100.0):
        o = oracle.OracleSim(sc, dict(newton_rel_tol=t))
        states = []
        for _ in range(steps):
            o.step(1)
            states.append(o.state())
        runs.append(states)
    ep = max(float(np.abs(a["pos"] - b["pos"]).max()) / L for a, b in zip(*runs))
    eq = max(qerr(a["quat"], b["quat"]) for a, b in zip(*runs))
    return ep, eq


def main(names):
    oracle.build()
    path = os.path.join(HERE, "newton_spread.json")
    out = {}
    if names and os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for name, (make, steps, tol) in CASES.items():
        if names and name not in names:
            continue
        ep, eq = spread(make, steps, tol)
        out[name] = {"steps": steps, "newton_rel_tol": tol, "pos": ep, "quat": eq}
        print(name, out[name], flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
