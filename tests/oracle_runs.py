"""Oracle trajectories for the parity tests, computed in parallel worker processes (test infrastructure).

Scenes of one simulation never interact (each has its own ground and contacts, and converges on its own), so a
batched case is split into its scenes and each scene's trajectory is computed by its own oracle instance in a pool of
worker processes started with the `spawn` method (never forked from a process that has touched the GPU). A single
scene runs in one worker. Only the oracle runs here; nothing from the CUDA path is used.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def split_scenes(sc):
    """One Scene per scene of a batched Scene (particles, bonds and materials re-indexed)."""
    from paper_2308_10459_gb300.scenes import Scene
    out = []
    off = np.asarray(sc.scene_offsets, np.int64)
    for s in range(len(off) - 1):
        a, b = int(off[s]), int(off[s + 1])
        m = (sc.bond_i >= a) & (sc.bond_i < b)
        out.append(Scene(pos=sc.pos[a:b].copy(), quat=sc.quat[a:b].copy(), vel=sc.vel[a:b].copy(),
                         quat_vel=sc.quat_vel[a:b].copy(), radius=sc.radius[a:b].copy(),
                         material=sc.material[a:b].copy(), kinematic=sc.kinematic[a:b].copy(),
                         scene_offsets=np.array([0, b - a], np.int64), bond_i=(sc.bond_i[m] - a).astype(np.int32),
                         bond_j=(sc.bond_j[m] - a).astype(np.int32), bond_material=sc.bond_material[m].copy(),
                         materials=list(sc.materials), config=dict(sc.config), name=f"{sc.name}[{s}]"))
    return out


def _trajectory(args):
    sc, steps, cfg = args
    if sc.n == 0:  # an empty scene has nothing to advance
        return ([{"pos": np.zeros((0, 3)), "quat": np.zeros((0, 4)), "broken": np.zeros(0, np.uint8)}] * steps,
                [{"newton_iters": 0, "pcg_iters": 0, "status": 0, "bonds_broken": 0}] * steps)
    import oracle
    oracle.build()
    o = oracle.OracleSim(sc, cfg)
    states, stats = [], []
    for _ in range(steps):
        stats.append(o.step(1)[0][0])
        st = o.state()
        states.append({k: st[k] for k in ("pos", "quat", "broken")})
    return states, stats


def _workers():
    try:
        return max(1, min(16, len(os.sched_getaffinity(0))))
    except Exception:
        return max(1, min(16, os.cpu_count() or 1))


def _assemble(sc, steps, res):
    """Per-step states and stats of a scene from its sub-scenes' trajectories (res in scene order)."""
    parts = sc.n_scenes if sc.n_scenes > 1 else 1
    off = np.asarray(sc.scene_offsets, np.int64)
    bond_scene = np.searchsorted(off, sc.bond_i, side="right") - 1
    states, stats = [], []
    for t in range(steps):
        pos = np.zeros((sc.n, 3))
        quat = np.zeros((sc.n, 4))
        broken = np.zeros(sc.nb, np.uint8)
        for s, (st, _) in enumerate(res):
            a, b = (int(off[s]), int(off[s + 1])) if parts > 1 else (0, sc.n)
            pos[a:b] = st[t]["pos"]
            quat[a:b] = st[t]["quat"]
            if parts == 1:
                broken[:] = st[t]["broken"]
            else:
                broken[bond_scene == s] = st[t]["broken"]
        states.append({"pos": pos, "quat": quat, "broken": broken})
        stats.append([r[1][t] for r in res])
    return states, stats


class Batch:
    """Oracle trajectories of several cases computed concurrently in one pool of spawned worker processes: submit()
    queues every scene of a case at once, result() waits for that case only."""

    def __init__(self, processes=None):
        import oracle
        oracle.build()  # compile once before the workers start
        self.pool = mp.get_context("spawn").Pool(processes or _workers())
        self.cases = {}

    def submit(self, name, sc, steps, cfg=None):
        parts = split_scenes(sc) if sc.n_scenes > 1 else [sc]
        order = sorted(range(len(parts)), key=lambda k: -(parts[k].n + parts[k].nb))
        handles = {k: self.pool.apply_async(_trajectory, ((parts[k], steps, cfg),)) for k in order}
        self.cases[name] = (sc, steps, [handles[k] for k in range(len(parts))])

    def result(self, name, timeout=3600):
        sc, steps, hs = self.cases[name]
        return _assemble(sc, steps, [h.get(timeout) for h in hs])

    def close(self):
        self.pool.terminate()
        self.pool.join()


def trajectories(sc, steps, cfg=None, processes=None):
    """Per-step oracle states of a (possibly batched) scene: a list over steps of dicts pos [N,3], quat [N,4] and
    broken [B] in the scene's own particle and bond order, plus per-step lists of per-scene stats."""
    import oracle
    oracle.build()  # compile once before the workers start
    parts = split_scenes(sc) if sc.n_scenes > 1 else [sc]
    jobs = [(p, steps, cfg) for p in parts]
    # largest scenes first so that the pool's tail is short
    order = sorted(range(len(jobs)), key=lambda k: -(parts[k].n + parts[k].nb))
    procs = min(processes or _workers(), len(jobs))
    if procs <= 1:
        res = [_trajectory(j) for j in jobs]
    else:
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs) as pool:
            got = pool.map(_trajectory, [jobs[k] for k in order], chunksize=1)
        res = [None] * len(jobs)
        for k, r in zip(order, got):
            res[k] = r
    return _assemble(sc, steps, res)
