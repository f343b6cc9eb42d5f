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
    """The oracle's trajectory of one scene at Newton setting cfg; with alternative settings `alts` (name -> cfg), also
    one step at each of them from every step's input state (the reference trajectory's previous state), recorded under
    states[k]["alt"][name] with its status under stats[k]["alt_status"][name]."""
    sc, steps, cfg = args[:3]
    alts = args[3] if len(args) > 3 else {}
    if sc.n == 0:  # an empty scene has nothing to advance
        z = {"pos": np.zeros((0, 3)), "quat": np.zeros((0, 4)), "vel": np.zeros((0, 3)),
             "quat_vel": np.zeros((0, 4)), "broken": np.zeros(0, np.uint8)}
        st0 = {"newton_iters": 0, "pcg_iters": 0, "status": 0, "bonds_broken": 0}
        return ([dict(z, alt={a: z for a in alts}) for _ in range(steps)],
                [dict(st0, alt_status={a: 0 for a in alts}) for _ in range(steps)])
    import oracle
    oracle.build()
    o = oracle.OracleSim(sc, cfg)
    others = {a: oracle.OracleSim(sc, dict(cfg or {}, **c)) for a, c in alts.items()}
    states, stats = [], []
    for _ in range(steps):
        prev = o.state()
        alt, alt_status = {}, {}
        for a, oa in others.items():
            oa.set_state(prev["pos"], prev["quat"], prev["vel"], prev["quat_vel"], prev["broken"])
            alt_status[a] = oa.step(1)[0][0]["status"]
            sa = oa.state()
            alt[a] = {k: sa[k] for k in ("pos", "quat", "broken")}
        stt = o.step(1)[0][0]
        stt["alt_status"] = alt_status
        stats.append(stt)
        st = o.state()
        states.append(dict({k: st[k] for k in ("pos", "quat", "vel", "quat_vel", "broken")}, alt=alt))
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
    alts = list(res[0][0][0].get("alt", {})) if res and steps else []

    def blank():
        return {"pos": np.zeros((sc.n, 3)), "quat": np.zeros((sc.n, 4)), "vel": np.zeros((sc.n, 3)),
                "quat_vel": np.zeros((sc.n, 4)), "broken": np.zeros(sc.nb, np.uint8)}

    for t in range(steps):
        out = blank()
        out["alt"] = {a: blank() for a in alts}
        for s, (st, _) in enumerate(res):
            a, b = (int(off[s]), int(off[s + 1])) if parts > 1 else (0, sc.n)
            sel = slice(None) if parts == 1 else (bond_scene == s)
            for dst, src in [(out, st[t])] + [(out["alt"][n], st[t]["alt"][n]) for n in alts]:
                for f in ("pos", "quat", "vel", "quat_vel"):
                    if f in src:
                        dst[f][a:b] = src[f]
                dst["broken"][sel] = src["broken"]
        states.append(out)
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

    def submit(self, name, sc, steps, cfg=None, alts=None):
        parts = split_scenes(sc) if sc.n_scenes > 1 else [sc]
        order = sorted(range(len(parts)), key=lambda k: -(parts[k].n + parts[k].nb))
        handles = {k: self.pool.apply_async(_trajectory, ((parts[k], steps, cfg, alts or {}),)) for k in order}
        self.cases[name] = (sc, steps, [handles[k] for k in range(len(parts))])

    def result(self, name, timeout=3600):
        sc, steps, hs = self.cases[name]
        return _assemble(sc, steps, [h.get(timeout) for h in hs])

    def close(self):
        self.pool.terminate()
        self.pool.join()


def trajectories(sc, steps, cfg=None, processes=None):
    """Per-step oracle states of a (possibly batched) scene: a list over steps of dicts pos [N,3], quat [N,4], vel
    [N,3], quat_vel [N,4] and broken [B] in the scene's own particle and bond order, plus per-step lists of per-scene
    stats."""
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
