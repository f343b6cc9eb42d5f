"""Seeded synthetic scene generators (inputs only).

These build the particle packings, bond lists, materials and solver settings of the workloads the
library is measured on. They hold none of the method's arithmetic: no energies, masses, stiffnesses
or rest data (each consumer derives those itself from the radii, materials and positions given here).
Both the CUDA library's tests/benchmark and the CPU oracle consume the same `Scene` objects.

Workload shapes follow the paper's demos (Table 1: ceramic plate drop, knitted cloth tear) and the
element packing of Sec. 3.4 (hexagonal close packing); the paper uses no public dataset, so every
scene here is synthetic and seeded.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # bond-neighbour search; scipy is present on both build and GPU machines
    from scipy.spatial import cKDTree
except Exception:  # pragma: no cover
    cKDTree = None


@dataclasses.dataclass
class Material:
    """Bond material. shear_scale multiplies the shear angle (1: the energy exactly as printed, in N/m;
    a length such as the rest bond length: the dimensionally consistent energy in J). A bond breaks when its
    tensile strain exceeds break_strain, or its stresses exceed tensile_strength (sigma_c) or shear_strength
    (tau_c); +inf switches a criterion off."""
    E: float
    nu: float
    density: float
    break_strain: float = math.inf
    bend_twist_scale: float = 1.0
    shear_scale: float = 1.0
    tensile_strength: float = math.inf
    shear_strength: float = math.inf


@dataclasses.dataclass
class Scene:
    """Particles (SoA, FP64), bonds, materials and solver settings of one or more independent scenes."""

    pos: np.ndarray            # [N,3]
    quat: np.ndarray           # [N,4] (x, y, z, w)
    vel: np.ndarray            # [N,3]
    quat_vel: np.ndarray       # [N,4]
    radius: np.ndarray         # [N]
    material: np.ndarray       # [N] int32 index into materials
    kinematic: np.ndarray      # [N] uint8
    scene_offsets: np.ndarray  # [S+1] int64
    bond_i: np.ndarray         # [B] int32
    bond_j: np.ndarray         # [B] int32
    bond_material: np.ndarray  # [B] int32
    materials: list
    config: dict
    name: str = "scene"

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nb(self) -> int:
        return int(self.bond_i.shape[0])

    @property
    def n_scenes(self) -> int:
        return int(self.scene_offsets.shape[0] - 1)

    def copy(self) -> "Scene":
        return dataclasses.replace(
            self, pos=self.pos.copy(), quat=self.quat.copy(), vel=self.vel.copy(), quat_vel=self.quat_vel.copy(),
            radius=self.radius.copy(), material=self.material.copy(), kinematic=self.kinematic.copy(),
            scene_offsets=self.scene_offsets.copy(), bond_i=self.bond_i.copy(), bond_j=self.bond_j.copy(),
            bond_material=self.bond_material.copy(), materials=list(self.materials), config=dict(self.config))


def default_config(**kw) -> dict:
    c = dict(dt=1e-3, gravity=(0.0, 0.0, -9.81), newton_rel_tol=1e-6, newton_max_iter=100, pcg_max_iter=1000,
             ls_max_halvings=30, ground_z=0.0, k_ground=0.0, k_self=0.0, contact_skin=0.0, friction_slide=0.0,
             friction_roll=0.0, optimizer=0, integrator=0, preconditioner=0, newton_abs_tol=0.0, pcg_refine=4,
             steps=100)
    c.update(kw)
    return c


def _pairs_within(pos: np.ndarray, cutoff: float) -> np.ndarray:
    """All index pairs i<j with |p_i - p_j| < cutoff, sorted lexicographically."""
    if pos.shape[0] < 2:
        return np.zeros((0, 2), np.int64)
    if cKDTree is not None:
        pr = cKDTree(pos).query_pairs(cutoff, output_type="ndarray").astype(np.int64)
    else:  # small inputs only
        d = np.linalg.norm(pos[:, None, :] - pos[None, :, :], axis=-1)
        i, j = np.nonzero(np.triu(d < cutoff, 1))
        pr = np.stack([i, j], 1)
    if pr.size == 0:
        return np.zeros((0, 2), np.int64)
    pr = np.sort(pr, axis=1)
    order = np.lexsort((pr[:, 1], pr[:, 0]))
    return pr[order]


def _assemble(pos, radius, mat, kin, pairs, materials, config, name, vel=None, offsets=None, bond_mat=None):
    n = pos.shape[0]
    q = np.zeros((n, 4))
    q[:, 3] = 1.0
    return Scene(
        pos=np.ascontiguousarray(pos, np.float64),
        quat=q,
        vel=np.zeros((n, 3)) if vel is None else np.ascontiguousarray(vel, np.float64),
        quat_vel=np.zeros((n, 4)),
        radius=np.ascontiguousarray(radius, np.float64),
        material=np.ascontiguousarray(mat, np.int32),
        kinematic=np.ascontiguousarray(kin, np.uint8),
        scene_offsets=np.array([0, n], np.int64) if offsets is None else np.asarray(offsets, np.int64),
        bond_i=np.ascontiguousarray(pairs[:, 0], np.int32),
        bond_j=np.ascontiguousarray(pairs[:, 1], np.int32),
        bond_material=(np.ascontiguousarray(mat[pairs[:, 0]], np.int32) if bond_mat is None
                       else np.ascontiguousarray(bond_mat, np.int32)),
        materials=materials, config=config, name=name)


# --------------------------------------------------------------------------------------------------
# Simple-cubic lattice cube (the 1,000-particle FP64 case and its small / contact variants)
# --------------------------------------------------------------------------------------------------

def cube_lattice(nx=10, spacing=0.01, r=0.005, z_bottom=0.2, E=1e7, nu=0.3, density=2500.0, dt=1e-3,
                 k_ground=1e6, steps=100, break_strain=math.inf, jitter=0.0, seed=1, vel=(0.0, 0.0, 0.0),
                 shear_scale=None, name=None, **cfg) -> Scene:
    """nx^3 particles, 6-neighbour bonds (3 nx^2 (nx-1) of them), identity orientations. The shear angle is
    scaled by the lattice spacing (the dimensionally consistent shear energy) unless shear_scale is given."""
    g = np.arange(nx) * spacing
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel() + z_bottom], 1)
    pairs = _pairs_within(pos, 1.05 * spacing)
    if jitter:
        pos = pos + np.random.default_rng(seed).uniform(-jitter, jitter, pos.shape)
    n = pos.shape[0]
    v = np.tile(np.asarray(vel, np.float64), (n, 1))
    mats = [Material(E, nu, density, break_strain, 1.0, spacing if shear_scale is None else shear_scale)]
    config = default_config(dt=dt, k_ground=k_ground, ground_z=0.0, steps=steps, **cfg)
    return _assemble(pos, np.full(n, r), np.zeros(n, np.int32), np.zeros(n, np.uint8), pairs, mats, config,
                     name or f"cube{nx}", vel=v)


def c1_cube() -> Scene:
    """1,000 particles, 10x10x10 lattice, spacing 10 mm, radius 5 mm, 2,700 bonds, lowest layer at 0.2 m."""
    return cube_lattice(name="c1_cube1000")


def c1b_cube_contact(nx=10, steps=300) -> Scene:
    """The same cube starting 5 mm above the ground (lowest sphere surface 5 mm up), exercising contact."""
    return cube_lattice(nx=nx, z_bottom=0.005 + 0.005, steps=steps, name=f"c1b_cube{nx}_contact")


# --------------------------------------------------------------------------------------------------
# Hexagonal-close-packed disk (the ceramic plate drop)
# --------------------------------------------------------------------------------------------------

def hcp_points(R, layers, r):
    """HCP lattice points (spacing 2r) inside a disk of radius R, `layers` layers (ABA stacking)."""
    a = 2.0 * r
    dy = a * math.sqrt(3.0) / 2.0
    dz = a * math.sqrt(2.0 / 3.0)
    nrow = int(math.ceil(R / dy)) + 2
    ncol = int(math.ceil(R / a)) + 2
    pts = []
    for k in range(layers):
        off = (0.0, 0.0) if k % 2 == 0 else (a / 2.0, dy / 3.0)
        jj, ii = np.meshgrid(np.arange(-nrow, nrow + 1), np.arange(-ncol, ncol + 1), indexing="ij")
        x = ii * a + (jj % 2) * (a / 2.0) + off[0]
        y = jj * dy + off[1]
        m = x * x + y * y <= R * R
        pts.append(np.stack([x[m], y[m], np.full(m.sum(), k * dz)], 1))
    return np.concatenate(pts, 0)


def c2_plate(R=0.284, layers=3, r=1e-3, E=5e9, nu=0.3, density=2500.0, break_strain=1e-3, vz=-3.0,
             tilt_deg=10.0, gap=1e-3, jitter=1e-5, seed=2, dt=5e-4, steps=200, name=None) -> Scene:
    """Ceramic-plate fracture: ~220K particles for R = 0.284 m (3 layers, r = 1 mm), bonds within
    1.05*2r on the unjittered lattice, +-1e-5 m jitter, tilted 10 deg about x, dropped at 3 m/s with its
    lowest point `gap` above the ground; penalty stiffness E*r for ground and self contact."""
    pts = hcp_points(R, layers, r)
    pairs = _pairs_within(pts, 1.05 * 2.0 * r)
    rng = np.random.default_rng(seed)
    pts = pts + rng.uniform(-jitter, jitter, pts.shape)
    t = math.radians(tilt_deg)
    rot = np.array([[1, 0, 0], [0, math.cos(t), -math.sin(t)], [0, math.sin(t), math.cos(t)]])
    pts = pts @ rot.T
    pts[:, 2] += (gap + r) - pts[:, 2].min()
    n = pts.shape[0]
    vel = np.zeros((n, 3))
    vel[:, 2] = vz
    mats = [Material(E, nu, density, break_strain, 1.0, 2.0 * r)]
    config = default_config(dt=dt, k_ground=E * r, k_self=E * r, contact_skin=r, ground_z=0.0, steps=steps)
    return _assemble(pts, np.full(n, r), np.zeros(n, np.int32), np.zeros(n, np.uint8), pairs, mats, config,
                     name or f"c2_plate{n}", vel=vel)


def c2_plate_small(R=0.02, **kw) -> Scene:
    """The same plate construction at a radius the oracle finishes quickly (R = 0.02 m: ~1.1K particles)."""
    return c2_plate(R=R, name=kw.pop("name", "c2_plate_small"), **kw)


# --------------------------------------------------------------------------------------------------
# Textile-like lattice (the knitted-cloth tear)
# --------------------------------------------------------------------------------------------------

def c3_textile(nx=300, spacing=2e-3, r=1e-3, E=1e9, nu=0.3, density=1500.0, bend_twist_scale=1e-3,
               break_strain=0.3, pull=0.5, dt=1e-3, steps=500, name=None) -> Scene:
    """nx x nx planar lattice, bonds along x, y and both diagonals; the columns x = 0 and x = max are
    kinematic and move apart at `pull` m/s each; gravity on, no ground."""
    g = np.arange(nx)
    y, x = np.meshgrid(g, g, indexing="ij")
    ix, iy = x.ravel(), y.ravel()
    pos = np.stack([ix * spacing, iy * spacing, np.zeros(ix.size)], 1)
    idx = (iy * nx + ix)
    pairs = []
    for dxo, dyo in ((1, 0), (0, 1), (1, 1), (1, -1)):
        m = (ix + dxo < nx) & (iy + dyo >= 0) & (iy + dyo < nx)
        pairs.append(np.stack([idx[m], (iy[m] + dyo) * nx + ix[m] + dxo], 1))
    pairs = np.sort(np.concatenate(pairs, 0), axis=1)
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    n = pos.shape[0]
    kin = ((ix == 0) | (ix == nx - 1)).astype(np.uint8)
    vel = np.zeros((n, 3))
    vel[ix == 0, 0] = -pull
    vel[ix == nx - 1, 0] = pull
    mats = [Material(E, nu, density, break_strain, bend_twist_scale, spacing)]
    config = default_config(dt=dt, k_ground=0.0, steps=steps)
    return _assemble(pos, np.full(n, r), np.zeros(n, np.int32), kin, pairs, mats, config,
                     name or f"c3_textile{nx}", vel=vel)


# --------------------------------------------------------------------------------------------------
# Poisson-disk packed boxes, batched scenes, slab impact
# --------------------------------------------------------------------------------------------------

def _dart_throw(sample, n_target, r, rng, batch, max_rounds=400, min_accept=None):
    """Dart throwing with minimum distance 2r, in rounds of `batch` darts drawn by sample(rng, batch): a dart is
    kept when it is at least 2r from every point already placed and from every earlier dart of its round that is
    itself not rejected by a placed point (a dart that conflicts with an earlier one of the same round is dropped,
    as sequential throwing would have dropped one of the two). Stops at n_target points or when a round keeps
    fewer than min_accept darts (default: 1% of a round)."""
    if min_accept is None:
        min_accept = max(2, batch // 100)
    d2 = 2.0 * r
    pts = np.zeros((0, 3))
    for _ in range(max_rounds):
        if pts.shape[0] >= n_target:
            break
        cand = sample(rng, batch)
        if pts.shape[0]:
            dist, _ = cKDTree(pts).query(cand, k=1, distance_upper_bound=d2)
            cand = cand[~(dist < d2)]
        if cand.shape[0] > 1:
            pr = cKDTree(cand).query_pairs(d2, output_type="ndarray")
            if pr.size:
                drop = np.zeros(cand.shape[0], bool)
                drop[np.maximum(pr[:, 0], pr[:, 1])] = True
                cand = cand[~drop]
        take = cand[: max(0, n_target - pts.shape[0])]
        pts = np.concatenate([pts, take], 0)
        if take.shape[0] < min_accept:
            break
    return pts


def poisson_box(n_target, r, rng, aspect=(1.0, 1.0, 1.0), fraction=0.28, **kw):
    """Dart-throwing packing of n_target spheres in a box of the given aspect, sized for the packing fraction
    `fraction` (round-based dart throwing stalls near 0.3, so the default reaches the target count)."""
    vol = n_target * (4.0 / 3.0) * math.pi * r ** 3 / fraction
    s = (vol / (aspect[0] * aspect[1] * aspect[2])) ** (1.0 / 3.0)
    ext = np.array(aspect) * s
    pts = _dart_throw(lambda g, m: g.uniform(0.0, 1.0, (m, 3)) * ext, n_target, r, rng, max(256, n_target // 8), **kw)
    return pts, ext


def poisson_ball(n_target, r, R, rng):
    """Dart-throwing packing of n_target spheres inside a ball of radius R centred at the origin."""
    def sample(g, m):
        v = g.normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        return v * (R * g.uniform(0.0, 1.0, (m, 1)) ** (1.0 / 3.0))
    return _dart_throw(sample, n_target, r, rng, max(256, n_target // 4))


def c4_batched(n_scenes=64, n_min=2000, n_max=50000, r=2e-3, E=1e8, nu=0.3, density=2500.0, break_strain=2e-3,
               cutoff_factor=1.1, dt=1e-3, steps=200, seed=4, heights=(0.1, 1.0), name=None) -> Scene:
    """Independent Poisson-disk boxes with log-uniform particle counts and drop heights U[0.1, 1] m; each
    scene has its own ground contact and no contact across scenes."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_scenes)).astype(int)
    heights = rng.uniform(heights[0], heights[1], n_scenes)
    pos_all, pairs_all, offsets = [], [], [0]
    for s in range(n_scenes):
        pts, ext = poisson_box(int(counts[s]), r, rng)
        pts = pts - np.array([ext[0] / 2.0, ext[1] / 2.0, 0.0]) + np.array([0.0, 0.0, heights[s] + r])
        pr = _pairs_within(pts, cutoff_factor * 2.0 * r) + offsets[-1]
        pos_all.append(pts)
        pairs_all.append(pr)
        offsets.append(offsets[-1] + pts.shape[0])
    pos = np.concatenate(pos_all, 0)
    pairs = np.concatenate(pairs_all, 0)
    n = pos.shape[0]
    mats = [Material(E, nu, density, break_strain, 1.0, 2.0 * r)]
    config = default_config(dt=dt, k_ground=E * r, k_self=E * r, contact_skin=r, steps=steps)
    return _assemble(pos, np.full(n, r), np.zeros(n, np.int32), np.zeros(n, np.uint8), pairs, mats, config,
                     name or f"c4_batched{n_scenes}", offsets=np.array(offsets))


def cutoff_for_degree(pts, target, lo, hi, sample=20000, iters=30, seed=0):
    """Bond cutoff giving a mean neighbour count `target` (bisection on a random sample of the points)."""
    rng = np.random.default_rng(seed)
    tree = cKDTree(pts)
    idx = rng.choice(pts.shape[0], size=min(sample, pts.shape[0]), replace=False)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        deg = np.mean(tree.query_ball_point(pts[idx], mid, return_length=True) - 1)
        lo, hi = (mid, hi) if deg < target else (lo, mid)
    return 0.5 * (lo + hi)


def c5_impact(n_slab=1_000_000, n_ball=2000, r=2e-3, footprint=0.5, ball_R=0.05, E=1e9, nu=0.3, density=2500.0,
              break_strain=1e-3, speed=20.0, degree=12.0, dt=2e-4, steps=300, seed=5, name=None) -> Scene:
    """Large impact: a Poisson-disk slab of n_slab particles on a footprint x footprint base (thickness set by the
    packing), bonds within the cutoff that gives `degree` neighbours on average; above it a ball of radius ball_R
    packed with n_ball particles, bonded by the same rule, unbreakable and 10x stiffer, moving down at `speed`.
    Two scenes' worth of particles in one scene (slab and ball interact through self contact); ground under the
    slab."""
    rng = np.random.default_rng(seed)
    vol = n_slab * (4.0 / 3.0) * math.pi * r ** 3 / 0.28
    thick = vol / footprint ** 2
    slab, ext = poisson_box(n_slab, r, rng, aspect=(footprint / thick, footprint / thick, 1.0))
    slab = slab - np.array([ext[0] / 2.0, ext[1] / 2.0, -r])
    ball = poisson_ball(n_ball, r, ball_R, rng)
    ball = ball + np.array([0.0, 0.0, slab[:, 2].max() + r + ball_R + 2.0 * r])
    cut_s = cutoff_for_degree(slab, degree, 2.0 * r, 4.0 * r)
    cut_b = cutoff_for_degree(ball, degree, 2.0 * r, 6.0 * r, sample=ball.shape[0])
    ps = _pairs_within(slab, cut_s)
    pb = _pairs_within(ball, cut_b) + slab.shape[0]
    pos = np.concatenate([slab, ball], 0)
    n = pos.shape[0]
    mat = np.zeros(n, np.int32)
    mat[slab.shape[0]:] = 1
    pairs = np.concatenate([ps, pb], 0)
    bond_mat = np.concatenate([np.zeros(len(ps), np.int32), np.ones(len(pb), np.int32)])
    mats = [Material(E, nu, density, break_strain, 1.0, 2.0 * r), Material(10.0 * E, nu, density, math.inf, 1.0, 2.0 * r)]
    vel = np.zeros((n, 3))
    vel[slab.shape[0]:, 2] = -speed
    config = default_config(dt=dt, k_ground=E * r, k_self=E * r, contact_skin=r, steps=steps)
    sc = _assemble(pos, np.full(n, r), mat, np.zeros(n, np.uint8), pairs, mats, config, name or "c5_impact",
                   vel=vel, bond_mat=bond_mat)
    sc.config["bond_cutoff_slab"] = float(cut_s)
    sc.config["bond_cutoff_ball"] = float(cut_b)
    return sc


def scene_by_name(name: str) -> Scene:
    table = {
        "c1": c1_cube, "c1b": c1b_cube_contact, "c2": c2_plate, "c2_small": c2_plate_small,
        "c3": c3_textile, "c4": c4_batched, "c5": c5_impact,
    }
    return table[name]()
