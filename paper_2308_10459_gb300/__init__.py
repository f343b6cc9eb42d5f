"""Python binding of libbdem (include/bdem.h): argument marshalling only.

Every stage of the implicit bonded-DEM step runs in the library's sm_103a CUDA kernels. The binding loads the
in-tree `_build/libbdem.so` (built by `paper_2308_10459_gb300.build.build()`); if it is missing or cannot be
loaded, importing a function that needs it raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build_mod

LIB_PATH = _build_mod.LIB

BDEM_OK, BDEM_E_INVALID, BDEM_E_NOMEM, BDEM_E_CUDA = 0, 1, 2, 3
BDEM_E_NEWTON_MAXITER, BDEM_E_LINESEARCH, BDEM_E_NONFINITE, BDEM_E_TIMEOUT = 4, 5, 6, 7
BDEM_FP64, BDEM_MIXED = 0, 1
BDEM_INT_EULER, BDEM_INT_MIDPOINT = 0, 1
BDEM_PRECOND_BLOCK_JACOBI, BDEM_PRECOND_AMG = 0, 1
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "CUDA", 4: "NEWTON_MAXITER", 5: "LINESEARCH", 6: "NONFINITE",
                7: "TIMEOUT"}


class bdem_material(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("density", ctypes.c_double),
                ("break_strain", ctypes.c_double), ("bend_twist_scale", ctypes.c_double),
                ("shear_scale", ctypes.c_double), ("tensile_strength", ctypes.c_double),
                ("shear_strength", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class bdem_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class bdem_config(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("newton_rel_tol", ctypes.c_double),
                ("newton_max_iter", ctypes.c_int32), ("pcg_max_iter", ctypes.c_int32),
                ("ls_max_halvings", ctypes.c_int32), ("precision", ctypes.c_int32), ("ground_z", ctypes.c_double),
                ("k_ground", ctypes.c_double), ("k_self", ctypes.c_double), ("contact_skin", ctypes.c_double),
                ("spd_mode", ctypes.c_int32), ("optimizer", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
                ("friction_slide", ctypes.c_double), ("friction_roll", ctypes.c_double),
                ("integrator", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
                ("newton_abs_tol", ctypes.c_double), ("pcg_refine", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("allocator", ctypes.POINTER(bdem_allocator))]


class bdem_step_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("newton_iters", ctypes.c_int32), ("pcg_iters", ctypes.c_int32),
                ("ls_halvings", ctypes.c_int32), ("bonds_broken", ctypes.c_int32),
                ("contact_candidates", ctypes.c_int32), ("status", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("g0_norm", ctypes.c_double), ("g_norm", ctypes.c_double),
                ("contact_entry_pcg_iters", ctypes.c_int64), ("intact_bonds", ctypes.c_int64),
                ("lin_rel_residual", ctypes.c_double), ("refine_rounds", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


PHASES = ["predict", "contact", "grad", "hess", "pcg", "linesearch", "finish"]


class bdem_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 7), ("intervals", ctypes.c_int64 * 7), ("pcg_iters", ctypes.c_int64),
                ("newton_iters", ctypes.c_int64), ("particle_newton_iters", ctypes.c_int64),
                ("steps", ctypes.c_int64)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)
_up = ctypes.POINTER(ctypes.c_uint8)
_vp = ctypes.c_void_p

# C prototypes (names identical to include/bdem.h)
_PROTOS = {
    "bdem_create": (ctypes.c_int, [ctypes.POINTER(bdem_config), ctypes.c_int32, _lp, _dp, _dp, _dp, _dp, _dp, _ip,
                                   ctypes.POINTER(bdem_material), ctypes.c_int32, _up, ctypes.POINTER(_vp)]),
    "bdem_add_bonds": (ctypes.c_int, [_vp, ctypes.c_int64, _ip, _ip, _ip]),
    "bdem_step": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(bdem_step_stats)]),
    "bdem_read_state": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp, _up]),
    "bdem_write_state": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp, _up]),
    "bdem_sizes": (ctypes.c_int, [_vp, _lp, _lp, _ip]),
    "bdem_bond_order": (ctypes.c_int, [_vp, _ip]),
    "bdem_destroy": (None, [_vp]),
    "bdem_last_error": (ctypes.c_char_p, [_vp]),
    "bdem_debug_system": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp, _dp, _lp]),
    "bdem_debug_system_at": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _lp]),
    "bdem_debug_zhat": (ctypes.c_int, [_vp, _dp, _dp]),
    "bdem_debug_matvec": (ctypes.c_int, [_vp, _dp, _dp]),
    "bdem_debug_bonds": (ctypes.c_int, [_vp, ctypes.c_int64, _ip, _dp]),
    "bdem_debug_bond_stress": (ctypes.c_int, [_vp, _dp]),
    "bdem_debug_wait_timeout": (ctypes.c_int, [_vp, ctypes.c_double]),
    "bdem_debug_pcg": (ctypes.c_int, [_vp, _dp, ctypes.c_double, ctypes.c_int32, _dp, _ip]),
    "bdem_launch_count": (ctypes.c_int64, [_vp]),
    "bdem_set_step_graph": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "bdem_graph_steps": (ctypes.c_int64, [_vp]),
    "bdem_graph_error": (ctypes.c_char_p, [_vp]),
    "bdem_pcg_static": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int32, _ip]),
    "bdem_set_pcg_shape": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "bdem_autotune_pcg": (ctypes.c_int, [_vp, ctypes.c_int32, _ip, _ip]),
    "bdem_set_pcg_product": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "bdem_set_bond_tile": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "bdem_autotune_bonds": (ctypes.c_int, [_vp, ctypes.c_int32, _ip, _ip]),
    "bdem_get_pcg_shape": (ctypes.c_int, [_vp, _ip, _ip, _ip]),
    "bdem_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "bdem_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(bdem_profile)]),
}

_lib = None


def load(path: str | None = None):
    """Load libbdem.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libbdem.so not found at {p}; run paper_2308_10459_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _PROTOS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_PROTOS)


class BdemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _arr(a, dtype, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ct)


class TorchAllocator:
    """A bdem_allocator hook that takes the library's device buffers from PyTorch's caching allocator (on the
    library's stream) and returns them to it. Keep the object alive while a simulation created with it exists."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.live = {}
        self.calls = 0

        def _alloc(ctx, nbytes, stream):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
            except Exception:
                return None
            self.live[ptr] = int(nbytes)
            self.calls += 1
            return ptr

        def _free(ctx, ptr, stream):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._alloc = ALLOC_FN(_alloc)  # the C function pointers must outlive every call through them
        self._free = FREE_FN(_free)
        self.struct = bdem_allocator(self._alloc, self._free, None)


def make_config(cfg: dict, precision=BDEM_FP64, cuda_stream=None) -> bdem_config:
    c = bdem_config()
    c.dt = cfg["dt"]
    for k in range(3):
        c.gravity[k] = cfg["gravity"][k]
    c.newton_rel_tol = cfg["newton_rel_tol"]
    c.newton_max_iter = int(cfg["newton_max_iter"])
    c.pcg_max_iter = int(cfg["pcg_max_iter"])
    c.ls_max_halvings = int(cfg["ls_max_halvings"])
    c.precision = int(precision)
    c.ground_z = cfg["ground_z"]
    c.k_ground = cfg["k_ground"]
    c.k_self = cfg["k_self"]
    c.contact_skin = cfg["contact_skin"]
    c.spd_mode = 0
    c.optimizer = int(cfg.get("optimizer", 0))
    c.cuda_stream = cuda_stream
    c.friction_slide = cfg.get("friction_slide", 0.0)
    c.friction_roll = cfg.get("friction_roll", 0.0)
    c.integrator = int(cfg.get("integrator", 0))
    c.preconditioner = int(cfg.get("preconditioner", 0))
    c.newton_abs_tol = float(cfg.get("newton_abs_tol", 0.0))
    c.pcg_refine = int(cfg.get("pcg_refine", 0))
    c.reserved0 = 0
    return c


def bdem_create(config: bdem_config, scene_offsets, pos, quat, vel, quat_vel, radius, particle_material, mats,
                kinematic=None):
    """Thin wrapper of bdem_create; returns an opaque handle (c_void_p)."""
    L = load()
    so = _arr(scene_offsets, np.int64)
    n = int(so[-1])
    pos, quat = _arr(pos, np.float64, (n, 3)), _arr(quat, np.float64, (n, 4))
    vel = None if vel is None else _arr(vel, np.float64, (n, 3))
    quat_vel = None if quat_vel is None else _arr(quat_vel, np.float64, (n, 4))
    radius, pm = _arr(radius, np.float64, (n,)), _arr(particle_material, np.int32, (n,))
    kin = None if kinematic is None else _arr(kinematic, np.uint8, (n,))
    M = (bdem_material * len(mats))()
    for k, m in enumerate(mats):
        M[k] = bdem_material(m.E, m.nu, m.density, m.break_strain, m.bend_twist_scale, m.shear_scale,
                             getattr(m, "tensile_strength", math.inf), getattr(m, "shear_strength", math.inf))
    h = _vp()
    st = L.bdem_create(ctypes.byref(config), len(so) - 1, _ptr(so, _lp), _ptr(pos, _dp), _ptr(quat, _dp),
                       _ptr(vel, _dp), _ptr(quat_vel, _dp), _ptr(radius, _dp), _ptr(pm, _ip), M, len(mats),
                       _ptr(kin, _up), ctypes.byref(h))
    if st != BDEM_OK:
        raise BdemError(st, L.bdem_last_error(None).decode())
    return h


class Sim:
    """Owns one bdem_sim. Methods mirror the C entry points."""

    def __init__(self, scene, precision=BDEM_FP64, config=None, cuda_stream=None, allocator=None):
        cfg = dict(scene.config)
        if config:
            cfg.update(config)
        self.scene = scene
        self.cfg = cfg
        self.precision = precision
        self.config = make_config(cfg, precision, cuda_stream)
        self.allocator = allocator  # a TorchAllocator (or any object with a bdem_allocator .struct), kept alive here
        if allocator is not None:
            self.config.allocator = ctypes.pointer(allocator.struct)
        self.L = load()
        self.h = bdem_create(self.config, scene.scene_offsets, scene.pos, scene.quat, scene.vel, scene.quat_vel,
                             scene.radius, scene.material, scene.materials, scene.kinematic)
        self.n = scene.n
        self.n_scenes = scene.n_scenes
        if scene.nb:
            self.bdem_add_bonds(scene.bond_i, scene.bond_j, scene.bond_material)

    def _check(self, st, ok=(BDEM_OK,)):
        if st not in ok:
            raise BdemError(st, self.L.bdem_last_error(self.h).decode())
        return st

    def bdem_add_bonds(self, i, j, m):
        i, j, m = _arr(i, np.int32), _arr(j, np.int32), _arr(m, np.int32)
        self._check(self.L.bdem_add_bonds(self.h, i.size, _ptr(i, _ip), _ptr(j, _ip), _ptr(m, _ip)))

    def bdem_step(self, n_steps=1, allow_warnings=True):
        stats = (bdem_step_stats * self.n_scenes)()
        ok = (BDEM_OK, BDEM_E_NEWTON_MAXITER, BDEM_E_LINESEARCH) if allow_warnings else (BDEM_OK,)
        st = self._check(self.L.bdem_step(self.h, int(n_steps), stats), ok)
        self.last_status = st
        return [{f: getattr(s, f) for f, _ in bdem_step_stats._fields_} for s in stats]

    step = bdem_step

    def sizes(self):
        n, nb, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        self._check(self.L.bdem_sizes(self.h, ctypes.byref(n), ctypes.byref(nb), ctypes.byref(ns)))
        return n.value, nb.value, ns.value

    def bond_order(self):
        nb = self.sizes()[1]
        pairs = np.zeros((max(nb, 1), 2), np.int32)
        self._check(self.L.bdem_bond_order(self.h, _ptr(pairs, _ip)))
        return pairs[:nb]

    def bdem_read_state(self, out=None):
        n, nb, _ = self.sizes()
        o = out or dict(pos=np.zeros((n, 3)), quat=np.zeros((n, 4)), vel=np.zeros((n, 3)), quat_vel=np.zeros((n, 4)),
                        broken=np.zeros(max(nb, 1), np.uint8))
        self._check(self.L.bdem_read_state(self.h, _ptr(o["pos"], _dp), _ptr(o["quat"], _dp), _ptr(o["vel"], _dp),
                                           _ptr(o["quat_vel"], _dp), _ptr(o["broken"], _up)))
        if out is None:
            o["broken"] = o["broken"][:nb]
        return o

    read_state = bdem_read_state

    def bdem_write_state(self, pos=None, quat=None, vel=None, quat_vel=None, broken=None):
        n = self.n
        a = [None if x is None else _arr(x, np.float64, s) for x, s in
             ((pos, (n, 3)), (quat, (n, 4)), (vel, (n, 3)), (quat_vel, (n, 4)))]
        b = None if broken is None else _arr(broken, np.uint8)
        self._check(self.L.bdem_write_state(self.h, _ptr(a[0], _dp), _ptr(a[1], _dp), _ptr(a[2], _dp),
                                            _ptr(a[3], _dp), _ptr(b, _up)))

    write_state = bdem_write_state

    def bdem_debug_system(self, phat, qhat, want_bonds=True, pos=None, quat=None):
        """The Newton system at the committed state, or at the iterate (pos, quat) when given (bdem_debug_system_at)."""
        n, nb, _ = self.sizes()
        phat, qhat = _arr(phat, np.float64, (n, 3)), _arr(qhat, np.float64, (n, 4))
        g, D = np.zeros((n, 6)), np.zeros((n, 6, 6))
        H = np.zeros((max(nb, 1), 12, 12)) if want_bonds else None
        nc = ctypes.c_int64()
        if pos is None:
            self._check(self.L.bdem_debug_system(self.h, _ptr(phat, _dp), _ptr(qhat, _dp), _ptr(g, _dp),
                                                 _ptr(D, _dp), _ptr(H, _dp) if want_bonds else None,
                                                 ctypes.byref(nc)))
        else:
            pos, quat = _arr(pos, np.float64, (n, 3)), _arr(quat, np.float64, (n, 4))
            self._check(self.L.bdem_debug_system_at(self.h, _ptr(pos, _dp), _ptr(quat, _dp), _ptr(phat, _dp),
                                                    _ptr(qhat, _dp), _ptr(g, _dp), _ptr(D, _dp),
                                                    _ptr(H, _dp) if want_bonds else None, ctypes.byref(nc)))
        return dict(g=g, diag=D, bondH=None if H is None else H[:nb], n_candidates=nc.value)

    def bdem_debug_zhat(self):
        """The inertia targets of a step from the committed state: xhat, or zhat in the midpoint form."""
        n = self.sizes()[0]
        zp, zq = np.zeros((n, 3)), np.zeros((n, 4))
        self._check(self.L.bdem_debug_zhat(self.h, _ptr(zp, _dp), _ptr(zq, _dp)))
        return zp, zq

    def bdem_debug_bonds(self, ids):
        ids = _arr(ids, np.int32)
        out = np.zeros((max(ids.size, 1), 12, 12))
        self._check(self.L.bdem_debug_bonds(self.h, ids.size, _ptr(ids, _ip), _ptr(out, _dp)))
        return out[:ids.size]

    def bdem_debug_bond_stress(self):
        """(sigma, tau) of every bond at the committed state, [n_bonds][2] in the order of addition."""
        nb = self.sizes()[1]
        out = np.zeros((max(nb, 1), 2))
        self._check(self.L.bdem_debug_bond_stress(self.h, _ptr(out, _dp)))
        return out[:nb]

    def bdem_debug_wait_timeout(self, limit_ms):
        """Status of a device wait that must run out after limit_ms (BDEM_E_TIMEOUT expected)."""
        return int(self.L.bdem_debug_wait_timeout(self.h, float(limit_ms)))

    def bdem_debug_matvec(self, x):
        x = _arr(x, np.float64, (self.n, 6))
        y = np.zeros((self.n, 6))
        self._check(self.L.bdem_debug_matvec(self.h, _ptr(x, _dp), _ptr(y, _dp)))
        return y

    def bdem_debug_pcg(self, b, eps_r, max_iter):
        b = _arr(b, np.float64, (self.n, 6))
        x = np.zeros((self.n, 6))
        it = np.zeros(self.n_scenes, np.int32)
        self._check(self.L.bdem_debug_pcg(self.h, _ptr(b, _dp), float(eps_r), int(max_iter), _ptr(x, _dp),
                                          _ptr(it, _ip)))
        return x, it

    def bdem_pcg_static(self, b_dev_ptr, x_dev_ptr, eps_r, max_iter):
        """Allocation-free PCG (see include/bdem.h): b and x are device addresses of [n][6] float64 arrays."""
        it = np.zeros(self.n_scenes, np.int32)
        self._check(self.L.bdem_pcg_static(self.h, ctypes.c_void_p(b_dev_ptr), ctypes.c_void_p(x_dev_ptr),
                                           float(eps_r), int(max_iter), _ptr(it, _ip)))
        return it

    def set_pcg_shape(self, lanes_per_row, blocks=0):
        self._check(self.L.bdem_set_pcg_shape(self.h, int(lanes_per_row), int(blocks)))

    def set_pcg_product(self, product):
        self._check(self.L.bdem_set_pcg_product(self.h, int(product)))

    def set_bond_tile(self, tile, capped=0):
        self._check(self.L.bdem_set_bond_tile(self.h, int(tile), int(capped)))

    def autotune_bonds(self, reps=3):
        t, c = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.L.bdem_autotune_bonds(self.h, int(reps), ctypes.byref(t), ctypes.byref(c)))
        return {"tile": t.value, "capped": c.value}

    def pcg_shape(self):
        lanes, blocks, product = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.L.bdem_get_pcg_shape(self.h, ctypes.byref(lanes), ctypes.byref(blocks), ctypes.byref(product)))
        return {"lanes_per_row": lanes.value, "blocks": blocks.value, "product": product.value}

    def autotune_pcg(self, iters=30):
        l, g = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.L.bdem_autotune_pcg(self.h, int(iters), ctypes.byref(l), ctypes.byref(g)))
        return l.value, g.value

    def profile_enable(self, on=True):
        self._check(self.L.bdem_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        p = bdem_profile()
        self._check(self.L.bdem_profile_read(self.h, ctypes.byref(p)))
        return dict(ms={k: p.ms[i] for i, k in enumerate(PHASES)},
                    intervals={k: p.intervals[i] for i, k in enumerate(PHASES)}, pcg_iters=p.pcg_iters,
                    newton_iters=p.newton_iters, particle_newton_iters=p.particle_newton_iters, steps=p.steps)

    def launch_count(self):
        return int(self.L.bdem_launch_count(self.h))

    def set_step_graph(self, on=True):
        self._check(self.L.bdem_set_step_graph(self.h, 1 if on else 0))

    def graph_steps(self):
        return int(self.L.bdem_graph_steps(self.h))

    def graph_error(self):
        return (self.L.bdem_graph_error(self.h) or b"").decode()

    def close(self):
        if getattr(self, "h", None):
            self.L.bdem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
