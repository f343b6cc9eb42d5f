"""CPU oracle for the implicit bonded-DEM step -- TEST INFRASTRUCTURE ONLY.

A ctypes front end to `bdem_oracle.c`, a plain single-threaded FP64 C restatement of the paper's method
(Sec. 3-5, Alg. 2 and Alg. 3). Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline /
reference legs may import this package; the CUDA library and its Python binding never do, and the two
share no code. Masses and bond rest data are derived here from the scene description, independently of
the library.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "bdem_oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bdem_oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-D_GNU_SOURCE",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _setup(_lib)
    return _lib


class OrcConfig(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("newton_rel_tol", ctypes.c_double),
                ("newton_max_iter", ctypes.c_int32), ("pcg_max_iter", ctypes.c_int32),
                ("ls_max_halvings", ctypes.c_int32), ("optimizer", ctypes.c_int32), ("ground_z", ctypes.c_double),
                ("k_ground", ctypes.c_double), ("k_self", ctypes.c_double), ("contact_skin", ctypes.c_double),
                ("mu_slide", ctypes.c_double), ("mu_roll", ctypes.c_double),
                ("integrator", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
                ("newton_abs_tol", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)
_up = ctypes.POINTER(ctypes.c_uint8)


class OrcProblem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nb", ctypes.c_int32), ("n_scenes", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("scene_start", _lp), ("p", _dp), ("q", _dp), ("v", _dp), ("u", _dp), ("radius", _dp), ("mass", _dp),
                ("kinematic", _up), ("bi", _ip), ("bj", _ip), ("l0", _dp), ("d0", _dp), ("R0", _dp), ("kn", _dp),
                ("kt", _dp), ("kbt", _dp), ("shear_scale", _dp), ("break_strain", _dp), ("broken", _up),
                ("tensile_strength", _dp), ("shear_strength", _dp), ("morton", _ip)]


class OrcStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int32), ("pcg_iters", ctypes.c_int32), ("ls_halvings", ctypes.c_int32),
                ("status", ctypes.c_int32), ("g0_norm", ctypes.c_double), ("g_norm", ctypes.c_double),
                ("n_candidates", ctypes.c_int32), ("bonds_broken", ctypes.c_int32)]


def _setup(L):
    P, C = ctypes.POINTER(OrcProblem), ctypes.POINTER(OrcConfig)
    L.orc_bond_rest.argtypes = [P, _dp, _dp, _dp, _dp, _dp]
    L.orc_step.argtypes = [C, P, ctypes.POINTER(OrcStats)]
    L.orc_bond_terms.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_bond_terms_at.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, _dp,
                                    _dp]
    L.orc_bond_terms_at.restype = None
    L.orc_bond_energy_parts.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_bond_stress.argtypes = [P, ctypes.c_int, _dp, _dp, _dp]
    L.orc_bond_stress.restype = None
    L.orc_system.argtypes = [C, P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _ip]
    L.orc_matvec.argtypes = [C, P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_zhat.argtypes = [C, P, ctypes.c_int, _dp, _dp, _dp, _dp]
    L.orc_morton_order.argtypes = [_lp, ctypes.c_int, _dp, _ip]
    L.orc_morton_order.restype = None
    L.orc_amg_apply.argtypes = [C, P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_amg_level1_apply.argtypes = [C, P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_pcg_solve.argtypes = [C, P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp]
    L.orc_energy_diff.argtypes = [C, P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_energy_diff.restype = ctypes.c_double
    L.orc_retract.argtypes = [_dp, _dp, _dp, ctypes.c_double, _dp, _dp]
    L.orc_retract.restype = None
    L.orc_precond_apply.argtypes = [_dp, _dp, _dp]
    L.orc_precond_apply.restype = ctypes.c_int
    L.orc_eig_clamp.argtypes = [ctypes.c_int, _dp]
    L.orc_eig_clamp.restype = None
    L.orc_eig_sym.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    L.orc_eig_sym.restype = None
    L.orc_contact_candidates.argtypes = [C, P, ctypes.c_int, _dp, _ip, ctypes.c_int, ctypes.c_int]
    for f in ("orc_Ql", "orc_Qr", "orc_Gl", "orc_Gr"):
        getattr(L, f).argtypes = [_dp, _dp]
        getattr(L, f).restype = None
    L.orc_qmul.argtypes = [_dp, _dp, _dp]
    L.orc_qmul.restype = None
    L.orc_rotate.argtypes = [_dp, _dp, _dp]
    L.orc_rotate.restype = None
    L.orc_jet_selftest.argtypes = [_dp, _dp, _dp, _dp]
    L.orc_jet_selftest.restype = None
    L.orc_bond_terms.restype = None
    L.orc_bond_energy_parts.restype = None


def _d(a):
    return a.ctypes.data_as(_dp)


def f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


# ---- quaternion algebra (App. A) ---------------------------------------------------------------

def _mat(fn, q, shape):
    out = np.zeros(shape)
    q = f64(q)
    getattr(lib(), fn)(_d(q), _d(out))
    return out


def Ql(q): return _mat("orc_Ql", q, (4, 4))
def Qr(q): return _mat("orc_Qr", q, (4, 4))
def Gl(q): return _mat("orc_Gl", q, (3, 4))
def Gr(q): return _mat("orc_Gr", q, (3, 4))


def qmul(a, b):
    out = np.zeros(4)
    a, b = f64(a), f64(b)
    lib().orc_qmul(_d(a), _d(b), _d(out))
    return out


def rotate(q, d0):
    out = np.zeros(3)
    q, d0 = f64(q), f64(d0)
    lib().orc_rotate(_d(q), _d(d0), _d(out))
    return out


def retract(p, q, step6, alpha=1.0):
    po, qo = np.zeros(3), np.zeros(4)
    p, q, s = f64(p), f64(q), f64(step6)
    lib().orc_retract(_d(p), _d(q), _d(s), float(alpha), _d(po), _d(qo))
    return po, qo


def precond_apply(D, r):
    """Block-Jacobi preconditioner of Sec. 5.3 on one 6x6 block: (z = D^-1 r, 1) by Cholesky, or the fallback
    (r_a / D_aa, 0) for a block that is not positive definite."""
    D = f64(D, (6, 6)).copy()
    r = f64(r, (6,)).copy()
    z = np.zeros(6)
    ok = lib().orc_precond_apply(_d(D), _d(r), _d(z))
    return z, int(ok)


def eig_clamp(A):
    A = f64(A).copy()
    lib().orc_eig_clamp(A.shape[0], _d(A))
    return A


def eig_sym(A):
    A = f64(A)
    n = A.shape[0]
    lam, V = np.zeros(n), np.zeros((n, n))
    lib().orc_eig_sym(n, _d(A), _d(lam), _d(V))
    return lam, V


def jet_selftest(x):
    x = f64(x)
    f, g, H = np.zeros(1), np.zeros(4), np.zeros((4, 4))
    lib().orc_jet_selftest(_d(x), _d(f), _d(g), _d(H))
    return f[0], g, H


# ---- simulation wrapper ------------------------------------------------------------------------

class OracleSim:
    """Holds a scene's state for the oracle. Masses m = density 4/3 pi r^3; bond rest data from the
    initial state (Sec. 3.2)."""

    def __init__(self, scene, config=None):
        self.scene = scene
        cfg = dict(scene.config)
        if config:
            cfg.update(config)
        self.cfg = cfg
        n, nb = scene.n, scene.nb
        self.p = f64(scene.pos, (n, 3)).copy()
        self.q = f64(scene.quat, (n, 4)).copy()
        self.v = f64(scene.vel, (n, 3)).copy()
        self.u = f64(scene.quat_vel, (n, 4)).copy()
        self.radius = f64(scene.radius).copy()
        dens = np.array([scene.materials[m].density for m in scene.material], np.float64)
        self.mass = dens * (4.0 / 3.0) * math.pi * self.radius ** 3
        self.kin = np.ascontiguousarray(scene.kinematic, np.uint8).copy()
        self.starts = np.ascontiguousarray(scene.scene_offsets, np.int64).copy()
        bi = np.ascontiguousarray(scene.bond_i, np.int32)
        bj = np.ascontiguousarray(scene.bond_j, np.int32)
        self.bi, self.bj = bi.copy(), bj.copy()
        self.l0, self.d0, self.R0 = np.zeros(nb), np.zeros((nb, 3)), np.zeros((nb, 9))
        self.kn, self.kt, self.kbt = np.zeros(nb), np.zeros(nb), np.zeros((nb, 3))
        self.shs, self.brk = np.zeros(nb), np.zeros(nb)
        self.broken = np.zeros(nb, np.uint8)
        mats = [scene.materials[m] for m in scene.bond_material]
        E = f64([m.E for m in mats]) if nb else np.zeros(0)
        nu = f64([m.nu for m in mats]) if nb else np.zeros(0)
        bts = f64([m.bend_twist_scale for m in mats]) if nb else np.zeros(0)
        shs = f64([m.shear_scale for m in mats]) if nb else np.zeros(0)
        brk = f64([m.break_strain for m in mats]) if nb else np.zeros(0)
        self.sig_c = f64([getattr(m, "tensile_strength", math.inf) for m in mats]) if nb else np.zeros(0)
        self.tau_c = f64([getattr(m, "shear_strength", math.inf) for m in mats]) if nb else np.zeros(0)
        self._build_problem()
        if nb:
            lib().orc_bond_rest(ctypes.byref(self.P), _d(E), _d(nu), _d(bts), _d(shs), _d(brk))
        self.C = self._config()

    def _config(self):
        c = self.cfg
        C = OrcConfig()
        C.dt = c["dt"]
        for k in range(3):
            C.gravity[k] = c["gravity"][k]
        C.newton_rel_tol = c["newton_rel_tol"]
        C.newton_max_iter = int(c["newton_max_iter"])
        C.pcg_max_iter = int(c["pcg_max_iter"])
        C.ls_max_halvings = int(c["ls_max_halvings"])
        C.ground_z = c["ground_z"]
        C.k_ground = c["k_ground"]
        C.k_self = c["k_self"]
        C.contact_skin = c["contact_skin"]
        C.optimizer = int(c.get("optimizer", 0))
        C.mu_slide = c.get("friction_slide", 0.0)
        C.mu_roll = c.get("friction_roll", 0.0)
        C.integrator = int(c.get("integrator", 0))
        C.preconditioner = int(c.get("preconditioner", 0))
        C.newton_abs_tol = float(c.get("newton_abs_tol", 0.0))
        return C

    def _build_problem(self):
        P = OrcProblem()
        P.n, P.nb, P.n_scenes = self.scene.n, self.scene.nb, self.scene.n_scenes
        P.scene_start = self.starts.ctypes.data_as(_lp)
        P.p, P.q, P.v, P.u = _d(self.p), _d(self.q), _d(self.v), _d(self.u)
        P.radius, P.mass = _d(self.radius), _d(self.mass)
        P.kinematic = self.kin.ctypes.data_as(_up)
        P.bi, P.bj = self.bi.ctypes.data_as(_ip), self.bj.ctypes.data_as(_ip)
        P.l0, P.d0, P.R0, P.kn, P.kt, P.kbt = _d(self.l0), _d(self.d0), _d(self.R0), _d(self.kn), _d(self.kt), _d(self.kbt)
        P.shear_scale, P.break_strain = _d(self.shs), _d(self.brk)
        P.broken = self.broken.ctypes.data_as(_up)
        P.tensile_strength, P.shear_strength = _d(self.sig_c), _d(self.tau_c)
        # Z-order of the initial positions (the AMG's aggregation order)
        self.morton = np.zeros(max(self.scene.n, 1), np.int32)
        if self.scene.n:
            pos0 = f64(self.scene.pos)
            lib().orc_morton_order(self.starts.ctypes.data_as(_lp), int(self.scene.n_scenes), _d(pos0),
                                   self.morton.ctypes.data_as(_ip))
        P.morton = self.morton.ctypes.data_as(_ip)
        self.P = P

    def step(self, n_steps=1):
        """Advance n_steps; returns a list (per step) of per-scene stats dicts."""
        out = []
        for _ in range(n_steps):
            st = (OrcStats * self.scene.n_scenes)()
            lib().orc_step(ctypes.byref(self.C), ctypes.byref(self.P), st)
            out.append([{f: getattr(s, f) for f, _ in OrcStats._fields_} for s in st])
        return out

    def state(self):
        return dict(pos=self.p.copy(), quat=self.q.copy(), vel=self.v.copy(), quat_vel=self.u.copy(),
                    broken=self.broken.copy())

    def set_state(self, pos, quat, vel, quat_vel, broken=None):
        self.p[:] = pos
        self.q[:] = quat
        self.v[:] = vel
        self.u[:] = quat_vel
        if broken is not None:
            self.broken[:] = broken

    def bond_terms(self, b, pi, qi, pj, qj):
        e, g, H, Hs = np.zeros(1), np.zeros(12), np.zeros((12, 12)), np.zeros((12, 12))
        pi, qi, pj, qj = f64(pi), f64(qi), f64(pj), f64(qj)
        lib().orc_bond_terms(ctypes.byref(self.P), int(b), _d(pi), _d(qi), _d(pj), _d(qj), _d(e), _d(g), _d(H), _d(Hs))
        return e[0], g, H, Hs

    def bond_terms_at(self, b, pvi, qvi, pvj, qvj, qi, qj, w):
        """Energy at the evaluation point, reduced gradient (12) and unprojected / projected reduced Hessians
        (12x12) of the bond term x -> V_b(w x + (1 - w) x_n), reduced at the state's quaternions (qi, qj)."""
        e, g, H, Hs = np.zeros(1), np.zeros(12), np.zeros((12, 12)), np.zeros((12, 12))
        args = [f64(x) for x in (pvi, qvi, pvj, qvj, qi, qj)]
        lib().orc_bond_terms_at(ctypes.byref(self.P), int(b), *[_d(x) for x in args], float(w), _d(e), _d(g), _d(H),
                                _d(Hs))
        return e[0], g, H, Hs

    def bond_energy_parts(self, b, pi, qi, pj, qj):
        out = np.zeros(3)
        pi, qi, pj, qj = f64(pi), f64(qi), f64(pj), f64(qj)
        lib().orc_bond_energy_parts(ctypes.byref(self.P), int(b), _d(pi), _d(qi), _d(pj), _d(qj), _d(out))
        return out

    def bond_stress(self, b, pos=None, quat=None):
        """(sigma, tau) of bond b at (pos, quat), default the current state (stress fracture criterion)."""
        pos = self.p if pos is None else f64(pos, (self.scene.n, 3))
        quat = self.q if quat is None else f64(quat, (self.scene.n, 4))
        out = np.zeros(2)
        lib().orc_bond_stress(ctypes.byref(self.P), int(b), _d(pos), _d(quat), _d(out))
        return out

    def bond_stresses(self, pos=None, quat=None):
        return np.array([self.bond_stress(b, pos, quat) for b in range(self.scene.nb)]).reshape(-1, 2)

    def _scene_range(self, scene):
        return int(self.starts[scene]), int(self.starts[scene + 1])

    def system(self, p, q, phat, qhat, scene=0):
        """Phi, reduced gradient [ns,6], diagonal blocks [ns,6,6], per-bond 12x12 blocks of the scene's
        intact bonds, candidate count at (p, q)."""
        a, b = self._scene_range(scene)
        ns = b - a
        sel = np.nonzero((self.bi >= a) & (self.bi < b) & (self.broken == 0))[0]
        phi, g, D = np.zeros(1), np.zeros((ns, 6)), np.zeros((ns, 6, 6))
        H = np.zeros((max(1, sel.size), 12, 12))
        nc = np.zeros(1, np.int32)
        p, q, phat, qhat = f64(p), f64(q), f64(phat), f64(qhat)
        lib().orc_system(ctypes.byref(self.C), ctypes.byref(self.P), scene, _d(p), _d(q), _d(phat), _d(qhat),
                         _d(phi), _d(g), _d(D), _d(H), nc.ctypes.data_as(_ip))
        return dict(phi=phi[0], g=g, diag=D, bondH=H[:sel.size], bond_ids=sel, n_candidates=int(nc[0]))

    def matvec(self, p, q, phat, qhat, x, scene=0):
        a, b = self._scene_range(scene)
        y = np.zeros((b - a, 6))
        p, q, phat, qhat, x = f64(p), f64(q), f64(phat), f64(qhat), f64(x)
        lib().orc_matvec(ctypes.byref(self.C), ctypes.byref(self.P), scene, _d(p), _d(q), _d(phat), _d(qhat), _d(x), _d(y))
        return y

    def pcg_solve(self, p, q, phat, qhat, b, eps_r, max_iter, scene=0):
        a, e = self._scene_range(scene)
        x = np.zeros((e - a, 6))
        p, q, phat, qhat, b = f64(p), f64(q), f64(phat), f64(qhat), f64(b)
        it = lib().orc_pcg_solve(ctypes.byref(self.C), ctypes.byref(self.P), scene, _d(p), _d(q), _d(phat), _d(qhat),
                                 _d(b), float(eps_r), int(max_iter), _d(x))
        return x, it

    def energy_diff(self, phat, qhat, p0, q0, p1, q1, scene=0):
        a0, a1 = np.zeros(1), np.zeros(1)
        args = [f64(x) for x in (phat, qhat, p0, q0, p1, q1)]
        d = lib().orc_energy_diff(ctypes.byref(self.C), ctypes.byref(self.P), scene, *[_d(x) for x in args],
                                  _d(a0), _d(a1))
        return d, a0[0], a1[0]

    def contact_candidates(self, p, scene=0, brute=False, cap=1 << 22):
        pairs = np.zeros((cap, 2), np.int32)
        p = f64(p)
        cnt = lib().orc_contact_candidates(ctypes.byref(self.C), ctypes.byref(self.P), scene, _d(p),
                                           pairs.ctypes.data_as(_ip), cap, 1 if brute else 0)
        return pairs[:min(cnt, cap)].copy()

    def amg_apply(self, p, q, phat, qhat, r, scene=0):
        """z = M^-1 r of the scene's AMG preconditioner at (p, q); returns (z [ns,6], number of levels)."""
        a, b = self._scene_range(scene)
        z = np.zeros((b - a, 6))
        args = [f64(x) for x in (p, q, phat, qhat, r)]
        nl = lib().orc_amg_apply(ctypes.byref(self.C), ctypes.byref(self.P), scene, *[_d(x) for x in args], _d(z))
        return z, nl

    def amg_level1_apply(self, p, q, phat, qhat, e, scene=0):
        """y = A_1 e with the AMG's level-1 (Galerkin) operator; e [n_agg,6] in Z-order of the aggregates."""
        e = f64(e)
        y = np.zeros_like(e)
        args = [f64(x) for x in (p, q, phat, qhat)]
        m = lib().orc_amg_level1_apply(ctypes.byref(self.C), ctypes.byref(self.P), scene, *[_d(x) for x in args],
                                       _d(e), _d(y))
        assert m == e.shape[0], (m, e.shape)
        return y

    def zhat(self, phat, qhat, scene=0):
        """The variational midpoint target zhat of the scene (Sec. 3.1, App. C) for the inertia targets
        (phat, qhat); contact candidates found at phat."""
        zp, zq = np.zeros((self.scene.n, 3)), np.zeros((self.scene.n, 4))
        phat, qhat = f64(phat), f64(qhat)
        lib().orc_zhat(ctypes.byref(self.C), ctypes.byref(self.P), scene, _d(phat), _d(qhat), _d(zp), _d(zq))
        return zp, zq

    def predict(self):
        """xhat = x_n + dt v_n and the initial guess (phat, qhat/|qhat|) of Alg. 3."""
        dt = self.cfg["dt"]
        ph = self.p + dt * self.v
        qh = self.q + dt * self.u
        return ph, qh, ph.copy(), qh / np.linalg.norm(qh, axis=1, keepdims=True)
