"""Pins of the oracle's variational midpoint integrator (Sec. 3.1, Eq. variational optimisation form; App. C).

Phi(x) = 1/(2 dt^2) (x - zhat)^T M_s (x - zhat) + V((x + x_n)/2),
zhat = xhat - 1/2 M_s^{-1} dt^2 grad V((x_{n-1} + x_n)/2),  xhat = 2 x_n - x_{n-1},  x_{n-1} = x_n - dt v_n.

Its stationarity condition is the discrete Euler-Lagrange equation of App. C,
M_s (x_{n+1} - 2 x_n + x_{n-1}) / dt^2 + 1/2 grad V((x_{n+1} + x_n)/2) + 1/2 grad V((x_n + x_{n-1})/2) = 0.
  - A uniform force field and rigid motion: gravity alone gives the same trajectory as the implicit-Euler-like form,
    p_n = p_0 + g dt^2 n (n + 1)/2 from rest.
  - A linear spring (two particles along x, w^2 = 2 kn / m): with a = w^2 dt^2 / 4 the equation becomes
    (1 + a) u_{n+1} - 2 (1 - a) u_n + (1 + a) u_{n-1} = 0, the trapezoidal rule: no amplitude decay, and the
    trajectory converges to the exact oscillation at second order (the implicit-Euler-like form at first order).
  - zhat of a stretched pair at rest has the closed form above with grad V = kn u e_x at the midpoint.
  - The reduced gradient and Hessian of the bond term x -> V_b((x + x_n)/2) equal the central differences of its
    pullback through the exponential-map retraction, and the system gradient those of Phi.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_10459_gb300 import scenes

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

G = np.array([0.0, 0.0, -9.81])
L0, R, E, NU, RHO = 0.01, 0.005, 1e7, 0.3, 2500.0
MASS = RHO * 4.0 / 3.0 * math.pi * R ** 3
KN = E * math.pi * R * R / L0


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def axial_pair(dt, integrator, gravity=(0.0, 0.0, 0.0), tol=1e-13):
    pos = np.array([[0.0, 0.0, 0.0], [L0, 0.0, 0.0]])
    cfg = scenes.default_config(dt=dt, gravity=gravity, k_ground=0.0, newton_rel_tol=tol, integrator=integrator)
    return scenes._assemble(pos, np.full(2, R), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.array([[0, 1]]),
                            [scenes.Material(E, NU, RHO)], cfg, "axial")


def test_free_fall_matches_the_closed_form():
    """Gravity is uniform and the lattice moves rigidly: p_n = p_0 + g dt^2 n (n+1)/2 from rest, as for the
    implicit-Euler-like form."""
    sc = scenes.cube_lattice(nx=3, k_ground=0.0, newton_rel_tol=1e-10, integrator=1)
    o = oracle.OracleSim(sc)
    p0, dt = sc.pos.copy(), sc.config["dt"]
    for n in range(1, 6):
        st = o.step(1)[0][0]
        assert st["status"] == 0
        ref = p0 + G * dt * dt * n * (n + 1) / 2.0
        assert np.abs(o.p - ref).max() <= 1e-8 * np.abs(ref - p0).max()
        assert np.abs(np.abs(o.q[:, 3]) - 1.0).max() < 1e-12


@pytest.mark.parametrize("v_rel", [0.0, 0.02])
def test_zhat_of_a_stretched_pair(v_rel):
    """grad V at the midpoint (x_{n-1} + x_n)/2 = x_n - dt v_n / 2 of a pair stretched by delta and separating at
    v_rel: kn u_m e_x on particle j (minus on i), u_m = delta - dt v_rel / 2; with gravity, -m g on each."""
    dt, delta = 2e-4, 1e-5
    sc = axial_pair(dt, 1, gravity=tuple(G))
    o = oracle.OracleSim(sc)
    p = o.p.copy()
    p[1, 0] += delta
    v = np.zeros((2, 3))
    v[0, 0], v[1, 0] = -0.5 * v_rel, 0.5 * v_rel
    o.set_state(p, o.q.copy(), v, np.zeros((2, 4)))
    ph, qh = p + dt * v, o.q.copy()
    zp, zq = o.zhat(ph, qh)
    um = delta - 0.5 * dt * v_rel
    f = KN * um
    ref = ph.copy()
    ref[1, 0] -= 0.5 * dt * dt * f / MASS
    ref[0, 0] += 0.5 * dt * dt * f / MASS
    ref += 0.5 * dt * dt * G
    # to the rounding floor of the literal shear term's gradient at zero shear angle (about kt eps / l0, here 5e-10
    # of the spring force)
    assert np.abs(zp - ref).max() <= 2e-9 * np.abs(ref - ph).max()
    assert np.abs(zq - qh).max() == 0.0


def axial_run(dt, steps, integrator, delta=1e-5):
    o = oracle.OracleSim(axial_pair(dt, integrator))
    p = o.p.copy()
    p[1, 0] += delta
    o.set_state(p, o.q.copy(), np.zeros((2, 3)), np.zeros((2, 4)))
    u = []
    for _ in range(steps):
        o.step(1)
        u.append(o.p[1, 0] - o.p[0, 0] - L0)
        assert abs(o.p[0, 1]) < 1e-20 and abs(o.p[1, 2]) < 1e-20
    return np.array(u), o


def test_axial_recurrence_is_the_trapezoidal_rule():
    dt, delta = 2e-4, 1e-5
    u, o = axial_run(dt, 60, 1, delta)
    a = (2.0 * KN / MASS) * dt * dt / 4.0
    u_prev, u_cur = delta, delta
    for n in range(60):
        u_next = (2.0 * (1.0 - a) * u_cur - (1.0 + a) * u_prev) / (1.0 + a)
        u_prev, u_cur = u_cur, u_next
        # the shear term's gradient floor at zero shear angle (5e-10 of the spring force) enters every step
        assert abs(u[n] - u_cur) <= 1e-8 * delta, (n, u[n], u_cur)
    # no amplitude decay: the recurrence's roots lie on the unit circle (amplitude delta / cos(w dt / 2) at most)
    w = math.sqrt(2.0 * KN / MASS)
    assert np.abs(u).max() <= delta / math.cos(math.atan(math.sqrt(a))) * (1 + 1e-9)
    assert np.abs(u).max() >= 0.99 * delta
    assert abs(o.v[:, 0].sum()) < 1e-9 * delta / dt  # centre of mass at rest
    assert w > 0


def test_second_order_against_first_order():
    """Error at t = 2e-4 s against the exact oscillation through both starting values (zero velocity at t = -dt/2:
    u(t) = A cos(w (t + dt/2)), A = delta / cos(w dt / 2)); halving dt divides the midpoint form's error by ~4 and
    the implicit-Euler-like form's by ~2."""
    w = math.sqrt(2.0 * KN / MASS)
    T, delta = 2e-4, 1e-5
    err = {0: [], 1: []}
    for dt in (1e-5, 5e-6, 2.5e-6):
        n = int(round(T / dt))
        exact = delta / math.cos(0.5 * w * dt) * math.cos(w * (n * dt + 0.5 * dt))
        for integ in (0, 1):
            u, _ = axial_run(dt, n, integ, delta)
            err[integ].append(abs(u[-1] - exact))
    r_mid = [err[1][k] / err[1][k + 1] for k in range(2)]
    r_eul = [err[0][k] / err[0][k + 1] for k in range(2)]
    assert all(3.5 < r < 4.5 for r in r_mid), r_mid
    assert all(1.7 < r < 2.3 for r in r_eul), r_eul
    assert err[1][-1] < 0.1 * err[0][-1]


def mid_pullback(o, x, xn, xi):
    pi, qi = oracle.retract(x[0], x[1], xi[:6])
    pj, qj = oracle.retract(x[2], x[3], xi[6:])
    return o.bond_energy_parts(0, 0.5 * (pi + xn[0]), 0.5 * (qi + xn[1]), 0.5 * (pj + xn[2]),
                               0.5 * (qj + xn[3])).sum()


def test_midpoint_bond_terms_against_pullback_differences():
    """Reduced gradient and unprojected Hessian of x -> V_b((x + x_n)/2) = first and second central differences of
    its pullback xi -> V_b((R_x(xi) + x_n)/2); the projected Hessian is the eigen-clamp of the unprojected one."""
    rng = np.random.default_rng(21)
    n0 = np.array([0.3, -0.2, 0.93])
    n0 /= np.linalg.norm(n0)
    pos = np.stack([np.zeros(3), L0 * n0])
    sc = scenes._assemble(pos, np.full(2, R), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.array([[0, 1]]),
                          [scenes.Material(E, NU, 2500.0)], scenes.default_config(integrator=1), "pair")
    o = oracle.OracleSim(sc)
    hs = np.array([1e-6] * 3 + [1e-4] * 3 + [1e-6] * 3 + [1e-4] * 3)

    def qrot(axis, ang):
        return Rotation.from_rotvec(np.asarray(axis, float) * ang).as_quat()

    for _ in range(3):
        pi = rng.normal(size=3) * 1e-3
        pj = pi + L0 * n0 * (1 + rng.uniform(-0.05, 0.05)) + rng.normal(size=3) * 5e-4
        x = (pi, qrot(rng.normal(size=3), 0.4), pj, qrot(rng.normal(size=3), 0.4))
        xn = (pi + rng.normal(size=3) * 2e-4, qrot(rng.normal(size=3), 0.3),
              pj + rng.normal(size=3) * 2e-4, qrot(rng.normal(size=3), 0.3))
        mid = [0.5 * (a + b) for a, b in zip(x, xn)]
        e, g, H, Hs = o.bond_terms_at(0, *mid, x[1], x[3], 0.5)
        assert np.isclose(e, mid_pullback(o, x, xn, np.zeros(12)), rtol=1e-13)
        gfd = np.zeros(12)
        for a in range(12):
            ea = np.zeros(12)
            ea[a] = hs[a]
            gfd[a] = (-mid_pullback(o, x, xn, 2 * ea) + 8 * mid_pullback(o, x, xn, ea)
                      - 8 * mid_pullback(o, x, xn, -ea) + mid_pullback(o, x, xn, -2 * ea)) / (12 * hs[a])
        sc_g = np.abs(g) + np.abs(gfd).max() * 1e-7
        assert np.all(np.abs(g - gfd) <= 1e-5 * sc_g + 1e-9 * np.abs(g).max()), (g, gfd)
        Hfd = np.zeros((12, 12))
        for a in range(12):
            for b in range(a, 12):
                ea, eb = np.zeros(12), np.zeros(12)
                ea[a], eb[b] = hs[a], hs[b]
                v = (mid_pullback(o, x, xn, ea + eb) - mid_pullback(o, x, xn, ea - eb)
                     - mid_pullback(o, x, xn, -ea + eb) + mid_pullback(o, x, xn, -ea - eb)) / (4 * hs[a] * hs[b])
                Hfd[a, b] = Hfd[b, a] = v
        d = np.sqrt(np.abs(np.outer(np.diag(H), np.diag(H)))) + 1e-12 * np.abs(H).max()
        assert np.all(np.abs(H - Hfd) <= 2e-5 * d + 1e-7 * np.abs(H).max()), np.abs(H - Hfd).max()
        lam, V = np.linalg.eigh(H)
        assert np.allclose(Hs, V @ np.diag(np.maximum(lam, 0)) @ V.T, atol=1e-11 * np.abs(H).max())


def test_system_gradient_matches_objective_differences():
    """Whole system (inertia towards zhat, gravity, ground, bonds and contacts at the midpoints with a start state
    x_n different from x): the reduced gradient is d/dxi of Phi(R_x(xi)) at 0, and the termwise line-search
    difference equals the plain difference of Phi."""
    sc = scenes.cube_lattice(nx=2, spacing=0.0098, r=0.005, k_ground=1e6, z_bottom=0.0045, k_self=1e5,
                             contact_skin=0.005, integrator=1)
    rng = np.random.default_rng(7)
    o = oracle.OracleSim(sc)
    pn = sc.pos + rng.normal(size=sc.pos.shape) * 2e-4
    qn = Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * 0.15).as_quat()
    o.set_state(pn, qn, np.zeros((sc.n, 3)), np.zeros((sc.n, 4)))
    p = pn + rng.normal(size=sc.pos.shape) * 3e-4
    q = (Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * 0.1) * Rotation.from_quat(qn)).as_quat()
    phat = sc.pos + rng.normal(size=sc.pos.shape) * 1e-4
    qhat = q + rng.normal(size=q.shape) * 0.01
    sysd = o.system(p, q, phat, qhat)
    n = p.shape[0]

    def phi(xi):
        pp, qq = np.zeros_like(p), np.zeros_like(q)
        for i in range(n):
            pp[i], qq[i] = oracle.retract(p[i], q[i], xi[i])
        return o.system(pp, qq, phat, qhat)["phi"]

    for _ in range(4):
        d = rng.normal(size=(n, 6)) * np.array([1e-4] * 3 + [1e-2] * 3)
        h = 1e-3
        fd = (-phi(2 * h * d) + 8 * phi(h * d) - 8 * phi(-h * d) + phi(-2 * h * d)) / (12 * h)
        an = (sysd["g"] * d).sum()
        assert abs(fd - an) <= 1e-6 * (np.abs(sysd["g"] * d).sum() + 1e-30), (fd, an)
    for scale in (1e-3, 1e-4):
        st = rng.normal(size=(n, 6)) * np.array([scale * 0.01] * 3 + [scale] * 3)
        p1, q1 = np.zeros_like(p), np.zeros_like(q)
        for i in range(n):
            p1[i], q1[i] = oracle.retract(p[i], q[i], st[i])
        dd, phi0, phi1 = o.energy_diff(phat, qhat, p, q, p1, q1)
        assert abs(dd - (phi1 - phi0)) <= 1e-9 * abs(phi1 - phi0) + 1e-13 * abs(phi0)


def test_sphere_bounce_matches_a_scalar_solve_of_the_discrete_equation():
    """A sphere dropped on the penalty ground: each step's z_{n+1} is the root, found by bracketing, of
    m (z_{n+1} - 2 z_n + z_{n-1}) / dt^2 + 1/2 V'((z_{n+1} + z_n)/2) + 1/2 V'((z_n + z_{n-1})/2) = 0 with
    V(z) = m 9.81 z + 1/2 k min(z - r, 0)^2. With the contact stiffness far beyond 1/dt^2 (w dt = 28) the one-sided
    contact switching inside a step makes the sphere leave faster than it arrived: a property of this form, reproduced
    here by the scalar solve."""
    brentq = pytest.importorskip("scipy.optimize").brentq
    k, dt, z0 = 1e6, 1e-3, 0.01
    cfg = scenes.default_config(dt=dt, k_ground=k, integrator=1, newton_rel_tol=1e-13)
    sc = scenes._assemble(np.array([[0.0, 0.0, z0]]), np.full(1, R), np.zeros(1, np.int32), np.zeros(1, np.uint8),
                          np.zeros((0, 2), np.int64), [scenes.Material(E, NU, RHO)], cfg, "sphere")
    o = oracle.OracleSim(sc)

    def dV(z):
        return MASS * 9.81 + (k * (z - R) if z < R else 0.0)

    zprev, z = z0, z0
    v_in = v_out = 0.0
    for n in range(45):
        def f(zn):
            return MASS * (zn - 2.0 * z + zprev) / dt ** 2 + 0.5 * dV(0.5 * (zn + z)) + 0.5 * dV(0.5 * (z + zprev))
        zn = brentq(f, z - 0.05, z + 0.05, xtol=1e-16, rtol=1e-15)
        zprev, z = z, zn
        o.step(1)
        assert abs(o.p[0, 2] - z) <= 1e-10 * z0, (n, o.p[0, 2], z)
        v = (z - zprev) / dt
        v_in, v_out = min(v_in, v), max(v_out, v)
    assert v_in < -0.3 and v_out > 2.0 * abs(v_in)


def test_midpoint_differs_from_euler_only_through_the_potential():
    """With no potential (free unbonded particles, no gravity, no contact) both forms reduce to x_{n+1} = xhat."""
    pos = np.array([[0.0, 0.0, 0.0], [0.05, 0.0, 0.0]])
    vel = np.array([[0.1, -0.2, 0.3], [0.0, 0.4, -0.1]])
    out = []
    for integ in (0, 1):
        cfg = scenes.default_config(dt=1e-3, gravity=(0.0, 0.0, 0.0), integrator=integ)
        sc = scenes._assemble(pos, np.full(2, R), np.zeros(2, np.int32), np.zeros(2, np.uint8),
                              np.zeros((0, 2), np.int64), [scenes.Material(E, NU, RHO)], cfg, "free", vel=vel)
        o = oracle.OracleSim(sc)
        o.step(3)
        out.append(o.p.copy())
    assert np.array_equal(out[0], out[1])
    assert np.allclose(out[1], pos + 3e-3 * vel, rtol=0, atol=1e-15)
