"""Pins of the oracle's time step (Alg. 3 with Alg. 2 inside) against closed forms, textbook linear
algebra and conservation laws."""
import math

import numpy as np
import pytest

import oracle
from paper_2308_10459_gb300 import scenes

G = np.array([0.0, 0.0, -9.81])


def free_particles(n=8, spacing=0.05, r=0.005, seed=0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 1, (n, 3)) * 0.01 + np.stack(np.unravel_index(np.arange(n), (2, 2, 2)), 1) * spacing
    cfg = scenes.default_config(dt=1e-3, k_ground=0.0)
    return scenes._assemble(pos, np.full(n, r), np.zeros(n, np.int32), np.zeros(n, np.uint8),
                            np.zeros((0, 2), np.int64), [scenes.Material(1e7, 0.3, 2500.0)], cfg, "free")


def test_free_fall_unbonded_is_exact_in_one_newton_iteration():
    """Without bonds the reduced Hessian is block diagonal, block-Jacobi PCG is exact, and each step is one
    Newton iteration: p_n = p_0 + g dt^2 n (n+1)/2 (Alg. 3 with xhat = x_n + dt v_n), q stays identity."""
    sc = free_particles()
    o = oracle.OracleSim(sc)
    p0, dt = sc.pos.copy(), sc.config["dt"]
    for n in range(1, 11):
        st = o.step(1)[0][0]
        assert st["newton_iters"] == 1 and st["status"] == 0
        ref = p0 + G * dt * dt * n * (n + 1) / 2.0
        assert np.abs(o.p - ref).max() <= 1e-12 * np.abs(ref - p0).max()
        assert np.allclose(o.q, [0, 0, 0, 1], atol=1e-15)


def test_free_fall_bonded_lattice():
    """A bonded lattice in free fall stays at rest in its own frame: the same closed form holds to the
    Newton tolerance."""
    sc = scenes.cube_lattice(nx=3, k_ground=0.0, newton_rel_tol=1e-9)
    o = oracle.OracleSim(sc)
    p0, dt = sc.pos.copy(), sc.config["dt"]
    for n in range(1, 6):
        st = o.step(1)[0][0]
        assert st["status"] == 0 and st["g_norm"] <= 1e-9 * st["g0_norm"]
        ref = p0 + G * dt * dt * n * (n + 1) / 2.0
        assert np.abs(o.p - ref).max() <= 1e-8 * np.abs(ref - p0).max()
        assert np.abs(np.abs(o.q[:, 3]) - 1.0).max() < 1e-12


def test_two_particle_axial_recurrence():
    """Two free particles joined along x, released with axial stretch delta: only the stretch term acts and
    u = l - l0 obeys (1 + w^2 dt^2) u_{n+1} - 2 u_n + u_{n-1} = 0 with w^2 = 2 kn / m."""
    l0, r, E, nu, rho, dt = 0.01, 0.005, 1e7, 0.3, 2500.0, 2e-4
    pos = np.array([[0.0, 0.0, 0.0], [l0, 0.0, 0.0]])
    cfg = scenes.default_config(dt=dt, gravity=(0.0, 0.0, 0.0), k_ground=0.0, newton_rel_tol=1e-13)
    sc = scenes._assemble(pos, np.full(2, r), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.array([[0, 1]]),
                          [scenes.Material(E, nu, rho)], cfg, "axial")
    o = oracle.OracleSim(sc)
    delta = 1e-5
    o.p[1, 0] += delta
    m = rho * 4.0 / 3.0 * math.pi * r ** 3
    kn = E * math.pi * r * r / l0
    w2 = 2.0 * kn / m
    u_prev, u = delta, delta
    for n in range(30):
        o.step(1)
        u_next = (2.0 * u - u_prev) / (1.0 + w2 * dt * dt)
        u_prev, u = u, u_next
        got = o.p[1, 0] - o.p[0, 0] - l0
        assert abs(got - u) <= 1e-9 * delta, (n, got, u)
        assert abs(o.p[0, 1]) < 1e-20 and abs(o.p[1, 2]) < 1e-20
    # centre of mass at rest (linear momentum zero)
    assert abs(o.v[:, 0].sum()) < 1e-9 * delta / dt


def spun_cube(nx=3, seed=5, gravity=(0.0, 0.0, 0.0), k_ground=0.0, z=0.2, tol=1e-10, dt=1e-3, **kw):
    sc = scenes.cube_lattice(nx=nx, z_bottom=z, k_ground=k_ground, gravity=gravity, newton_rel_tol=tol, dt=dt, **kw)
    rng = np.random.default_rng(seed)
    n = sc.n
    c = sc.pos.mean(0)
    w = np.array([3.0, -2.0, 5.0])
    sc.vel[:] = np.cross(w, sc.pos - c) + rng.normal(size=(n, 3)) * 0.05 + np.array([0.1, 0.0, -0.3])
    # quaternion velocity of a common spin w: qdot = 1/2 (w, 0) q
    sc.quat_vel[:] = 0.5 * np.array([w[0], w[1], w[2], 0.0])
    return sc


def test_monotone_objective_over_newton_iterations():
    """The line search only accepts Phi(x') <= Phi(x), so Phi is non-increasing over Newton iterations."""
    sc = spun_cube(gravity=(0.0, 0.0, -9.81), k_ground=1e6, z=0.004, tol=1e-12)
    dt = sc.config["dt"]
    phat = sc.pos + dt * sc.vel
    qhat = sc.quat + dt * sc.quat_vel
    phis = []
    for k in range(1, 7):
        o = oracle.OracleSim(sc, dict(newton_max_iter=k))
        st = o.step(1)[0][0]
        phis.append(o.system(o.p, o.q, phat, qhat)["phi"])
    x0q = qhat / np.linalg.norm(qhat, axis=1, keepdims=True)
    phi0 = oracle.OracleSim(sc).system(phat, x0q, phat, qhat)["phi"]
    seq = [phi0] + phis
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(seq, seq[1:])), seq
    assert seq[-1] < seq[0]


def test_linear_momentum_conserved_without_external_forces():
    sc = spun_cube(tol=1e-9)
    o = oracle.OracleSim(sc)
    P0 = (o.mass[:, None] * o.v).sum(0)
    scale = (o.mass * np.linalg.norm(o.v, axis=1)).sum()
    for _ in range(20):
        st = o.step(1)[0][0]
        assert st["status"] == 0
    P = (o.mass[:, None] * o.v).sum(0)
    assert np.abs(P - P0).max() <= 1e-8 * scale
    assert np.abs(np.linalg.norm(o.q, axis=1) - 1.0).max() <= 1e-14


def angular_momentum(o):
    L = (o.mass[:, None] * np.cross(o.p, o.v)).sum(0)
    J = 0.4 * o.mass * o.radius ** 2
    for i in range(o.p.shape[0]):
        qc = np.array([-o.q[i, 0], -o.q[i, 1], -o.q[i, 2], o.q[i, 3]])
        w = 2.0 * oracle.qmul(o.u[i], qc)[:3]
        L += J[i] * w
    return L


def test_angular_momentum_conserved_without_external_forces():
    """No gravity or contact: total angular momentum (orbital m p x v plus spin J w, w = 2 vec(qdot conj q),
    J = 2/5 m r^2) stays within 1e-5 of its value for a spinning, vibrating bonded cube, at two time steps."""
    for dt in (4e-4, 2e-4):
        sc = spun_cube(tol=1e-9, dt=dt)
        o = oracle.OracleSim(sc)
        o.step(1)
        L0 = angular_momentum(o)
        for _ in range(10):
            o.step(1)
            assert np.linalg.norm(angular_momentum(o) - L0) <= 1e-5 * np.linalg.norm(L0)


def deformed_small_system(seed=7, k_self=1e5):
    sc = scenes.cube_lattice(nx=2, spacing=0.0098, r=0.005, k_ground=1e6, z_bottom=0.0045, k_self=k_self,
                             contact_skin=0.005)
    rng = np.random.default_rng(seed)
    o = oracle.OracleSim(sc)
    p = sc.pos + rng.normal(size=sc.pos.shape) * 3e-4
    from scipy.spatial.transform import Rotation
    q = Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * 0.2).as_quat()
    phat = sc.pos + rng.normal(size=sc.pos.shape) * 1e-4
    qhat = q + rng.normal(size=q.shape) * 0.01
    return o, p, q, phat, qhat


def dense_hessian(o, p, q, phat, qhat):
    n6 = 6 * p.shape[0]
    H = np.zeros((n6, n6))
    for c in range(n6):
        e = np.zeros(n6)
        e[c] = 1.0
        H[:, c] = o.matvec(p, q, phat, qhat, e.reshape(-1, 6)).ravel()
    return H


def test_assembled_hessian_is_symmetric_psd_and_matches_blocks():
    o, p, q, phat, qhat = deformed_small_system()
    H = dense_hessian(o, p, q, phat, qhat)
    sysd = o.system(p, q, phat, qhat)
    assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > -1e-10 * np.abs(H).max()
    # the diagonal 6x6 blocks are the assembled preconditioner blocks
    for i in range(p.shape[0]):
        assert np.allclose(H[6 * i:6 * i + 6, 6 * i:6 * i + 6], sysd["diag"][i], atol=1e-12 * np.abs(H).max())
    # off-diagonal blocks of bonded pairs are the bonds' (i, j) sub-blocks
    for k, b in enumerate(sysd["bond_ids"]):
        i, j = o.bi[b], o.bj[b]
        blk = H[6 * i:6 * i + 6, 6 * j:6 * j + 6]
        assert np.allclose(blk, sysd["bondH"][k][:6, 6:], atol=1e-12 * np.abs(H).max())


def test_pcg_matches_dense_solve():
    """Sec. 5.3 PCG driven to a tiny relative residual equals a dense Cholesky solve of the same system."""
    o, p, q, phat, qhat = deformed_small_system()
    H = dense_hessian(o, p, q, phat, qhat)
    b = np.random.default_rng(3).normal(size=H.shape[0])
    x, it = o.pcg_solve(p, q, phat, qhat, b.reshape(-1, 6), 1e-14, 500)
    L = np.linalg.cholesky(H)
    ref = np.linalg.solve(L.T, np.linalg.solve(L, b))
    assert np.allclose(x.ravel(), ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    x2, it2 = o.pcg_solve(p, q, phat, qhat, b.reshape(-1, 6), 0.5, 500)
    r = b - H @ x2.ravel()
    assert np.linalg.norm(r) <= 0.5 * np.linalg.norm(b) and it2 <= it


def test_gradient_matches_objective_differences():
    """The assembled reduced gradient is d/dxi of Phi(R_x(xi)) at 0 (whole system, inertia + gravity +
    ground + bonds + contacts)."""
    o, p, q, phat, qhat = deformed_small_system()
    sysd = o.system(p, q, phat, qhat)
    n = p.shape[0]

    def phi(xi):
        pp, qq = np.zeros_like(p), np.zeros_like(q)
        for i in range(n):
            pp[i], qq[i] = oracle.retract(p[i], q[i], xi[i])
        return o.system(pp, qq, phat, qhat)["phi"]

    rng = np.random.default_rng(4)
    for _ in range(4):
        d = rng.normal(size=(n, 6)) * np.array([1e-4] * 3 + [1e-2] * 3)
        h = 1e-3
        fd = (-phi(2 * h * d) + 8 * phi(h * d) - 8 * phi(-h * d) + phi(-2 * h * d)) / (12 * h)
        an = (sysd["g"] * d).sum()
        assert abs(fd - an) <= 1e-6 * (np.abs(sysd["g"] * d).sum() + 1e-30), (fd, an)


def test_contact_candidates_grid_equals_brute_force():
    rng = np.random.default_rng(8)
    pos = rng.uniform(0, 0.05, (300, 3))
    pairs = scenes._pairs_within(pos, 0.006)[::3]
    cfg = scenes.default_config(k_self=1e5, contact_skin=0.002)
    sc = scenes._assemble(pos, rng.uniform(0.001, 0.003, 300), np.zeros(300, np.int32), np.zeros(300, np.uint8),
                          pairs, [scenes.Material(1e7, 0.3, 2500.0)], cfg, "cloud")
    o = oracle.OracleSim(sc)
    a = o.contact_candidates(o.p, brute=False)
    b = o.contact_candidates(o.p, brute=True)
    assert a.shape[0] > 50 and np.array_equal(a, b)
    bonded = set(map(tuple, pairs.tolist()))
    assert not any(tuple(x) in bonded for x in a.tolist())


def test_self_contact_energy_and_force():
    """Sec. 5.4: V_self = 1/2 k_ec (|p_i - p_j| - r_i - r_j)^2 when overlapping, zero otherwise."""
    r, k, delta = 0.005, 2e5, 4e-4
    pos = np.array([[0.0, 0.0, 1.0], [2 * r - delta, 0.0, 1.0]])
    cfg = scenes.default_config(gravity=(0.0, 0.0, 0.0), k_self=k, contact_skin=r)
    sc = scenes._assemble(pos, np.full(2, r), np.zeros(2, np.int32), np.zeros(2, np.uint8), np.zeros((0, 2), np.int64),
                          [scenes.Material(1e7, 0.3, 2500.0)], cfg, "touch")
    o = oracle.OracleSim(sc)
    s = o.system(o.p, o.q, o.p, o.q)
    assert s["n_candidates"] == 1
    assert np.isclose(s["phi"], 0.5 * k * delta ** 2, rtol=1e-10)
    assert np.allclose(s["g"][0, :3], [k * delta, 0, 0], rtol=1e-10) and np.allclose(s["g"][1, :3], [-k * delta, 0, 0], rtol=1e-10)
    o.p[1, 0] = 2 * r + 1e-4
    s = o.system(o.p, o.q, o.p, o.q)
    assert s["n_candidates"] == 1 and s["phi"] == 0.0 and np.abs(s["g"]).max() == 0.0


def test_ground_contact_rest_state():
    """A single sphere settles on the ground at the penalty equilibrium p_z = z0 + r - m |g| / k_c."""
    r, k = 0.005, 1e4
    pos = np.array([[0.0, 0.0, r + 0.001]])
    cfg = scenes.default_config(dt=1e-3, k_ground=k, newton_rel_tol=1e-12)
    sc = scenes._assemble(pos, np.full(1, r), np.zeros(1, np.int32), np.zeros(1, np.uint8), np.zeros((0, 2), np.int64),
                          [scenes.Material(1e7, 0.3, 2500.0)], cfg, "rest")
    o = oracle.OracleSim(sc)
    o.step(400)
    m = 2500.0 * 4.0 / 3.0 * math.pi * r ** 3
    assert abs(o.p[0, 2] - (r - m * 9.81 / k)) < 1e-9


def test_kinematic_particles_and_strain_fracture():
    """Kinematic particles follow their velocity exactly; a bond breaks at the first converged step whose tensile
    strain (|p_j - p_i| - l0)/l0 strictly exceeds its limit, every intact bond tested at once on the step's converged
    state (Alg. 3, bond update). The two end particles of a 3-particle chain move apart at v each, so by symmetry
    each bond's strain is v dt n / l0 = 0.05 n at step n: with limit 0.27 both bonds break together at n = 6
    (0.30 > 0.27 while 0.25 at n = 5 is below), and not one step earlier or later."""
    l0, v, dt, lim = 0.01, 0.5, 1e-3, 0.27
    pos = np.array([[0.0, 0.0, 0.0], [l0, 0.0, 0.0], [2 * l0, 0.0, 0.0]])
    cfg = scenes.default_config(dt=dt, gravity=(0.0, 0.0, 0.0), newton_rel_tol=1e-10)
    sc = scenes._assemble(pos, np.full(3, 0.005), np.zeros(3, np.int32), np.array([1, 0, 1], np.uint8),
                          np.array([[0, 1], [1, 2]]), [scenes.Material(1e7, 0.3, 2500.0, lim)], cfg, "pull")
    sc.vel[0, 0], sc.vel[2, 0] = -v, v
    o = oracle.OracleSim(sc)
    broke_at = None
    for n in range(1, 9):
        was = o.broken.copy()
        st = o.step(1)[0][0]
        assert np.isclose(o.p[0, 0], -v * dt * n, rtol=0, atol=1e-15) and np.isclose(o.p[2, 0], 2 * l0 + v * dt * n, atol=1e-15)
        strain = np.array([(np.linalg.norm(o.p[o.bj[b]] - o.p[o.bi[b]]) - l0) / l0 for b in range(2)])
        if not was.any():
            assert np.allclose(strain, v * dt * n / l0, rtol=0, atol=1e-9)  # the closed form before the break
            # broken exactly where the converged state's strain is above the limit, nowhere else
            assert np.array_equal(o.broken.astype(bool), strain > lim)
            assert st["bonds_broken"] == int((strain > lim).sum())
        if st["bonds_broken"] and broke_at is None:
            broke_at = n
    assert broke_at == 6 and o.broken.sum() == 2


def test_fracture_tests_each_bond_against_its_own_limit():
    """Bonds of different limits in the same stretched chain: only the weaker one breaks, at the first step its
    strain is above its own limit; the stronger one, at the same strain, stays intact."""
    l0, v, dt = 0.01, 0.5, 1e-3
    pos = np.array([[0.0, 0.0, 0.0], [l0, 0.0, 0.0], [2 * l0, 0.0, 0.0]])
    cfg = scenes.default_config(dt=dt, gravity=(0.0, 0.0, 0.0), newton_rel_tol=1e-10)
    mats = [scenes.Material(1e7, 0.3, 2500.0, 0.17), scenes.Material(1e7, 0.3, 2500.0, 0.5)]
    sc = scenes._assemble(pos, np.full(3, 0.005), np.zeros(3, np.int32), np.array([1, 0, 1], np.uint8),
                          np.array([[0, 1], [1, 2]]), mats, cfg, "pull2", bond_mat=np.array([0, 1], np.int32))
    sc.vel[0, 0], sc.vel[2, 0] = -v, v
    o = oracle.OracleSim(sc)
    for n in range(1, 5):
        st = o.step(1)[0][0]
        if n < 4:  # strains 0.05 n <= 0.15 < 0.17
            assert st["bonds_broken"] == 0 and not o.broken.any()
    # n = 4: both strains 0.20 (the middle particle is still centred before the test): only bond 0 is above its limit
    assert o.broken.tolist() == [1, 0]


def test_literal_shear_gradient_noise_floor():
    """With the shear energy exactly as printed (shear_scale = 1, N/m) the transverse stiffness is ~1e5 times
    the stretch stiffness at 10 mm spacing, and FP64 rounding of positions 0.2 m from the origin alone puts the
    gradient's noise floor near 1e-6 of |g_0| in free fall: the Newton loop cannot certify 1e-6 there and ends
    with a line-search failure. The dimensionally consistent scaling converges."""
    lit = oracle.OracleSim(scenes.cube_lattice(nx=3, k_ground=0.0, shear_scale=1.0, newton_rel_tol=1e-8))
    st = lit.step(1)[0][0]
    assert st["status"] == 5 and st["g_norm"] > 1e-8 * st["g0_norm"]
    ok = oracle.OracleSim(scenes.cube_lattice(nx=3, k_ground=0.0, newton_rel_tol=1e-8))
    st = ok.step(1)[0][0]
    assert st["status"] == 0


def test_newton_cap_reports_status():
    sc = spun_cube(gravity=(0.0, 0.0, -9.81), k_ground=1e6, z=0.004, tol=1e-14)
    o = oracle.OracleSim(sc, dict(newton_max_iter=1))
    st = o.step(1)[0][0]
    assert st["status"] == 4 and st["newton_iters"] == 1


def test_termwise_energy_difference_matches_plain_difference():
    """The line search's Phi(x') - Phi(x) (exact difference identities, term by term) equals the plain
    difference of the objective for steps large enough that the plain difference is accurate."""
    o, p, q, phat, qhat = deformed_small_system()
    rng = np.random.default_rng(11)
    n = p.shape[0]
    for scale in (1e-3, 1e-4):
        st = rng.normal(size=(n, 6)) * np.array([scale * 0.01] * 3 + [scale] * 3)
        p1, q1 = np.zeros_like(p), np.zeros_like(q)
        for i in range(n):
            p1[i], q1[i] = oracle.retract(p[i], q[i], st[i])
        d, phi0, phi1 = o.energy_diff(phat, qhat, p, q, p1, q1)
        assert abs(d - (phi1 - phi0)) <= 1e-9 * abs(phi1 - phi0) + 1e-13 * abs(phi0)
