"""Pins of the oracle's algebra against the paper's identities (App. A, App. C) and library routines.

Each test checks the oracle against something other than itself: scipy's rotation algebra, numpy's
symmetric eigensolver, sympy's symbolic derivatives, or an identity printed in the paper.
"""
import math

import numpy as np
import pytest

import oracle

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def rand_quats(n, seed=0, unit=True):
    q = np.random.default_rng(seed).normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True) if unit else q


def test_nullspace_identities():
    """App. A: G_l q = G_r q = 0; G_l^T G_l = |q|^2 I4 - q q^T; G_l G_l^T = |q|^2 I3 (also for G_r)."""
    for q in rand_quats(20, seed=1, unit=False):
        n2 = q @ q
        for G in (oracle.Gl(q), oracle.Gr(q)):
            assert np.allclose(G @ q, 0.0, atol=1e-14)
            assert np.allclose(G.T @ G, n2 * np.eye(4) - np.outer(q, q), atol=1e-13)
            assert np.allclose(G @ G.T, n2 * np.eye(3), atol=1e-13)


def test_multiplication_matrices_from_nullspace_operators():
    """App. A: Q_l(q) = [G_l(q)^T  q], Q_r(q) = [G_r(q)^T  q]."""
    for q in rand_quats(10, seed=2, unit=False):
        assert np.allclose(oracle.Ql(q), np.column_stack([oracle.Gl(q).T, q]), atol=0)
        assert np.allclose(oracle.Qr(q), np.column_stack([oracle.Gr(q).T, q]), atol=0)


def test_quaternion_product_matches_scipy_composition():
    """q_i q_j = Q_l(q_i) q_j = Q_r(q_j) q_i is the Hamilton product (composition of rotations)."""
    qs = rand_quats(20, seed=3)
    for a, b in zip(qs[:10], qs[10:]):
        ref = (Rotation.from_quat(a) * Rotation.from_quat(b)).as_quat()
        got = oracle.qmul(a, b)
        assert min(np.abs(got - ref).max(), np.abs(got + ref).max()) < 1e-14
        assert np.allclose(oracle.Ql(a) @ b, got, atol=1e-15)
        assert np.allclose(oracle.Qr(b) @ a, got, atol=1e-15)


def test_rotation_operator_matches_scipy():
    """(d, 0) = q (d0, 0) conj(q) is the active rotation of d0 by q."""
    qs = rand_quats(10, seed=4)
    d0s = np.random.default_rng(5).normal(size=(10, 3))
    for q, d0 in zip(qs, d0s):
        assert np.allclose(oracle.rotate(q, d0), Rotation.from_quat(q).apply(d0), atol=1e-14)


def test_conjugate_product_is_identity():
    """App. A: conj(q) q = {0, 0, 0, 1} for a unit quaternion."""
    for q in rand_quats(10, seed=6):
        qc = np.array([-q[0], -q[1], -q[2], q[3]])
        assert np.allclose(oracle.qmul(qc, q), [0, 0, 0, 1], atol=1e-15)


def test_extended_mass_matrix_identity():
    """App. C: for a sphere (J = 2/5 m r^2 I3) and unit q, 4 G^T J G + 2 tr(J) q q^T = 8/5 m r^2 (I4 + q q^T / 2).
    (The printed 'G J G^T' has mismatched shapes; the 4x4 reading G^T J G is used.)"""
    m, r = 0.7, 0.013
    Jc = 0.4 * m * r * r
    for q in rand_quats(5, seed=7):
        G = oracle.Gl(q)
        Mq = 4.0 * G.T @ (Jc * np.eye(3)) @ G + 2.0 * (3 * Jc) * np.outer(q, q)
        ref = 1.6 * m * r * r * (np.eye(4) + 0.5 * np.outer(q, q))
        assert np.allclose(Mq, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_angular_velocity_relation():
    """App. A: w4 = 2 qdot conj(q) for q(t) rotating at constant world angular velocity w."""
    w = np.array([0.3, -1.1, 0.7])
    q0 = rand_quats(1, seed=8)[0]
    q = lambda t: (Rotation.from_rotvec(w * t) * Rotation.from_quat(q0)).as_quat()
    t, h = 0.4, 1e-6
    qa, qb, qm = q(t + h), q(t - h), q(t)
    if qa @ qm < 0:
        qa = -qa
    if qb @ qm < 0:
        qb = -qb
    qdot = (qa - qb) / (2 * h)
    w4 = 2.0 * oracle.qmul(qdot, np.array([-qm[0], -qm[1], -qm[2], qm[3]]))
    assert np.allclose(w4, [*w, 0.0], atol=1e-8)


def test_retraction_is_right_composition_with_exponential():
    """Eq. manifold-update-2 with dq = G_l(q)^T y: q' = q (y/|y| sin|y|, cos|y|), i.e. a body-frame
    rotation by 2|alpha y| about y; p' = p + alpha dp; |q'| = 1."""
    rng = np.random.default_rng(9)
    for k in range(10):
        p, q = rng.normal(size=3), rand_quats(1, seed=10 + k)[0]
        st = rng.normal(size=6) * (0.3 if k % 2 else 1e-7)
        alpha = [1.0, 0.5, 0.25][k % 3]
        po, qo = oracle.retract(p, q, st, alpha)
        assert np.allclose(po, p + alpha * st[:3], atol=1e-15)
        assert abs(np.linalg.norm(qo) - 1.0) <= 1e-14
        ref = (Rotation.from_quat(q) * Rotation.from_rotvec(2.0 * alpha * st[3:])).as_quat()
        assert min(np.abs(qo - ref).max(), np.abs(qo + ref).max()) < 1e-13
    # first order: d q'/d alpha at 0 equals G_l(q)^T y
    q = rand_quats(1, seed=30)[0]
    y = np.array([0.2, -0.1, 0.4])
    st = np.concatenate([np.zeros(3), y])
    h = 1e-6
    d = (oracle.retract(np.zeros(3), q, st, h)[1] - oracle.retract(np.zeros(3), q, st, -h)[1]) / (2 * h)
    assert np.allclose(d, oracle.Gl(q).T @ y, atol=1e-9)


def test_jacobi_eigensolver_matches_numpy():
    rng = np.random.default_rng(11)
    for n in (3, 6, 9, 12):
        A = rng.normal(size=(n, n))
        A = A + A.T
        lam, V = oracle.eig_sym(A)
        assert np.allclose(np.sort(lam), np.linalg.eigvalsh(A), atol=1e-12 * np.abs(A).max())
        assert np.allclose(V @ np.diag(lam) @ V.T, A, atol=1e-12 * np.abs(A).max())
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)


def test_eig_clamp_matches_reconstruction():
    """Sec. 5.2 projection: negative eigenvalues set to zero, V max(L, 0) V^T."""
    rng = np.random.default_rng(12)
    for n in (6, 12):
        for scale in (1.0, 1e6):
            A = rng.normal(size=(n, n)) * scale
            A = A + A.T
            lam, V = np.linalg.eigh(A)
            ref = V @ np.diag(np.maximum(lam, 0.0)) @ V.T
            got = oracle.eig_clamp(A)
            assert np.allclose(got, ref, atol=1e-12 * np.abs(A).max())
            assert np.linalg.eigvalsh(got).min() > -1e-11 * np.abs(A).max()
            assert np.allclose(oracle.eig_clamp(got), got, atol=1e-12 * np.abs(A).max())
    B = rng.normal(size=(12, 12))
    B = B @ B.T
    assert np.allclose(oracle.eig_clamp(B), B, atol=1e-12 * np.abs(B).max())
    # a degenerate case: the zero matrix and a rank-one negative matrix
    assert np.allclose(oracle.eig_clamp(np.zeros((6, 6))), 0.0)
    v = rng.normal(size=6)
    assert np.allclose(oracle.eig_clamp(-np.outer(v, v)), 0.0, atol=1e-12 * (v @ v))


def test_jets_match_symbolic_derivatives():
    """The oracle's second-order forward-mode arithmetic against sympy's exact derivatives."""
    sp = pytest.importorskip("sympy")
    xs = sp.symbols("x0:4")
    f = sp.sin(xs[0] * xs[1]) + sp.sqrt(xs[2]) / (1 + xs[0] ** 2) + sp.acos(xs[3]) ** 2
    grad = [sp.diff(f, v) for v in xs]
    hess = [[sp.diff(f, a, b) for b in xs] for a in xs]
    for x in ([0.3, 0.7, 1.3, 0.2], [1.1, -0.4, 0.05, 0.999], [-0.6, 2.0, 3.0, 0.9999999]):
        sub = {v: sp.Float(repr(c), 50) for v, c in zip(xs, x)}  # evaluate in 50-digit arithmetic
        ev = lambda e: float(e.evalf(40, subs=sub))
        fv, g, H = oracle.jet_selftest(np.array(x))
        assert abs(fv - ev(f)) < 1e-14
        assert np.allclose(g, [ev(e) for e in grad], rtol=1e-12, atol=1e-13)
        assert np.allclose(H, [[ev(e) for e in row] for row in hess], rtol=1e-9, atol=1e-10)
