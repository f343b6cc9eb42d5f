/*
 * bdem_oracle.c -- CPU oracle for one implicit bonded-DEM time step. TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of the paper's method, written to be checked by eye
 * against it. Only tests/, the smoke check and the benchmark's cpu_baseline / reference legs may load
 * it; the CUDA library never does, and the two share no code.
 *
 *  - Objective (Sec. 3.1, Eq. optimization form):
 *      Phi(x) = 1/(2 dt^2) (x - xhat)^T M_s (x - xhat) + V(x),  M_s = diag(m I3, 8/5 m r^2 I4),
 *      xhat = 2 x_n - x_{n-1} = x_n + dt v_n.
 *  - Potential V (Sec. 3.2): stretch 1/2 kn (|p_i - p_j| - l0)^2, shear 1/2 kt theta^2,
 *    bend-twist 1/2 t^T K t with t = R0 G_l(q_j) q_i; gravity -m g.p; penalty contact (Sec. 5.4).
 *  - Derivatives: second-order forward-mode arithmetic ("jets") over the Euclidean coordinates
 *    (p_i, q_i, p_j, q_j) in R^14, then the Riemannian gradient of Sec. 4.1, the Riemannian Hessian of
 *    Eq. manifold-hessian-1..4 and the nullspace reduction G H G^T y = z, z = G b of Sec. 4.2.
 *  - Semi-positive-definite projection (Sec. 5.2): per-term eigenvalue clamp by cyclic Jacobi.
 *  - PCG with block-Jacobi preconditioner and relative tolerance eps_r = min(0.5, sqrt|grad f|) (Sec. 5.3).
 *  - Line search along the retraction of Eq. manifold-update-1/2, then normalisation (Sec. 4.1).
 *  - Alg. 3: prediction, Newton loop, velocity update, bond state update (strain fracture).
 *
 * Readings of points the paper leaves open (the shear angle, R0, d0, double cover, stopping rules,
 * line-search rule, contact activation, fracture by strain) are stated where they are used.
 */
#include "bdem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------------ */
/* Quaternion algebra, App. A. q = {u, v, w, s}.                                                     */
/* ------------------------------------------------------------------------------------------------ */

/* Left multiplication matrix: q_i q_j = Q_l(q_i) q_j, Q_l = [[s I + t^x, t], [-t^T, s]]. */
void orc_Ql(const double q[4], double M[16]) {
  double u = q[0], v = q[1], w = q[2], s = q[3];
  double m[16] = {s, -w, v, u,  w, s, -u, v,  -v, u, s, w,  -u, -v, -w, s};
  memcpy(M, m, sizeof m);
}

/* Right multiplication matrix: q_i q_j = Q_r(q_j) q_i, Q_r = [[s I - t^x, t], [-t^T, s]]. */
void orc_Qr(const double q[4], double M[16]) {
  double u = q[0], v = q[1], w = q[2], s = q[3];
  double m[16] = {s, w, -v, u,  -w, s, u, v,  v, -u, s, w,  -u, -v, -w, s};
  memcpy(M, m, sizeof m);
}

/* Nullspace operators G_l = [s I - t^x, -t], G_r = [s I + t^x, -t] (3x4, row-major). */
void orc_Gl(const double q[4], double M[12]) {
  double u = q[0], v = q[1], w = q[2], s = q[3];
  double m[12] = {s, w, -v, -u,  -w, s, u, -v,  v, -u, s, -w};
  memcpy(M, m, sizeof m);
}

void orc_Gr(const double q[4], double M[12]) {
  double u = q[0], v = q[1], w = q[2], s = q[3];
  double m[12] = {s, -w, v, -u,  w, s, -u, -v,  -v, u, s, -w};
  memcpy(M, m, sizeof m);
}

void orc_qmul(const double a[4], const double b[4], double out[4]) {
  double M[16];
  orc_Ql(a, M);
  for (int r = 0; r < 4; ++r) out[r] = M[4 * r] * b[0] + M[4 * r + 1] * b[1] + M[4 * r + 2] * b[2] + M[4 * r + 3] * b[3];
}

/* Direction rotation operator: (d, 0) = q (d0, 0) conj(q). */
void orc_rotate(const double q[4], const double d0[3], double d[3]) {
  double a[4], qc[4] = {-q[0], -q[1], -q[2], q[3]}, x[4] = {d0[0], d0[1], d0[2], 0.0}, r[4];
  orc_qmul(q, x, a);
  orc_qmul(a, qc, r);
  d[0] = r[0]; d[1] = r[1]; d[2] = r[2];
}

/* ------------------------------------------------------------------------------------------------ */
/* Jets: value, gradient and (packed symmetric) Hessian with respect to NV variables.                 */
/* The variables of a pair term are (p_a[3], q_a[4], p_b[3], q_b[4]).                                */
/* ------------------------------------------------------------------------------------------------ */

#define NV 14
#define NH (NV * (NV + 1) / 2)
typedef struct { double v; double g[NV]; double h[NH]; } jet;

static int g_order = 2; /* 0: values only; 2: values, gradients and Hessians */

static int hidx(int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  return a * NV - a * (a - 1) / 2 + (b - a);
}

static jet jc(double c) {
  jet r;
  r.v = c;
  if (g_order) { memset(r.g, 0, sizeof r.g); memset(r.h, 0, sizeof r.h); }
  return r;
}

static jet jvar(double x, int k) {
  jet r = jc(x);
  if (g_order) r.g[k] = 1.0;
  return r;
}

static jet jadd(jet a, jet b) {
  jet r; r.v = a.v + b.v;
  if (g_order) {
    for (int k = 0; k < NV; ++k) r.g[k] = a.g[k] + b.g[k];
    for (int k = 0; k < NH; ++k) r.h[k] = a.h[k] + b.h[k];
  }
  return r;
}

static jet jsub(jet a, jet b) {
  jet r; r.v = a.v - b.v;
  if (g_order) {
    for (int k = 0; k < NV; ++k) r.g[k] = a.g[k] - b.g[k];
    for (int k = 0; k < NH; ++k) r.h[k] = a.h[k] - b.h[k];
  }
  return r;
}

static jet jscale(jet a, double s) {
  jet r; r.v = s * a.v;
  if (g_order) {
    for (int k = 0; k < NV; ++k) r.g[k] = s * a.g[k];
    for (int k = 0; k < NH; ++k) r.h[k] = s * a.h[k];
  }
  return r;
}

static jet jaddc(jet a, double c) { a.v += c; return a; }

/* product rule: (ab)'' = a b'' + b a'' + a' b'^T + b' a'^T */
static jet jmul(jet a, jet b) {
  jet r; r.v = a.v * b.v;
  if (g_order) {
    for (int k = 0; k < NV; ++k) r.g[k] = a.v * b.g[k] + b.v * a.g[k];
    int k = 0;
    for (int i = 0; i < NV; ++i)
      for (int j = i; j < NV; ++j, ++k) r.h[k] = a.v * b.h[k] + b.v * a.h[k] + a.g[i] * b.g[j] + a.g[j] * b.g[i];
  }
  return r;
}

/* chain rule for a scalar function with value f0, first derivative f1 and second derivative f2 */
static jet jfun(jet a, double f0, double f1, double f2) {
  jet r; r.v = f0;
  if (g_order) {
    for (int k = 0; k < NV; ++k) r.g[k] = f1 * a.g[k];
    int k = 0;
    for (int i = 0; i < NV; ++i)
      for (int j = i; j < NV; ++j, ++k) r.h[k] = f1 * a.h[k] + f2 * a.g[i] * a.g[j];
  }
  return r;
}

static jet jrecip(jet a) { double x = a.v; return jfun(a, 1.0 / x, -1.0 / (x * x), 2.0 / (x * x * x)); }
static jet jsqrt(jet a) { double s = sqrt(a.v); return jfun(a, s, 0.5 / s, -0.25 / (s * a.v)); }
static jet jsin(jet a) { return jfun(a, sin(a.v), cos(a.v), -sin(a.v)); }

/* f(c) = theta^2 with c = cos(theta); theta is taken from atan2(sin, cos) for accuracy at small angles.
 * f'(c) = -2 theta / sin(theta), f''(c) = 2 (sin(theta) - theta cos(theta)) / sin(theta)^3, with their
 * Taylor series below 1e-3 (limits -2 and 2/3). */
static jet jangle2(jet c, double sin_theta) {
  double th = atan2(sin_theta, c.v), f1, f2;
  if (th < 1e-3) {
    double t2 = th * th;
    f1 = -2.0 - t2 / 3.0 - 7.0 * t2 * t2 / 180.0;
    f2 = 2.0 / 3.0 + 4.0 * t2 / 15.0;
  } else {
    double s = sin(th), co = cos(th);
    f1 = -2.0 * th / s;
    f2 = 2.0 * (s - th * co) / (s * s * s);
  }
  return jfun(c, th * th, f1, f2);
}

static void jet_grad_hess(const jet* f, double* g, double* H /* NV x NV */) {
  for (int i = 0; i < NV; ++i) g[i] = f->g[i];
  for (int i = 0; i < NV; ++i)
    for (int j = 0; j < NV; ++j) H[i * NV + j] = f->h[hidx(i, j)];
}

void orc_jet_selftest(const double x[4], double* f, double g[4], double H[16]) {
  g_order = 2;
  jet a = jvar(x[0], 0), b = jvar(x[1], 1), c = jvar(x[2], 2), d = jvar(x[3], 3);
  jet t1 = jsin(jmul(a, b));
  jet t2 = jmul(jsqrt(c), jrecip(jaddc(jmul(a, a), 1.0)));
  double s = sqrt(fmax(0.0, (1.0 - x[3]) * (1.0 + x[3])));
  jet t3 = jangle2(d, s);
  jet r = jadd(jadd(t1, t2), t3);
  *f = r.v;
  for (int i = 0; i < 4; ++i) {
    g[i] = r.g[i];
    for (int j = 0; j < 4; ++j) H[4 * i + j] = r.h[hidx(i, j)];
  }
}

/* ------------------------------------------------------------------------------------------------ */
/* Dense helpers                                                                                     */
/* ------------------------------------------------------------------------------------------------ */

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double dot4(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3]; }

/* C (m x n) = A (m x k) B (k x n) */
static void matmul(int m, int k, int n, const double* A, const double* B, double* C) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * n + j];
      C[i * n + j] = s;
    }
}

static void transpose(int m, int n, const double* A, double* At) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) At[j * m + i] = A[i * n + j];
}

/* ------------------------------------------------------------------------------------------------ */
/* Symmetric eigen-decomposition by the cyclic Jacobi method and the eigenvalue clamp (Sec. 5.2).     */
/* ------------------------------------------------------------------------------------------------ */

void orc_eig_sym(int n, const double* A0, double* evals, double* V) {
  double A[144];
  memcpy(A, A0, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off += A[i * n + j] * A[i * n + j];
    if (sqrt(off) <= 1e-15 * fro || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        /* rotation that annihilates A[p][q] (symmetric Schur 2x2) */
        double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) { /* A <- A J */
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* A <- J^T A */
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) { /* V <- V J */
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) evals[i] = A[i * n + i];
}

void orc_eig_clamp(int n, double* A) {
  double lam[12], V[144];
  orc_eig_sym(n, A, lam, V);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        if (lam[k] > 0.0) s += V[i * n + k] * lam[k] * V[j * n + k];
      A[i * n + j] = s;
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Riemannian gradient / Hessian on (R^3 x S^3)^m and the nullspace reduction (Sec. 4.1, 4.2).        */
/* Input: Euclidean gradient ge[7m] and Hessian He[7m x 7m] in the order (p_1, q_1, ..., p_m, q_m).   */
/* Output: reduced gradient gr[6m] and Hessian Hr[6m x 6m] in the order (dp_1, y_1, ..., dp_m, y_m).  */
/* ------------------------------------------------------------------------------------------------ */

static void riemann_reduce(int m, const double* const* qe, const double* ge, const double* He, double* gr, double* Hr) {
  int ne = 7 * m, nr = 6 * m;
  double P[2][16], gR[14], HR[196], T[12 * 14], tmp[12 * 14], Tt[14 * 12];
  for (int e = 0; e < m; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) P[e][4 * a + b] = (a == b ? 1.0 : 0.0) - qe[e][a] * qe[e][b];
  /* Riemannian gradient: grad_p f = grad_p fbar, grad_q f = (I - q q^T) grad_q fbar */
  for (int e = 0; e < m; ++e) {
    for (int a = 0; a < 3; ++a) gR[7 * e + a] = ge[7 * e + a];
    for (int a = 0; a < 4; ++a) {
      double s = 0.0;
      for (int b = 0; b < 4; ++b) s += P[e][4 * a + b] * ge[7 * e + 3 + b];
      gR[7 * e + 3 + a] = s;
    }
  }
  /* Riemannian Hessian, Eq. manifold-hessian-1..4 */
  for (int e = 0; e < m; ++e)
    for (int f = 0; f < m; ++f) {
      for (int a = 0; a < 7; ++a)
        for (int b = 0; b < 7; ++b) {
          int ia = a < 3 ? -1 : a - 3, ib = b < 3 ? -1 : b - 3;
          double h;
          if (ia < 0 && ib < 0) { /* p-p */
            h = He[(7 * e + a) * ne + 7 * f + b];
          } else if (ia < 0) { /* p-q: Hbar_pq (I - q_f q_f^T) */
            h = 0.0;
            for (int c = 0; c < 4; ++c) h += He[(7 * e + a) * ne + 7 * f + 3 + c] * P[f][4 * c + ib];
          } else if (ib < 0) { /* q-p: (I - q_e q_e^T) Hbar_qp */
            h = 0.0;
            for (int c = 0; c < 4; ++c) h += P[e][4 * ia + c] * He[(7 * e + 3 + c) * ne + 7 * f + b];
          } else { /* q-q: P_e Hbar_qq P_f - delta_ef (q_e^T grad_qe fbar) P_e */
            h = 0.0;
            for (int c = 0; c < 4; ++c)
              for (int d = 0; d < 4; ++d) h += P[e][4 * ia + c] * He[(7 * e + 3 + c) * ne + 7 * f + 3 + d] * P[f][4 * d + ib];
            if (e == f) h -= dot4(qe[e], ge + 7 * e + 3) * P[e][4 * ia + ib];
          }
          HR[(7 * e + a) * ne + 7 * f + b] = h;
        }
    }
  /* reduction with T = blockdiag(I3, G_l(q_e)): z = T grad f, H_red = T Hess f T^T */
  memset(T, 0, sizeof(double) * nr * ne);
  for (int e = 0; e < m; ++e) {
    double G[12];
    orc_Gl(qe[e], G);
    for (int a = 0; a < 3; ++a) T[(6 * e + a) * ne + 7 * e + a] = 1.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 4; ++b) T[(6 * e + 3 + a) * ne + 7 * e + 3 + b] = G[4 * a + b];
  }
  matmul(nr, ne, 1, T, gR, gr);
  matmul(nr, ne, ne, T, HR, tmp);
  transpose(nr, ne, T, Tt);
  matmul(nr, ne, nr, tmp, Tt, Hr);
  /* symmetrise (the exact Riemannian Hessian is symmetric) */
  for (int i = 0; i < nr; ++i)
    for (int j = i + 1; j < nr; ++j) {
      double s = 0.5 * (Hr[i * nr + j] + Hr[j * nr + i]);
      Hr[i * nr + j] = Hr[j * nr + i] = s;
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Bond rest data (Sec. 3.2) with the readings:                                                     */
/*  - d0 is the rest bond direction expressed in the frame of the common rotation q_c, so that       */
/*    q_c (.) d0 equals the current bond direction at rest;                                          */
/*  - q0 is the shortest-arc rotation taking e_x to d0 (180 deg about e_z when d0 = -e_x) and        */
/*    R0 = G_l(q0) G_r(q0)^T, the inverse rotation, maps d0 to e_x (twist axis x);                  */
/*  - r0 = (r_i + r_j)/2, S = pi r0^2, I = pi r0^4/4, J = pi r0^4/2, G = E / (2 (1 + nu)).           */
/* ------------------------------------------------------------------------------------------------ */

static void common_rotation(const double qi[4], const double qj[4], double qc[4]) {
  /* q_c = (q_i + q_j)/|q_i + q_j|, taking -q_j when q_i.q_j < 0 (double cover) */
  double sg = dot4(qi, qj) < 0.0 ? -1.0 : 1.0, m[4], nm = 0.0;
  for (int k = 0; k < 4; ++k) { m[k] = qi[k] + sg * qj[k]; nm += m[k] * m[k]; }
  nm = sqrt(nm);
  for (int k = 0; k < 4; ++k) qc[k] = m[k] / nm;
}

int orc_bond_rest(orc_problem* P, const double* E, const double* nu, const double* bts, const double* shs,
                  const double* brk) {
  for (int b = 0; b < P->nb; ++b) {
    int i = P->bi[b], j = P->bj[b];
    const double *pi = P->p + 3 * i, *pj = P->p + 3 * j, *qi = P->q + 4 * i, *qj = P->q + 4 * j;
    double dx[3] = {pj[0] - pi[0], pj[1] - pi[1], pj[2] - pi[2]};
    double l0 = sqrt(dot3(dx, dx));
    double n0[3] = {dx[0] / l0, dx[1] / l0, dx[2] / l0};
    double qc[4], qcc[4], d0[3];
    common_rotation(qi, qj, qc);
    qcc[0] = -qc[0]; qcc[1] = -qc[1]; qcc[2] = -qc[2]; qcc[3] = qc[3];
    orc_rotate(qcc, n0, d0);
    double q0[4];
    if (1.0 + d0[0] > 1e-12) {
      double m[4] = {0.0, -d0[2], d0[1], 1.0 + d0[0]};
      double nm = sqrt(dot4(m, m));
      for (int k = 0; k < 4; ++k) q0[k] = m[k] / nm;
    } else {
      q0[0] = 0.0; q0[1] = 0.0; q0[2] = 1.0; q0[3] = 0.0;
    }
    double Gl0[12], Gr0[12], Grt[12];
    orc_Gl(q0, Gl0);
    orc_Gr(q0, Gr0);
    transpose(3, 4, Gr0, Grt);
    matmul(3, 4, 3, Gl0, Grt, P->R0 + 9 * b);
    double r0 = 0.5 * (P->radius[i] + P->radius[j]);
    double S = M_PI * r0 * r0, I = M_PI * pow(r0, 4) / 4.0, J = M_PI * pow(r0, 4) / 2.0;
    double G = E[b] / (2.0 * (1.0 + nu[b]));
    P->l0[b] = l0;
    P->d0[3 * b] = d0[0]; P->d0[3 * b + 1] = d0[1]; P->d0[3 * b + 2] = d0[2];
    P->kn[b] = E[b] * S / l0;
    P->kt[b] = G * S / l0;
    P->kbt[3 * b + 0] = bts[b] * G * J / l0;
    P->kbt[3 * b + 1] = bts[b] * E[b] * I / l0;
    P->kbt[3 * b + 2] = bts[b] * E[b] * I / l0;
    P->shear_scale[b] = shs[b];
    P->break_strain[b] = brk[b];
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------------ */
/* Bond energy in jets (Sec. 3.2).                                                                   */
/* Shear reading: theta is the angle between the rotated rest direction d = q_c (.) d0 and the       */
/* current bond direction n = (p_j - p_i)/|p_j - p_i| (the literal angle between d0 and d would      */
/* penalise rigid rotation); V_shear = 1/2 kt (shear_scale theta)^2.                                 */
/* ------------------------------------------------------------------------------------------------ */

static void jrotate(const jet q[4], const double d0[3], jet d[3]) {
  /* a = Q_l(q) (d0, 0), then (d, .) = Q_r(conj q) a */
  double x[4] = {d0[0], d0[1], d0[2], 0.0};
  /* Q_l(q) rows as linear forms in q: row r, column c coefficient of q components */
  jet a[4];
  /* Q_l = [[s, -w, v, u], [w, s, -u, v], [-v, u, s, w], [-u, -v, -w, s]] */
  const jet *u = &q[0], *v = &q[1], *w = &q[2], *s = &q[3];
  a[0] = jadd(jadd(jscale(*s, x[0]), jscale(*w, -x[1])), jadd(jscale(*v, x[2]), jscale(*u, x[3])));
  a[1] = jadd(jadd(jscale(*w, x[0]), jscale(*s, x[1])), jadd(jscale(*u, -x[2]), jscale(*v, x[3])));
  a[2] = jadd(jadd(jscale(*v, -x[0]), jscale(*u, x[1])), jadd(jscale(*s, x[2]), jscale(*w, x[3])));
  a[3] = jadd(jadd(jscale(*u, -x[0]), jscale(*v, -x[1])), jadd(jscale(*w, -x[2]), jscale(*s, x[3])));
  /* Q_r(b) = [[s, w, -v, u], [-w, s, u, v], [v, -u, s, w], [-u, -v, -w, s]] with b = conj q = (-u,-v,-w,s) */
  jet bu = jscale(*u, -1.0), bv = jscale(*v, -1.0), bw = jscale(*w, -1.0);
  d[0] = jadd(jadd(jmul(*s, a[0]), jmul(bw, a[1])), jadd(jmul(jscale(bv, -1.0), a[2]), jmul(bu, a[3])));
  d[1] = jadd(jadd(jmul(jscale(bw, -1.0), a[0]), jmul(*s, a[1])), jadd(jmul(bu, a[2]), jmul(bv, a[3])));
  d[2] = jadd(jadd(jmul(bv, a[0]), jmul(jscale(bu, -1.0), a[1])), jadd(jmul(*s, a[2]), jmul(bw, a[3])));
}

/* returns total energy; parts: stretch, shear, bend-twist */
static jet bond_energy_jet(const orc_problem* P, int b, const double pi[3], const double qi[4], const double pj[3],
                           const double qj[4], double parts[3], double* l_out, double t_out[3], jet part_jets[3]) {
  jet Pi[3], Qi[4], Pj[3], Qj[4];
  for (int k = 0; k < 3; ++k) { Pi[k] = jvar(pi[k], k); Pj[k] = jvar(pj[k], 7 + k); }
  for (int k = 0; k < 4; ++k) { Qi[k] = jvar(qi[k], 3 + k); Qj[k] = jvar(qj[k], 10 + k); }
  double l0 = P->l0[b], kn = P->kn[b], kt = P->kt[b], ss = P->shear_scale[b];
  const double* d0 = P->d0 + 3 * b;
  const double* R0 = P->R0 + 9 * b;
  const double* K = P->kbt + 3 * b;

  /* stretch: 1/2 kn (|p_i - p_j| - l0)^2 */
  jet dx[3];
  for (int k = 0; k < 3; ++k) dx[k] = jsub(Pj[k], Pi[k]);
  jet l = jsqrt(jadd(jadd(jmul(dx[0], dx[0]), jmul(dx[1], dx[1])), jmul(dx[2], dx[2])));
  jet e = jaddc(l, -l0);
  jet Vs = jscale(jmul(e, e), 0.5 * kn);

  /* shear: q_c = (q_i + q_j)/|q_i + q_j|, d = q_c (.) d0, n = (p_j - p_i)/|p_j - p_i| */
  double sg = dot4(qi, qj) < 0.0 ? -1.0 : 1.0;
  jet m[4];
  for (int k = 0; k < 4; ++k) m[k] = jadd(Qi[k], jscale(Qj[k], sg));
  jet inm = jrecip(jsqrt(jadd(jadd(jmul(m[0], m[0]), jmul(m[1], m[1])), jadd(jmul(m[2], m[2]), jmul(m[3], m[3])))));
  jet qc[4];
  for (int k = 0; k < 4; ++k) qc[k] = jmul(m[k], inm);
  jet d[3], n[3];
  jrotate(qc, d0, d);
  jet il = jrecip(l);
  for (int k = 0; k < 3; ++k) n[k] = jmul(dx[k], il);
  jet c = jadd(jadd(jmul(d[0], n[0]), jmul(d[1], n[1])), jmul(d[2], n[2]));
  double cr[3] = {d[1].v * n[2].v - d[2].v * n[1].v, d[2].v * n[0].v - d[0].v * n[2].v, d[0].v * n[1].v - d[1].v * n[0].v};
  jet th2 = jangle2(c, sqrt(dot3(cr, cr)));
  jet Vsh = jscale(th2, 0.5 * kt * ss * ss);

  /* bend-twist: t = R0 G_l(q_j) q_i, V = 1/2 t^T K t, K = diag(GJ, EI, EI)/l0 */
  /* G_l(q) = [[s, w, -v, -u], [-w, s, u, -v], [v, -u, s, -w]] */
  const jet *u = &Qj[0], *v = &Qj[1], *w = &Qj[2], *s = &Qj[3];
  jet wv[3];
  wv[0] = jadd(jadd(jmul(*s, Qi[0]), jmul(*w, Qi[1])), jsub(jmul(jscale(*v, -1.0), Qi[2]), jmul(*u, Qi[3])));
  wv[1] = jadd(jadd(jmul(jscale(*w, -1.0), Qi[0]), jmul(*s, Qi[1])), jsub(jmul(*u, Qi[2]), jmul(*v, Qi[3])));
  wv[2] = jadd(jadd(jmul(*v, Qi[0]), jmul(jscale(*u, -1.0), Qi[1])), jsub(jmul(*s, Qi[2]), jmul(*w, Qi[3])));
  jet t[3];
  for (int r = 0; r < 3; ++r) t[r] = jadd(jadd(jscale(wv[0], R0[3 * r]), jscale(wv[1], R0[3 * r + 1])), jscale(wv[2], R0[3 * r + 2]));
  jet Vbt = jscale(jadd(jadd(jscale(jmul(t[0], t[0]), K[0]), jscale(jmul(t[1], t[1]), K[1])), jscale(jmul(t[2], t[2]), K[2])), 0.5);

  if (parts) { parts[0] = Vs.v; parts[1] = Vsh.v; parts[2] = Vbt.v; }
  if (part_jets) { part_jets[0] = Vs; part_jets[1] = Vsh; part_jets[2] = Vbt; }
  if (l_out) *l_out = l.v;
  if (t_out) { t_out[0] = t[0].v; t_out[1] = t[1].v; t_out[2] = t[2].v; }
  return jadd(jadd(Vs, Vsh), Vbt);
}

void orc_bond_energy_parts(const orc_problem* P, int b, const double pi[3], const double qi[4], const double pj[3],
                           const double qj[4], double parts[3]) {
  int save = g_order;
  g_order = 0;
  bond_energy_jet(P, b, pi, qi, pj, qj, parts, NULL, NULL, NULL);
  g_order = save;
}

/* Bond stresses of the stress fracture criterion (Sec. 3.2, Fracture Criteria), from the implicit potentials:
 *   F_n = grad_p V_stretch, F_s = grad_p V_shear (gradients with respect to the position of endpoint j; the
 *   endpoint i gradients are their negatives), (K t) the generalised moment of the bend-twist potential in the
 *   bond frame (e_0 the twist axis), M_t = <K t, e_0> e_0, M_b = <K t, e_1> e_1 + <K t, e_2> e_2;
 *   sigma = |F_n| / S + |M_b| r0 / I, tau = |F_s| / S + |M_t| r0 / J with r0 = (r_i + r_j)/2, S = pi r0^2,
 *   I = pi r0^4 / 4, J = pi r0^4 / 2.
 * The gradients come from the jets of the energy parts (first derivatives). */
void orc_bond_stress(const orc_problem* P, int b, const double* p, const double* q, double out[2]) {
  int i = P->bi[b], j = P->bj[b], save = g_order;
  g_order = 2;
  jet parts[3];
  double t[3];
  bond_energy_jet(P, b, p + 3 * i, q + 4 * i, p + 3 * j, q + 4 * j, NULL, NULL, t, parts);
  g_order = save;
  double fn = 0.0, fs = 0.0;
  for (int k = 0; k < 3; ++k) {  /* variables 7..9 are p_j */
    fn += parts[0].g[7 + k] * parts[0].g[7 + k];
    fs += parts[1].g[7 + k] * parts[1].g[7 + k];
  }
  const double* K = P->kbt + 3 * b;
  double mt = fabs(K[0] * t[0]);
  double mb = sqrt(K[1] * t[1] * K[1] * t[1] + K[2] * t[2] * K[2] * t[2]);
  double r0 = 0.5 * (P->radius[i] + P->radius[j]);
  double S = M_PI * r0 * r0, I = M_PI * pow(r0, 4) / 4.0, J = M_PI * pow(r0, 4) / 2.0;
  out[0] = sqrt(fn) / S + mb * r0 / I;
  out[1] = sqrt(fs) / S + mt * r0 / J;
}

static double bond_energy(const orc_problem* P, int b, const double* p, const double* q) {
  int i = P->bi[b], j = P->bj[b], save = g_order;
  g_order = 0;
  jet V = bond_energy_jet(P, b, p + 3 * i, q + 4 * i, p + 3 * j, q + 4 * j, NULL, NULL, NULL, NULL);
  g_order = save;
  return V.v;
}

/* V_b(x1) - V_b(x0), with the stretch and bend-twist parts written as exact difference identities
 * (l1 - l0 = (d1 - d0).(d1 + d0)/(l1 + l0); t1 - t0 = R0 (G_l(q_j1 - q_j0) q_i1 + G_l(q_j0)(q_i1 - q_i0)))
 * so that the difference is accurate relative to itself; the shear part is differenced directly. The differences
 * x1 - x0 are taken from (dp, dq) when given (x0 and x1 are then rounded midpoints whose own difference would
 * carry their rounding), else formed from x1 and x0. */
static double bond_energy_diff(const orc_problem* P, int b, const double* p0, const double* q0, const double* p1,
                               const double* q1, const double* dp, const double* dq) {
  int i = P->bi[b], j = P->bj[b], save = g_order;
  double e0[3], e1[3], l0v, l1v, t0[3], t1[3];
  g_order = 0;
  bond_energy_jet(P, b, p0 + 3 * i, q0 + 4 * i, p0 + 3 * j, q0 + 4 * j, e0, &l0v, t0, NULL);
  bond_energy_jet(P, b, p1 + 3 * i, q1 + 4 * i, p1 + 3 * j, q1 + 4 * j, e1, &l1v, t1, NULL);
  g_order = save;
  double dd[3], ds[3];
  for (int k = 0; k < 3; ++k) {
    dd[k] = dp ? dp[3 * j + k] - dp[3 * i + k] : (p1[3 * j + k] - p0[3 * j + k]) - (p1[3 * i + k] - p0[3 * i + k]);
    ds[k] = (p0[3 * j + k] - p0[3 * i + k]) + (p1[3 * j + k] - p1[3 * i + k]);
  }
  double dl = dot3(dd, ds) / (l0v + l1v);
  double dVs = 0.5 * P->kn[b] * dl * ((l0v - P->l0[b]) + (l1v - P->l0[b]));
  double dqi[4], dqj[4], G1[12], G0[12], dw[3];
  for (int k = 0; k < 4; ++k) {
    dqi[k] = dq ? dq[4 * i + k] : q1[4 * i + k] - q0[4 * i + k];
    dqj[k] = dq ? dq[4 * j + k] : q1[4 * j + k] - q0[4 * j + k];
  }
  orc_Gl(dqj, G1);
  orc_Gl(q0 + 4 * j, G0);
  for (int r = 0; r < 3; ++r) {
    dw[r] = 0.0;
    for (int c = 0; c < 4; ++c) dw[r] += G1[4 * r + c] * q1[4 * i + c] + G0[4 * r + c] * dqi[c];
  }
  const double* R0 = P->R0 + 9 * b;
  double dVbt = 0.0;
  for (int r = 0; r < 3; ++r) {
    double dt = R0[3 * r] * dw[0] + R0[3 * r + 1] * dw[1] + R0[3 * r + 2] * dw[2];
    dVbt += 0.5 * P->kbt[3 * b + r] * dt * (t0[r] + t1[r]);
  }
  return dVs + (e1[1] - e0[1]) + dVbt;
}

/* pair term derivatives -> reduced gradient g12 and reduced Hessian H12 (unprojected). The term is evaluated at a
 * point whose Euclidean coordinates move by w times those of the state (w = 1: the state itself; w = 1/2: the
 * midpoint with the step's start state), so its Euclidean gradient and Hessian with respect to the state are w and
 * w^2 times those at the evaluation point; the reduction takes place at the state's quaternions (qa, qb). */
static void pair_reduce(const jet* V, const double qa[4], const double qb[4], double w, double* g12, double* H12) {
  double ge[14], He[196];
  jet_grad_hess(V, ge, He);
  for (int k = 0; k < 14; ++k) ge[k] *= w;
  for (int k = 0; k < 196; ++k) He[k] *= w * w;
  const double* qe[2] = {qa, qb};
  riemann_reduce(2, qe, ge, He, g12, H12);
}

void orc_bond_terms(const orc_problem* P, int b, const double pi[3], const double qi[4], const double pj[3],
                    const double qj[4], double* energy, double* grad12, double* hess12, double* hess12_spd) {
  orc_bond_terms_at(P, b, pi, qi, pj, qj, qi, qj, 1.0, energy, grad12, hess12, hess12_spd);
}

void orc_bond_terms_at(const orc_problem* P, int b, const double pvi[3], const double qvi[4], const double pvj[3],
                       const double qvj[4], const double qi[4], const double qj[4], double w, double* energy,
                       double* grad12, double* hess12, double* hess12_spd) {
  g_order = 2;
  jet V = bond_energy_jet(P, b, pvi, qvi, pvj, qvj, NULL, NULL, NULL, NULL);
  double g12[12], H12[144];
  pair_reduce(&V, qi, qj, w, g12, H12);
  if (energy) *energy = V.v;
  if (grad12) memcpy(grad12, g12, sizeof g12);
  if (hess12) memcpy(hess12, H12, sizeof H12);
  if (hess12_spd) { memcpy(hess12_spd, H12, sizeof H12); orc_eig_clamp(12, hess12_spd); }
}

/* ------------------------------------------------------------------------------------------------ */
/* Contact (Sec. 5.4) with the reading: a candidate pair is active when |p_i - p_j| < r_i + r_j,     */
/* V_self = 1/2 k_ec (|p_i - p_j| - r_i - r_j)^2; the ground is the plane z = ground_z with signed    */
/* distance g(p) = p_z - ground_z - r (|grad g| = 1), active when g < 0, V_ext = 1/2 k_c g^2.        */
/* ------------------------------------------------------------------------------------------------ */

static jet contact_energy_jet(double k, double R, const double pa[3], const double pb[3]) {
  jet A[3], B[3];
  for (int c = 0; c < 3; ++c) { A[c] = jvar(pa[c], c); B[c] = jvar(pb[c], 7 + c); }
  jet dx[3];
  for (int c = 0; c < 3; ++c) dx[c] = jsub(A[c], B[c]);
  jet d = jsqrt(jadd(jadd(jmul(dx[0], dx[0]), jmul(dx[1], dx[1])), jmul(dx[2], dx[2])));
  if (d.v >= R) return jc(0.0);
  jet e = jaddc(d, -R);
  return jscale(jmul(e, e), 0.5 * k);
}

static double contact_energy(double k, double R, const double pa[3], const double pb[3]) {
  int save = g_order;
  g_order = 0;
  jet V = contact_energy_jet(k, R, pa, pb);
  g_order = save;
  return V.v;
}

/* contact energy difference; when active at both states, 1/2 k (d1 - d0)(e1 + e0) with
 * d1 - d0 = (x1 - x0).(x1 + x0)/(d1 + d0), x = p_a - p_b; (dpa, dpb), when given, are the endpoint differences */
static double contact_energy_diff(double k, double R, const double* pa0, const double* pb0, const double* pa1,
                                  const double* pb1, const double* dpa, const double* dpb) {
  double x0[3], x1[3], dx[3], sx[3];
  for (int c = 0; c < 3; ++c) {
    x0[c] = pa0[c] - pb0[c];
    x1[c] = pa1[c] - pb1[c];
    dx[c] = dpa ? dpa[c] - dpb[c] : (pa1[c] - pa0[c]) - (pb1[c] - pb0[c]);
    sx[c] = x0[c] + x1[c];
  }
  double d0 = sqrt(dot3(x0, x0)), d1 = sqrt(dot3(x1, x1));
  if (d0 < R && d1 < R) return 0.5 * k * (dot3(dx, sx) / (d0 + d1)) * ((d0 - R) + (d1 - R));
  return contact_energy(k, R, pa1, pb1) - contact_energy(k, R, pa0, pb0);
}

/* Per-particle term: inertia 1/(2dt^2) (x - xhat)^T M_s (x - xhat) at the state (p, q), gravity -m g.pv and the
 * ground at the potential's evaluation point pv (the state itself, or the midpoint with the step's start state). */
static double particle_energy(const orc_config* C, double m, double r, const double p[3], const double q[4],
                              const double pv[3], const double ph[3], const double qh[4]) {
  double dt2 = C->dt * C->dt, cp = m / dt2, cq = 1.6 * m * r * r / dt2, e = 0.0;
  for (int k = 0; k < 3; ++k) e += 0.5 * cp * (p[k] - ph[k]) * (p[k] - ph[k]);
  for (int k = 0; k < 4; ++k) e += 0.5 * cq * (q[k] - qh[k]) * (q[k] - qh[k]);
  e -= m * dot3(C->gravity, pv);
  if (C->k_ground > 0.0) {
    double gd = pv[2] - C->ground_z - r;
    if (gd < 0.0) e += 0.5 * C->k_ground * gd * gd;
  }
  return e;
}

/* particle-term difference written with dp = p1 - p0: 1/2 c (|p1 - ph|^2 - |p0 - ph|^2) = c dp.((p0 - ph) + dp/2),
 * the same for q, -m g.dv, and for the ground 1/2 k (g1 - g0)(g1 + g0) when active at both evaluation points
 * (v0, v1: the potential's evaluation points, dv = v1 - v0; the state itself, or the midpoints with the step's
 * start state and dv = dp/2) */
static double particle_energy_diff(const orc_config* C, double m, double r, const double* p0, const double* q0,
                                   const double* p1, const double* q1, const double* v0, const double* v1,
                                   double wv, const double* ph, const double* qh) {
  double dt2 = C->dt * C->dt, cp = m / dt2, cq = 1.6 * m * r * r / dt2, e = 0.0;
  for (int k = 0; k < 3; ++k) {
    double dp = p1[k] - p0[k];
    e += cp * dp * ((p0[k] - ph[k]) + 0.5 * dp) - m * C->gravity[k] * (wv * dp);
  }
  for (int k = 0; k < 4; ++k) {
    double dq = q1[k] - q0[k];
    e += cq * dq * ((q0[k] - qh[k]) + 0.5 * dq);
  }
  if (C->k_ground > 0.0) {
    double g0 = v0[2] - C->ground_z - r, g1 = v1[2] - C->ground_z - r;
    if (g0 < 0.0 && g1 < 0.0) e += 0.5 * C->k_ground * (wv * (p1[2] - p0[2])) * (g0 + g1);
    else e += 0.5 * C->k_ground * ((g1 < 0.0 ? g1 * g1 : 0.0) - (g0 < 0.0 ? g0 * g0 : 0.0));
  }
  return e;
}

/* reduced gradient (6) and projected reduced Hessian (6x6) of the particle term; gravity and the ground are
 * evaluated at pv, whose coordinates move by w times those of the state (see pair_reduce) */
static void particle_terms(const orc_config* C, double m, double r, const double p[3], const double q[4],
                           const double pv[3], double w, const double ph[3], const double qh[4], double g6[6],
                           double H6[36]) {
  double dt2 = C->dt * C->dt, cp = m / dt2, cq = 1.6 * m * r * r / dt2;
  double ge[7], He[49];
  memset(He, 0, sizeof He);
  for (int k = 0; k < 3; ++k) { ge[k] = cp * (p[k] - ph[k]) - w * m * C->gravity[k]; He[8 * k] = cp; }
  for (int k = 0; k < 4; ++k) { ge[3 + k] = cq * (q[k] - qh[k]); He[8 * (3 + k)] = cq; }
  if (C->k_ground > 0.0) {
    double gd = pv[2] - C->ground_z - r;
    if (gd < 0.0) { ge[2] += w * C->k_ground * gd; He[8 * 2] += w * w * C->k_ground; }
  }
  const double* qe[1] = {q};
  riemann_reduce(1, qe, ge, He, g6, H6);
  orc_eig_clamp(6, H6);
}

/* ------------------------------------------------------------------------------------------------ */
/* Retraction: Eq. manifold-update-1/2 with dq = G_l(q)^T y, then q <- q/|q| (Sec. 4.1).             */
/* ------------------------------------------------------------------------------------------------ */

void orc_retract(const double p[3], const double q[4], const double st[6], double alpha, double po[3], double qo[4]) {
  for (int k = 0; k < 3; ++k) po[k] = p[k] + alpha * st[k];
  double G[12], dq[4];
  orc_Gl(q, G);
  for (int c = 0; c < 4; ++c) dq[c] = alpha * (G[c] * st[3] + G[4 + c] * st[4] + G[8 + c] * st[5]);
  double a = sqrt(dot4(dq, dq));
  if (a == 0.0) {
    for (int k = 0; k < 4; ++k) qo[k] = q[k];
  } else {
    double ca = cos(a), sa = sin(a);
    for (int k = 0; k < 4; ++k) qo[k] = q[k] * ca + dq[k] / a * sa;
  }
  double nq = sqrt(dot4(qo, qo));
  for (int k = 0; k < 4; ++k) qo[k] /= nq;
}

/* ------------------------------------------------------------------------------------------------ */
/* Contact candidates: unbonded pairs of the scene with |p_i - p_j| < r_i + r_j + skin.               */
/* ------------------------------------------------------------------------------------------------ */

typedef struct { long long key[3]; int id; } cell_entry;

static int cmp_cell(const void* a, const void* b) {
  const cell_entry *x = a, *y = b;
  for (int k = 0; k < 3; ++k) {
    if (x->key[k] < y->key[k]) return -1;
    if (x->key[k] > y->key[k]) return 1;
  }
  return (x->id > y->id) - (x->id < y->id);
}

static int cmp_pair(const void* a, const void* b) {
  const int32_t *x = a, *y = b;
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  return (x[1] > y[1]) - (x[1] < y[1]);
}

/* intact-bond adjacency of a scene: CSR over local particle index */
typedef struct { int* start; int* nbr; } adjacency;

static void build_adjacency(const orc_problem* P, int n0, int ns, adjacency* A) {
  size_t nsz = ns > 0 ? (size_t)ns : 1;
  A->start = calloc(nsz + 1, sizeof(int));
  int cnt = 0;
  for (int b = 0; b < P->nb; ++b) {
    if (P->broken && P->broken[b]) continue;
    int i = P->bi[b], j = P->bj[b];
    if (i < n0 || i >= n0 + ns) continue;
    A->start[i - n0 + 1]++; A->start[j - n0 + 1]++; cnt += 2;
  }
  for (int i = 0; i < ns; ++i) A->start[i + 1] += A->start[i];
  A->nbr = malloc(sizeof(int) * (cnt + 1));
  int* fill = calloc(nsz, sizeof(int));
  for (int b = 0; b < P->nb; ++b) {
    if (P->broken && P->broken[b]) continue;
    int i = P->bi[b], j = P->bj[b];
    if (i < n0 || i >= n0 + ns) continue;
    A->nbr[A->start[i - n0] + fill[i - n0]++] = j;
    A->nbr[A->start[j - n0] + fill[j - n0]++] = i;
  }
  free(fill);
}

static int bonded(const adjacency* A, int n0, int i, int j) {
  for (int k = A->start[i - n0]; k < A->start[i - n0 + 1]; ++k)
    if (A->nbr[k] == j) return 1;
  return 0;
}

static int find_candidates(const orc_config* C, const orc_problem* P, int scene, const double* p, int32_t** out,
                           int brute) {
  int n0 = (int)P->scene_start[scene], ns = (int)(P->scene_start[scene + 1] - P->scene_start[scene]);
  adjacency A;
  build_adjacency(P, n0, ns, &A);
  int cap = 1024, cnt = 0;
  int32_t* pairs = malloc(sizeof(int32_t) * 2 * cap);
  double rmax = 0.0;
  for (int i = n0; i < n0 + ns; ++i) rmax = fmax(rmax, P->radius[i]);
  double h = 2.0 * rmax + C->contact_skin;
#define PUSH_PAIR(a, b)                                                   \
  do {                                                                    \
    if (cnt == cap) { cap *= 2; pairs = realloc(pairs, sizeof(int32_t) * 2 * cap); } \
    pairs[2 * cnt] = (a); pairs[2 * cnt + 1] = (b); cnt++;                \
  } while (0)
  if (brute || ns < 2) {
    for (int i = n0; i < n0 + ns; ++i)
      for (int j = i + 1; j < n0 + ns; ++j) {
        double dx[3] = {p[3 * i] - p[3 * j], p[3 * i + 1] - p[3 * j + 1], p[3 * i + 2] - p[3 * j + 2]};
        double lim = P->radius[i] + P->radius[j] + C->contact_skin;
        if (dot3(dx, dx) < lim * lim && !bonded(&A, n0, i, j)) PUSH_PAIR(i, j);
      }
  } else {
    cell_entry* E = malloc(sizeof(cell_entry) * ns);
    for (int i = 0; i < ns; ++i) {
      for (int k = 0; k < 3; ++k) E[i].key[k] = (long long)floor(p[3 * (n0 + i) + k] / h);
      E[i].id = n0 + i;
    }
    qsort(E, ns, sizeof(cell_entry), cmp_cell);
    for (int a = 0; a < ns; ++a) {
      int i = E[a].id;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dxc = -1; dxc <= 1; ++dxc) {
            cell_entry key = {{E[a].key[0] + dxc, E[a].key[1] + dy, E[a].key[2] + dz}, -1};
            /* first entry with cell >= key */
            int lo = 0, hi = ns;
            while (lo < hi) {
              int mid = (lo + hi) / 2;
              if (cmp_cell(&E[mid], &key) < 0) lo = mid + 1; else hi = mid;
            }
            for (int c = lo; c < ns && E[c].key[0] == key.key[0] && E[c].key[1] == key.key[1] && E[c].key[2] == key.key[2]; ++c) {
              int j = E[c].id;
              if (j <= i) continue;
              double dx[3] = {p[3 * i] - p[3 * j], p[3 * i + 1] - p[3 * j + 1], p[3 * i + 2] - p[3 * j + 2]};
              double lim = P->radius[i] + P->radius[j] + C->contact_skin;
              if (dot3(dx, dx) < lim * lim && !bonded(&A, n0, i, j)) PUSH_PAIR(i, j);
            }
          }
    }
    free(E);
  }
#undef PUSH_PAIR
  qsort(pairs, cnt, 2 * sizeof(int32_t), cmp_pair);
  free(A.start); free(A.nbr);
  *out = pairs;
  return cnt;
}

int orc_contact_candidates(const orc_config* C, const orc_problem* P, int scene, const double* p, int32_t* pairs,
                           int cap, int brute) {
  int32_t* all;
  int cnt = find_candidates(C, P, scene, p, &all, brute);
  for (int k = 0; k < cnt && k < cap; ++k) { pairs[2 * k] = all[2 * k]; pairs[2 * k + 1] = all[2 * k + 1]; }
  free(all);
  return cnt;
}

/* ------------------------------------------------------------------------------------------------ */
/* The Newton system of one scene.                                                                   */
/* ------------------------------------------------------------------------------------------------ */

typedef struct {
  const orc_config* C;
  const orc_problem* P;
  int n0, ns;
  const double *phat, *qhat;   /* global [n][3], [n][4] */
  int nbond; int* bonds;       /* intact bonds of the scene */
  int ncand; int32_t* cand;    /* contact candidate pairs (global ids) */
  double* g;                   /* [6 ns] reduced gradient (kinematic entries zeroed) */
  double* Hp;                  /* [ns][36] particle-term blocks */
  double* Hb;                  /* [nbond][144] bond blocks */
  double* Hc;                  /* [ncand][144] contact blocks */
  double* D;                   /* [ns][36] assembled diagonal blocks (preconditioner) */
  int mid;                     /* variational midpoint form: potentials at (x + x_n)/2 */
  const double *pn, *qn;       /* the step's start state x_n (the problem's state arrays) */
  double *pm0, *qm0, *pm1, *qm1, *dpm, *dqm;  /* [n][3], [n][4] midpoints and their differences (mid only) */
  const double *cur_p, *cur_q; /* the state of the last sys_assemble (the AMG's rigid modes are taken there) */
} scene_sys;

static void sys_init(scene_sys* S, const orc_config* C, const orc_problem* P, int scene, const double* phat,
                     const double* qhat) {
  memset(S, 0, sizeof *S);
  S->C = C; S->P = P; S->phat = phat; S->qhat = qhat;
  S->n0 = (int)P->scene_start[scene];
  S->ns = (int)(P->scene_start[scene + 1] - P->scene_start[scene]);
  S->bonds = malloc(sizeof(int) * (P->nb + 1));
  for (int b = 0; b < P->nb; ++b)
    if (!(P->broken && P->broken[b]) && P->bi[b] >= S->n0 && P->bi[b] < S->n0 + S->ns) S->bonds[S->nbond++] = b;
  S->g = malloc(sizeof(double) * 6 * S->ns);
  S->Hp = malloc(sizeof(double) * 36 * S->ns);
  S->D = malloc(sizeof(double) * 36 * S->ns);
  S->Hb = malloc(sizeof(double) * 144 * (S->nbond + 1));
  S->mid = C->integrator == 1;
  S->pn = P->p;
  S->qn = P->q;
  if (S->mid) {
    S->pm0 = calloc(3 * (size_t)P->n, sizeof(double)); S->qm0 = calloc(4 * (size_t)P->n, sizeof(double));
    S->pm1 = calloc(3 * (size_t)P->n, sizeof(double)); S->qm1 = calloc(4 * (size_t)P->n, sizeof(double));
    S->dpm = calloc(3 * (size_t)P->n, sizeof(double)); S->dqm = calloc(4 * (size_t)P->n, sizeof(double));
  }
}

/* the midpoint (x + x_n)/2 of the scene's particles (Sec. 3.1, Eq. variational optimisation form) */
static void sys_midpoint(const scene_sys* S, const double* p, const double* q, double* pm, double* qm) {
  for (int i = S->n0; i < S->n0 + S->ns; ++i) {
    for (int k = 0; k < 3; ++k) pm[3 * i + k] = 0.5 * (p[3 * i + k] + S->pn[3 * i + k]);
    for (int k = 0; k < 4; ++k) qm[4 * i + k] = 0.5 * (q[4 * i + k] + S->qn[4 * i + k]);
  }
}

static void sys_free(scene_sys* S) {
  free(S->bonds); free(S->g); free(S->Hp); free(S->D); free(S->Hb); free(S->Hc); free(S->cand);
  free(S->pm0); free(S->qm0); free(S->pm1); free(S->qm1); free(S->dpm); free(S->dqm);
}

static void sys_set_candidates(scene_sys* S, int scene, const double* p) {
  free(S->cand); free(S->Hc);
  S->cand = NULL; S->ncand = 0;
  if (S->C->k_self > 0.0) S->ncand = find_candidates(S->C, S->P, scene, p, &S->cand, 0);
  S->Hc = malloc(sizeof(double) * 144 * (S->ncand + 1));
}

static int is_kin(const orc_problem* P, int i) { return P->kinematic && P->kinematic[i]; }

/* Phi(x) summed term by term (potentials at x, or at the midpoint (x + x_n)/2) */
static double sys_energy(const scene_sys* S, const double* p, const double* q) {
  const orc_problem* P = S->P;
  const double *pv = p, *qv = q;
  if (S->mid) {
    sys_midpoint(S, p, q, S->pm0, S->qm0);
    pv = S->pm0; qv = S->qm0;
  }
  double e = 0.0;
  for (int i = S->n0; i < S->n0 + S->ns; ++i)
    e += particle_energy(S->C, P->mass[i], P->radius[i], p + 3 * i, q + 4 * i, pv + 3 * i, S->phat + 3 * i,
                         S->qhat + 4 * i);
  for (int k = 0; k < S->nbond; ++k) e += bond_energy(P, S->bonds[k], pv, qv);
  for (int k = 0; k < S->ncand; ++k) {
    int a = S->cand[2 * k], b = S->cand[2 * k + 1];
    e += contact_energy(S->C->k_self, P->radius[a] + P->radius[b], pv + 3 * a, pv + 3 * b);
  }
  return e;
}

/* Phi(x1) - Phi(x0): each term's difference is formed first (accurately, see the *_diff helpers) and the
 * differences are summed; near convergence the total is far below the rounding of Phi itself */
static double sys_energy_diff(const scene_sys* S, const double* p0, const double* q0, const double* p1, const double* q1) {
  const orc_problem* P = S->P;
  /* evaluation points of the potentials and, at the midpoints, their exact differences (x1 - x0)/2 */
  const double *v0 = p0, *w0 = q0, *v1 = p1, *w1 = q1, *dv = NULL, *dw = NULL;
  double wv = 1.0;
  if (S->mid) {
    sys_midpoint(S, p0, q0, S->pm0, S->qm0);
    sys_midpoint(S, p1, q1, S->pm1, S->qm1);
    for (int i = S->n0; i < S->n0 + S->ns; ++i) {
      for (int k = 0; k < 3; ++k) S->dpm[3 * i + k] = 0.5 * (p1[3 * i + k] - p0[3 * i + k]);
      for (int k = 0; k < 4; ++k) S->dqm[4 * i + k] = 0.5 * (q1[4 * i + k] - q0[4 * i + k]);
    }
    v0 = S->pm0; w0 = S->qm0; v1 = S->pm1; w1 = S->qm1; dv = S->dpm; dw = S->dqm;
    wv = 0.5;
  }
  double e = 0.0;
  for (int i = S->n0; i < S->n0 + S->ns; ++i)
    e += particle_energy_diff(S->C, P->mass[i], P->radius[i], p0 + 3 * i, q0 + 4 * i, p1 + 3 * i, q1 + 4 * i,
                              v0 + 3 * i, v1 + 3 * i, wv, S->phat + 3 * i, S->qhat + 4 * i);
  for (int k = 0; k < S->nbond; ++k) e += bond_energy_diff(P, S->bonds[k], v0, w0, v1, w1, dv, dw);
  for (int k = 0; k < S->ncand; ++k) {
    int a = S->cand[2 * k], b = S->cand[2 * k + 1];
    e += contact_energy_diff(S->C->k_self, P->radius[a] + P->radius[b], v0 + 3 * a, v0 + 3 * b, v1 + 3 * a,
                             v1 + 3 * b, dv ? dv + 3 * a : NULL, dv ? dv + 3 * b : NULL);
  }
  return e;
}

double orc_energy_diff(const orc_config* C, const orc_problem* P, int scene, const double* phat, const double* qhat,
                       const double* p0, const double* q0, const double* p1, const double* q1, double* phi0,
                       double* phi1) {
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, p0);
  double d = sys_energy_diff(&S, p0, q0, p1, q1);
  if (phi0) *phi0 = sys_energy(&S, p0, q0);
  if (phi1) *phi1 = sys_energy(&S, p1, q1);
  sys_free(&S);
  return d;
}

/* gradient and projected Hessian blocks at (p, q); mask_kin zeroes kinematic gradient entries */
static void sys_assemble(scene_sys* S, const double* p, const double* q, int mask_kin) {
  const orc_problem* P = S->P;
  int n0 = S->n0, ns = S->ns;
  S->cur_p = p;
  S->cur_q = q;
  /* potentials at x (w = 1) or at the midpoint (x + x_n)/2 (w = 1/2), reduced at x */
  const double *pv = p, *qv = q;
  double w = 1.0;
  if (S->mid) {
    sys_midpoint(S, p, q, S->pm0, S->qm0);
    pv = S->pm0; qv = S->qm0; w = 0.5;
  }
  memset(S->g, 0, sizeof(double) * 6 * ns);
  memset(S->D, 0, sizeof(double) * 36 * ns);
  for (int i = n0; i < n0 + ns; ++i) {
    double g6[6], H6[36];
    particle_terms(S->C, P->mass[i], P->radius[i], p + 3 * i, q + 4 * i, pv + 3 * i, w, S->phat + 3 * i,
                   S->qhat + 4 * i, g6, H6);
    for (int a = 0; a < 6; ++a) S->g[6 * (i - n0) + a] += g6[a];
    memcpy(S->Hp + 36 * (i - n0), H6, sizeof H6);
    for (int a = 0; a < 36; ++a) S->D[36 * (i - n0) + a] += H6[a];
  }
  for (int k = 0; k < S->nbond + S->ncand; ++k) {
    int a, b;
    double g12[12], *H12;
    if (k < S->nbond) {
      int bd = S->bonds[k];
      a = P->bi[bd]; b = P->bj[bd];
      H12 = S->Hb + 144 * k;
      orc_bond_terms_at(P, bd, pv + 3 * a, qv + 4 * a, pv + 3 * b, qv + 4 * b, q + 4 * a, q + 4 * b, w, NULL, g12,
                        NULL, H12);
    } else {
      int c = k - S->nbond;
      a = S->cand[2 * c]; b = S->cand[2 * c + 1];
      H12 = S->Hc + 144 * c;
      g_order = 2;
      jet V = contact_energy_jet(S->C->k_self, P->radius[a] + P->radius[b], pv + 3 * a, pv + 3 * b);
      pair_reduce(&V, q + 4 * a, q + 4 * b, w, g12, H12);
      orc_eig_clamp(12, H12);
    }
    int ia = a - n0, ib = b - n0;
    for (int r = 0; r < 6; ++r) {
      S->g[6 * ia + r] += g12[r];
      S->g[6 * ib + r] += g12[6 + r];
      for (int c = 0; c < 6; ++c) {
        S->D[36 * ia + 6 * r + c] += H12[12 * r + c];
        S->D[36 * ib + 6 * r + c] += H12[12 * (6 + r) + 6 + c];
      }
    }
  }
  if (mask_kin)
    for (int i = n0; i < n0 + ns; ++i)
      if (is_kin(P, i)) {
        for (int a = 0; a < 6; ++a) S->g[6 * (i - n0) + a] = 0.0;
        for (int a = 0; a < 36; ++a) S->D[36 * (i - n0) + a] = (a % 7 == 0) ? 1.0 : 0.0;
      }
}

/* y = H x, H = sum of the projected term Hessians; kinematic rows and columns removed when masked */
static void sys_matvec(const scene_sys* S, const double* x, double* y, int mask_kin) {
  const orc_problem* P = S->P;
  int n0 = S->n0, ns = S->ns;
  memset(y, 0, sizeof(double) * 6 * ns);
  for (int i = 0; i < ns; ++i) {
    if (mask_kin && is_kin(P, n0 + i)) continue;
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) y[6 * i + r] += S->Hp[36 * i + 6 * r + c] * x[6 * i + c];
  }
  for (int k = 0; k < S->nbond + S->ncand; ++k) {
    int a, b;
    const double* H12;
    if (k < S->nbond) { a = P->bi[S->bonds[k]]; b = P->bj[S->bonds[k]]; H12 = S->Hb + 144 * k; }
    else { int c = k - S->nbond; a = S->cand[2 * c]; b = S->cand[2 * c + 1]; H12 = S->Hc + 144 * c; }
    int ka = mask_kin && is_kin(P, a), kb = mask_kin && is_kin(P, b);
    double xv[12], yv[12];
    for (int r = 0; r < 6; ++r) { xv[r] = ka ? 0.0 : x[6 * (a - n0) + r]; xv[6 + r] = kb ? 0.0 : x[6 * (b - n0) + r]; }
    matmul(12, 12, 1, H12, xv, yv);
    for (int r = 0; r < 6; ++r) {
      if (!ka) y[6 * (a - n0) + r] += yv[r];
      if (!kb) y[6 * (b - n0) + r] += yv[6 + r];
    }
  }
}

/* block-Jacobi preconditioner: z_i = D_i^{-1} r_i by Cholesky; a block that is not positive definite
 * falls back to the inverse of its diagonal (entries <= 0 leave r unchanged) */
static int precond_apply(const double* D, const double* r, double* z) {
  double L[36];
  memset(L, 0, sizeof L);
  int ok = 1;
  for (int j = 0; j < 6 && ok; ++j) {
    double s = D[6 * j + j];
    for (int k = 0; k < j; ++k) s -= L[6 * j + k] * L[6 * j + k];
    if (!(s > 0.0)) { ok = 0; break; }
    L[6 * j + j] = sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = D[6 * i + j];
      for (int k = 0; k < j; ++k) t -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = t / L[6 * j + j];
    }
  }
  if (!ok) {
    for (int a = 0; a < 6; ++a) z[a] = D[7 * a] > 0.0 ? r[a] / D[7 * a] : r[a];
    return 0;
  }
  double w[6];
  for (int i = 0; i < 6; ++i) {
    double s = r[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * w[k];
    w[i] = s / L[7 * i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = w[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * z[k];
    z[i] = s / L[7 * i];
  }
  return 1;
}

int orc_precond_apply(const double D[36], const double r[6], double z[6]) { return precond_apply(D, r, z); }

static double vdot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Preconditioned conjugate gradient on H x = b from x = 0, stopping when |r| <= eps_r |b| (Sec. 5.3) */

/* ------------------------------------------------------------------------------------------------ */
/* Algebraic multigrid preconditioner (Sec. 5.3 names an AMG preconditioner for the PCG and nothing    */
/* more). Reading, an aggregation AMG built for this method's block structure:                       */
/*  - level 0: the scene's particles in the Z-order (Morton order) of their initial positions, as      */
/*    defined by orc_morton_order; level l+1: consecutive groups of 8 level-l nodes; coarsest level: the */
/*    first level above 0 with at most 8 nodes, solved exactly (dense Cholesky);                       */
/*  - the coarse space of an aggregate is its infinitesimal rigid motions (t, w): a level-0 node i in  */
/*    aggregate I moves by dp_i = t + w x (p_i - c_I) and turns by y_i = 1/2 R(q_i)^T w (dq = q (x)     */
/*    (y, 0) for the world rotation dq = 1/2 (w, 0) (x) q); a level-l node k (l >= 1) by t_k =          */
/*    t + w x (c_k - c_I), w_k = w; c = centroid (mean of the members' positions or centroids);        */
/*  - A_0 = the assembled system without the off-diagonal blocks of the contact terms (each dropped   */
/*    block leaves its PSD diagonal part, so A_0 stays SPD), kinematic rows and columns replaced by    */
/*    identity; A_{l+1} = P_l^T A_l P_l (Galerkin);                                                     */
/*  - symmetric V(1,1) cycle: x = w D^-1 r; x += P A_c^-1-cycle P^T (r - A x); x += w D^-1 (r - A x)    */
/*    with D the block diagonal of A_l and w = 0.6.                                                     */
/* ------------------------------------------------------------------------------------------------ */

#define AMG_AGG 8
#define AMG_OMEGA 0.6

typedef struct { int r, c; double v[36]; } blk_entry;
typedef struct {
  int n;              /* nodes */
  int nnz;            /* block entries, sorted by (r, c), unique */
  int* rs;            /* [n+1] row starts */
  blk_entry* e;
  double* Dinv;       /* [n][36] inverse of the diagonal block */
  double* P;          /* [n][36] prolongation block of each node into its aggregate (none on the coarsest) */
  double* cen;        /* [n][3] centroid */
  double *r, *x, *t;  /* [6n] work vectors */
} amg_level;
typedef struct {
  int nl;
  amg_level L[16];
  double* chol;       /* coarsest level: dense Cholesky factor, (6 n_L)^2 */
  int mask0;          /* level 0 nodes that are kinematic get zeroed by the caller */
} amg_hier;

static int cmp_blk(const void* a, const void* b) {
  const blk_entry *x = a, *y = b;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  return 0;
}

/* sorts the entries and sums duplicates in their order of appearance (qsort on (r, c, position)) */
typedef struct { blk_entry e; int pos; } blk_tmp;
static int cmp_blk_tmp(const void* a, const void* b) {
  const blk_tmp *x = a, *y = b;
  int c = cmp_blk(&x->e, &y->e);
  if (c) return c;
  return x->pos < y->pos ? -1 : (x->pos > y->pos);
}
static void amg_finish_level(amg_level* L, blk_entry* raw, int nraw) {
  blk_tmp* t = malloc(sizeof(blk_tmp) * (nraw + 1));
  for (int k = 0; k < nraw; ++k) { t[k].e = raw[k]; t[k].pos = k; }
  qsort(t, nraw, sizeof(blk_tmp), cmp_blk_tmp);
  L->e = malloc(sizeof(blk_entry) * (nraw + 1));
  int m = 0;
  for (int k = 0; k < nraw; ++k) {
    if (m > 0 && L->e[m - 1].r == t[k].e.r && L->e[m - 1].c == t[k].e.c) {
      for (int a = 0; a < 36; ++a) L->e[m - 1].v[a] += t[k].e.v[a];
    } else {
      L->e[m++] = t[k].e;
    }
  }
  free(t);
  L->nnz = m;
  L->rs = calloc(L->n + 1, sizeof(int));
  for (int k = 0; k < m; ++k) L->rs[L->e[k].r + 1]++;
  for (int i = 0; i < L->n; ++i) L->rs[i + 1] += L->rs[i];
  L->r = calloc(6 * (size_t)L->n, sizeof(double));
  L->x = calloc(6 * (size_t)L->n, sizeof(double));
  L->t = calloc(6 * (size_t)L->n, sizeof(double));
}

static void inv6(const double* A, double* Ai) {  /* inverse of an SPD 6x6 block by solving A X = I */
  for (int c = 0; c < 6; ++c) {
    double e[6] = {0, 0, 0, 0, 0, 0}, z[6];
    e[c] = 1.0;
    precond_apply(A, e, z);
    for (int r = 0; r < 6; ++r) Ai[6 * r + c] = z[r];
  }
}

static void rot_of(const double q[4], double R[9]) {  /* R(q) for a unit quaternion {x, y, z, w} */
  double x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

/* the rigid-motion block of a node at position c_k in an aggregate with centroid c_I: [[I, -[c_k - c_I]x], [0, B]] */
static void rigid_block(const double* ck, const double* cI, const double* B3, double* P) {
  double d[3] = {ck[0] - cI[0], ck[1] - cI[1], ck[2] - cI[2]};
  memset(P, 0, sizeof(double) * 36);
  for (int a = 0; a < 3; ++a) P[6 * a + a] = 1.0;
  /* -[d]x: rows of (w x d) = -d x w */
  P[6 * 0 + 4] = d[2];  P[6 * 0 + 5] = -d[1];
  P[6 * 1 + 3] = -d[2]; P[6 * 1 + 5] = d[0];
  P[6 * 2 + 3] = d[1];  P[6 * 2 + 4] = -d[0];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) P[6 * (3 + a) + 3 + b] = B3[3 * a + b];
}

static void amg_free(amg_hier* H) {
  for (int l = 0; l < H->nl; ++l) {
    amg_level* L = &H->L[l];
    free(L->rs); free(L->e); free(L->Dinv); free(L->P); free(L->cen); free(L->r); free(L->x); free(L->t);
  }
  free(H->chol);
}

static void amg_cholesky(int n, double* A) {  /* in place, lower triangle */
  for (int j = 0; j < n; ++j) {
    double s = A[n * j + j];
    for (int k = 0; k < j; ++k) s -= A[n * j + k] * A[n * j + k];
    A[n * j + j] = sqrt(s > 0.0 ? s : 1e-300);
    for (int i = j + 1; i < n; ++i) {
      double t = A[n * i + j];
      for (int k = 0; k < j; ++k) t -= A[n * i + k] * A[n * j + k];
      A[n * i + j] = t / A[n * j + j];
    }
  }
}

/* builds the hierarchy of one scene from its assembled system (sys_assemble with the kinematic mask) */
static void amg_build(const scene_sys* S, const double* p, const double* q, amg_hier* H) {
  const orc_problem* P = S->P;
  int n0 = S->n0, ns = S->ns;
  memset(H, 0, sizeof *H);
  /* level 0: node k = particle morton[n0 + k]; pos[] local node index of each particle */
  int* node_of = malloc(sizeof(int) * (ns + 1));
  for (int k = 0; k < ns; ++k) node_of[P->morton[n0 + k] - n0] = k;
  amg_level* L0 = &H->L[0];
  L0->n = ns;
  int nraw = 0, cap = ns + 2 * S->nbond + 1;
  blk_entry* raw = malloc(sizeof(blk_entry) * cap);
  for (int k = 0; k < ns; ++k) {
    int i = P->morton[n0 + k];
    raw[nraw].r = raw[nraw].c = k;
    memcpy(raw[nraw].v, S->D + 36 * (i - n0), sizeof(double) * 36);
    ++nraw;
  }
  for (int k = 0; k < S->nbond; ++k) {
    int a = P->bi[S->bonds[k]], b = P->bj[S->bonds[k]];
    if (is_kin(P, a) || is_kin(P, b)) continue;
    const double* H12 = S->Hb + 144 * k;
    int na = node_of[a - n0], nb = node_of[b - n0];
    raw[nraw].r = na; raw[nraw].c = nb;
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) raw[nraw].v[6 * r + c] = H12[12 * r + 6 + c];
    ++nraw;
    raw[nraw].r = nb; raw[nraw].c = na;
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) raw[nraw].v[6 * r + c] = H12[12 * (6 + r) + c];
    ++nraw;
  }
  amg_finish_level(L0, raw, nraw);
  free(raw);
  L0->cen = malloc(sizeof(double) * 3 * (ns + 1));
  for (int k = 0; k < ns; ++k) memcpy(L0->cen + 3 * k, p + 3 * P->morton[n0 + k], sizeof(double) * 3);
  int l = 0;
  for (;;) {
    amg_level* L = &H->L[l];
    L->Dinv = malloc(sizeof(double) * 36 * (L->n + 1));
    for (int i = 0; i < L->n; ++i)
      for (int k = L->rs[i]; k < L->rs[i + 1]; ++k)
        if (L->e[k].c == i) inv6(L->e[k].v, L->Dinv + 36 * i);
    if ((L->n <= AMG_AGG && l > 0) || l == 15) break;  /* at least one coarse level */
    /* aggregates of consecutive groups of AMG_AGG nodes: centroids, prolongation blocks, Galerkin product */
    amg_level* C = &H->L[l + 1];
    C->n = (L->n + AMG_AGG - 1) / AMG_AGG;
    C->cen = calloc(3 * (size_t)C->n + 3, sizeof(double));
    for (int I = 0; I < C->n; ++I) {
      int a = I * AMG_AGG, b = a + AMG_AGG < L->n ? a + AMG_AGG : L->n;
      for (int k = a; k < b; ++k)
        for (int c = 0; c < 3; ++c) C->cen[3 * I + c] += L->cen[3 * k + c];
      for (int c = 0; c < 3; ++c) C->cen[3 * I + c] /= (double)(b - a);
    }
    L->P = malloc(sizeof(double) * 36 * (L->n + 1));
    for (int k = 0; k < L->n; ++k) {
      double B3[9];
      if (l == 0) {
        double R[9];
        rot_of(q + 4 * P->morton[n0 + k], R);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) B3[3 * a + b] = 0.5 * R[3 * b + a];  /* 1/2 R^T */
      } else {
        for (int a = 0; a < 9; ++a) B3[a] = (a % 4 == 0) ? 1.0 : 0.0;
      }
      rigid_block(L->cen + 3 * k, C->cen + 3 * (k / AMG_AGG), B3, L->P + 36 * k);
    }
    blk_entry* craw = malloc(sizeof(blk_entry) * (L->nnz + 1));
    for (int k = 0; k < L->nnz; ++k) {
      const blk_entry* e = &L->e[k];
      double T[36], Pt[36];
      craw[k].r = e->r / AMG_AGG;
      craw[k].c = e->c / AMG_AGG;
      matmul(6, 6, 6, e->v, L->P + 36 * e->c, T);        /* A_rc P_c */
      transpose(6, 6, L->P + 36 * e->r, Pt);
      matmul(6, 6, 6, Pt, T, craw[k].v);                  /* P_r^T A_rc P_c */
    }
    amg_finish_level(C, craw, L->nnz);
    free(craw);
    ++l;
  }
  H->nl = l + 1;
  /* coarsest: dense Cholesky */
  amg_level* Lc = &H->L[l];
  int m = 6 * Lc->n;
  H->chol = calloc((size_t)m * m + 1, sizeof(double));
  for (int k = 0; k < Lc->nnz; ++k)
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) H->chol[(size_t)m * (6 * Lc->e[k].r + a) + 6 * Lc->e[k].c + b] = Lc->e[k].v[6 * a + b];
  amg_cholesky(m, H->chol);
  free(node_of);
}

static void amg_spmv_res(const amg_level* L, const double* x, const double* r, double* t) {  /* t = r - A x */
  for (int i = 0; i < L->n; ++i) {
    double s[6];
    for (int a = 0; a < 6; ++a) s[a] = r[6 * i + a];
    for (int k = L->rs[i]; k < L->rs[i + 1]; ++k) {
      const blk_entry* e = &L->e[k];
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) s[a] -= e->v[6 * a + b] * x[6 * e->c + b];
    }
    for (int a = 0; a < 6; ++a) t[6 * i + a] = s[a];
  }
}

static void amg_cycle(amg_hier* H, int l, const double* r, double* x) {
  amg_level* L = &H->L[l];
  int n6 = 6 * L->n;
  if (l == H->nl - 1) {  /* exact solve with the Cholesky factor */
    double* w = malloc(sizeof(double) * (n6 + 1));
    for (int i = 0; i < n6; ++i) {
      double s = r[i];
      for (int k = 0; k < i; ++k) s -= H->chol[(size_t)n6 * i + k] * w[k];
      w[i] = s / H->chol[(size_t)n6 * i + i];
    }
    for (int i = n6 - 1; i >= 0; --i) {
      double s = w[i];
      for (int k = i + 1; k < n6; ++k) s -= H->chol[(size_t)n6 * k + i] * x[k];
      x[i] = s / H->chol[(size_t)n6 * i + i];
    }
    free(w);
    return;
  }
  amg_level* C = &H->L[l + 1];
  /* pre-smoothing from zero */
  for (int i = 0; i < L->n; ++i) {
    double z[6];
    matmul(6, 6, 1, L->Dinv + 36 * i, r + 6 * i, z);
    for (int a = 0; a < 6; ++a) x[6 * i + a] = AMG_OMEGA * z[a];
  }
  /* restriction of the residual, coarse correction, prolongation */
  amg_spmv_res(L, x, r, L->t);
  memset(C->r, 0, sizeof(double) * 6 * C->n);
  for (int k = 0; k < L->n; ++k) {
    double Pt[36], v[6];
    transpose(6, 6, L->P + 36 * k, Pt);
    matmul(6, 6, 1, Pt, L->t + 6 * k, v);
    for (int a = 0; a < 6; ++a) C->r[6 * (k / AMG_AGG) + a] += v[a];
  }
  double* e = malloc(sizeof(double) * (6 * C->n + 1));
  double* rc = malloc(sizeof(double) * (6 * C->n + 1));
  memcpy(rc, C->r, sizeof(double) * 6 * C->n);
  amg_cycle(H, l + 1, rc, e);
  for (int k = 0; k < L->n; ++k) {
    double v[6];
    matmul(6, 6, 1, L->P + 36 * k, e + 6 * (k / AMG_AGG), v);
    for (int a = 0; a < 6; ++a) x[6 * k + a] += v[a];
  }
  free(e); free(rc);
  /* post-smoothing */
  amg_spmv_res(L, x, r, L->t);
  for (int i = 0; i < L->n; ++i) {
    double z[6];
    matmul(6, 6, 1, L->Dinv + 36 * i, L->t + 6 * i, z);
    for (int a = 0; a < 6; ++a) x[6 * i + a] += AMG_OMEGA * z[a];
  }
}

/* z = M^-1 r for the scene's vectors in particle order (kinematic entries of z zeroed) */
static void amg_apply(const scene_sys* S, amg_hier* H, const double* r, double* z) {
  const orc_problem* P = S->P;
  int n0 = S->n0, ns = S->ns;
  double *rn = calloc(6 * (size_t)ns + 1, sizeof(double)), *xn = calloc(6 * (size_t)ns + 1, sizeof(double));
  for (int k = 0; k < ns; ++k) {
    int i = P->morton[n0 + k];
    for (int a = 0; a < 6; ++a) rn[6 * k + a] = is_kin(P, i) ? 0.0 : r[6 * (i - n0) + a];
  }
  amg_cycle(H, 0, rn, xn);
  for (int k = 0; k < ns; ++k) {
    int i = P->morton[n0 + k];
    for (int a = 0; a < 6; ++a) z[6 * (i - n0) + a] = is_kin(P, i) ? 0.0 : xn[6 * k + a];
  }
  free(rn); free(xn);
}

/* z = M^-1 r: block Jacobi (the assembled diagonal blocks), or the AMG cycle when H is given */
static void prec(const scene_sys* S, amg_hier* H, const double* r, double* z) {
  if (H) { amg_apply(S, H, r, z); return; }
  for (int i = 0; i < S->ns; ++i) precond_apply(S->D + 36 * i, r + 6 * i, z + 6 * i);
}

static int pcg_with(const scene_sys* S, amg_hier* H, const double* b, double eps_r, int max_iter, double* x);

static int pcg(const scene_sys* S, const double* b, double eps_r, int max_iter, double* x) {
  if (S->C->preconditioner == 1 && S->P->morton) {
    amg_hier H;
    amg_build(S, S->cur_p, S->cur_q, &H);
    int it = pcg_with(S, &H, b, eps_r, max_iter, x);
    amg_free(&H);
    return it;
  }
  return pcg_with(S, NULL, b, eps_r, max_iter, x);
}

static int pcg_with(const scene_sys* S, amg_hier* H, const double* b, double eps_r, int max_iter, double* x) {
  int n = 6 * S->ns;
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *pv = malloc(sizeof(double) * n),
         *qv = malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
  double bn = sqrt(vdot(n, b, b)), rz;
  int it = 0;
  if (sqrt(vdot(n, r, r)) > eps_r * bn) {
    prec(S, H, r, z);
    for (int i = 0; i < n; ++i) pv[i] = z[i];
    rz = vdot(n, r, z);
    while (it < max_iter) {
      sys_matvec(S, pv, qv, 1);
      double pq = vdot(n, pv, qv);
      ++it;
      if (!(pq > 0.0)) break;
      double alpha = rz / pq;
      for (int i = 0; i < n; ++i) { x[i] += alpha * pv[i]; r[i] -= alpha * qv[i]; }
      if (sqrt(vdot(n, r, r)) <= eps_r * bn) break;
      prec(S, H, r, z);
      double rz1 = vdot(n, r, z), beta = rz1 / rz;
      rz = rz1;
      for (int i = 0; i < n; ++i) pv[i] = z[i] + beta * pv[i];
    }
  }
  free(r); free(z); free(pv); free(qv);
  return it;
}

static void sys_zhat(const scene_sys* S, const double* phat, const double* qhat, double* zp, double* zq);

int orc_zhat(const orc_config* C, const orc_problem* P, int scene, const double* phat, const double* qhat,
             double* zp, double* zq) {
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, phat);
  memcpy(zp, phat, sizeof(double) * 3 * P->n);
  memcpy(zq, qhat, sizeof(double) * 4 * P->n);
  sys_zhat(&S, phat, qhat, zp, zq);
  int nc = S.ncand;
  sys_free(&S);
  return nc;
}

int orc_system(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
               const double* phat, const double* qhat, double* phi, double* g, double* diag, double* bondH,
               int32_t* n_candidates) {
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, p);
  sys_assemble(&S, p, q, 0);
  if (phi) *phi = sys_energy(&S, p, q);
  if (g) memcpy(g, S.g, sizeof(double) * 6 * S.ns);
  if (diag) memcpy(diag, S.D, sizeof(double) * 36 * S.ns);
  if (bondH) memcpy(bondH, S.Hb, sizeof(double) * 144 * S.nbond);
  if (n_candidates) *n_candidates = S.ncand;
  sys_free(&S);
  return 0;
}

int orc_matvec(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
               const double* phat, const double* qhat, const double* x, double* y) {
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, p);
  sys_assemble(&S, p, q, 0);
  sys_matvec(&S, x, y, 0);
  sys_free(&S);
  return 0;
}

static uint64_t spread_bits3(uint64_t x) {  /* bit k of x moves to bit 3k (21 bits) */
  uint64_t out = 0;
  for (int k = 0; k < 21; ++k) out |= ((x >> k) & 1ull) << (3 * k);
  return out;
}

typedef struct { uint64_t code; int32_t id; } morton_key;
static int cmp_morton(const void* a, const void* b) {
  const morton_key *x = a, *y = b;
  if (x->code != y->code) return x->code < y->code ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

void orc_morton_order(const int64_t* scene_start, int n_scenes, const double* pos, int32_t* out) {
  for (int s = 0; s < n_scenes; ++s) {
    int64_t a = scene_start[s], b = scene_start[s + 1];
    if (b <= a) continue;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = a; i < b; ++i)
      for (int k = 0; k < 3; ++k) {
        if (pos[3 * i + k] < lo[k]) lo[k] = pos[3 * i + k];
        if (pos[3 * i + k] > hi[k]) hi[k] = pos[3 * i + k];
      }
    double ext = 1e-300;
    for (int k = 0; k < 3; ++k) if (hi[k] - lo[k] > ext) ext = hi[k] - lo[k];
    double scale = 2097151.0 / ext;
    morton_key* keys = malloc(sizeof(morton_key) * (size_t)(b - a));
    for (int64_t i = a; i < b; ++i) {
      uint64_t c = 0;
      for (int k = 0; k < 3; ++k) {
        double v = (pos[3 * i + k] - lo[k]) * scale;
        if (v < 0.0) v = 0.0;
        if (v > 2097151.0) v = 2097151.0;
        c |= spread_bits3((uint64_t)v) << k;
      }
      keys[i - a].code = c;
      keys[i - a].id = (int32_t)i;
    }
    qsort(keys, (size_t)(b - a), sizeof(morton_key), cmp_morton);
    for (int64_t i = a; i < b; ++i) out[i] = keys[i - a].id;
    free(keys);
  }
}

int orc_amg_apply(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
                  const double* phat, const double* qhat, const double* r, double* z) {
  if (!P->morton) return -1;
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, p);
  sys_assemble(&S, p, q, 1);
  amg_hier H;
  amg_build(&S, p, q, &H);
  amg_apply(&S, &H, r, z);
  int nl = H.nl;
  amg_free(&H);
  sys_free(&S);
  return nl;
}

int orc_amg_level1_apply(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
                         const double* phat, const double* qhat, const double* e, double* y) {
  if (!P->morton) return -1;
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, p);
  sys_assemble(&S, p, q, 1);
  amg_hier H;
  amg_build(&S, p, q, &H);
  int m = -1;
  if (H.nl > 1) {
    amg_level* L1 = &H.L[1];
    m = L1->n;
    memset(y, 0, sizeof(double) * 6 * m);
    for (int k = 0; k < L1->nnz; ++k)
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) y[6 * L1->e[k].r + a] += L1->e[k].v[6 * a + b] * e[6 * L1->e[k].c + b];
  }
  amg_free(&H);
  sys_free(&S);
  return m;
}

int orc_pcg_solve(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
                  const double* phat, const double* qhat, const double* b, double eps_r, int max_iter, double* x) {
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, p);
  sys_assemble(&S, p, q, 1);
  int it = pcg(&S, b, eps_r, max_iter, x);
  sys_free(&S);
  return it;
}

/* ------------------------------------------------------------------------------------------------ */
/* Alg. 3: one time step.                                                                           */
/* Readings: Newton stops when |g_k| <= tol |g_0| (g_0 at the initial guess), or, when an absolute   */
/* tolerance is set, when |g_k| <= newton_abs_tol (Alg. 3's own test |grad f| < eps); eps_r uses the  */
/* absolute |g_k|; the line search halves alpha from 1 until Phi(x') - Phi(x) <= 0 (at most           */
/* ls_max_halvings halvings), and a direction with g.dx >= 0 is replaced by -g; after convergence a   */
/* bond breaks when its tensile strain (|p_j - p_i| - l0)/l0 exceeds its limit; kinematic particles    */
/* move with their velocity and are excluded from the solve.                                          */
/* ------------------------------------------------------------------------------------------------ */

/* The target of the variational midpoint form (Sec. 3.1; App. C):
 *   zhat = xhat - 1/2 M_s^{-1} dt^2 grad V((x_{n-1} + x_n)/2),  x_{n-1} = x_n - dt v_n,
 * with the Euclidean gradient (R^3 x R^4 per particle) of every potential term of the scene at that midpoint: the
 * intact bonds, gravity, the ground and the step's contact candidates. Kinematic particles keep zhat = xhat. */
static void sys_zhat(const scene_sys* S, const double* phat, const double* qhat, double* zp, double* zq) {
  const orc_problem* P = S->P;
  const orc_config* C = S->C;
  int n = P->n, n0 = S->n0, ns = S->ns;
  double *pm = malloc(sizeof(double) * 3 * n), *qm = malloc(sizeof(double) * 4 * n);
  double* ge = calloc(7 * (size_t)n, sizeof(double));
  double dt = C->dt;
  for (int i = n0; i < n0 + ns; ++i) {
    for (int k = 0; k < 3; ++k) pm[3 * i + k] = P->p[3 * i + k] - 0.5 * dt * P->v[3 * i + k];
    for (int k = 0; k < 4; ++k) qm[4 * i + k] = P->q[4 * i + k] - 0.5 * dt * P->u[4 * i + k];
    double m = P->mass[i];
    for (int k = 0; k < 3; ++k) ge[7 * i + k] = -m * C->gravity[k];
    if (C->k_ground > 0.0) {
      double gd = pm[3 * i + 2] - C->ground_z - P->radius[i];
      if (gd < 0.0) ge[7 * i + 2] += C->k_ground * gd;
    }
  }
  g_order = 2;
  for (int k = 0; k < S->nbond + S->ncand; ++k) {
    int a, b;
    jet V;
    if (k < S->nbond) {
      int bd = S->bonds[k];
      a = P->bi[bd]; b = P->bj[bd];
      V = bond_energy_jet(P, bd, pm + 3 * a, qm + 4 * a, pm + 3 * b, qm + 4 * b, NULL, NULL, NULL, NULL);
    } else {
      int c = k - S->nbond;
      a = S->cand[2 * c]; b = S->cand[2 * c + 1];
      V = contact_energy_jet(C->k_self, P->radius[a] + P->radius[b], pm + 3 * a, pm + 3 * b);
    }
    double g14[14], H[196];
    jet_grad_hess(&V, g14, H);
    for (int c = 0; c < 7; ++c) { ge[7 * a + c] += g14[c]; ge[7 * b + c] += g14[7 + c]; }
  }
  for (int i = n0; i < n0 + ns; ++i) {
    double m = P->mass[i], r = P->radius[i];
    double cp = m / (dt * dt), cq = 1.6 * m * r * r / (dt * dt);
    int kin = P->kinematic && P->kinematic[i];
    for (int k = 0; k < 3; ++k) zp[3 * i + k] = kin ? phat[3 * i + k] : phat[3 * i + k] - 0.5 * ge[7 * i + k] / cp;
    for (int k = 0; k < 4; ++k) zq[4 * i + k] = kin ? qhat[4 * i + k] : qhat[4 * i + k] - 0.5 * ge[7 * i + 3 + k] / cq;
  }
  free(pm); free(qm); free(ge);
}

static int newton_scene(const orc_config* C, orc_problem* P, int scene, double* xp, double* xq, const double* phat,
                        const double* qhat, orc_scene_stats* st) {
  scene_sys S;
  sys_init(&S, C, P, scene, phat, qhat);
  sys_set_candidates(&S, scene, xp);
  st->n_candidates = S.ncand;
  double *zp = NULL, *zq = NULL;
  if (S.mid) {  /* the inertia targets become zhat */
    zp = malloc(sizeof(double) * 3 * P->n);
    zq = malloc(sizeof(double) * 4 * P->n);
    sys_zhat(&S, phat, qhat, zp, zq);
    S.phat = zp;
    S.qhat = zq;
  }
  int n0 = S.n0, ns = S.ns, n6 = 6 * ns, status = 0;
  double *dx = malloc(sizeof(double) * n6), *rhs = malloc(sizeof(double) * n6);
  double *tp = malloc(sizeof(double) * 3 * P->n), *tq = malloc(sizeof(double) * 4 * P->n);
  memcpy(tp, xp, sizeof(double) * 3 * P->n);
  memcpy(tq, xq, sizeof(double) * 4 * P->n);
  int k = 0;
  for (;;) {
    sys_assemble(&S, xp, xq, 1);
    double gn = sqrt(vdot(n6, S.g, S.g));
    if (k == 0) st->g0_norm = gn;
    st->g_norm = gn;
    if (gn <= C->newton_rel_tol * st->g0_norm || gn <= C->newton_abs_tol) break;
    if (k >= C->newton_max_iter) { status = 4; break; }
    if (C->optimizer == 1) {
      /* Alg. 1: the descent direction is -grad f; in the reduced coordinates dq = G_l(q)^T y, so y = -g_y gives
       * dq = -(I - q q^T) grad_q F, the projected gradient of the first-order method */
      for (int i = 0; i < n6; ++i) dx[i] = -S.g[i];
    } else {
      double eps_r = fmin(0.5, sqrt(gn));
      for (int i = 0; i < n6; ++i) rhs[i] = -S.g[i];
      st->pcg_iters += pcg(&S, rhs, eps_r, C->pcg_max_iter, dx);
      if (vdot(n6, S.g, dx) >= 0.0)
        for (int i = 0; i < n6; ++i) dx[i] = -S.g[i];
    }
    ++k;
    double alpha = 1.0;
    int accepted = 0;
    for (int h = 0; h <= C->ls_max_halvings; ++h) {
      for (int i = n0; i < n0 + ns; ++i)
        orc_retract(xp + 3 * i, xq + 4 * i, dx + 6 * (i - n0), alpha, tp + 3 * i, tq + 4 * i);
      if (sys_energy_diff(&S, xp, xq, tp, tq) <= 0.0) { accepted = 1; break; }
      alpha *= 0.5;
      st->ls_halvings++;
    }
    if (!accepted) { status = 5; break; }
    for (int i = n0; i < n0 + ns; ++i) {
      memcpy(xp + 3 * i, tp + 3 * i, sizeof(double) * 3);
      memcpy(xq + 4 * i, tq + 4 * i, sizeof(double) * 4);
    }
  }
  st->newton_iters = k;
  st->status = status;
  free(dx); free(rhs); free(tp); free(tq); free(zp); free(zq);
  sys_free(&S);
  return status;
}

/* ------------------------------------------------------------------------------------------------ */
/* Friction (Sec. 5.4, Friction; Alg. 3: project v_{n+1} to the friction cone), an explicit velocity   */
/* correction after the velocity update, with the readings:                                          */
/*  - the contacts are those active at x_{n+1}: the ground when g = p_z - z_ground - r < 0 (normal     */
/*    e_z, |F_n| = k_c |g|), and the step's self-contact candidates that overlap at x_{n+1} (normal    */
/*    (p_i - p_j)/|p_i - p_j|, |F_n| = k_ec |d - r_i - r_j|);                                           */
/*  - v_ij = v_i - v_j (v_i for the ground), w_ij = w_i - w_j (w_i) with w the angular velocity in the  */
/*    world frame, q' = 1/2 (w, 0) (x) q;                                                              */
/*  - each contact contributes dv = -min(1, mu_s |F_n| dt / (m_i |v_t|)) v_t and                       */
/*    dw = -min(1, mu_r |F_n| r_i^3 dt / (I_i |w_ij|)) w_ij with I_i = 2/5 m_i r_i^2; the contributions */
/*    of all contacts add, computed from the velocities before any correction;                        */
/*  - the sums are projected on the directions of v_i and w_i and clamped to [-|v_i|, 0] and           */
/*    [-|w_i|, 0] along them (the correction only slows the element, down to rest at most);            */
/*  - q' changes by 1/2 (dw, 0) (x) q; kinematic particles keep their velocities.                      */
/* ------------------------------------------------------------------------------------------------ */

static void ang_vel(const double q[4], const double u[4], double w[3]) {
  double qc[4] = {-q[0], -q[1], -q[2], q[3]}, t[4];
  orc_qmul(u, qc, t);
  w[0] = 2.0 * t[0]; w[1] = 2.0 * t[1]; w[2] = 2.0 * t[2];
}

static void contact_friction(const orc_config* C, const double* p, const double* vv, const double* ww, int i, int j,
                             const double* radius, double mi, double dv[3], double dw[3]) {
  /* j < 0: the ground */
  double n[3], fn, vij[3], wij[3];
  double ri = radius[i];
  if (j < 0) {
    double g = p[3 * i + 2] - C->ground_z - ri;
    if (!(g < 0.0)) return;
    n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
    fn = C->k_ground * fabs(g);
    for (int k = 0; k < 3; ++k) { vij[k] = vv[3 * i + k]; wij[k] = ww[3 * i + k]; }
  } else {
    double e[3] = {p[3 * i] - p[3 * j], p[3 * i + 1] - p[3 * j + 1], p[3 * i + 2] - p[3 * j + 2]};
    double d = sqrt(dot3(e, e)), R = ri + radius[j];
    if (!(d < R)) return;
    for (int k = 0; k < 3; ++k) n[k] = e[k] / d;
    fn = C->k_self * fabs(d - R);
    for (int k = 0; k < 3; ++k) { vij[k] = vv[3 * i + k] - vv[3 * j + k]; wij[k] = ww[3 * i + k] - ww[3 * j + k]; }
  }
  double vn = dot3(vij, n), vt[3] = {vij[0] - vn * n[0], vij[1] - vn * n[1], vij[2] - vn * n[2]};
  double nvt = sqrt(dot3(vt, vt)), nw = sqrt(dot3(wij, wij));
  if (nvt > 0.0) {
    double c = C->mu_slide * fn * C->dt / (mi * nvt);
    if (c > 1.0) c = 1.0;
    for (int k = 0; k < 3; ++k) dv[k] -= c * vt[k];
  }
  if (nw > 0.0) {
    double I = 0.4 * mi * ri * ri;
    double c = C->mu_roll * fn * ri * ri * ri * C->dt / (I * nw);
    if (c > 1.0) c = 1.0;
    for (int k = 0; k < 3; ++k) dw[k] -= c * wij[k];
  }
}

/* clamps the correction d to the direction of x: d <- s x/|x| with s = d.x/|x| limited to [-|x|, 0] */
static void slow_only(const double x[3], double d[3]) {
  double nx = sqrt(dot3(x, x));
  if (!(nx > 0.0)) { d[0] = d[1] = d[2] = 0.0; return; }
  double s = dot3(d, x) / nx;
  if (s > 0.0) s = 0.0;
  if (s < -nx) s = -nx;
  for (int k = 0; k < 3; ++k) d[k] = s * x[k] / nx;
}

static void apply_friction(const orc_config* C, orc_problem* P, const double* pred) {
  int n = P->n;
  double *vv = malloc(sizeof(double) * 3 * n), *ww = malloc(sizeof(double) * 3 * n);
  double *dv = calloc(3 * (size_t)n, sizeof(double)), *dw = calloc(3 * (size_t)n, sizeof(double));
  memcpy(vv, P->v, sizeof(double) * 3 * n);
  for (int i = 0; i < n; ++i) ang_vel(P->q + 4 * i, P->u + 4 * i, ww + 3 * i);
  for (int s = 0; s < P->n_scenes; ++s) {
    int32_t* cand = NULL;
    int nc = C->k_self > 0.0 ? find_candidates(C, P, s, pred, &cand, 0) : 0;  /* the step's candidates */
    for (int i = (int)P->scene_start[s]; i < (int)P->scene_start[s + 1]; ++i)
      if (C->k_ground > 0.0) contact_friction(C, P->p, vv, ww, i, -1, P->radius, P->mass[i], dv + 3 * i, dw + 3 * i);
    for (int k = 0; k < nc; ++k) {
      int a = cand[2 * k], b = cand[2 * k + 1];
      contact_friction(C, P->p, vv, ww, a, b, P->radius, P->mass[a], dv + 3 * a, dw + 3 * a);
      contact_friction(C, P->p, vv, ww, b, a, P->radius, P->mass[b], dv + 3 * b, dw + 3 * b);
    }
    free(cand);
  }
  for (int i = 0; i < n; ++i) {
    if (is_kin(P, i)) continue;
    slow_only(vv + 3 * i, dv + 3 * i);
    slow_only(ww + 3 * i, dw + 3 * i);
    for (int k = 0; k < 3; ++k) P->v[3 * i + k] += dv[3 * i + k];
    double x[4] = {dw[3 * i], dw[3 * i + 1], dw[3 * i + 2], 0.0}, t[4];
    orc_qmul(x, P->q + 4 * i, t);
    for (int k = 0; k < 4; ++k) P->u[4 * i + k] += 0.5 * t[k];
  }
  free(vv); free(ww); free(dv); free(dw);
}

int orc_step(const orc_config* C, orc_problem* P, orc_scene_stats* stats) {
  int n = P->n, worst = 0;
  double dt = C->dt;
  double *phat = malloc(sizeof(double) * 3 * n), *qhat = malloc(sizeof(double) * 4 * n);
  double *xp = malloc(sizeof(double) * 3 * n), *xq = malloc(sizeof(double) * 4 * n);
  /* prediction xhat = x_n + dt v_n (= 2 x_n - x_{n-1}); initial guess x_0 = (phat, qhat/|qhat|) */
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) phat[3 * i + k] = P->p[3 * i + k] + dt * P->v[3 * i + k];
    for (int k = 0; k < 4; ++k) qhat[4 * i + k] = P->q[4 * i + k] + dt * P->u[4 * i + k];
    double nq = sqrt(dot4(qhat + 4 * i, qhat + 4 * i));
    for (int k = 0; k < 3; ++k) xp[3 * i + k] = phat[3 * i + k];
    for (int k = 0; k < 4; ++k) xq[4 * i + k] = qhat[4 * i + k] / nq;
  }
  for (int s = 0; s < P->n_scenes; ++s) {
    memset(&stats[s], 0, sizeof stats[s]);
    int st = newton_scene(C, P, s, xp, xq, phat, qhat, &stats[s]);
    if (st > worst) worst = st;
  }
  /* velocity update v_{n+1} = (x_{n+1} - x_n)/dt, then the new state */
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) { P->v[3 * i + k] = (xp[3 * i + k] - P->p[3 * i + k]) / dt; P->p[3 * i + k] = xp[3 * i + k]; }
    for (int k = 0; k < 4; ++k) { P->u[4 * i + k] = (xq[4 * i + k] - P->q[4 * i + k]) / dt; P->q[4 * i + k] = xq[4 * i + k]; }
  }
  /* friction correction of the new velocities (contacts from the step's candidates, found at the prediction) */
  if (C->mu_slide > 0.0 || C->mu_roll > 0.0) apply_friction(C, P, phat);
  /* bond state update, all bonds at once at the new state: tensile strain fracture, and the stress criterion
   * sigma > sigma_c or tau > tau_c of Sec. 3.2 where the bond's strengths are finite */
  for (int b = 0; b < P->nb; ++b) {
    if (P->broken[b]) continue;
    int i = P->bi[b], j = P->bj[b];
    double d[3] = {P->p[3 * j] - P->p[3 * i], P->p[3 * j + 1] - P->p[3 * i + 1], P->p[3 * j + 2] - P->p[3 * i + 2]};
    double strain = (sqrt(dot3(d, d)) - P->l0[b]) / P->l0[b];
    int brk = strain > P->break_strain[b];
    if (!brk && P->tensile_strength && P->shear_strength &&
        (isfinite(P->tensile_strength[b]) || isfinite(P->shear_strength[b]))) {
      double st[2];
      orc_bond_stress(P, b, P->p, P->q, st);
      brk = st[0] > P->tensile_strength[b] || st[1] > P->shear_strength[b];
    }
    if (brk) {
      P->broken[b] = 1;
      for (int s = 0; s < P->n_scenes; ++s)
        if (i >= P->scene_start[s] && i < P->scene_start[s + 1]) stats[s].bonds_broken++;
    }
  }
  free(phat); free(qhat); free(xp); free(xq);
  return worst;
}
