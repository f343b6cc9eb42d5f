// bdem_device.cuh -- device math of the implicit bonded-DEM Newton iteration.
//
// Per-bond energy, reduced gradient and reduced Riemannian Hessian (Sec. 3.2 potential, Sec. 4.1 gradient,
// Eq. manifold-hessian-1..4 with the nullspace reduction of Sec. 4.2). Derivatives are taken directly in the
// tangent coordinates of the exponential-map retraction (Eq. manifold-update-2): q -> q (x) (y sin|y|/|y|, cos|y|),
// whose pullback Hessian at y = 0 equals the Riemannian Hessian (a second-order retraction). Bond energies depend on
// p_j - p_i only, so each bond is evaluated in 9 variables (d = dp_j - dp_i, y_i, y_j); the translation direction
// is an exact null space and the 12x12 Hessian is rebuilt from the 9x9 one by the map (dp_i, dp_j) -> dp_j - dp_i.
//
// Quaternions are stored (x, y, z, w) with the scalar last, as in App. A.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define BDEM_HD __host__ __device__ __forceinline__

namespace bdem {

// ------------------------------------------------------------------------------------------------
// small dense helpers
// ------------------------------------------------------------------------------------------------

// packed upper triangle of an n x n symmetric matrix, row major
template <int N>
BDEM_HD constexpr int sidx(int a, int b) {
  return a <= b ? a * N - a * (a - 1) / 2 + (b - a) : b * N - b * (b - 1) / 2 + (a - b);
}

template <typename T>
struct V3 {
  T x, y, z;
};

template <typename T>
BDEM_HD V3<T> v3(T x, T y, T z) { return V3<T>{x, y, z}; }
template <typename T>
BDEM_HD V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
BDEM_HD V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
BDEM_HD V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T>
BDEM_HD T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
BDEM_HD V3<T> cross(V3<T> a, V3<T> b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
template <typename T>
BDEM_HD T comp(V3<T> a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

template <typename T>
struct Q4 {
  T x, y, z, w;  // vector part (x, y, z), scalar w
};

// Hamilton product a (x) b
template <typename T>
BDEM_HD Q4<T> qmul(Q4<T> a, Q4<T> b) {
  return {a.w * b.x + b.w * a.x + a.y * b.z - a.z * b.y, a.w * b.y + b.w * a.y + a.z * b.x - a.x * b.z,
          a.w * b.z + b.w * a.z + a.x * b.y - a.y * b.x, a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z};
}
template <typename T>
BDEM_HD Q4<T> qconj(Q4<T> a) { return {-a.x, -a.y, -a.z, a.w}; }
template <typename T>
BDEM_HD V3<T> qvec(Q4<T> a) { return {a.x, a.y, a.z}; }
template <typename T>
BDEM_HD T qdot(Q4<T> a, Q4<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
template <typename T>
BDEM_HD T qcomp(Q4<T> a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : (k == 2 ? a.z : a.w)); }

BDEM_HD Q4<double> to_q(double4 a) { return {a.x, a.y, a.z, a.w}; }
BDEM_HD V3<double> to_v(double4 a) { return {a.x, a.y, a.z}; }

// ------------------------------------------------------------------------------------------------
// shear angle function f(c) = theta^2, c = cos(theta); derivatives with respect to c
// ------------------------------------------------------------------------------------------------

struct AngleFn {
  double f, f1, f2;
};

__device__ __forceinline__ AngleFn angle2(double sin_t, double cos_t) {
  double th = atan2(sin_t, cos_t);
  AngleFn r;
  r.f = th * th;
  if (th < 1e-3) {  // Taylor series: theta/sin(theta), (sin - theta cos)/sin^3
    double t2 = th * th;
    r.f1 = -2.0 - t2 * (1.0 / 3.0) - t2 * t2 * (7.0 / 180.0);
    r.f2 = 2.0 / 3.0 + t2 * (4.0 / 15.0);
  } else {
    double s, c;
    sincos(th, &s, &c);
    r.f1 = -2.0 * th / s;
    r.f2 = 2.0 * (s - th * c) / (s * s * s);
  }
  return r;
}

// ------------------------------------------------------------------------------------------------
// bond inputs and first-order evaluation (always FP64)
// ------------------------------------------------------------------------------------------------

struct BondParams {
  V3<double> d0;   // rest direction in the frame of the common rotation
  double l0;
  double kn;       // E S / l0
  double kt;       // G S / l0 * shear_scale^2
  double kb;       // bend_twist_scale E I / l0
  double ktw;      // bend_twist_scale G J / l0
};

__device__ __forceinline__ BondParams load_bond(double4 rest, double4 stiff) {
  BondParams b;
  b.d0 = {rest.x, rest.y, rest.z};
  b.l0 = rest.w;
  b.kn = stiff.x;
  b.kt = stiff.y;
  b.kb = stiff.z;
  b.ktw = stiff.w;
  return b;
}

// Everything the Hessian needs, from one FP64 evaluation at (p_i, q_i, p_j, q_j).
struct BondEval {
  double energy, e_stretch, e_shear, e_bt;
  double g[9];          // gradient in (d, y_i, y_j)
  // stretch
  V3<double> n;
  double l, elong;      // |d|, l - l0
  // bend-twist: rho = conj(q_j) q_i = (r, s_r); kappa = K r
  V3<double> r, kappa;
  double sr;
  // shear: m = q_i + sigma q_j, c = d_hat . n
  Q4<double> m, gm;     // gm = grad_m c
  V3<double> dhat, cd;  // cd = grad_d c
  double rho_m, c, sigma;
  AngleFn fa;
  // variational midpoint form only (bond_first_order_mid): the bend-twist chain factors at the reduction
  // quaternions (ri, rj) of the state, conj(q_j^mid) ri = (ra, sa) and conj(q_i^mid) rj = (rb, sb), and
  // conj(ri) rj = (sv, ss)
  V3<double> ra, rb, sv;
  double sa, sb, ss;
};

// K r with K = ktw d0 d0^T + kb (I - d0 d0^T) (the bend-twist stiffness in the bond frame, expressed in the frame of
// q_j: t = R0 r with R0 d0 = e_x gives t^T diag(GJ, EI, EI) t / l0 = this form)
__device__ __forceinline__ V3<double> kmul(const BondParams& b, V3<double> r) {
  double a = dot(b.d0, r);
  return (b.kb) * r + ((b.ktw - b.kb) * a) * b.d0;
}

// u = R(m) d0 for an unnormalised quaternion m: (w^2 - |v|^2) d0 + 2 w (v x d0) + 2 (v.d0) v
__device__ __forceinline__ V3<double> rot_unnorm(Q4<double> m, V3<double> d0) {
  V3<double> v = qvec(m);
  return (m.w * m.w - dot(v, v)) * d0 + (2.0 * m.w) * cross(v, d0) + (2.0 * dot(v, d0)) * v;
}

// A(n) m with m^T A m = n . R(m) d0: A = [[-(n.d0) I + d0 n^T + n d0^T, d0 x n], [(d0 x n)^T, n.d0]]
__device__ __forceinline__ Q4<double> amul(V3<double> n, V3<double> d0, Q4<double> m) {
  V3<double> v = qvec(m), w = cross(d0, n);
  double ga = dot(n, d0);
  V3<double> av = (-ga) * v + dot(n, v) * d0 + dot(d0, v) * n + m.w * w;
  return {av.x, av.y, av.z, dot(w, v) + ga * m.w};
}

// G_l(q) v = vec(conj(q) (x) v) for v in R^4 (App. A nullspace operator)
template <typename T>
BDEM_HD V3<T> gl_mul(Q4<T> q, Q4<T> v) { return qvec(qmul(qconj(q), v)); }

__device__ __forceinline__ void bond_first_order(const BondParams& b, V3<double> pi, Q4<double> qi, V3<double> pj,
                                                 Q4<double> qj, BondEval& E) {
  // stretch: 1/2 kn (|d| - l0)^2
  V3<double> d = pj - pi;
  double l = sqrt(dot(d, d));
  double il = 1.0 / l;
  V3<double> n = il * d;
  double el = l - b.l0;
  E.n = n;
  E.l = l;
  E.elong = el;
  E.e_stretch = 0.5 * b.kn * el * el;
  V3<double> gd = (b.kn * el) * n;

  // bend-twist: r = vec(conj(q_j) q_i), V = 1/2 r^T K r; dr/dy_i = s_r I + [r]x, dr/dy_j = -s_r I + [r]x
  Q4<double> rho = qmul(qconj(qj), qi);
  V3<double> r = qvec(rho);
  double sr = rho.w;
  V3<double> ka = kmul(b, r);
  E.r = r;
  E.sr = sr;
  E.kappa = ka;
  E.e_bt = 0.5 * dot(r, ka);
  V3<double> rxk = cross(r, ka);
  V3<double> gyi = sr * ka - rxk;
  V3<double> gyj = (-sr) * ka - rxk;

  // shear: theta = angle(q_c (.) d0, n), q_c = m/|m|, m = q_i + sigma q_j; V = 1/2 kt theta^2
  double sg = qdot(qi, qj) < 0.0 ? -1.0 : 1.0;
  Q4<double> m = {qi.x + sg * qj.x, qi.y + sg * qj.y, qi.z + sg * qj.z, qi.w + sg * qj.w};
  double rm = qdot(m, m), irm = 1.0 / rm;
  V3<double> dh = irm * rot_unnorm(m, b.d0);  // unit
  double c = dot(dh, n);
  double st = sqrt(dot(cross(dh, n), cross(dh, n)));
  AngleFn fa = angle2(st, c);
  Q4<double> am = amul(n, b.d0, m);
  Q4<double> gm = {2.0 * irm * (am.x - c * m.x), 2.0 * irm * (am.y - c * m.y), 2.0 * irm * (am.z - c * m.z),
                   2.0 * irm * (am.w - c * m.w)};
  V3<double> cd = il * (dh - c * n);
  E.m = m;
  E.gm = gm;
  E.dhat = dh;
  E.cd = cd;
  E.rho_m = rm;
  E.c = c;
  E.sigma = sg;
  E.fa = fa;
  double hk = 0.5 * b.kt;
  E.e_shear = hk * fa.f;
  // grad_y c = G_l(q) grad_m c (dm/dy_i = G_l(q_i)^T, dm/dy_j = sigma G_l(q_j)^T)
  V3<double> cyi = gl_mul(qi, gm);
  V3<double> cyj = sg * gl_mul(qj, gm);
  double s1 = hk * fa.f1;
  gd = gd + s1 * cd;
  gyi = gyi + s1 * cyi;
  gyj = gyj + s1 * cyj;

  E.energy = E.e_stretch + E.e_shear + E.e_bt;
  E.g[0] = gd.x; E.g[1] = gd.y; E.g[2] = gd.z;
  E.g[3] = gyi.x; E.g[4] = gyi.y; E.g[5] = gyi.z;
  E.g[6] = gyj.x; E.g[7] = gyj.y; E.g[8] = gyj.z;
}

// The bond term x -> V_b((x + x_n)/2) of the variational midpoint form (Sec. 3.1; App. C): the energy and its
// Euclidean derivatives are taken at the midpoint (pvi, qvi, pvj, qvj), scaled by 1/2 per derivative, and reduced
// at the state's quaternions (ri, rj), whose retraction moves the midpoint by 1/2 G_l(r)^T y. With
// J_i = G_l(q_j^mid) G_l(ri)^T = sa I + [ra]x and J_j = -G_l(q_i^mid) G_l(rj)^T = -(sb I + [rb]x) (the bend-twist
// vector r = vec(conj(q_j) q_i) = G_l(q_j) q_i = -G_l(q_i) q_j is bilinear), the gradient is
// (1/2 grad_d V, 1/2 (J_i^T kappa + s1 G_l(ri) grad_m c), 1/2 (J_j^T kappa + s1 sigma G_l(rj) grad_m c)).
__device__ __forceinline__ void bond_first_order_mid(const BondParams& b, V3<double> pvi, Q4<double> qvi,
                                                     V3<double> pvj, Q4<double> qvj, Q4<double> ri, Q4<double> rj,
                                                     BondEval& E) {
  bond_first_order(b, pvi, qvi, pvj, qvj, E);  // every value at the midpoint
  Q4<double> ta = qmul(qconj(qvj), ri), tb = qmul(qconj(qvi), rj), tv = qmul(qconj(ri), rj);
  E.ra = qvec(ta);
  E.sa = ta.w;
  E.rb = qvec(tb);
  E.sb = tb.w;
  E.sv = qvec(tv);
  E.ss = tv.w;
  V3<double> ka = E.kappa;
  V3<double> gyi = E.sa * ka - cross(E.ra, ka);
  V3<double> gyj = cross(E.rb, ka) - E.sb * ka;
  double s1 = 0.5 * b.kt * E.fa.f1;
  V3<double> gd = (b.kn * E.elong) * E.n + s1 * E.cd;
  gyi = gyi + s1 * gl_mul(ri, E.gm);
  gyj = gyj + (s1 * E.sigma) * gl_mul(rj, E.gm);
  E.g[0] = 0.5 * gd.x; E.g[1] = 0.5 * gd.y; E.g[2] = 0.5 * gd.z;
  E.g[3] = 0.5 * gyi.x; E.g[4] = 0.5 * gyi.y; E.g[5] = 0.5 * gyi.z;
  E.g[6] = 0.5 * gyj.x; E.g[7] = 0.5 * gyj.y; E.g[8] = 0.5 * gyj.z;
}

// Euclidean gradient of the bond energy at (pi, qi, pj, qj) in (d = p_j - p_i, q_i, q_j) (11 values): grad_d,
// G_l(q_j)^T kappa + s1 grad_m c = q_j (x) (kappa, 0) + s1 grad_m c, and -q_i (x) (kappa, 0) + s1 sigma grad_m c
__device__ __forceinline__ void bond_euclid_grad(const BondParams& b, V3<double> pi, Q4<double> qi, V3<double> pj,
                                                 Q4<double> qj, double g[11]) {
  BondEval E;
  bond_first_order(b, pi, qi, pj, qj, E);
  double s1 = 0.5 * b.kt * E.fa.f1;
  V3<double> gd = (b.kn * E.elong) * E.n + s1 * E.cd;
  Q4<double> kq = {E.kappa.x, E.kappa.y, E.kappa.z, 0.0};
  Q4<double> ga = qmul(qj, kq), gb = qmul(qi, kq);
  g[0] = gd.x; g[1] = gd.y; g[2] = gd.z;
  g[3] = ga.x + s1 * E.gm.x; g[4] = ga.y + s1 * E.gm.y; g[5] = ga.z + s1 * E.gm.z; g[6] = ga.w + s1 * E.gm.w;
  double s2 = s1 * E.sigma;
  g[7] = -gb.x + s2 * E.gm.x; g[8] = -gb.y + s2 * E.gm.y; g[9] = -gb.z + s2 * E.gm.z; g[10] = -gb.w + s2 * E.gm.w;
}

// stresses of the stress fracture criterion (Sec. 3.2, Fracture Criteria) from the implicit potentials:
// |F_n| = |grad_p V_stretch| = kn |l - l0|; |F_s| = |grad_p V_shear| = |1/2 kt f'(c)| |grad_d c|; the bend-twist
// moment kappa = K r split into its twist part along the bond axis d0 and its bending part;
// sigma = |F_n| / S + |M_b| r0 / I, tau = |F_s| / S + |M_t| r0 / J with geo = (1/S, r0/I, r0/J)
__device__ __forceinline__ void bond_stress(const BondParams& b, double4 geo, V3<double> pi, Q4<double> qi,
                                            V3<double> pj, Q4<double> qj, double& sigma, double& tau) {
  BondEval E;
  bond_first_order(b, pi, qi, pj, qj, E);
  double fn = fabs(b.kn * E.elong);
  double fs = fabs(0.5 * b.kt * E.fa.f1) * sqrt(dot(E.cd, E.cd));
  double mt = dot(b.d0, E.kappa);
  V3<double> mb = E.kappa - mt * b.d0;
  sigma = fn * geo.x + sqrt(dot(mb, mb)) * geo.y;
  tau = fs * geo.x + fabs(mt) * geo.z;
}

// ------------------------------------------------------------------------------------------------
// Hessian in the 9 variables (d, y_i, y_j), packed symmetric, precision T
// ------------------------------------------------------------------------------------------------

template <typename T>
struct M3 {
  T a[3][3];
};

// 3x4 matrix of G_l(q): rows are vec(conj(q) (x) e_c) for columns c
template <typename T>
__device__ __forceinline__ void gl_matrix(Q4<double> q, T G[3][4]) {
  // G_l = [s I - t^x, -t] with t = (x, y, z), s = w
  T u = (T)q.x, v = (T)q.y, w = (T)q.z, s = (T)q.w;
  G[0][0] = s;  G[0][1] = w;  G[0][2] = -v; G[0][3] = -u;
  G[1][0] = -w; G[1][1] = s;  G[1][2] = u;  G[1][3] = -v;
  G[2][0] = v;  G[2][1] = -u; G[2][2] = s;  G[2][3] = -w;
}

template <typename T>
__device__ __forceinline__ void hadd(T* H, int a, int b, T v) {  // H[a][b] += v for a <= b (packed)
  H[sidx<9>(a, b)] += v;
}

// MID: the bond term x -> V_b((x + x_n)/2) of the variational midpoint form; E from bond_first_order_mid, (qi, qj)
// the state's quaternions at which the reduction takes place. Every second derivative of the energy enters with
// the factor 1/4, the retraction's second-order (curvature) terms with 1/2.
template <typename T, bool MID = false>
__device__ void bond_hessian(const BondParams& b, Q4<double> qi, Q4<double> qj, const BondEval& E, T* H /*45*/) {
#pragma unroll
  for (int k = 0; k < 45; ++k) H[k] = (T)0;
  // ---- stretch: kn n n^T + kn (l - l0)/l (I - n n^T) on the d block
  {
    T nn[3] = {(T)E.n.x, (T)E.n.y, (T)E.n.z};
    T kn = (T)(MID ? 0.25 * b.kn : b.kn), kp = (T)(MID ? 0.25 * (b.kn * E.elong / E.l) : b.kn * E.elong / E.l);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = a; c < 3; ++c) hadd(H, a, c, (kn - kp) * nn[a] * nn[c] + (a == c ? kp : (T)0));
  }
  // ---- bend-twist on the y blocks
  {
    T r[3] = {(T)E.r.x, (T)E.r.y, (T)E.r.z};
    T kap[3] = {(T)E.kappa.x, (T)E.kappa.y, (T)E.kappa.z};
    T sr = (T)E.sr, kr = (T)dot(E.kappa, E.r);
    T d0[3] = {(T)b.d0.x, (T)b.d0.y, (T)b.d0.z};
    T kb = (T)b.kb, kdiff = (T)(b.ktw - b.kb);
    // J_i = s_r I + [r]x, J_j = -s_r I + [r]x ; [r]x = [[0,-rz,ry],[rz,0,-rx],[-ry,rx,0]]
    T Ji[3][3], Jj[3][3], KJi[3][3], KJj[3][3];
    if constexpr (MID) {  // J_i = sa I + [ra]x, J_j = -(sb I + [rb]x)
      T ra[3] = {(T)E.ra.x, (T)E.ra.y, (T)E.ra.z}, rb[3] = {(T)E.rb.x, (T)E.rb.y, (T)E.rb.z};
      T sa = (T)E.sa, sb = (T)E.sb;
      T ax[3][3] = {{0, -ra[2], ra[1]}, {ra[2], 0, -ra[0]}, {-ra[1], ra[0], 0}};
      T bx[3][3] = {{0, -rb[2], rb[1]}, {rb[2], 0, -rb[0]}, {-rb[1], rb[0], 0}};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Ji[a][c] = ax[a][c] + (a == c ? sa : (T)0);
          Jj[a][c] = -bx[a][c] - (a == c ? sb : (T)0);
        }
    } else {
      T rx[3][3] = {{0, -r[2], r[1]}, {r[2], 0, -r[0]}, {-r[1], r[0], 0}};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Ji[a][c] = rx[a][c] + (a == c ? sr : (T)0);
          Jj[a][c] = rx[a][c] - (a == c ? sr : (T)0);
        }
    }
    // K J: K = kb I + (ktw - kb) d0 d0^T
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T di = d0[0] * Ji[0][c] + d0[1] * Ji[1][c] + d0[2] * Ji[2][c];
      T dj = d0[0] * Jj[0][c] + d0[1] * Jj[1][c] + d0[2] * Jj[2][c];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        KJi[a][c] = kb * Ji[a][c] + kdiff * d0[a] * di;
        KJj[a][c] = kb * Jj[a][c] + kdiff * d0[a] * dj;
      }
    }
    T kx[3][3] = {{0, -kap[2], kap[1]}, {kap[2], 0, -kap[0]}, {-kap[1], kap[0], 0}};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T ii = Ji[0][a] * KJi[0][c] + Ji[1][a] * KJi[1][c] + Ji[2][a] * KJi[2][c];
        T jj = Jj[0][a] * KJj[0][c] + Jj[1][a] * KJj[1][c] + Jj[2][a] * KJj[2][c];
        T ij = Ji[0][a] * KJj[0][c] + Ji[1][a] * KJj[1][c] + Ji[2][a] * KJj[2][c];
        if constexpr (MID) {
          // 1/4 J^T K J; retraction terms -1/2 (kappa.ra) I and +1/2 (kappa.rb) I on the diagonal blocks; on the
          // (y_i, y_j) block 1/4 of the bilinear term G_l(ri) Q_r((kappa, 0)) G_l(rj)^T =
          // -ss [kappa]x - sv kappa^T - kappa sv^T + (sv.kappa) I with conj(ri) rj = (sv, ss)
          T sv[3] = {(T)E.sv.x, (T)E.sv.y, (T)E.sv.z};
          T svk = (T)dot(E.sv, E.kappa), ss = (T)E.ss;
          T da = (a == c) ? (T)(0.5 * dot(E.kappa, E.ra)) : (T)0;
          T db = (a == c) ? (T)(0.5 * dot(E.kappa, E.rb)) : (T)0;
          T m = -ss * kx[a][c] - sv[a] * kap[c] - kap[a] * sv[c] + ((a == c) ? svk : (T)0);
          if (c >= a) {
            hadd(H, 3 + a, 3 + c, (T)0.25 * ii - da);
            hadd(H, 6 + a, 6 + c, (T)0.25 * jj + db);
          }
          hadd(H, 3 + a, 6 + c, (T)0.25 * (ij + m));
        } else {
          // second-order terms of the retraction: -(kappa.r) I on both diagonal blocks;
          // r kappa^T + kappa r^T - (kappa.r) I - s_r [kappa]x on the (y_i, y_j) block
          T dg = (a == c) ? kr : (T)0;
          ij += r[a] * kap[c] + kap[a] * r[c] - dg - sr * kx[a][c];
          if (c >= a) {
            hadd(H, 3 + a, 3 + c, ii - dg);
            hadd(H, 6 + a, 6 + c, jj - dg);
          }
          hadd(H, 3 + a, 6 + c, ij);
        }
      }
  }
  // ---- shear: 1/2 kt (f'' grad c grad c^T + f' Hess c)
  {
    const double hk = 0.5 * b.kt;
    const T s1 = (T)(hk * E.fa.f1), s2 = (T)(hk * E.fa.f2);
    const T il = (T)(1.0 / E.l), c = (T)E.c, irm = (T)(1.0 / E.rho_m), sg = (T)E.sigma;
    T n[3] = {(T)E.n.x, (T)E.n.y, (T)E.n.z};
    T cd[3] = {(T)E.cd.x, (T)E.cd.y, (T)E.cd.z};
    T dh[3] = {(T)E.dhat.x, (T)E.dhat.y, (T)E.dhat.z};
    T m[4] = {(T)E.m.x, (T)E.m.y, (T)E.m.z, (T)E.m.w};
    T gm[4] = {(T)E.gm.x, (T)E.gm.y, (T)E.gm.z, (T)E.gm.w};
    T d0[3] = {(T)b.d0.x, (T)b.d0.y, (T)b.d0.z};
    T nv[3] = {n[0], n[1], n[2]};
    T Gi[3][4], Gj[3][4];
    gl_matrix<T>(qi, Gi);
    gl_matrix<T>(qj, Gj);
    // full gradient of c in (d, y_i, y_j)
    T gc[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      gc[a] = cd[a];
      T si = 0, sj = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) { si += Gi[a][k] * gm[k]; sj += Gj[a][k] * gm[k]; }
      gc[3 + a] = si;
      gc[6 + a] = sg * sj;
    }
    // Hess_mm c = 2 (A - c I - m gm^T - gm m^T) / |m|^2 with A(n)
    T ga = n[0] * d0[0] + n[1] * d0[1] + n[2] * d0[2];
    T w[3] = {d0[1] * nv[2] - d0[2] * nv[1], d0[2] * nv[0] - d0[0] * nv[2], d0[0] * nv[1] - d0[1] * nv[0]};
    T Amm[4][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int k = 0; k < 3; ++k) Amm[a][k] = (a == k ? -ga : (T)0) + d0[a] * nv[k] + nv[a] * d0[k];
      Amm[a][3] = w[a];
      Amm[3][a] = w[a];
    }
    Amm[3][3] = ga;
    T Hm[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        Hm[a][k] = (T)2 * irm * (Amm[a][k] - (a == k ? c : (T)0) - m[a] * gm[k] - gm[a] * m[k]);
    // d dhat / d m = (J_u - 2 dhat m^T) / |m|^2, u = (w^2 - |v|^2) d0 + 2 w v x d0 + 2 (v.d0) v
    T Ju[3][4];
    {
      T vx = m[0], vy = m[1], vz = m[2], ws = m[3];
      T vd = vx * d0[0] + vy * d0[1] + vz * d0[2];
      T v[3] = {vx, vy, vz};
      // column s: 2 w d0 + 2 v x d0
      T vxd[3] = {vy * d0[2] - vz * d0[1], vz * d0[0] - vx * d0[2], vx * d0[1] - vy * d0[0]};
#pragma unroll
      for (int a = 0; a < 3; ++a) Ju[a][3] = (T)2 * (ws * d0[a] + vxd[a]);
      // column v_k: -2 v_k d0 + 2 w (e_k x d0) + 2 d0_k v + 2 (v.d0) e_k
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T ek[3] = {(T)(k == 0), (T)(k == 1), (T)(k == 2)};
        T exd[3] = {ek[1] * d0[2] - ek[2] * d0[1], ek[2] * d0[0] - ek[0] * d0[2], ek[0] * d0[1] - ek[1] * d0[0]};
#pragma unroll
        for (int a = 0; a < 3; ++a)
          Ju[a][k] = (T)2 * (-v[k] * d0[a] + ws * exd[a] + d0[k] * v[a] + vd * ek[a]);
      }
    }
    T Dm[3][4];  // (P / l) d dhat / dm
    {
      T dd[3][4];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) dd[a][k] = irm * (Ju[a][k] - (T)2 * dh[a] * m[k]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        T nd = n[0] * dd[0][k] + n[1] * dd[1][k] + n[2] * dd[2][k];
#pragma unroll
        for (int a = 0; a < 3; ++a) Dm[a][k] = il * (dd[a][k] - n[a] * nd);
      }
    }
    // blocks of Hess c
    T Hc[9][9];
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int k = 0; k < 9; ++k) Hc[a][k] = 0;
    // dd: -(n cd^T + cd n^T)/l - c P / l^2
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Hc[a][k] = -il * (n[a] * cd[k] + cd[a] * n[k]) - c * il * il * ((a == k ? (T)1 : (T)0) - n[a] * n[k]);
    // d-y blocks: Dm G^T
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T si = 0, sj = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) { si += Dm[a][t] * Gi[k][t]; sj += Dm[a][t] * Gj[k][t]; }
        Hc[a][3 + k] = si;
        Hc[a][6 + k] = sg * sj;
      }
    // y-y blocks: G Hm G^T with the retraction terms -(q.grad_m c) I (sigma for j)
    T GiH[3][4], GjH[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        T si = 0, sj = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) { si += Gi[a][t] * Hm[t][k]; sj += Gj[a][t] * Hm[t][k]; }
        GiH[a][k] = si;
        GjH[a][k] = sj;
      }
    T qgi = (T)(qi.x * E.gm.x + qi.y * E.gm.y + qi.z * E.gm.z + qi.w * E.gm.w);
    T qgj = (T)(qj.x * E.gm.x + qj.y * E.gm.y + qj.z * E.gm.z + qj.w * E.gm.w);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T ii = 0, jj = 0, ij = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          ii += GiH[a][t] * Gi[k][t];
          jj += GjH[a][t] * Gj[k][t];
          ij += GiH[a][t] * Gj[k][t];
        }
        Hc[3 + a][3 + k] = ii - (a == k ? qgi : (T)0);
        Hc[6 + a][6 + k] = jj - (a == k ? sg * qgj : (T)0);
        Hc[3 + a][6 + k] = sg * ij;
      }
    if constexpr (MID) {  // chain factors: 1/2 on the gradient of c, 1/4 on its Hessian, 1/2 on the retraction terms
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        gc[a] *= (T)0.5;
#pragma unroll
        for (int k = 0; k < 9; ++k) Hc[a][k] *= (T)0.25;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Hc[3 + a][3 + a] -= (T)0.25 * qgi;
        Hc[6 + a][6 + a] -= (T)0.25 * sg * qgj;
      }
    }
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int k = a; k < 9; ++k) {
        T hc = (k >= a) ? Hc[a][k] : Hc[k][a];
        hadd(H, a, k, s2 * gc[a] * gc[k] + s1 * hc);
      }
  }
}

// ------------------------------------------------------------------------------------------------
// Eigenvalue clamp (Sec. 5.2 projection) of a packed symmetric N x N matrix by cyclic Jacobi rotations.
// ------------------------------------------------------------------------------------------------

template <typename T>
struct JacobiTol;
template <>
struct JacobiTol<float> {
  static constexpr float rel = 4e-7f;
  static constexpr int sweeps = 12;
};
template <>
struct JacobiTol<double> {
  static constexpr double rel = 1e-15;
  static constexpr int sweeps = 16;
};

// The clamp is applied as H+ = H - sum_{lambda_k < 0} lambda_k v_k v_k^T, which equals V max(Lambda, 0) V^T; its
// rounding error scales with the clamped eigenvalues instead of the largest one. Rotations use the relative test
// |a_pq| > tol sqrt(|a_pp a_qq|), which resolves the small eigenpairs of graded matrices (translation stiffness far
// above rotation stiffness) to relative accuracy.
template <typename T, int N>
__device__ void eig_clamp(T* A /*packed N*(N+1)/2*/) {
  constexpr int NP = N * (N + 1) / 2;
  T H0[NP];
  T fro = 0;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    H0[k] = A[k];
    fro += A[k] * A[k];
  }
  if (!(fro > (T)0)) return;
  T V[N][N];
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int c = 0; c < N; ++c) V[a][c] = (a == c) ? (T)1 : (T)0;
  const T tol = JacobiTol<T>::rel;
  for (int sweep = 0; sweep < JacobiTol<T>::sweeps; ++sweep) {
    bool rotated = false;
#pragma unroll
    for (int p = 0; p < N - 1; ++p)
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        T apq = A[sidx<N>(p, q)];
        T app = A[sidx<N>(p, p)], aqq = A[sidx<N>(q, q)];
        if (apq != (T)0 && fabs(apq) > tol * sqrt(fabs(app * aqq))) {
          rotated = true;
          T th = (aqq - app) / ((T)2 * apq);
          T t = (th >= (T)0 ? (T)1 : (T)-1) / (fabs(th) + sqrt(th * th + (T)1));
          T cs = (T)1 / sqrt(t * t + (T)1), sn = t * cs;
          A[sidx<N>(p, p)] = app - t * apq;
          A[sidx<N>(q, q)] = aqq + t * apq;
          A[sidx<N>(p, q)] = 0;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            if (k != p && k != q) {
              T akp = A[sidx<N>(k, p)], akq = A[sidx<N>(k, q)];
              A[sidx<N>(k, p)] = cs * akp - sn * akq;
              A[sidx<N>(k, q)] = sn * akp + cs * akq;
            }
            T vkp = V[k][p], vkq = V[k][q];
            V[k][p] = cs * vkp - sn * vkq;
            V[k][q] = sn * vkp + cs * vkq;
          }
        }
      }
    if (!rotated) break;
  }
  T neg[N];
#pragma unroll
  for (int k = 0; k < N; ++k) neg[k] = A[sidx<N>(k, k)] < (T)0 ? A[sidx<N>(k, k)] : (T)0;
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int c = a; c < N; ++c) {
      T s = H0[sidx<N>(a, c)];
#pragma unroll
      for (int k = 0; k < N; ++k) s -= V[a][k] * neg[k] * V[c][k];
      A[sidx<N>(a, c)] = s;
    }
}

// ------------------------------------------------------------------------------------------------
// 6x6 symmetric positive definite inverse (block-Jacobi preconditioner) by Cholesky
// ------------------------------------------------------------------------------------------------

template <typename T>
__device__ void spd_inverse6(const T* Dp /*21 packed*/, T* Ip /*21 packed*/) {
  T L[6][6];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int c = 0; c < 6; ++c) L[a][c] = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    T s = Dp[sidx<6>(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > (T)0)) ok = false;
    T ljj = ok ? sqrt(s) : (T)1;
    L[j][j] = ljj;
    T il = (T)1 / ljj;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      T t = Dp[sidx<6>(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t * il;
    }
  }
  if (!ok) {  // not positive definite: inverse of the diagonal (entries <= 0 act as identity)
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = a; c < 6; ++c) {
        T d = Dp[sidx<6>(a, a)];
        Ip[sidx<6>(a, c)] = (a == c) ? (d > (T)0 ? (T)1 / d : (T)1) : (T)0;
      }
    return;
  }
  // W = L^{-1} (lower triangular)
  T W[6][6];
#pragma unroll
  for (int c = 0; c < 6; ++c)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i < c) { W[i][c] = 0; continue; }
      T s = (i == c) ? (T)1 : (T)0;
#pragma unroll
      for (int k = c; k < i; ++k) s -= L[i][k] * W[k][c];
      W[i][c] = s / L[i][i];
    }
  // D^{-1} = W^T W
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int c = a; c < 6; ++c) {
      T s = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s += W[k][a] * W[k][c];
      Ip[sidx<6>(a, c)] = s;
    }
}

}  // namespace bdem
