// bdem_kernels.cu -- sm_103a kernels of one implicit bonded-DEM time step (Alg. 3) and their launchers.
//
// Stage map (one Newton iteration of Alg. 3 / Alg. 2 on every active scene):
//   k_predict            xhat = x_n + dt v_n, x_0 = (phat, qhat/|qhat|)                       (Alg. 3, Sec. 3.1)
//   k_cell_* / k_contact spatial hash -> per-particle contact candidate lists at x_0             (Sec. 5.4)
//   k_bond_grad          per-bond FP64 energy gradient in (d, y_i, y_j)                       (Sec. 3.2, 4.1)
//   k_particle_grad      per-particle gather: inertia, gravity, ground, bonds, contacts -> g      (Sec. 4.1)
//   k_bond_hess          per-bond reduced Riemannian Hessian, eigen-clamp, block store     (Eq. manifold-hessian, 5.2)
//   k_particle_hess      diagonal blocks + block-Jacobi inverses                                (Sec. 5.3)
//   k_pcg                persistent cooperative PCG, per-scene FP64 dot products              (Sec. 5.3)
//   k_ls_*               exp-map retraction, term-wise energy difference, accept / halve  (Eq. manifold-update-1/2)
//   k_finish / k_fracture velocity update, tensile-strain (and stress) bond breaking     (Alg. 3, Sec. 3.2)
//   k_friction           post-step friction correction of the new velocities                  (Sec. 5.4)
//   k_zhat_*             target zhat of the variational midpoint form                    (Sec. 3.1, App. C)
//   k_amg_*, k_apcg_*    aggregation AMG coarse operators, V(1,1) cycle, AMG-preconditioned PCG stages (Sec. 5.3)
// Every reduction is deterministic: per-tile partial sums (fixed order) reduced per scene in tile order.
#include <math.h>

#include <atomic>

#include "bdem_device.cuh"
#include "bdem_internal.h"

namespace bdem {

// ================================================================================================
// helpers
// ================================================================================================

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum of K values over a 256-thread block; the result is returned to every thread
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double sh[K][kTile / 32];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][w] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kTile / 32; ++j) s += sh[k][j];
    v[k] = s;
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
struct Vec6 {
  T v[6];
};

template <typename T>
__device__ __forceinline__ Vec6<T> load6(const T* base, int i) {
  Vec6<T> r;
  const T* p = base + 6 * (size_t)i;
#pragma unroll
  for (int k = 0; k < 6; ++k) r.v[k] = p[k];
  return r;
}

// L2-coherent load (data written by other blocks of the same persistent kernel)
template <typename T>
__device__ __forceinline__ Vec6<T> load6_cg(const T* base, int i);
template <>
__device__ __forceinline__ Vec6<float> load6_cg<float>(const float* base, int i) {
  const float2* p = reinterpret_cast<const float2*>(base + 6 * (size_t)i);
  float2 a = __ldcg(p), b = __ldcg(p + 1), c = __ldcg(p + 2);
  return Vec6<float>{{a.x, a.y, b.x, b.y, c.x, c.y}};
}
template <>
__device__ __forceinline__ Vec6<double> load6_cg<double>(const double* base, int i) {
  const double2* p = reinterpret_cast<const double2*>(base + 6 * (size_t)i);
  double2 a = __ldcg(p), b = __ldcg(p + 1), c = __ldcg(p + 2);
  return Vec6<double>{{a.x, a.y, b.x, b.y, c.x, c.y}};
}

// 6-word row stores as three 8-byte (FP32) or 16-byte (FP64) stores: rows start at 24 B / 48 B multiples
template <typename T>
__device__ __forceinline__ void store6(T* base, int i, const T (&v)[6]);
template <>
__device__ __forceinline__ void store6<float>(float* base, int i, const float (&v)[6]) {
  float2* p = reinterpret_cast<float2*>(base + 6 * (size_t)i);
  p[0] = make_float2(v[0], v[1]);
  p[1] = make_float2(v[2], v[3]);
  p[2] = make_float2(v[4], v[5]);
}
template <>
__device__ __forceinline__ void store6<double>(double* base, int i, const double (&v)[6]) {
  double2* p = reinterpret_cast<double2*>(base + 6 * (size_t)i);
  p[0] = make_double2(v[0], v[1]);
  p[1] = make_double2(v[2], v[3]);
  p[2] = make_double2(v[4], v[5]);
}

template <typename T>
struct T4 {
  T x, y, z, w;
};

// Dot products of FP32 vectors accumulated without FP64 arithmetic per element: each product is split exactly into
// p + e (p = a b rounded, e = fma(a, b, -p)) and summed with error-free two-sums (the Dot2 scheme of Ogita, Rump
// and Oishi, "Accurate sum and dot product", 2005); the result carries about twice the FP32 precision and is
// converted to FP64 once per thread before the FP64 reductions. For FP64 vectors plain FP64 products are used.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    float p = a * b;
    float e = fmaf(a, b, -p);
    float s = hi + p;
    float z = s - hi;
    float t = (hi - (s - z)) + (p - z);
    hi = s;
    lo += t + e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <>
struct DotAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double value() const { return v; }
};

// ================================================================================================
// step initialisation and prediction
// ================================================================================================

__global__ void k_step_init(DevArrays d) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) {
    d.cnt->loops_newton = 0;
    d.cnt->loops_ls = 0;
    d.cnt->ls_total = 0;
    d.cnt->loops_refine = 0;
    d.cnt->loops_amg = 0;
  }
  if (s >= d.n_scenes) return;
  SceneCtl c = {};
  c.newton_active = 1;
  c.lin_res = -1.0;
  d.sc[s] = c;
}

// a step that must not be committed: a device wait gave up, the residual became non-finite, the contact arrays
// were too small (graph path) or a device-driven loop passed its cap
__device__ __forceinline__ bool step_aborted(const DevArrays& d) {
  const Counters* c = d.cnt;
  return c->timeout || c->nonfinite || c->overflow || c->runaway;
}

// the variational midpoint form (Sec. 3.1; App. C) evaluates every potential at the plain average (x + x_n)/2 of the
// state and the step's start state in R^3 x R^4 (.w of a position keeps the radius)
__device__ __forceinline__ double4 mid4(double4 a, double4 b) {
  return make_double4(0.5 * (a.x + b.x), 0.5 * (a.y + b.y), 0.5 * (a.z + b.z), a.w);
}
__device__ __forceinline__ Q4<double> midq(double4 a, double4 b) {
  return {0.5 * (a.x + b.x), 0.5 * (a.y + b.y), 0.5 * (a.z + b.z), 0.5 * (a.w + b.w)};
}
// evaluation point of the potentials for particle i at the iterate arrays x (xp or tp)
__device__ __forceinline__ double4 pot_p(const DevArrays& d, const double4* x, int i) {
  return d.midpoint ? mid4(x[i], d.x0p[i]) : x[i];
}

// xhat = x_n + dt v_n; the initial guess x_0 = (phat, qhat/|qhat|) (Alg. 3; qhat itself stays unnormalised)
__global__ void k_predict(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double4 p = d.x0p[i], q = d.x0q[i], v = d.vp[i], u = d.vq[i];
  double dt = d.dt;
  double mass = d.hp[i].w;
  double4 hp = make_double4(p.x + dt * v.x, p.y + dt * v.y, p.z + dt * v.z, mass);
  double4 hq = make_double4(q.x + dt * u.x, q.y + dt * u.y, q.z + dt * u.z, q.w + dt * u.w);
  double nq = sqrt(hq.x * hq.x + hq.y * hq.y + hq.z * hq.z + hq.w * hq.w);
  d.hp[i] = hp;
  d.hq[i] = hq;
  d.xp[i] = make_double4(hp.x, hp.y, hp.z, p.w);
  d.xq[i] = make_double4(hq.x / nq, hq.y / nq, hq.z / nq, hq.w / nq);
}

// The target of the variational midpoint form (Sec. 3.1; App. C): zhat = xhat - 1/2 M_s^{-1} dt^2 grad V(m) at the
// midpoint m = (x_{n-1} + x_n)/2 = x_n - dt v_n / 2 (x_{n-1} = x_n - dt v_n), with the Euclidean gradient (R^3 x R^4
// per particle) of the intact bonds, gravity, the ground and the step's contact candidates. The per-bond gradients
// (d, q_i, q_j: 11 values, padded to 12) go to the bond-Hessian buffer, unused until the step's first Hessian.
__global__ void __launch_bounds__(kTile) k_zhat_bonds(DevArrays d) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nb || d.bbroken[b]) return;
  int2 ij = d.bij[b];
  double hdt = 0.5 * d.dt;
  double4 pi = d.x0p[ij.x], pj = d.x0p[ij.y], vi = d.vp[ij.x], vj = d.vp[ij.y];
  double4 qi = d.x0q[ij.x], qj = d.x0q[ij.y], ui = d.vq[ij.x], uj = d.vq[ij.y];
  V3<double> mpi = {pi.x - hdt * vi.x, pi.y - hdt * vi.y, pi.z - hdt * vi.z};
  V3<double> mpj = {pj.x - hdt * vj.x, pj.y - hdt * vj.y, pj.z - hdt * vj.z};
  Q4<double> mqi = {qi.x - hdt * ui.x, qi.y - hdt * ui.y, qi.z - hdt * ui.z, qi.w - hdt * ui.w};
  Q4<double> mqj = {qj.x - hdt * uj.x, qj.y - hdt * uj.y, qj.z - hdt * uj.z, qj.w - hdt * uj.w};
  double g[11];
  bond_euclid_grad(load_bond(d.brest[b], d.bstiff[b]), mpi, mqi, mpj, mqj, g);
  double* out = reinterpret_cast<double*>(d.bM) + 12 * (size_t)b;
#pragma unroll
  for (int k = 0; k < 11; ++k) out[k] = g[k];
}

__device__ __forceinline__ double4 zhat_mid_p(const DevArrays& d, int i) {
  double4 p = d.x0p[i], v = d.vp[i];
  double hdt = 0.5 * d.dt;
  return make_double4(p.x - hdt * v.x, p.y - hdt * v.y, p.z - hdt * v.z, p.w);
}

__global__ void __launch_bounds__(kTile) k_zhat_particles(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || d.kin[i]) return;  // kinematic particles keep zhat = xhat
  double4 hp = d.hp[i], hq = d.hq[i];
  double m = hp.w;
  double4 pm = zhat_mid_p(d, i);
  double gp[3] = {-m * d.gx, -m * d.gy, -m * d.gz}, gq[4] = {0.0, 0.0, 0.0, 0.0};
  if (d.k_ground > 0.0) {
    double gd = pm.z - d.ground_z - pm.w;
    if (gd < 0.0) gp[2] += d.k_ground * gd;
  }
  const double* gall = reinterpret_cast<const double*>(d.bM);
  for (int e = d.inc_start[i]; e < d.inc_start[i + 1]; ++e) {
    int ent = d.inc2[e].x, b = ent >> 1;
    if (d.bbroken[b]) continue;
    const double* g = gall + 12 * (size_t)b;
    double sg = (ent & 1) ? 1.0 : -1.0;  // dV/dp_j = dV/dd, dV/dp_i = -dV/dd
    const double* gqe = g + ((ent & 1) ? 7 : 3);
#pragma unroll
    for (int k = 0; k < 3; ++k) gp[k] += sg * g[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) gq[k] += gqe[k];
  }
  if (d.k_self > 0.0)
    for (int e = d.c_start[i]; e < d.c_start[i + 1]; ++e) {
      double4 pj = zhat_mid_p(d, d.c_nbr[e]);
      double ex = pm.x - pj.x, ey = pm.y - pj.y, ez = pm.z - pj.z;
      double dd = sqrt(ex * ex + ey * ey + ez * ez), R = pm.w + pj.w;
      if (dd < R) {
        double f = d.k_self * (dd - R) / dd;
        gp[0] += f * ex; gp[1] += f * ey; gp[2] += f * ez;
      }
    }
  double2 cf = d.coef[i];
  d.hp[i] = make_double4(hp.x - 0.5 * gp[0] / cf.x, hp.y - 0.5 * gp[1] / cf.x, hp.z - 0.5 * gp[2] / cf.x, m);
  d.hq[i] = make_double4(hq.x - 0.5 * gq[0] / cf.y, hq.y - 0.5 * gq[1] / cf.y, hq.z - 0.5 * gq[2] / cf.y,
                         hq.w - 0.5 * gq[3] / cf.y);
}

// ================================================================================================
// spatial hash contact candidates (Sec. 5.4 repulsion between elements)
// ================================================================================================

__device__ __forceinline__ int3 cell_of(const DevArrays& d, double4 p) {
  double ih = 1.0 / d.cell_h;
  return make_int3((int)floor(p.x * ih), (int)floor(p.y * ih), (int)floor(p.z * ih));
}

__device__ __forceinline__ int hash_cell(int3 c, int scene, int size) {
  unsigned h = (unsigned)c.x * 73856093u ^ (unsigned)c.y * 19349663u ^ (unsigned)c.z * 83492791u ^
               (unsigned)scene * 2654435761u;
  return (int)(h & (unsigned)(size - 1));
}

__global__ void k_cell_count(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  int key = hash_cell(cell_of(d, d.xp[i]), d.pscene[i], d.hash_size);
  d.cell_key[i] = key;
  atomicAdd(&d.hash_count[key], 1);
}

__global__ void k_cell_fill(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  int key = d.cell_key[i];
  int pos = d.hash_start[key] + atomicAdd(&d.cnt_tmp[key], 1);
  d.hash_ids[pos] = i;
}

// order each bucket by particle index so that candidate lists do not depend on atomic order
__global__ void k_cell_sort(DevArrays d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.hash_size) return;
  int a = d.hash_start[k], b = d.hash_start[k + 1];
  for (int x = a + 1; x < b; ++x) {
    int v = d.hash_ids[x], y = x - 1;
    while (y >= a && d.hash_ids[y] > v) {
      d.hash_ids[y + 1] = d.hash_ids[y];
      --y;
    }
    d.hash_ids[y + 1] = v;
  }
}

__device__ __forceinline__ bool bonded_intact(const DevArrays& d, int i, int j) {
  for (int e = d.inc_start[i]; e < d.inc_start[i + 1]; ++e) {
    int2 ent = d.inc2[e];
    if (ent.y == j && !d.bbroken[ent.x >> 1]) return true;
  }
  return false;
}

// stage 0 counts, stage 1 fills (same traversal order: 27 cells in fixed order, buckets sorted by index)
template <int FILL>
__global__ void k_contact_scan(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double4 pi = d.xp[i];
  int si = d.pscene[i];
  int3 ci = cell_of(d, pi);
  int count = 0, out = FILL ? d.c_start[i] : 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int3 c = make_int3(ci.x + dx, ci.y + dy, ci.z + dz);
        int key = hash_cell(c, si, d.hash_size);
        for (int e = d.hash_start[key]; e < d.hash_start[key + 1]; ++e) {
          int j = d.hash_ids[e];
          if (j == i || d.pscene[j] != si) continue;
          double4 pj = d.xp[j];
          int3 cj = cell_of(d, pj);
          if (cj.x != c.x || cj.y != c.y || cj.z != c.z) continue;
          double ex = pi.x - pj.x, ey = pi.y - pj.y, ez = pi.z - pj.z;
          double lim = pi.w + pj.w + d.skin;
          if (ex * ex + ey * ey + ez * ez >= lim * lim) continue;
          if (bonded_intact(d, i, j)) continue;
          if (FILL) {
            if (out < d.c_cap) d.c_nbr[out] = j;
            ++out;
          } else {
            ++count;
          }
        }
      }
  if (!FILL) d.cnt_tmp[i] = count;
}

// capacity guard of the graph path: the host sizes the contact arrays between steps, a captured step cannot, so
// a step whose candidates do not fit records the count it needs and runs with empty candidate lists (it is not
// committed and the host repeats it after growing the arrays)
__global__ void k_contact_check(DevArrays d) {
  int need = d.c_start[d.n];
  d.cnt->overflow = (need < 0) ? 0x7fffffff : (need > d.c_cap ? need : 0);
}
__global__ void k_contact_clear(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > d.n) return;
  if (d.cnt->overflow) d.c_start[i] = 0;
}

// ---- exclusive scan of int32 counts (n) into starts (n+1) --------------------------------------------------------
__global__ void k_scan_block_sums(const int32_t* in, int n, int64_t* bsum) {
  __shared__ int64_t sh[1024];
  int i = blockIdx.x * 1024 + threadIdx.x;
  sh[threadIdx.x] = (i < n) ? in[i] : 0;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

__global__ void k_scan_top(int64_t* bsum, int nb) {  // one block: exclusive scan of nb block sums in place
  __shared__ int64_t carry;
  __shared__ int64_t sh[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    int64_t v = (i < nb) ? bsum[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int64_t t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_apply(const int32_t* in, int n, const int64_t* bsum, int nblk, int32_t* out) {
  __shared__ int64_t sh[1024];
  int i = blockIdx.x * 1024 + threadIdx.x;
  int64_t v = (i < n) ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = (int32_t)(bsum[blockIdx.x] + sh[threadIdx.x] - v);
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int32_t)bsum[nblk];
}

// ================================================================================================
// gradient
// ================================================================================================

__global__ void __launch_bounds__(kTile) k_bond_grad(DevArrays d, int all) {
  int t = blockIdx.x;
  int b = d.btile_start[t] + threadIdx.x;
  if (b >= d.btile_start[t + 1]) return;
  int s = d.btile_scene[t];
  if (!all && !d.sc[s].newton_active) return;
  double* g = d.bg + 9 * (size_t)b;
  if (d.bbroken[b]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = 0.0;
    return;
  }
  int2 ij = d.bij[b];
  BondParams bp = load_bond(d.brest[b], d.bstiff[b]);
  BondEval E;
  if (d.midpoint)
    bond_first_order_mid(bp, to_v(mid4(d.xp[ij.x], d.x0p[ij.x])), midq(d.xq[ij.x], d.x0q[ij.x]),
                         to_v(mid4(d.xp[ij.y], d.x0p[ij.y])), midq(d.xq[ij.y], d.x0q[ij.y]), to_q(d.xq[ij.x]),
                         to_q(d.xq[ij.y]), E);
  else
    bond_first_order(bp, to_v(d.xp[ij.x]), to_q(d.xq[ij.x]), to_v(d.xp[ij.y]), to_q(d.xq[ij.y]), E);
#pragma unroll
  for (int k = 0; k < 9; ++k) g[k] = E.g[k];
}

// inertia + gravity + ground (particle term) reduced gradient: (c_p (p - phat) - m g + ground, -c_q vec(conj(q) qhat));
// in the midpoint form gravity and the ground act at the midpoint with the chain factor 1/2
__device__ __forceinline__ void particle_term_grad(const DevArrays& d, int i, double g[6]) {
  double4 p = d.xp[i], q = d.xq[i], hp = d.hp[i], hq = d.hq[i];
  double2 cf = d.coef[i];
  double m = hp.w;
  double w = d.midpoint ? 0.5 : 1.0;
  double4 pv = d.midpoint ? mid4(p, d.x0p[i]) : p;
  g[0] = cf.x * (p.x - hp.x) - w * m * d.gx;
  g[1] = cf.x * (p.y - hp.y) - w * m * d.gy;
  g[2] = cf.x * (p.z - hp.z) - w * m * d.gz;
  if (d.k_ground > 0.0) {
    double gd = pv.z - d.ground_z - pv.w;
    if (gd < 0.0) g[2] += w * d.k_ground * gd;
  }
  V3<double> gy = gl_mul(to_q(q), to_q(hq));
  g[3] = -cf.y * gy.x;
  g[4] = -cf.y * gy.y;
  g[5] = -cf.y * gy.z;
}

__global__ void __launch_bounds__(kTile) k_particle_grad(DevArrays d, int mask, int all) {
  int t = blockIdx.x;
  int i = d.ptile_start[t] + threadIdx.x;
  int s = d.ptile_scene[t];
  bool act = (i < d.ptile_start[t + 1]) && (all || d.sc[s].newton_active);
  double acc[1] = {0.0};
  if (act) {
    double g[6];
    particle_term_grad(d, i, g);
    for (int e = d.inc_start[i]; e < d.inc_start[i + 1]; ++e) {
      int ent = d.inc2[e].x, b = ent >> 1;
      if (d.bbroken[b]) continue;
      const double* bg = d.bg + 9 * (size_t)b;
      if (ent & 1) {  // particle is j: dV/dp_j = dV/dd
        g[0] += bg[0]; g[1] += bg[1]; g[2] += bg[2];
        g[3] += bg[6]; g[4] += bg[7]; g[5] += bg[8];
      } else {        // particle is i: dV/dp_i = -dV/dd
        g[0] -= bg[0]; g[1] -= bg[1]; g[2] -= bg[2];
        g[3] += bg[3]; g[4] += bg[4]; g[5] += bg[5];
      }
    }
    if (d.k_self > 0.0) {
      double4 pi = pot_p(d, d.xp, i);
      double w = d.midpoint ? 0.5 : 1.0;
      for (int e = d.c_start[i]; e < d.c_start[i + 1]; ++e) {
        int j = d.c_nbr[e];
        double4 pj = pot_p(d, d.xp, j);
        double ex = pi.x - pj.x, ey = pi.y - pj.y, ez = pi.z - pj.z;
        double dd = sqrt(ex * ex + ey * ey + ez * ez), R = pi.w + pj.w;
        if (dd < R) {
          double f = w * d.k_self * (dd - R) / dd;
          g[0] += f * ex; g[1] += f * ey; g[2] += f * ez;
        }
      }
    }
    if (mask && d.kin[i])
#pragma unroll
      for (int k = 0; k < 6; ++k) g[k] = 0.0;
    double* go = d.g + 6 * (size_t)i;
#pragma unroll
    for (int k = 0; k < 6; ++k) { go[k] = g[k]; acc[0] += g[k] * g[k]; }
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) d.part_p[kPartials * t] = acc[0];
}

// ================================================================================================
// Hessian
// ================================================================================================

// MINB: resident 256-thread blocks the register budget is set for (1: up to 255 registers, as the 9x9 clamp wants;
// 2: 128 registers, twice the resident warps at the price of spills); the block size is d.bond_tile (64, 128, 256)
template <typename T, bool MID, int MINB>
__global__ void __launch_bounds__(256, MINB) k_bond_hess(DevArrays d, int all) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nb) return;
  int s = d.bscene[b];
  if (!all && !d.sc[s].newton_active) return;
  T* M = reinterpret_cast<T*>(d.bM) + 36 * (size_t)b;
  T* Eo = reinterpret_cast<T*>(d.bE) + 12 * (size_t)b;
  if (d.bbroken[b]) {
#pragma unroll
    for (int k = 0; k < 36; ++k) M[k] = (T)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) Eo[k] = (T)0;
    return;
  }
  int2 ij = d.bij[b];
  BondParams bp = load_bond(d.brest[b], d.bstiff[b]);
  Q4<double> qi = to_q(d.xq[ij.x]), qj = to_q(d.xq[ij.y]);
  BondEval E;
  if constexpr (MID)
    bond_first_order_mid(bp, to_v(mid4(d.xp[ij.x], d.x0p[ij.x])), midq(d.xq[ij.x], d.x0q[ij.x]),
                         to_v(mid4(d.xp[ij.y], d.x0p[ij.y])), midq(d.xq[ij.y], d.x0q[ij.y]), qi, qj, E);
  else
    bond_first_order(bp, to_v(d.xp[ij.x]), qi, to_v(d.xp[ij.y]), qj, E);
  T H[45];
  bond_hessian<T, MID>(bp, qi, qj, E, H);
  // orthonormal coordinates u = d / sqrt(2): H_uu = 2 H_dd, H_uy = sqrt(2) H_dy; clamp; back to d
  const T r2 = (T)1.4142135623730951;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int c = a; c < 3; ++c) H[sidx<9>(a, c)] *= (T)2;
#pragma unroll
    for (int c = 3; c < 9; ++c) H[sidx<9>(a, c)] *= r2;
  }
  eig_clamp<T, 9>(H);
  const T ir2 = (T)0.7071067811865476;
  // 1/2 A (= clamped H_dd), B/sqrt2, C/sqrt2, F, E, G
  M[0] = (T)0.5 * H[sidx<9>(0, 0)]; M[1] = (T)0.5 * H[sidx<9>(0, 1)]; M[2] = (T)0.5 * H[sidx<9>(0, 2)];
  M[3] = (T)0.5 * H[sidx<9>(1, 1)]; M[4] = (T)0.5 * H[sidx<9>(1, 2)]; M[5] = (T)0.5 * H[sidx<9>(2, 2)];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      M[6 + 3 * a + c] = ir2 * H[sidx<9>(a, 3 + c)];
      M[15 + 3 * a + c] = ir2 * H[sidx<9>(a, 6 + c)];
      M[24 + 3 * a + c] = H[sidx<9>(3 + a, 6 + c)];
    }
  M[33] = M[34] = M[35] = (T)0;
  int k = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = a; c < 3; ++c) {
      Eo[k] = H[sidx<9>(3 + a, 3 + c)];
      Eo[6 + k] = H[sidx<9>(6 + a, 6 + c)];
      ++k;
    }
}

__device__ __forceinline__ int s3(int a, int c) { return sidx<3>(a, c); }

template <typename T>
__global__ void __launch_bounds__(kTile) k_particle_hess(DevArrays d, int mask, int all) {
  int t = blockIdx.x;
  int i = d.ptile_start[t] + threadIdx.x;
  if (i >= d.ptile_start[t + 1]) return;
  int s = d.ptile_scene[t];
  if (!all && !d.sc[s].newton_active) return;
  T D[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) D[k] = (T)0;
  double4 q = d.xq[i], hq = d.hq[i];
  double4 p = pot_p(d, d.xp, i);  // the potentials' evaluation point
  double w2 = d.midpoint ? 0.25 : 1.0;
  double2 cf = d.coef[i];
  // particle term: diag(c_p I (+ k_ground e_z e_z^T), max(c_q q.qhat, 0) I), already clamped
  double cy = cf.y * (q.x * hq.x + q.y * hq.y + q.z * hq.z + q.w * hq.w);
  cy = cy > 0.0 ? cy : 0.0;
  D[sidx<6>(0, 0)] = (T)cf.x;
  D[sidx<6>(1, 1)] = (T)cf.x;
  D[sidx<6>(2, 2)] = (T)cf.x;
  if (d.k_ground > 0.0 && p.z - d.ground_z - p.w < 0.0) D[sidx<6>(2, 2)] += (T)(w2 * d.k_ground);
  D[sidx<6>(3, 3)] = (T)cy;
  D[sidx<6>(4, 4)] = (T)cy;
  D[sidx<6>(5, 5)] = (T)cy;
  const T* Mall = reinterpret_cast<const T*>(d.bM);
  const T* Eall = reinterpret_cast<const T*>(d.bE);
  for (int e = d.inc_start[i]; e < d.inc_start[i + 1]; ++e) {
    int ent = d.inc2[e].x, b = ent >> 1;
    if (d.bbroken[b]) continue;
    const T* M = Mall + 36 * (size_t)b;
    const T* Eb = Eall + 12 * (size_t)b + ((ent & 1) ? 6 : 0);
    const T* X = M + ((ent & 1) ? 15 : 6);  // Cs for j, Bs for i
    T sgn = (ent & 1) ? (T)1 : (T)-1;        // D_j += [[Ah, Cs], ...], D_i += [[Ah, -Bs], ...]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = a; c < 3; ++c) {
        D[sidx<6>(a, c)] += M[s3(a, c)];
        D[sidx<6>(3 + a, 3 + c)] += Eb[s3(a, c)];
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) D[sidx<6>(a, 3 + c)] += sgn * X[3 * a + c];
  }
  int nact = 0;
  if (d.k_self > 0.0) {
    // active contacts (overlapping candidates) compacted to the front of the particle's candidate range
    T4<T>* blk = reinterpret_cast<T4<T>*>(d.c_blk);
    int c0 = d.c_start[i];
    for (int e = c0; e < d.c_start[i + 1]; ++e) {
      int j = d.c_nbr[e];
      double4 pj = pot_p(d, d.xp, j);
      double ex = p.x - pj.x, ey = p.y - pj.y, ez = p.z - pj.z;
      double dd = sqrt(ex * ex + ey * ey + ez * ez), R = p.w + pj.w;
      if (dd < R) {  // clamped penalty Hessian k n n^T (the transverse part k (d - R)/d < 0 is removed)
        T n[3] = {(T)(ex / dd), (T)(ey / dd), (T)(ez / dd)};
        T k = (T)(w2 * d.k_self);
        blk[c0 + nact] = T4<T>{n[0], n[1], n[2], k};
        d.c_anbr[c0 + nact] = j;
        ++nact;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int c = a; c < 3; ++c) D[sidx<6>(a, c)] += k * n[a] * n[c];
      }
    }
  }
  d.c_act[i] = nact;
  if (d.k_self > 0.0) {  // per-scene count of the active entries (each tile lies inside one scene)
    unsigned m = __activemask();
    int wsum = __reduce_add_sync(m, nact);
    if ((threadIdx.x & 31) == __ffs(m) - 1 && wsum)
      atomicAdd(reinterpret_cast<unsigned long long*>(&d.sc[s].act_cur), (unsigned long long)wsum);
  }
  if (mask && d.kin[i]) {
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = a; c < 6; ++c) D[sidx<6>(a, c)] = (a == c) ? (T)1 : (T)0;
  }
  T* Do = reinterpret_cast<T*>(d.D) + kDiagStride * (size_t)i;
  T* Io = reinterpret_cast<T*>(d.Dinv) + kDiagStride * (size_t)i;
  T I[21];
  spd_inverse6<T>(D, I);
#pragma unroll
  for (int k = 0; k < 21; ++k) { Do[k] = D[k]; Io[k] = I[k]; }
#pragma unroll
  for (int k = 21; k < kDiagStride; ++k) { Do[k] = (T)0; Io[k] = (T)0; }
}

// ================================================================================================
// block-sparse matrix-vector product: y_i = D_i x_i + sum_b H_ib x_other + sum_c (-k n n^T) x_c
// ================================================================================================

// 128-bit loads of a padded block of n words (n a multiple of 4 floats / 2 doubles; 16-byte aligned)
template <int NW>
__device__ __forceinline__ void load_words(const float* src, float (&dst)[NW]) {
  static_assert(NW % 4 == 0, "float blocks load in float4");
  const float4* p = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < NW / 4; ++k) {
    float4 v = __ldg(p + k);
    dst[4 * k] = v.x; dst[4 * k + 1] = v.y; dst[4 * k + 2] = v.z; dst[4 * k + 3] = v.w;
  }
}
template <int NW>
__device__ __forceinline__ void load_words(const double* src, double (&dst)[NW]) {
  static_assert(NW % 2 == 0, "double blocks load in double2");
  const double2* p = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int k = 0; k < NW / 2; ++k) {
    double2 v = __ldg(p + k);
    dst[2 * k] = v.x; dst[2 * k + 1] = v.y;
  }
}

// a stored symmetric 6x6 block (words of type TS) times x, in arithmetic of type TA
template <typename TS, typename TA>
__device__ __forceinline__ void sym6_mul_as(const TS* Pg, const TA (&x)[6], TA (&y)[6]) {
  TS Ps[kDiagStride];
  load_words<kDiagStride>(Pg, Ps);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    TA s = 0;
#pragma unroll
    for (int c = 0; c < 6; ++c) s += (TA)Ps[sidx<6>(a, c)] * x[c];
    y[a] = s;
  }
}
// 16-byte asynchronous copy global -> shared (cp.async, L2 only) and the wait for all of this thread's copies
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most N of this thread's most recently committed copy groups are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// a block of NW words from shared memory (128-bit reads)
template <int NW>
__device__ __forceinline__ void load_words_shared(const float* src, float (&dst)[NW]) {
  const float4* p = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < NW / 4; ++k) {
    float4 v = p[k];
    dst[4 * k] = v.x; dst[4 * k + 1] = v.y; dst[4 * k + 2] = v.z; dst[4 * k + 3] = v.w;
  }
}
template <int NW>
__device__ __forceinline__ void load_words_shared(const double* src, double (&dst)[NW]) {
  const double2* p = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int k = 0; k < NW / 2; ++k) {
    double2 v = p[k];
    dst[2 * k] = v.x; dst[2 * k + 1] = v.y;
  }
}

template <typename T>
__device__ __forceinline__ void sym6_mul(const T* Pg, const T (&x)[6], T (&y)[6]) {
  sym6_mul_as<T, T>(Pg, x, y);
}

// one off-diagonal bond block (stored words of type TS) times the other endpoint's vector, added to y (arithmetic
// of type TA)
template <typename TA>
__device__ __forceinline__ void bond_block_apply(const TA (&M)[36], int side, const Vec6<TA>& xo, TA (&y)[6]);
template <typename TS, typename TA>
__device__ __forceinline__ void bond_block_mul_as(const TS* Mg, int side, const Vec6<TA>& xo, TA (&y)[6]) {
  TS Ms[36];
  load_words<36>(Mg, Ms);
  TA M[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) M[k] = (TA)Ms[k];
  bond_block_apply<TA>(M, side, xo, y);
}
// the same with the block in shared memory
template <typename T>
__device__ __forceinline__ void bond_block_mul_shared(const T* Ms, int side, const Vec6<T>& xo, T (&y)[6]) {
  T M[36];
  load_words_shared<36>(Ms, M);
  bond_block_apply<T>(M, side, xo, y);
}
template <typename TA>
__device__ __forceinline__ void bond_block_apply(const TA (&M)[36], int side, const Vec6<TA>& xo, TA (&y)[6]) {
  TA a0 = xo.v[0], a1 = xo.v[1], a2 = xo.v[2], b0 = xo.v[3], b1 = xo.v[4], b2 = xo.v[5];
  TA Ah[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) Ah[k] = M[k];
  y[0] -= Ah[0] * a0 + Ah[1] * a1 + Ah[2] * a2;
  y[1] -= Ah[1] * a0 + Ah[3] * a1 + Ah[4] * a2;
  y[2] -= Ah[2] * a0 + Ah[4] * a1 + Ah[5] * a2;
  const TA* Bs = M + 6;
  const TA* Cs = M + 15;
  const TA* F = M + 24;
  if (!side) {  // the row is i (= bi): H_ij = [[-Ah, -Cs], [Bs^T, F]]
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      y[r] -= Cs[3 * r] * b0 + Cs[3 * r + 1] * b1 + Cs[3 * r + 2] * b2;
      y[3 + r] += Bs[r] * a0 + Bs[3 + r] * a1 + Bs[6 + r] * a2 + F[3 * r] * b0 + F[3 * r + 1] * b1 + F[3 * r + 2] * b2;
    }
  } else {      // the row is j (= bj): H_ij^T = [[-Ah, Bs], [-Cs^T, F^T]]
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      y[r] += Bs[3 * r] * b0 + Bs[3 * r + 1] * b1 + Bs[3 * r + 2] * b2;
      y[3 + r] += -(Cs[r] * a0 + Cs[3 + r] * a1 + Cs[6 + r] * a2) + F[r] * b0 + F[3 + r] * b1 + F[6 + r] * b2;
    }
  }
}
template <typename T>
__device__ __forceinline__ void bond_block_mul(const T* Mg, int side, const Vec6<T>& xo, T (&y)[6]) {
  bond_block_mul_as<T, T>(Mg, side, xo, y);
}

// entry k of row i (bonds first, then active contacts), added to y
template <typename T, bool CG>
__device__ __forceinline__ void row_entry(const DevArrays& d, int i, int k, int nbond, const T* x, T (&y)[6]) {
  if (k < nbond) {
    int2 ent = d.inc2[d.inc_start[i] + k];
    Vec6<T> xo = CG ? load6_cg<T>(x, ent.y) : load6<T>(x, ent.y);
    bond_block_mul<T>(reinterpret_cast<const T*>(d.bM) + 36 * (size_t)(ent.x >> 1), ent.x & 1, xo, y);
  } else {
    int e = d.c_start[i] + (k - nbond);
    T4<T> c = reinterpret_cast<const T4<T>*>(d.c_blk)[e];
    Vec6<T> xo = CG ? load6_cg<T>(x, d.c_anbr[e]) : load6<T>(x, d.c_anbr[e]);
    T t = c.w * (c.x * xo.v[0] + c.y * xo.v[1] + c.z * xo.v[2]);
    y[0] -= t * c.x;
    y[1] -= t * c.y;
    y[2] -= t * c.z;
  }
}

// one thread per row (inspection product)
template <typename T>
__global__ void __launch_bounds__(kTile) k_matvec(DevArrays d, int mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  T y[6] = {0, 0, 0, 0, 0, 0};
  if (!(mask && d.kin[i])) {
    Vec6<T> xi = load6<T>(reinterpret_cast<const T*>(d.vp_), i);
    sym6_mul<T>(reinterpret_cast<const T*>(d.D) + kDiagStride * (size_t)i, xi.v, y);
    int nbond = d.inc_start[i + 1] - d.inc_start[i];
    int nent = nbond + (d.k_self > 0.0 ? d.c_act[i] : 0);
    for (int k = 0; k < nent; ++k) row_entry<T, false>(d, i, k, nbond, reinterpret_cast<const T*>(d.vp_), y);
  }
  store6<T>(reinterpret_cast<T*>(d.vq_), i, y);
}

// ================================================================================================
// a scene takes part in a PCG launch while its Newton loop runs and its current solve is not complete (the
// FP64-residual refinement re-solves only the scenes whose true residual is still above the target)
__device__ __forceinline__ bool pcg_on(const SceneCtl& c) { return c.newton_active && !c.pcg_skip; }

// persistent PCG (Sec. 5.3) in the Chronopoulos-Gear arrangement: per iteration one product w = H z fused with the
// three dot products (r.z, w.z, r.r) and one grid-wide reduction, then one vector update. In exact arithmetic it
// produces the iterates of the textbook PCG (x0 = 0, block-Jacobi preconditioner, stop at |r| <= eps_r |b| or the
// iteration cap): alpha_k = gamma_k / (delta_k - beta_k gamma_k / alpha_{k-1}), beta_k = gamma_k / gamma_{k-1},
// p = z + beta p, s = w + beta s (= H p), x += alpha p, r -= alpha s, z = M^-1 r.
// ================================================================================================

// the one form of device-side waiting in the library: until *word differs from old (acquire loads), for at most
// d.wait_ns nanoseconds; on giving up it sets the timeout flag (the host reports BDEM_E_TIMEOUT) and returns false
__device__ bool bounded_wait_change(const DevArrays& d, const unsigned* word, unsigned old) {
  unsigned long long t0 = global_ns();
  while (ld_acquire(word) == old) {
    __nanosleep(32);
    if (global_ns() - t0 > d.wait_ns) {
      atomicExch(&d.cnt->timeout, 1);
      return false;
    }
  }
  return true;
}

// a wait on a word that nothing writes, for testing the time limit and the host's handling of it
__global__ void k_wait_test(DevArrays d) {
  if (threadIdx.x == 0) bounded_wait_change(d, &d.cnt->never, ld_acquire(&d.cnt->never));
}

int launch_wait_test(const DevArrays& d, cudaStream_t s) {
  k_wait_test<<<1, 32, 0, s>>>(d);
  return 1;
}

// grid barrier with a bounded wait; the last block to arrive runs `work` (whole block) before releasing the others
template <typename F>
__device__ bool grid_barrier(const DevArrays& d, F&& work) {
  __shared__ int s_last, s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen = ld_acquire(&d.cnt->sync_gen);
    __threadfence();
    bool last = atomicAdd(&d.cnt->sync_count, 1u) + 1u == gridDim.x;
    s_last = last;
    s_ok = last ? 1 : (bounded_wait_change(d, &d.cnt->sync_gen, gen) ? 1 : 0);
    __threadfence();
  }
  __syncthreads();
  if (s_last) {
    work();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      d.cnt->sync_count = 0u;
      __threadfence();
      atomicAdd(&d.cnt->sync_gen, 1u);
    }
  }
  __syncthreads();
  return s_ok != 0;
}

// deterministic per-scene sums of partial slot k over a scene's tiles (particle tiles), one warp per scene
__device__ __forceinline__ double scene_partial(const DevArrays& d, int s, int k, int lane) {
  int a = d.ptile_begin[s], b = d.ptile_begin[s + 1];
  double v = 0.0;
  for (int t = a + lane; t < b; t += 32) v += __ldcg(d.part_p + kPartials * t + k);
  return warp_sum(v);
}

// the PCG decision of one scene from its reduced dots (run by a single thread): convergence test, then the
// Chronopoulos-Gear step lengths; returns whether the scene keeps iterating
// the fields of a scene's control block that the PCG decision reads, loaded together from L2 (other blocks wrote
// them since this SM last cached them) and issued before the partial dots so that both loads overlap
struct PcgPrev {
  int newton_active, pcg_active, it;
  double eps_r, bnorm, rz, alpha, beta, pq, thr2;
};
__device__ __forceinline__ PcgPrev load_prev(const SceneCtl* c) {
  return {__ldcg(&c->newton_active) && !__ldcg(&c->pcg_skip), __ldcg(&c->pcg_active), __ldcg(&c->pcg_iters),
          __ldcg(&c->eps_r),
          __ldcg(&c->bnorm), __ldcg(&c->rz), __ldcg(&c->alpha), __ldcg(&c->beta), __ldcg(&c->pq),
          __ldcg(&c->pcg_thr2)};
}

// the PCG decision of one scene from its reduced dots: convergence test, then the Chronopoulos-Gear step lengths.
// Updates the scene's solver state in place and returns whether the scene keeps iterating.
// FP64 division and square root are long dependent sequences on this part, so the decision keeps them off its
// critical path: the stopping test compares squares (|r| <= eps_r |b| as rho <= eps_r^2 |b|^2), and the
// reciprocals of the previous gamma and alpha (needed for beta and for the denominator) are taken when the state is
// loaded, while the block still waits for the partial dots; one division (alpha) remains on the path.
struct PcgState {
  int newton_active, pcg_active, it;
  double eps_r, bnorm, rz, alpha, beta, pq;
  double thr2, inv_rz, inv_alpha;  // (eps_r |b|)^2; 1 / previous gamma; 1 / previous alpha
};
__device__ __forceinline__ void pcg_prepare(PcgState& s) {
  s.inv_rz = s.it > 0 ? 1.0 / s.rz : 0.0;
  s.inv_alpha = s.it > 0 ? s.pq * s.inv_rz : 0.0;  // 1 / alpha = den / gamma
}
__device__ bool pcg_decision(PcgState& s, double gam, double del, double rho, int k_iter, int pcg_max) {
  if (!s.newton_active) return false;
  if (k_iter == 0) {
    s.thr2 = s.eps_r * s.eps_r * rho;
    s.bnorm = sqrt(rho);
    s.it = 0;
    s.pcg_active = 1;
  }
  if (!s.pcg_active) return false;
  bool stop = !(rho > s.thr2) || s.it >= pcg_max;
  if (!stop) {
    double beta = (s.it == 0) ? 0.0 : gam * s.inv_rz;
    double den = (s.it == 0) ? del : del - beta * gam * s.inv_alpha;
    if (!(den > 0.0) || !(gam > 0.0)) {
      stop = true;  // breakdown: no further decrease along this Krylov space
    } else {
      s.beta = beta;
      s.alpha = gam / den;
      s.rz = gam;
      s.pq = den;
      s.it += 1;
    }
  }
  if (stop) s.pcg_active = 0;
  return !stop;
}

__device__ __forceinline__ void store_pcg_state(SceneCtl* c, const PcgState& s) {
  c->bnorm = s.bnorm;
  c->pcg_thr2 = s.thr2;
  c->pcg_iters = s.it;
  c->pcg_active = s.pcg_active;
  c->alpha = s.alpha;
  c->beta = s.beta;
  c->rz = s.rz;
  c->pq = s.pq;
}

// the decision of one scene whose solver state lives in its control block (run by a single thread)
__device__ bool pcg_decide_scene(const DevArrays& d, SceneCtl* c, PcgPrev pv, double gam, double del, double rho,
                                 int k_iter) {
  PcgState s = {pv.newton_active, pv.pcg_active, pv.it, pv.eps_r, pv.bnorm, pv.rz, pv.alpha, pv.beta, pv.pq,
                pv.thr2, 0.0, 0.0};
  if (!s.newton_active) return false;
  pcg_prepare(s);
  bool go = pcg_decision(s, gam, del, rho, k_iter, d.pcg_max);
  store_pcg_state(c, s);
  return go;
}

// few scenes: the last block to reach the barrier sums every scene's partial dots in a fixed order, and every block
// then takes the same decisions from those sums with its own copy of the solver state (no control-block reads after
// the barrier); block 0 keeps the control blocks current for the host
constexpr int kLocalScenes = kLocalPcgScenes;
struct LocalPcg {
  PcgState st[kLocalScenes];
  double acc[3][kTile / 32];
  int n_active;
};

// the scenes' sums of this iteration's partial dots, formed by the last block to reach the barrier (threads over the
// scene's segments, then the warps' sums in order) into slots n_seg + scene, so that the other blocks read three
// words per scene instead of every segment's partials (all blocks reading every slot makes those lines an L2 hot spot)
__device__ void pcg_local_totals(const DevArrays& d, const int* ss, LocalPcg& L) {
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int s = 0; s < d.n_scenes; ++s) {
    int a = ss[s], b = ss[s + 1];
    double gam = 0.0, del = 0.0, rho = 0.0;
    for (int t = a + threadIdx.x; t < b; t += blockDim.x) {
      gam += __ldcg(d.part_s + kPartials * t);
      del += __ldcg(d.part_s + kPartials * t + 1);
      rho += __ldcg(d.part_s + kPartials * t + 2);
    }
    gam = warp_sum(gam);
    del = warp_sum(del);
    rho = warp_sum(rho);
    if (lane == 0) {
      L.acc[0][warp] = gam;
      L.acc[1][warp] = del;
      L.acc[2][warp] = rho;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double G = 0.0, D = 0.0, R = 0.0;
      for (int w = 0; w < nw; ++w) {
        G += L.acc[0][w];
        D += L.acc[1][w];
        R += L.acc[2][w];
      }
      double* tot = d.part_s + kPartials * ((size_t)d.n_seg + s);
      tot[0] = G;
      tot[1] = D;
      tot[2] = R;
    }
    __syncthreads();
  }
}

// every scene's decision from the sums (after the barrier that formed them), one thread per scene, the same in every
// block
__device__ void pcg_decide_local(const DevArrays& d, int k_iter, LocalPcg& L) {
  bool go = false;
  if (threadIdx.x < d.n_scenes) {
    const int s = threadIdx.x;
    const double* tot = d.part_s + kPartials * ((size_t)d.n_seg + s);
    const double G = __ldcg(tot), D = __ldcg(tot + 1), R = __ldcg(tot + 2);
    pcg_prepare(L.st[s]);
    go = pcg_decision(L.st[s], G, D, R, k_iter, d.pcg_max);
    if (blockIdx.x == 0) store_pcg_state(d.sc + s, L.st[s]);
  }
  const int active = __syncthreads_count(go);
  if (threadIdx.x == 0) L.n_active = active;
  __syncthreads();
}

// many scenes (DevArrays::pcg_dist): each block decides the scenes its own rows belong to (the scenes of its product
// and update segments, a contiguous range of at most kDistPcgScenes) with its own copy of their solver state, after a
// plain barrier. Every block sums a scene's partial dots in the same fixed order (one warp per scene, lanes over the
// scene's segments, then the warp's shuffle tree), so all copies agree. The block holding a scene's first product
// segment keeps its control block current and counts it, if it iterates on, in the active-scene counter of the
// iteration (dist_active[k % 3]), which every block reads after the iteration's next barrier; block 0 clears the
// counter two iterations ahead.
struct DistPcg {
  PcgState st[kDistPcgScenes];
  int lo, n;  // first scene of the block's range, scenes in it
};

// the block's scene range and its copies of their solver states; block 0 also writes the final state of the scenes
// without rows (no block decides them) and clears the active-scene counters
__device__ void pcg_dist_init(const DevArrays& d, int seg0, int seg1, int useg0, int useg1, DistPcg& D) {
  if (threadIdx.x == 0) {
    int lo = 0x7fffffff, hi = -1;
    if (seg1 > seg0) {
      lo = min(lo, d.seg_scene[seg0]);
      hi = max(hi, d.seg_scene[seg1 - 1]);
    }
    if (useg1 > useg0) {
      lo = min(lo, d.useg_scene[useg0]);
      hi = max(hi, d.useg_scene[useg1 - 1]);
    }
    int n = hi >= 0 ? hi - lo + 1 : 0;
    if (n > kDistPcgScenes) {  // never taken: the host enables this path only when every range fits
      atomicExch(&d.cnt->timeout, 1);
      n = kDistPcgScenes;
    }
    D.lo = hi >= 0 ? lo : 0;
    D.n = n;
    if (blockIdx.x == 0) {
      d.cnt->dist_active[0] = d.cnt->dist_active[1] = d.cnt->dist_active[2] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x < D.n) {
    const SceneCtl* c = d.sc + D.lo + threadIdx.x;
    int on = pcg_on(*c);
    D.st[threadIdx.x] = PcgState{on, on, 0, c->eps_r, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  }
  if (blockIdx.x == 0)
    for (int s = threadIdx.x; s < d.n_scenes; s += blockDim.x)
      if (d.scene_seg[s] == d.scene_seg[s + 1] && pcg_on(d.sc[s]))
        store_pcg_state(d.sc + s, PcgState{1, 0, 0, d.sc[s].eps_r, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0});
}

// this block's decisions of iteration k_iter (after a plain grid barrier); ss: the scenes' first product segments
__device__ void pcg_decide_dist(const DevArrays& d, int k_iter, const int* ss, int seg0, int seg1, DistPcg& D) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < D.n; j += nw) {
    const int s = D.lo + j, a = ss[s], b = ss[s + 1];
    if (lane == 0) pcg_prepare(D.st[j]);  // overlaps the partial loads below
    double gam = 0.0, del = 0.0, rho = 0.0;
    for (int t = a + lane; t < b; t += 32) {
      gam += __ldcg(d.part_s + kPartials * t);
      del += __ldcg(d.part_s + kPartials * t + 1);
      rho += __ldcg(d.part_s + kPartials * t + 2);
    }
    gam = warp_sum(gam);
    del = warp_sum(del);
    rho = warp_sum(rho);
    if (lane == 0 && a < b) {
      const bool go = pcg_decision(D.st[j], gam, del, rho, k_iter, d.pcg_max);
      if (a >= seg0 && a < seg1) {  // this block holds the scene's first product segment
        store_pcg_state(d.sc + s, D.st[j]);
        if (go) atomicAdd(&d.cnt->dist_active[k_iter % 3], 1);
      }
    }
  }
  __syncthreads();
}

// many scenes whose solves stop after different numbers of iterations (DevArrays::pcg_even): at every iteration the
// rows of the scenes still iterating are split evenly over the grid (a block's share may span several scenes: its
// segments), every block keeps every scene's solver state and takes every scene's decision from the same sums in the
// same order, so the blocks whose scenes have stopped take rows of the others instead of waiting at the barriers. A
// segment's partial dots go to slot blockIdx.x * kEvenPcgSegs + its index in the block; a scene's slots are found
// from the iteration's active-row prefix (the blocks whose shares its rows fall in, its index in the first of them)
// and summed in block order by the last block to reach the barrier, so that every other block reads one sum per
// scene (all blocks reading every slot made the slots' L2 lines a hot spot: 19-36 us per iteration on 64 scenes).
struct EvenPcg {
  PcgState st[kEvenPcgScenes];
  int off[kEvenPcgScenes + 1];    // first row of each scene
  int pre[kEvenPcgScenes + 1];    // rows of the iterating scenes before each scene (this iteration)
  int arank[kEvenPcgScenes + 1];  // iterating scenes with rows before each scene
  int4 seg[kEvenPcgSegs];          // this block's segments: scene, first row, end row
  int nseg, n_active;
};
size_t pcg_even_bytes() { return sizeof(EvenPcg); }

// the first of the N active rows in block b's share (shares [floor(b N / G), floor((b + 1) N / G)))
__device__ __forceinline__ long long even_share(long long b, long long N, long long G) { return b * N / G; }
// the block whose share holds active row x: the largest b with floor(b N / G) <= x
__device__ __forceinline__ int even_block_of(long long x, long long N, long long G) {
  return (int)(((x + 1) * G - 1) / N);
}

__device__ void pcg_even_init(const DevArrays& d, EvenPcg& E) {
  for (int s = threadIdx.x; s <= d.n_scenes; s += blockDim.x) E.off[s] = d.ptile_start[d.ptile_begin[s]];
  for (int s = threadIdx.x; s < d.n_scenes; s += blockDim.x) {
    const SceneCtl* c = d.sc + s;
    int on = pcg_on(*c);
    E.st[s] = PcgState{on, on, 0, c->eps_r, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  }
}

// this iteration's active-row prefix and the block's segments (thread 0; the block waits)
__device__ void pcg_even_partition(const DevArrays& d, EvenPcg& E) {
  if (threadIdx.x == 0) {
    const int S = d.n_scenes;
    int p = 0, r = 0;
    for (int s = 0; s < S; ++s) {
      E.pre[s] = p;
      E.arank[s] = r;
      const int rows = E.off[s + 1] - E.off[s];
      if (E.st[s].pcg_active && rows > 0) {
        p += rows;
        ++r;
      }
    }
    E.pre[S] = p;
    E.arank[S] = r;
    E.n_active = 0;
    E.nseg = 0;
    const long long N = p, G = gridDim.x;
    const long long lo = N > 0 ? even_share(blockIdx.x, N, G) : 0, hi = N > 0 ? even_share(blockIdx.x + 1, N, G) : 0;
    if (hi > lo) {
      int a = 0, b = S - 1;  // the first scene with rows after lo: smallest s with pre[s + 1] > lo
      while (a < b) {
        const int m = (a + b) >> 1;
        if (E.pre[m + 1] > lo) b = m;
        else a = m + 1;
      }
      for (int s = a; s < S && E.pre[s] < hi; ++s) {
        const long long x0 = lo > E.pre[s] ? lo : E.pre[s], x1 = hi < E.pre[s + 1] ? hi : E.pre[s + 1];
        if (x1 <= x0) continue;
        if (E.nseg < kEvenPcgSegs)
          E.seg[E.nseg++] = make_int4(s, E.off[s] + (int)(x0 - E.pre[s]), E.off[s] + (int)(x1 - E.pre[s]), 0);
        else
          atomicExch(&d.cnt->timeout, 1);  // never taken: the host enables this path only when every share fits
      }
    }
  }
  __syncthreads();
}

// the scenes' sums of this iteration's partial dots, formed by the last block to reach the barrier (all of its
// threads): a group of threads per scene (a power of two, up to 32) strides over the scene's slots in block order
// and adds its partial sums by a shuffle tree; the sums go to slot G * kEvenPcgSegs + scene
__device__ void pcg_even_totals(const DevArrays& d, const EvenPcg& E) {
  const long long N = E.pre[d.n_scenes], G = gridDim.x;
  int T = 1;
  while (T < 32 && 2 * T * d.n_scenes <= (int)blockDim.x) T *= 2;
  const int lane = threadIdx.x & 31, t = threadIdx.x % T, ngroups = blockDim.x / T;
  const unsigned gmask = (T == 32 ? 0xffffffffu : ((1u << T) - 1u)) << (lane & ~(T - 1));
  for (int s = threadIdx.x / T; s < d.n_scenes; s += ngroups) {
    double gam = 0.0, del = 0.0, rho = 0.0;
    const int a = E.pre[s], b = E.pre[s + 1];
    if (b > a) {
      const int blo = even_block_of(a, N, G), bhi = even_block_of(b - 1, N, G);
      // the scene's index among block blo's segments: the scenes with rows between blo's first row and this one
      const long long x = even_share(blo, N, G);
      int u = 0, v = s;
      while (u < v) {
        const int m = (u + v) >> 1;
        if (E.pre[m + 1] > x) v = m;
        else u = m + 1;
      }
      const int k0 = E.arank[s] - E.arank[u];
      for (int bb = blo + t; bb <= bhi; bb += T) {
        // with fewer active rows than blocks some shares are empty and wrote no slot
        if (N < G && even_share(bb + 1, N, G) <= even_share(bb, N, G)) continue;
        const int slot = bb * kEvenPcgSegs + (bb == blo ? k0 : 0);
        gam += __ldcg(d.part_s + kPartials * slot);
        del += __ldcg(d.part_s + kPartials * slot + 1);
        rho += __ldcg(d.part_s + kPartials * slot + 2);
      }
    }
    for (int o = T / 2; o >= 1; o >>= 1) {
      gam += __shfl_xor_sync(gmask, gam, o, T);
      del += __shfl_xor_sync(gmask, del, o, T);
      rho += __shfl_xor_sync(gmask, rho, o, T);
    }
    if (t == 0) {
      double* tot = d.part_s + kPartials * ((size_t)G * kEvenPcgSegs + s);
      tot[0] = gam;
      tot[1] = del;
      tot[2] = rho;
    }
  }
}

// every scene's decision of iteration k_iter from the sums (after the barrier that formed them), the same in every
// block, one thread per scene
__device__ void pcg_decide_even(const DevArrays& d, int k_iter, EvenPcg& E) {
  const size_t base = (size_t)gridDim.x * kEvenPcgSegs;
  for (int s = threadIdx.x; s < d.n_scenes; s += blockDim.x) {
    PcgState& st = E.st[s];
    double gam = 0.0, del = 0.0, rho = 0.0;
    if (E.pre[s + 1] > E.pre[s]) {
      const double* tot = d.part_s + kPartials * (base + s);
      gam = __ldcg(tot);
      del = __ldcg(tot + 1);
      rho = __ldcg(tot + 2);
    }
    pcg_prepare(st);
    const bool go = pcg_decision(st, gam, del, rho, k_iter, d.pcg_max);
    if (blockIdx.x == 0) store_pcg_state(d.sc + s, st);
    if (go) atomicAdd(&E.n_active, 1);
  }
  __syncthreads();
}

constexpr int kBlockScene = 64;  // scenes with more PCG segments than this are reduced by the whole block

// per-scene decision after the fused product, run by the last block to reach the barrier. The partial dots of a
// scene's segments are summed in a fixed order: by one warp (lanes stride over the segments) for a scene with at
// most kBlockScene segments, by the whole block (threads stride, then warps in order) for a larger one, so that a
// large scene costs one round of loads instead of a serial walk over its segments. sseg: the scenes' first
// segments staged in shared memory (NULL: read them from global memory).
__device__ __noinline__ void pcg_decide(const DevArrays& d, int k_iter, const int* sseg) {
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int s_active[kTile / 32];
  __shared__ double s_acc[3][kTile / 32];
  __shared__ int s_big[kTile], s_nbig;
  if (threadIdx.x == 0) s_nbig = 0;
  __syncthreads();
  const int* ss = sseg ? sseg : d.scene_seg;
  int active = 0;
  for (int s = warp; s < d.n_scenes; s += nw) {
    int a = ss[s], b = ss[s + 1];
    if (b - a > kBlockScene) {
      if (lane == 0) {
        int k = atomicAdd(&s_nbig, 1);  // list order is irrelevant: each scene is reduced on its own
        if (k < kTile) s_big[k] = s;
      }
      continue;
    }
    PcgPrev pv;
    if (lane == 0) pv = load_prev(d.sc + s);
    double gam = 0.0, del = 0.0, rho = 0.0;
    for (int t = a + lane; t < b; t += 32) {
      gam += __ldcg(d.part_s + kPartials * t);
      del += __ldcg(d.part_s + kPartials * t + 1);
      rho += __ldcg(d.part_s + kPartials * t + 2);
    }
    gam = warp_sum(gam);
    del = warp_sum(del);
    rho = warp_sum(rho);
    if (lane == 0 && pcg_decide_scene(d, d.sc + s, pv, gam, del, rho, k_iter)) ++active;
  }
  if (lane == 0) s_active[warp] = active;
  __syncthreads();
  int nbig = s_nbig < kTile ? s_nbig : kTile;  // at most pcg_grid / kBlockScene + 1 scenes, far below kTile
  int big_active = 0;
  for (int k = 0; k < nbig; ++k) {
    int s = s_big[k];
    int a = ss[s], b = ss[s + 1];
    PcgPrev pv;
    if (threadIdx.x == 0) pv = load_prev(d.sc + s);
    double gam = 0.0, del = 0.0, rho = 0.0;
    for (int t = a + threadIdx.x; t < b; t += blockDim.x) {
      gam += __ldcg(d.part_s + kPartials * t);
      del += __ldcg(d.part_s + kPartials * t + 1);
      rho += __ldcg(d.part_s + kPartials * t + 2);
    }
    gam = warp_sum(gam);
    del = warp_sum(del);
    rho = warp_sum(rho);
    if (lane == 0) {
      s_acc[0][warp] = gam;
      s_acc[1][warp] = del;
      s_acc[2][warp] = rho;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double G = 0.0, D = 0.0, R = 0.0;
      for (int w = 0; w < nw; ++w) {
        G += s_acc[0][w];
        D += s_acc[1][w];
        R += s_acc[2][w];
      }
      if (pcg_decide_scene(d, d.sc + s, pv, G, D, R, k_iter)) ++big_active;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int tot = big_active;
    for (int w = 0; w < nw; ++w) tot += s_active[w];
    d.cnt->n_active = tot;
  }
}

// MODE (DevArrays::pcg_mode) selects how the product reaches the bond blocks:
//   0: each lane loads its own entries' blocks from L2/DRAM (128-bit loads); row descriptors and incidence entries are
//      read from global memory at every product;
//   1: as 0, with the block's row descriptors and incidence entries staged in shared memory once per solve (for
//      systems whose block row ranges fit: about 25 KB per 1,000 rows of degree 12);
//   2: row descriptors staged once per solve; the product runs in waves of one entry per lane, and before each wave
//      the warp copies the wave's 32 bond blocks into shared memory with 16-byte cp.async copies in which
//      consecutive lanes take consecutive 16-byte pieces of the same block, so that a copy request covers a few cache
//      lines instead of one line per lane (with per-lane loads the L1 data pipe, not DRAM, bounds the product); each
//      lane then multiplies its own entry's block from shared memory;
//   3: as 2 with two slot buffers per warp: the copies of wave w + 1 are in flight while wave w is multiplied
// resident blocks the register budget is set for: 4 of 256 threads per SM in FP32 (64 registers), 3 with the
// cooperative product (85 registers; its shared-memory slots leave room for 3 or 4) and 2 with its double-buffered
// form, 2 in FP64 (1 double-buffered)
template <typename T, int MODE>
constexpr int pcg_min_blocks() {
  return sizeof(T) == 4 ? (MODE == 3 ? 2 : MODE == 2 ? 3 : 4) : (MODE == 3 ? 1 : 2);
}

template <typename T, int G, int MODE>
__global__ void __launch_bounds__(kTile, pcg_min_blocks<T, MODE>()) k_pcg(DevArrays d, int rhs_from_g, int mask) {
  constexpr bool STAGED = MODE == 1;  // incidence entries in shared memory
  // row descriptors in shared memory (always with MODE 1; with MODE 2 and 3 when the block's rows fit beside its SM's
  // other blocks, else read from L2 at every product)
  const bool ROWS = MODE == 1 || (MODE >= 2 && d.pcg_rows_sm);
  constexpr bool COOP = MODE >= 2;
  constexpr int NB = MODE == 3 ? 2 : 1;  // slot buffers per warp of the cooperative product
  T* X = reinterpret_cast<T*>(d.vx);
  T* R = reinterpret_cast<T*>(d.vr);
  T* Z = reinterpret_cast<T*>(d.vz);
  T* P = reinterpret_cast<T*>(d.vp_);
  T* W = reinterpret_cast<T*>(d.vq_);
  T* S = reinterpret_cast<T*>(d.vs);
  const T* Dinv = reinterpret_cast<const T*>(d.Dinv);
  const T* Dm = reinterpret_cast<const T*>(d.D);
  const int seg0 = d.block_seg[blockIdx.x], seg1 = d.block_seg[blockIdx.x + 1];
  const T zero6[6] = {0, 0, 0, 0, 0, 0};
  // per-row descriptors of the block's rows, fixed for the whole solve: first incidence entry, bond count,
  // active-contact count with the kinematic flag in bit 30, first contact entry
  // and the incidence entries of those rows (staged once; every product reads them from shared memory)
  extern __shared__ int4 s_rows[];
  int2* s_ent = reinterpret_cast<int2*>(s_rows + d.pcg_max_rows);
  // COOP: this warp's 32 block slots (36 words each) after the row descriptors
  T* s_blk = reinterpret_cast<T*>(s_rows + (ROWS ? d.pcg_max_rows : 1)) + (threadIdx.x >> 5) * NB * 32 * 36;
  const int R0 = d.seg_row[seg0], R1 = d.seg_row[seg1];
  const int E0 = d.inc_start[R0], E1 = d.inc_start[R1];
  // row descriptor: first incidence entry (relative to the block's first when staged), bond count, active-contact
  // count with the kinematic flag in bit 30, first contact entry
  auto row_desc = [&](int i) {
    int a = d.inc_start[i];
    int na = (d.k_self > 0.0) ? d.c_act[i] : 0;
    int kin = (mask && d.kin[i]) ? (1 << 30) : 0;
    return make_int4(STAGED ? a - E0 : a, d.inc_start[i + 1] - a, na | kin, d.c_start[i]);
  };
  if (ROWS)
    for (int i = R0 + threadIdx.x; i < R1; i += blockDim.x) s_rows[i - R0] = row_desc(i);
  if (STAGED)
    for (int e = E0 + threadIdx.x; e < E1; e += blockDim.x) s_ent[e - E0] = d.inc2[e];
  const int2* ent_all = STAGED ? s_ent : d.inc2;
  __shared__ int s_sseg[kTile + 1];  // first PCG segment of each scene, for the decision (up to kTile scenes)
  const bool sseg_ok = d.n_scenes <= kTile;
  if (sseg_ok)
    for (int x = threadIdx.x; x <= d.n_scenes; x += blockDim.x) s_sseg[x] = d.scene_seg[x];
  __shared__ LocalPcg s_loc;
  const bool local = d.n_scenes <= kLocalScenes;
  if (local && threadIdx.x < d.n_scenes) {
    const SceneCtl* c = d.sc + threadIdx.x;
    int on = pcg_on(*c);
    s_loc.st[threadIdx.x] = PcgState{on, on, 0, c->eps_r, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  }
  // the elementwise phases (init and B) use the equal-rows partition: their cost is per row, while the product's
  // partition balances rows against incidence entries
  const int useg0 = d.ublock_seg[blockIdx.x], useg1 = d.ublock_seg[blockIdx.x + 1];
  __shared__ DistPcg s_dist;
  const bool even = !local && d.pcg_even;
  const bool dist = !local && !even && d.pcg_dist;
  if (dist) pcg_dist_init(d, seg0, seg1, useg0, useg1, s_dist);
  EvenPcg& E = *reinterpret_cast<EvenPcg*>(reinterpret_cast<char*>(s_rows) + d.pcg_even_off);
  if (even) pcg_even_init(d, E);
  __syncthreads();
  // ---- init: x = p = s = 0, r = b, z = M^-1 r
  for (int g = useg0; g < useg1; ++g) {
    int sc = d.useg_scene[g];
    if (!pcg_on(d.sc[sc])) continue;
    for (int i = d.useg_row[g] + threadIdx.x; i < d.useg_row[g + 1]; i += blockDim.x) {
      T r[6], z[6];
      if (rhs_from_g) {
        const double* gg = d.g + 6 * (size_t)i;
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = (T)(-gg[k]);
      } else {
        Vec6<T> b = load6<T>(R, i);
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = b.v[k];
      }
      if (mask && d.kin[i])
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = (T)0;
      sym6_mul<T>(Dinv + kDiagStride * (size_t)i, r, z);
      store6<T>(X, i, zero6);
      store6<T>(P, i, zero6);
      store6<T>(S, i, zero6);
      store6<T>(R, i, r);
      store6<T>(Z, i, z);
    }
  }
  if (!grid_barrier(d, [] {})) return;
  const int sub = threadIdx.x % G, grp = threadIdx.x / G, rows_per_pass = blockDim.x / G;
  for (int k_iter = 0;; ++k_iter) {
    if (even) pcg_even_partition(d, E);
    // ---- A: w = H z, gamma = r.z, delta = w.z, rho = r.r (per segment, deterministic)
    const int nseg = even ? E.nseg : seg1 - seg0;
    for (int q = 0; q < nseg; ++q) {
      const int g = even ? blockIdx.x * kEvenPcgSegs + q : seg0 + q;  // partial slot
      const int sc = even ? E.seg[q].x : d.seg_scene[g];
      bool act = local  ? s_loc.st[sc].pcg_active != 0
                 : even ? E.st[sc].pcg_active != 0
                 : dist ? s_dist.st[sc - s_dist.lo].pcg_active != 0
                        : pcg_on(d.sc[sc]) && (k_iter == 0 || __ldcg(&d.sc[sc].pcg_active));
      DotAcc<T> dg, dd, dr;
      if (act) {
        const int r0 = even ? E.seg[q].y : d.seg_row[g], r1 = even ? E.seg[q].z : d.seg_row[g + 1];
        for (int base = r0; base < r1; base += rows_per_pass) {
          int i = base + grp;
          bool valid = i < r1;
          T y[6] = {0, 0, 0, 0, 0, 0};
          int4 rd = valid ? (ROWS ? s_rows[i - R0] : row_desc(i)) : make_int4(0, 0, 1 << 30, 0);
          bool live = valid && !(rd.z & (1 << 30));
          if (live && sub == 0) {
            Vec6<T> zi = load6_cg<T>(Z, i);
            sym6_mul<T>(Dm + kDiagStride * (size_t)i, zi.v, y);
          }
          const T* Mall = reinterpret_cast<const T*>(d.bM);
          if (COOP) {
            // waves of one entry per lane (warp-uniform count: every lane takes part in the copies)
            const int lane = threadIdx.x & 31;
            const int nwave = __reduce_max_sync(0xffffffffu, live ? (rd.y + G - 1) / G : 0);
            constexpr int PP = 36 * (int)sizeof(T) / 16;  // 16-byte pieces of one block
            constexpr int PW = 16 / (int)sizeof(T);       // words of one piece
            // copies of one wave's blocks (bond -1: no entry in that lane's slot) into a 32-slot buffer, as one group
            auto copy_wave = [&](int bond, T* buf) {
#pragma unroll
              for (int m = 0; m < PP; ++m) {
                const int p = lane + 32 * m, slot = p / PP, q = p - slot * PP;
                const int bs = __shfl_sync(0xffffffffu, bond, slot);
                if (bs >= 0) cp_async16(buf + 36 * slot + PW * q, Mall + 36 * (size_t)bs + PW * q);
              }
              cp_async_commit();
            };
            // the wave's incidence entry and the other endpoint's z are loaded one wave ahead, so that the wait of a
            // wave covers only its block copies
            bool has = live && sub < rd.y;
            int2 e = has ? __ldg(d.inc2 + rd.x + sub) : make_int2(-2, 0);
            Vec6<T> xo;
            if (has) xo = load6_cg<T>(Z, e.y);
            if (NB == 2 && nwave > 0) copy_wave(e.x >> 1, s_blk);
            for (int w = 0; w < nwave; ++w) {
              T* cur = s_blk + (NB == 2 ? (w & 1) * 32 * 36 : 0);
              if (NB == 1) copy_wave(e.x >> 1, cur);
              const int kn = (w + 1) * G + sub;
              const bool hasn = live && kn < rd.y;
              const int2 en = hasn ? __ldg(d.inc2 + rd.x + kn) : make_int2(-2, 0);
              Vec6<T> xon;
              if (hasn) xon = load6_cg<T>(Z, en.y);
              if (NB == 2) {
                // the next wave's copies go to the other buffer, whose previous wave every lane has finished reading
                if (w + 1 < nwave) copy_wave(en.x >> 1, s_blk + ((w + 1) & 1) * 32 * 36);
                else cp_async_commit();  // an empty group keeps the count of pending groups uniform
                cp_async_wait_group<1>();
              } else {
                cp_async_wait_group<0>();
              }
              __syncwarp();
              if (has) bond_block_mul_shared<T>(cur + 36 * lane, e.x & 1, xo, y);
              __syncwarp();  // every lane has read its slot before a later wave's copies overwrite it
              has = hasn;
              e = en;
              xo = xon;
            }
          } else if (live) {
            const int2* ent = ent_all + rd.x;
#pragma unroll 2
            for (int k = sub; k < rd.y; k += G) {
              int2 e = ent[k];
              Vec6<T> xo = load6_cg<T>(Z, e.y);
              bond_block_mul<T>(Mall + 36 * (size_t)(e.x >> 1), e.x & 1, xo, y);
            }
          }
          if (live) {
            int nact = rd.z & ((1 << 30) - 1);
            for (int k = sub; k < nact; k += G) {
              int e = rd.w + k;
              T4<T> c = reinterpret_cast<const T4<T>*>(d.c_blk)[e];
              Vec6<T> xo = load6_cg<T>(Z, d.c_anbr[e]);
              T t = c.w * (c.x * xo.v[0] + c.y * xo.v[1] + c.z * xo.v[2]);
              y[0] -= t * c.x;
              y[1] -= t * c.y;
              y[2] -= t * c.z;
            }
          }
#pragma unroll
          for (int o = G / 2; o >= 1; o >>= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) y[k] += __shfl_xor_sync(0xffffffffu, y[k], o, G);
          if (valid && sub == 0) {
            store6<T>(W, i, y);
            Vec6<T> zi = load6_cg<T>(Z, i), ri = load6_cg<T>(R, i);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              dg.add(ri.v[k], zi.v[k]);
              dd.add(y[k], zi.v[k]);
              dr.add(ri.v[k], ri.v[k]);
            }
          }
        }
      }
      double acc[3] = {dg.value(), dd.value(), dr.value()};
      block_sum<3>(acc);
      if (threadIdx.x == 0) {
        d.part_s[kPartials * g] = acc[0];
        d.part_s[kPartials * g + 1] = acc[1];
        d.part_s[kPartials * g + 2] = acc[2];
      }
    }
    if (local) {
      if (!grid_barrier(d, [&] { pcg_local_totals(d, s_sseg, s_loc); })) return;
      pcg_decide_local(d, k_iter, s_loc);
      if (s_loc.n_active == 0 || __ldcg(&d.cnt->timeout)) break;
    } else if (even) {
      if (!grid_barrier(d, [&] { pcg_even_totals(d, E); })) return;
      pcg_decide_even(d, k_iter, E);
      if (E.n_active == 0 || __ldcg(&d.cnt->timeout)) break;
    } else if (dist) {
      if (!grid_barrier(d, [] {})) return;
      pcg_decide_dist(d, k_iter, sseg_ok ? s_sseg : d.scene_seg, seg0, seg1, s_dist);
    } else {
      if (!grid_barrier(d, [&] { pcg_decide(d, k_iter, sseg_ok ? s_sseg : nullptr); })) return;
      if (__ldcg(&d.cnt->n_active) == 0 || __ldcg(&d.cnt->timeout)) break;
    }
    // ---- B: p = z + beta p, s = w + beta s, x += alpha p, r -= alpha s, z = M^-1 r (with the even re-partition
    // over the product's segments, else over the equal-rows partition)
    const int nuseg = even ? E.nseg : useg1 - useg0;
    for (int q = 0; q < nuseg; ++q) {
      const int g = useg0 + q;
      const int sc = even ? E.seg[q].x : d.useg_scene[g];
      const int u0 = even ? E.seg[q].y : d.useg_row[g], u1 = even ? E.seg[q].z : d.useg_row[g + 1];
      T al, be;
      if (even) {
        if (!E.st[sc].pcg_active) continue;
        al = (T)E.st[sc].alpha;
        be = (T)E.st[sc].beta;
      } else if (local) {
        if (!s_loc.st[sc].pcg_active) continue;
        al = (T)s_loc.st[sc].alpha;
        be = (T)s_loc.st[sc].beta;
      } else if (dist) {
        const PcgState& st = s_dist.st[sc - s_dist.lo];
        if (!st.pcg_active) continue;
        al = (T)st.alpha;
        be = (T)st.beta;
      } else {
        if (!pcg_on(d.sc[sc]) || !__ldcg(&d.sc[sc].pcg_active)) continue;
        al = (T)__ldcg(&d.sc[sc].alpha);
        be = (T)__ldcg(&d.sc[sc].beta);
      }
      for (int i = u0 + threadIdx.x; i < u1; i += blockDim.x) {
        Vec6<T> z = load6_cg<T>(Z, i), w = load6_cg<T>(W, i), p = load6_cg<T>(P, i), s = load6_cg<T>(S, i);
        Vec6<T> x = load6_cg<T>(X, i), r = load6_cg<T>(R, i);
        T pn[6], sn[6], xn[6], rn[6], zn[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          pn[k] = z.v[k] + be * p.v[k];
          sn[k] = w.v[k] + be * s.v[k];
          xn[k] = x.v[k] + al * pn[k];
          rn[k] = r.v[k] - al * sn[k];
        }
        sym6_mul<T>(Dinv + kDiagStride * (size_t)i, rn, zn);
        store6<T>(P, i, pn);
        store6<T>(S, i, sn);
        store6<T>(X, i, xn);
        store6<T>(R, i, rn);
        store6<T>(Z, i, zn);
      }
    }
    if (!grid_barrier(d, [] {})) return;
    if (dist) {  // every block's decisions of this iteration are counted
      if (__ldcg(&d.cnt->dist_active[k_iter % 3]) == 0 || __ldcg(&d.cnt->timeout)) break;
      if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt->dist_active[(k_iter + 1) % 3] = 0;
    }
  }
}

// ================================================================================================
// fused PCG (MODE 4): the same Chronopoulos-Gear iterates with one grid barrier per iteration instead of two. The
// vector update of iteration k (p = z + beta p, s = w + beta s, x += alpha p, r -= alpha s, z = M^-1 r) and the product
// w = H z of iteration k + 1 run in one phase: every block updates its own rows (the product partition's) and keeps
// their new z in shared memory, and recomputes the new z of its halo rows (the rows outside its range its bond entries
// reference) from their previous r, s, w and block-Jacobi inverse, so that no other block's update has to be waited
// for. r, s and w alternate between two buffers (the halo recomputation of iteration k reads the buffers of
// iteration k - 1 while their owners write those of iteration k); x, p and z are only read by their owners and stay
// in place. Active-contact neighbours outside the block recompute their z the same way. The bond blocks reach shared
// memory as in MODE 2 (one wave of 32 entries per warp, warp-cooperative 16-byte copies).
// ================================================================================================

template <typename T>
__device__ __forceinline__ void pcg_update_z(const T* Dinv, int i, const T* Rp, const T* Sp, const T* Wp, T al, T be,
                                             T (&z)[6]) {
  Vec6<T> r = load6_cg<T>(Rp, i), s = load6_cg<T>(Sp, i), w = load6_cg<T>(Wp, i);
  T rn[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) rn[k] = r.v[k] - al * (w.v[k] + be * s.v[k]);
  sym6_mul<T>(Dinv + kDiagStride * (size_t)i, rn, z);
}

template <typename T, int G>
__global__ void __launch_bounds__(kTile, sizeof(T) == 4 ? 2 : 1) k_pcg_fused(DevArrays d, int rhs_from_g, int mask) {
  T* X = reinterpret_cast<T*>(d.vx);
  T* Zg = reinterpret_cast<T*>(d.vz);
  T* P = reinterpret_cast<T*>(d.vp_);
  T* const R_0 = reinterpret_cast<T*>(d.vr);
  T* const R_1 = reinterpret_cast<T*>(d.vr2);
  T* const S_0 = reinterpret_cast<T*>(d.vs);
  T* const S_1 = reinterpret_cast<T*>(d.vs2);
  T* const W_0 = reinterpret_cast<T*>(d.vq_);
  T* const W_1 = reinterpret_cast<T*>(d.vq2);
  const T* Dinv = reinterpret_cast<const T*>(d.Dinv);
  const T* Dm = reinterpret_cast<const T*>(d.D);
  const T* Mall = reinterpret_cast<const T*>(d.bM);
  const int seg0 = d.block_seg[blockIdx.x], seg1 = d.block_seg[blockIdx.x + 1];
  const int R0 = d.seg_row[seg0], R1 = d.seg_row[seg1], nown = R1 - R0;
  const int h0 = d.halo_start[blockIdx.x], h1 = d.halo_start[blockIdx.x + 1];
  extern __shared__ int4 s_rows[];                                      // [pcg_max_rows] row descriptors
  T* s_z = reinterpret_cast<T*>(s_rows + d.pcg_max_rows);              // [pcg_max_zslots][6]: own rows, then halo
  T* s_blk = s_z + 6 * (size_t)d.pcg_max_zslots + (threadIdx.x >> 5) * 32 * 36;  // this warp's 32 block slots
  for (int i = R0 + threadIdx.x; i < R1; i += blockDim.x) {
    int a = d.inc_start[i];
    int na = (d.k_self > 0.0) ? d.c_act[i] : 0;
    int kin = (mask && d.kin[i]) ? (1 << 30) : 0;
    s_rows[i - R0] = make_int4(a, d.inc_start[i + 1] - a, na | kin, d.c_start[i]);
  }
  __shared__ int s_sseg[kTile + 1];
  const bool sseg_ok = d.n_scenes <= kTile;
  if (sseg_ok)
    for (int x = threadIdx.x; x <= d.n_scenes; x += blockDim.x) s_sseg[x] = d.scene_seg[x];
  __shared__ LocalPcg s_loc;
  const bool local = d.n_scenes <= kLocalScenes;
  if (local && threadIdx.x < d.n_scenes) {
    const SceneCtl* c = d.sc + threadIdx.x;
    int on = pcg_on(*c);
    s_loc.st[threadIdx.x] = PcgState{on, on, 0, c->eps_r, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  }
  // every phase of this kernel works on the block's own rows (halo and contact neighbours are in the same scenes)
  __shared__ DistPcg s_dist;
  const bool dist = !local && d.pcg_dist;
  if (dist) pcg_dist_init(d, seg0, seg1, 0, 0, s_dist);
  __syncthreads();
  const T zero6[6] = {0, 0, 0, 0, 0, 0};
  // ---- init (own rows): x = p = s = 0, r = b, z = M^-1 r
  for (int g = seg0; g < seg1; ++g) {
    if (!pcg_on(d.sc[d.seg_scene[g]])) continue;
    for (int i = d.seg_row[g] + threadIdx.x; i < d.seg_row[g + 1]; i += blockDim.x) {
      T r[6], z[6];
      if (rhs_from_g) {
        const double* gg = d.g + 6 * (size_t)i;
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = (T)(-gg[k]);
      } else {
        Vec6<T> b = load6<T>(R_0, i);
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = b.v[k];
      }
      if (mask && d.kin[i])
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = (T)0;
      sym6_mul<T>(Dinv + kDiagStride * (size_t)i, r, z);
      store6<T>(X, i, zero6);
      store6<T>(P, i, zero6);
      store6<T>(S_0, i, zero6);
      store6<T>(R_0, i, r);
      store6<T>(Zg, i, z);
    }
  }
  if (!grid_barrier(d, [] {})) return;
  const int sub = threadIdx.x % G, grp = threadIdx.x / G, rows_per_pass = blockDim.x / G, lane = threadIdx.x & 31;
  constexpr int PP = 36 * (int)sizeof(T) / 16;
  constexpr int PW = 16 / (int)sizeof(T);
  for (int k_iter = 0;; ++k_iter) {
    // this iteration's r, s, w buffers and the previous iteration's
    const bool odd = k_iter & 1;
    T* const Rc = odd ? R_1 : R_0;
    T* const Sc = odd ? S_1 : S_0;
    T* const Wc = odd ? W_1 : W_0;
    T* const Rp = odd ? R_0 : R_1;
    T* const Sp = odd ? S_0 : S_1;
    T* const Wp = odd ? W_0 : W_1;
    // the scalars of the decision that closed the previous iteration, per scene
    auto coef = [&](int sc, T& al, T& be) -> bool {
      if (local) {
        al = (T)s_loc.st[sc].alpha;
        be = (T)s_loc.st[sc].beta;
        return s_loc.st[sc].pcg_active != 0;
      }
      if (dist) {
        const PcgState& st = s_dist.st[sc - s_dist.lo];
        al = (T)st.alpha;
        be = (T)st.beta;
        return st.pcg_active != 0;
      }
      al = (T)__ldcg(&d.sc[sc].alpha);
      be = (T)__ldcg(&d.sc[sc].beta);
      return pcg_on(d.sc[sc]) && (k_iter == 0 || __ldcg(&d.sc[sc].pcg_active));
    };
    // ---- U: own rows' update (from iteration 1 on) with their new z kept in shared memory; halo rows' new z
    for (int g = seg0; g < seg1; ++g) {
      T al, be;
      if (!coef(d.seg_scene[g], al, be)) continue;
      for (int i = d.seg_row[g] + threadIdx.x; i < d.seg_row[g + 1]; i += blockDim.x) {
        T zn[6];
        if (k_iter == 0) {
          Vec6<T> z = load6_cg<T>(Zg, i);
#pragma unroll
          for (int k = 0; k < 6; ++k) zn[k] = z.v[k];
        } else {
          Vec6<T> z = load6_cg<T>(Zg, i), w = load6_cg<T>(Wp, i), p = load6_cg<T>(P, i);
          Vec6<T> s = load6_cg<T>(Sp, i), x = load6_cg<T>(X, i), r = load6_cg<T>(Rp, i);
          T pn[6], sn[6], xn[6], rn[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            pn[k] = z.v[k] + be * p.v[k];
            sn[k] = w.v[k] + be * s.v[k];
            xn[k] = x.v[k] + al * pn[k];
            rn[k] = r.v[k] - al * sn[k];
          }
          sym6_mul<T>(Dinv + kDiagStride * (size_t)i, rn, zn);
          store6<T>(P, i, pn);
          store6<T>(Sc, i, sn);
          store6<T>(X, i, xn);
          store6<T>(Rc, i, rn);
          store6<T>(Zg, i, zn);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) s_z[6 * (i - R0) + k] = zn[k];
      }
    }
    for (int h = h0 + threadIdx.x; h < h1; h += blockDim.x) {
      const int j = d.halo_rows[h];
      T al, be;
      if (!coef(d.pscene[j], al, be)) continue;
      T zn[6];
      if (k_iter == 0) {
        Vec6<T> z = load6_cg<T>(Zg, j);
#pragma unroll
        for (int k = 0; k < 6; ++k) zn[k] = z.v[k];
      } else {
        pcg_update_z<T>(Dinv, j, Rp, Sp, Wp, al, be, zn);
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) s_z[6 * (nown + h - h0) + k] = zn[k];
    }
    __syncthreads();
    // ---- A: w = H z from the shared z, gamma = r.z, delta = w.z, rho = r.r (per segment, deterministic)
    for (int g = seg0; g < seg1; ++g) {
      const int sc = d.seg_scene[g];
      T al, be;
      const bool act = coef(sc, al, be);
      DotAcc<T> dg, dd, dr;
      if (act) {
        const int r0 = d.seg_row[g], r1 = d.seg_row[g + 1];
        for (int base = r0; base < r1; base += rows_per_pass) {
          const int i = base + grp;
          const bool valid = i < r1;
          T y[6] = {0, 0, 0, 0, 0, 0};
          const int4 rd = valid ? s_rows[i - R0] : make_int4(0, 0, 1 << 30, 0);
          const bool live = valid && !(rd.z & (1 << 30));
          Vec6<T> zi;
          if (valid)
#pragma unroll
            for (int k = 0; k < 6; ++k) zi.v[k] = s_z[6 * (i - R0) + k];
          if (live && sub == 0) sym6_mul<T>(Dm + kDiagStride * (size_t)i, zi.v, y);
          const int nwave = __reduce_max_sync(0xffffffffu, live ? (rd.y + G - 1) / G : 0);
          for (int w = 0; w < nwave; ++w) {
            const int k = w * G + sub;
            const bool has = live && k < rd.y;
            const int2 e = has ? __ldg(d.inc2_loc + rd.x + k) : make_int2(-2, 0);
            const int bond = e.x >> 1;
#pragma unroll
            for (int m = 0; m < PP; ++m) {
              const int p = lane + 32 * m, slot = p / PP, q = p - slot * PP;
              const int bs = __shfl_sync(0xffffffffu, bond, slot);
              if (bs >= 0) cp_async16(s_blk + 36 * slot + PW * q, Mall + 36 * (size_t)bs + PW * q);
            }
            cp_async_commit();
            Vec6<T> xo;
            if (has)
#pragma unroll
              for (int c = 0; c < 6; ++c) xo.v[c] = s_z[6 * e.y + c];
            cp_async_wait_group<0>();
            __syncwarp();
            if (has) bond_block_mul_shared<T>(s_blk + 36 * lane, e.x & 1, xo, y);
            __syncwarp();
          }
          if (live) {
            const int nact = rd.z & ((1 << 30) - 1);
            for (int k = sub; k < nact; k += G) {
              const int e = rd.w + k;
              const int c = d.c_anbr[e];
              T4<T> cb = reinterpret_cast<const T4<T>*>(d.c_blk)[e];
              Vec6<T> xo;
              if (c >= R0 && c < R1) {
#pragma unroll
                for (int q = 0; q < 6; ++q) xo.v[q] = s_z[6 * (c - R0) + q];
              } else if (k_iter == 0) {
                xo = load6_cg<T>(Zg, c);
              } else {
                T a2, b2;
                coef(d.pscene[c], a2, b2);
                pcg_update_z<T>(Dinv, c, Rp, Sp, Wp, a2, b2, xo.v);
              }
              T t = cb.w * (cb.x * xo.v[0] + cb.y * xo.v[1] + cb.z * xo.v[2]);
              y[0] -= t * cb.x;
              y[1] -= t * cb.y;
              y[2] -= t * cb.z;
            }
          }
#pragma unroll
          for (int o = G / 2; o >= 1; o >>= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) y[k] += __shfl_xor_sync(0xffffffffu, y[k], o, G);
          if (valid && sub == 0) {
            store6<T>(Wc, i, y);
            Vec6<T> ri = load6_cg<T>(Rc, i);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              dg.add(ri.v[k], zi.v[k]);
              dd.add(y[k], zi.v[k]);
              dr.add(ri.v[k], ri.v[k]);
            }
          }
        }
      }
      double acc[3] = {dg.value(), dd.value(), dr.value()};
      block_sum<3>(acc);
      if (threadIdx.x == 0) {
        d.part_s[kPartials * g] = acc[0];
        d.part_s[kPartials * g + 1] = acc[1];
        d.part_s[kPartials * g + 2] = acc[2];
      }
    }
    if (local) {
      if (!grid_barrier(d, [&] { pcg_local_totals(d, s_sseg, s_loc); })) return;
      pcg_decide_local(d, k_iter, s_loc);
      if (s_loc.n_active == 0 || __ldcg(&d.cnt->timeout)) break;
    } else if (dist) {
      if (!grid_barrier(d, [] {})) return;
      pcg_decide_dist(d, k_iter, sseg_ok ? s_sseg : d.scene_seg, seg0, seg1, s_dist);
      // the previous iteration's decisions are all counted (this iteration's may still be under way): none went on
      // means this iteration updated and multiplied nothing, and neither will the next
      if ((k_iter > 0 && __ldcg(&d.cnt->dist_active[(k_iter - 1) % 3]) == 0) || __ldcg(&d.cnt->timeout)) break;
      if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt->dist_active[(k_iter + 1) % 3] = 0;
    } else {
      if (!grid_barrier(d, [&] { pcg_decide(d, k_iter, sseg_ok ? s_sseg : nullptr); })) return;
      if (__ldcg(&d.cnt->n_active) == 0 || __ldcg(&d.cnt->timeout)) break;
    }
  }
}

// ================================================================================================
// per-scene reductions outside the PCG (Newton residual, descent check, line search decision)
// ================================================================================================

__global__ void k_scene_reduce(DevArrays d, int mode, unsigned long long cond) {
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int s_cnt[32];
  int cnt = 0;
  for (int s = warp; s < d.n_scenes; s += nw) {
    SceneCtl* c = d.sc + s;
    double v = scene_partial(d, s, 0, lane);
    if (mode == RED_LS) {
      int a = d.btile_begin[s], b = d.btile_begin[s + 1];
      double w = 0.0;
      for (int t = a + lane; t < b; t += 32) w += d.part_b[kPartials * t];
      v += warp_sum(w);
    }
    if (lane != 0) continue;
    if (mode == RED_GRAD) {
      if (!c->newton_active) continue;
      c->act_cur = 0;
      if (!isfinite(v)) {
        c->newton_active = 0;
        c->status = 6;
        d.cnt->nonfinite = 1;
        continue;
      }
      double gn = sqrt(v);
      if (c->newton_iters == 0) c->g0 = gn;  // first residual of the step
      c->gnorm = gn;
      if (gn <= d.tol * c->g0 || gn <= d.tol_abs) {
        c->newton_active = 0;
      } else if (c->newton_iters >= d.newton_max) {
        c->newton_active = 0;
        c->status = 4;
      } else {
        c->eps_r = fmin(0.5, sqrt(gn));
        c->pcg_skip = 0;
        ++cnt;
      }
    } else if (mode == RED_GDX) {
      if (!c->newton_active) continue;
      c->gdx = v;
      c->use_neg_grad = d.first_order || !(v < 0.0);  // first order (Alg. 1): always -grad f
      c->ls_alpha = 1.0;
      c->ls_state = 0;
      c->pad1 = 0;  // halvings in this line search
      c->newton_iters += 1;
      int its = d.refine ? c->pcg_acc : c->pcg_iters;  // every round of a refined solve
      c->pcg_total += its;
      c->act_pcg += c->act_cur * (long long)its;
      ++cnt;
    } else if (mode == RED_LS) {
      if (!c->newton_active || c->ls_state != 0) continue;
      c->dphi = v;
      if (v <= 0.0) {
        c->ls_state = 1;
      } else {
        if (c->pad1 >= d.ls_max) {
          c->ls_state = 2;
          c->status = c->status > 5 ? c->status : 5;
          c->newton_active = 0;
        } else {
          c->pad1 += 1;
          c->ls_halvings += 1;
          c->ls_alpha *= 0.5;
          ++cnt;
        }
      }
    } else if (mode == RED_REFINE0 || mode == RED_REFINE) {
      // after a PCG launch: v = |b - H x64|^2 of the accumulated FP64 solution. The solve is complete when the true
      // residual meets the Newton solve's target eps_r |b|, after d.refine rounds, when a round did not reduce the
      // residual, or when the solve has used pcg_max iterations; otherwise the next round solves H d = r with the
      // relative target eps_r |b| / |r|, which reaches the solve's target where the FP32 recurrence is exact
      if (!pcg_on(*c)) continue;
      double res = sqrt(v);
      if (mode == RED_REFINE0) {
        c->eps_out = c->eps_r;
        c->b_out = c->bnorm;
        c->pcg_acc = c->pcg_iters;
        c->refine_round = 0;
      } else {
        c->pcg_acc += c->pcg_iters;
      }
      double tgt = c->eps_out * c->b_out;
      bool worse = mode == RED_REFINE && !(res < c->res64);
      c->lin_res = c->b_out > 0.0 ? res / c->b_out : 0.0;
      c->res64 = res;
      if (!(res > tgt) || c->refine_round >= d.refine || worse || c->pcg_acc >= d.pcg_max || !isfinite(res)) {
        c->pcg_skip = 1;
      } else {
        c->refine_round += 1;
        c->refine_total += 1;
        c->eps_r = tgt / res;
        ++cnt;
      }
    } else if (mode == RED_FORCE_ACTIVE) {
      c->newton_active = 1;
      c->pcg_skip = 0;
      ++cnt;
    } else if (mode == RED_CAND) {
      int a = d.ptile_start[d.ptile_begin[s]], b = d.ptile_start[d.ptile_begin[s + 1]];
      c->pad2 = d.c_start[b] - d.c_start[a];
    }
  }
  if (lane == 0) s_cnt[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < nw; ++w) tot += s_cnt[w];
    if (mode == RED_LS) d.cnt->n_pending = tot;
    else d.cnt->n_active = tot;
    if (cond) {  // device-driven loop of the step graph: the same decisions as the host-driven loop
      unsigned go = tot > 0;
      if (mode == RED_GRAD) {
        int trips = ++d.cnt->loops_newton;
        if (go && trips > d.newton_max + 2) d.cnt->runaway = 1;
      } else if (mode == RED_GDX) {
        d.cnt->loops_ls = 0;
      } else if (mode == RED_LS) {
        int trials = ++d.cnt->loops_ls;
        d.cnt->ls_total += 1;
        if (trials >= d.ls_max + 2) go = 0;
      } else if (mode == RED_REFINE) {
        d.cnt->loops_refine += 1;
      }
      if (step_aborted(d)) go = 0;
      cudaGraphSetConditional((cudaGraphConditionalHandle)cond, go);
    }
  }
}

// ================================================================================================
// FP64 products and the FP64-residual refinement of the mixed-precision Newton solve
// ================================================================================================

// row i of y = H x in FP64 arithmetic on the stored blocks of type T (x [N][6] FP64, internal order). The products of
// FP32 words in FP64 are exact, so the only rounding is that of the FP64 sums: this is the true product of the
// matrix the PCG iterates with.
template <typename T>
__device__ __forceinline__ void row_product64(const DevArrays& d, int i, const double* x, double (&y)[6]) {
  Vec6<double> xi = load6<double>(x, i);
  sym6_mul_as<T, double>(reinterpret_cast<const T*>(d.D) + kDiagStride * (size_t)i, xi.v, y);
  const int a = d.inc_start[i], nbond = d.inc_start[i + 1] - a;
  const T* Mall = reinterpret_cast<const T*>(d.bM);
  for (int k = 0; k < nbond; ++k) {
    int2 e = d.inc2[a + k];
    Vec6<double> xo = load6<double>(x, e.y);
    bond_block_mul_as<T, double>(Mall + 36 * (size_t)(e.x >> 1), e.x & 1, xo, y);
  }
  if (d.k_self > 0.0) {
    const int na = d.c_act[i];
    for (int k = 0; k < na; ++k) {
      int e = d.c_start[i] + k;
      T4<T> c = reinterpret_cast<const T4<T>*>(d.c_blk)[e];
      Vec6<double> xo = load6<double>(x, d.c_anbr[e]);
      double cx = (double)c.x, cy = (double)c.y, cz = (double)c.z;
      double t = (double)c.w * (cx * xo.v[0] + cy * xo.v[1] + cz * xo.v[2]);
      y[0] -= t * cx;
      y[1] -= t * cy;
      y[2] -= t * cz;
    }
  }
}

// y = H x in FP64 (inspection product; mask: kinematic rows give 0)
template <typename T>
__global__ void __launch_bounds__(kTile) k_matvec64(DevArrays d, const double* x, double* y, int mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (!(mask && d.kin[i])) row_product64<T>(d, i, x, v);
#pragma unroll
  for (int k = 0; k < 6; ++k) y[6 * (size_t)i + k] = v[k];
}

// x64 = x (first) or x64 += x for the rows of the scenes that solved in the last PCG launch
template <typename T>
__global__ void k_refine_acc(DevArrays d, int first) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || !pcg_on(d.sc[d.pscene[i]])) return;
  Vec6<T> x = load6<T>(reinterpret_cast<const T*>(d.vx), i);
  double* o = d.x64 + 6 * (size_t)i;
#pragma unroll
  for (int k = 0; k < 6; ++k) o[k] = (first ? 0.0 : o[k]) + (double)x.v[k];
}

// r = b - H x64 in FP64 for the rows of the scenes that solved in the last PCG launch (b = -g, or b64 for an
// inspection solve; kinematic rows 0), r rounded into vr as the next launch's right-hand side, per-tile |r|^2
template <typename T>
__global__ void __launch_bounds__(kTile) k_refine_res(DevArrays d) {
  int t = blockIdx.x;
  int i = d.ptile_start[t] + threadIdx.x;
  double acc[1] = {0.0};
  if (i < d.ptile_start[t + 1] && pcg_on(d.sc[d.ptile_scene[t]])) {
    double r[6] = {0, 0, 0, 0, 0, 0};
    if (!d.kin[i]) {
      double y[6];
      row_product64<T>(d, i, d.x64, y);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        double b = d.b64 ? d.b64[6 * (size_t)i + k] : -d.g[6 * (size_t)i + k];
        r[k] = b - y[k];
        acc[0] += r[k] * r[k];
      }
    }
    T rt[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) rt[k] = (T)r[k];
    store6<T>(reinterpret_cast<T*>(d.vr), i, rt);
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) d.part_p[kPartials * t] = acc[0];
}

// partial g . dx for the descent check
template <typename T>
__global__ void __launch_bounds__(kTile) k_gdx(DevArrays d) {
  int t = blockIdx.x;
  int i = d.ptile_start[t] + threadIdx.x;
  int s = d.ptile_scene[t];
  double acc[1] = {0.0};
  if (i < d.ptile_start[t + 1] && d.sc[s].newton_active) {
    const double* g = d.g + 6 * (size_t)i;
    if (d.refine) {
      const double* x = d.x64 + 6 * (size_t)i;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[0] += g[k] * x[k];
    } else {
      Vec6<T> x = load6<T>(reinterpret_cast<const T*>(d.vx), i);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[0] += g[k] * (double)x.v[k];
    }
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) d.part_p[kPartials * t] = acc[0];
}

// ================================================================================================
// line search along the retraction (Eq. manifold-update-1/2, then normalisation)
// ================================================================================================

template <typename T>
__global__ void k_ls_trial(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const SceneCtl& c = d.sc[d.pscene[i]];
  if (!c.newton_active || c.ls_state != 0) return;
  double4 p = d.xp[i], q = d.xq[i];
  if (d.kin[i]) {
    d.tp[i] = p;
    d.tq[i] = q;
    return;
  }
  double st[6];
  if (c.use_neg_grad) {
    const double* g = d.g + 6 * (size_t)i;
#pragma unroll
    for (int k = 0; k < 6; ++k) st[k] = -g[k];
  } else if (d.refine) {  // the refined FP64 solution
#pragma unroll
    for (int k = 0; k < 6; ++k) st[k] = d.x64[6 * (size_t)i + k];
  } else {
    Vec6<T> x = load6<T>(reinterpret_cast<const T*>(d.vx), i);
#pragma unroll
    for (int k = 0; k < 6; ++k) st[k] = (double)x.v[k];
  }
  double al = c.ls_alpha;
  double4 pn = make_double4(p.x + al * st[0], p.y + al * st[1], p.z + al * st[2], p.w);
  // dq = G_l(q)^T (alpha y) = q (x) (alpha y, 0)
  Q4<double> qq = to_q(q);
  Q4<double> dq = qmul(qq, Q4<double>{al * st[3], al * st[4], al * st[5], 0.0});
  double a = sqrt(qdot(dq, dq));
  Q4<double> qn = qq;
  if (a != 0.0) {
    double sa, ca;
    sincos(a, &sa, &ca);
    double f = sa / a;
    qn = {qq.x * ca + dq.x * f, qq.y * ca + dq.y * f, qq.z * ca + dq.z * f, qq.w * ca + dq.w * f};
  }
  double nq = sqrt(qdot(qn, qn));
  d.tp[i] = pn;
  d.tq[i] = make_double4(qn.x / nq, qn.y / nq, qn.z / nq, qn.w / nq);
}

// particle-term difference with dp = p1 - p0: c dp.((p0 - phat) + dp/2) - m g.dp (+ ground), the same for q; in the
// midpoint form gravity and the ground see the midpoints, whose difference is exactly dp/2
__device__ __forceinline__ double particle_dphi(const DevArrays& d, int i) {
  double4 p0 = d.xp[i], q0 = d.xq[i], p1 = d.tp[i], q1 = d.tq[i], hp = d.hp[i], hq = d.hq[i];
  double2 cf = d.coef[i];
  double m = hp.w;
  double dpx = p1.x - p0.x, dpy = p1.y - p0.y, dpz = p1.z - p0.z;
  double e = cf.x * (dpx * ((p0.x - hp.x) + 0.5 * dpx) + dpy * ((p0.y - hp.y) + 0.5 * dpy) + dpz * ((p0.z - hp.z) + 0.5 * dpz));
  double wv = 1.0;
  if (d.midpoint) {
    double4 pn = d.x0p[i];
    wv = 0.5;
    p0 = mid4(p0, pn);
    p1 = mid4(p1, pn);
  }
  e -= m * (d.gx * (wv * dpx) + d.gy * (wv * dpy) + d.gz * (wv * dpz));
  double dqx = q1.x - q0.x, dqy = q1.y - q0.y, dqz = q1.z - q0.z, dqw = q1.w - q0.w;
  e += cf.y * (dqx * ((q0.x - hq.x) + 0.5 * dqx) + dqy * ((q0.y - hq.y) + 0.5 * dqy) + dqz * ((q0.z - hq.z) + 0.5 * dqz) +
               dqw * ((q0.w - hq.w) + 0.5 * dqw));
  if (d.k_ground > 0.0) {
    double g0 = p0.z - d.ground_z - p0.w, g1 = p1.z - d.ground_z - p0.w;
    if (g0 < 0.0 && g1 < 0.0) e += 0.5 * d.k_ground * (wv * dpz) * (g0 + g1);
    else e += 0.5 * d.k_ground * ((g1 < 0.0 ? g1 * g1 : 0.0) - (g0 < 0.0 ? g0 * g0 : 0.0));
  }
  return e;
}

// contact difference; when overlapping at both states 1/2 k (d1 - d0)(e1 + e0), d1 - d0 = (x1 - x0).(x1 + x0)/(d1 + d0);
// in the midpoint form at the midpoints, with the endpoint differences (p1 - p0)/2
__device__ __forceinline__ double contact_dphi(const DevArrays& d, int i, int j) {
  double4 a0 = d.xp[i], b0 = d.xp[j], a1 = d.tp[i], b1 = d.tp[j];
  double dx[3] = {(a1.x - a0.x) - (b1.x - b0.x), (a1.y - a0.y) - (b1.y - b0.y), (a1.z - a0.z) - (b1.z - b0.z)};
  if (d.midpoint) {
    double4 an = d.x0p[i], bn = d.x0p[j];
    dx[0] = 0.5 * (a1.x - a0.x) - 0.5 * (b1.x - b0.x);
    dx[1] = 0.5 * (a1.y - a0.y) - 0.5 * (b1.y - b0.y);
    dx[2] = 0.5 * (a1.z - a0.z) - 0.5 * (b1.z - b0.z);
    a0 = mid4(a0, an); a1 = mid4(a1, an); b0 = mid4(b0, bn); b1 = mid4(b1, bn);
  }
  double x0[3] = {a0.x - b0.x, a0.y - b0.y, a0.z - b0.z}, x1[3] = {a1.x - b1.x, a1.y - b1.y, a1.z - b1.z};
  double d0 = sqrt(x0[0] * x0[0] + x0[1] * x0[1] + x0[2] * x0[2]);
  double d1 = sqrt(x1[0] * x1[0] + x1[1] * x1[1] + x1[2] * x1[2]);
  double R = a0.w + b0.w, k = d.k_self;
  if (d0 < R && d1 < R) {
    double dd = (dx[0] * (x0[0] + x1[0]) + dx[1] * (x0[1] + x1[1]) + dx[2] * (x0[2] + x1[2])) / (d0 + d1);
    return 0.5 * k * dd * ((d0 - R) + (d1 - R));
  }
  double e1 = d1 < R ? 0.5 * k * (d1 - R) * (d1 - R) : 0.0;
  double e0 = d0 < R ? 0.5 * k * (d0 - R) * (d0 - R) : 0.0;
  return e1 - e0;
}

__global__ void __launch_bounds__(kTile) k_ls_energy_particles(DevArrays d) {
  int t = blockIdx.x;
  int i = d.ptile_start[t] + threadIdx.x;
  int s = d.ptile_scene[t];
  double acc[1] = {0.0};
  if (i < d.ptile_start[t + 1] && d.sc[s].newton_active && d.sc[s].ls_state == 0) {
    acc[0] = particle_dphi(d, i);
    if (d.k_self > 0.0)
      for (int e = d.c_start[i]; e < d.c_start[i + 1]; ++e) {
        int j = d.c_nbr[e];
        if (j > i) acc[0] += contact_dphi(d, i, j);
      }
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) d.part_p[kPartials * t] = acc[0];
}

// bond difference: stretch via l1 - l0 = (d1 - d0).(d1 + d0)/(l1 + l0); bend-twist via the bilinear identity
// r1 - r0 = vec((conj q_j1 - conj q_j0) q_i1) + vec(conj q_j0 (q_i1 - q_i0)); shear differenced directly
__global__ void __launch_bounds__(kTile) k_ls_energy_bonds(DevArrays d) {
  int t = blockIdx.x;
  int b = d.btile_start[t] + threadIdx.x;
  int s = d.btile_scene[t];
  double acc[1] = {0.0};
  if (b < d.btile_start[t + 1] && d.sc[s].newton_active && d.sc[s].ls_state == 0 && !d.bbroken[b]) {
    int2 ij = d.bij[b];
    BondParams bp = load_bond(d.brest[b], d.bstiff[b]);
    double4 pi0 = d.xp[ij.x], pj0 = d.xp[ij.y], pi1 = d.tp[ij.x], pj1 = d.tp[ij.y];
    Q4<double> qi0 = to_q(d.xq[ij.x]), qj0 = to_q(d.xq[ij.y]), qi1 = to_q(d.tq[ij.x]), qj1 = to_q(d.tq[ij.y]);
    V3<double> ddd = (to_v(pj1) - to_v(pj0)) - (to_v(pi1) - to_v(pi0));
    Q4<double> dqj = {qj1.x - qj0.x, qj1.y - qj0.y, qj1.z - qj0.z, qj1.w - qj0.w};
    Q4<double> dqi = {qi1.x - qi0.x, qi1.y - qi0.y, qi1.z - qi0.z, qi1.w - qi0.w};
    if (d.midpoint) {  // midpoints with the start state; their differences are exactly half the state's
      double4 ai = d.x0p[ij.x], aj = d.x0p[ij.y], bi = d.x0q[ij.x], bj = d.x0q[ij.y];
      ddd = 0.5 * (to_v(pj1) - to_v(pj0)) - 0.5 * (to_v(pi1) - to_v(pi0));
      dqj = {0.5 * (qj1.x - qj0.x), 0.5 * (qj1.y - qj0.y), 0.5 * (qj1.z - qj0.z), 0.5 * (qj1.w - qj0.w)};
      dqi = {0.5 * (qi1.x - qi0.x), 0.5 * (qi1.y - qi0.y), 0.5 * (qi1.z - qi0.z), 0.5 * (qi1.w - qi0.w)};
      qi0 = midq(d.xq[ij.x], bi); qj0 = midq(d.xq[ij.y], bj); qi1 = midq(d.tq[ij.x], bi); qj1 = midq(d.tq[ij.y], bj);
      pi0 = mid4(pi0, ai); pj0 = mid4(pj0, aj); pi1 = mid4(pi1, ai); pj1 = mid4(pj1, aj);
    }
    // stretch
    V3<double> dd0 = to_v(pj0) - to_v(pi0), dd1 = to_v(pj1) - to_v(pi1);
    double l0 = sqrt(dot(dd0, dd0)), l1 = sqrt(dot(dd1, dd1));
    double dl = dot(ddd, dd0 + dd1) / (l0 + l1);
    double e = 0.5 * bp.kn * dl * ((l0 - bp.l0) + (l1 - bp.l0));
    // bend-twist
    V3<double> r0 = qvec(qmul(qconj(qj0), qi0)), r1 = qvec(qmul(qconj(qj1), qi1));
    V3<double> dr = qvec(qmul(qconj(dqj), qi1)) + qvec(qmul(qconj(qj0), dqi));
    e += 0.5 * dot(dr, kmul(bp, r0 + r1));
    // shear
    BondEval E0, E1;
    bond_first_order(bp, to_v(pi0), qi0, to_v(pj0), qj0, E0);
    bond_first_order(bp, to_v(pi1), qi1, to_v(pj1), qj1, E1);
    e += E1.e_shear - E0.e_shear;
    acc[0] = e;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) d.part_b[kPartials * t] = acc[0];
}

__global__ void k_ls_commit(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const SceneCtl& c = d.sc[d.pscene[i]];
  if (c.ls_state == 1 && c.newton_active) {
    d.xp[i] = d.tp[i];
    d.xq[i] = d.tq[i];
  }
}

// ================================================================================================
// end of step: velocities (Alg. 3) and tensile-strain fracture (bond state update)
// ================================================================================================

__global__ void k_finish(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || step_aborted(d)) return;  // an aborted step leaves the committed state untouched
  double4 p = d.xp[i], q = d.xq[i], p0 = d.x0p[i], q0 = d.x0q[i];
  double idt = 1.0 / d.dt;
  d.vp[i] = make_double4((p.x - p0.x) * idt, (p.y - p0.y) * idt, (p.z - p0.z) * idt, 0.0);
  d.vq[i] = make_double4((q.x - q0.x) * idt, (q.y - q0.y) * idt, (q.z - q0.z) * idt, (q.w - q0.w) * idt);
  d.x0p[i] = p;
  d.x0q[i] = q;
}

// friction (Sec. 5.4, Friction; Alg. 3): explicit correction of the new velocities from the contacts active at the
// committed state x_{n+1} (the ground, and the step's self-contact candidates that overlap), Jacobi style: every
// particle reads the uncorrected velocities and writes its corrected ones to the trial arrays
__device__ __forceinline__ V3<double> ang_vel(double4 q, double4 u) {  // q' = 1/2 (w, 0) (x) q
  Q4<double> t = qmul(Q4<double>{u.x, u.y, u.z, u.w}, qconj(to_q(q)));
  return {2.0 * t.x, 2.0 * t.y, 2.0 * t.z};
}

__device__ __forceinline__ void friction_term(const DevArrays& d, double fn, V3<double> n, V3<double> vij,
                                              V3<double> wij, double m, double r, V3<double>& dv, V3<double>& dw) {
  V3<double> vt = vij - dot(vij, n) * n;
  double nvt = sqrt(dot(vt, vt)), nw = sqrt(dot(wij, wij));
  if (nvt > 0.0) dv = dv - fmin(1.0, d.mu_slide * fn * d.dt / (m * nvt)) * vt;
  if (nw > 0.0) dw = dw - fmin(1.0, d.mu_roll * fn * r * r * r * d.dt / (0.4 * m * r * r * nw)) * wij;
}

// the correction d along x only, limited to bring x to rest at most
__device__ __forceinline__ V3<double> slow_only(V3<double> x, V3<double> dd) {
  double nx = sqrt(dot(x, x));
  if (!(nx > 0.0)) return {0.0, 0.0, 0.0};
  double s = fmax(-nx, fmin(0.0, dot(dd, x) / nx));
  return (s / nx) * x;
}

__global__ void k_friction(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || step_aborted(d)) return;
  double4 v4 = d.vp[i], u4 = d.vq[i];
  d.tp[i] = v4;
  d.tq[i] = u4;
  if (d.kin[i]) return;
  double4 p = d.x0p[i], q = d.x0q[i];
  double m = d.hp[i].w, r = p.w;
  V3<double> vi = to_v(v4), wi = ang_vel(q, u4), dv = {0.0, 0.0, 0.0}, dw = {0.0, 0.0, 0.0};
  if (d.k_ground > 0.0) {
    double g = p.z - d.ground_z - r;
    if (g < 0.0) friction_term(d, d.k_ground * fabs(g), V3<double>{0.0, 0.0, 1.0}, vi, wi, m, r, dv, dw);
  }
  if (d.k_self > 0.0)
    for (int e = d.c_start[i]; e < d.c_start[i + 1]; ++e) {
      int j = d.c_nbr[e];
      double4 pj = d.x0p[j];
      V3<double> ev = to_v(p) - to_v(pj);
      double dist = sqrt(dot(ev, ev)), R = r + pj.w;
      if (!(dist < R)) continue;
      friction_term(d, d.k_self * fabs(dist - R), (1.0 / dist) * ev, vi - to_v(d.vp[j]),
                    wi - ang_vel(d.x0q[j], d.vq[j]), m, r, dv, dw);
    }
  dv = slow_only(vi, dv);
  dw = slow_only(wi, dw);
  Q4<double> du = qmul(Q4<double>{dw.x, dw.y, dw.z, 0.0}, to_q(q));
  d.tp[i] = make_double4(v4.x + dv.x, v4.y + dv.y, v4.z + dv.z, v4.w);
  d.tq[i] = make_double4(u4.x + 0.5 * du.x, u4.y + 0.5 * du.y, u4.z + 0.5 * du.z, u4.w + 0.5 * du.w);
}

__global__ void k_friction_commit(DevArrays d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || step_aborted(d)) return;
  d.vp[i] = d.tp[i];
  d.vq[i] = d.tq[i];
}

__global__ void k_fracture(DevArrays d) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  bool live = b < d.nb && !d.bbroken[b] && !step_aborted(d);
  int s = b < d.nb ? d.bscene[b] : -1;
  bool intact = false;
  if (live) {
    int2 ij = d.bij[b];
    double4 pi = d.x0p[ij.x], pj = d.x0p[ij.y];
    double ex = pj.x - pi.x, ey = pj.y - pi.y, ez = pj.z - pi.z;
    double l0 = d.brest[b].w;
    double strain = (sqrt(ex * ex + ey * ey + ez * ez) - l0) / l0;
    bool brk = strain > d.bbrk[b];
    if (!brk && d.stress_on) {
      double2 lim = d.bsstr[b];
      if (isfinite(lim.x) || isfinite(lim.y)) {
        double sg, ta;
        bond_stress(load_bond(d.brest[b], d.bstiff[b]), d.bsgeo[b], to_v(pi), to_q(d.x0q[ij.x]), to_v(pj),
                    to_q(d.x0q[ij.y]), sg, ta);
        brk = sg > lim.x || ta > lim.y;
      }
    }
    if (brk) {
      d.bbroken[b] = 1;
      atomicAdd(&d.sc[s].bonds_broken, 1);
    } else {
      intact = true;
    }
  }
  // intact bonds per scene, one atomic per scene present in the warp (bonds are grouped by scene)
  unsigned m = __activemask();
  unsigned grp = __match_any_sync(m, s);
  unsigned cnt = __popc(__ballot_sync(m, intact) & grp);
  if (s >= 0 && cnt && (threadIdx.x & 31) == __ffs(grp) - 1)
    atomicAdd(reinterpret_cast<unsigned long long*>(&d.sc[s].intact), (unsigned long long)cnt);
}

// ================================================================================================
// inspection helpers
// ================================================================================================

// (sigma, tau) of every bond at the committed state, written at its caller index
__global__ void k_bond_stress(DevArrays d, double* out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nb) return;
  int2 ij = d.bij[b];
  double sg, ta;
  bond_stress(load_bond(d.brest[b], d.bstiff[b]), d.bsgeo[b], to_v(d.x0p[ij.x]), to_q(d.x0q[ij.x]),
              to_v(d.x0p[ij.y]), to_q(d.x0q[ij.y]), sg, ta);
  size_t e = (size_t)d.bond_int2ext[b];
  out[2 * e] = sg;
  out[2 * e + 1] = ta;
}

// ids: NULL (every bond, written at its caller index) or a list of caller bond indices (written in list order)
template <typename T>
__global__ void k_unpack_bond_hess(DevArrays d, double* out, const int32_t* ids, int count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (ids ? count : d.nb)) return;
  int b = ids ? d.bond_ext2int[ids[t]] : t;
  size_t slot = ids ? (size_t)t : (size_t)d.bond_int2ext[b];
  const T* M = reinterpret_cast<const T*>(d.bM) + 36 * (size_t)b;
  const T* E = reinterpret_cast<const T*>(d.bE) + 12 * (size_t)b;
  double H[12][12];
  for (int a = 0; a < 12; ++a)
    for (int c = 0; c < 12; ++c) H[a][c] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      double ah = M[s3(a, c)], bs = M[6 + 3 * a + c], cs = M[15 + 3 * a + c], f = M[24 + 3 * a + c];
      double e = E[s3(a, c)], g = E[6 + s3(a, c)];
      H[a][c] = ah; H[6 + a][6 + c] = ah; H[a][6 + c] = -ah; H[6 + a][c] = -ah;   // p_i, p_j
      H[a][3 + c] = -bs; H[3 + c][a] = -bs;                                        // p_i y_i
      H[6 + a][3 + c] = bs; H[3 + c][6 + a] = bs;                                  // p_j y_i
      H[a][9 + c] = -cs; H[9 + c][a] = -cs;                                        // p_i y_j
      H[6 + a][9 + c] = cs; H[9 + c][6 + a] = cs;                                  // p_j y_j
      H[3 + a][3 + c] = e; H[9 + a][9 + c] = g;
      H[3 + a][9 + c] = f; H[9 + c][3 + a] = f;
    }
  // stored bonds are oriented by internal index; report them oriented like the caller's pair (lower caller index
  // first), swapping the two endpoint blocks when the orders disagree
  int2 bp = d.bij[b];
  int flip = d.perm[bp.x] > d.perm[bp.y] ? 6 : 0;
  double* o = out + 144 * slot;
  for (int a = 0; a < 12; ++a)
    for (int c = 0; c < 12; ++c) o[12 * a + c] = H[(a + flip) % 12][(c + flip) % 12];
}

template <typename T>
__global__ void k_unpack_diag(DevArrays d, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const T* D = reinterpret_cast<const T*>(d.D) + kDiagStride * (size_t)i;
  size_t u = (size_t)d.perm[i];
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 6; ++c) out[36 * u + 6 * a + c] = (double)D[sidx<6>(a, c)];
}

__global__ void k_convert(const void* src, int sd, void* dst, int dd, int64_t count) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count) return;
  double v = sd ? reinterpret_cast<const double*>(src)[k] : (double)reinterpret_cast<const float*>(src)[k];
  if (dd) reinterpret_cast<double*>(dst)[k] = v;
  else reinterpret_cast<float*>(dst)[k] = (float)v;
}

static inline int blocks_for(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

// ================================================================================================
// Allocation-free PCG: the solver's scratch (per-scene control blocks, barrier counters, partial sums and the
// PCG vectors) lives in this fixed static device array instead of memory the library allocates. Every GPU that
// loads the library holds the array until the process exits. All calls share it.
// ================================================================================================

constexpr size_t kStaticPcgBytes = size_t(24) << 20;  // 24 MiB
static __device__ __align__(256) unsigned char g_static_pcg_scratch[kStaticPcgBytes];

size_t static_pcg_capacity() { return kStaticPcgBytes; }

// Device address of the static array for the current device. The first call on a device looks the symbol up
// (cudaGetSymbolAddress) with that device current and caches it; later calls reuse the cached address.
// The cache entries are atomics: two host threads making their first call on one device may both look the address
// up, and both store the same value.
cudaError_t static_pcg_address(void** out) {
  static std::atomic<void*> cache[256];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  void* p = cache[dev].load(std::memory_order_acquire);
  if (p == nullptr) {
    e = cudaGetSymbolAddress(&p, g_static_pcg_scratch);
    if (e != cudaSuccess) return e;
    cache[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return cudaSuccess;
}

// clears the control blocks and counters that must start at zero and sets every scene active with eps_r
__global__ void k_static_pcg_init(DevArrays d, double eps_r) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *d.cnt = Counters{};
  if (s >= d.n_scenes) return;
  SceneCtl c = {};
  c.newton_active = 1;
  c.eps_r = eps_r;
  d.sc[s] = c;
}

int launch_static_pcg_init(const DevArrays& d, double eps_r, cudaStream_t s) {
  int n = d.n_scenes > 1 ? d.n_scenes : 1;
  k_static_pcg_init<<<blocks_for(n, 128), 128, 0, s>>>(d, eps_r);
  return 1;
}

// ================================================================================================
// launchers
// ================================================================================================


int launch_predict(const DevArrays& d, cudaStream_t s) {
  k_step_init<<<blocks_for(d.n_scenes, 128), 128, 0, s>>>(d);
  if (d.n == 0) return 1;
  k_predict<<<blocks_for(d.n, 256), 256, 0, s>>>(d);
  return 2;
}

int launch_zhat(const DevArrays& d, cudaStream_t s) {
  if (!d.midpoint || d.n == 0) return 0;
  int k = 0;
  if (d.nb) {
    k_zhat_bonds<<<blocks_for(d.nb, kTile), kTile, 0, s>>>(d);
    ++k;
  }
  k_zhat_particles<<<blocks_for(d.n, kTile), kTile, 0, s>>>(d);
  return k + 1;
}

int launch_contacts(const DevArrays& d, int stage, cudaStream_t s) {
  if (d.n == 0) return 0;
  if (stage == 0) {
    cudaMemsetAsync(d.hash_count, 0, sizeof(int32_t) * d.hash_size, s);
    cudaMemsetAsync(d.cnt_tmp, 0, sizeof(int32_t) * (d.hash_size > d.n ? d.hash_size : d.n), s);
    k_cell_count<<<blocks_for(d.n, 256), 256, 0, s>>>(d);
    int k = 1 + launch_scan_counts(d, d.hash_count, d.hash_start, d.hash_size, s);
    k_cell_fill<<<blocks_for(d.n, 256), 256, 0, s>>>(d);
    k_cell_sort<<<blocks_for(d.hash_size, 256), 256, 0, s>>>(d);
    k_contact_scan<0><<<blocks_for(d.n, 128), 128, 0, s>>>(d);
    k += 3 + launch_scan_counts(d, d.cnt_tmp, d.c_start, d.n, s);
    return k;
  }
  if (stage == 2) {
    k_contact_check<<<1, 1, 0, s>>>(d);
    k_contact_clear<<<blocks_for(d.n + 1, 256), 256, 0, s>>>(d);
    return 2;
  }
  k_contact_scan<1><<<blocks_for(d.n, 128), 128, 0, s>>>(d);
  return 1;
}

int launch_scan_counts(const DevArrays& d, const int32_t* counts, int32_t* starts, int n, cudaStream_t s) {
  int nblk = blocks_for(n, 1024);
  if (nblk == 0) {
    cudaMemsetAsync(starts, 0, sizeof(int32_t), s);
    return 0;
  }
  k_scan_block_sums<<<nblk, 1024, 0, s>>>(counts, n, d.scan_tmp);
  k_scan_top<<<1, 1024, 0, s>>>(d.scan_tmp, nblk);
  k_scan_apply<<<nblk, 1024, 0, s>>>(counts, n, d.scan_tmp, nblk, starts);
  return 3;
}

int launch_bond_grad(const DevArrays& d, int all, cudaStream_t s) {
  if (d.n_btiles == 0) return 0;
  k_bond_grad<<<d.n_btiles, kTile, 0, s>>>(d, all);
  return 1;
}

int launch_particle_grad(const DevArrays& d, int mask, int all, cudaStream_t s) {
  if (d.n_ptiles == 0) return 0;
  k_particle_grad<<<d.n_ptiles, kTile, 0, s>>>(d, mask, all);
  return 1;
}

int launch_bond_hess(const DevArrays& d, int all, cudaStream_t s) {
  if (d.nb == 0) return 0;
  const int bs = (d.bond_tile == 64 || d.bond_tile == 256) ? d.bond_tile : 128;
  const int nbk = blocks_for(d.nb, bs);
  if (d.midpoint) {
    if (d.mixed) k_bond_hess<float, true, 1><<<nbk, bs, 0, s>>>(d, all);
    else k_bond_hess<double, true, 1><<<nbk, bs, 0, s>>>(d, all);
  } else if (d.mixed) {
    if (d.bond_capped) k_bond_hess<float, false, 2><<<nbk, bs, 0, s>>>(d, all);
    else k_bond_hess<float, false, 1><<<nbk, bs, 0, s>>>(d, all);
  } else {
    k_bond_hess<double, false, 1><<<nbk, bs, 0, s>>>(d, all);
  }
  return 1;
}

int launch_particle_hess(const DevArrays& d, int mask, int all, cudaStream_t s) {
  if (d.n_ptiles == 0) return 0;
  if (d.mixed) k_particle_hess<float><<<d.n_ptiles, kTile, 0, s>>>(d, mask, all);
  else k_particle_hess<double><<<d.n_ptiles, kTile, 0, s>>>(d, mask, all);
  return 1;
}

int launch_scene_reduce(const DevArrays& d, int mode, unsigned long long cond, cudaStream_t s) {
  k_scene_reduce<<<1, 1024, 0, s>>>(d, mode, cond);
  return 1;
}

size_t pcg_smem_bytes_for(int mode, int mixed, int max_rows, int max_entries, int max_zslots) {
  size_t rows = sizeof(int4) * (size_t)(max_rows > 0 ? max_rows : 1);
  size_t w = mixed ? sizeof(float) : sizeof(double);
  if (mode == 1) return rows + sizeof(int2) * (size_t)(max_entries > 0 ? max_entries : 1);
  if (mode == 2) return rows + (size_t)kTile * 36 * w;
  if (mode == 3) return rows + (size_t)2 * kTile * 36 * w;
  if (mode == 4) return rows + (size_t)(max_zslots > 0 ? max_zslots : 2) * 6 * w + (size_t)kTile * 36 * w;
  return 0;
}
size_t pcg_smem_bytes(const DevArrays& d) {
  if (d.pcg_even) return (size_t)d.pcg_even_off + sizeof(EvenPcg);
  const bool rows = !(d.pcg_mode == 2 || d.pcg_mode == 3) || d.pcg_rows_sm;
  return pcg_smem_bytes_for(d.pcg_mode, d.mixed, rows ? d.pcg_max_rows : 0, d.pcg_max_entries, d.pcg_max_zslots);
}

template <typename T, int MODE>
static const void* pcg_kernel_m(int lanes) {
  switch (lanes) {
    case 1: return (const void*)k_pcg<T, 1, MODE>;
    case 2: return (const void*)k_pcg<T, 2, MODE>;
    case 8: return (const void*)k_pcg<T, 8, MODE>;
    default: return (const void*)k_pcg<T, 4, MODE>;
  }
}
template <typename T>
static const void* pcg_kernel(int lanes, int mode) {
  if (mode == 4) switch (lanes) {
      case 1: return (const void*)k_pcg_fused<T, 1>;
      case 2: return (const void*)k_pcg_fused<T, 2>;
      case 8: return (const void*)k_pcg_fused<T, 8>;
      default: return (const void*)k_pcg_fused<T, 4>;
    }
  if (mode == 3) return pcg_kernel_m<T, 3>(lanes);
  if (mode == 2) return pcg_kernel_m<T, 2>(lanes);
  if (mode == 1) return pcg_kernel_m<T, 1>(lanes);
  return pcg_kernel_m<T, 0>(lanes);
}

int pcg_max_blocks(int mixed, int lanes, size_t smem, int mode) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* k = mixed ? pcg_kernel<float>(lanes, mode) : pcg_kernel<double>(lanes, mode);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kTile, smem) != cudaSuccess) return 0;
  return sms * per;
}

int launch_pcg(const DevArrays& d, int rhs_from_g, int mask, cudaStream_t s, cudaError_t* err) {
  if (d.n == 0 || d.pcg_grid < 1) {
    *err = cudaSuccess;
    return 0;
  }
  DevArrays dd = d;
  void* args[] = {&dd, &rhs_from_g, &mask};
  const void* k = d.mixed ? pcg_kernel<float>(d.pcg_lanes, d.pcg_mode) : pcg_kernel<double>(d.pcg_lanes, d.pcg_mode);
  size_t smem = pcg_smem_bytes(d);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  *err = cudaLaunchCooperativeKernel(k, d.pcg_grid, kTile, args, smem, s);
  return 1;
}

int launch_matvec64(const DevArrays& d, const double* x64, double* y64, int mask, cudaStream_t s) {
  if (d.n == 0) return 0;
  if (d.mixed) k_matvec64<float><<<blocks_for(d.n, kTile), kTile, 0, s>>>(d, x64, y64, mask);
  else k_matvec64<double><<<blocks_for(d.n, kTile), kTile, 0, s>>>(d, x64, y64, mask);
  return 1;
}

int launch_refine(const DevArrays& d, int first, cudaStream_t s) {
  if (d.n == 0 || !d.refine || d.n_ptiles == 0) return 0;
  if (d.mixed) {
    k_refine_acc<float><<<blocks_for(d.n, 256), 256, 0, s>>>(d, first);
    k_refine_res<float><<<d.n_ptiles, kTile, 0, s>>>(d);
  } else {
    k_refine_acc<double><<<blocks_for(d.n, 256), 256, 0, s>>>(d, first);
    k_refine_res<double><<<d.n_ptiles, kTile, 0, s>>>(d);
  }
  return 2;
}

int launch_gdx(const DevArrays& d, cudaStream_t s) {
  if (d.n_ptiles == 0) return 0;
  if (d.mixed) k_gdx<float><<<d.n_ptiles, kTile, 0, s>>>(d);
  else k_gdx<double><<<d.n_ptiles, kTile, 0, s>>>(d);
  return 1;
}

int launch_ls_trial(const DevArrays& d, cudaStream_t s) {
  if (d.n == 0) return 0;
  if (d.mixed) k_ls_trial<float><<<blocks_for(d.n, 256), 256, 0, s>>>(d);
  else k_ls_trial<double><<<blocks_for(d.n, 256), 256, 0, s>>>(d);
  return 1;
}

int launch_ls_energy(const DevArrays& d, cudaStream_t s) {
  int k = 0;
  if (d.n_ptiles) { k_ls_energy_particles<<<d.n_ptiles, kTile, 0, s>>>(d); ++k; }
  if (d.n_btiles) { k_ls_energy_bonds<<<d.n_btiles, kTile, 0, s>>>(d); ++k; }
  return k;
}

int launch_ls_commit(const DevArrays& d, cudaStream_t s) {
  if (d.n == 0) return 0;
  k_ls_commit<<<blocks_for(d.n, 256), 256, 0, s>>>(d);
  return 1;
}

int launch_finish(const DevArrays& d, cudaStream_t s) {
  int k = 0;
  if (d.n) { k_finish<<<blocks_for(d.n, 256), 256, 0, s>>>(d); ++k; }
  if (d.n && (d.mu_slide > 0.0 || d.mu_roll > 0.0)) {
    k_friction<<<blocks_for(d.n, 128), 128, 0, s>>>(d);
    k_friction_commit<<<blocks_for(d.n, 256), 256, 0, s>>>(d);
    k += 2;
  }
  if (d.nb) { k_fracture<<<blocks_for(d.nb, 256), 256, 0, s>>>(d); ++k; }
  return k;
}

int launch_matvec(const DevArrays& d, int mask, cudaStream_t s) {
  if (d.n == 0) return 0;
  if (d.mixed) k_matvec<float><<<blocks_for(d.n, kTile), kTile, 0, s>>>(d, mask);
  else k_matvec<double><<<blocks_for(d.n, kTile), kTile, 0, s>>>(d, mask);
  return 1;
}

int launch_unpack_bond_hess(const DevArrays& d, double* out, const int32_t* ids, int count, cudaStream_t s) {
  int m = ids ? count : d.nb;
  if (m == 0) return 0;
  if (d.mixed) k_unpack_bond_hess<float><<<blocks_for(m, 64), 64, 0, s>>>(d, out, ids, count);
  else k_unpack_bond_hess<double><<<blocks_for(m, 64), 64, 0, s>>>(d, out, ids, count);
  return 1;
}

int launch_bond_stress(const DevArrays& d, double* out, cudaStream_t s) {
  if (d.nb == 0) return 0;
  k_bond_stress<<<blocks_for(d.nb, 128), 128, 0, s>>>(d, out);
  return 1;
}

int launch_unpack_diag(const DevArrays& d, double* out, cudaStream_t s) {
  if (d.n == 0) return 0;
  if (d.mixed) k_unpack_diag<float><<<blocks_for(d.n, 128), 128, 0, s>>>(d, out);
  else k_unpack_diag<double><<<blocks_for(d.n, 128), 128, 0, s>>>(d, out);
  return 1;
}

// state transfers between the caller's particle order (perm[k] = caller index of internal particle k) and the
// library's internal space-filling-curve order
__global__ void k_pack_state(DevArrays d, double* pos3, double* quat4, double* vel3, double* qvel4) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  size_t u = (size_t)d.perm[k];
  if (pos3) { double4 p = d.x0p[k]; pos3[3 * u] = p.x; pos3[3 * u + 1] = p.y; pos3[3 * u + 2] = p.z; }
  if (vel3) { double4 v = d.vp[k]; vel3[3 * u] = v.x; vel3[3 * u + 1] = v.y; vel3[3 * u + 2] = v.z; }
  // [n][4] arrays are accessed element by element: the caller layout guarantees only 8-byte alignment
  if (quat4) { double4 q = d.x0q[k]; quat4[4 * u] = q.x; quat4[4 * u + 1] = q.y; quat4[4 * u + 2] = q.z; quat4[4 * u + 3] = q.w; }
  if (qvel4) { double4 q = d.vq[k]; qvel4[4 * u] = q.x; qvel4[4 * u + 1] = q.y; qvel4[4 * u + 2] = q.z; qvel4[4 * u + 3] = q.w; }
}

__global__ void k_unpack_state(DevArrays d, const double* pos3, const double* quat4, const double* vel3,
                               const double* qvel4) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  size_t u = (size_t)d.perm[k];
  if (pos3) { double r = d.x0p[k].w; d.x0p[k] = make_double4(pos3[3 * u], pos3[3 * u + 1], pos3[3 * u + 2], r); }
  if (vel3) d.vp[k] = make_double4(vel3[3 * u], vel3[3 * u + 1], vel3[3 * u + 2], 0.0);
  if (quat4) d.x0q[k] = make_double4(quat4[4 * u], quat4[4 * u + 1], quat4[4 * u + 2], quat4[4 * u + 3]);
  if (qvel4) d.vq[k] = make_double4(qvel4[4 * u], qvel4[4 * u + 1], qvel4[4 * u + 2], qvel4[4 * u + 3]);
}

// inertia targets given in the caller's order (inspection calls); the mass in hp.w is kept
__global__ void k_set_hat(DevArrays d, const double* phat3, const double* qhat4) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  size_t u = (size_t)d.perm[k];
  double m = d.hp[k].w;
  d.hp[k] = make_double4(phat3[3 * u], phat3[3 * u + 1], phat3[3 * u + 2], m);
  d.hq[k] = make_double4(qhat4[4 * u], qhat4[4 * u + 1], qhat4[4 * u + 2], qhat4[4 * u + 3]);
}

__global__ void k_pack_hat(DevArrays d, double* phat3, double* qhat4) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  size_t u = (size_t)d.perm[k];
  double4 p = d.hp[k], q = d.hq[k];
  phat3[3 * u] = p.x; phat3[3 * u + 1] = p.y; phat3[3 * u + 2] = p.z;
  qhat4[4 * u] = q.x; qhat4[4 * u + 1] = q.y; qhat4[4 * u + 2] = q.z; qhat4[4 * u + 3] = q.w;
}

// the iterate (xp, xq) given in the caller's order (inspection calls); the radius in xp.w is kept
__global__ void k_set_iterate(DevArrays d, const double* pos3, const double* quat4) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  size_t u = (size_t)d.perm[k];
  double r = d.x0p[k].w;
  d.xp[k] = make_double4(pos3[3 * u], pos3[3 * u + 1], pos3[3 * u + 2], r);
  d.xq[k] = make_double4(quat4[4 * u], quat4[4 * u + 1], quat4[4 * u + 2], quat4[4 * u + 3]);
}

// bond flags between the caller's bond order (order of addition) and the stored order: ext2int[e] = stored index
__global__ void k_bond_flags(DevArrays d, uint8_t* ext, int to_device) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.nb) return;
  int b = d.bond_ext2int[e];
  if (to_device) d.bbroken[b] = ext[e] ? 1 : 0;
  else ext[e] = d.bbroken[b];
}

int launch_pack_state(const DevArrays& d, double* pos3, double* quat4, double* vel3, double* qvel4, cudaStream_t s) {
  if (d.n == 0) return 0;
  k_pack_state<<<blocks_for(d.n, 256), 256, 0, s>>>(d, pos3, quat4, vel3, qvel4);
  return 1;
}

int launch_unpack_state(const DevArrays& d, const double* pos3, const double* quat4, const double* vel3,
                        const double* qvel4, cudaStream_t s) {
  if (d.n == 0) return 0;
  k_unpack_state<<<blocks_for(d.n, 256), 256, 0, s>>>(d, pos3, quat4, vel3, qvel4);
  return 1;
}

int launch_set_hat(const DevArrays& d, const double* phat3, const double* qhat4, cudaStream_t s) {
  if (d.n == 0) return 0;
  k_set_hat<<<blocks_for(d.n, 256), 256, 0, s>>>(d, phat3, qhat4);
  return 1;
}

int launch_pack_hat(const DevArrays& d, double* phat3, double* qhat4, cudaStream_t s) {
  if (d.n == 0) return 0;
  k_pack_hat<<<blocks_for(d.n, 256), 256, 0, s>>>(d, phat3, qhat4);
  return 1;
}

int launch_set_iterate(const DevArrays& d, const double* pos3, const double* quat4, cudaStream_t s) {
  if (d.n == 0) return 0;
  k_set_iterate<<<blocks_for(d.n, 256), 256, 0, s>>>(d, pos3, quat4);
  return 1;
}

int launch_bond_flags(const DevArrays& d, uint8_t* ext, int to_device, cudaStream_t s) {
  if (d.nb == 0) return 0;
  k_bond_flags<<<blocks_for(d.nb, 256), 256, 0, s>>>(d, ext, to_device);
  return 1;
}

// [n][6] vectors with precision conversion and reordering: dir 0 caller -> internal, dir 1 internal -> caller
__global__ void k_convert_perm(const void* src, int sd, void* dst, int dd, const int32_t* perm, int dir, int n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 6 * (int64_t)n) return;
  int64_t k = t / 6, c = t % 6;
  int64_t u = perm[k];
  int64_t si = dir ? t : 6 * u + c, di = dir ? 6 * u + c : t;
  double v = sd ? reinterpret_cast<const double*>(src)[si] : (double)reinterpret_cast<const float*>(src)[si];
  if (dd) reinterpret_cast<double*>(dst)[di] = v;
  else reinterpret_cast<float*>(dst)[di] = (float)v;
}

int launch_convert_perm(const void* src, int sd, void* dst, int dd, const int32_t* perm, int dir, int n,
                        cudaStream_t s) {
  if (n == 0) return 0;
  k_convert_perm<<<blocks_for(6 * (int64_t)n, 256), 256, 0, s>>>(src, sd, dst, dd, perm, dir, n);
  return 1;
}

int launch_convert(const void* src, int sd, void* dst, int dd, int64_t count, cudaStream_t s) {
  if (count == 0) return 0;
  k_convert<<<blocks_for(count, 256), 256, 0, s>>>(src, sd, dst, dd, count);
  return 1;
}

// ================================================================================================
// aggregation AMG preconditioner (Sec. 5.3): coarse operators and the V(1,1) cycle
// ================================================================================================

// R(q) of a unit quaternion (x, y, z, w), row major
__device__ __forceinline__ void amg_rot(double4 q, double R[9]) {
  double x = q.x, y = q.y, z = q.z, w = q.w;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

// the rigid-motion block of a node at offset dv from its aggregate's centroid: [[I, -[dv]x], [0, B]]; B = 1/2 R(q)^T
// on level 0 (a world rotation w turns the particle by y = 1/2 R(q)^T w), identity above
__device__ __forceinline__ void amg_pblock(const double dv[3], const double* B3, double P[36]) {
#pragma unroll
  for (int k = 0; k < 36; ++k) P[k] = 0.0;
  P[0] = P[7] = P[14] = 1.0;
  P[4] = dv[2];  P[5] = -dv[1];
  P[9] = -dv[2]; P[11] = dv[0];
  P[15] = dv[1]; P[16] = -dv[0];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) P[6 * (3 + a) + 3 + b] = B3 ? B3[3 * a + b] : (a == b ? 1.0 : 0.0);
}

__device__ __forceinline__ void amg_p0(const DevArrays& d, const AmgDev& a, int i, double P[36]) {
  int I = a.L[0].parent[i];
  double4 p = d.xp[i];
  const double* c = a.L[1].cen + 3 * (size_t)I;
  double dv[3] = {p.x - c[0], p.y - c[1], p.z - c[2]};
  double R[9], B[9];
  amg_rot(d.xq[i], R);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2) B[3 * r + c2] = 0.5 * R[3 * c2 + r];
  amg_pblock(dv, B, P);
}

__device__ __forceinline__ void amg_pl(const AmgDev& a, int l, int k, double P[36]) {  // node k of level l >= 1
  int I = a.L[l].parent[k];
  const double *ck = a.L[l].cen + 3 * (size_t)k, *cI = a.L[l + 1].cen + 3 * (size_t)I;
  double dv[3] = {ck[0] - cI[0], ck[1] - cI[1], ck[2] - cI[2]};
  amg_pblock(dv, nullptr, P);
}

// acc += P_r^T A P_c (all 6x6, A row major)
__device__ __forceinline__ void amg_triple(const double Pr[36], const double A[36], const double Pc[36], double acc[36]) {
  double T[36];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s += A[6 * r + k] * Pc[6 * k + c];
      T[6 * r + c] = s;
    }
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s += Pr[6 * k + r] * T[6 * k + c];
      acc[6 * r + c] += s;
    }
}

__global__ void k_amg_cent(DevArrays d, AmgDev a, int l) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  const AmgLevel& L = a.L[l];
  if (I >= L.n) return;
  int c0 = L.cbeg[I], c1 = L.cend[I];
  double s[3] = {0.0, 0.0, 0.0};
  for (int k = c0; k < c1; ++k) {
    if (l == 1) {
      double4 p = d.xp[k];
      s[0] += p.x; s[1] += p.y; s[2] += p.z;
    } else {
      const double* c = a.L[l - 1].cen + 3 * (size_t)k;
      s[0] += c[0]; s[1] += c[1]; s[2] += c[2];
    }
  }
  double inv = 1.0 / (double)(c1 - c0);
  double* o = L.cen + 3 * (size_t)I;
  o[0] = s[0] * inv; o[1] = s[1] * inv; o[2] = s[2] * inv;
}

// the (i, j) block of bond b in (dp_i, y_i) x (dp_j, y_j) from its factored storage: [[-Ah, -Cs], [Bs^T, F]]
template <typename T>
__device__ __forceinline__ void amg_bond_block(const DevArrays& d, int b, T H[36]) {
  const T* M = reinterpret_cast<const T*>(d.bM) + 36 * (size_t)b;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      H[6 * r + c] = -M[sidx<3>(r, c)];
      H[6 * r + 3 + c] = -M[15 + 3 * r + c];
      H[6 * (3 + r) + c] = M[6 + 3 * c + r];
      H[6 * (3 + r) + 3 + c] = M[24 + 3 * r + c];
    }
}

// per particle, once per Newton iteration: offset from the aggregate's centroid and 1/2 R(q)^T
template <typename T>
__global__ void k_amg_p0(DevArrays d, AmgDev a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  int I = a.L[0].parent[i];
  double4 p = d.xp[i];
  const double* c = a.L[1].cen + 3 * (size_t)I;
  double R[9];
  amg_rot(d.xq[i], R);
  T* o = reinterpret_cast<T*>(a.p0) + 12 * (size_t)i;
  o[0] = (T)(p.x - c[0]); o[1] = (T)(p.y - c[1]); o[2] = (T)(p.z - c[2]);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) o[3 + 3 * r + k] = (T)(0.5 * R[3 * k + r]);  // 1/2 R^T
}

// the block [[I, -[dv]x], [0, B]] from the stored (dv, B) of a particle (or B = I)
template <typename T>
__device__ __forceinline__ void amg_pblock_t(T dx, T dy, T dz, const T* B3, T P[36]) {
#pragma unroll
  for (int k = 0; k < 36; ++k) P[k] = (T)0;
  P[0] = P[7] = P[14] = (T)1;
  P[4] = dz;  P[5] = -dy;
  P[9] = -dz; P[11] = dx;
  P[15] = dy; P[16] = -dx;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) P[6 * (3 + r) + 3 + c] = B3 ? B3[3 * r + c] : (r == c ? (T)1 : (T)0);
}
template <typename T>
__device__ __forceinline__ void amg_p0_load(const AmgDev& a, int i, T P[36]) {
  const T* o = reinterpret_cast<const T*>(a.p0) + 12 * (size_t)i;
  T B[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) B[k] = o[3 + k];
  amg_pblock_t<T>(o[0], o[1], o[2], B, P);
}

// acc += P_r^T A P_c in the path's precision
template <typename T>
__device__ __forceinline__ void amg_triple_t(const T Pr[36], const T A[36], const T Pc[36], T acc[36]) {
  T W[36];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      T s = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s += A[6 * r + k] * Pc[6 * k + c];
      W[6 * r + c] = s;
    }
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      T s = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s += Pr[6 * k + r] * W[6 * k + c];
      acc[6 * r + c] += s;
    }
}

template <typename T>
__global__ void k_amg_gal1(DevArrays d, AmgDev a) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  const AmgLevel& L = a.L[1];
  if (e >= L.nnz) return;
  int I = L.erow[e], J = L.col[e];
  T acc[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) acc[k] = (T)0;
  T Pr[36], Pc[36], H[36];
  if (I == J) {  // the assembled diagonal blocks of the aggregate's particles
    for (int i = L.cbeg[I]; i < L.cend[I]; ++i) {
      const T* Dp = reinterpret_cast<const T*>(d.D) + kDiagStride * (size_t)i;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) H[6 * r + c] = Dp[sidx<6>(r, c)];
      amg_p0_load<T>(a, i, Pr);
      amg_triple_t<T>(Pr, H, Pr, acc);
    }
  }
  for (int k = L.gs[e]; k < L.gs[e + 1]; ++k) {
    int code = L.gsrc[k], b = code >> 1;
    if (d.bbroken[b]) continue;
    int2 ij = d.bij[b];
    if (d.kin[ij.x] || d.kin[ij.y]) continue;  // the kinematic rows and columns of the system are identity
    amg_bond_block<T>(d, b, H);
    if (code & 1) {  // P_j^T H_ij^T P_i
      T Ht[36];
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) Ht[6 * r + c] = H[6 * c + r];
      amg_p0_load<T>(a, ij.y, Pr);
      amg_p0_load<T>(a, ij.x, Pc);
      amg_triple_t<T>(Pr, Ht, Pc, acc);
    } else {
      amg_p0_load<T>(a, ij.x, Pr);
      amg_p0_load<T>(a, ij.y, Pc);
      amg_triple_t<T>(Pr, H, Pc, acc);
    }
  }
  T* o = reinterpret_cast<T*>(L.val) + 36 * (size_t)e;
#pragma unroll
  for (int k = 0; k < 36; ++k) o[k] = acc[k];
}

template <typename T>
__global__ void k_amg_gal(AmgDev a, int l) {  // level l >= 2 from level l - 1
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  const AmgLevel& L = a.L[l];
  const AmgLevel& F = a.L[l - 1];
  if (e >= L.nnz) return;
  T acc[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) acc[k] = (T)0;
  T Pr[36], Pc[36], A[36];
  for (int k = L.gs[e]; k < L.gs[e + 1]; ++k) {
    int f = L.gsrc[k];
    const T* v = reinterpret_cast<const T*>(F.val) + 36 * (size_t)f;
#pragma unroll
    for (int t = 0; t < 36; ++t) A[t] = v[t];
    int r = F.erow[f], c = F.col[f];
    const double *cr = F.cen + 3 * (size_t)r, *cc = F.cen + 3 * (size_t)c;
    const double *Cr = L.cen + 3 * (size_t)F.parent[r], *Cc = L.cen + 3 * (size_t)F.parent[c];
    amg_pblock_t<T>((T)(cr[0] - Cr[0]), (T)(cr[1] - Cr[1]), (T)(cr[2] - Cr[2]), nullptr, Pr);
    amg_pblock_t<T>((T)(cc[0] - Cc[0]), (T)(cc[1] - Cc[1]), (T)(cc[2] - Cc[2]), nullptr, Pc);
    amg_triple_t<T>(Pr, A, Pc, acc);
  }
  T* o = reinterpret_cast<T*>(L.val) + 36 * (size_t)e;
#pragma unroll
  for (int k = 0; k < 36; ++k) o[k] = acc[k];
}

// inverse of an SPD 6x6 block (FP64 Cholesky; a non-positive pivot falls back to the inverse diagonal)
__device__ __forceinline__ void amg_inv6(const double A[36], double X[36]) {
  double Lc[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) Lc[k] = 0.0;
  bool ok = true;
  for (int j = 0; j < 6 && ok; ++j) {
    double s = A[7 * j];
    for (int k = 0; k < j; ++k) s -= Lc[6 * j + k] * Lc[6 * j + k];
    if (!(s > 0.0)) { ok = false; break; }
    Lc[7 * j] = sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = A[6 * i + j];
      for (int k = 0; k < j; ++k) t -= Lc[6 * i + k] * Lc[6 * j + k];
      Lc[6 * i + j] = t / Lc[7 * j];
    }
  }
  for (int c = 0; c < 6; ++c) {
    double w[6], z[6];
    if (!ok) {
      for (int r = 0; r < 6; ++r) X[6 * r + c] = (r == c && A[7 * r] > 0.0) ? 1.0 / A[7 * r] : (r == c ? 1.0 : 0.0);
      continue;
    }
    for (int i = 0; i < 6; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= Lc[6 * i + k] * w[k];
      w[i] = s / Lc[7 * i];
    }
    for (int i = 5; i >= 0; --i) {
      double s = w[i];
      for (int k = i + 1; k < 6; ++k) s -= Lc[6 * k + i] * z[k];
      z[i] = s / Lc[7 * i];
    }
    for (int r = 0; r < 6; ++r) X[6 * r + c] = z[r];
  }
}

template <typename T>
__global__ void k_amg_dinv(AmgDev a, int l) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  const AmgLevel& L = a.L[l];
  if (I >= L.n) return;
  double A[36], X[36];
  if (L.diag[I] >= 0) {
    const T* v = reinterpret_cast<const T*>(L.val) + 36 * (size_t)L.diag[I];
#pragma unroll
    for (int k = 0; k < 36; ++k) A[k] = (double)v[k];
  } else {  // not reached: every node carries its diagonal entry
#pragma unroll
    for (int k = 0; k < 36; ++k) A[k] = (k % 7 == 0) ? 1.0 : 0.0;
  }
  amg_inv6(A, X);
  T* o = reinterpret_cast<T*>(L.dinv) + 36 * (size_t)I;
#pragma unroll
  for (int k = 0; k < 36; ++k) o[k] = (T)X[k];
}

// one block per scene: the dense operator of the scene's coarsest level and its Cholesky factor (FP64)
template <typename T>
__global__ void k_amg_cfactor(AmgDev a) {
  int s = blockIdx.x;
  int l = a.sc_level[s], o = a.sc_off[s], m = a.sc_m[s];
  if (l <= 0 || m <= 0 || m > kAmgAgg) return;
  int n = 6 * m;
  __shared__ double A[kAmgDense * kAmgDense];
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k] = 0.0;
  __syncthreads();
  const AmgLevel& L = a.L[l];
  for (int I = o + (int)threadIdx.x; I < o + m; I += blockDim.x)
    for (int e = L.rs[I]; e < L.rs[I + 1]; ++e) {
      if (L.col[e] < o || L.col[e] >= o + m) continue;  // not reached: entries stay inside their scene
      const T* v = reinterpret_cast<const T*>(L.val) + 36 * (size_t)e;
      int r0 = 6 * (I - o), c0 = 6 * (L.col[e] - o);
      for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) A[n * (r0 + r) + c0 + c] += (double)v[6 * r + c];
    }
  __syncthreads();
  for (int j = 0; j < n; ++j) {  // right-looking Cholesky, rows below the pivot in parallel
    if (threadIdx.x == 0) {
      double dj = A[n * j + j];
      A[n * j + j] = sqrt(dj > 0.0 ? dj : 1e-300);
    }
    __syncthreads();
    double piv = A[n * j + j];
    for (int i = j + 1 + (int)threadIdx.x; i < n; i += blockDim.x) A[n * i + j] /= piv;
    __syncthreads();
    for (int i = j + 1 + (int)threadIdx.x; i < n; i += blockDim.x) {
      double lij = A[n * i + j];
      for (int k = j + 1; k <= i; ++k) A[n * i + k] -= lij * A[n * k + j];
    }
    __syncthreads();
  }
  double* out = a.chol + (size_t)kAmgDense * kAmgDense * s;
  for (int k = threadIdx.x; k < n * n; k += blockDim.x)  // the diagonal stored as its reciprocal
    out[k] = (k % (n + 1) == 0) ? 1.0 / A[k] : A[k];
}

// ---- the cycle --------------------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void amg_mat6(const T* Mg, const double (&x)[6], double (&y)[6]) {
  T M[36];
  load_words<36>(Mg, M);  // 16-byte loads: the blocks start at multiples of 144 (FP32) or 288 (FP64) bytes
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) s += (double)M[6 * r + c] * x[c];
    y[r] = s;
  }
}

template <typename T>
__device__ __forceinline__ void amg_load(const void* base, int i, double (&v)[6]) {
  const T* p = reinterpret_cast<const T*>(base) + 6 * (size_t)i;
#pragma unroll
  for (int k = 0; k < 6; ++k) v[k] = (double)p[k];
}
template <typename T>
__device__ __forceinline__ void amg_store(void* base, int i, const double (&v)[6]) {
  T* p = reinterpret_cast<T*>(base) + 6 * (size_t)i;
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = (T)v[k];
}

// restriction from level l to l + 1: r_{l+1}[I] = sum over the children k of P_k^T t_l[k]
// (P^T (v_p, v_y) = (v_p, dv x v_p + B^T v_y)), one lane per child (8 per coarse node), in the path's precision;
// then the coarse node's pre-smoothing x = w Dinv r when it is not its scene's coarsest node
template <typename T>
__global__ void __launch_bounds__(256) k_amg_restrict(DevArrays d, AmgDev a, int l) {
  constexpr int G = kAmgAgg;
  int I = blockIdx.x * (256 / G) + threadIdx.x / G, sub = threadIdx.x % G;
  const AmgLevel& C = a.L[l + 1];
  bool valid = I < C.n;
  T acc[6] = {0, 0, 0, 0, 0, 0};
  if (valid) {
    int k = C.cbeg[I] + sub;
    if (k < C.cend[I]) {
      Vec6<T> v = load6<T>(reinterpret_cast<const T*>(a.L[l].t), k);
      T dv[3], w[3];
      if (l == 0) {  // the particle's stored offset and B = 1/2 R(q)^T: B^T v_y
        const T* o = reinterpret_cast<const T*>(a.p0) + 12 * (size_t)k;
        dv[0] = o[0]; dv[1] = o[1]; dv[2] = o[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) w[r] = o[3 + r] * v.v[3] + o[6 + r] * v.v[4] + o[9 + r] * v.v[5];
      } else {
        const double *ck = a.L[l].cen + 3 * (size_t)k, *cI = C.cen + 3 * (size_t)I;
        dv[0] = (T)(ck[0] - cI[0]); dv[1] = (T)(ck[1] - cI[1]); dv[2] = (T)(ck[2] - cI[2]);
        w[0] = v.v[3]; w[1] = v.v[4]; w[2] = v.v[5];
      }
      acc[0] = v.v[0]; acc[1] = v.v[1]; acc[2] = v.v[2];
      acc[3] = dv[1] * v.v[2] - dv[2] * v.v[1] + w[0];
      acc[4] = dv[2] * v.v[0] - dv[0] * v.v[2] + w[1];
      acc[5] = dv[0] * v.v[1] - dv[1] * v.v[0] + w[2];
    }
  }
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o, G);
  if (!valid || sub != 0) return;
  store6<T>(reinterpret_cast<T*>(C.r), I, acc);
  if (C.parent[I] >= 0) {
    T M[36], y[6];
    load_words<36>(reinterpret_cast<const T*>(C.dinv) + 36 * (size_t)I, M);
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      T sum = 0;
#pragma unroll
      for (int c = 0; c < 6; ++c) sum += M[6 * r + c] * acc[c];
      y[r] = (T)a.omega * sum;
    }
    store6<T>(reinterpret_cast<T*>(C.x), I, y);
  }
}

// level l >= 1, non-coarsest nodes: mode 0 x = w Dinv r; mode 1 t = r - A x; mode 2 x += w Dinv t (the cycle uses
// mode 2; the pre-smoothing is part of the restriction and the residual has its own multi-lane kernel)
template <typename T>
__global__ void k_amg_level(AmgDev a, int l, int mode) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  const AmgLevel& L = a.L[l];
  if (I >= L.n || L.parent[I] < 0) return;
  double r[6], y[6];
  if (mode == 1) {
    amg_load<T>(L.r, I, r);
    for (int e = L.rs[I]; e < L.rs[I + 1]; ++e) {
      double x[6];
      amg_load<T>(L.x, L.col[e], x);
      amg_mat6<T>(reinterpret_cast<const T*>(L.val) + 36 * (size_t)e, x, y);
#pragma unroll
      for (int k = 0; k < 6; ++k) r[k] -= y[k];
    }
    amg_store<T>(L.t, I, r);
    return;
  }
  amg_load<T>(mode ? L.t : L.r, I, r);
  amg_mat6<T>(reinterpret_cast<const T*>(L.dinv) + 36 * (size_t)I, r, y);
  if (mode) {
    double x[6];
    amg_load<T>(L.x, I, x);
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] = x[k] + a.omega * y[k];
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] = a.omega * y[k];
  }
  amg_store<T>(L.x, I, y);
}

// one warp per scene: x = A^-1 r on the scene's coarsest level with its Cholesky factor (in shared memory, diagonal
// as reciprocals); lane t owns rows t and t + 32, the substitutions broadcast each solved entry with a shuffle
template <typename T>
__global__ void k_amg_csolve(AmgDev a) {
  int s = blockIdx.x;
  int l = a.sc_level[s], o = a.sc_off[s], m = a.sc_m[s];
  if (l <= 0 || m <= 0 || m > kAmgAgg) return;
  int n = 6 * m, t = threadIdx.x;
  __shared__ double Ls[kAmgDense * kAmgDense];
  const double* Lc = a.chol + (size_t)kAmgDense * kAmgDense * s;
  for (int k = t; k < n * n; k += 32) Ls[k] = Lc[k];
  const AmgLevel& L = a.L[l];
  const T* R = reinterpret_cast<const T*>(L.r) + 6 * (size_t)o;
  double w0 = t < n ? (double)R[t] : 0.0, w1 = t + 32 < n ? (double)R[t + 32] : 0.0;
  __syncwarp();
  for (int j = 0; j < n; ++j) {  // forward: L w = r
    double wj = __shfl_sync(0xffffffffu, j < 32 ? w0 : w1, j & 31) * Ls[n * j + j];
    if (t == (j & 31)) { if (j < 32) w0 = wj; else w1 = wj; }
    if (t > j && t < n) w0 -= Ls[n * t + j] * wj;
    if (t + 32 > j && t + 32 < n) w1 -= Ls[n * (t + 32) + j] * wj;
  }
  for (int j = n - 1; j >= 0; --j) {  // backward: L^T z = w
    double wj = __shfl_sync(0xffffffffu, j < 32 ? w0 : w1, j & 31) * Ls[n * j + j];
    if (t == (j & 31)) { if (j < 32) w0 = wj; else w1 = wj; }
    if (t < j) w0 -= Ls[n * j + t] * wj;
    if (t + 32 < j) w1 -= Ls[n * j + t + 32] * wj;
  }
  T* X = reinterpret_cast<T*>(L.x) + 6 * (size_t)o;
  if (t < n) X[t] = (T)w0;
  if (t + 32 < n) X[t + 32] = (T)w1;
}

// prolongation from level l + 1 to l (nodes whose scene has level l + 1): x_l[k] += P_k e[parent(k)]
// (P (t, w) = (t + w x dv, B w)); on level 0 the result goes to the PCG's z, kinematic rows kept at zero
template <typename T>
__global__ void k_amg_prolong(DevArrays d, AmgDev a, int l) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int n = l == 0 ? d.n : a.L[l].n;
  if (k >= n) return;
  int I = a.L[l].parent[k];
  if (I < 0) return;
  Vec6<T> e = load6<T>(reinterpret_cast<const T*>(a.L[l + 1].x), I);
  void* X = l == 0 ? d.vz : a.L[l].x;
  Vec6<T> x = load6<T>(reinterpret_cast<const T*>(X), k);
  T dv[3], wv[3];
  if (l == 0) {  // stored offset and B = 1/2 R(q)^T: B w
    const T* o = reinterpret_cast<const T*>(a.p0) + 12 * (size_t)k;
    dv[0] = o[0]; dv[1] = o[1]; dv[2] = o[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) wv[r] = o[3 + 3 * r] * e.v[3] + o[4 + 3 * r] * e.v[4] + o[5 + 3 * r] * e.v[5];
  } else {
    const double *ck = a.L[l].cen + 3 * (size_t)k, *cI = a.L[l + 1].cen + 3 * (size_t)I;
    dv[0] = (T)(ck[0] - cI[0]); dv[1] = (T)(ck[1] - cI[1]); dv[2] = (T)(ck[2] - cI[2]);
    wv[0] = e.v[3]; wv[1] = e.v[4]; wv[2] = e.v[5];
  }
  T o6[6];
  o6[0] = x.v[0] + e.v[0] + e.v[4] * dv[2] - e.v[5] * dv[1];
  o6[1] = x.v[1] + e.v[1] + e.v[5] * dv[0] - e.v[3] * dv[2];
  o6[2] = x.v[2] + e.v[2] + e.v[3] * dv[1] - e.v[4] * dv[0];
  o6[3] = x.v[3] + wv[0]; o6[4] = x.v[4] + wv[1]; o6[5] = x.v[5] + wv[2];
  if (l == 0 && d.kin[k])
#pragma unroll
    for (int t = 0; t < 6; ++t) o6[t] = (T)0;
  store6<T>(reinterpret_cast<T*>(X), k, o6);
}

// fine-level products with G lanes per row (the lanes split the row's entries, the diagonal block goes to lane 0):
// mode 0: q = H p (the PCG's product: bonds and active contacts, kinematic rows zero); mode 1: t = r - A_0 x
// (the cycle's residual: bonds only; kinematic rows t = r - x, x vanishes on them)
template <typename T, int G>
__global__ void __launch_bounds__(256) k_amg_fine(DevArrays d, AmgDev a, int mode) {
  int i = blockIdx.x * (256 / G) + threadIdx.x / G;
  int sub = threadIdx.x % G;
  bool valid = i < d.n;
  const T* X = reinterpret_cast<const T*>(mode ? d.vz : d.vp_);
  T y[6] = {0, 0, 0, 0, 0, 0};
  bool kin = valid && d.kin[i];
  if (valid && !kin) {
    if (sub == 0) {
      Vec6<T> xi = load6<T>(X, i);
      sym6_mul<T>(reinterpret_cast<const T*>(d.D) + kDiagStride * (size_t)i, xi.v, y);
    }
    int nbond = d.inc_start[i + 1] - d.inc_start[i];
    int nent = nbond + ((mode == 0 && d.k_self > 0.0) ? d.c_act[i] : 0);
    for (int k = sub; k < nent; k += G) row_entry<T, false>(d, i, k, nbond, X, y);
  }
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] += __shfl_down_sync(0xffffffffu, y[k], o, G);
  if (!valid || sub != 0) return;
  if (mode == 0) {
    if (kin)
#pragma unroll
      for (int k = 0; k < 6; ++k) y[k] = (T)0;
    store6<T>(reinterpret_cast<T*>(d.vq_), i, y);
  } else {
    Vec6<T> r = load6<T>(reinterpret_cast<const T*>(d.vr), i);
    T t[6];
    if (kin) {
      Vec6<T> xi = load6<T>(X, i);
#pragma unroll
      for (int k = 0; k < 6; ++k) t[k] = r.v[k] - xi.v[k];
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) t[k] = r.v[k] - y[k];
    }
    store6<T>(reinterpret_cast<T*>(a.L[0].t), i, t);
  }
}

// coarse-level residual t = r - A x with 8 lanes per row (non-coarsest rows), in the path's precision (the coarse
// operators are stored in it; FP64 arithmetic here would make the mixed path's coarse levels FP64-bound)
template <typename T>
__global__ void __launch_bounds__(256) k_amg_cresid(AmgDev a, int l) {
  constexpr int G = 8;
  int I = blockIdx.x * (256 / G) + threadIdx.x / G;
  int sub = threadIdx.x % G;
  const AmgLevel& L = a.L[l];
  bool valid = I < L.n && L.parent[I] >= 0;
  T y[6] = {0, 0, 0, 0, 0, 0};
  const T* X = reinterpret_cast<const T*>(L.x);
  if (valid)
    for (int e = L.rs[I] + sub; e < L.rs[I + 1]; e += G) {
      Vec6<T> x = load6<T>(X, L.col[e]);
      T M[36];
      load_words<36>(reinterpret_cast<const T*>(L.val) + 36 * (size_t)e, M);
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        T s = y[r];
#pragma unroll
        for (int c = 0; c < 6; ++c) s += M[6 * r + c] * x.v[c];
        y[r] = s;
      }
    }
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] += __shfl_down_sync(0xffffffffu, y[k], o, G);
  if (!valid || sub != 0) return;
  Vec6<T> r = load6<T>(reinterpret_cast<const T*>(L.r), I);
  T t[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) t[k] = r.v[k] - y[k];
  store6<T>(reinterpret_cast<T*>(L.t), I, t);
}

static inline int amg_blocks(int64_t n) { return (int)((n + 127) / 128); }
static inline int amg_lane_blocks(int64_t n, int g) { return (int)((n * g + 255) / 256); }

template <typename T>
static int amg_setup_t(const DevArrays& d, const AmgDev& a, int n_scenes, cudaStream_t s) {
  int k = 0;
  for (int l = 1; l < a.nl; ++l) {
    if (a.L[l].n == 0) continue;
    k_amg_cent<<<amg_blocks(a.L[l].n), 128, 0, s>>>(d, a, l);
    ++k;
  }
  k_amg_p0<T><<<amg_blocks(d.n), 128, 0, s>>>(d, a);
  ++k;
  for (int l = 1; l < a.nl; ++l) {
    if (a.L[l].nnz == 0) continue;
    if (l == 1) k_amg_gal1<T><<<amg_blocks(a.L[1].nnz), 128, 0, s>>>(d, a);
    else k_amg_gal<T><<<amg_blocks(a.L[l].nnz), 128, 0, s>>>(a, l);
    k_amg_dinv<T><<<amg_blocks(a.L[l].n), 128, 0, s>>>(a, l);
    k += 2;
  }
  if (n_scenes > 0) {
    k_amg_cfactor<T><<<n_scenes, 64, 0, s>>>(a);
    ++k;
  }
  return k;
}

int launch_amg_setup(const DevArrays& d, const AmgDev& a, int n_scenes, cudaStream_t s) {
  if (d.n == 0 || a.nl < 2) return 0;
  return d.mixed ? amg_setup_t<float>(d, a, n_scenes, s) : amg_setup_t<double>(d, a, n_scenes, s);
}

template <typename T>
static int amg_cycle_t(const DevArrays& d, const AmgDev& a, int n_scenes, cudaStream_t s) {
  // the level-0 pre-smoothing (z = w Dinv r) was written by the PCG stage that produced r
  int k = 0, top = a.nl - 1;
  k_amg_fine<T, 4><<<amg_lane_blocks(d.n, 4), 256, 0, s>>>(d, a, 1);
  k_amg_restrict<T><<<amg_lane_blocks(a.L[1].n, kAmgAgg), 256, 0, s>>>(d, a, 0);
  k += 2;
  for (int l = 1; l < top; ++l) {
    if (a.L[l + 1].n == 0) break;
    k_amg_cresid<T><<<amg_lane_blocks(a.L[l].n, 8), 256, 0, s>>>(a, l);
    k_amg_restrict<T><<<amg_lane_blocks(a.L[l + 1].n, kAmgAgg), 256, 0, s>>>(d, a, l);
    k += 2;
  }
  k_amg_csolve<T><<<n_scenes, 32, 0, s>>>(a);
  ++k;
  for (int l = top - 1; l >= 1; --l) {
    if (a.L[l + 1].n == 0) continue;
    k_amg_prolong<T><<<amg_blocks(a.L[l].n), 128, 0, s>>>(d, a, l);
    k_amg_cresid<T><<<amg_lane_blocks(a.L[l].n, 8), 256, 0, s>>>(a, l);
    k_amg_level<T><<<amg_blocks(a.L[l].n), 128, 0, s>>>(a, l, 2);
    k += 3;
  }
  k_amg_prolong<T><<<amg_blocks(d.n), 128, 0, s>>>(d, a, 0);
  k_amg_fine<T, 4><<<amg_lane_blocks(d.n, 4), 256, 0, s>>>(d, a, 1);
  return k + 2;  // the post-smoothing is finished by the PCG stage that reads z
}

int launch_amg_cycle(const DevArrays& d, const AmgDev& a, int n_scenes, cudaStream_t s) {
  if (d.n == 0 || a.nl < 2) return 0;
  return d.mixed ? amg_cycle_t<float>(d, a, n_scenes, s) : amg_cycle_t<double>(d, a, n_scenes, s);
}

// ---- PCG with the cycle as preconditioner (textbook form, per-scene state in SceneCtl) ---------------------------

// w Dinv v (the cycle's level-0 smoothing step) for particle i
template <typename T>
__device__ __forceinline__ void amg_smooth_row(const DevArrays& d, double omega, int i, const T (&v)[6], T (&y)[6]) {
  sym6_mul<T>(reinterpret_cast<const T*>(d.Dinv) + kDiagStride * (size_t)i, v, y);
#pragma unroll
  for (int k = 0; k < 6; ++k) y[k] = (T)omega * y[k];
}

// The level-0 smoothing steps of the cycle are done here: the stages that produce a new residual r (0, 6, 3) also
// write the pre-smoothed z = w Dinv r, and the stages that read the cycle's result (1, 4) first finish it with the
// post-smoothing z += w Dinv t (t = the cycle's last level-0 residual).
template <typename T>
__global__ void __launch_bounds__(kTile) k_apcg_vec(DevArrays d, AmgDev a, int stage) {
  int t = blockIdx.x;
  int i = d.ptile_start[t] + threadIdx.x;
  int s = d.ptile_scene[t];
  double acc[1] = {0.0};
  if (i < d.ptile_start[t + 1]) {
    SceneCtl& c = d.sc[s];
    T* X = reinterpret_cast<T*>(d.vx);
    T* R = reinterpret_cast<T*>(d.vr);
    T* Z = reinterpret_cast<T*>(d.vz);
    T* P = reinterpret_cast<T*>(d.vp_);
    T* Q = reinterpret_cast<T*>(d.vq_);
    if (stage == 0 || stage == 6) {  // r = b (-g, or the given vr) with kinematic rows zero, x = 0, acc = |b|^2
      T r[6], x[6] = {0, 0, 0, 0, 0, 0};
      const double* g = d.g + 6 * (size_t)i;
      Vec6<T> rv = load6<T>(R, i);
      bool on = c.newton_active && !d.kin[i];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        double b = on ? (stage == 0 ? -g[k] : (double)rv.v[k]) : 0.0;
        r[k] = (T)b;
        acc[0] += (double)r[k] * (double)r[k];
      }
      store6<T>(X, i, x);
      store6<T>(R, i, r);
      T z[6];
      amg_smooth_row<T>(d, a.omega, i, r, z);
      store6<T>(Z, i, z);
    } else if (stage == 1 || stage == 4) {  // z += w Dinv t (kinematic rows zero), acc = r.z
      DotAcc<T> dot;
      Vec6<T> r = load6<T>(R, i), z = load6<T>(Z, i), t = load6<T>(reinterpret_cast<const T*>(a.L[0].t), i);
      T y[6];
      amg_smooth_row<T>(d, a.omega, i, t.v, y);
      bool kin = d.kin[i];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        z.v[k] = kin ? (T)0 : z.v[k] + y[k];
        dot.add(r.v[k], z.v[k]);
      }
      store6<T>(Z, i, z.v);
      acc[0] = dot.value();
    } else if (stage == 2) {  // acc = p.q
      DotAcc<T> dot;
      Vec6<T> p = load6<T>(P, i), q = load6<T>(Q, i);
#pragma unroll
      for (int k = 0; k < 6; ++k) dot.add(p.v[k], q.v[k]);
      acc[0] = dot.value();
    } else if (stage == 3) {  // x += alpha p, r -= alpha q, acc = |r|^2
      Vec6<T> r = load6<T>(R, i);
      if (c.pcg_active) {
        Vec6<T> x = load6<T>(X, i), p = load6<T>(P, i), q = load6<T>(Q, i);
        T al = (T)c.alpha;
        T xo[6], ro[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          xo[k] = x.v[k] + al * p.v[k];
          ro[k] = r.v[k] - al * q.v[k];
          r.v[k] = ro[k];
        }
        store6<T>(X, i, xo);
        store6<T>(R, i, ro);
      }
      DotAcc<T> dot;
#pragma unroll
      for (int k = 0; k < 6; ++k) dot.add(r.v[k], r.v[k]);
      acc[0] = dot.value();
      T z[6];
      amg_smooth_row<T>(d, a.omega, i, r.v, z);
      store6<T>(Z, i, z);
    } else if (stage == 5) {  // p = z + beta p (beta = 0 on the first step)
      if (c.pcg_active) {
        Vec6<T> z = load6<T>(Z, i), p = load6<T>(P, i);
        T be = (T)c.beta;
        T po[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) po[k] = z.v[k] + be * p.v[k];
        store6<T>(P, i, po);
      }
    }
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) d.part_p[kPartials * t] = acc[0];
}

// per scene (one warp): the tile partials of the last k_apcg_vec (lane-strided sums and a fixed shuffle tree, so
// the order is fixed), then the stage's scalar update
__global__ void k_apcg_scene(DevArrays d, int stage) {
  int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= d.n_scenes) return;
  SceneCtl& c = d.sc[s];
  double v = 0.0;
  for (int t = d.ptile_begin[s] + lane; t < d.ptile_begin[s + 1]; t += 32) v += d.part_p[kPartials * t];
  v = warp_sum(v);
  if (lane != 0) return;
  if (stage == 0 || stage == 6) {
    c.pcg_iters = 0;
    c.pcg_thr2 = c.eps_r * c.eps_r * v;
    c.bnorm = sqrt(v);
    c.pcg_active = c.newton_active && v > c.pcg_thr2;
    c.beta = 0.0;
  } else if (stage == 1) {
    c.rz = v;
  } else if (stage == 2) {
    if (c.pcg_active) {
      if (!(v > 0.0) || !(c.rz > 0.0)) c.pcg_active = 0;  // breakdown
      else c.alpha = c.rz / v;
    }
  } else if (stage == 3) {
    if (c.pcg_active) {
      c.pcg_iters += 1;
      if (!(v > c.pcg_thr2) || c.pcg_iters >= d.pcg_max) c.pcg_active = 0;
    }
    if (c.pcg_active) atomicAdd(&d.cnt->n_active, 1);
  } else if (stage == 4) {
    if (c.pcg_active) {
      c.beta = v / c.rz;
      c.rz = v;
    }
  }
}

__global__ void k_amg_loop(DevArrays d, unsigned long long cond, int what) {
  if (what == 0) {  // a solve starts: its first trip always runs
    d.cnt->amg_trips = 0;
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 1u);
  } else if (what == 1) {  // a trip starts
    d.cnt->n_active = 0;
  } else {  // a trip ends
    int trips = ++d.cnt->amg_trips;
    d.cnt->loops_amg += 1;
    unsigned go = d.cnt->n_active > 0 && trips <= d.pcg_max && !step_aborted(d);
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, go);
  }
}

int launch_amg_loop_init(const DevArrays& d, unsigned long long cond, cudaStream_t s) {
  k_amg_loop<<<1, 1, 0, s>>>(d, cond, 0);
  return 1;
}
int launch_amg_iteration_begin(const DevArrays& d, cudaStream_t s) {
  k_amg_loop<<<1, 1, 0, s>>>(d, 0ull, 1);
  return 1;
}
int launch_amg_loop_cond(const DevArrays& d, unsigned long long cond, cudaStream_t s) {
  k_amg_loop<<<1, 1, 0, s>>>(d, cond, 2);
  return 1;
}

int launch_amg_pcg_stage(const DevArrays& d, const AmgDev& a, int stage, cudaStream_t s) {
  if (d.n == 0) return 0;
  int k = 0;
  if (stage == 2) {  // q = H p first
    if (d.mixed) k_amg_fine<float, 4><<<amg_lane_blocks(d.n, 4), 256, 0, s>>>(d, a, 0);
    else k_amg_fine<double, 4><<<amg_lane_blocks(d.n, 4), 256, 0, s>>>(d, a, 0);
    ++k;
  }
  if (stage != 5) {
    if (d.mixed) k_apcg_vec<float><<<d.n_ptiles, kTile, 0, s>>>(d, a, stage);
    else k_apcg_vec<double><<<d.n_ptiles, kTile, 0, s>>>(d, a, stage);
    k_apcg_scene<<<(d.n_scenes + 3) / 4, 128, 0, s>>>(d, stage);
    k += 2;
  }
  if (stage == 1 || stage == 4 || stage == 5) {  // then p = z + beta p
    if (d.mixed) k_apcg_vec<float><<<d.n_ptiles, kTile, 0, s>>>(d, a, 5);
    else k_apcg_vec<double><<<d.n_ptiles, kTile, 0, s>>>(d, a, 5);
    ++k;
  }
  return k;
}

}  // namespace bdem
