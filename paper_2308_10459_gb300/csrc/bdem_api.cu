// bdem_api.cu -- host implementation of the C ABI in include/bdem.h: validation, bond rest data (Sec. 3.2),
// device memory, and the host-driven Newton / line-search loop of Alg. 3 around the device kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bdem.h"
#include "bdem_internal.h"

using namespace bdem;

struct bdem_sim {
  bdem_config cfg;
  bdem_allocator hook{};              // caller's device-memory hook (alloc == NULL: cudaMalloc)
  int32_t n = 0, n_scenes = 0;
  int64_t nb = 0;
  cudaStream_t stream = 0;
  std::vector<int64_t> offsets;
  std::vector<int32_t> pscene;
  std::vector<double> radius, mass;
  std::vector<uint8_t> kin;
  std::vector<bdem_material> mats;
  std::vector<int32_t> perm, iperm;  // internal -> caller particle index, caller -> internal
  std::vector<int32_t> deg;          // bonds per particle (internal order), weights of the PCG partition
  std::vector<int32_t> ext_i, ext_j;  // bonds in the caller's order of addition (caller indices, i < j)
  std::vector<int32_t> bond_ext2int_h;
  std::vector<int32_t> bi, bj, bmat;  // stored bond order (internal indices), i < j, sorted by (i, j)
  std::vector<double4> rest, stiff;   // host copies of the bond rest data (d0, l0), (kn, kt, kb, ktw)
  std::vector<double> brk;
  DevArrays d{};
  std::vector<void*> allocs;          // every device buffer owned by the sim
  std::string err;
  int64_t launches = 0;
  int pcg_blocks = 0;
  int pcg_product = 1;                // 1: warp-cooperative staging of the bond blocks (k_pcg MODE 2); 0: per-lane
  double* dbg_buf = nullptr;          // device scratch of the inspection calls
  size_t dbg_cap = 0;
  double* stage = nullptr;            // device staging for the caller-order state arrays (14 doubles per particle)
  uint8_t* flag_stage = nullptr;      // device staging for bond flags
  bool system_ready = false;
  // phase timing
  bool prof_on = false;
  bdem_profile prof{};
  std::vector<cudaEvent_t> ev_pool;
  struct Pending { int ph; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  cudaEvent_t ev_open = nullptr;
  int ph_open = -1;
  bool nvtx_open = false;
  // captured step graph: one graph launch per step, the Newton and line-search loops run as conditional while
  // nodes decided on the device
  bool graph_enabled = true;
  bool graph_failed = false;          // capture or instantiation was refused: steps use the host-driven loop
  bool contacts_sized = false;        // a host-driven step has sized the contact arrays
  std::string graph_err;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  DevArrays graph_d{};                // the arrays the graph was captured with (kernel arguments are by value)
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  int g_pre = 0, g_body = 0, g_ls = 0, g_post = 0, g_ref = 0, g_amg = 0;  // kernels per graph segment
  AmgDev graph_amg{};                 // the AMG hierarchy the step graph was captured with
  int64_t graph_steps = 0;
  // aggregation AMG preconditioner (bdem_config.preconditioner)
  AmgDev amg{};
  int64_t amg_nb = -1;                // bond count the AMG patterns were built for (-1: not built)
  std::vector<void*> amg_allocs;
  cudaStream_t amg_cap = nullptr;     // capture stream of the AMG-PCG iteration graph
  cudaGraphExec_t amg_exec = nullptr; // one PCG iteration (product, update, stop test, cycle, direction)
  DevArrays amg_gd{};                 // the arrays and hierarchy the iteration graph was captured with
  AmgDev amg_ga{};
  int amg_gk = 0;                     // kernels per iteration graph
};

static cudaEvent_t ev_get(bdem_sim* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// phases of the host-driven step: an NVTX range each (for timeline tools), and CUDA events when timing is on
static const char* const kPhaseName[BDEM_N_PHASES] = {"predict", "contact", "grad", "hess", "pcg", "linesearch",
                                                      "finish"};

static void phase_begin(bdem_sim* s, int ph) {
  if (s->nvtx_open) nvtxRangePop();  // a phase left open by an early loop exit
  nvtxRangePushA(kPhaseName[ph]);
  s->nvtx_open = true;
  if (!s->prof_on) return;
  s->ev_open = ev_get(s);
  s->ph_open = ph;
  cudaEventRecord(s->ev_open, s->stream);
}

static void phase_end(bdem_sim* s) {
  if (s->nvtx_open) {
    nvtxRangePop();
    s->nvtx_open = false;
  }
  if (!s->prof_on || s->ph_open < 0) return;
  cudaEvent_t b = ev_get(s);
  cudaEventRecord(b, s->stream);
  s->pending.push_back({s->ph_open, s->ev_open, b});
  s->ph_open = -1;
  s->ev_open = nullptr;
}

// called after a stream synchronisation: every pending interval has completed
static void phase_collect(bdem_sim* s) {
  for (auto& p : s->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      s->prof.ms[p.ph] += ms;
      s->prof.intervals[p.ph] += 1;
    }
    s->ev_pool.push_back(p.a);
    s->ev_pool.push_back(p.b);
  }
  s->pending.clear();
}

static std::string g_create_err;

static bdem_status fail(bdem_sim* s, bdem_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  else g_create_err = buf;
  return st;
}

#define CUDA_TRY(sim, call)                                                                            \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess)                                                                             \
      return fail(sim, e_ == cudaErrorMemoryAllocation ? BDEM_E_NOMEM : BDEM_E_CUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                             \
  } while (0)

#define TRY(expr)                  \
  do {                             \
    bdem_status st_ = (expr);      \
    if (st_ != BDEM_OK) return st_; \
  } while (0)

// device buffers of the sim: from the caller's allocator hook when one was given, else cudaMalloc; zero-filled
static void raw_free(bdem_sim* s, void* p) {
  if (s->hook.alloc) s->hook.free(s->hook.ctx, p, (void*)s->stream);
  else cudaFree(p);
}

static bdem_status dalloc(bdem_sim* s, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (s->hook.alloc) {
    *p = s->hook.alloc(s->hook.ctx, bytes, (void*)s->stream);
    if (!*p) return fail(s, BDEM_E_NOMEM, "the allocator hook returned NULL for %zu bytes", bytes);
    if (reinterpret_cast<uintptr_t>(*p) % 256 != 0) {
      raw_free(s, *p);
      *p = nullptr;
      return fail(s, BDEM_E_INVALID, "the allocator hook returned memory that is not 256-byte aligned");
    }
    s->allocs.push_back(*p);
    cudaError_t e2 = cudaMemsetAsync(*p, 0, bytes, s->stream);
    if (e2 != cudaSuccess) return fail(s, BDEM_E_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e2));
    return BDEM_OK;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(s, e == cudaErrorMemoryAllocation ? BDEM_E_NOMEM : BDEM_E_CUDA, "cudaMalloc(%zu bytes): %s", bytes,
                cudaGetErrorString(e));
  }
  cudaError_t e2 = cudaMemset(*p, 0, bytes);
  s->allocs.push_back(*p);
  if (e2 != cudaSuccess) return fail(s, BDEM_E_CUDA, "cudaMemset: %s", cudaGetErrorString(e2));
  return BDEM_OK;
}

template <typename P>
static bdem_status dalloc_t(bdem_sim* s, P** p, size_t count) {
  return dalloc(s, reinterpret_cast<void**>(p), sizeof(P) * count);
}

static void dfree(bdem_sim* s, void* p) {
  if (!p) return;
  auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
  if (it != s->allocs.end()) s->allocs.erase(it);
  raw_free(s, p);
}

static bool fin(double x) { return std::isfinite(x); }

static bdem_status check_launch(bdem_sim* s, int k) {
  s->launches += k;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(s, BDEM_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return BDEM_OK;
}

static void phase_collect(bdem_sim* s);

static bdem_status sync(bdem_sim* s) {
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return fail(s, BDEM_E_CUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
  phase_collect(s);
  return BDEM_OK;
}

// ------------------------------------------------------------------------------------------------
// quaternion helpers for the host-side rest data (App. A conventions, scalar last)
// ------------------------------------------------------------------------------------------------

static void hq_mul(const double a[4], const double b[4], double o[4]) {
  o[0] = a[3] * b[0] + b[3] * a[0] + a[1] * b[2] - a[2] * b[1];
  o[1] = a[3] * b[1] + b[3] * a[1] + a[2] * b[0] - a[0] * b[2];
  o[2] = a[3] * b[2] + b[3] * a[2] + a[0] * b[1] - a[1] * b[0];
  o[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
}

// d = q (.) v = vec(q (v, 0) conj(q))
static void hq_rotate(const double q[4], const double v[3], double d[3]) {
  double x[4] = {v[0], v[1], v[2], 0.0}, t[4], qc[4] = {-q[0], -q[1], -q[2], q[3]}, r[4];
  hq_mul(q, x, t);
  hq_mul(t, qc, r);
  d[0] = r[0];
  d[1] = r[1];
  d[2] = r[2];
}

// ------------------------------------------------------------------------------------------------
// create
// ------------------------------------------------------------------------------------------------

static bdem_status check_config(const bdem_config* c) {
  if (!c) return fail(nullptr, BDEM_E_INVALID, "config is NULL");
  if (!(c->dt > 0.0) || !fin(c->dt)) return fail(nullptr, BDEM_E_INVALID, "dt must be positive and finite");
  for (int k = 0; k < 3; ++k)
    if (!fin(c->gravity[k])) return fail(nullptr, BDEM_E_INVALID, "gravity must be finite");
  if (!(c->newton_rel_tol >= 0.0) || !fin(c->newton_rel_tol))
    return fail(nullptr, BDEM_E_INVALID, "newton_rel_tol must be finite and >= 0");
  if (!(c->newton_abs_tol >= 0.0) || !fin(c->newton_abs_tol))
    return fail(nullptr, BDEM_E_INVALID, "newton_abs_tol must be finite and >= 0");
  if (c->pcg_refine < 0 || c->pcg_refine > 16) return fail(nullptr, BDEM_E_INVALID, "pcg_refine must be in [0, 16]");
  if (c->newton_max_iter < 1 || c->pcg_max_iter < 1 || c->ls_max_halvings < 0 || c->ls_max_halvings > 1000)
    return fail(nullptr, BDEM_E_INVALID, "iteration caps must be newton >= 1, pcg >= 1, 0 <= line search <= 1000");
  if (c->precision != BDEM_FP64 && c->precision != BDEM_MIXED)
    return fail(nullptr, BDEM_E_INVALID, "precision must be BDEM_FP64 or BDEM_MIXED");
  if (c->spd_mode != BDEM_SPD_EIG) return fail(nullptr, BDEM_E_INVALID, "spd_mode must be BDEM_SPD_EIG");
  if (c->optimizer != BDEM_OPT_SECOND_ORDER && c->optimizer != BDEM_OPT_FIRST_ORDER)
    return fail(nullptr, BDEM_E_INVALID, "optimizer must be BDEM_OPT_SECOND_ORDER or BDEM_OPT_FIRST_ORDER");
  if (c->integrator != BDEM_INT_EULER && c->integrator != BDEM_INT_MIDPOINT)
    return fail(nullptr, BDEM_E_INVALID, "integrator must be BDEM_INT_EULER or BDEM_INT_MIDPOINT");
  if (c->preconditioner != BDEM_PRECOND_BLOCK_JACOBI && c->preconditioner != BDEM_PRECOND_AMG)
    return fail(nullptr, BDEM_E_INVALID, "preconditioner must be BDEM_PRECOND_BLOCK_JACOBI or BDEM_PRECOND_AMG");
  if (!(c->k_ground >= 0.0) || !(c->k_self >= 0.0) || !(c->contact_skin >= 0.0) || !fin(c->ground_z) ||
      !fin(c->k_ground) || !fin(c->k_self) || !fin(c->contact_skin))
    return fail(nullptr, BDEM_E_INVALID, "contact parameters must be finite and >= 0");
  if (!(c->friction_slide >= 0.0) || !(c->friction_roll >= 0.0) || !fin(c->friction_slide) || !fin(c->friction_roll))
    return fail(nullptr, BDEM_E_INVALID, "friction coefficients must be finite and >= 0");
  return BDEM_OK;
}

static size_t wsize(const bdem_sim* s) { return s->cfg.precision == BDEM_MIXED ? sizeof(float) : sizeof(double); }

static bdem_status alloc_particles(bdem_sim* s) {
  DevArrays& d = s->d;
  size_t n = (size_t)std::max(s->n, 1);
  double4** p4[] = {&d.xp, &d.xq, &d.x0p, &d.x0q, &d.vp, &d.vq, &d.hp, &d.hq, &d.tp, &d.tq};
  for (double4** p : p4) TRY(dalloc_t(s, p, n));
  size_t w = wsize(s);
  TRY(dalloc_t(s, &d.coef, n));
  TRY(dalloc_t(s, &d.pscene, n));
  TRY(dalloc_t(s, &d.kin, n));
  TRY(dalloc_t(s, &d.g, 6 * n));
  TRY(dalloc(s, &d.D, w * kDiagStride * n));
  TRY(dalloc(s, &d.Dinv, w * kDiagStride * n));
  void** pv[] = {&d.vx, &d.vr, &d.vz, &d.vp_, &d.vq_, &d.vs, &d.vr2, &d.vs2, &d.vq2};
  for (void** p : pv) TRY(dalloc(s, p, w * 6 * n));
  if (d.refine) TRY(dalloc_t(s, &d.x64, 6 * n));
  int hs = 1024;
  while (hs < 2 * (int)n) hs <<= 1;
  d.hash_size = hs;
  size_t mx = std::max((size_t)hs, n);
  TRY(dalloc_t(s, &d.c_start, n + 1));
  TRY(dalloc_t(s, &d.cell_key, n));
  TRY(dalloc_t(s, &d.hash_count, (size_t)hs));
  TRY(dalloc_t(s, &d.hash_start, (size_t)hs + 1));
  TRY(dalloc_t(s, &d.hash_ids, n));
  TRY(dalloc_t(s, &d.cnt_tmp, mx));
  TRY(dalloc_t(s, &d.scan_tmp, mx / 1024 + 4));
  d.c_cap = (int32_t)std::max<size_t>(1024, (s->cfg.k_self > 0.0 ? 16 : 1) * n);
  TRY(dalloc_t(s, &d.c_nbr, (size_t)d.c_cap));
  TRY(dalloc_t(s, &d.c_anbr, (size_t)d.c_cap));
  TRY(dalloc(s, &d.c_blk, 4 * w * d.c_cap));
  TRY(dalloc_t(s, &d.c_act, n));
  TRY(dalloc_t(s, &s->stage, 14 * n + 128));
  TRY(dalloc_t(s, &d.perm, n));
  TRY(dalloc_t(s, &d.sc, (size_t)std::max(s->n_scenes, 1)));
  TRY(dalloc_t(s, &d.cnt, 1));
  return BDEM_OK;
}

// particle tiles (<= kTile rows inside one scene) and their per-scene ranges
static bdem_status build_particle_tiles(bdem_sim* s) {
  std::vector<int32_t> start, scene, begin(s->n_scenes + 1, 0);
  for (int sc = 0; sc < s->n_scenes; ++sc) {
    begin[sc] = (int32_t)scene.size();
    for (int64_t a = s->offsets[sc]; a < s->offsets[sc + 1]; a += kTile) {
      start.push_back((int32_t)a);
      scene.push_back(sc);
    }
  }
  begin[s->n_scenes] = (int32_t)scene.size();
  start.push_back(s->n);
  DevArrays& d = s->d;
  d.n_ptiles = (int32_t)scene.size();
  TRY(dalloc_t(s, &d.ptile_start, start.size()));
  TRY(dalloc_t(s, &d.ptile_scene, std::max<size_t>(scene.size(), 1)));
  TRY(dalloc_t(s, &d.ptile_begin, begin.size()));
  TRY(dalloc_t(s, &d.part_p, (size_t)kPartials * std::max(d.n_ptiles, 1)));
  CUDA_TRY(s, cudaMemcpy(d.ptile_start, start.data(), sizeof(int32_t) * start.size(), cudaMemcpyHostToDevice));
  if (!scene.empty())
    CUDA_TRY(s, cudaMemcpy(d.ptile_scene, scene.data(), sizeof(int32_t) * scene.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.ptile_begin, begin.data(), sizeof(int32_t) * begin.size(), cudaMemcpyHostToDevice));
  return BDEM_OK;
}

// 21-bit spread for 3-D Morton codes (bits of x land at every third position)
static uint64_t spread3(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

// internal order: inside each scene, particles sorted by the Morton code of their initial position (ties by index)
static void morton_order(const int64_t* offsets, int n_scenes, const double* pos, std::vector<int32_t>& perm) {
  int64_t n = offsets[n_scenes];
  perm.resize(n);
  std::vector<uint64_t> code(n);
  for (int sc = 0; sc < n_scenes; ++sc) {
    int64_t a = offsets[sc], b = offsets[sc + 1];
    if (b <= a) continue;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = a; i < b; ++i)
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], pos[3 * i + k]);
        hi[k] = std::max(hi[k], pos[3 * i + k]);
      }
    double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    double sc_q = 2097151.0 / ext;
    for (int64_t i = a; i < b; ++i) {
      uint64_t q[3];
      for (int k = 0; k < 3; ++k) q[k] = (uint64_t)std::min(2097151.0, std::max(0.0, (pos[3 * i + k] - lo[k]) * sc_q));
      code[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
      perm[i] = (int32_t)i;
    }
    std::sort(perm.begin() + a, perm.begin() + b, [&](int32_t x, int32_t y) {
      return code[x] != code[y] ? code[x] < code[y] : x < y;
    });
  }
}

// kernel variant (DevArrays::pcg_mode) of a product setting: 3 the fused one-barrier PCG, 2 and 1 the double- and
// single-buffered cooperative staging, 0 per-lane loads (with the rows and entries staged when they fit)
static int pcg_mode_of(int product, int staged) {
  return product == 3 ? 4 : product == 2 ? 3 : product == 1 ? 2 : (staged ? 1 : 0);
}

// balanced PCG row ranges per block and their intersections with the scenes (segments)

static bdem_status build_pcg_segments(bdem_sim* s, int lanes, int grid) {
  DevArrays& d = s->d;
  int64_t n = s->n;
  if (grid < 1) grid = 1;
  if (grid > kPcgMaxBlocks) grid = kPcgMaxBlocks;
  if (n > 0 && grid > n) grid = (int)n;
  std::vector<int32_t> seg_row, seg_scene, block_seg(grid + 1, 0), scene_seg(s->n_scenes + 1, 0);
  // block boundaries at equal cumulative work, a row weighing 4 + its bond count (the product's entries)
  std::vector<int64_t> cum(n + 1, 0), bounds(grid + 1, 0);
  for (int64_t i = 0; i < n; ++i) cum[i + 1] = cum[i] + 4 + s->deg[i];
  for (int b = 1; b < grid; ++b) {
    int64_t target = cum[n] * b / grid;
    bounds[b] = std::lower_bound(cum.begin(), cum.end(), target) - cum.begin();
    bounds[b] = std::max(bounds[b], bounds[b - 1]);
  }
  bounds[grid] = n;
  int64_t max_rows = 0, max_ent = 0;
  for (int b = 0; b < grid; ++b) {
    max_rows = std::max(max_rows, bounds[b + 1] - bounds[b]);
    int64_t ent = 0;
    for (int64_t i = bounds[b]; i < bounds[b + 1]; ++i) ent += s->deg[i];
    max_ent = std::max(max_ent, ent);
  }
  // the rows and entries are staged in shared memory when a block's share fits beside the other blocks of its SM
  // (the grid's blocks per SM share 227 KB); otherwise they are read from L2 at every product
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t per_sm = std::max(1, (grid + sms - 1) / std::max(sms, 1));
  const int64_t budget = std::min<int64_t>(200 * 1024, 227 * 1024 / per_sm - 4 * 1024);
  const int staged = max_rows * (int64_t)sizeof(int4) + max_ent * (int64_t)sizeof(int2) <= budget;
  // the cooperative product stages the row descriptors and one bond block per thread (its grid is shrunk to what is
  // co-resident with that shared memory by apply_pcg_shape)
  // many scenes (at most kEvenPcgScenes) and a product that can read its rows from L2: the rows of the scenes still
  // iterating are split evenly over the grid at every iteration, when no block's share can span more than
  // kEvenPcgSegs scenes (a share never exceeds ceil(n / grid) rows, the smallest scene with rows bounds how many it
  // spans)
  int even = 0;
  if (s->n_scenes > kLocalPcgScenes && s->n_scenes <= kEvenPcgScenes && s->pcg_product <= 2 && n > 0) {
    int64_t min_rows = n;
    for (int sc = 0; sc < s->n_scenes; ++sc) {
      const int64_t r = s->offsets[sc + 1] - s->offsets[sc];
      if (r > 0) min_rows = std::min(min_rows, r);
    }
    const int64_t share = (n + grid - 1) / grid;
    even = 2 + (share + min_rows - 1) / min_rows <= kEvenPcgSegs;
  }
  const int mode = even && s->pcg_product == 0 ? 0 : pcg_mode_of(s->pcg_product, staged);
  // the cooperative products stage the row descriptors beside their slot buffers when both fit the same budget;
  // otherwise (and always with the even re-partition, whose rows change) the rows are read from L2 and more blocks
  // fit an SM
  const int64_t slots = (mode == 3 ? 2 : 1) * (int64_t)kTile * 36 * (int64_t)wsize(s);
  const int rows_sm =
      (mode == 2 || mode == 3) ? (!even && max_rows * (int64_t)sizeof(int4) + slots <= budget) : 1;
  // cuts block row ranges at scene boundaries
  auto cut = [&](const std::vector<int64_t>& bnd, std::vector<int32_t>& row, std::vector<int32_t>& scn,
                 std::vector<int32_t>& blk) {
    int sc = 0;
    for (int b = 0; b < grid; ++b) {
      int64_t r0 = bnd[b], r1 = bnd[b + 1];
      blk[b] = (int32_t)scn.size();
      int64_t r = r0;
      while (r < r1) {
        while (sc < s->n_scenes && s->offsets[sc + 1] <= r) ++sc;
        int64_t e = std::min<int64_t>(r1, s->offsets[sc + 1]);
        row.push_back((int32_t)r);
        scn.push_back(sc);
        r = e;
      }
    }
    blk[grid] = (int32_t)scn.size();
    row.push_back((int32_t)n);
  };
  cut(bounds, seg_row, seg_scene, block_seg);
  std::vector<int64_t> ubounds(grid + 1);
  for (int b = 0; b <= grid; ++b) ubounds[b] = n * b / grid;
  std::vector<int32_t> useg_row, useg_scene, ublock_seg(grid + 1, 0);
  cut(ubounds, useg_row, useg_scene, ublock_seg);
  for (int x = 0, k = 0; x <= s->n_scenes; ++x) {  // first segment of each scene (segments are in row order)
    while (k < (int)seg_scene.size() && seg_scene[k] < x) ++k;
    scene_seg[x] = k;
  }
  void* olds[] = {d.seg_row, d.seg_scene, d.block_seg, d.scene_seg, d.part_s, d.useg_row, d.useg_scene, d.ublock_seg};
  for (void* p : olds) dfree(s, p);
  size_t ns = std::max<size_t>(seg_scene.size(), 1);
  TRY(dalloc_t(s, &d.seg_row, seg_row.size()));
  TRY(dalloc_t(s, &d.seg_scene, ns));
  TRY(dalloc_t(s, &d.block_seg, block_seg.size()));
  TRY(dalloc_t(s, &d.scene_seg, scene_seg.size()));
  // segments' partials, then the few-scene sums (n_seg + scene); or the even re-split's block slots and scene sums
  const size_t part_slots =
      std::max<size_t>(ns + kLocalPcgScenes, even ? (size_t)grid * kEvenPcgSegs + kEvenPcgScenes : 0);
  TRY(dalloc_t(s, &d.part_s, (size_t)kPartials * part_slots));
  CUDA_TRY(s, cudaMemcpy(d.seg_row, seg_row.data(), sizeof(int32_t) * seg_row.size(), cudaMemcpyHostToDevice));
  if (!seg_scene.empty())
    CUDA_TRY(s, cudaMemcpy(d.seg_scene, seg_scene.data(), sizeof(int32_t) * seg_scene.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.block_seg, block_seg.data(), sizeof(int32_t) * block_seg.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.scene_seg, scene_seg.data(), sizeof(int32_t) * scene_seg.size(), cudaMemcpyHostToDevice));
  TRY(dalloc_t(s, &d.useg_row, useg_row.size()));
  TRY(dalloc_t(s, &d.useg_scene, std::max<size_t>(useg_scene.size(), 1)));
  TRY(dalloc_t(s, &d.ublock_seg, ublock_seg.size()));
  CUDA_TRY(s, cudaMemcpy(d.useg_row, useg_row.data(), sizeof(int32_t) * useg_row.size(), cudaMemcpyHostToDevice));
  if (!useg_scene.empty())
    CUDA_TRY(s, cudaMemcpy(d.useg_scene, useg_scene.data(), sizeof(int32_t) * useg_scene.size(),
                           cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.ublock_seg, ublock_seg.data(), sizeof(int32_t) * ublock_seg.size(), cudaMemcpyHostToDevice));
  d.n_seg = (int32_t)seg_scene.size();
  d.pcg_grid = n > 0 ? grid : 0;
  d.pcg_lanes = lanes;
  d.pcg_max_rows = (int32_t)std::max<int64_t>(max_rows, 1);
  d.pcg_max_entries = (int32_t)std::max<int64_t>(max_ent, 1);
  d.pcg_mode = mode;
  d.pcg_rows_sm = rows_sm;
  d.pcg_part_slots = (int32_t)part_slots;
  d.pcg_even = even;
  d.pcg_even_off = 0;
  if (even) d.pcg_even_off = (int32_t)((pcg_smem_bytes_for(mode, d.mixed, 0, 1, 0) + 15) & ~size_t(15));
  // many scenes: each block decides its own scenes when every block's rows (product and update partitions) span at
  // most kDistPcgScenes scenes
  {
    int dist = s->n_scenes > kLocalPcgScenes && !even;
    for (int b = 0; b < grid && dist; ++b) {
      int lo = 0x7fffffff, hi = -1;
      if (block_seg[b + 1] > block_seg[b]) {
        lo = std::min(lo, seg_scene[block_seg[b]]);
        hi = std::max(hi, seg_scene[block_seg[b + 1] - 1]);
      }
      if (ublock_seg[b + 1] > ublock_seg[b]) {
        lo = std::min(lo, useg_scene[ublock_seg[b]]);
        hi = std::max(hi, useg_scene[ublock_seg[b + 1] - 1]);
      }
      if (hi >= 0 && hi - lo + 1 > kDistPcgScenes) dist = 0;
    }
    d.pcg_dist = dist;
  }
  // the fused PCG's halo rows and local neighbour slots (the incidence of the bonds in the device's entry order)
  {
    void* holds[] = {d.halo_start, d.halo_rows, d.inc2_loc};
    for (void* p : holds) dfree(s, p);
    d.halo_start = d.halo_rows = nullptr;
    d.inc2_loc = nullptr;
    d.pcg_max_zslots = 0;
  }
  if (mode == 4) {
    const int64_t nb = s->nb;
    std::vector<int32_t> ist(n + 1, 0);
    for (int64_t k = 0; k < nb; ++k) {
      ist[s->bi[k] + 1]++;
      ist[s->bj[k] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) ist[i + 1] += ist[i];
    std::vector<int2> inc(std::max<int64_t>(2 * nb, 1));
    {
      std::vector<int32_t> fill(ist.begin(), ist.end() - 1);
      for (int64_t k = 0; k < nb; ++k) {
        inc[fill[s->bi[k]]++] = make_int2((int32_t)(k << 1), s->bj[k]);
        inc[fill[s->bj[k]]++] = make_int2((int32_t)((k << 1) | 1), s->bi[k]);
      }
    }
    std::vector<int32_t> hstart(grid + 1, 0), hrows, halo;
    int64_t max_slots = 2;
    for (int b = 0; b < grid; ++b) {
      const int64_t r0 = bounds[b], r1 = bounds[b + 1];
      hstart[b] = (int32_t)hrows.size();
      halo.clear();
      for (int64_t e = ist[r0]; e < ist[r1]; ++e)
        if (inc[e].y < r0 || inc[e].y >= r1) halo.push_back(inc[e].y);
      std::sort(halo.begin(), halo.end());
      halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
      for (int64_t e = ist[r0]; e < ist[r1]; ++e) {
        int32_t o = inc[e].y;
        int64_t slot = (o >= r0 && o < r1) ? o - r0
                                           : (r1 - r0) + (std::lower_bound(halo.begin(), halo.end(), o) - halo.begin());
        inc[e].y = (int32_t)slot;
      }
      hrows.insert(hrows.end(), halo.begin(), halo.end());
      max_slots = std::max<int64_t>(max_slots, (r1 - r0) + (int64_t)halo.size());
    }
    hstart[grid] = (int32_t)hrows.size();
    TRY(dalloc_t(s, &d.halo_start, (size_t)grid + 1));
    TRY(dalloc_t(s, &d.halo_rows, std::max<size_t>(hrows.size(), 1)));
    TRY(dalloc_t(s, &d.inc2_loc, inc.size()));
    CUDA_TRY(s, cudaMemcpy(d.halo_start, hstart.data(), sizeof(int32_t) * hstart.size(), cudaMemcpyHostToDevice));
    if (!hrows.empty())
      CUDA_TRY(s, cudaMemcpy(d.halo_rows, hrows.data(), sizeof(int32_t) * hrows.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(s, cudaMemcpy(d.inc2_loc, inc.data(), sizeof(int2) * inc.size(), cudaMemcpyHostToDevice));
    d.pcg_max_zslots = (int32_t)((max_slots + 1) & ~int64_t(1));  // even: the bond-block slots start 16-byte aligned
  }
  return BDEM_OK;
}

// default PCG launch shape: 4 lanes per row, every co-resident block, at least 64 rows per block
// co-resident PCG blocks as the registers allow (the partition's shared memory is checked in apply_pcg_shape)
static int pcg_blocks_by_regs(const bdem_sim* s, int lanes) {
  int mode = pcg_mode_of(s->pcg_product, 1);
  return pcg_max_blocks(s->d.mixed, lanes, pcg_smem_bytes_for(mode, s->d.mixed, 64, 64, 128), mode);
}

// builds the partition for (lanes, grid) and shrinks the grid until every block is co-resident with the partition's
// actual shared-memory need (a cooperative launch requires it)
static bdem_status apply_pcg_shape(bdem_sim* s, int lanes, int grid) {
  for (int tries = 0; tries < 16; ++tries) {
    TRY(build_pcg_segments(s, lanes, grid));
    int mx = pcg_max_blocks(s->d.mixed, lanes, pcg_smem_bytes(s->d), s->d.pcg_mode);
    if (mx < 1) return fail(s, BDEM_E_INVALID, "the PCG blocks' shared memory does not fit an SM at this shape");
    if (s->d.pcg_grid <= mx) return BDEM_OK;
    grid = mx;
  }
  return fail(s, BDEM_E_CUDA, "could not fit the PCG grid on the device");
}

static bdem_status default_pcg_shape(bdem_sim* s) {
  int lanes = 2;
  int mx = pcg_blocks_by_regs(s, lanes);
  if (mx < 1) return fail(s, BDEM_E_CUDA, "no resident blocks for the PCG kernel");
  int grid = (int)std::min<int64_t>(mx, std::max<int64_t>(1, (s->n + 63) / 64));
  s->pcg_blocks = mx;
  return apply_pcg_shape(s, lanes, grid);
}

extern "C" bdem_status bdem_create(const bdem_config* config, int32_t n_scenes, const int64_t* scene_offsets,
                                   const double* pos, const double* quat, const double* vel, const double* quat_vel,
                                   const double* radius, const int32_t* particle_material, const bdem_material* mats,
                                   int32_t n_mats, const uint8_t* kinematic, bdem_sim** out) {
  if (!out) return fail(nullptr, BDEM_E_INVALID, "out is NULL");
  *out = nullptr;
  TRY(check_config(config));
  if (n_scenes < 1 || !scene_offsets) return fail(nullptr, BDEM_E_INVALID, "need n_scenes >= 1 and scene_offsets");
  if (scene_offsets[0] != 0) return fail(nullptr, BDEM_E_INVALID, "scene_offsets[0] must be 0");
  for (int s = 0; s < n_scenes; ++s)
    if (scene_offsets[s + 1] < scene_offsets[s]) return fail(nullptr, BDEM_E_INVALID, "scene_offsets must not decrease");
  int64_t n = scene_offsets[n_scenes];
  if (n < 0 || n > (int64_t)1 << 30) return fail(nullptr, BDEM_E_INVALID, "particle count out of range");
  if (n > 0 && (!pos || !quat || !radius || !particle_material))
    return fail(nullptr, BDEM_E_INVALID, "pos, quat, radius and particle_material are required");
  if (n_mats < 1 || !mats) return fail(nullptr, BDEM_E_INVALID, "need at least one material");
  for (int m = 0; m < n_mats; ++m) {
    const bdem_material& M = mats[m];
    if (!(M.E > 0.0) || !fin(M.E) || !(M.nu > -1.0 && M.nu < 0.5) || !(M.density > 0.0) || !fin(M.density) ||
        !(M.break_strain > 0.0) || !(M.bend_twist_scale >= 0.0) || !fin(M.bend_twist_scale) ||
        !(M.tensile_strength > 0.0) || !(M.shear_strength > 0.0) ||
        !(M.shear_scale >= 0.0) || !fin(M.shear_scale))
      return fail(nullptr, BDEM_E_INVALID, "material %d is invalid", m);
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k)
      if (!fin(pos[3 * i + k]) || (vel && !fin(vel[3 * i + k])))
        return fail(nullptr, BDEM_E_INVALID, "particle %lld: non-finite position or velocity", (long long)i);
    double nq = 0.0;
    for (int k = 0; k < 4; ++k) {
      if (!fin(quat[4 * i + k]) || (quat_vel && !fin(quat_vel[4 * i + k])))
        return fail(nullptr, BDEM_E_INVALID, "particle %lld: non-finite quaternion", (long long)i);
      nq += quat[4 * i + k] * quat[4 * i + k];
    }
    if (std::fabs(std::sqrt(nq) - 1.0) > 1e-6)
      return fail(nullptr, BDEM_E_INVALID, "particle %lld: quaternion is not unit", (long long)i);
    if (!(radius[i] > 0.0) || !fin(radius[i]))
      return fail(nullptr, BDEM_E_INVALID, "particle %lld: radius must be positive", (long long)i);
    if (particle_material[i] < 0 || particle_material[i] >= n_mats)
      return fail(nullptr, BDEM_E_INVALID, "particle %lld: material index out of range", (long long)i);
  }
  bdem_sim* s = new bdem_sim();
  s->cfg = *config;
  if (config->allocator) {
    s->hook = *config->allocator;
    if (!s->hook.alloc != !s->hook.free) {
      delete s;
      return fail(nullptr, BDEM_E_INVALID, "the allocator hook needs both alloc and free");
    }
  }
  s->cfg.allocator = nullptr;  // copied into s->hook
  s->n = (int32_t)n;
  s->n_scenes = n_scenes;
  s->stream = (cudaStream_t)config->cuda_stream;
  s->offsets.assign(scene_offsets, scene_offsets + n_scenes + 1);
  s->mats.assign(mats, mats + n_mats);
  s->pscene.resize(n);
  for (int sc = 0; sc < n_scenes; ++sc)
    for (int64_t i = scene_offsets[sc]; i < scene_offsets[sc + 1]; ++i) s->pscene[i] = sc;
  morton_order(scene_offsets, n_scenes, pos, s->perm);
  s->iperm.resize(n);
  s->deg.assign(n, 0);
  for (int64_t k = 0; k < n; ++k) s->iperm[s->perm[k]] = (int32_t)k;
  s->radius.resize(n);
  s->mass.resize(n);
  s->kin.assign(n, 0);
  for (int64_t k = 0; k < n; ++k) {
    s->radius[k] = radius[s->perm[k]];
    if (kinematic) s->kin[k] = kinematic[s->perm[k]] ? 1 : 0;
  }
  const bdem_config& c = s->cfg;
  DevArrays& d = s->d;
  d.n = (int32_t)n;
  d.nb = 0;
  d.n_scenes = n_scenes;
  d.mixed = c.precision == BDEM_MIXED;
  d.dt = c.dt;
  d.gx = c.gravity[0];
  d.gy = c.gravity[1];
  d.gz = c.gravity[2];
  d.tol = c.newton_rel_tol;
  d.tol_abs = c.newton_abs_tol;
  d.ground_z = c.ground_z;
  d.k_ground = c.k_ground;
  d.k_self = c.k_self;
  d.skin = c.contact_skin;
  d.mu_slide = c.friction_slide;
  d.wait_ns = 2000000000ull;  // 2 s
  d.first_order = c.optimizer == BDEM_OPT_FIRST_ORDER;
  d.midpoint = c.integrator == BDEM_INT_MIDPOINT;
  s->amg.on = c.preconditioner == BDEM_PRECOND_AMG;
  // FP64-residual refinement: the mixed path's second-order solves with the block-Jacobi PCG
  d.refine = (d.mixed && !d.first_order && !s->amg.on) ? c.pcg_refine : 0;
  s->amg.omega = 0.6;
  d.mu_roll = c.friction_roll;
  double rmax = 0.0;
  for (int64_t i = 0; i < n; ++i) rmax = std::max(rmax, radius[i]);
  d.cell_h = std::max(2.0 * rmax + c.contact_skin, 1e-12);
  d.newton_max = c.newton_max_iter;
  d.pcg_max = c.pcg_max_iter;
  d.ls_max = c.ls_max_halvings;
  bdem_status st = alloc_particles(s);
  if (st == BDEM_OK) st = build_particle_tiles(s);
  if (st == BDEM_OK) {
    std::vector<double4> xp(std::max<int64_t>(n, 1)), xq(std::max<int64_t>(n, 1)), vp(std::max<int64_t>(n, 1)),
        vq(std::max<int64_t>(n, 1)), hp(std::max<int64_t>(n, 1));
    std::vector<double2> coef(std::max<int64_t>(n, 1));
    for (int64_t i = 0; i < n; ++i) {  // i internal, u the caller's index
      int64_t u = s->perm[i];
      const bdem_material& M = mats[particle_material[u]];
      double r = radius[u], m = M.density * 4.0 / 3.0 * M_PI * r * r * r;
      s->mass[i] = m;
      double qn = std::sqrt(quat[4 * u] * quat[4 * u] + quat[4 * u + 1] * quat[4 * u + 1] +
                            quat[4 * u + 2] * quat[4 * u + 2] + quat[4 * u + 3] * quat[4 * u + 3]);
      xp[i] = make_double4(pos[3 * u], pos[3 * u + 1], pos[3 * u + 2], r);
      xq[i] = make_double4(quat[4 * u] / qn, quat[4 * u + 1] / qn, quat[4 * u + 2] / qn, quat[4 * u + 3] / qn);
      vp[i] = vel ? make_double4(vel[3 * u], vel[3 * u + 1], vel[3 * u + 2], 0.0) : make_double4(0, 0, 0, 0);
      vq[i] = quat_vel ? make_double4(quat_vel[4 * u], quat_vel[4 * u + 1], quat_vel[4 * u + 2], quat_vel[4 * u + 3])
                       : make_double4(0, 0, 0, 0);
      hp[i] = make_double4(0, 0, 0, m);
      coef[i] = make_double2(m / (c.dt * c.dt), 1.6 * m * r * r / (c.dt * c.dt));
    }
    size_t nn = (size_t)n;
    if (nn) {
      cudaMemcpy(d.x0p, xp.data(), sizeof(double4) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.x0q, xq.data(), sizeof(double4) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.xp, xp.data(), sizeof(double4) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.xq, xq.data(), sizeof(double4) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.vp, vp.data(), sizeof(double4) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.vq, vq.data(), sizeof(double4) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.hp, hp.data(), sizeof(double4) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.coef, coef.data(), sizeof(double2) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.pscene, s->pscene.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.kin, s->kin.data(), nn, cudaMemcpyHostToDevice);
      cudaMemcpy(d.perm, s->perm.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice);
    }
    // no bonds yet: empty incidence lists and an empty bond-tile table (every scene owns zero bond tiles)
    st = BDEM_OK;
    if (dalloc_t(s, &d.inc_start, nn + 1) != BDEM_OK || dalloc_t(s, &d.inc2, 1) != BDEM_OK ||
        dalloc_t(s, &d.btile_start, 1) != BDEM_OK || dalloc_t(s, &d.btile_scene, 1) != BDEM_OK ||
        dalloc_t(s, &d.btile_begin, (size_t)n_scenes + 1) != BDEM_OK ||
        dalloc_t(s, &d.part_b, (size_t)kPartials) != BDEM_OK)
      st = BDEM_E_NOMEM;
    d.n_btiles = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (st == BDEM_OK && e != cudaSuccess) st = fail(s, BDEM_E_CUDA, "upload: %s", cudaGetErrorString(e));
    if (st == BDEM_OK) st = default_pcg_shape(s);
  }
  if (st != BDEM_OK) {
    g_create_err = s->err;
    bdem_destroy(s);
    return st;
  }
  *out = s;
  return BDEM_OK;
}

// ------------------------------------------------------------------------------------------------
// bonds
// ------------------------------------------------------------------------------------------------

// staging sub-arrays of the caller-order state: pos [n][3], quat [n][4], vel [n][3], quat_vel [n][4], each starting
// on a 256-byte boundary
static size_t stage_off(size_t n, int k) {
  const size_t len[4] = {3 * n, 4 * n, 3 * n, 4 * n};
  size_t off = 0;
  for (int i = 0; i < k; ++i) off += (len[i] + 31) & ~(size_t)31;
  return off;
}

static bdem_status download_committed(bdem_sim* s, std::vector<double4>& xp, std::vector<double4>& xq) {
  xp.resize(std::max(s->n, 1));
  xq.resize(std::max(s->n, 1));
  if (s->n == 0) return BDEM_OK;
  CUDA_TRY(s, cudaStreamSynchronize(s->stream));
  CUDA_TRY(s, cudaMemcpy(xp.data(), s->d.x0p, sizeof(double4) * s->n, cudaMemcpyDeviceToHost));
  CUDA_TRY(s, cudaMemcpy(xq.data(), s->d.x0q, sizeof(double4) * s->n, cudaMemcpyDeviceToHost));
  return BDEM_OK;
}

extern "C" bdem_status bdem_add_bonds(bdem_sim* s, int64_t n, const int32_t* I, const int32_t* J, const int32_t* M) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (n < 0) return fail(s, BDEM_E_INVALID, "negative bond count");
  if (n == 0) return BDEM_OK;
  if (!I || !J || !M) return fail(s, BDEM_E_INVALID, "bond arrays are NULL");
  if (s->nb + n > ((int64_t)1 << 29)) return fail(s, BDEM_E_INVALID, "too many bonds");
  std::vector<double4> xp, xq;
  TRY(download_committed(s, xp, xq));
  struct NB { int32_t a, b, m; int64_t old, ext; };
  std::vector<NB> all;
  all.reserve(s->nb + n);
  std::vector<int64_t> old_ext(s->nb);  // stored index -> caller index of the existing bonds
  for (int64_t e = 0; e < s->nb; ++e) old_ext[s->bond_ext2int_h[e]] = e;
  for (int64_t k = 0; k < s->nb; ++k) all.push_back({s->bi[k], s->bj[k], s->bmat[k], k, old_ext[k]});
  for (int64_t k = 0; k < n; ++k) {
    int32_t iu = I[k], ju = J[k], m = M[k];
    if (iu < 0 || ju < 0 || iu >= s->n || ju >= s->n)
      return fail(s, BDEM_E_INVALID, "bond %lld: index out of range", (long long)k);
    if (iu == ju) return fail(s, BDEM_E_INVALID, "bond %lld: i == j", (long long)k);
    int32_t i = s->iperm[iu], j = s->iperm[ju];
    if (s->pscene[i] != s->pscene[j]) return fail(s, BDEM_E_INVALID, "bond %lld joins two scenes", (long long)k);
    if (m < 0 || m >= (int32_t)s->mats.size()) return fail(s, BDEM_E_INVALID, "bond %lld: material out of range", (long long)k);
    double4 qi = xq[i], qj = xq[j];
    double qd = qi.x * qj.x + qi.y * qj.y + qi.z * qj.z + qi.w * qj.w;
    if (!(qd >= 1.0 - 1e-12))
      return fail(s, BDEM_E_INVALID, "bond %lld: endpoint orientations differ (q_i.q_j = %.17g)", (long long)k, qd);
    double dx = xp[j].x - xp[i].x, dy = xp[j].y - xp[i].y, dz = xp[j].z - xp[i].z;
    if (!(dx * dx + dy * dy + dz * dz > 0.0)) return fail(s, BDEM_E_INVALID, "bond %lld: zero length", (long long)k);
    all.push_back({std::min(i, j), std::max(i, j), m, -1 - k, s->nb + k});
  }
  std::sort(all.begin(), all.end(), [](const NB& x, const NB& y) { return x.a != y.a ? x.a < y.a : x.b < y.b; });
  for (size_t k = 1; k < all.size(); ++k)
    if (all[k].a == all[k - 1].a && all[k].b == all[k - 1].b)
      return fail(s, BDEM_E_INVALID, "duplicate bond (%d, %d)", s->perm[all[k].a], s->perm[all[k].b]);
  // broken flags of the existing bonds
  std::vector<uint8_t> old_broken(std::max<int64_t>(s->nb, 1), 0);
  if (s->nb) CUDA_TRY(s, cudaMemcpy(old_broken.data(), s->d.bbroken, s->nb, cudaMemcpyDeviceToHost));
  int64_t nb = (int64_t)all.size();
  std::vector<int2> bij(nb);
  std::vector<double4> rest(nb), stiff(nb);
  std::vector<double> brk(nb);
  std::vector<double4> sgeo(nb);
  std::vector<double2> sstr(nb);
  int stress_on = 0;
  std::vector<uint8_t> broken(nb, 0);
  std::vector<int32_t> bscene(nb), bi(nb), bj(nb), bm(nb), e2i(nb), i2e(nb);
  for (int64_t k = 0; k < nb; ++k) {
    const NB& e = all[k];
    e2i[e.ext] = (int32_t)k;
    i2e[k] = (int32_t)e.ext;
    bij[k] = make_int2(e.a, e.b);
    bi[k] = e.a;
    bj[k] = e.b;
    bm[k] = e.m;
    bscene[k] = s->pscene[e.a];
    const bdem_material& mt = s->mats[e.m];
    brk[k] = mt.break_strain;
    {  // stress criterion: cross-section of the bond (r0 = (r_i + r_j)/2) and strengths
      double r0 = 0.5 * (s->radius[e.a] + s->radius[e.b]);
      double S = M_PI * r0 * r0, Ia = M_PI * r0 * r0 * r0 * r0 / 4.0, Ja = M_PI * r0 * r0 * r0 * r0 / 2.0;
      sgeo[k] = make_double4(1.0 / S, r0 / Ia, r0 / Ja, 0.0);
      sstr[k] = make_double2(mt.tensile_strength, mt.shear_strength);
      if (fin(mt.tensile_strength) || fin(mt.shear_strength)) stress_on = 1;
    }
    if (e.old >= 0) {
      rest[k] = s->rest[e.old];
      stiff[k] = s->stiff[e.old];
      broken[k] = old_broken[e.old];
      continue;
    }
    // rest data from the current state (Sec. 3.2 with the readings of the bond frame)
    double pi[3] = {xp[e.a].x, xp[e.a].y, xp[e.a].z}, pj[3] = {xp[e.b].x, xp[e.b].y, xp[e.b].z};
    double qi[4] = {xq[e.a].x, xq[e.a].y, xq[e.a].z, xq[e.a].w}, qj[4] = {xq[e.b].x, xq[e.b].y, xq[e.b].z, xq[e.b].w};
    double dd[3] = {pj[0] - pi[0], pj[1] - pi[1], pj[2] - pi[2]};
    double l0 = std::sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    double n0[3] = {dd[0] / l0, dd[1] / l0, dd[2] / l0};
    double sg = (qi[0] * qj[0] + qi[1] * qj[1] + qi[2] * qj[2] + qi[3] * qj[3]) < 0.0 ? -1.0 : 1.0;
    double m4[4], mm = 0.0;
    for (int c = 0; c < 4; ++c) {
      m4[c] = qi[c] + sg * qj[c];
      mm += m4[c] * m4[c];
    }
    mm = std::sqrt(mm);
    double qcc[4] = {-m4[0] / mm, -m4[1] / mm, -m4[2] / mm, m4[3] / mm}, d0[3];
    hq_rotate(qcc, n0, d0);
    double r0 = 0.5 * (s->radius[e.a] + s->radius[e.b]);
    double S = M_PI * r0 * r0, Ia = M_PI * r0 * r0 * r0 * r0 / 4.0, Ja = M_PI * r0 * r0 * r0 * r0 / 2.0;
    double G = mt.E / (2.0 * (1.0 + mt.nu));
    rest[k] = make_double4(d0[0], d0[1], d0[2], l0);
    stiff[k] = make_double4(mt.E * S / l0, G * S / l0 * mt.shear_scale * mt.shear_scale,
                            mt.bend_twist_scale * mt.E * Ia / l0, mt.bend_twist_scale * G * Ja / l0);
  }
  // incidence CSR (entries ordered by bond index within each particle)
  std::vector<int32_t> inc_start(s->n + 1, 0);
  std::vector<int2> inc(2 * nb);
  for (int64_t k = 0; k < nb; ++k) {
    inc_start[bi[k] + 1]++;
    inc_start[bj[k] + 1]++;
  }
  for (int i = 0; i < s->n; ++i) inc_start[i + 1] += inc_start[i];
  {
    std::vector<int32_t> fill(inc_start.begin(), inc_start.end() - 1);
    for (int64_t k = 0; k < nb; ++k) {
      inc[fill[bi[k]]++] = make_int2((int32_t)(k << 1), bj[k]);
      inc[fill[bj[k]]++] = make_int2((int32_t)((k << 1) | 1), bi[k]);
    }
  }
  // bond tiles per scene
  std::vector<int32_t> tstart, tscene, tbegin(s->n_scenes + 1, 0);
  {
    int64_t k = 0;
    for (int sc = 0; sc < s->n_scenes; ++sc) {
      tbegin[sc] = (int32_t)tscene.size();
      int64_t a = k;
      while (k < nb && bscene[k] == sc) ++k;
      for (int64_t t = a; t < k; t += kTile) {
        tstart.push_back((int32_t)t);
        tscene.push_back(sc);
      }
    }
    tbegin[s->n_scenes] = (int32_t)tscene.size();
    tstart.push_back((int32_t)nb);
  }
  // replace the device bond arrays
  DevArrays& d = s->d;
  void* olds[] = {d.bij, d.brest, d.bstiff, d.bbrk, d.bsgeo, d.bsstr, d.bbroken, d.bscene, d.bg, d.bM, d.bE, d.inc2, d.inc_start, d.bond_ext2int, d.bond_int2ext, s->flag_stage,
                  d.btile_start, d.btile_scene, d.btile_begin, d.part_b};
  for (void* p : olds) dfree(s, p);
  size_t w = wsize(s);
  TRY(dalloc_t(s, &d.bij, nb));
  TRY(dalloc_t(s, &d.brest, nb));
  TRY(dalloc_t(s, &d.bstiff, nb));
  TRY(dalloc_t(s, &d.bbrk, nb));
  TRY(dalloc_t(s, &d.bsgeo, nb));
  TRY(dalloc_t(s, &d.bsstr, nb));
  TRY(dalloc_t(s, &d.bbroken, nb));
  TRY(dalloc_t(s, &d.bscene, nb));
  TRY(dalloc_t(s, &d.bg, 9 * (size_t)nb));
  TRY(dalloc(s, &d.bM, w * 36 * nb));
  TRY(dalloc(s, &d.bE, w * 12 * nb));
  TRY(dalloc_t(s, &d.inc2, 2 * (size_t)nb));
  TRY(dalloc_t(s, &d.bond_ext2int, nb));
  TRY(dalloc_t(s, &d.bond_int2ext, nb));
  TRY(dalloc_t(s, &s->flag_stage, nb));
  TRY(dalloc_t(s, &d.inc_start, (size_t)s->n + 1));
  TRY(dalloc_t(s, &d.btile_start, tstart.size()));
  TRY(dalloc_t(s, &d.btile_scene, std::max<size_t>(1, tscene.size())));
  TRY(dalloc_t(s, &d.btile_begin, tbegin.size()));
  TRY(dalloc_t(s, &d.part_b, (size_t)kPartials * std::max<size_t>(1, tscene.size())));
  CUDA_TRY(s, cudaMemcpy(d.bij, bij.data(), sizeof(int2) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.brest, rest.data(), sizeof(double4) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.bstiff, stiff.data(), sizeof(double4) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.bbrk, brk.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.bsgeo, sgeo.data(), sizeof(double4) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.bsstr, sstr.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice));
  d.stress_on = stress_on;
  CUDA_TRY(s, cudaMemcpy(d.bbroken, broken.data(), nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.bscene, bscene.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.inc2, inc.data(), sizeof(int2) * 2 * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.bond_ext2int, e2i.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.bond_int2ext, i2e.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.inc_start, inc_start.data(), sizeof(int32_t) * (s->n + 1), cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.btile_start, tstart.data(), sizeof(int32_t) * tstart.size(), cudaMemcpyHostToDevice));
  if (!tscene.empty())
    CUDA_TRY(s, cudaMemcpy(d.btile_scene, tscene.data(), sizeof(int32_t) * tscene.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(s, cudaMemcpy(d.btile_begin, tbegin.data(), sizeof(int32_t) * tbegin.size(), cudaMemcpyHostToDevice));
  d.nb = (int32_t)nb;
  d.n_btiles = (int32_t)tscene.size();
  s->nb = nb;
  for (int64_t k = 0; k < n; ++k) {
    s->ext_i.push_back(std::min(I[k], J[k]));
    s->ext_j.push_back(std::max(I[k], J[k]));
  }
  s->bond_ext2int_h.swap(e2i);
  for (int i = 0; i < s->n; ++i) s->deg[i] = inc_start[i + 1] - inc_start[i];
  s->bi.swap(bi);
  s->bj.swap(bj);
  s->bmat.swap(bm);
  s->rest.swap(rest);
  s->stiff.swap(stiff);
  s->brk.swap(brk);
  s->system_ready = false;
  // the PCG partition weighs rows by their bond counts: rebuild it for the new bonds (same shape)
  return apply_pcg_shape(s, s->d.pcg_lanes, s->d.pcg_grid);
}

// ------------------------------------------------------------------------------------------------
// step
// ------------------------------------------------------------------------------------------------

// clears the device counters after a step that did not complete (a wait that gave up leaves the grid barrier's
// arrival count behind)
static void reset_counters(bdem_sim* s, unsigned sync_gen) {
  Counters z{};
  z.sync_gen = sync_gen;
  cudaMemcpy(s->d.cnt, &z, sizeof z, cudaMemcpyHostToDevice);
}

static bdem_status read_counters(bdem_sim* s, Counters* c) {
  CUDA_TRY(s, cudaMemcpyAsync(c, s->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
  TRY(sync(s));
  if (c->timeout) {
    reset_counters(s, c->sync_gen);
    return fail(s, BDEM_E_TIMEOUT, "a device-side wait gave up; the step was rolled back");
  }
  return BDEM_OK;
}

static bdem_status build_contacts(bdem_sim* s) {
  DevArrays& d = s->d;
  TRY(check_launch(s, launch_contacts(d, 0, s->stream)));
  int32_t total = 0;
  CUDA_TRY(s, cudaMemcpyAsync(&total, d.c_start + d.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  TRY(sync(s));
  if (total < 0) return fail(s, BDEM_E_CUDA, "contact count overflow");
  if (total > d.c_cap) {
    dfree(s, d.c_nbr);
    dfree(s, d.c_anbr);
    dfree(s, d.c_blk);
    d.c_nbr = d.c_anbr = nullptr;
    d.c_blk = nullptr;
    int64_t cap = (int64_t)total + total / 2 + 1024;
    if (cap > ((int64_t)1 << 31) - 1) return fail(s, BDEM_E_NOMEM, "too many contact candidates");
    TRY(dalloc_t(s, &d.c_nbr, (size_t)cap));
    TRY(dalloc_t(s, &d.c_anbr, (size_t)cap));
    TRY(dalloc(s, &d.c_blk, 4 * wsize(s) * (size_t)cap));
    d.c_cap = (int32_t)cap;
  }
  TRY(check_launch(s, launch_contacts(d, 1, s->stream)));
  return BDEM_OK;
}

static bdem_status run_pcg(bdem_sim* s, const DevArrays& d, int rhs_from_g, int mask) {
  cudaError_t e = cudaSuccess;
  int k = launch_pcg(d, rhs_from_g, mask, s->stream, &e);
  s->launches += k;
  if (e != cudaSuccess) return fail(s, BDEM_E_CUDA, "cooperative PCG launch: %s", cudaGetErrorString(e));
  return check_launch(s, 0);
}

// FP64-residual refinement of the Newton solve just computed by run_pcg (mixed path): accumulate the solution in
// FP64, form the true residual, and re-solve for the scenes whose residual is still above the target (host-driven:
// one counter read per round)
static bdem_status run_refine(bdem_sim* s, const DevArrays& d) {
  if (!d.refine) return BDEM_OK;
  cudaStream_t st = s->stream;
  TRY(check_launch(s, launch_refine(d, 1, st)));
  TRY(check_launch(s, launch_scene_reduce(d, RED_REFINE0, 0, st)));
  Counters c{};
  TRY(read_counters(s, &c));
  for (int r = 0; r < d.refine && c.n_active > 0; ++r) {
    TRY(run_pcg(s, d, 0, 1));
    TRY(check_launch(s, launch_refine(d, 0, st)));
    TRY(check_launch(s, launch_scene_reduce(d, RED_REFINE, 0, st)));
    TRY(read_counters(s, &c));
  }
  return BDEM_OK;
}

// ---- aggregation AMG (Sec. 5.3): static patterns from the bond list --------------------------------------------

static void amg_release(bdem_sim* s) {
  for (void* p : s->amg_allocs) dfree(s, p);
  s->amg_allocs.clear();
  double om = s->amg.omega;
  int on = s->amg.on;
  s->amg = AmgDev{};
  s->amg.omega = om;
  s->amg.on = on;
  s->amg_nb = -1;
}

template <typename P>
static bdem_status amg_upload(bdem_sim* s, P** dst, const std::vector<P>& src) {
  TRY(dalloc_t(s, dst, std::max<size_t>(src.size(), 1)));
  s->amg_allocs.push_back(*dst);
  if (!src.empty()) CUDA_TRY(s, cudaMemcpy(*dst, src.data(), sizeof(P) * src.size(), cudaMemcpyHostToDevice));
  return BDEM_OK;
}

static bdem_status amg_zeros(bdem_sim* s, void** dst, size_t bytes) {
  TRY(dalloc(s, dst, bytes));
  s->amg_allocs.push_back(*dst);
  return BDEM_OK;
}

// Level 0: the particles in internal (Z-) order, each scene contiguous. A scene gets level 1 always and level l + 1
// while it has more than kAmgAgg nodes on level l; its nodes on a level are consecutive. Entries of A_1: the diagonal
// of every node and, per bond, (agg i, agg j) with the code b << 1 and (agg j, agg i) with b << 1 | 1; entries of
// A_{l+1}: the parents of each level-l entry. Sorted by (row, column, source), so every coarse entry sums its sources
// in one fixed order.
static bdem_status build_amg(bdem_sim* s) {
  amg_release(s);
  AmgDev& a = s->amg;
  const int S = s->n_scenes;
  const size_t wsz = wsize(s);
  std::vector<std::vector<int64_t>> cnt(1, std::vector<int64_t>(S)), off(1, std::vector<int64_t>(S + 1));
  for (int sc = 0; sc < S; ++sc) {
    cnt[0][sc] = s->offsets[sc + 1] - s->offsets[sc];
    off[0][sc] = s->offsets[sc];
  }
  off[0][S] = s->n;
  std::vector<int64_t> nl_nodes(1, s->n);
  for (int l = 0; l + 1 < kAmgMaxLevels; ++l) {
    std::vector<int64_t> c(S, 0), o(S + 1, 0);
    bool any = false;
    for (int sc = 0; sc < S; ++sc) {
      bool next = l == 0 ? cnt[0][sc] > 0 : cnt[l][sc] > kAmgAgg;
      c[sc] = next ? (cnt[l][sc] + kAmgAgg - 1) / kAmgAgg : 0;
      any = any || next;
    }
    if (!any) break;
    for (int sc = 0; sc < S; ++sc) o[sc + 1] = o[sc] + c[sc];
    cnt.push_back(c);
    off.push_back(o);
    nl_nodes.push_back(o[S]);
  }
  a.nl = (int)cnt.size();
  if (a.nl < 2) return BDEM_OK;
  // per level: children ranges and parents
  std::vector<std::vector<int32_t>> parent(a.nl), cbeg(a.nl), cend(a.nl);
  for (int l = 0; l < a.nl; ++l) parent[l].assign(std::max<int64_t>(nl_nodes[l], 1), -1);
  for (int l = 1; l < a.nl; ++l) {
    cbeg[l].assign(std::max<int64_t>(nl_nodes[l], 1), 0);
    cend[l].assign(std::max<int64_t>(nl_nodes[l], 1), 0);
    for (int sc = 0; sc < S; ++sc)
      for (int64_t k = 0; k < cnt[l][sc]; ++k) {
        int64_t I = off[l][sc] + k;
        int64_t c0 = off[l - 1][sc] + kAmgAgg * k, c1 = std::min(c0 + kAmgAgg, off[l - 1][sc] + cnt[l - 1][sc]);
        cbeg[l][I] = (int32_t)c0;
        cend[l][I] = (int32_t)c1;
        for (int64_t ch = c0; ch < c1; ++ch) parent[l - 1][ch] = (int32_t)I;
      }
  }
  // patterns
  struct Ent { int32_t r, c, src; };
  std::vector<Ent> raw;
  raw.reserve(nl_nodes[1] + 2 * s->bi.size());
  for (int64_t I = 0; I < nl_nodes[1]; ++I) raw.push_back({(int32_t)I, (int32_t)I, -1});
  for (size_t b = 0; b < s->bi.size(); ++b) {
    int32_t I = parent[0][s->bi[b]], J = parent[0][s->bj[b]];
    raw.push_back({I, J, (int32_t)(b << 1)});
    raw.push_back({J, I, (int32_t)(b << 1 | 1)});
  }
  std::vector<int32_t> prev_row, prev_col;  // entries of the level below (l >= 2 sources)
  for (int l = 1; l < a.nl; ++l) {
    if (l >= 2) {
      raw.clear();
      for (size_t e = 0; e < prev_row.size(); ++e) {
        int32_t I = parent[l - 1][prev_row[e]], J = parent[l - 1][prev_col[e]];
        if (I >= 0 && J >= 0) raw.push_back({I, J, (int32_t)e});
      }
    }
    std::sort(raw.begin(), raw.end(), [](const Ent& x, const Ent& y) {
      return x.r != y.r ? x.r < y.r : (x.c != y.c ? x.c < y.c : x.src < y.src);
    });
    std::vector<int32_t> rs(nl_nodes[l] + 1, 0), col, erow, gs(1, 0), gsrc, diag(std::max<int64_t>(nl_nodes[l], 1), -1);
    for (size_t k = 0; k < raw.size(); ++k) {
      bool fresh = k == 0 || raw[k].r != raw[k - 1].r || raw[k].c != raw[k - 1].c;
      if (fresh) {
        if (k) gs.push_back((int32_t)gsrc.size());
        col.push_back(raw[k].c);
        erow.push_back(raw[k].r);
        rs[raw[k].r + 1] += 1;
        if (raw[k].r == raw[k].c) diag[raw[k].r] = (int32_t)col.size() - 1;
      }
      if (raw[k].src >= 0) gsrc.push_back(raw[k].src);
    }
    gs.push_back((int32_t)gsrc.size());
    for (int64_t I = 0; I < nl_nodes[l]; ++I) rs[I + 1] += rs[I];
    AmgLevel& L = a.L[l];
    L.n = (int32_t)nl_nodes[l];
    L.nnz = (int32_t)col.size();
    TRY(amg_upload(s, &L.cbeg, cbeg[l]));
    TRY(amg_upload(s, &L.cend, cend[l]));
    TRY(amg_upload(s, &L.parent, parent[l]));
    TRY(amg_upload(s, &L.rs, rs));
    TRY(amg_upload(s, &L.col, col));
    TRY(amg_upload(s, &L.erow, erow));
    TRY(amg_upload(s, &L.diag, diag));
    TRY(amg_upload(s, &L.gs, gs));
    TRY(amg_upload(s, &L.gsrc, gsrc));
    TRY(amg_zeros(s, &L.val, 36 * wsz * std::max<size_t>(col.size(), 1)));
    TRY(amg_zeros(s, &L.dinv, 36 * wsz * std::max<int64_t>(L.n, 1)));
    void* cen = nullptr;
    TRY(amg_zeros(s, &cen, 3 * sizeof(double) * std::max<int64_t>(L.n, 1)));
    L.cen = reinterpret_cast<double*>(cen);
    TRY(amg_zeros(s, &L.r, 6 * wsz * std::max<int64_t>(L.n, 1)));
    TRY(amg_zeros(s, &L.x, 6 * wsz * std::max<int64_t>(L.n, 1)));
    TRY(amg_zeros(s, &L.t, 6 * wsz * std::max<int64_t>(L.n, 1)));
    prev_row = erow;
    prev_col = col;
  }
  a.L[0].n = s->n;
  TRY(amg_upload(s, &a.L[0].parent, parent[0]));
  TRY(amg_zeros(s, &a.p0, 12 * wsz * std::max<int32_t>(s->n, 1)));
  TRY(amg_zeros(s, &a.L[0].t, 6 * wsz * std::max<int32_t>(s->n, 1)));
  std::vector<int32_t> lev(S, 0), o(S, 0), m(S, 0);
  for (int sc = 0; sc < S; ++sc)
    for (int l = 1; l < a.nl; ++l)
      if (cnt[l][sc] > 0) {
        lev[sc] = l;
        o[sc] = (int32_t)off[l][sc];
        m[sc] = (int32_t)cnt[l][sc];
      }
  TRY(amg_upload(s, &a.sc_level, lev));
  TRY(amg_upload(s, &a.sc_off, o));
  TRY(amg_upload(s, &a.sc_m, m));
  void* ch = nullptr;
  TRY(amg_zeros(s, &ch, sizeof(double) * kAmgDense * kAmgDense * std::max(S, 1)));
  a.chol = reinterpret_cast<double*>(ch);
  s->amg_nb = s->nb;
  return BDEM_OK;
}

static cudaError_t capture_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body);

// captures one AMG-PCG iteration (q = H p and alpha, the update with the stop test, the cycle, the new direction) on
// stream st into `body`, closed by the kernel that sets the loop's condition h; returns the kernels per trip
static int capture_amg_body(bdem_sim* s, const DevArrays& d, cudaGraph_t body, cudaGraphConditionalHandle h,
                            cudaStream_t st, cudaError_t* err) {
  *err = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (*err != cudaSuccess) return 0;
  int k = launch_amg_iteration_begin(d, st);
  k += launch_amg_pcg_stage(d, s->amg, 2, st);
  k += launch_amg_pcg_stage(d, s->amg, 3, st);
  k += launch_amg_cycle(d, s->amg, s->n_scenes, st);
  k += launch_amg_pcg_stage(d, s->amg, 4, st);
  k += launch_amg_loop_cond(d, (unsigned long long)h, st);
  cudaError_t e1 = cudaGetLastError();
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &out);
  *err = e1 != cudaSuccess ? e1 : e2;
  return k;
}

// PCG with the AMG cycle as preconditioner on the assembled Newton system. from_g: b = -g; else b is read from vr
// (inspection calls). The solution is left in vx. The iterations run as one graph launch whose conditional while node
// is decided on the device (every scene's stop test, at most pcg_max + 1 trips), so the host neither reads nor waits
// between iterations; if that graph cannot be captured the same kernels run from a host loop that reads the count of
// scenes still iterating after each iteration.
static bdem_status run_amg_pcg(bdem_sim* s, const DevArrays& d, int from_g) {
  if (s->amg_nb != s->nb) TRY(build_amg(s));
  AmgDev& a = s->amg;
  cudaStream_t st = s->stream;
  if (a.nl < 2 || d.n == 0) return BDEM_OK;
  TRY(check_launch(s, launch_amg_setup(d, a, s->n_scenes, st)));
  TRY(check_launch(s, launch_amg_pcg_stage(d, a, from_g ? 0 : 6, st)));
  TRY(check_launch(s, launch_amg_cycle(d, a, s->n_scenes, st)));
  TRY(check_launch(s, launch_amg_pcg_stage(d, a, 1, st)));
  if (!s->amg_exec || memcmp(&s->amg_gd, &d, sizeof(DevArrays)) != 0 || memcmp(&s->amg_ga, &a, sizeof(AmgDev)) != 0) {
    if (s->amg_exec) cudaGraphExecDestroy(s->amg_exec);
    s->amg_exec = nullptr;
    if (!s->amg_cap && cudaStreamCreateWithFlags(&s->amg_cap, cudaStreamNonBlocking) != cudaSuccess) s->amg_cap = nullptr;
    cudaGraph_t g = nullptr, body = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaError_t e = s->amg_cap ? cudaGraphCreate(&g, 0) : cudaErrorNotReady;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s->amg_cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      launch_amg_loop_init(d, (unsigned long long)h, s->amg_cap);
      cudaError_t e1 = cudaGetLastError();
      if (e1 == cudaSuccess) e1 = capture_while(s->amg_cap, h, &body);
      cudaGraph_t out = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(s->amg_cap, &out);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    int k = 0;
    if (e == cudaSuccess) k = capture_amg_body(s, d, body, h, s->amg_cap, &e);
    if (e == cudaSuccess && cudaGraphInstantiate(&s->amg_exec, g, 0) == cudaSuccess) {
      s->amg_gd = d;
      s->amg_ga = a;
      s->amg_gk = k;
    } else {
      s->amg_exec = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
  }
  if (s->amg_exec) {
    CUDA_TRY(s, cudaGraphLaunch(s->amg_exec, st));
    s->launches += 1;  // the loop's kernels are counted from the device's trip count (amg_trip_launches)
    return BDEM_OK;
  }
  for (int it = 0; it <= d.pcg_max; ++it) {
    CUDA_TRY(s, cudaMemsetAsync(&d.cnt->n_active, 0, sizeof(int32_t), st));
    TRY(check_launch(s, launch_amg_pcg_stage(d, a, 2, st)));  // q = H p, then alpha
    TRY(check_launch(s, launch_amg_pcg_stage(d, a, 3, st)));
    TRY(check_launch(s, launch_amg_cycle(d, a, s->n_scenes, st)));
    TRY(check_launch(s, launch_amg_pcg_stage(d, a, 4, st)));
    int32_t act = 0;
    CUDA_TRY(s, cudaMemcpyAsync(&act, &d.cnt->n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(sync(s));
    if (act == 0) break;
  }
  return BDEM_OK;
}

// one time step; on success ctl holds the per-scene control blocks of the step
static bdem_status do_step(bdem_sim* s, std::vector<SceneCtl>& ctl) {
  DevArrays& d = s->d;
  cudaStream_t st = s->stream;
  phase_begin(s, BDEM_PH_PREDICT);
  TRY(check_launch(s, launch_predict(d, st)));
  phase_end(s);
  phase_begin(s, BDEM_PH_CONTACT);
  if (d.k_self > 0.0 && d.n > 0) {
    TRY(build_contacts(s));
  } else if (d.n > 0) {
    CUDA_TRY(s, cudaMemsetAsync(d.c_start, 0, sizeof(int32_t) * (d.n + 1), st));
  }
  TRY(check_launch(s, launch_scene_reduce(d, RED_CAND, 0, st)));
  TRY(check_launch(s, launch_zhat(d, st)));
  phase_end(s);
  Counters c{};
  for (int k = 0;; ++k) {
    phase_begin(s, BDEM_PH_GRAD);
    TRY(check_launch(s, launch_bond_grad(d, 0, st)));
    TRY(check_launch(s, launch_particle_grad(d, 1, 0, st)));
    TRY(check_launch(s, launch_scene_reduce(d, RED_GRAD, 0, st)));
    phase_end(s);
    TRY(read_counters(s, &c));
    if (c.nonfinite) {
      reset_counters(s, c.sync_gen);
      return fail(s, BDEM_E_NONFINITE, "the Newton residual became non-finite; the step was rolled back");
    }
    if (c.n_active == 0) break;
    if (k > d.newton_max + 1) return fail(s, BDEM_E_CUDA, "Newton loop did not terminate");
    if (!d.first_order) {
      phase_begin(s, BDEM_PH_HESS);
      TRY(check_launch(s, launch_bond_hess(d, 0, st)));
      TRY(check_launch(s, launch_particle_hess(d, 1, 0, st)));
      phase_end(s);
      phase_begin(s, BDEM_PH_PCG);
      if (s->amg.on) {
        TRY(run_amg_pcg(s, d, 1));
      } else {
        TRY(run_pcg(s, d, 1, 1));
        TRY(run_refine(s, d));
      }
      phase_end(s);
    }
    phase_begin(s, BDEM_PH_LINESEARCH);
    if (!d.first_order) TRY(check_launch(s, launch_gdx(d, st)));
    TRY(check_launch(s, launch_scene_reduce(d, RED_GDX, 0, st)));
    for (int h = 0; h <= d.ls_max + 1; ++h) {
      TRY(check_launch(s, launch_ls_trial(d, st)));
      TRY(check_launch(s, launch_ls_energy(d, st)));
      TRY(check_launch(s, launch_scene_reduce(d, RED_LS, 0, st)));
      phase_end(s);
      TRY(read_counters(s, &c));
      if (c.n_pending == 0) break;
      phase_begin(s, BDEM_PH_LINESEARCH);
    }
    phase_begin(s, BDEM_PH_LINESEARCH);
    TRY(check_launch(s, launch_ls_commit(d, st)));
    phase_end(s);
  }
  if (s->amg.on && s->amg_exec) s->launches += (int64_t)c.loops_amg * s->amg_gk;  // trips of the device-driven loop
  phase_begin(s, BDEM_PH_FINISH);
  TRY(check_launch(s, launch_finish(d, st)));
  phase_end(s);
  ctl.resize(s->n_scenes);
  CUDA_TRY(s, cudaMemcpyAsync(ctl.data(), d.sc, sizeof(SceneCtl) * s->n_scenes, cudaMemcpyDeviceToHost, st));
  TRY(sync(s));
  if (s->prof_on) {
    s->prof.steps += 1;
    for (int sc = 0; sc < s->n_scenes; ++sc) {
      s->prof.pcg_iters += ctl[sc].pcg_total;
      s->prof.newton_iters += ctl[sc].newton_iters;
      s->prof.particle_newton_iters += (int64_t)ctl[sc].newton_iters * (s->offsets[sc + 1] - s->offsets[sc]);
    }
  }
  return BDEM_OK;
}

// ---- the step as one CUDA graph -------------------------------------------------------------------------------
// predict -> contacts (+ capacity guard) -> gradient -> WHILE(Newton active) { Hessian -> PCG -> descent check ->
// WHILE(line search pending) { trial -> energy difference -> decision } -> commit -> gradient } -> finish.
// The reductions that close each loop body set the loop's condition on the device (k_scene_reduce), with the same
// decisions and caps as the host-driven loop of do_step, so both run the same kernels on the same data.

static void destroy_step_graph(bdem_sim* s) {
  if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->graph_exec = nullptr;
  s->graph = nullptr;
}

// appends a conditional WHILE node after the capture's current frontier and returns its body graph
static cudaError_t capture_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};  // the remaining members zero-initialised
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, deps, edges, nd, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

static bool build_step_graph(bdem_sim* s) {
  destroy_step_graph(s);
  const DevArrays& d = s->d;
  for (auto& c : s->cap)
    if (!c && cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) {
      s->graph_err = "cudaStreamCreateWithFlags failed";
      return false;
    }
  cudaGraph_t G = nullptr, bodyN = nullptr, bodyL = nullptr, bodyR = nullptr, bodyA = nullptr;
  cudaGraphConditionalHandle hN = 0, hL = 0, hR = 0, hA = 0;
  cudaError_t e = cudaSuccess, pe = cudaSuccess, pe2 = cudaSuccess;
  int pre = 0, body = 0, ls = 0, post = 0, ref = 0, amgk = 0;
  const bool amg = s->amg.on && !d.first_order;
  const char* where = "";
#define G_TRY(what, call)        \
  do {                           \
    if (e == cudaSuccess) {      \
      e = (call);                \
      if (e != cudaSuccess) where = what; \
    }                            \
  } while (0)
  G_TRY("cudaGraphCreate", cudaGraphCreate(&G, 0));
  G_TRY("cudaGraphConditionalHandleCreate", cudaGraphConditionalHandleCreate(&hN, G, 0, cudaGraphCondAssignDefault));
  // top level
  G_TRY("begin capture", cudaStreamBeginCaptureToGraph(s->cap[0], G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  if (e == cudaSuccess) {
    cudaStream_t st = s->cap[0];
    pre += launch_predict(d, st);
    if (d.k_self > 0.0) {
      pre += launch_contacts(d, 0, st);
      pre += launch_contacts(d, 1, st);
      pre += launch_contacts(d, 2, st);
    } else {
      cudaMemsetAsync(d.c_start, 0, sizeof(int32_t) * (d.n + 1), st);
    }
    pre += launch_scene_reduce(d, RED_CAND, 0, st);
    pre += launch_zhat(d, st);
    pre += launch_bond_grad(d, 0, st);
    pre += launch_particle_grad(d, 1, 0, st);
    pre += launch_scene_reduce(d, RED_GRAD, hN, st);
    G_TRY("top-level launches", cudaGetLastError());
    G_TRY("Newton while node", capture_while(st, hN, &bodyN));
    post += launch_finish(d, st);
    G_TRY("finish launches", cudaGetLastError());
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &out);
    if (e == cudaSuccess && e2 != cudaSuccess) { e = e2; where = "end capture"; }
  }
  G_TRY("line-search handle", cudaGraphConditionalHandleCreate(&hL, bodyN, 0, 0));
  if (d.refine) G_TRY("refinement handle", cudaGraphConditionalHandleCreate(&hR, bodyN, 0, 0));
  if (amg) G_TRY("AMG loop handle", cudaGraphConditionalHandleCreate(&hA, bodyN, 0, 0));
  // Newton body
  G_TRY("begin body capture", cudaStreamBeginCaptureToGraph(s->cap[1], bodyN, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  if (e == cudaSuccess) {
    cudaStream_t st = s->cap[1];
    if (amg) {  // the AMG-preconditioned solve: setup, first residual and cycle, WHILE(a scene iterates) { iteration }
      body += launch_bond_hess(d, 0, st);
      body += launch_particle_hess(d, 1, 0, st);
      body += launch_amg_setup(d, s->amg, s->n_scenes, st);
      body += launch_amg_pcg_stage(d, s->amg, 0, st);
      body += launch_amg_cycle(d, s->amg, s->n_scenes, st);
      body += launch_amg_pcg_stage(d, s->amg, 1, st);
      body += launch_amg_loop_init(d, (unsigned long long)hA, st);
      G_TRY("AMG launches", cudaGetLastError());
      G_TRY("AMG while node", capture_while(st, hA, &bodyA));
      body += launch_gdx(d, st);
    } else if (!d.first_order) {
      body += launch_bond_hess(d, 0, st);
      body += launch_particle_hess(d, 1, 0, st);
      body += launch_pcg(d, 1, 1, st, &pe);
      if (d.refine) {  // WHILE(a scene's true residual is above its target) { PCG on the residual, refine }
        body += launch_refine(d, 1, st);
        body += launch_scene_reduce(d, RED_REFINE0, hR, st);
        G_TRY("PCG launch", pe);
        G_TRY("refinement launches", cudaGetLastError());
        G_TRY("refinement while node", capture_while(st, hR, &bodyR));
      }
      body += launch_gdx(d, st);
    }
    body += launch_scene_reduce(d, RED_GDX, hL, st);
    G_TRY("PCG launch", pe);
    G_TRY("Newton body launches", cudaGetLastError());
    G_TRY("line-search while node", capture_while(st, hL, &bodyL));
    body += launch_ls_commit(d, st);
    body += launch_bond_grad(d, 0, st);
    body += launch_particle_grad(d, 1, 0, st);
    body += launch_scene_reduce(d, RED_GRAD, hN, st);
    G_TRY("Newton body launches", cudaGetLastError());
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &out);
    if (e == cudaSuccess && e2 != cudaSuccess) { e = e2; where = "end body capture"; }
  }
  // line-search body
  G_TRY("begin line-search capture", cudaStreamBeginCaptureToGraph(s->cap[2], bodyL, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  if (e == cudaSuccess) {
    cudaStream_t st = s->cap[2];
    ls += launch_ls_trial(d, st);
    ls += launch_ls_energy(d, st);
    ls += launch_scene_reduce(d, RED_LS, hL, st);
    G_TRY("line-search launches", cudaGetLastError());
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &out);
    if (e == cudaSuccess && e2 != cudaSuccess) { e = e2; where = "end line-search capture"; }
  }
  // refinement body
  if (d.refine && !d.first_order) {
    G_TRY("begin refinement capture",
          cudaStreamBeginCaptureToGraph(s->cap[2], bodyR, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    if (e == cudaSuccess) {
      cudaStream_t st = s->cap[2];
      ref += launch_pcg(d, 0, 1, st, &pe2);
      ref += launch_refine(d, 0, st);
      ref += launch_scene_reduce(d, RED_REFINE, hR, st);
      G_TRY("refinement PCG launch", pe2);
      G_TRY("refinement launches", cudaGetLastError());
      cudaGraph_t out = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(st, &out);
      if (e == cudaSuccess && e2 != cudaSuccess) { e = e2; where = "end refinement capture"; }
    }
  }
  // AMG iteration body
  if (amg && e == cudaSuccess) {
    cudaError_t ea = cudaSuccess;
    amgk = capture_amg_body(s, d, bodyA, hA, s->cap[2], &ea);
    if (ea != cudaSuccess) { e = ea; where = "AMG iteration capture"; }
  }
  G_TRY("cudaGraphInstantiate", cudaGraphInstantiate(&s->graph_exec, G, 0));
#undef G_TRY
  s->graph = G;
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_step_graph(s);
    s->graph_err = std::string(where) + ": " + cudaGetErrorString(e);
    return false;
  }
  s->graph_d = d;
  s->g_pre = pre;
  s->g_body = body;
  s->g_ls = ls;
  s->g_post = post;
  s->g_ref = ref;
  s->g_amg = amgk;
  s->graph_amg = s->amg;
  return true;
}

// one step through the graph; *redo when the contact arrays were too small (the step was not committed)
static bdem_status graph_step(bdem_sim* s, std::vector<SceneCtl>& ctl, bool* redo) {
  *redo = false;
  DevArrays& d = s->d;
  CUDA_TRY(s, cudaGraphLaunch(s->graph_exec, s->stream));
  Counters c{};
  ctl.resize(s->n_scenes);
  CUDA_TRY(s, cudaMemcpyAsync(&c, d.cnt, sizeof c, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(s, cudaMemcpyAsync(ctl.data(), d.sc, sizeof(SceneCtl) * s->n_scenes, cudaMemcpyDeviceToHost, s->stream));
  TRY(sync(s));
  s->launches += s->g_pre + (int64_t)std::max(0, c.loops_newton - 1) * s->g_body + (int64_t)c.ls_total * s->g_ls +
                 (int64_t)c.loops_refine * s->g_ref + (int64_t)c.loops_amg * s->g_amg + s->g_post;
  if (c.timeout || c.nonfinite || c.overflow || c.runaway) {
    reset_counters(s, c.sync_gen);
    if (c.timeout) return fail(s, BDEM_E_TIMEOUT, "a device-side wait gave up; the step was rolled back");
    if (c.nonfinite)
      return fail(s, BDEM_E_NONFINITE, "the Newton residual became non-finite; the step was rolled back");
    if (c.runaway) return fail(s, BDEM_E_CUDA, "Newton loop did not terminate");
    *redo = true;  // contact arrays too small: the host-driven step grows them
    return BDEM_OK;
  }
  s->graph_steps += 1;
  return BDEM_OK;
}

static bool graph_usable(bdem_sim* s) {
  if (!s->graph_enabled || s->graph_failed || s->prof_on || s->d.n == 0 || !s->contacts_sized) return false;
  if (s->amg.on && s->amg_nb != s->nb) return false;  // the host-driven step builds the AMG hierarchy first
  if (s->graph_exec && memcmp(&s->graph_d, &s->d, sizeof(DevArrays)) == 0 &&
      (!s->amg.on || memcmp(&s->graph_amg, &s->amg, sizeof(AmgDev)) == 0))
    return true;
  if (build_step_graph(s)) return true;
  s->graph_failed = true;
  return false;
}

extern "C" bdem_status bdem_step(bdem_sim* s, int32_t n_steps, bdem_step_stats* stats) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (n_steps < 0) return fail(s, BDEM_E_INVALID, "n_steps must be >= 0");
  if (stats) memset(stats, 0, sizeof(bdem_step_stats) * s->n_scenes);
  s->system_ready = false;
  int worst = BDEM_OK;
  std::vector<SceneCtl> ctl;
  for (int t = 0; t < n_steps; ++t) {
    bool redo = true;
    if (graph_usable(s)) {
      bdem_status st = graph_step(s, ctl, &redo);
      if (st != BDEM_OK) return st;
    }
    if (redo) {
      bdem_status st = do_step(s, ctl);
      if (st != BDEM_OK) return st;
      s->contacts_sized = true;
    }
    for (int sc = 0; sc < s->n_scenes; ++sc) {
      const SceneCtl& c = ctl[sc];
      worst = std::max(worst, (int)c.status);
      if (!stats) continue;
      bdem_step_stats& o = stats[sc];
      o.steps += 1;
      o.newton_iters += c.newton_iters;
      o.pcg_iters += c.pcg_total;
      o.ls_halvings += c.ls_halvings;
      o.bonds_broken += c.bonds_broken;
      o.contact_candidates = c.pad2;
      o.status = std::max(o.status, c.status);
      o.g0_norm = c.g0;
      o.g_norm = c.gnorm;
      o.contact_entry_pcg_iters += c.act_pcg;
      o.intact_bonds = c.intact;
      o.lin_rel_residual = c.lin_res;
      o.refine_rounds += c.refine_total;
    }
  }
  if (worst == BDEM_E_NEWTON_MAXITER) fail(s, BDEM_E_NEWTON_MAXITER, "a scene reached newton_max_iter");
  if (worst == BDEM_E_LINESEARCH) fail(s, BDEM_E_LINESEARCH, "a line search found no decrease");
  return (bdem_status)worst;
}

// ------------------------------------------------------------------------------------------------
// state access
// ------------------------------------------------------------------------------------------------

extern "C" bdem_status bdem_read_state(bdem_sim* s, double* pos, double* quat, double* vel, double* quat_vel,
                                       uint8_t* bond_broken) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  DevArrays& d = s->d;
  size_t n = (size_t)s->n;
  cudaStream_t st = s->stream;
  double *sp = s->stage + stage_off(n, 0), *sq = s->stage + stage_off(n, 1), *sv = s->stage + stage_off(n, 2),
         *su = s->stage + stage_off(n, 3);
  if (n && (pos || quat || vel || quat_vel)) {
    TRY(check_launch(s, launch_pack_state(d, pos ? sp : nullptr, quat ? sq : nullptr, vel ? sv : nullptr,
                                          quat_vel ? su : nullptr, st)));
    if (pos) CUDA_TRY(s, cudaMemcpyAsync(pos, sp, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (quat) CUDA_TRY(s, cudaMemcpyAsync(quat, sq, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, st));
    if (vel) CUDA_TRY(s, cudaMemcpyAsync(vel, sv, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (quat_vel) CUDA_TRY(s, cudaMemcpyAsync(quat_vel, su, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, st));
  }
  if (bond_broken && s->nb) {
    TRY(check_launch(s, launch_bond_flags(d, s->flag_stage, 0, st)));
    CUDA_TRY(s, cudaMemcpyAsync(bond_broken, s->flag_stage, s->nb, cudaMemcpyDeviceToHost, st));
  }
  return sync(s);
}

extern "C" bdem_status bdem_write_state(bdem_sim* s, const double* pos, const double* quat, const double* vel,
                                        const double* quat_vel, const uint8_t* bond_broken) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  size_t n = (size_t)s->n;
  for (size_t i = 0; i < n; ++i) {
    if (pos)
      for (int k = 0; k < 3; ++k)
        if (!fin(pos[3 * i + k])) return fail(s, BDEM_E_INVALID, "particle %zu: non-finite position", i);
    if (vel)
      for (int k = 0; k < 3; ++k)
        if (!fin(vel[3 * i + k])) return fail(s, BDEM_E_INVALID, "particle %zu: non-finite velocity", i);
    if (quat_vel)
      for (int k = 0; k < 4; ++k)
        if (!fin(quat_vel[4 * i + k])) return fail(s, BDEM_E_INVALID, "particle %zu: non-finite quaternion velocity", i);
    if (quat) {
      double nq = 0.0;
      for (int k = 0; k < 4; ++k) nq += quat[4 * i + k] * quat[4 * i + k];
      if (!fin(nq) || std::fabs(std::sqrt(nq) - 1.0) > 1e-6)
        return fail(s, BDEM_E_INVALID, "particle %zu: quaternion is not unit", i);
    }
  }
  DevArrays& d = s->d;
  cudaStream_t st = s->stream;
  double *sp = s->stage + stage_off(n, 0), *sq = s->stage + stage_off(n, 1), *sv = s->stage + stage_off(n, 2),
         *su = s->stage + stage_off(n, 3);
  if (n && (pos || quat || vel || quat_vel)) {
    if (pos) CUDA_TRY(s, cudaMemcpyAsync(sp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    if (quat) CUDA_TRY(s, cudaMemcpyAsync(sq, quat, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, st));
    if (vel) CUDA_TRY(s, cudaMemcpyAsync(sv, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    if (quat_vel) CUDA_TRY(s, cudaMemcpyAsync(su, quat_vel, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, st));
    TRY(check_launch(s, launch_unpack_state(d, pos ? sp : nullptr, quat ? sq : nullptr, vel ? sv : nullptr,
                                            quat_vel ? su : nullptr, st)));
  }
  if (bond_broken && s->nb) {
    CUDA_TRY(s, cudaMemcpyAsync(s->flag_stage, bond_broken, s->nb, cudaMemcpyHostToDevice, st));
    TRY(check_launch(s, launch_bond_flags(d, s->flag_stage, 1, st)));
  }
  s->system_ready = false;
  return sync(s);
}

extern "C" bdem_status bdem_sizes(const bdem_sim* s, int64_t* n_particles, int64_t* n_bonds, int32_t* n_scenes) {
  if (!s) return BDEM_E_INVALID;
  if (n_particles) *n_particles = s->n;
  if (n_bonds) *n_bonds = s->nb;
  if (n_scenes) *n_scenes = s->n_scenes;
  return BDEM_OK;
}

extern "C" bdem_status bdem_bond_order(const bdem_sim* s, int32_t* pairs) {
  if (!s || (!pairs && s->nb)) return BDEM_E_INVALID;
  for (int64_t k = 0; k < s->nb; ++k) {  // the caller's order of addition, caller indices
    pairs[2 * k] = s->ext_i[k];
    pairs[2 * k + 1] = s->ext_j[k];
  }
  return BDEM_OK;
}

extern "C" bdem_status bdem_set_step_graph(bdem_sim* s, int32_t on) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  s->graph_enabled = on != 0;
  s->graph_failed = false;
  s->graph_err.clear();
  if (!s->graph_enabled) destroy_step_graph(s);
  return BDEM_OK;
}

extern "C" int64_t bdem_graph_steps(const bdem_sim* s) { return s ? s->graph_steps : 0; }

extern "C" const char* bdem_graph_error(const bdem_sim* s) { return s ? s->graph_err.c_str() : ""; }

extern "C" void bdem_destroy(bdem_sim* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  phase_collect(s);
  destroy_step_graph(s);
  if (s->amg_exec) cudaGraphExecDestroy(s->amg_exec);
  if (s->amg_cap) cudaStreamDestroy(s->amg_cap);
  for (cudaStream_t c : s->cap)
    if (c) cudaStreamDestroy(c);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->hook.alloc) cudaStreamSynchronize(s->stream);  // the pool may hand the buffers out again at once
  for (void* p : s->allocs) raw_free(s, p);
  s->allocs.clear();
  delete s;
}

extern "C" const char* bdem_last_error(const bdem_sim* s) { return s ? s->err.c_str() : g_create_err.c_str(); }

extern "C" int64_t bdem_launch_count(const bdem_sim* s) { return s ? s->launches : 0; }

// ------------------------------------------------------------------------------------------------
// inspection
// ------------------------------------------------------------------------------------------------

static bdem_status dbg_reserve(bdem_sim* s, size_t count) {
  if (s->dbg_cap >= count) return BDEM_OK;
  dfree(s, s->dbg_buf);
  s->dbg_buf = nullptr;
  s->dbg_cap = 0;
  TRY(dalloc_t(s, &s->dbg_buf, count));
  s->dbg_cap = count;
  return BDEM_OK;
}

extern "C" bdem_status bdem_debug_system(bdem_sim* s, const double* phat, const double* qhat, double* g, double* diag,
                                         double* bond_hess, int64_t* n_candidates) {
  return bdem_debug_system_at(s, nullptr, nullptr, phat, qhat, g, diag, bond_hess, n_candidates);
}

extern "C" bdem_status bdem_debug_system_at(bdem_sim* s, const double* pos, const double* quat, const double* phat,
                                            const double* qhat, double* g, double* diag, double* bond_hess,
                                            int64_t* n_candidates) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (!phat || !qhat) return fail(s, BDEM_E_INVALID, "phat and qhat are required");
  if ((pos == nullptr) != (quat == nullptr)) return fail(s, BDEM_E_INVALID, "pos and quat go together");
  DevArrays& d = s->d;
  cudaStream_t st = s->stream;
  size_t n = (size_t)s->n;
  if (n) {
    double *sp = s->stage + stage_off(n, 0), *sq = s->stage + stage_off(n, 1);
    CUDA_TRY(s, cudaMemcpyAsync(sp, phat, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(s, cudaMemcpyAsync(sq, qhat, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, st));
    TRY(check_launch(s, launch_set_hat(d, sp, sq, st)));
    if (pos) {
      double *sx = s->stage + stage_off(n, 2), *sy = s->stage + stage_off(n, 3);
      CUDA_TRY(s, cudaMemcpyAsync(sx, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
      CUDA_TRY(s, cudaMemcpyAsync(sy, quat, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, st));
      TRY(check_launch(s, launch_set_iterate(d, sx, sy, st)));
    } else {
      CUDA_TRY(s, cudaMemcpyAsync(d.xp, d.x0p, sizeof(double4) * n, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(s, cudaMemcpyAsync(d.xq, d.x0q, sizeof(double4) * n, cudaMemcpyDeviceToDevice, st));
    }
  }
  TRY(check_launch(s, launch_scene_reduce(d, RED_FORCE_ACTIVE, 0, st)));
  if (d.k_self > 0.0 && d.n > 0) TRY(build_contacts(s));
  else if (d.n > 0) CUDA_TRY(s, cudaMemsetAsync(d.c_start, 0, sizeof(int32_t) * (d.n + 1), st));
  TRY(check_launch(s, launch_bond_grad(d, 1, st)));
  TRY(check_launch(s, launch_particle_grad(d, 0, 1, st)));
  TRY(check_launch(s, launch_bond_hess(d, 1, st)));
  TRY(check_launch(s, launch_particle_hess(d, 0, 1, st)));
  if (g && n) {
    TRY(dbg_reserve(s, 6 * n));
    TRY(check_launch(s, launch_convert_perm(d.g, 1, s->dbg_buf, 1, d.perm, 1, (int)n, st)));
    CUDA_TRY(s, cudaMemcpyAsync(g, s->dbg_buf, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st));
    TRY(sync(s));
  }
  if (diag && n) {
    TRY(dbg_reserve(s, 36 * n));
    TRY(check_launch(s, launch_unpack_diag(d, s->dbg_buf, st)));
    CUDA_TRY(s, cudaMemcpyAsync(diag, s->dbg_buf, sizeof(double) * 36 * n, cudaMemcpyDeviceToHost, st));
    TRY(sync(s));
  }
  if (bond_hess && s->nb) {
    TRY(dbg_reserve(s, 144 * (size_t)s->nb));
    TRY(check_launch(s, launch_unpack_bond_hess(d, s->dbg_buf, nullptr, 0, st)));
    CUDA_TRY(s, cudaMemcpyAsync(bond_hess, s->dbg_buf, sizeof(double) * 144 * s->nb, cudaMemcpyDeviceToHost, st));
  }
  if (n_candidates) {
    int32_t c = 0;
    if (n) CUDA_TRY(s, cudaMemcpyAsync(&c, d.c_start + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(sync(s));
    *n_candidates = c / 2;  // directed entries: each pair appears in both lists
  }
  TRY(sync(s));
  s->system_ready = true;
  return BDEM_OK;
}

extern "C" bdem_status bdem_debug_zhat(bdem_sim* s, double* zp, double* zq) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (!zp || !zq) return fail(s, BDEM_E_INVALID, "zp and zq are required");
  DevArrays& d = s->d;
  cudaStream_t st = s->stream;
  size_t n = (size_t)s->n;
  if (n == 0) return BDEM_OK;
  TRY(check_launch(s, launch_predict(d, st)));
  if (d.k_self > 0.0) TRY(build_contacts(s));
  else CUDA_TRY(s, cudaMemsetAsync(d.c_start, 0, sizeof(int32_t) * (d.n + 1), st));
  TRY(check_launch(s, launch_zhat(d, st)));
  // hp, hq (double4) to the caller's order through the staging buffer
  double *sp = s->stage + stage_off(n, 0), *sq = s->stage + stage_off(n, 1);
  TRY(check_launch(s, launch_pack_hat(d, sp, sq, st)));
  CUDA_TRY(s, cudaMemcpyAsync(zp, sp, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(s, cudaMemcpyAsync(zq, sq, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, st));
  s->system_ready = false;
  return sync(s);
}

extern "C" bdem_status bdem_debug_bonds(bdem_sim* s, int64_t count, const int32_t* ids, double* out) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (!s->system_ready) return fail(s, BDEM_E_INVALID, "call bdem_debug_system first");
  if (count < 0 || (count && (!ids || !out))) return fail(s, BDEM_E_INVALID, "bad arguments");
  for (int64_t k = 0; k < count; ++k)
    if (ids[k] < 0 || ids[k] >= s->nb) return fail(s, BDEM_E_INVALID, "bond id %d out of range", ids[k]);
  if (count == 0) return BDEM_OK;
  cudaStream_t st = s->stream;
  size_t need = 144 * (size_t)count + ((size_t)count + 1) / 2 + 1;
  TRY(dbg_reserve(s, need));
  int32_t* dids = reinterpret_cast<int32_t*>(s->dbg_buf + 144 * (size_t)count);
  CUDA_TRY(s, cudaMemcpyAsync(dids, ids, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
  TRY(check_launch(s, launch_unpack_bond_hess(s->d, s->dbg_buf, dids, (int)count, st)));
  CUDA_TRY(s, cudaMemcpyAsync(out, s->dbg_buf, sizeof(double) * 144 * count, cudaMemcpyDeviceToHost, st));
  return sync(s);
}

extern "C" bdem_status bdem_debug_bond_stress(bdem_sim* s, double* out) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (s->nb && !out) return fail(s, BDEM_E_INVALID, "out is NULL");
  if (s->nb == 0) return BDEM_OK;
  cudaStream_t st = s->stream;
  TRY(dbg_reserve(s, 2 * (size_t)s->nb));
  TRY(check_launch(s, launch_bond_stress(s->d, s->dbg_buf, st)));
  CUDA_TRY(s, cudaMemcpyAsync(out, s->dbg_buf, sizeof(double) * 2 * s->nb, cudaMemcpyDeviceToHost, st));
  return sync(s);
}

extern "C" bdem_status bdem_debug_wait_timeout(bdem_sim* s, double limit_ms) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (!(limit_ms >= 0.0) || !(limit_ms <= 10000.0)) return fail(s, BDEM_E_INVALID, "limit_ms must be in [0, 10000]");
  DevArrays d = s->d;
  d.wait_ns = (unsigned long long)(limit_ms * 1e6);
  TRY(check_launch(s, launch_wait_test(d, s->stream)));
  Counters c{};
  return read_counters(s, &c);  // BDEM_E_TIMEOUT once the wait has given up; the counters are reset
}

extern "C" bdem_status bdem_debug_matvec(bdem_sim* s, const double* x, double* y) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (!s->system_ready) return fail(s, BDEM_E_INVALID, "call bdem_debug_system first");
  if (!x || !y) return fail(s, BDEM_E_INVALID, "x and y are required");
  size_t n = (size_t)s->n;
  if (!n) return BDEM_OK;
  DevArrays& d = s->d;
  cudaStream_t st = s->stream;
  TRY(dbg_reserve(s, 18 * n));
  double* xc = s->dbg_buf;           // caller order
  double* xi = s->dbg_buf + 6 * n;   // internal order
  double* yi = s->dbg_buf + 12 * n;
  CUDA_TRY(s, cudaMemcpyAsync(xc, x, sizeof(double) * 6 * n, cudaMemcpyHostToDevice, st));
  TRY(check_launch(s, launch_convert_perm(xc, 1, xi, 1, d.perm, 0, (int)n, st)));
  TRY(check_launch(s, launch_matvec64(d, xi, yi, 0, st)));
  TRY(check_launch(s, launch_convert_perm(yi, 1, xc, 1, d.perm, 1, (int)n, st)));
  CUDA_TRY(s, cudaMemcpyAsync(y, xc, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st));
  return sync(s);
}

extern "C" bdem_status bdem_debug_pcg(bdem_sim* s, const double* b, double eps_r, int32_t max_iter, double* dx,
                                      int32_t* iters) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (!s->system_ready) return fail(s, BDEM_E_INVALID, "call bdem_debug_system first");
  if (!b || !dx || max_iter < 1 || !(eps_r >= 0.0)) return fail(s, BDEM_E_INVALID, "bad PCG arguments");
  size_t n = (size_t)s->n;
  if (!n) return BDEM_OK;
  DevArrays d = s->d;
  d.pcg_max = max_iter;
  cudaStream_t st = s->stream;
  // the solve removes kinematic rows: rebuild the diagonal blocks with them masked
  TRY(check_launch(s, launch_particle_hess(d, 1, 1, st)));
  std::vector<SceneCtl> ctl(s->n_scenes);
  CUDA_TRY(s, cudaMemcpyAsync(ctl.data(), d.sc, sizeof(SceneCtl) * s->n_scenes, cudaMemcpyDeviceToHost, st));
  TRY(sync(s));
  for (auto& c : ctl) {
    c.newton_active = 1;
    c.pcg_skip = 0;
    c.eps_r = eps_r;
  }
  CUDA_TRY(s, cudaMemcpy(d.sc, ctl.data(), sizeof(SceneCtl) * s->n_scenes, cudaMemcpyHostToDevice));
  TRY(dbg_reserve(s, 18 * n));
  CUDA_TRY(s, cudaMemcpyAsync(s->dbg_buf, b, sizeof(double) * 6 * n, cudaMemcpyHostToDevice, st));
  TRY(check_launch(s, launch_convert_perm(s->dbg_buf, 1, d.vr, !d.mixed, d.perm, 0, (int)n, st)));
  if (s->amg.on) {
    CUDA_TRY(s, cudaMemsetAsync(&d.cnt->loops_amg, 0, sizeof(int32_t), st));
    TRY(run_amg_pcg(s, d, 0));
  } else {
    TRY(run_pcg(s, d, 0, 1));
    if (d.refine) {  // the refinement's residual takes the caller's FP64 right-hand side
      d.b64 = s->dbg_buf + 12 * n;
      TRY(check_launch(s, launch_convert_perm(s->dbg_buf, 1, d.b64, 1, d.perm, 0, (int)n, st)));
      TRY(run_refine(s, d));
    }
  }
  Counters c{};
  TRY(read_counters(s, &c));
  if (s->amg.on && s->amg_exec) s->launches += (int64_t)c.loops_amg * s->amg_gk;
  if (d.refine && !s->amg.on)
    TRY(check_launch(s, launch_convert_perm(d.x64, 1, s->dbg_buf + 6 * n, 1, d.perm, 1, (int)n, st)));
  else
    TRY(check_launch(s, launch_convert_perm(d.vx, !d.mixed, s->dbg_buf + 6 * n, 1, d.perm, 1, (int)n, st)));
  CUDA_TRY(s, cudaMemcpyAsync(dx, s->dbg_buf + 6 * n, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(s, cudaMemcpyAsync(ctl.data(), d.sc, sizeof(SceneCtl) * s->n_scenes, cudaMemcpyDeviceToHost, st));
  TRY(sync(s));
  if (iters)
    for (int sc = 0; sc < s->n_scenes; ++sc) iters[sc] = (d.refine && !s->amg.on) ? ctl[sc].pcg_acc : ctl[sc].pcg_iters;
  // restore the unmasked diagonal blocks of the inspected system
  TRY(check_launch(s, launch_particle_hess(s->d, 0, 1, st)));
  return sync(s);
}

extern "C" bdem_status bdem_profile_enable(bdem_sim* s, int32_t on) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  TRY(sync(s));
  s->prof_on = on != 0;
  s->prof = bdem_profile{};
  return BDEM_OK;
}

extern "C" bdem_status bdem_profile_read(bdem_sim* s, bdem_profile* out) {
  if (!s || !out) return fail(s, BDEM_E_INVALID, "NULL argument");
  TRY(sync(s));
  *out = s->prof;
  return BDEM_OK;
}

// ------------------------------------------------------------------------------------------------
// allocation-free PCG solve (scratch in the library's static device array)
// ------------------------------------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" bdem_status bdem_pcg_static(bdem_sim* s, const double* b_dev, double* x_dev, double eps_r,
                                       int32_t max_iter, int32_t* iters) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (!b_dev || !x_dev || max_iter < 1 || !(eps_r >= 0.0)) return fail(s, BDEM_E_INVALID, "bad PCG arguments");
  DevArrays d = s->d;
  size_t n = (size_t)s->n, w = wsize(s);
  // scratch layout: scene control blocks | counters | segment partials | PCG vectors x r z p w s
  constexpr int kVecs = 6;
  size_t off_sc = 0;
  size_t off_cnt = off_sc + align256(sizeof(SceneCtl) * (size_t)std::max(s->n_scenes, 1));
  size_t off_part = off_cnt + align256(sizeof(Counters));
  size_t off_vec = off_part + align256(sizeof(double) * kPartials * (size_t)std::max(d.pcg_part_slots, 1));
  size_t vec_bytes = align256(w * 6 * std::max<size_t>(n, 1));
  size_t need = off_vec + kVecs * vec_bytes;
  if (need > static_pcg_capacity())
    return fail(s, BDEM_E_INVALID,
                "system too large for the static PCG scratch: needs %zu bytes, the array holds %zu bytes "
                "(about %zu particles in this precision)",
                need, static_pcg_capacity(), (size_t)(static_pcg_capacity() / (kVecs * 6 * w + 1)));
  if (!s->system_ready) return fail(s, BDEM_E_INVALID, "call bdem_debug_system first");
  if (n == 0) return BDEM_OK;
  void* base = nullptr;
  cudaError_t e = static_pcg_address(&base);
  if (e != cudaSuccess) return fail(s, BDEM_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  unsigned char* b8 = static_cast<unsigned char*>(base);
  d.sc = reinterpret_cast<SceneCtl*>(b8 + off_sc);
  d.cnt = reinterpret_cast<Counters*>(b8 + off_cnt);
  d.part_s = reinterpret_cast<double*>(b8 + off_part);
  void** vecs[] = {&d.vx, &d.vr, &d.vz, &d.vp_, &d.vq_, &d.vs};
  for (int k = 0; k < kVecs; ++k) *vecs[k] = b8 + off_vec + k * vec_bytes;
  d.pcg_max = max_iter;
  if (d.pcg_mode == 4) d.pcg_mode = 2;  // the fused PCG's second buffers are not in the static array
  cudaStream_t st = s->stream;
  int k = launch_static_pcg_init(d, eps_r, st);
  k += launch_convert_perm(b_dev, 1, d.vr, !d.mixed, d.perm, 0, (int)n, st);
  TRY(check_launch(s, k));
  TRY(run_pcg(s, d, 0, 1));
  TRY(check_launch(s, launch_convert_perm(d.vx, !d.mixed, x_dev, 1, d.perm, 1, (int)n, st)));
  Counters c{};
  CUDA_TRY(s, cudaMemcpyAsync(&c, d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  if (iters)
    for (int sc = 0; sc < s->n_scenes; ++sc)
      CUDA_TRY(s, cudaMemcpyAsync(iters + sc, &d.sc[sc].pcg_iters, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(s, cudaStreamSynchronize(s->stream));
  if (c.timeout) return fail(s, BDEM_E_TIMEOUT, "a device-side wait gave up");
  return BDEM_OK;
}

// ------------------------------------------------------------------------------------------------
// PCG launch shape and its autotuner
// ------------------------------------------------------------------------------------------------

extern "C" bdem_status bdem_set_pcg_shape(bdem_sim* s, int32_t lanes, int32_t blocks) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) return fail(s, BDEM_E_INVALID, "lanes must be 1, 2, 4 or 8");
  if (blocks < 0) return fail(s, BDEM_E_INVALID, "blocks must be >= 0");
  int mx = pcg_blocks_by_regs(s, lanes);
  if (mx < 1) return fail(s, BDEM_E_CUDA, "no resident blocks for the PCG kernel");
  // default: every co-resident block but at least 64 rows per block; an explicit count is honoured up to one row per
  // block (and the co-resident limit)
  int cap = (int)std::min<int64_t>(mx, std::max<int64_t>(1, (s->n + 63) / 64));
  int grid = blocks == 0 ? cap : (int)std::min<int64_t>(std::min(blocks, mx), std::max<int64_t>(1, s->n));
  TRY(sync(s));
  TRY(apply_pcg_shape(s, lanes, grid));
  s->pcg_blocks = mx;
  return BDEM_OK;
}

extern "C" bdem_status bdem_set_pcg_product(bdem_sim* s, int32_t product) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (product < 0 || product > 3) return fail(s, BDEM_E_INVALID, "product must be 0, 1, 2 or 3");
  const int old = s->pcg_product, lanes = s->d.pcg_lanes, grid = s->d.pcg_grid;
  s->pcg_product = product;
  bdem_status st = bdem_set_pcg_shape(s, lanes, grid);
  if (st == BDEM_E_INVALID) {  // this product does not fit the current shape: the previous setting stays
    std::string why = s->err;
    s->pcg_product = old;
    TRY(bdem_set_pcg_shape(s, lanes, grid));
    s->err = why;
  }
  return st;
}

extern "C" bdem_status bdem_get_pcg_shape(const bdem_sim* s, int32_t* lanes, int32_t* blocks, int32_t* product) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (lanes) *lanes = s->d.pcg_lanes;
  if (blocks) *blocks = s->d.pcg_grid;
  if (product) *product = s->d.pcg_mode >= 2 ? s->d.pcg_mode - 1 : 0;
  return BDEM_OK;
}

// assemble the Newton system at the committed state with xhat = x + dt v (the step's prediction)
static bdem_status assemble_at_committed(bdem_sim* s) {
  DevArrays& d = s->d;
  cudaStream_t st = s->stream;
  TRY(check_launch(s, launch_predict(d, st)));
  if (d.k_self > 0.0 && d.n > 0) TRY(build_contacts(s));
  else if (d.n > 0) CUDA_TRY(s, cudaMemsetAsync(d.c_start, 0, sizeof(int32_t) * (d.n + 1), st));
  TRY(check_launch(s, launch_scene_reduce(d, RED_FORCE_ACTIVE, 0, st)));
  TRY(check_launch(s, launch_bond_grad(d, 1, st)));
  TRY(check_launch(s, launch_particle_grad(d, 1, 1, st)));
  TRY(check_launch(s, launch_bond_hess(d, 1, st)));
  TRY(check_launch(s, launch_particle_hess(d, 1, 1, st)));
  return sync(s);
}

extern "C" bdem_status bdem_set_bond_tile(bdem_sim* s, int32_t tile, int32_t capped) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (tile != 64 && tile != 128 && tile != 256) return fail(s, BDEM_E_INVALID, "tile must be 64, 128 or 256");
  if (capped != 0 && capped != 1) return fail(s, BDEM_E_INVALID, "capped must be 0 or 1");
  TRY(sync(s));
  s->d.bond_tile = tile;
  s->d.bond_capped = capped;
  return BDEM_OK;
}

extern "C" bdem_status bdem_autotune_bonds(bdem_sim* s, int32_t reps, int32_t* tile_out, int32_t* capped_out) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (reps < 1) return fail(s, BDEM_E_INVALID, "reps must be >= 1");
  if (s->nb == 0 || s->n == 0) return BDEM_OK;
  TRY(assemble_at_committed(s));
  cudaEvent_t a = ev_get(s), b = ev_get(s);
  float best = 1e30f;
  int best_t = s->d.bond_tile ? s->d.bond_tile : 128, best_c = s->d.bond_capped;
  const int tiles[] = {64, 128, 256};
  const int caps = (s->d.mixed && !s->d.midpoint) ? 2 : 1;  // the capped variant exists for the FP32 first-order form
  for (int capped = 0; capped < caps; ++capped)
    for (int tile : tiles) {
      DevArrays d = s->d;
      d.bond_tile = tile;
      d.bond_capped = capped;
      TRY(check_launch(s, launch_bond_hess(d, 1, s->stream)));  // warm-up
      cudaEventRecord(a, s->stream);
      for (int r = 0; r < reps; ++r) TRY(check_launch(s, launch_bond_hess(d, 1, s->stream)));
      cudaEventRecord(b, s->stream);
      TRY(sync(s));
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) { best = ms; best_t = tile; best_c = capped; }
    }
  s->ev_pool.push_back(a);
  s->ev_pool.push_back(b);
  s->d.bond_tile = best_t;
  s->d.bond_capped = best_c;
  if (tile_out) *tile_out = best_t;
  if (capped_out) *capped_out = best_c;
  return BDEM_OK;
}

extern "C" bdem_status bdem_autotune_pcg(bdem_sim* s, int32_t iters, int32_t* lanes_out, int32_t* blocks_out) {
  if (!s) return fail(nullptr, BDEM_E_INVALID, "sim is NULL");
  if (iters < 1) return fail(s, BDEM_E_INVALID, "iters must be >= 1");
  if (s->n == 0) return BDEM_OK;
  TRY(assemble_at_committed(s));
  cudaEvent_t a = ev_get(s), b = ev_get(s);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float best = 1e30f;
  int best_l = s->d.pcg_lanes, best_g = s->d.pcg_grid, best_p = s->pcg_product;
  const int lanes_c[] = {1, 2, 4, 8};
  for (int product = 3; product >= 0; --product)
  for (int lanes : lanes_c) {
    s->pcg_product = product;
    int mx = pcg_blocks_by_regs(s, lanes);
    if (mx < 1) continue;  // this product's shared memory leaves no resident block
    for (int per = 1; per <= std::max(1, mx / sms); ++per) {
      bdem_status sst = bdem_set_pcg_shape(s, lanes, per * sms);
      if (sst == BDEM_E_INVALID) continue;  // the block row ranges do not fit this shape's shared memory
      if (sst != BDEM_OK) return sst;
      DevArrays d = s->d;
      d.pcg_max = iters;
      float t_min = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        std::vector<SceneCtl> ctl(s->n_scenes);
        CUDA_TRY(s, cudaMemcpy(ctl.data(), d.sc, sizeof(SceneCtl) * s->n_scenes, cudaMemcpyDeviceToHost));
        for (auto& c : ctl) { c.newton_active = 1; c.pcg_skip = 0; c.eps_r = 0.0; }
        CUDA_TRY(s, cudaMemcpy(d.sc, ctl.data(), sizeof(SceneCtl) * s->n_scenes, cudaMemcpyHostToDevice));
        cudaEventRecord(a, s->stream);
        TRY(run_pcg(s, d, 1, 1));
        cudaEventRecord(b, s->stream);
        TRY(sync(s));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        t_min = std::min(t_min, ms);
      }
      if (t_min < best) { best = t_min; best_l = lanes; best_g = s->d.pcg_grid; best_p = product; }
      if (s->d.pcg_grid >= (s->n + 63) / 64) break;  // larger grids are capped to the same shape
    }
  }
  s->ev_pool.push_back(a);
  s->ev_pool.push_back(b);
  s->pcg_product = best_p;
  TRY(bdem_set_pcg_shape(s, best_l, best_g));
  if (lanes_out) *lanes_out = best_l;
  if (blocks_out) *blocks_out = best_g;
  return BDEM_OK;
}
