/*
 * bdem.h -- C ABI of the GB300 implicit bonded-DEM library (libbdem.so).
 *
 * The library advances particles that carry a position p in R^3 and a unit quaternion q
 * (stored {x, y, z, w}, scalar last) by the implicit bonded discrete element method of
 * "Implicit Bonded Discrete Element Method with Manifold Optimization":
 *   - each time step minimises Phi(x) = 1/(2 dt^2) (x - xhat)^T M_s (x - xhat) + V(x)
 *     (Sec. 3.1, Eq. optimization form; M_s = diag(m I3, 8/5 m r^2 I4), xhat = 2 x_n - x_{n-1}),
 *   - V is the bond potential of Sec. 3.2 (stretch, shear, bend-twist) plus gravity and the penalty
 *     contact of Sec. 5.4 (ground plane and self contact),
 *   - the minimisation is the second-order manifold optimisation of Sec. 4.2 / Alg. 2 inside the stable
 *     integrator of Alg. 3: Riemannian gradient and Hessian (Eq. manifold-hessian-1..4), nullspace
 *     reduction to 6 unknowns per particle, per-term eigenvalue clamp (Sec. 5.2), block-Jacobi PCG with
 *     relative tolerance min(0.5, sqrt|grad f|) (Sec. 5.3), exponential-map retraction with an
 *     energy-decrease line search (Eq. manifold-update-1/2), velocity update, and a tensile-strain bond
 *     break test after every converged step.
 * All arithmetic runs in CUDA kernels on the device; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *   - host pointers are caller-owned and only read (or written, for outputs) during the call; the library
 *     copies what it keeps;
 *   - device memory is owned by the library and released by bdem_destroy;
 *   - no call throws, aborts or traps; each returns a bdem_status and keeps a message readable through
 *     bdem_last_error(sim);
 *   - on any status other than BDEM_OK, BDEM_E_NEWTON_MAXITER and BDEM_E_LINESEARCH the simulation state
 *     is left at the last committed time step;
 *   - a simulation object must not be used from two host threads at once.
 */
#ifndef BDEM_H
#define BDEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdem_sim bdem_sim;

typedef enum {
  BDEM_OK = 0,
  BDEM_E_INVALID = 1,         /* an argument failed validation; nothing changed */
  BDEM_E_NOMEM = 2,           /* a device allocation failed */
  BDEM_E_CUDA = 3,            /* a CUDA runtime call failed */
  BDEM_E_NEWTON_MAXITER = 4,  /* warning: a scene hit newton_max_iter; its best iterate was committed */
  BDEM_E_LINESEARCH = 5,      /* warning: no step length in the halving sequence decreased Phi; the scene
                                 stopped at its current (best) iterate, which was committed */
  BDEM_E_NONFINITE = 6,       /* a residual norm became NaN/Inf; the step was rolled back */
  BDEM_E_TIMEOUT = 7          /* a device-side wait gave up; the step was rolled back */
} bdem_status;

enum { BDEM_FP64 = 0, BDEM_MIXED = 1 };   /* bdem_config.precision */
enum { BDEM_SPD_EIG = 0 };                /* bdem_config.spd_mode */
enum { BDEM_OPT_SECOND_ORDER = 0, BDEM_OPT_FIRST_ORDER = 1 };  /* bdem_config.optimizer */
enum { BDEM_INT_EULER = 0, BDEM_INT_MIDPOINT = 1 };             /* bdem_config.integrator */
enum { BDEM_PRECOND_BLOCK_JACOBI = 0, BDEM_PRECOND_AMG = 1 };   /* bdem_config.preconditioner */

/* Bond material (Sec. 3.2). G = E / (2 (1 + nu)) (isotropic relation; the paper does not define G). */
typedef struct {
  double E;                 /* Young's modulus > 0 */
  double nu;                /* Poisson ratio in (-1, 0.5) */
  double density;           /* > 0; particle mass m = density * 4/3 pi r^3 */
  double break_strain;      /* tensile strain limit > 0; +inf: unbreakable */
  double bend_twist_scale;  /* >= 0, multiplies K = diag(GJ, EI, EI)/l0 */
  double shear_scale;       /* >= 0, multiplies the shear angle: 1 gives 1/2 kt theta^2 as printed (N/m);
                               a length (e.g. the rest bond length) gives the dimensionally consistent energy */
  double tensile_strength;  /* sigma_c > 0 of the stress fracture criterion (Sec. 3.2); +inf: off */
  double shear_strength;    /* tau_c > 0 of the stress fracture criterion; +inf: off */
} bdem_material;

/* Optional device-memory hook (bdem_config.allocator): every device buffer a simulation owns is obtained from alloc
 * and returned to free, with ctx passed through and cuda_stream the library's stream, e.g. to draw from a caller's
 * memory pool such as PyTorch's caching allocator. alloc returns NULL on failure (the call then fails with
 * BDEM_E_NOMEM) and must return memory aligned to 256 bytes that stays valid until free; the library clears it on its
 * stream. The hook's functions are called from the host thread that calls the library, until bdem_destroy returns. */
typedef struct {
  void* (*alloc)(void* ctx, size_t bytes, void* cuda_stream);
  void (*free)(void* ctx, void* ptr, void* cuda_stream);
  void* ctx;
} bdem_allocator;

typedef struct {
  double dt;                /* time step > 0 */
  double gravity[3];        /* V_g = -m g.p */
  double newton_rel_tol;    /* a scene converges when |g_k|_2 <= tol |g_0|_2 (g_0 at the initial guess) or when
                               |g_k|_2 <= newton_abs_tol */
  int32_t newton_max_iter;  /* >= 1 */
  int32_t pcg_max_iter;     /* >= 1 */
  int32_t ls_max_halvings;  /* >= 0; the line search tries alpha = 1, 1/2, ..., 2^-ls_max_halvings */
  int32_t precision;        /* BDEM_FP64: every stage in FP64. BDEM_MIXED: bond Hessians, block-sparse matrix,
                               preconditioner and PCG vectors in FP32; gradient, residual norms, PCG dot
                               products, line-search energy sums and the state in FP64 */
  double ground_z;          /* ground plane z = ground_z */
  double k_ground;          /* ground penalty stiffness; 0 disables the ground */
  double k_self;            /* particle-particle penalty stiffness; 0 disables self contact */
  double contact_skin;      /* >= 0; candidate pairs are collected once per step at the initial guess when
                               |p_i - p_j| < r_i + r_j + contact_skin (same scene, not joined by an intact bond) */
  int32_t spd_mode;         /* BDEM_SPD_EIG: per-term eigenvalue clamp */
  int32_t optimizer;        /* BDEM_OPT_SECOND_ORDER (0): Newton directions from the projected Riemannian Hessian and
                               PCG (Alg. 2 inside Alg. 3); BDEM_OPT_FIRST_ORDER (1): the direction -grad f with the
                               same line search and stopping test (Alg. 1), no Hessian and no linear solve */
  void* cuda_stream;        /* cudaStream_t the library launches on (NULL: the legacy default stream) */
  double friction_slide;    /* >= 0, mu_s of the post-step friction correction (Sec. 5.4, Friction); 0: off */
  double friction_roll;     /* >= 0, mu_r of the rotation friction; 0: off. After the velocity update each element's
                               linear and angular velocity is corrected from the contacts active at x_{n+1}:
                               dv = -min(1, mu_s |F_n| dt / (m |v_t|)) v_t and
                               dw = -min(1, mu_r |F_n| r^3 dt / (I |w_ij|)) w_ij per contact (I = 2/5 m r^2,
                               relative velocities of the element pair, the ground at rest), summed, projected on
                               the element's own velocity direction and clamped so that it only slows down */
  int32_t integrator;       /* BDEM_INT_EULER (0): Phi(x) = 1/(2 dt^2) (x - xhat)^T M_s (x - xhat) + V(x), the
                               first-order form the paper uses in its experiments (Sec. 3.1, Eq.
                               implicit_euler_integrator). BDEM_INT_MIDPOINT (1): the variational midpoint form
                               (Sec. 3.1, App. C): Phi(x) = 1/(2 dt^2) (x - zhat)^T M_s (x - zhat) + V((x + x_n)/2)
                               with zhat = xhat - 1/2 M_s^{-1} dt^2 grad V((x_{n-1} + x_n)/2), x_{n-1} = x_n - dt v_n;
                               every potential (bonds, gravity, ground, self contact) at the plain average of the two
                               states in R^3 x R^4 (quaternions not renormalised); contact candidates and fracture as
                               for BDEM_INT_EULER */
  int32_t preconditioner;   /* BDEM_PRECOND_BLOCK_JACOBI (0): block-Jacobi PCG in one persistent kernel (and the step
                               graph). BDEM_PRECOND_AMG (1): the algebraic multigrid preconditioner Sec. 5.3 names,
                               read as an aggregation AMG: Z-order aggregates of 8 (levels until a scene has at most
                               8 nodes, at least one), rigid-motion coarse spaces (t, w) per aggregate, Galerkin
                               coarse operators of the assembled diagonal and bond blocks (contact off-diagonal
                               blocks left out), a symmetric V(1,1) cycle with block-Jacobi smoothing damped by 0.6,
                               exact solves of each scene's coarsest level; the textbook PCG around it runs from the
                               host-driven step loop (no step graph) */
  double newton_abs_tol;    /* >= 0; a scene also converges when |g_k|_2 <= newton_abs_tol, the absolute test
                               |grad f| < eps of Alg. 3 (0: off, only the relative test) */
  int32_t pcg_refine;       /* >= 0 (at most 16): rounds of FP64-residual refinement of each Newton solve in
                               BDEM_MIXED with block-Jacobi PCG (0: off; ignored in BDEM_FP64 and with the AMG). After
                               the FP32 PCG stops, the correction is accumulated in FP64, the true residual
                               r = b - H dx is formed with FP64 arithmetic on the stored blocks, and while
                               |r| > eps_r |b| the FP32 PCG is run again on H d = r (relative target
                               eps_r |b| / |r|), at most pcg_refine times, stopping early when |r| grows; the
                               line search takes the FP64 direction */
  int32_t reserved0;        /* set to 0 */
  const bdem_allocator* allocator; /* NULL: cudaMalloc / cudaFree; else the hook, copied by bdem_create */
} bdem_config;

/* Per-scene statistics of one bdem_step call (sums over its steps, norms of the last step). */
typedef struct {
  int32_t steps;
  int32_t newton_iters;     /* linear solves performed */
  int32_t pcg_iters;
  int32_t ls_halvings;
  int32_t bonds_broken;
  int32_t contact_candidates; /* of the last step */
  int32_t status;           /* worst bdem_status of the scene in this call */
  int32_t reserved0;
  double g0_norm;           /* |g_0| of the last step */
  double g_norm;            /* |g| at exit of the last step */
  int64_t contact_entry_pcg_iters; /* sum over linear solves of (active self-contact matrix entries x PCG iterations) */
  int64_t intact_bonds;     /* intact bonds of the scene after the last step */
  double lin_rel_residual;  /* |b - H dx| / |b| of the last linear solve of the last step, evaluated in FP64 when
                               pcg_refine > 0 in BDEM_MIXED (-1: not evaluated) */
  int32_t refine_rounds;    /* FP64-residual refinement rounds (extra PCG launches) summed over the call's steps */
  int32_t reserved1;
} bdem_step_stats;

/* Creates a simulation of n particles split into n_scenes independent scenes: scene s owns particles
 * [scene_offsets[s], scene_offsets[s+1]) (scene_offsets[0] = 0, non-decreasing, scene_offsets[n_scenes] = n).
 * Scenes share the configuration but never interact, and each converges on its own.
 *   pos[n][3], quat[n][4] (unit, +-1e-6; normalised on input), vel[n][3] or NULL (zero), quat_vel[n][4] or NULL
 *   (zero; dq/dt), radius[n] > 0, particle_material[n] in [0, n_mats), kinematic[n] or NULL: nonzero marks a
 *   particle that moves with its given velocity and is excluded from the solve (Sec. 3.1 boundary condition).
 * Returns BDEM_E_INVALID on bad input, BDEM_E_NOMEM / BDEM_E_CUDA on device failure; *out is NULL then. */
bdem_status bdem_create(const bdem_config* config, int32_t n_scenes, const int64_t* scene_offsets, const double* pos,
                        const double* quat, const double* vel, const double* quat_vel, const double* radius,
                        const int32_t* particle_material, const bdem_material* mats, int32_t n_mats,
                        const uint8_t* kinematic, bdem_sim** out);

/* Adds n bonds (i[k], j[k]) with material bond_material[k] (Sec. 3.2). Rest data comes from the current state:
 * l0 = |p_j - p_i|, d0 = conj(q_c) (.) (p_j - p_i)/l0 with q_c = (q_i + q_j)/|q_i + q_j|, r0 = (r_i + r_j)/2,
 * S = pi r0^2, I = pi r0^4/4, J = pi r0^4/2, kn = E S/l0, kt = G S/l0, K = bend_twist_scale diag(GJ, EI, EI)/l0.
 * Requires i != j, both in the same scene, no duplicate pair (also against earlier calls), l0 > 0 and
 * q_i . q_j >= 1 - 1e-12 (equal rest orientations); otherwise BDEM_E_INVALID and nothing is added.
 * Bond flags (bdem_read_state, bdem_write_state) and per-bond outputs are in the order of addition across all calls,
 * which bdem_bond_order() lists. */
bdem_status bdem_add_bonds(bdem_sim* sim, int64_t n, const int32_t* i, const int32_t* j, const int32_t* bond_material);

/* Advances n_steps >= 0 time steps (Alg. 3). stats: NULL or an array of n_scenes entries. Host-blocking: returns
 * when the last step has completed on the device.
 * By default every step after the first is one launch of a captured CUDA graph whose Newton and line-search loops
 * are conditional while nodes decided on the device (one host synchronisation per step); the first step, a step
 * whose contact candidates outgrow the arrays sized so far (repeated, not committed twice), and every step while
 * phase timing is on run the same kernels from a host-driven loop. Both orders give bit-identical results. */
bdem_status bdem_step(bdem_sim* sim, int32_t n_steps, bdem_step_stats* stats);

/* on = 0: every step uses the host-driven loop; on = 1 (default): steps use the captured step graph when the
 * device supports it. Clears a recorded capture failure. */
bdem_status bdem_set_step_graph(bdem_sim* sim, int32_t on);

/* Steps that ran through the captured graph since creation. */
int64_t bdem_graph_steps(const bdem_sim* sim);

/* Why the step graph could not be captured or instantiated ("" if it could); steps then use the host-driven
 * loop. */
const char* bdem_graph_error(const bdem_sim* sim);

/* Copies the committed state to caller host buffers; any pointer may be NULL. pos[n][3], quat[n][4], vel[n][3],
 * quat_vel[n][4], bond_broken[n_bonds] (1 = broken). Synchronises the library's stream. */
bdem_status bdem_read_state(bdem_sim* sim, double* pos, double* quat, double* vel, double* quat_vel,
                            uint8_t* bond_broken);

/* Overwrites the dynamic state (for checkpoint / resume); NULL leaves a field unchanged. Rest data is kept.
 * quat must be unit (+-1e-6). */
bdem_status bdem_write_state(bdem_sim* sim, const double* pos, const double* quat, const double* vel,
                             const double* quat_vel, const uint8_t* bond_broken);

/* Sizes: particles, intact + broken bonds, scenes. */
bdem_status bdem_sizes(const bdem_sim* sim, int64_t* n_particles, int64_t* n_bonds, int32_t* n_scenes);

/* The bonds in their order of addition: pairs[2k], pairs[2k+1] = (min(i, j), max(i, j)) of the k-th bond added. */
bdem_status bdem_bond_order(const bdem_sim* sim, int32_t* pairs);

/* Releases every device and host resource of sim (NULL is ignored). */
void bdem_destroy(bdem_sim* sim);

/* Message of the last failed call on sim ("" if none); valid until the next call on sim. NULL sim: the message of
 * the last failed bdem_create. */
const char* bdem_last_error(const bdem_sim* sim);

/* ---- inspection entry points (the Newton system the step builds, for verification) --------------------------
 * They evaluate at the current committed state x with inertia targets (phat, qhat) given by the caller (host,
 * [n][3], [n][4]); contact candidates are collected at x. They run the same kernels as bdem_step. */

/* Reduced gradient g[n][6] (FP64), assembled projected diagonal blocks diag[n][6][6], per-bond projected reduced
 * Hessians bond_hess[n_bonds][12][12] in the order (dp_i, y_i, dp_j, y_j) (zero for broken bonds), and the number
 * of contact candidates; any output may be NULL. Kinematic rows are not masked. Rows and particles are in the
 * caller's order, bonds in their order of addition. */
bdem_status bdem_debug_system(bdem_sim* sim, const double* phat, const double* qhat, double* g, double* diag,
                              double* bond_hess, int64_t* n_candidates);

/* The same at the iterate x = (pos [n][3], quat [n][4]) given by the caller (both NULL: the committed state). The
 * committed state is the step's start state x_n of the variational midpoint form (bdem_config.integrator), whose
 * potentials are then evaluated at (x + x_n)/2; contact candidates are collected at x. */
bdem_status bdem_debug_system_at(bdem_sim* sim, const double* pos, const double* quat, const double* phat,
                                 const double* qhat, double* g, double* diag, double* bond_hess, int64_t* n_candidates);

/* The inertia targets a step from the committed state uses, in the caller's order: xhat = x_n + dt v_n with
 * BDEM_INT_EULER; with BDEM_INT_MIDPOINT zhat = xhat - 1/2 M_s^{-1} dt^2 grad V((x_{n-1} + x_n)/2) (Sec. 3.1,
 * App. C; x_{n-1} = x_n - dt v_n; the step's contact candidates, collected at (xhat, qhat/|qhat|)). zp [n][3],
 * zq [n][4] host. Replaces the system of the last bdem_debug_system call. */
bdem_status bdem_debug_zhat(bdem_sim* sim, double* zp, double* zq);

/* Per-bond projected reduced Hessians [count][12][12] of the bonds ids[k] (order of addition) from the system of the
 * last bdem_debug_system call (called with bond_hess = NULL to skip the full download). */
bdem_status bdem_debug_bonds(bdem_sim* sim, int64_t count, const int32_t* ids, double* bond_hess);

/* Stresses (sigma, tau) of the stress fracture criterion (Sec. 3.2) of every bond at the committed state, computed
 * in FP64 by the kernel the fracture test uses: out host [n_bonds][2] in the order of addition (broken bonds
 * included, evaluated as if intact). */
bdem_status bdem_debug_bond_stress(bdem_sim* sim, double* out);

/* Runs one device-side wait on a word that nothing writes, with a time limit of limit_ms (0..10000) instead of the
 * 2 s every wait of the library uses: the wait gives up, sets the device's timeout flag, and the call returns
 * BDEM_E_TIMEOUT as a step would (the simulation stays usable). For testing the failure path without a GPU fault. */
bdem_status bdem_debug_wait_timeout(bdem_sim* sim, double limit_ms);

/* y = H x with the system of the last bdem_debug_system call; x, y host [n][6]. The product is formed in FP64
 * arithmetic on the stored blocks (FP32 words in BDEM_MIXED), so it is the exact product of the stored matrix up to
 * the rounding of the FP64 sums. */
bdem_status bdem_debug_matvec(bdem_sim* sim, const double* x, double* y);

/* PCG (Sec. 5.3) on H dx = b with the system of the last bdem_debug_system call (kinematic rows removed), from
 * dx = 0 until |r| <= eps_r |b| or max_iter iterations. b, dx host [n][6]; iters[n_scenes] or NULL. With
 * pcg_refine > 0 in BDEM_MIXED the solve is refined as a Newton solve is (the FP64 residual b - H dx of the
 * accumulated FP64 solution must meet eps_r |b|; iters counts the iterations of every round). */
bdem_status bdem_debug_pcg(bdem_sim* sim, const double* b, double eps_r, int32_t max_iter, double* dx,
                           int32_t* iters);

/* Kernel launches issued by this sim since creation (for launch accounting). */
int64_t bdem_launch_count(const bdem_sim* sim);

/* ---- launch shape of the persistent PCG kernel ---------------------------------------------------------------------
 * lanes_per_row in {1, 2, 4, 8}: threads that share one block row of the product (the rows of a warp = 32 / lanes);
 * blocks: PCG grid size, 0 = every co-resident block (capped at one block per 64 rows). Changing the shape changes
 * the grouping of the FP64 partial sums, so results differ at rounding level between shapes; a fixed shape gives
 * bit-identical runs. With 5 to 128 scenes and products 0-2 (bdem_set_pcg_product) the rows of the scenes still
 * iterating are split evenly over the blocks again at every PCG iteration, when no block's share can span more than
 * 32 scenes; that partition is part of the shape, so runs stay bit-identical. */
bdem_status bdem_set_pcg_shape(bdem_sim* sim, int32_t lanes_per_row, int32_t blocks);


/* How the PCG product reaches the off-diagonal bond blocks: product = 1 (default): in waves of one entry per thread,
 * each warp first copies its wave's 32 blocks into shared memory with 16-byte asynchronous copies taken by
 * consecutive threads from the same block (few cache lines per request); product = 2: the same with two buffers, the
 * next wave's copies in flight while a wave is multiplied (twice the shared memory, fewer resident blocks);
 * product = 0: each thread loads its own entries' blocks (with the row descriptors and incidence entries staged in
 * shared memory when they fit); these three give the same sums in the same order. product = 3: the fused PCG, one
 * grid barrier per iteration: the vector update is folded into the next product (each block keeps its rows' new z in
 * shared memory and recomputes its halo rows' z from their previous r, s and w, which alternate between two buffers),
 * with the bond blocks staged as in product 1; the same iterates up to rounding. Keeps the lanes and grid (the grid
 * shrinks if the blocks no longer fit); BDEM_E_INVALID when no block of the product fits an SM beside its share of
 * the rows, with the previous product kept. */
bdem_status bdem_set_pcg_product(bdem_sim* sim, int32_t product);

/* The current PCG launch shape: lanes per row, grid size and product (as bdem_set_pcg_product); NULL skips. */
bdem_status bdem_get_pcg_shape(const bdem_sim* sim, int32_t* lanes_per_row, int32_t* blocks, int32_t* product);

/* Times the PCG kernel for `iters` iterations on the system at the current committed state for each candidate shape
 * (products 3, 2, 1, 0 x lanes 1, 2, 4, 8 x 1..all co-resident blocks per SM; shapes whose blocks do not fit an SM are
 * skipped), keeps the fastest, and reports its lanes and grid (either pointer may be NULL; bdem_get_pcg_shape gives
 * the product). Every scene iterates while it is timed (no stopping test), so the even re-split of many scenes is
 * timed without the savings it makes once scenes stop. Host-blocking. */
bdem_status bdem_autotune_pcg(bdem_sim* sim, int32_t iters, int32_t* lanes_per_row, int32_t* blocks);

/* ---- bond-Hessian tile ------------------------------------------------------------------------------------------
 * The bond kernel that evaluates each bond's 12x12 reduced Hessian and its eigenvalue clamp (one thread per bond)
 * runs in blocks of `tile` threads (64, 128 or 256; default 128); capped = 1 selects its variant compiled for 128
 * registers per thread (twice the resident warps, with spills; FP32 path, first-order form only, else ignored). */
bdem_status bdem_set_bond_tile(bdem_sim* sim, int32_t tile, int32_t capped);

/* Times the bond-Hessian kernel `reps` times on the system at the current committed state for each tile and register
 * variant, keeps the fastest and reports it (either pointer may be NULL). Host-blocking. */
bdem_status bdem_autotune_bonds(bdem_sim* sim, int32_t reps, int32_t* tile, int32_t* capped);

/* ---- allocation-free solve ---------------------------------------------------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that cannot allocate device memory, for
 * example code running under an external memory pool that forbids extra cudaMalloc calls, or a host thread that
 * must not trigger allocation while other work is being captured or scheduled.
 * It runs the block-Jacobi PCG solve (kinematic rows removed) on the system assembled by the last bdem_debug_system
 * call, whatever bdem_config.preconditioner and pcg_refine say: this is bdem_debug_pcg's solve when the
 * preconditioner is block Jacobi and pcg_refine is 0 (no FP64-residual refinement). It keeps all of its scratch
 * (per-scene control blocks, barrier
 * counters, partial sums, PCG vectors) in one static device array of 24 MiB inside the library, so the call itself
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine). That caps the system at about 87,000
 * particles in BDEM_FP64 and 174,000 in BDEM_MIXED; larger systems get BDEM_E_INVALID with the byte counts.
 *   b_dev, x_dev: caller-owned DEVICE arrays [n][6] of double (right-hand side in, solution out).
 *   iters: NULL or host int32_t[n_scenes] receiving the iterations per scene.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that device current
 * and caches it (the cache is safe to fill from several host threads), so make that first call before any stream
 * capture. Every GPU that loads the library holds the array until the process exits. All calls share the array and
 * each call overwrites it, clearing what must start at zero; calls whose work overlaps on the GPU (other host
 * threads, other streams, other sims) race on it and must be serialised by the caller. Host-blocking: returns after
 * the solve has completed. */
bdem_status bdem_pcg_static(bdem_sim* sim, const double* b_dev, double* x_dev, double eps_r, int32_t max_iter,
                            int32_t* iters);

/* ---- phase timing: CUDA events recorded on the library's stream around each stage's launches ------------------ */
enum {
  BDEM_PH_PREDICT = 0,     /* prediction and step set-up */
  BDEM_PH_CONTACT = 1,     /* spatial hash and contact candidate lists */
  BDEM_PH_GRAD = 2,        /* bond gradients, per-particle gradient gather, residual norms */
  BDEM_PH_HESS = 3,        /* bond Hessians with eigenvalue clamp, diagonal blocks and their inverses */
  BDEM_PH_PCG = 4,         /* the persistent PCG kernel */
  BDEM_PH_LINESEARCH = 5,  /* descent check, retraction trials, energy differences, commit */
  BDEM_PH_FINISH = 6,      /* velocity update and fracture */
  BDEM_N_PHASES = 7
};
typedef struct {
  double ms[BDEM_N_PHASES];         /* summed event time per phase */
  int64_t intervals[BDEM_N_PHASES]; /* timed intervals per phase (the PCG phase: one per kernel launch) */
  int64_t pcg_iters;                /* PCG iterations summed over scenes */
  int64_t newton_iters;             /* linear solves summed over scenes */
  int64_t particle_newton_iters;    /* sum over scenes of particles x Newton iterations */
  int64_t steps;
} bdem_profile;

/* on != 0 enables timing and clears the counters; on == 0 disables it. */
bdem_status bdem_profile_enable(bdem_sim* sim, int32_t on);
bdem_status bdem_profile_read(bdem_sim* sim, bdem_profile* out);

#ifdef __cplusplus
}
#endif
#endif
