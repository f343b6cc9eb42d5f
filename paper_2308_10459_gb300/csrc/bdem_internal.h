// bdem_internal.h -- device data layout and kernel launchers shared by bdem_kernels.cu and bdem_api.cu.
//
// Layout in HBM (N particles, B bonds, S scenes; T = float in the mixed path, double in the FP64 path):
//   particles are stored in a space-filling-curve (Morton) order inside each scene, so that bonded and contacting
//             particles are close in memory; every transfer across the ABI is reordered on the device
//   particles, AoS of double4 (32 B, two per particle state): xp = (p, radius), xq = q       current iterate
//             x0p, x0q committed state of the step; vp = (v, 0), vq = dq/dt; hp = (phat, mass), hq = qhat (raw);
//             tp, tq line-search trial; coef = (c_p, c_q) = (m/dt^2, 8/5 m r^2/dt^2); g [N][6] FP64 gradient;
//             D, Dinv [N][24] T packed symmetric diagonal blocks (21 words + 3 pad) and their inverses (block Jacobi);
//             PCG vectors [N][6] T (x, r, z, p, q)
//   bonds, sorted by (i, j) with i < j (so each scene's bonds are contiguous):
//             bij int2; brest double4 (d0, l0); bstiff double4 (kn, kt s^2, kb, ktw); bbrk double; bbroken u8;
//             bsgeo double4 (1/S, r0/I, r0/J, 0) and bsstr double2 (sigma_c, tau_c) of the stress criterion;
//             bg [B][9] FP64 gradient in (d = p_j - p_i, y_i, y_j);
//             bM [B][36] T: the (i, j) off-diagonal 6x6 block in factored form (1/2 A sym6 | B/sqrt2 3x3 |
//             C/sqrt2 3x3 | F 3x3 | 3 pad) of the clamped 9x9 Hessian in (u = (dp_j - dp_i)/sqrt2, y_i, y_j);
//             bE [B][12] T: its E (y_i y_i) and G (y_j y_j) blocks, sym6 each
//   incidence CSR inc_start [N+1], inc2 [2B] int2 entries (bond << 1 | side, other particle), side 0: particle is
//             i, 1: particle is j; entries of a particle are in bond order
//   contact CSR c_start [N+1], c_nbr [C] candidates; per Newton iteration the active ones are compacted to the front
//             of each particle's range: c_anbr [C], c_blk [C] T4 (n, k) of the clamped contact Hessian k n n^T,
//             c_act [N] counts
//   tiles: particle tiles of <= 256 rows inside one scene, bond tiles of <= 256 bonds inside one scene
//   PCG segments: the persistent PCG grid gives block b a row range of the product balanced by rows + incidence
//             entries; its intersections with the scenes are the segments (seg_row [nseg+1], seg_scene,
//             block_seg [P+1], scene_seg [S+1]); one partial per segment and quantity (part_s [nseg][4]). The
//             elementwise phases use the equal-rows ranges [b N / P, (b+1) N / P) cut the same way at scene
//             boundaries (useg_row, useg_scene, ublock_seg)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bdem {

constexpr int kTile = 256;      // rows (particles or bonds) per tile = threads per block of tile kernels
constexpr int kPartials = 4;    // partial sums per tile
constexpr int kDiagStride = 24; // words per stored 6x6 symmetric block (21 used, padded for 128-bit loads)
constexpr int kLocalPcgScenes = 4;   // up to this many scenes every PCG block decides every scene
constexpr int kDistPcgScenes = 16;   // with more, a block decides its own scenes when its rows span at most this many
constexpr int kEvenPcgScenes = 128;  // up to this many scenes the PCG can re-split the active rows every iteration
constexpr int kEvenPcgSegs = 32;     // most scenes one block's share of the active rows may span
constexpr int kPcgMaxBlocks = 2048;  // largest PCG grid (grids are at most 8 blocks of kTile threads per SM)

struct SceneCtl {
  double g0, gnorm, eps_r, bnorm;
  double rz, pq, alpha, beta;
  double dphi, ls_alpha, gdx, pcg_thr2;  // pcg_thr2: (eps_r |b|)^2 of the current solve
  long long act_cur;            // active self-contact matrix entries of the current Newton system
  long long act_pcg;            // sum over this step's solves of act_cur x PCG iterations
  long long intact;             // intact bonds after the step's fracture test
  int32_t newton_active;        // still iterating Newton in this step
  int32_t pcg_active;
  int32_t pcg_iters;            // in the current solve
  int32_t use_neg_grad;         // the PCG direction was not a descent direction
  int32_t ls_state;             // 0 pending, 1 accepted, 2 failed
  int32_t newton_iters;         // in this step
  int32_t pcg_total, ls_halvings;
  int32_t status;               // bdem_status of the scene in this step
  int32_t bonds_broken;
  int32_t pad1;                 // halvings in the current line search
  int32_t pad2;                 // contact candidates of the step
  // FP64-residual refinement of the mixed-precision Newton solve (DevArrays::refine > 0)
  double eps_out, b_out;        // the solve's relative target eps_r and |b| (the first PCG launch's)
  double res64;                 // |b - H dx| of the accumulated FP64 solution after the last round
  double lin_res;               // |b - H dx| / |b| of the last completed solve (-1: not evaluated)
  int32_t pcg_skip;             // 1: the scene takes no part in the current PCG launch (its solve is complete)
  int32_t refine_round;         // refinement rounds of the current solve
  int32_t pcg_acc;              // PCG iterations of the current solve over its rounds
  int32_t refine_total;         // refinement rounds in this step
};

struct Counters {               // small device-side summary read by the host after reductions
  int32_t n_active;             // scenes with work left in the current loop
  int32_t n_pending;
  int32_t timeout;              // a device wait gave up
  int32_t nonfinite;
  unsigned int sync_count;      // grid barrier arrival counter
  unsigned int sync_gen;        // grid barrier generation
  int32_t overflow;             // graph path: contact candidates needed when the contact arrays were too small
  int32_t runaway;              // graph path: a device-driven loop passed its iteration cap
  int32_t loops_newton;         // gradient reductions in this step (device-driven Newton loop trips + 1)
  int32_t loops_ls;             // trials of the current line search
  int32_t ls_total;             // line-search trials in this step
  unsigned int never;           // written by nothing: the word the wait test waits on
  int32_t loops_refine;         // refinement rounds in this step (graph path: trips of the refinement loop)
  int32_t loops_amg;            // AMG-PCG iterations in this step (trips of the device-driven iteration loop)
  int32_t amg_trips;            // trips of the current AMG-PCG solve's loop
  int32_t dist_active[3];       // PCG with per-block decisions: scenes still iterating after iteration k, in [k % 3]
};

struct DevArrays {
  int32_t n, nb, n_scenes, n_ptiles, n_btiles;
  int32_t mixed;                // T = float when 1, double when 0
  int32_t c_cap;                // capacity of the contact arrays
  int32_t hash_size;            // power of two
  double dt, gx, gy, gz, tol, ground_z, k_ground, k_self, skin, cell_h;
  double tol_abs;               // absolute Newton tolerance (0: off)
  double mu_slide, mu_roll;     // friction coefficients of the post-step correction (0: off)
  unsigned long long wait_ns;   // time limit of every device-side wait
  int32_t newton_max, pcg_max, ls_max;
  int32_t stress_on;            // some bond has a finite tensile or shear strength
  int32_t first_order;          // descent direction -g (Alg. 1) instead of the Newton direction
  int32_t midpoint;             // variational midpoint form: potentials at (x + x0)/2, inertia targets zhat
  int32_t refine;               // rounds of FP64-residual refinement per Newton solve (0: off; mixed + block Jacobi)
  int32_t bond_tile;            // threads per block of the bond-Hessian kernel (64, 128, 256)
  int32_t bond_capped;          // 1: its register-capped variant (FP32, first-order form)
  double* x64;                  // [N][6] FP64 accumulated solution of the refined solve (refine > 0)
  double* b64;                  // [N][6] FP64 right-hand side of an inspection solve (NULL: b = -g)
  // particles
  double4 *xp, *xq, *x0p, *x0q, *vp, *vq, *hp, *hq, *tp, *tq;
  double2* coef;
  int32_t* pscene;
  int32_t* perm;                // caller index of internal particle k (internal order: Morton order per scene)
  uint8_t* kin;
  double* g;
  void *D, *Dinv;
  void *vx, *vr, *vz, *vp_, *vq_, *vs;   // x, r, z, p, w (= H z; also the inspection product), s (= H p)
  void *vr2, *vs2, *vq2;        // second buffers of r, s, w for the fused PCG (k_pcg_fused)
  // bonds
  int2* bij;
  double4 *brest, *bstiff;
  double* bbrk;
  double4* bsgeo;               // (1/S, r0/I, r0/J, 0) of the stress criterion
  double2* bsstr;               // (sigma_c, tau_c); +inf: off
  uint8_t* bbroken;
  int32_t* bscene;
  int32_t *bond_ext2int, *bond_int2ext;  // caller bond order (order of addition) <-> stored order
  double* bg;
  void *bM, *bE;
  int32_t* inc_start;
  int2* inc2;
  // contacts
  int32_t *c_start, *c_nbr, *c_anbr, *c_act;
  void* c_blk;
  int32_t *cell_key, *hash_count, *hash_start, *hash_ids, *cnt_tmp;
  int64_t* scan_tmp;
  // tiles
  int32_t *ptile_start, *ptile_scene, *ptile_begin;   // ptile_begin [S+1]: first tile of each scene
  int32_t *btile_start, *btile_scene, *btile_begin;
  double *part_p, *part_b;      // [tiles][kPartials]
  int32_t n_seg, pcg_grid, pcg_lanes, pcg_max_rows;  // pcg_max_rows: most rows of one PCG block
  int32_t pcg_max_entries, pcg_mode;                 // most incidence entries of one PCG block's rows; how the
                                                     // product reaches the bond blocks (k_pcg MODE 0, 1, 2)
  int32_t *seg_row, *seg_scene, *block_seg, *scene_seg;
  int32_t *useg_row, *useg_scene, *ublock_seg;      // equal-rows partition of the elementwise PCG phases
  // fused PCG (pcg_mode 4): each block's halo rows (rows outside its product range that its bond entries reference),
  // halo_start [P+1] into halo_rows; the incidence entries with their neighbour's slot in the block's shared z array
  // (own rows first, then the halo); the most slots of one block
  int32_t *halo_start, *halo_rows;
  int2* inc2_loc;
  int32_t pcg_max_zslots;
  int32_t pcg_rows_sm;          // pcg_mode 2, 3: 1 when each block stages its row descriptors in shared memory
  int32_t pcg_even;             // 1: the rows of the scenes still iterating are split evenly over the grid at every
                                // iteration, and every block decides every scene (pcg_even_off: the byte offset of
                                // the per-block state in the dynamic shared memory)
  int32_t pcg_even_off;
  int32_t pcg_part_slots;       // partial-dot slots of the PCG (part_s): segments, or blocks x kEvenPcgSegs
  int32_t pcg_dist;             // 1: more scenes than kLocalPcgScenes and every PCG block's rows span at most
                                // kDistPcgScenes scenes, so each block takes its own scenes' decisions
  double* part_s;               // [n_seg][kPartials]
  SceneCtl* sc;
  Counters* cnt;
};

// ---- aggregation AMG preconditioner (Sec. 5.3) --------------------------------------------------------------------
// Level 0: the particles (internal order = Z-order of the initial positions inside each scene); level l+1: groups of
// kAmgAgg consecutive level-l nodes of one scene, built while the scene has more than kAmgAgg nodes (at least one
// coarse level); coarse spaces of rigid motions (t, w) per node; A_1 = Galerkin product of the assembled diagonal
// blocks and bond blocks (contact off-diagonal blocks left out), A_{l+1} = P^T A_l P; the coarsest level of each
// scene (<= kAmgAgg nodes) is solved by a dense Cholesky factor. Patterns and Galerkin source lists are built on the
// host from the bond list; values are recomputed on the device at every Newton iteration.
constexpr int kAmgMaxLevels = 12;
constexpr int kAmgAgg = 8;
constexpr int kAmgDense = 6 * kAmgAgg;  // largest coarsest system per scene
struct AmgLevel {
  int32_t n, nnz;
  int32_t *cbeg, *cend;  // [n] children [cbeg, cend) of each node (level l-1 nodes; on level 1 internal particles)
  int32_t* parent;  // [n] node of level l+1 holding this node; -1 on the scene's coarsest level
  int32_t *rs, *col, *erow, *diag;  // block CSR of A_l: row starts [n+1], columns and rows [nnz], diagonal entry [n]
  int32_t *gs, *gsrc;  // Galerkin sources per entry: level 1 bond codes (b << 1 | o, o = 1: the transposed block),
                       // level l >= 2 entries of level l-1
  void *val, *dinv;    // [nnz][36], [n][36] T
  double* cen;         // [n][3] centroids
  void *r, *x, *t;     // [n][6] T cycle vectors
};
struct AmgDev {
  int32_t nl, on;              // number of levels (level 0 included); the preconditioner is in use
  double omega;                // damping of the block-Jacobi smoothing
  AmgLevel L[kAmgMaxLevels];   // L[0]: only parent (= level-1 node of each particle) and t are used
  int32_t *sc_level, *sc_off, *sc_m;  // per scene: coarsest level, its first node there, its node count
  void* p0;                    // [N][12] T per particle: offset from its aggregate's centroid (3), 1/2 R(q)^T (9)
  double* chol;                // [S][kAmgDense^2] dense Cholesky factors of the coarsest operators
};

// ---- launchers (bdem_kernels.cu); each returns the number of kernels launched -----------------------------------
int launch_predict(const DevArrays& d, cudaStream_t s);
// variational midpoint form: zhat = xhat - 1/2 M^-1 dt^2 grad V((x_{n-1} + x_n)/2) into hp, hq (after the contact
// candidates of the step exist); no launch otherwise
int launch_zhat(const DevArrays& d, cudaStream_t s);
// the iterate x (xp, xq) from the caller's order (inspection calls)
int launch_set_iterate(const DevArrays& d, const double* pos3, const double* quat4, cudaStream_t s);
// stage 0: hash + count, 1: fill, 2: capacity guard of the graph path (records the overflow and empties every
// candidate list, so that no later kernel reads past the contact arrays)
int launch_contacts(const DevArrays& d, int stage, cudaStream_t s);
int launch_scan_counts(const DevArrays& d, const int32_t* counts, int32_t* starts, int n, cudaStream_t s);
int launch_bond_grad(const DevArrays& d, int all_scenes, cudaStream_t s);
int launch_particle_grad(const DevArrays& d, int mask_kin, int all_scenes, cudaStream_t s);
int launch_bond_hess(const DevArrays& d, int all_scenes, cudaStream_t s);
int launch_particle_hess(const DevArrays& d, int mask_kin, int all_scenes, cudaStream_t s);
// reduction modes of the per-scene reduce kernel
enum ReduceMode { RED_GRAD = 0, RED_GDX = 1, RED_LS = 2, RED_FORCE_ACTIVE = 3, RED_CAND = 4, RED_REFINE0 = 5,
                  RED_REFINE = 6 };
// cond: 0, or the conditional handle of the device-driven loop that this reduction controls in the step graph
// (RED_GRAD: the Newton loop, RED_GDX and RED_LS: the line-search loop)
int launch_scene_reduce(const DevArrays& d, int mode, unsigned long long cond, cudaStream_t s);
// PCG: rhs_from_g = 1 uses b = -g; else b is read from vr (already T) and eps from sc.eps_r
int launch_pcg(const DevArrays& d, int rhs_from_g, int mask_kin, cudaStream_t s, cudaError_t* err);
int pcg_max_blocks(int mixed, int lanes, size_t smem, int mode);  // co-resident PCG blocks on this device (0: none)
size_t pcg_smem_bytes(const DevArrays& d);  // dynamic shared memory of a PCG block in the arrays' mode
size_t pcg_smem_bytes_for(int mode, int mixed, int max_rows, int max_entries, int max_zslots);
size_t pcg_even_bytes();  // the per-block state of the even re-partition (in dynamic shared memory)
int launch_gdx(const DevArrays& d, cudaStream_t s);
int launch_ls_trial(const DevArrays& d, cudaStream_t s);
int launch_ls_energy(const DevArrays& d, cudaStream_t s);
int launch_ls_commit(const DevArrays& d, cudaStream_t s);
int launch_finish(const DevArrays& d, cudaStream_t s);
int launch_matvec(const DevArrays& d, int mask_kin, cudaStream_t s);  // vq_ = H vp_
// y64 = H x64 in FP64 arithmetic on the stored blocks (both [N][6] double, internal order)
int launch_matvec64(const DevArrays& d, const double* x64, double* y64, int mask_kin, cudaStream_t s);
// FP64-residual refinement: first = 1 sets x64 = x (the PCG solution), else x64 += x, for the scenes of the last PCG
// launch; then r = b - H x64 in FP64 (b = -g, or b64 when set), r rounded into vr for the next PCG launch, and the
// per-tile |r|^2 partials (reduced by RED_REFINE0 / RED_REFINE)
int launch_refine(const DevArrays& d, int first, cudaStream_t s);
int launch_unpack_bond_hess(const DevArrays& d, double* out, const int32_t* ids, int count, cudaStream_t s);
int launch_unpack_diag(const DevArrays& d, double* out /*device [n][36]*/, cudaStream_t s);
int launch_bond_stress(const DevArrays& d, double* out /*device [nb][2], caller bond order*/, cudaStream_t s);
// transfers in the caller's particle order (any pointer may be NULL): committed state <-> [n][3] / [n][4] arrays
int launch_pack_state(const DevArrays& d, double* pos3, double* quat4, double* vel3, double* qvel4, cudaStream_t s);
int launch_unpack_state(const DevArrays& d, const double* pos3, const double* quat4, const double* vel3,
                        const double* qvel4, cudaStream_t s);
int launch_set_hat(const DevArrays& d, const double* phat3, const double* qhat4, cudaStream_t s);
int launch_pack_hat(const DevArrays& d, double* phat3, double* qhat4, cudaStream_t s);  // hp, hq -> caller order
int launch_bond_flags(const DevArrays& d, uint8_t* ext, int to_device, cudaStream_t s);
int launch_convert_perm(const void* src, int src_double, void* dst, int dst_double, const int32_t* perm, int dir,
                        int n, cudaStream_t s);
// allocation-free PCG scratch (static device array in bdem_kernels.cu)
size_t static_pcg_capacity();
cudaError_t static_pcg_address(void** out);
int launch_static_pcg_init(const DevArrays& d, double eps_r, cudaStream_t s);
int launch_wait_test(const DevArrays& d, cudaStream_t s);  // a bounded wait that always runs out
int launch_convert(const void* src, int src_double, void* dst, int dst_double, int64_t count, cudaStream_t s);
// AMG: coarse operators of the current Newton system (centroids, Galerkin products, block inverses, coarsest
// factors); one V(1,1) cycle z = M^-1 r (r = PCG residual vr, z = vz; its level-0 smoothing steps belong to the PCG
// stages around it: the stages that produce r pre-smooth, the stages that read z post-smooth); PCG steps with the
// cycle as preconditioner
int launch_amg_setup(const DevArrays& d, const AmgDev& a, int n_scenes, cudaStream_t s);
int launch_amg_cycle(const DevArrays& d, const AmgDev& a, int n_scenes, cudaStream_t s);
// AMG-preconditioned PCG pieces (per-scene state in SceneCtl): stage 0 r = b = -g (masked), x = 0, |b|^2 -> thr2;
// 1 gamma = r.z, p = z; 2 q = H p and alpha from p.q; 3 x += alpha p, r -= alpha q, stop test (counts active scenes into
// cnt->n_active); 4 beta from the new r.z, p = z + beta p
int launch_amg_pcg_stage(const DevArrays& d, const AmgDev& a, int stage, cudaStream_t s);
// the AMG-PCG iteration loop decided on the device: loop_init (before the conditional while node) starts a solve's
// trip count and sets the loop's condition; iteration_begin opens each trip (clears the active-scene count);
// loop_cond (closing the body) continues while a scene is still iterating, up to pcg_max + 1 trips
int launch_amg_loop_init(const DevArrays& d, unsigned long long cond, cudaStream_t s);
int launch_amg_iteration_begin(const DevArrays& d, cudaStream_t s);
int launch_amg_loop_cond(const DevArrays& d, unsigned long long cond, cudaStream_t s);

}  // namespace bdem
