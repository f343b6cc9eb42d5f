/*
 * bdem_oracle.h -- interface of the CPU oracle for the implicit bonded DEM step.
 *
 * TEST INFRASTRUCTURE ONLY. The oracle is a plain, slow, single-threaded FP64 restatement of the
 * method of "Implicit Bonded Discrete Element Method with Manifold Optimization": the
 * optimisation-based integrator (Sec. 3.1, Eq. implicit_euler_integrator / optimization form), the
 * bond potential (Sec. 3.2), penalty contact (Sec. 5.4), the second-order manifold optimisation
 * (Sec. 4.2, Alg. 2, Eq. manifold-hessian-1..4 and the nullspace reduction) inside the stable
 * integrator of Alg. 3 (Sec. 5), plus a strain fracture test after each converged step.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it. It shares
 * no code, header, table or helper with the CUDA library; neither side includes the other.
 *
 * Conventions: quaternions are stored {u, v, w, s} (vector part first, scalar last, App. A).
 * Reduced (tangent) coordinates are 6 per particle: (dp in R^3, y in R^3) with dq = G_l(q)^T y.
 */
#ifndef BDEM_ORACLE_H
#define BDEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double dt;               /* time step */
  double gravity[3];       /* gravitational acceleration, V_g = -m g.p */
  double newton_rel_tol;   /* stop when |g_k| <= tol |g_0| */
  int32_t newton_max_iter;
  int32_t pcg_max_iter;
  int32_t ls_max_halvings;
  int32_t optimizer;       /* 0: second-order manifold optimisation (Alg. 2); 1: first-order (Alg. 1) */
  double ground_z;         /* ground plane z = ground_z */
  double k_ground;         /* 0: no ground */
  double k_self;           /* 0: no self contact */
  double contact_skin;     /* candidate distance margin */
  double mu_slide;         /* sliding friction coefficient of the post-step friction (0: off) */
  double mu_roll;          /* rotation friction coefficient (0: off) */
  int32_t integrator;      /* 0: the implicit-Euler-like form (V at x_{n+1}); 1: the variational midpoint form of
                              Sec. 3.1 / App. C (V at (x_{n+1} + x_n)/2 and the target zhat) */
  int32_t preconditioner;  /* 0: block Jacobi; 1: the aggregation AMG cycle (Sec. 5.3; needs P->morton) */
  double newton_abs_tol;   /* also stop when |g_k| <= newton_abs_tol: Alg. 3's absolute test |grad f| < eps (0: off) */
} orc_config;

/* Particle, bond and scene arrays. Bond rest data is filled by orc_bond_rest(). */
typedef struct {
  int32_t n, nb, n_scenes, pad0;
  const int64_t* scene_start;   /* [n_scenes+1] */
  double* p;                    /* [n][3] position at step start (in/out) */
  double* q;                    /* [n][4] unit quaternion (in/out) */
  double* v;                    /* [n][3] linear velocity (in/out) */
  double* u;                    /* [n][4] quaternion velocity dq/dt (in/out) */
  const double* radius;         /* [n] */
  const double* mass;           /* [n] */
  const uint8_t* kinematic;     /* [n] or NULL */
  const int32_t* bi;            /* [nb] */
  const int32_t* bj;            /* [nb] */
  double* l0;                   /* [nb] rest length */
  double* d0;                   /* [nb][3] rest direction in the frame of q_c */
  double* R0;                   /* [nb][9] row-major, maps d0 to e_x */
  double* kn;                   /* [nb] ES/l0 */
  double* kt;                   /* [nb] GS/l0 */
  double* kbt;                  /* [nb][3] bend_twist_scale * (GJ, EI, EI)/l0 */
  double* shear_scale;          /* [nb] multiplies theta in the shear energy */
  double* break_strain;         /* [nb] tensile strain limit (+inf: unbreakable) */
  uint8_t* broken;              /* [nb] */
  const double* tensile_strength; /* [nb] sigma_c of the stress criterion (+inf: off), or NULL */
  const double* shear_strength;   /* [nb] tau_c of the stress criterion (+inf: off), or NULL */
  const int32_t* morton;          /* [n] the particles of each scene in the Z-order of their initial positions
                                     (orc_morton_order), or NULL (no AMG) */
} orc_problem;

typedef struct {
  int32_t newton_iters;
  int32_t pcg_iters;
  int32_t ls_halvings;
  int32_t status;               /* 0 ok, 4 newton cap, 5 line search failed */
  double g0_norm;
  double g_norm;
  int32_t n_candidates;
  int32_t bonds_broken;
} orc_scene_stats;

/* Sec. 3.2: per-bond rest data from the current state and per-bond material constants. */
int orc_bond_rest(orc_problem* P, const double* E, const double* nu, const double* bend_twist_scale,
                  const double* shear_scale, const double* break_strain);

/* The Z-order (Morton order) of each scene's particles: positions quantised to 21 bits per axis over the scene's
 * bounding box (largest extent), bits interleaved x, y, z from the lowest, particles sorted by code, ties by
 * index; out[scene_start[s] + k] = index of the k-th particle of scene s. */
void orc_morton_order(const int64_t* scene_start, int n_scenes, const double* pos, int32_t* out);

/* z = M^-1 r of the AMG preconditioner of one scene's system at (p, q) (arguments as orc_system; r, z [6 n_s]). */
int orc_amg_apply(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
                  const double* phat, const double* qhat, const double* r, double* z);

/* The AMG's level-1 operator A_1 = P_0^T A_0 P_0 applied to a coarse vector e [n_agg][6] (aggregates in Z-order):
 * y = A_1 e. Returns n_agg. */
int orc_amg_level1_apply(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
                         const double* phat, const double* qhat, const double* e, double* y);

/* One time step of Alg. 3 for every scene. stats: [n_scenes]. Returns the worst status. */
int orc_step(const orc_config* C, orc_problem* P, orc_scene_stats* stats);

/* Energy, reduced gradient (12) and projected / unprojected reduced Hessian (12x12 row-major) of one
 * intact bond at the given endpoint states. Any output may be NULL. */
void orc_bond_terms(const orc_problem* P, int b, const double pi[3], const double qi[4], const double pj[3],
                    const double qj[4], double* energy, double* grad12, double* hess12, double* hess12_spd);

/* The same for the bond term x -> V_b(w x + (1 - w) x_n) of the variational midpoint form (w = 1/2): the energy
 * and its Euclidean derivatives are taken at the evaluation point (pv, qv), scaled by w and w^2, and reduced at the
 * state's quaternions (qi, qj). orc_bond_terms is the case pv = p, qv = q, w = 1. */
void orc_bond_terms_at(const orc_problem* P, int b, const double pvi[3], const double qvi[4], const double pvj[3],
                       const double qvj[4], const double qi[4], const double qj[4], double w, double* energy,
                       double* grad12, double* hess12, double* hess12_spd);

/* Stresses (sigma, tau) of one bond at the state (p[n][3], q[n][4]) for the stress fracture criterion. */
void orc_bond_stress(const orc_problem* P, int b, const double* p, const double* q, double out[2]);

/* Plain bond energy (stretch, shear, bend-twist parts). */
void orc_bond_energy_parts(const orc_problem* P, int b, const double pi[3], const double qi[4],
                           const double pj[3], const double qj[4], double parts[3]);

/* With integrator = 1 every potential term below is evaluated at the midpoint ((p, q) + (P->p, P->q))/2 of the
 * state and the step's start state held in the problem, its Euclidean derivatives scaled by 1/2 (gradient) and
 * 1/4 (Hessian) and reduced at (p, q); the inertia targets are then zhat.
 *
 * The Newton system of one scene at state (p, q) with inertia targets (phat, qhat) and the contact
 * candidates found at (p, q): objective Phi, reduced gradient g[6n_s], assembled projected diagonal
 * blocks diag[n_s][36], per-bond projected 12x12 Hessians bondH[nb][144] (intact bonds of the scene,
 * NULL allowed), and the number of contact candidates. Kinematic particles are not masked here. */
int orc_system(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
               const double* phat, const double* qhat, double* phi, double* g, double* diag, double* bondH,
               int32_t* n_candidates);

/* The variational midpoint target zhat = xhat - 1/2 M_s^{-1} dt^2 grad V((x_{n-1} + x_n)/2) of one scene (Sec. 3.1,
 * App. C), x_n the problem's state and x_{n-1} = x_n - dt v_n, contact candidates found at phat; zp [n][3], zq
 * [n][4] get xhat outside the scene. Returns the number of contact candidates. */
int orc_zhat(const orc_config* C, const orc_problem* P, int scene, const double* phat, const double* qhat,
             double* zp, double* zq);

/* y = H x for the projected Hessian of orc_system (same arguments), x and y [6 n_s]. */
int orc_matvec(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
               const double* phat, const double* qhat, const double* x, double* y);

/* PCG of Sec. 5.3 on H x = b at the same system (kinematic rows removed), from x = 0, stopping at
 * |r| <= eps_r |b| or max_iter iterations; returns the iteration count. */
int orc_pcg_solve(const orc_config* C, const orc_problem* P, int scene, const double* p, const double* q,
                  const double* phat, const double* qhat, const double* b, double eps_r, int max_iter, double* x);

/* Phi(x1) - Phi(x0) as the line search forms it (term by term, with exact difference identities), and
 * Phi at both states (contact candidates taken at x0). */
double orc_energy_diff(const orc_config* C, const orc_problem* P, int scene, const double* phat, const double* qhat,
                       const double* p0, const double* q0, const double* p1, const double* q1, double* phi0,
                       double* phi1);

/* Retraction of Eq. manifold-update-1/2 followed by normalisation (Sec. 4.1). */
void orc_retract(const double p[3], const double q[4], const double step6[6], double alpha, double p_out[3],
                 double q_out[4]);

/* Block-Jacobi preconditioner of Sec. 5.3 applied to one 6x6 block: z = D^-1 r by a Cholesky factorisation of D
 * (row-major 6x6, symmetric); a block that is not positive definite falls back to z_a = r_a / D_aa (r_a unchanged
 * where D_aa <= 0). Returns 1 when the Cholesky path was taken, 0 for the fallback. */
int orc_precond_apply(const double D[36], const double r[6], double z[6]);

/* Symmetric eigen-clamp by cyclic Jacobi (eigenvalues < 0 set to 0); A is n x n row-major, in place. */
void orc_eig_clamp(int n, double* A);
void orc_eig_sym(int n, const double* A, double* evals, double* evecs);

/* Contact candidates of one scene at (p): unbonded pairs i<j with |p_i-p_j| < r_i+r_j+skin.
 * Returns the count; writes up to cap pairs into pairs[2*k]. Brute force when brute != 0. */
int orc_contact_candidates(const orc_config* C, const orc_problem* P, int scene, const double* p, int32_t* pairs,
                           int cap, int brute);

/* Quaternion algebra of App. A (for identity tests). */
void orc_Ql(const double q[4], double M[16]);
void orc_Qr(const double q[4], double M[16]);
void orc_Gl(const double q[4], double M[12]);
void orc_Gr(const double q[4], double M[12]);
void orc_qmul(const double a[4], const double b[4], double out[4]);
void orc_rotate(const double q[4], const double d0[3], double d[3]);

/* Second-order forward-mode derivative test hook: value, gradient and Hessian of
 * f(x) = sin(x0 x1) + sqrt(x2) / (1 + x0^2) + acos-squared of x3 via the oracle's jet arithmetic. */
void orc_jet_selftest(const double x[4], double* f, double g[4], double H[16]);

#ifdef __cplusplus
}
#endif
#endif
