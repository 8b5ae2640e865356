/*
 * lbm_oracle.h -- plain FP64 CPU oracle for the regularized lattice Boltzmann
 * step of "Thread-safe lattice Boltzmann for high-performance computing on
 * GPUs" (arXiv 2304.06437).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this code: only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; it keeps its own lattice tables built from the textbook rule.
 *
 * What it computes (paper section 2 and section 3):
 *   state   : f_a(x, t), the post-streaming, pre-collision populations;
 *   collide : f*_a = f^eq_a + (1 - omega) * fhat^neq_a + S_a      (Eq. LBexp,
 *             with f^neq replaced by its order-2 Hermite projection, Eq. hermite)
 *   stream  : f_a(x, t+1) = f*_a(x - c_a, t), periodic wrap or halfway
 *             bounce-back at walls                                  (Eq. pushLB,
 *             written as a pull)
 * Readings of points the paper leaves open (the incompressible velocity
 * u = (j + F/2)/rho0, the forcing term, the wall rule) are stated beside the
 * function that implements them.
 *
 * Layout: every field is structure-of-arrays, f[a][N] with node index
 * idx = x + nx*(y + ny*z); vectors u[d][N]; a symmetric tensor is stored as
 * [3][N] in 2D (xx, yy, xy) and [6][N] in 3D (xx, yy, zz, xy, xz, yz).
 * Velocity order ("canonical"): rest first, then by |c|^2, then
 * lexicographically on (cx, cy, cz) with -1 < 0 < 1.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1, ORC_D3Q27 = 2 };
enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_MOVING_WALL = 2 };

typedef struct {
  int lattice;          /* ORC_D2Q9 / ORC_D3Q19 / ORC_D3Q27 */
  int nx, ny, nz;       /* fluid nodes per axis; nz = 1 for D2Q9 */
  double tau;           /* relaxation time, omega = 1/tau */
  double rho0;          /* reference density of the He-Luo equilibrium */
  double force[3];      /* body force per unit volume (lattice units) */
  int face_kind[6];     /* faces -x,+x,-y,+y,-z,+z: ORC_PERIODIC/WALL/MOVING_WALL */
  double wall_u[6][3];  /* wall velocity of each face (used for MOVING_WALL) */
} orc_cfg;

/* Lattice tables.  c is [q][3] (cz = 0 in 2D), w is [q], opp is [q].
 * Returns q, or -1 for an unknown lattice. */
int orc_lattice(int lattice, int* c, double* w, int* opp);
int orc_q(int lattice);
int orc_dim(int lattice);

/* He-Luo incompressible equilibrium (Eq. equil) for one node. */
int orc_equilibrium(const orc_cfg* cfg, double rho, const double* u, double* feq);

/* Regularized post-collision set of one node (Eq. LBexp + Eq. hermite +
 * forcing reading).  f and fpc are [q].  If pineq_out is not NULL it receives
 * the non-equilibrium momentum flux (3 or 6 components). */
int orc_collide_node(const orc_cfg* cfg, const double* f, double* fpc, double* pineq_out);

/* Order-2 Hermite projection of an arbitrary non-equilibrium set g[q]. */
int orc_project_neq(int lattice, const double* g, double* ghat);

/* Initial populations from moments: f = f^eq(rho, u) + fhat^neq(pineq)
 * (pineq may be NULL for pure equilibrium).  u is the velocity the state
 * should report, so with a force the stored momentum is rho0*u - F/2. */
int orc_init(const orc_cfg* cfg, const double* rho, const double* u,
             const double* pineq, double* f);

/* Advance f (in/out, [q][N]) by `steps` time steps.  nthreads <= 0 uses the
 * OpenMP default.  Returns 0, or a negative value on bad arguments / OOM. */
int orc_run(const orc_cfg* cfg, double* f, long steps, int nthreads);

/* Density and velocity of the stored state: rho = sum f, u = (j + F/2)/rho0. */
int orc_moments(const orc_cfg* cfg, const double* f, double* rho, double* u);

/* Two-component colour-gradient model (section 2.1), periodic box, D2Q9 or
 * D3Q19.  The two colours are stored as f_R, f_B ([q][N] each); see
 * lbm_oracle.c for the step and the readings it takes. */
typedef struct {
  int lattice;          /* ORC_D2Q9 / ORC_D3Q19 */
  int nx, ny, nz;
  double tau, rho0;
  double sigma;         /* surface tension parameter of the perturbation */
  double beta;          /* recolouring parameter (interface width) */
  /* near-contact interactions (section 2.2); nci_amp = 0 switches them off */
  double nci_amp;       /* force amplitude A: F = A rho_R n at flagged nodes */
  double nci_eps;       /* bulk threshold: a node is bulk if phi < -1 + eps */
  int nci_h;            /* sampling distance along the lattice directions */
} orc_cg_cfg;
int orc_cg_weights(int lattice, double* B);  /* perturbation weights B_a; returns q */
int orc_cg_gradient(const orc_cg_cfg* cfg, const double* phi, double* grad);  /* [d][N] */
int orc_cg_init(const orc_cg_cfg* cfg, const double* rho_r, const double* rho_b, const double* u,
                double* fr, double* fb);
int orc_cg_run(const orc_cg_cfg* cfg, double* fr, double* fb, long steps, int nthreads);
int orc_cg_fields(const orc_cg_cfg* cfg, const double* fr, const double* fb, double* rho_r, double* rho_b,
                  double* u);
/* Near-contact flags of a phase field phi[N] (1 = the repulsive force acts
 * on the node in the next collision). */
int orc_cg_nci_flags(const orc_cg_cfg* cfg, const double* phi, unsigned char* flags);

/* Number of OpenMP threads a parallel region would use (0 without OpenMP). */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
