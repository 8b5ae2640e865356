/*
 * lbm_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * lbm_oracle.h).  Two population arrays, collide-then-stream, every step
 * written out in the order of the paper's formulas, no blocking or fusion.
 *
 * Paper: "Thread-safe lattice Boltzmann for high-performance computing on
 * GPUs", arXiv 2304.06437.  Section 2 (Eq. lbe, Eq. equil, the moment
 * definitions and nu = c_s^2 (1/omega - 1/2)), section 3 (Eq. LBexp, Eq.
 * pushLB, Eq. hermite and the compact order-2 form of fhat^neq), section 5.1
 * (bounce-back walls with a moving lid).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)   /* speed of sound squared, section 2 */
#define QMAX 27

/* ------------------------------------------------------------------------ */
/* Lattice tables, built from the textbook rule: the velocity set is the    */
/* subset of {-1,0,1}^d with |c|^2 <= 2 (D2Q9 keeps all 9, D3Q19 drops the  */
/* 8 corners, D3Q27 keeps all 27); weights depend on |c|^2 only.            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int q, d;
  int c[QMAX][3];
  double w[QMAX];
  int opp[QMAX];
} lattice_t;

static double weight_of(int lattice, int c2) {
  if (lattice == ORC_D2Q9) {
    static const double w[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    return w[c2];
  }
  if (lattice == ORC_D3Q19) {
    static const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    return w[c2];
  }
  {
    static const double w[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    return w[c2];
  }
}

/* ordering key: |c|^2 first, then (cx, cy, cz) lexicographically */
static int vel_less(const int* a, const int* b) {
  int a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  int b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  if (a2 != b2) return a2 < b2;
  for (int k = 0; k < 3; ++k)
    if (a[k] != b[k]) return a[k] < b[k];
  return 0;
}

static int build_lattice(int lattice, lattice_t* L) {
  if (lattice != ORC_D2Q9 && lattice != ORC_D3Q19 && lattice != ORC_D3Q27) return -1;
  L->d = (lattice == ORC_D2Q9) ? 2 : 3;
  L->q = 0;
  int zr = (L->d == 2) ? 0 : 1;
  for (int cx = -1; cx <= 1; ++cx)
    for (int cy = -1; cy <= 1; ++cy)
      for (int cz = -zr; cz <= zr; ++cz) {
        int c2 = cx * cx + cy * cy + cz * cz;
        if (lattice == ORC_D3Q19 && c2 > 2) continue;
        L->c[L->q][0] = cx;
        L->c[L->q][1] = cy;
        L->c[L->q][2] = cz;
        L->q++;
      }
  /* insertion sort into the canonical order */
  for (int i = 1; i < L->q; ++i) {
    int t[3] = {L->c[i][0], L->c[i][1], L->c[i][2]};
    int j = i - 1;
    while (j >= 0 && vel_less(t, L->c[j])) {
      memcpy(L->c[j + 1], L->c[j], sizeof(t));
      --j;
    }
    memcpy(L->c[j + 1], t, sizeof(t));
  }
  for (int a = 0; a < L->q; ++a) {
    int c2 = L->c[a][0] * L->c[a][0] + L->c[a][1] * L->c[a][1] + L->c[a][2] * L->c[a][2];
    L->w[a] = weight_of(lattice, c2);
    L->opp[a] = -1;
    for (int b = 0; b < L->q; ++b)
      if (L->c[b][0] == -L->c[a][0] && L->c[b][1] == -L->c[a][1] && L->c[b][2] == -L->c[a][2])
        L->opp[a] = b;
  }
  return L->q;
}

int orc_lattice(int lattice, int* c, double* w, int* opp) {
  lattice_t L;
  if (build_lattice(lattice, &L) < 0) return -1;
  for (int a = 0; a < L.q; ++a) {
    if (c) { c[3 * a] = L.c[a][0]; c[3 * a + 1] = L.c[a][1]; c[3 * a + 2] = L.c[a][2]; }
    if (w) w[a] = L.w[a];
    if (opp) opp[a] = L.opp[a];
  }
  return L.q;
}

int orc_q(int lattice) { lattice_t L; return build_lattice(lattice, &L); }
int orc_dim(int lattice) {
  lattice_t L;
  if (build_lattice(lattice, &L) < 0) return -1;
  return L.d;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 0;
#endif
}

/* ------------------------------------------------------------------------ */
/* Equilibrium, Eq. equil (He & Luo incompressible form):                  */
/*   f^eq_a = t_a [ rho + rho0 ( c_a.u / cs2 + (c_a c_a - cs2 I):uu / (2 cs2^2) ) ] */
/* ------------------------------------------------------------------------ */
static void equilibrium(const lattice_t* L, double rho0, double rho, const double* u, double* feq) {
  for (int a = 0; a < L->q; ++a) {
    double cu = 0.0;
    for (int al = 0; al < 3; ++al) cu += L->c[a][al] * u[al];
    double quu = 0.0; /* (c c - cs2 I) : u u, over the d lattice axes */
    for (int al = 0; al < L->d; ++al)
      for (int be = 0; be < L->d; ++be)
        quu += (L->c[a][al] * L->c[a][be] - (al == be ? CS2 : 0.0)) * u[al] * u[be];
    feq[a] = L->w[a] * (rho + rho0 * (cu / CS2 + quu / (2.0 * CS2 * CS2)));
  }
}

/* ------------------------------------------------------------------------ */
/* Order-2 Hermite projection, Eq. hermite: fhat_a = t_a sum_n a^n:H^n(c_a) */
/* / (n! cs2^n), with H^0 = 1, H^1 = c, H^2 = c c - cs2 I and the moments    */
/* a^n = sum_b g_b H^n(c_b).  For a non-equilibrium set with a^0 = a^1 = 0  */
/* this is the compact form t_a (c c - cs2 I):Pi^neq / (2 cs2^2).           */
/* ------------------------------------------------------------------------ */
static void hermite_project(const lattice_t* L, const double* g, double* ghat) {
  const int d = L->d; /* tensor indices run over the d lattice axes only */
  double a0 = 0.0, a1[3] = {0, 0, 0}, a2[3][3] = {{0}};
  for (int b = 0; b < L->q; ++b) {
    a0 += g[b];
    for (int al = 0; al < d; ++al) {
      a1[al] += g[b] * L->c[b][al];
      for (int be = 0; be < d; ++be)
        a2[al][be] += g[b] * (L->c[b][al] * L->c[b][be] - (al == be ? CS2 : 0.0));
    }
  }
  for (int a = 0; a < L->q; ++a) {
    double h1 = 0.0, h2 = 0.0;
    for (int al = 0; al < d; ++al) {
      h1 += a1[al] * L->c[a][al];
      for (int be = 0; be < d; ++be)
        h2 += a2[al][be] * (L->c[a][al] * L->c[a][be] - (al == be ? CS2 : 0.0));
    }
    ghat[a] = L->w[a] * (a0 + h1 / CS2 + h2 / (2.0 * CS2 * CS2));
  }
}

int orc_project_neq(int lattice, const double* g, double* ghat) {
  lattice_t L;
  if (build_lattice(lattice, &L) < 0) return -1;
  hermite_project(&L, g, ghat);
  return 0;
}

int orc_equilibrium(const orc_cfg* cfg, double rho, const double* u, double* feq) {
  lattice_t L;
  if (!cfg || build_lattice(cfg->lattice, &L) < 0) return -1;
  double u3[3] = {u[0], u[1], L.d == 3 ? u[2] : 0.0};
  equilibrium(&L, cfg->rho0, rho, u3, feq);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One node's regularized collision.                                        */
/*  1. rho = sum f, j = sum f c                        (moment definitions)  */
/*  2. u = (j + F/2) / rho0   -- reading: the He-Luo equilibrium carries     */
/*     rho0 u as its momentum, so u = j/rho0 keeps the collision exactly     */
/*     momentum conserving; the F/2 shift is the usual second-order forcing. */
/*  3. f^neq = f - f^eq(rho, u), Pi^neq = sum f^neq c c                      */
/*  4. fhat^neq = order-2 Hermite projection of f^neq         (Eq. hermite)  */
/*  5. f* = f^eq + (1 - omega) fhat^neq + S                   (Eq. LBexp)    */
/*     S_a = (1 - omega/2) t_a [ c.F/cs2 + (c c - cs2 I):(u F + F u)/(2 cs2^2) ] */
/*     -- reading of the body-force term the paper mentions without a        */
/*     formula; S = 0 when F = 0, which leaves Eq. LBexp unchanged.          */
/* ------------------------------------------------------------------------ */
static void collide(const lattice_t* L, const orc_cfg* cfg, const double* f, double* fpc,
                    double* pineq_out) {
  const double omega = 1.0 / cfg->tau;
  const double* F = cfg->force;
  double rho = 0.0, j[3] = {0, 0, 0};
  for (int a = 0; a < L->q; ++a) {
    rho += f[a];
    for (int al = 0; al < 3; ++al) j[al] += f[a] * L->c[a][al];
  }
  double u[3];
  for (int al = 0; al < 3; ++al) u[al] = (j[al] + 0.5 * F[al]) / cfg->rho0;

  double feq[QMAX], fneq[QMAX], fhat[QMAX];
  equilibrium(L, cfg->rho0, rho, u, feq);
  for (int a = 0; a < L->q; ++a) fneq[a] = f[a] - feq[a];

  if (pineq_out) {
    double P[3][3] = {{0}};
    for (int a = 0; a < L->q; ++a)
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) P[al][be] += fneq[a] * L->c[a][al] * L->c[a][be];
    if (L->d == 2) {
      pineq_out[0] = P[0][0]; pineq_out[1] = P[1][1]; pineq_out[2] = P[0][1];
    } else {
      pineq_out[0] = P[0][0]; pineq_out[1] = P[1][1]; pineq_out[2] = P[2][2];
      pineq_out[3] = P[0][1]; pineq_out[4] = P[0][2]; pineq_out[5] = P[1][2];
    }
  }

  hermite_project(L, fneq, fhat);

  for (int a = 0; a < L->q; ++a) {
    double cF = 0.0, quf = 0.0;
    for (int al = 0; al < L->d; ++al) {
      cF += L->c[a][al] * F[al];
      for (int be = 0; be < L->d; ++be)
        quf += (L->c[a][al] * L->c[a][be] - (al == be ? CS2 : 0.0)) *
               (u[al] * F[be] + F[al] * u[be]);
    }
    double S = (1.0 - 0.5 * omega) * L->w[a] * (cF / CS2 + quf / (2.0 * CS2 * CS2));
    fpc[a] = feq[a] + (1.0 - omega) * fhat[a] + S;
  }
}

static int check_cfg(const orc_cfg* cfg, lattice_t* L) {
  if (!cfg || build_lattice(cfg->lattice, L) < 0) return -1;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return -1;
  if (L->d == 2 && cfg->nz != 1) return -1;
  if (!(cfg->tau > 0.5)) return -1;
  if (!(cfg->rho0 > 0.0)) return -1;
  for (int ax = 0; ax < 3; ++ax) {
    int lo = cfg->face_kind[2 * ax], hi = cfg->face_kind[2 * ax + 1];
    if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return -1;
    if ((lo == ORC_PERIODIC) != (hi == ORC_PERIODIC)) return -1;
  }
  return 0;
}

int orc_collide_node(const orc_cfg* cfg, const double* f, double* fpc, double* pineq_out) {
  lattice_t L;
  if (!cfg || build_lattice(cfg->lattice, &L) < 0) return -1;
  collide(&L, cfg, f, fpc, pineq_out);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Streaming (Eq. pushLB read as a pull): f_a(y, t+1) = f*_a(y - c_a, t).   */
/* Periodic axes wrap.  Reading of the wall rule (section 5.1 names         */
/* bounce-back walls and a moving lid without formulas): halfway bounce-back,*/
/* the wall half a link outside the outermost fluid node, so                */
/*   f_a(y, t+1) = f*_abar(y, t) + 2 t_a rho0 (c_a . u_w) / cs2,             */
/* where u_w is the velocity of the wall the link y -> y - c_a crosses.  A   */
/* link that leaves through several non-periodic faces at once uses a        */
/* stationary wall if any of them is stationary, else the velocity of the    */
/* first crossed face in the order -x,+x,-y,+y,-z,+z.                        */
/* ------------------------------------------------------------------------ */
static void stream(const lattice_t* L, const orc_cfg* cfg, const double* fpc, double* fout) {
  const long nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
  const long N = nx * ny * nz;
  const long n[3] = {nx, ny, nz};
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    long p[3] = {idx % nx, (idx / nx) % ny, idx / (nx * ny)};
    for (int a = 0; a < L->q; ++a) {
      long s[3];
      int out_wall = 0, any_stationary = 0, first_face = -1;
      for (int ax = 0; ax < 3; ++ax) {
        s[ax] = p[ax] - L->c[a][ax];
        if (s[ax] < 0 || s[ax] >= n[ax]) {
          int face = 2 * ax + (s[ax] < 0 ? 0 : 1);
          int kind = cfg->face_kind[face];
          if (kind == ORC_PERIODIC) {
            s[ax] = (s[ax] + n[ax]) % n[ax];
          } else {
            out_wall = 1;
            if (kind == ORC_WALL) any_stationary = 1;
            if (first_face < 0) first_face = face;
          }
        }
      }
      double v;
      if (out_wall) {
        double cu = 0.0;
        if (!any_stationary)
          for (int al = 0; al < 3; ++al) cu += L->c[a][al] * cfg->wall_u[first_face][al];
        v = fpc[(long)L->opp[a] * N + idx] + 2.0 * L->w[a] * cfg->rho0 * cu / CS2;
      } else {
        long sidx = s[0] + nx * (s[1] + ny * s[2]);
        v = fpc[(long)a * N + sidx];
      }
      fout[(long)a * N + idx] = v;
    }
  }
}

int orc_run(const orc_cfg* cfg, double* f, long steps, int nthreads) {
  lattice_t L;
  if (check_cfg(cfg, &L) < 0 || !f || steps < 0) return -1;
#ifdef _OPENMP
  int saved = omp_get_max_threads();
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const long N = (long)cfg->nx * cfg->ny * cfg->nz;
  double* fpc = (double*)malloc(sizeof(double) * (size_t)L.q * (size_t)N);
  if (!fpc) return -2;
  for (long t = 0; t < steps; ++t) {
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < N; ++idx) {
      double fn[QMAX], fc[QMAX];
      for (int a = 0; a < L.q; ++a) fn[a] = f[(long)a * N + idx];
      collide(&L, cfg, fn, fc, NULL);
      for (int a = 0; a < L.q; ++a) fpc[(long)a * N + idx] = fc[a];
    }
    stream(&L, cfg, fpc, f);
  }
  free(fpc);
#ifdef _OPENMP
  omp_set_num_threads(saved);
#endif
  return 0;
}

int orc_moments(const orc_cfg* cfg, const double* f, double* rho, double* u) {
  lattice_t L;
  if (check_cfg(cfg, &L) < 0 || !f) return -1;
  const long N = (long)cfg->nx * cfg->ny * cfg->nz;
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    double r = 0.0, j[3] = {0, 0, 0};
    for (int a = 0; a < L.q; ++a) {
      double fa = f[(long)a * N + idx];
      r += fa;
      for (int al = 0; al < 3; ++al) j[al] += fa * L.c[a][al];
    }
    if (rho) rho[idx] = r;
    if (u)
      for (int al = 0; al < L.d; ++al) u[(long)al * N + idx] = (j[al] + 0.5 * cfg->force[al]) / cfg->rho0;
  }
  return 0;
}

int orc_init(const orc_cfg* cfg, const double* rho, const double* u, const double* pineq, double* f) {
  lattice_t L;
  if (check_cfg(cfg, &L) < 0 || !rho || !u || !f) return -1;
  const long N = (long)cfg->nx * cfg->ny * cfg->nz;
  const int np = (L.d == 2) ? 3 : 6;
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    double uu[3] = {0, 0, 0};
    for (int al = 0; al < L.d; ++al) uu[al] = u[(long)al * N + idx];
    double feq[QMAX];
    equilibrium(&L, cfg->rho0, rho[idx], uu, feq);
    double P[3][3] = {{0}};
    if (pineq) {
      double p[6];
      for (int k = 0; k < np; ++k) p[k] = pineq[(long)k * N + idx];
      if (L.d == 2) {
        P[0][0] = p[0]; P[1][1] = p[1]; P[0][1] = P[1][0] = p[2];
      } else {
        P[0][0] = p[0]; P[1][1] = p[1]; P[2][2] = p[2];
        P[0][1] = P[1][0] = p[3]; P[0][2] = P[2][0] = p[4]; P[1][2] = P[2][1] = p[5];
      }
    }
    for (int a = 0; a < L.q; ++a) {
      double qp = 0.0, cF = 0.0;
      for (int al = 0; al < L.d; ++al) {
        cF += L.c[a][al] * cfg->force[al];
        for (int be = 0; be < L.d; ++be)
          qp += (L.c[a][al] * L.c[a][be] - (al == be ? CS2 : 0.0)) * P[al][be];
      }
      /* stored momentum is rho0 u - F/2 so that the reported u is u */
      f[(long)a * N + idx] = feq[a] + L.w[a] * qp / (2.0 * CS2 * CS2) - L.w[a] * 0.5 * cF / CS2;
    }
  }
  return 0;
}

/* ======================================================================== */
/* Two-component colour-gradient model (paper section 2.1), periodic box.   */
/* Per step, in the paper's order:                                          */
/*  1. rho_R = sum f_R, rho_B = sum f_B, rho = rho_R + rho_B; the total     */
/*     distribution g = f_R + f_B carries j = sum g c; u = j / rho0.        */
/*  2. relaxation of g as in the single-component step (Eq. LBexp with the  */
/*     Hermite-projected f^neq), plus the perturbation                       */
/*       Omega1_a = (9/4) sigma omega |grad phi| [ t_a (c_a.grad phi)^2 /    */
/*                  |grad phi|^2 - B_a ]                                     */
/*     -- reading: the paper prints (c_a.grad phi) without the square, which */
/*     would inject momentum; the squared form (the one of the cited CG     */
/*     models) conserves mass and momentum when sum B = cs2 and sum B c c =  */
/*     cs2 I.  phi = (rho_R - rho_B) / rho; grad phi by the isotropic        */
/*     stencil (1/cs2) sum_a t_a c_a phi(x + c_a).                           */
/*  3. recolouring (Latva-Kokko):                                            */
/*       f_R* = (rho_R/rho) g* + beta (rho_R rho_B / rho) t_a cos(theta_a)   */
/*       f_B* = (rho_B/rho) g* - beta (rho_R rho_B / rho) t_a cos(theta_a)   */
/*     cos(theta_a) = c_a.grad phi / (|c_a| |grad phi|), 0 for the rest      */
/*     vector or a vanishing gradient -- reading: the paper prints + for     */
/*     both colours; the opposite signs keep f_R* + f_B* = g*, and the zero- */
/*     velocity equilibrium is taken per unit density (t_a).                 */
/*  4. each colour streams (pull, periodic wrap).                            */
/* Near-contact interactions (section 2.2), when nci_amp > 0: before the     */
/* collision every node is checked for a thin film of the continuous (blue) */
/* phase between two interfaces, and flagged nodes collide with a body      */
/* force (the forcing term of the single-component step):                  */
/*   flag(y) = 1 if, for some direction a, the node x = y - h c_a is bulk    */
/*   (phi(x) < -1 + eps) and both points sampled from it along the pair of  */
/*   opposite directions, x + h c_a = y and x - h c_a, are not bulk          */
/*   (phi > -1 + eps);                                                       */
/*   F(y) = A rho_R(y) grad phi / |grad phi|  (0 where grad phi = 0).        */
/* -- readings: the paper states the test from the bulk node ("flag the two  */
/* points"); written from the flagged node it is race free.  "Larger than   */
/* phi_bulk" is read as "not bulk" (a bulk minimum of phi would otherwise   */
/* flag noise); the dispersed phase is red (phi > 0), and the force points  */
/* along the interface normal into it, away from the film.  eps, h and A    */
/* are parameters: the paper gives no values.                              */
/* ======================================================================== */

/* perturbation weights B_a by |c|^2 shell (they satisfy sum B = cs2 and
 * sum B c_x^2 = cs2; the remaining freedom as in the D2Q9 / D3Q19 CG models
 * the paper cites) */
static double cg_B_of(int lattice, int c2) {
  if (lattice == ORC_D2Q9) {
    static const double b[3] = {-4.0 / 27.0, 2.0 / 27.0, 5.0 / 108.0};
    return b[c2];
  }
  static const double b[3] = {-2.0 / 9.0, 1.0 / 54.0, 1.0 / 27.0};
  return b[c2];
}

int orc_cg_weights(int lattice, double* B) {
  lattice_t L;
  if (lattice == ORC_D3Q27 || build_lattice(lattice, &L) < 0) return -1;
  for (int a = 0; a < L.q; ++a)
    B[a] = cg_B_of(lattice, L.c[a][0] * L.c[a][0] + L.c[a][1] * L.c[a][1] + L.c[a][2] * L.c[a][2]);
  return L.q;
}

static int cg_check(const orc_cg_cfg* cfg, lattice_t* L) {
  if (!cfg || cfg->lattice == ORC_D3Q27 || build_lattice(cfg->lattice, L) < 0) return -1;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || !(cfg->tau > 0.5) || !(cfg->rho0 > 0.0)) return -1;
  if (L->d == 2 && cfg->nz != 1) return -1;
  return 0;
}

static long cg_wrap(long v, long n) { v %= n; return v < 0 ? v + n : v; }

int orc_cg_gradient(const orc_cg_cfg* cfg, const double* phi, double* grad) {
  lattice_t L;
  if (cg_check(cfg, &L) < 0 || !phi || !grad) return -1;
  const long nx = cfg->nx, ny = cfg->ny, nz = cfg->nz, N = nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    const long x = idx % nx, y = (idx / nx) % ny, z = idx / (nx * ny);
    double gsum[3] = {0, 0, 0};
    for (int a = 0; a < L.q; ++a) {
      const long xn = cg_wrap(x + L.c[a][0], nx), yn = cg_wrap(y + L.c[a][1], ny), zn = cg_wrap(z + L.c[a][2], nz);
      const double p = phi[xn + nx * (yn + ny * zn)];
      for (int al = 0; al < 3; ++al) gsum[al] += L.w[a] * L.c[a][al] * p;
    }
    for (int al = 0; al < L.d; ++al) grad[al * N + idx] = gsum[al] / CS2;
  }
  return 0;
}

int orc_cg_init(const orc_cg_cfg* cfg, const double* rho_r, const double* rho_b, const double* u, double* fr,
                double* fb) {
  lattice_t L;
  if (cg_check(cfg, &L) < 0 || !rho_r || !rho_b || !fr || !fb) return -1;
  const long N = (long)cfg->nx * cfg->ny * cfg->nz;
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    double uu[3] = {0, 0, 0};
    if (u)
      for (int al = 0; al < L.d; ++al) uu[al] = u[al * N + idx];
    const double rho = rho_r[idx] + rho_b[idx];
    double feq[QMAX];
    equilibrium(&L, cfg->rho0, rho, uu, feq);
    for (int a = 0; a < L.q; ++a) {
      fr[(long)a * N + idx] = rho_r[idx] / rho * feq[a];
      fb[(long)a * N + idx] = rho_b[idx] / rho * feq[a];
    }
  }
  return 0;
}

int orc_cg_fields(const orc_cg_cfg* cfg, const double* fr, const double* fb, double* rho_r, double* rho_b,
                  double* u) {
  lattice_t L;
  if (cg_check(cfg, &L) < 0 || !fr || !fb) return -1;
  const long N = (long)cfg->nx * cfg->ny * cfg->nz;
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    double rr = 0.0, rb = 0.0, j[3] = {0, 0, 0};
    for (int a = 0; a < L.q; ++a) {
      const double r = fr[(long)a * N + idx], b = fb[(long)a * N + idx];
      rr += r;
      rb += b;
      for (int al = 0; al < 3; ++al) j[al] += (r + b) * L.c[a][al];
    }
    if (rho_r) rho_r[idx] = rr;
    if (rho_b) rho_b[idx] = rb;
    if (u)
      for (int al = 0; al < L.d; ++al) u[al * N + idx] = j[al] / cfg->rho0;
  }
  return 0;
}

int orc_cg_nci_flags(const orc_cg_cfg* cfg, const double* phi, unsigned char* flags) {
  lattice_t L;
  if (cg_check(cfg, &L) < 0 || !phi || !flags || cfg->nci_h < 1) return -1;
  const long nx = cfg->nx, ny = cfg->ny, nz = cfg->nz, N = nx * ny * nz;
  const long h = cfg->nci_h;
  const double bulk = -1.0 + cfg->nci_eps;
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    const long x = idx % nx, y = (idx / nx) % ny, z = idx / (nx * ny);
    unsigned char fl = 0;
    if (phi[idx] > bulk) {
      for (int a = 1; a < L.q && !fl; ++a) {
        /* the bulk candidate one sampling distance upstream, and the point
         * one further sampling distance beyond it */
        const long x1 = cg_wrap(x - h * L.c[a][0], nx), y1 = cg_wrap(y - h * L.c[a][1], ny),
                   z1 = cg_wrap(z - h * L.c[a][2], nz);
        const long x2 = cg_wrap(x - 2 * h * L.c[a][0], nx), y2 = cg_wrap(y - 2 * h * L.c[a][1], ny),
                   z2 = cg_wrap(z - 2 * h * L.c[a][2], nz);
        if (phi[x1 + nx * (y1 + ny * z1)] < bulk && phi[x2 + nx * (y2 + ny * z2)] > bulk) fl = 1;
      }
    }
    flags[idx] = fl;
  }
  return 0;
}

int orc_cg_run(const orc_cg_cfg* cfg, double* fr, double* fb, long steps, int nthreads) {
  lattice_t L;
  if (cg_check(cfg, &L) < 0 || !fr || !fb || steps < 0) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const long nx = cfg->nx, ny = cfg->ny, nz = cfg->nz, N = nx * ny * nz;
  const int q = L.q, d = L.d;
  const double omega = 1.0 / cfg->tau;
  double B[QMAX];
  for (int a = 0; a < q; ++a)
    B[a] = cg_B_of(cfg->lattice, L.c[a][0] * L.c[a][0] + L.c[a][1] * L.c[a][1] + L.c[a][2] * L.c[a][2]);
  const int nci = cfg->nci_amp != 0.0;
  if (nci && cfg->nci_h < 1) return -1;
  double* phi = (double*)malloc(sizeof(double) * N);
  double* grad = (double*)malloc(sizeof(double) * 3 * N);
  double* pr = (double*)malloc(sizeof(double) * q * N);
  double* pb = (double*)malloc(sizeof(double) * q * N);
  unsigned char* flags = (unsigned char*)calloc((size_t)N, 1);
  if (!phi || !grad || !pr || !pb || !flags) {
    free(phi); free(grad); free(pr); free(pb); free(flags);
    return -2;
  }
  for (long t = 0; t < steps; ++t) {
    /* phase field of the current state, then its gradient */
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < N; ++idx) {
      double rr = 0.0, rb = 0.0;
      for (int a = 0; a < q; ++a) {
        rr += fr[(long)a * N + idx];
        rb += fb[(long)a * N + idx];
      }
      phi[idx] = (rr - rb) / (rr + rb);
    }
    orc_cg_gradient(cfg, phi, grad);
    if (nci) orc_cg_nci_flags(cfg, phi, flags);
    /* collide: relax + perturb the total set, then recolour */
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < N; ++idx) {
      double g[QMAX], gpc[QMAX];
      double rr = 0.0, rb = 0.0;
      for (int a = 0; a < q; ++a) {
        const double r = fr[(long)a * N + idx], b = fb[(long)a * N + idx];
        rr += r;
        rb += b;
        g[a] = r + b;
      }
      const double rho = rr + rb;
      double gv[3] = {0, 0, 0}, g2 = 0.0;
      for (int al = 0; al < d; ++al) {
        gv[al] = grad[al * N + idx];
        g2 += gv[al] * gv[al];
      }
      const double gn = sqrt(g2);
      orc_cfg one = {cfg->lattice, 1, 1, 1, cfg->tau, cfg->rho0, {0, 0, 0}, {0, 0, 0, 0, 0, 0}, {{0}}};
      if (nci && flags[idx] && gn > 0.0)
        for (int al = 0; al < d; ++al) one.force[al] = cfg->nci_amp * rr * gv[al] / gn;
      collide(&L, &one, g, gpc, 0);
      for (int a = 0; a < q; ++a) {
        double cg = 0.0, c2 = 0.0;
        for (int al = 0; al < d; ++al) {
          cg += L.c[a][al] * gv[al];
          c2 += L.c[a][al] * L.c[a][al];
        }
        double pert = 0.0, cosv = 0.0;
        if (gn > 0.0) {
          pert = 2.25 * cfg->sigma * omega * gn * (L.w[a] * cg * cg / g2 - B[a]);
          if (c2 > 0.0) cosv = cg / (sqrt(c2) * gn);
        }
        const double gs = gpc[a] + pert;
        const double rec = cfg->beta * rr * rb / rho * L.w[a] * cosv;
        pr[(long)a * N + idx] = rr / rho * gs + rec;
        pb[(long)a * N + idx] = rb / rho * gs - rec;
      }
    }
    /* stream each colour: pull from x - c_a with periodic wrap */
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < N; ++idx) {
      const long x = idx % nx, y = (idx / nx) % ny, z = idx / (nx * ny);
      for (int a = 0; a < q; ++a) {
        const long xs = cg_wrap(x - L.c[a][0], nx), ys = cg_wrap(y - L.c[a][1], ny), zs = cg_wrap(z - L.c[a][2], nz);
        const long src = xs + nx * (ys + ny * zs);
        fr[(long)a * N + idx] = pr[(long)a * N + src];
        fb[(long)a * N + idx] = pb[(long)a * N + src];
      }
    }
  }
  free(phi); free(grad); free(pr); free(pb); free(flags);
  return 0;
}
