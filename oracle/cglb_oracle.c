/*
 * FP64 CPU oracle for one time step of the two-component colour-gradient
 * lattice Boltzmann scheme on D3Q27 with the coarse-grained near-contact
 * repulsion (arXiv 2405.14551, Sec. III.B, III.C.1, III.D).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is plain, slow, obviously-correct C in
 * double precision.  It shares no code, header, table or helper with the CUDA
 * path under paper_2405_14551_gb300/csrc.  Only tests/, the smoke check and the
 * bench's cpu_baseline / reference arm may load it.
 *
 * State convention: the oracle stores the PRE-collision populations f_i^k(x,t)
 * of both components ("two population sets", Eq. CGLBE).  One step is
 *   moments -> colour gradient -> near-contact scan -> force, velocity ->
 *   BGK + perturbation + forcing -> recolouring -> streaming / bounce-back.
 *
 * Readings of the paper where it is silent or garbled: lattice order and weights, isotropic gradient stencil, neutral
 * wetting of phi at walls, B_i = w_i(|c_i|^2 - 2/3), omega_bar = 2/(6 nu_bar + 1),
 * Guo forcing, Latva-Kokko f^{eq,0} = w_i rho, the regularised collision as
 * the projection of the non-equilibrium part on Hermite orders 1 and 2, the near-contact scan along the
 * outward normal with lround() steps, F_rep = (A_h/2) grad(phi), halfway
 * bounce-back walls, the sharp droplet initial condition.
 *
 * Parity pins: tests/test_oracle_*.py check this file against closed forms
 * (lattice isotropy, equilibrium moments, the perturbation's stress identity
 * that reproduces Eq. sigmaA, Guo moments), exact invariants (per-component
 * mass), hand-counted near-contact distances, Laplace's law, the Poiseuille
 * parabola and the non-coalescence control.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 27
#define NFIELD 14 /* phi, rho, ux, uy, uz, rhoA, rhoB, Frx, Fry, Frz, h, gx, gy, gz */

/* ------------------------------------------------------------------------ */
/* D3Q27 lattice, built by loops (Sec. III.B, Fig. lattice_vel).            */
/* Order: rest, 6 faces, 12 edges, 8 corners; lexicographic (z,y,x) within  */
/* each shell.  Weights are products of the 1D weights {2/3, 1/6, 1/6},     */
/* which gives the D3Q27 set with c_s^2 = 1/3.                              */
/* ------------------------------------------------------------------------ */
static int LC[Q][3];
static double LW[Q];
static int LOPP[Q];
static double LB[Q];   /* perturbation weights B_i */
static double LNORM[Q]; /* |c_i| */
static int lattice_ready = 0;

static void lattice_build(void) {
  if (lattice_ready) return;
  int q = 0;
  for (int shell = 0; shell <= 3; ++shell)
    for (int cz = -1; cz <= 1; ++cz)
      for (int cy = -1; cy <= 1; ++cy)
        for (int cx = -1; cx <= 1; ++cx) {
          if (cx * cx + cy * cy + cz * cz != shell) continue;
          LC[q][0] = cx; LC[q][1] = cy; LC[q][2] = cz;
          double w = 1.0;
          int comp[3] = {cx, cy, cz};
          for (int a = 0; a < 3; ++a) w *= (comp[a] == 0) ? (2.0 / 3.0) : (1.0 / 6.0);
          LW[q] = w;
          LNORM[q] = sqrt((double)shell);
          /* Reading of the isotropy constraints on B_i (Sec. III.C.1):
             B_i = w_i (|c_i|^2 - 2/3) gives sum B = 1/3, sum B c = 0 and
             sum B c c = I/3. */
          LB[q] = w * ((double)shell - 2.0 / 3.0);
          ++q;
        }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j)
      if (LC[j][0] == -LC[i][0] && LC[j][1] == -LC[i][1] && LC[j][2] == -LC[i][2]) LOPP[i] = j;
  lattice_ready = 1;
}

/* Canonical external direction index used to exchange populations with other
 * programs: (cx+1) + 3(cy+1) + 9(cz+1). */
static int canon_index(int i) { return (LC[i][0] + 1) + 3 * (LC[i][1] + 1) + 9 * (LC[i][2] + 1); }

void orc_lattice(int32_t c[Q][3], double w[Q], int32_t opp[Q], double B[Q]) {
  lattice_build();
  for (int i = 0; i < Q; ++i) {
    for (int a = 0; a < 3; ++a) c[i][a] = LC[i][a];
    w[i] = LW[i];
    opp[i] = LOPP[i];
    B[i] = LB[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Parameters (Sec. III.C.1 and the near-contact paragraph).                */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t nx, ny, nz;
  uint32_t walls; /* bit0: x, bit1: y, bit2: z -> solid layers at 0 and n-1 */
  double tau_a, tau_b;
  double A_a, A_b;
  double beta;
  double A_h, h_min, h_max;
  double phi_I;
  double g[3];
  int32_t g_mode; /* 0 none, 1 rho*g, 2 s(z)*rhoA*g (mirror-opposite halves) */
  int32_t collision; /* 0 BGK, 1 regularised (non-equilibrium projected on Hermite orders 1 and 2) */
  int32_t model;     /* 0 colour gradient, 1 Shan-Chen pseudo-potential (Sec. III.C.3) */
  double G;          /* Shan-Chen coupling G_AB = G_BA (G_AA = G_BB = 0) */
  double psi0;       /* rho_0 of the pseudo-potential psi(rho) = rho_0 (1 - exp(-rho/rho_0)) */
} orc_params;

#define GRAD_EPS 1e-12
#define NORMAL_FLOOR 1e-4
/* Near-contact scan: a node with |grad phi| below NC_GRAD_MIN has no defined
   normal (e.g. the stagnation point midway between two droplets) and is
   neither a scan origin nor a target; normals count as antiparallel when
   their cosine is below -NC_COS_TOL, so that exact ties break the same way in
   every precision. */
#define NC_GRAD_MIN 1e-2
#define NC_COS_TOL 1e-6

/* ------------------------------------------------------------------------ */
/* Per-node building blocks.                                                */
/* ------------------------------------------------------------------------ */

/* Second-order equilibrium, Eq. disteq, with c_s^2 = 1/3. */
void orc_feq(double rho, const double u[3], double out[Q]) {
  lattice_build();
  const double cs2 = 1.0 / 3.0;
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    double cu = LC[i][0] * u[0] + LC[i][1] * u[1] + LC[i][2] * u[2];
    /* (c c - cs2 I):u u = (c.u)^2 - cs2 |u|^2 */
    out[i] = LW[i] * rho * (1.0 + cu / cs2 + (cu * cu - cs2 * uu) / (2.0 * cs2 * cs2));
  }
}

/* Surface-tension perturbation summed over both components (Sec. III.C.1):
 * sum_k (A_k/2)|grad phi| [ w_i (c_i.grad phi)^2/|grad phi|^2 - B_i ]. */
void orc_omega2(double A_a, double A_b, const double grad[3], double out[Q]) {
  lattice_build();
  double g = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
  if (g < GRAD_EPS) {
    for (int i = 0; i < Q; ++i) out[i] = 0.0;
    return;
  }
  for (int i = 0; i < Q; ++i) {
    double cg = LC[i][0] * grad[0] + LC[i][1] * grad[1] + LC[i][2] * grad[2];
    out[i] = 0.5 * (A_a + A_b) * g * (LW[i] * cg * cg / (g * g) - LB[i]);
  }
}

/* Guo forcing source (reading of the forcing term, Sec. III.C.1 near-contact
 * paragraph "forcing contribution"):
 * S_i = (1 - 1/(2 tau)) w_i [ (c_i - u)/cs2 + (c_i.u) c_i / cs2^2 ] . F  */
void orc_guo(double tau, const double u[3], const double F[3], double out[Q]) {
  lattice_build();
  const double cs2 = 1.0 / 3.0;
  double pref = 1.0 - 1.0 / (2.0 * tau);
  for (int i = 0; i < Q; ++i) {
    double cu = LC[i][0] * u[0] + LC[i][1] * u[1] + LC[i][2] * u[2];
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s += ((LC[i][a] - u[a]) / cs2 + cu * LC[i][a] / (cs2 * cs2)) * F[a];
    out[i] = pref * LW[i] * s;
  }
}

/* Mixture relaxation time: harmonic kinematic viscosity (Eq. sigmaA and the
 * sentence after it), nu_k = cs2 (tau_k - 1/2), omega_bar = 1/tau_bar =
 * 2/(6 nu_bar + 1).  Equal taus return tau itself. */
double orc_tau_bar(double tau_a, double tau_b, double rhoA, double rhoB) {
  if (tau_a == tau_b) return tau_a;
  double rho = rhoA + rhoB;
  double nu_a = (tau_a - 0.5) / 3.0, nu_b = (tau_b - 0.5) / 3.0;
  double inv_nu = (rhoA / rho) / nu_a + (rhoB / rho) / nu_b;
  double nu = 1.0 / inv_nu;
  return 3.0 * nu + 0.5;
}

/* Regularised non-equilibrium part (the regularised colour-gradient collision
 * that Sec. III.C.1 cites for filtering the non-hydrodynamic "ghost" modes;
 * the paper gives no formula, the reading is the Hermite projection of the
 * regularised LB method): the non-equilibrium part fneq_i = f_i - feq_i of the
 * total is replaced by its projection on the Hermite polynomials of orders 1
 * and 2,
 *   fneq_reg_i = w_i [ c_i.J / cs2 + (c_i c_i - cs2 I) : Pi / (2 cs2^2) ],
 *   J = sum_i c_i fneq_i,   Pi = sum_i c_i c_i fneq_i,
 * which keeps the moments of orders 0, 1 and 2 of fneq (J = -F/2 with the
 * half-force velocity shift) and removes every higher-order part. */
void orc_regularise(const double f[Q], const double feq[Q], double out[Q]) {
  lattice_build();
  const double cs2 = 1.0 / 3.0;
  double J[3] = {0, 0, 0}, Pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int i = 0; i < Q; ++i) {
    double d = f[i] - feq[i];
    for (int a = 0; a < 3; ++a) {
      J[a] += LC[i][a] * d;
      for (int b = 0; b < 3; ++b) Pi[a][b] += LC[i][a] * LC[i][b] * d;
    }
  }
  for (int i = 0; i < Q; ++i) {
    double cj = 0.0, qp = 0.0;
    for (int a = 0; a < 3; ++a) {
      cj += LC[i][a] * J[a];
      for (int b = 0; b < 3; ++b) qp += (LC[i][a] * LC[i][b] - (a == b ? cs2 : 0.0)) * Pi[a][b];
    }
    out[i] = LW[i] * (cj / cs2 + qp / (2.0 * cs2 * cs2));
  }
}

/* Latva-Kokko recolouring, Eqs. ome3_1 / ome3_2, with f^{eq,0}_i = w_i rho and
 * cos(theta_i) = c_i.n/|c_i| (0 for the rest direction). */
void orc_recolour(double beta, double rhoA, double rhoB, const double fstar[Q], const double grad[3],
                  double outA[Q], double outB[Q]) {
  lattice_build();
  double rho = rhoA + rhoB;
  double g = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
  /* Reading: where |grad phi| < NORMAL_FLOOR the direction of grad phi is set
     by round-off, not by an interface; the normal is taken as
     grad phi / max(|grad phi|, NORMAL_FLOOR) so that the segregation term
     fades out continuously there.  At every interface |grad phi| is orders of
     magnitude above the floor and the term is exactly Eq. ome3_1. */
  double gn = g > NORMAL_FLOOR ? g : NORMAL_FLOOR;
  for (int i = 0; i < Q; ++i) {
    double cosv = 0.0;
    if (i != 0) {
      double cg = LC[i][0] * grad[0] + LC[i][1] * grad[1] + LC[i][2] * grad[2];
      cosv = cg / (gn * LNORM[i]);
    }
    double feq0 = LW[i] * rho;
    double seg = beta * rhoA * rhoB / (rho * rho) * cosv * feq0;
    outA[i] = rhoA / rho * fstar[i] + seg;
    outB[i] = rhoB / rho * fstar[i] - seg;
  }
}

/* One node's collision: moments, velocity with the half-force shift, BGK on
 * the total, perturbation, forcing, recolouring.  F is the total force
 * (near-contact + body).  u_out (nullable) receives u = (j + F/2)/rho. */
void orc_node_collide(const orc_params* p, const double fA[Q], const double fB[Q], const double grad[3],
                      const double F[3], double outA[Q], double outB[Q], double u_out[3]) {
  lattice_build();
  double rhoA = 0, rhoB = 0, j[3] = {0, 0, 0};
  double f[Q];
  for (int i = 0; i < Q; ++i) {
    rhoA += fA[i];
    rhoB += fB[i];
    f[i] = fA[i] + fB[i];
    for (int a = 0; a < 3; ++a) j[a] += f[i] * LC[i][a];
  }
  double rho = rhoA + rhoB;
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
  if (u_out)
    for (int a = 0; a < 3; ++a) u_out[a] = u[a];
  double tau = orc_tau_bar(p->tau_a, p->tau_b, rhoA, rhoB);
  double feq[Q], om2[Q], S[Q], fstar[Q];
  orc_feq(rho, u, feq);
  orc_omega2(p->A_a, p->A_b, grad, om2);
  orc_guo(tau, u, F, S);
  if (p->collision == 1) {
    /* regularised: f* = feq + (1 - 1/tau) fneq_reg + Omega2 + S */
    double fr[Q];
    orc_regularise(f, feq, fr);
    for (int i = 0; i < Q; ++i) fstar[i] = feq[i] + (1.0 - 1.0 / tau) * fr[i] + om2[i] + S[i];
  } else {
    for (int i = 0; i < Q; ++i) fstar[i] = f[i] + (feq[i] - f[i]) / tau + om2[i] + S[i];
  }
  orc_recolour(p->beta, rhoA, rhoB, fstar, grad, outA, outB);
}

/* Shan-Chen multicomponent model (Sec. III.C.3, lattice pseudo-potential
 * approach).  Pseudo-potential of a component, Shan and Chen's choice as the
 * paper states it: psi(rho) = rho_0 (1 - exp(-rho/rho_0)). */
double orc_sc_psi(double rho, double psi0) { return psi0 * (1.0 - exp(-rho / psi0)); }

/* One node's Shan-Chen collision: each component relaxes by BGK with its own
 * tau_k towards its own equilibrium f^eq(rho_k, u') at the common velocity
 * of Shan and Chen's scheme, weighted by 1/tau_k and shifted by half the
 * force, u' = sum_k (j_k + F_k/2)/tau_k / sum_k rho_k/tau_k, and receives the
 * Guo source of its own force F_k (reading: the forcing term of the
 * colour-gradient path applied per component).  With this u' the collision
 * adds exactly F_A + F_B to the total momentum for any tau_A, tau_B; for
 * equal taus u' = (j + F/2)/rho.  FA, FB include the body forces.  u_out
 * (nullable) receives u'. */
void orc_node_collide_sc(const orc_params* p, const double fA[Q], const double fB[Q], const double FA[3],
                         const double FB[3], double outA[Q], double outB[Q], double u_out[3]) {
  lattice_build();
  double rhoA = 0, rhoB = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < Q; ++i) {
    rhoA += fA[i];
    rhoB += fB[i];
    for (int a = 0; a < 3; ++a) j[a] += (fA[i] + fB[i]) * LC[i][a];
  }
  double jA[3] = {0, 0, 0}, u[3];
  for (int i = 0; i < Q; ++i)
    for (int a = 0; a < 3; ++a) jA[a] += fA[i] * LC[i][a];
  const double wa = 1.0 / p->tau_a, wb = 1.0 / p->tau_b;
  for (int a = 0; a < 3; ++a)
    u[a] = (wa * (jA[a] + 0.5 * FA[a]) + wb * (j[a] - jA[a] + 0.5 * FB[a])) / (wa * rhoA + wb * rhoB);
  if (u_out)
    for (int a = 0; a < 3; ++a) u_out[a] = u[a];
  double feqA[Q], feqB[Q], SA[Q], SB[Q];
  orc_feq(rhoA, u, feqA);
  orc_feq(rhoB, u, feqB);
  orc_guo(p->tau_a, u, FA, SA);
  orc_guo(p->tau_b, u, FB, SB);
  for (int i = 0; i < Q; ++i) {
    outA[i] = fA[i] + (feqA[i] - fA[i]) / p->tau_a + SA[i];
    outB[i] = fB[i] + (feqB[i] - fB[i]) / p->tau_b + SB[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Whole-lattice simulation.                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
  orc_params p;
  int64_t N;
  double* f[2]; /* [comp] -> [Q][N] pre-collision populations */
  double* fn[2];
  uint8_t* solid;
  /* per-node work arrays at the current time level */
  double *rhoA, *rhoB, *phi, *jx, *jy, *jz;
  double *gx, *gy, *gz;
  double *frx, *fry, *frz;
  double *psiA, *psiB;           /* Shan-Chen pseudo-potentials */
  double *fax, *fay, *faz;       /* Shan-Chen force on component A (B: total minus A) */
  int32_t* h;
  int64_t t;
} orc_sim;

static inline int64_t nid(const orc_sim* s, int x, int y, int z) {
  return (int64_t)x + (int64_t)s->p.nx * ((int64_t)y + (int64_t)s->p.ny * z);
}

static inline int axis_wall(const orc_sim* s, int a) { return (s->p.walls >> a) & 1u; }

static int is_solid_xyz(const orc_sim* s, int x, int y, int z) {
  int n[3] = {s->p.nx, s->p.ny, s->p.nz};
  int v[3] = {x, y, z};
  for (int a = 0; a < 3; ++a)
    if (axis_wall(s, a) && (v[a] <= 0 || v[a] >= n[a] - 1)) return 1;
  return 0;
}

/* Neighbour coordinate along one axis: periodic wrap on open axes (Sec. III.D,
 * periodic paragraph); on wall axes the raw coordinate is returned and the
 * caller checks for solid / out of range. */
static inline int wrap(int v, int n, int wall) {
  if (wall) return v;
  v %= n;
  if (v < 0) v += n;
  return v;
}

orc_sim* orc_create(const orc_params* p) {
  lattice_build();
  if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return NULL;
  if (p->tau_a <= 0.5 || p->tau_b <= 0.5) return NULL;
  if (p->model == 1 && (p->A_h != 0.0 || p->collision != 0 || !(p->psi0 > 0.0))) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->p = *p;
  s->N = (int64_t)p->nx * p->ny * p->nz;
  for (int k = 0; k < 2; ++k) {
    s->f[k] = (double*)calloc((size_t)Q * s->N, sizeof(double));
    s->fn[k] = (double*)calloc((size_t)Q * s->N, sizeof(double));
  }
  s->solid = (uint8_t*)calloc(s->N, 1);
  double** arrs[] = {&s->rhoA, &s->rhoB, &s->phi, &s->jx, &s->jy, &s->jz, &s->gx,  &s->gy,
                     &s->gz,   &s->frx,  &s->fry, &s->frz, &s->psiA, &s->psiB, &s->fax, &s->fay, &s->faz};
  for (unsigned a = 0; a < sizeof(arrs) / sizeof(arrs[0]); ++a) *arrs[a] = (double*)calloc(s->N, sizeof(double));
  s->h = (int32_t*)calloc(s->N, sizeof(int32_t));
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) s->solid[nid(s, x, y, z)] = (uint8_t)is_solid_xyz(s, x, y, z);
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  for (int k = 0; k < 2; ++k) {
    free(s->f[k]);
    free(s->fn[k]);
  }
  free(s->solid);
  double* arrs[] = {s->rhoA, s->rhoB, s->phi, s->jx, s->jy, s->jz, s->gx, s->gy, s->gz,
                    s->frx,  s->fry,  s->frz, s->psiA, s->psiB, s->fax, s->fay, s->faz};
  for (unsigned a = 0; a < sizeof(arrs) / sizeof(arrs[0]); ++a) free(arrs[a]);
  free(s->h);
  free(s);
}

int64_t orc_time(const orc_sim* s) { return s->t; }

/* Set every fluid node to the component equilibria f_i^k = f^eq(rho_k, u). */
void orc_init_fields(orc_sim* s, const double* phi, const double* rho, const double* u /* [3][N] or NULL */) {
  int64_t N = s->N;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    double fa[Q], fb[Q];
    if (s->solid[n]) {
      for (int i = 0; i < Q; ++i) s->f[0][i * N + n] = s->f[1][i * N + n] = 0.0;
      continue;
    }
    double r = rho ? rho[n] : 1.0;
    double ra = r * (1.0 + phi[n]) / 2.0, rb = r * (1.0 - phi[n]) / 2.0;
    double uu[3] = {0, 0, 0};
    if (u)
      for (int a = 0; a < 3; ++a) uu[a] = u[a * N + n];
    orc_feq(ra, uu, fa);
    orc_feq(rb, uu, fb);
    for (int i = 0; i < Q; ++i) {
      s->f[0][i * N + n] = fa[i];
      s->f[1][i * N + n] = fb[i];
    }
  }
  s->t = 0;
}

/* Droplet initial condition (reading of the initial state): phi = +1 inside
 * any droplet (periodic distance on open axes, union), -1 outside; with
 * width > 0, phi = max_j tanh((R_j - d_j)/width).  rho = 1, u = 0. */
void orc_init_droplets(orc_sim* s, int32_t nd, const double* centres, const double* radii, double width) {
  int64_t N = s->N;
  double* phi = (double*)malloc(sizeof(double) * N);
  int nn[3] = {s->p.nx, s->p.ny, s->p.nz};
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    int v[3] = {(int)(n % nn[0]), (int)((n / nn[0]) % nn[1]), (int)(n / ((int64_t)nn[0] * nn[1]))};
    double best = -1.0;
    for (int d = 0; d < nd; ++d) {
      double d2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        double dx = v[a] - centres[3 * d + a];
        if (!axis_wall(s, a)) {
          dx = fmod(dx, (double)nn[a]);
          if (dx > 0.5 * nn[a]) dx -= nn[a];
          if (dx < -0.5 * nn[a]) dx += nn[a];
        }
        d2 += dx * dx;
      }
      double dist = sqrt(d2);
      double ph;
      if (width > 0.0)
        ph = tanh((radii[d] - dist) / width);
      else
        ph = (dist <= radii[d]) ? 1.0 : -1.0;
      if (ph > best) best = ph;
    }
    phi[n] = best;
  }
  orc_init_fields(s, phi, NULL, NULL);
  free(phi);
}

/* Populations in or out, canonical direction order [comp][9(cz+1)+3(cy+1)+(cx+1)][N]. */
void orc_set_populations(orc_sim* s, const double* fA, const double* fB) {
  int64_t N = s->N;
  for (int i = 0; i < Q; ++i) {
    int ci = canon_index(i);
    memcpy(s->f[0] + (int64_t)i * N, fA + (int64_t)ci * N, sizeof(double) * N);
    memcpy(s->f[1] + (int64_t)i * N, fB + (int64_t)ci * N, sizeof(double) * N);
  }
}

void orc_get_populations(const orc_sim* s, double* fA, double* fB) {
  int64_t N = s->N;
  for (int i = 0; i < Q; ++i) {
    int ci = canon_index(i);
    memcpy(fA + (int64_t)ci * N, s->f[0] + (int64_t)i * N, sizeof(double) * N);
    memcpy(fB + (int64_t)ci * N, s->f[1] + (int64_t)i * N, sizeof(double) * N);
  }
}

void orc_set_time(orc_sim* s, int64_t t) { s->t = t; }

/* Body force density at a node (reading of the body forces of the workloads). */
static void body_force(const orc_sim* s, int z, double rho, double rhoA, double F[3]) {
  F[0] = F[1] = F[2] = 0.0;
  if (s->p.g_mode == 1) {
    for (int a = 0; a < 3; ++a) F[a] = rho * s->p.g[a];
  } else if (s->p.g_mode == 2) {
    int nz = s->p.nz;
    double sg = (z == 0 || 2 * z == nz) ? 0.0 : (2 * z < nz ? 1.0 : -1.0);
    for (int a = 0; a < 3; ++a) F[a] = sg * rhoA * s->p.g[a];
  }
}

/* Pass 1-3 at the current time level: moments (Eqs. eq:rho, eq:u and the
 * component sums of Sec. III.C.1), phase field (Eq. order_param), isotropic
 * colour gradient, and the near-contact distance h and force (Eqs.
 * stress_jump, near_cont_force). */
static void compute_levels(orc_sim* s) {
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const int64_t N = s->N;
  const int wx = axis_wall(s, 0), wy = axis_wall(s, 1), wz = axis_wall(s, 2);

#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    if (s->solid[n]) {
      s->rhoA[n] = s->rhoB[n] = s->phi[n] = s->jx[n] = s->jy[n] = s->jz[n] = 0.0;
      continue;
    }
    double ra = 0, rb = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      double a = s->f[0][i * N + n], b = s->f[1][i * N + n];
      ra += a;
      rb += b;
      for (int d = 0; d < 3; ++d) j[d] += (a + b) * LC[i][d];
    }
    s->rhoA[n] = ra;
    s->rhoB[n] = rb;
    s->phi[n] = (ra - rb) / (ra + rb);
    s->jx[n] = j[0];
    s->jy[n] = j[1];
    s->jz[n] = j[2];
  }

  /* colour gradient: grad phi(x) = (1/cs2) sum_i w_i c_i phi(x + c_i), with a
     solid neighbour contributing phi(x) (neutral wetting reading). */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t n = nid(s, x, y, z);
        if (s->solid[n]) {
          s->gx[n] = s->gy[n] = s->gz[n] = 0.0;
          continue;
        }
        double gr[3] = {0, 0, 0};
        for (int i = 1; i < Q; ++i) {
          int xx = wrap(x + LC[i][0], nx, wx), yy = wrap(y + LC[i][1], ny, wy), zz = wrap(z + LC[i][2], nz, wz);
          int64_t m = nid(s, xx, yy, zz);
          double ph = s->solid[m] ? s->phi[n] : s->phi[m];
          for (int d = 0; d < 3; ++d) gr[d] += LW[i] * LC[i][d] * ph;
        }
        s->gx[n] = 3.0 * gr[0];
        s->gy[n] = 3.0 * gr[1];
        s->gz[n] = 3.0 * gr[2];
      }

  if (s->p.model == 1) {
    /* Shan-Chen force (Sec. III.C.3, discretised on the lattice links):
       F_k(x) = -psi_k(x) sum_{k'} G_{kk'} sum_i w_i psi_{k'}(x + c_i) c_i with
       G_AB = G_BA = G and G_AA = G_BB = 0; a solid neighbour contributes the
       node's own psi (the neutral-wall reading of the colour gradient).
       frx.. hold the total F_A + F_B, fax.. the force on A. */
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
      s->psiA[n] = s->solid[n] ? 0.0 : orc_sc_psi(s->rhoA[n], s->p.psi0);
      s->psiB[n] = s->solid[n] ? 0.0 : orc_sc_psi(s->rhoB[n], s->p.psi0);
    }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          int64_t n = nid(s, x, y, z);
          s->h[n] = 0;
          s->frx[n] = s->fry[n] = s->frz[n] = s->fax[n] = s->fay[n] = s->faz[n] = 0.0;
          if (s->solid[n]) continue;
          double sa[3] = {0, 0, 0}, sb[3] = {0, 0, 0}; /* sum_i w_i psi_k(x + c_i) c_i */
          for (int i = 1; i < Q; ++i) {
            int xx = wrap(x + LC[i][0], nx, wx), yy = wrap(y + LC[i][1], ny, wy), zz = wrap(z + LC[i][2], nz, wz);
            int64_t m = nid(s, xx, yy, zz);
            double pa = s->solid[m] ? s->psiA[n] : s->psiA[m];
            double pb = s->solid[m] ? s->psiB[n] : s->psiB[m];
            for (int d = 0; d < 3; ++d) {
              sa[d] += LW[i] * pa * LC[i][d];
              sb[d] += LW[i] * pb * LC[i][d];
            }
          }
          double fa[3], fb[3];
          for (int d = 0; d < 3; ++d) {
            fa[d] = -s->psiA[n] * s->p.G * sb[d];
            fb[d] = -s->psiB[n] * s->p.G * sa[d];
          }
          s->fax[n] = fa[0];
          s->fay[n] = fa[1];
          s->faz[n] = fa[2];
          s->frx[n] = fa[0] + fb[0];
          s->fry[n] = fa[1] + fb[1];
          s->frz[n] = fa[2] + fb[2];
        }
    return;
  }

  /* near-contact scan: from an interface node x (|phi| < phi_I with a defined
     normal), step along the outward normal n_out = -grad phi/|grad phi| in
     lround(k n_out) increments, k = 1..floor(h_max); the first interface node
     y whose normal is antiparallel to n(x) gives h = k.  The scan stops at
     solids. */
  const int K = (int)floor(s->p.h_max);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t n = nid(s, x, y, z);
        s->h[n] = 0;
        s->frx[n] = s->fry[n] = s->frz[n] = 0.0;
        if (s->solid[n] || s->p.A_h == 0.0) continue;
        double g = sqrt(s->gx[n] * s->gx[n] + s->gy[n] * s->gy[n] + s->gz[n] * s->gz[n]);
        if (!(fabs(s->phi[n]) < s->p.phi_I) || g < NC_GRAD_MIN) continue;
        double no[3] = {-s->gx[n] / g, -s->gy[n] / g, -s->gz[n] / g};
        int hit = 0;
        for (int k = 1; k <= K && !hit; ++k) {
          int v[3] = {x + (int)lround(k * no[0]), y + (int)lround(k * no[1]), z + (int)lround(k * no[2])};
          int nn3[3] = {nx, ny, nz};
          int out = 0;
          for (int a = 0; a < 3; ++a) {
            if (axis_wall(s, a)) {
              if (v[a] <= 0 || v[a] >= nn3[a] - 1) out = 1;
            } else {
              v[a] = wrap(v[a], nn3[a], 0);
            }
          }
          if (out) break; /* reached a wall: no droplet-wall repulsion */
          int64_t m = nid(s, v[0], v[1], v[2]);
          double gm = sqrt(s->gx[m] * s->gx[m] + s->gy[m] * s->gy[m] + s->gz[m] * s->gz[m]);
          if (!(fabs(s->phi[m]) < s->p.phi_I) || gm < NC_GRAD_MIN) continue;
          double dot = s->gx[n] * s->gx[m] + s->gy[n] * s->gy[m] + s->gz[n] * s->gz[m];
          if (dot < -NC_COS_TOL * g * gm) hit = k;
        }
        if (!hit) continue;
        double Ah;
        if ((double)hit <= s->p.h_min)
          Ah = s->p.A_h;
        else if ((double)hit <= s->p.h_max)
          Ah = s->p.A_h * pow(s->p.h_min / (double)hit, 3.0);
        else
          Ah = 0.0;
        s->h[n] = hit;
        /* F_rep = -A_h n_out delta_I with delta_I = |grad phi|/2, i.e. (A_h/2) grad phi */
        s->frx[n] = 0.5 * Ah * s->gx[n];
        s->fry[n] = 0.5 * Ah * s->gy[n];
        s->frz[n] = 0.5 * Ah * s->gz[n];
      }
}

/* Fields at the current time level, [NFIELD][N]:
 * phi, rho, ux, uy, uz, rhoA, rhoB, F_rep (3), h, grad phi (3).  u includes the half force
 * of the total force (near-contact + body).  Solid nodes hold zeros. */
void orc_fields(orc_sim* s, double* out) {
  compute_levels(s);
  const int64_t N = s->N;
  const int nx = s->p.nx, ny = s->p.ny;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    int z = (int)(n / ((int64_t)nx * ny));
    for (int k = 0; k < NFIELD; ++k) out[k * N + n] = 0.0;
    if (s->solid[n]) continue;
    double rho = s->rhoA[n] + s->rhoB[n];
    double F[3];
    body_force(s, z, rho, s->rhoA[n], F);
    F[0] += s->frx[n];
    F[1] += s->fry[n];
    F[2] += s->frz[n];
    out[0 * N + n] = s->phi[n];
    out[1 * N + n] = rho;
    out[2 * N + n] = (s->jx[n] + 0.5 * F[0]) / rho;
    out[3 * N + n] = (s->jy[n] + 0.5 * F[1]) / rho;
    out[4 * N + n] = (s->jz[n] + 0.5 * F[2]) / rho;
    out[5 * N + n] = s->rhoA[n];
    out[6 * N + n] = s->rhoB[n];
    out[7 * N + n] = s->frx[n];
    out[8 * N + n] = s->fry[n];
    out[9 * N + n] = s->frz[n];
    out[10 * N + n] = (double)s->h[n];
    out[11 * N + n] = s->gx[n];
    out[12 * N + n] = s->gy[n];
    out[13 * N + n] = s->gz[n];
  }
}

/* One full step: Eq. CGLBE with the collision split of Sec. III.C.1, then
 * streaming with periodic wrap and halfway bounce-back at solid neighbours
 * (Eq. eq:lbm, Sec. III.D no-slip paragraph read as halfway bounce-back). */
static void step_once(orc_sim* s) {
  compute_levels(s);
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const int64_t N = s->N;
  const int wx = axis_wall(s, 0), wy = axis_wall(s, 1), wz = axis_wall(s, 2);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t n = nid(s, x, y, z);
        if (s->solid[n]) continue;
        double fa[Q], fb[Q], oa[Q], ob[Q];
        for (int i = 0; i < Q; ++i) {
          fa[i] = s->f[0][i * N + n];
          fb[i] = s->f[1][i * N + n];
        }
        double rho = s->rhoA[n] + s->rhoB[n];
        double F[3];
        body_force(s, z, rho, s->rhoA[n], F);
        F[0] += s->frx[n];
        F[1] += s->fry[n];
        F[2] += s->frz[n];
        if (s->p.model == 1) {
          /* the body force acts on each component by its own density (g_mode
             1) or on A only (g_mode 2); the Shan-Chen forces of each component */
          double FA[3], FB[3], bA[3] = {0, 0, 0};
          if (s->p.g_mode == 1)
            for (int a = 0; a < 3; ++a) bA[a] = s->rhoA[n] * s->p.g[a];
          else if (s->p.g_mode == 2)
            body_force(s, z, rho, s->rhoA[n], bA);
          double sf[3] = {s->fax[n], s->fay[n], s->faz[n]}, tf[3] = {s->frx[n], s->fry[n], s->frz[n]};
          for (int a = 0; a < 3; ++a) {
            double body = F[a] - tf[a];  /* total body force of the node */
            FA[a] = sf[a] + bA[a];
            FB[a] = (tf[a] - sf[a]) + (body - bA[a]);
          }
          orc_node_collide_sc(&s->p, fa, fb, FA, FB, oa, ob, NULL);
        } else {
          double grad[3] = {s->gx[n], s->gy[n], s->gz[n]};
          orc_node_collide(&s->p, fa, fb, grad, F, oa, ob, NULL);
        }
        for (int i = 0; i < Q; ++i) {
          int xx = wrap(x + LC[i][0], nx, wx), yy = wrap(y + LC[i][1], ny, wy), zz = wrap(z + LC[i][2], nz, wz);
          int64_t m = nid(s, xx, yy, zz);
          if (s->solid[m]) {
            int o = LOPP[i];
            s->fn[0][o * N + n] = oa[i];
            s->fn[1][o * N + n] = ob[i];
          } else {
            s->fn[0][i * N + m] = oa[i];
            s->fn[1][i * N + m] = ob[i];
          }
        }
      }
  for (int k = 0; k < 2; ++k) {
    double* tmp = s->f[k];
    s->f[k] = s->fn[k];
    s->fn[k] = tmp;
  }
  s->t += 1;
}

void orc_step(orc_sim* s, int64_t nsteps) {
  for (int64_t k = 0; k < nsteps; ++k) step_once(s);
}

/* FP64 global sums over fluid nodes at the current time level:
 * [0] mass A, [1] mass B, [2..4] momentum rho u (with half force),
 * [5] A volume sum (1+phi)/2, [6] near-contact active node count,
 * [7] kinetic energy sum rho|u|^2/2. */
void orc_reduce(orc_sim* s, double out[8]) {
  double* fl = (double*)malloc(sizeof(double) * NFIELD * s->N);
  orc_fields(s, fl);
  const int64_t N = s->N;
  for (int k = 0; k < 8; ++k) out[k] = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    if (s->solid[n]) continue;
    double rho = fl[1 * N + n];
    out[0] += fl[5 * N + n];
    out[1] += fl[6 * N + n];
    out[2] += rho * fl[2 * N + n];
    out[3] += rho * fl[3 * N + n];
    out[4] += rho * fl[4 * N + n];
    out[5] += 0.5 * (1.0 + fl[0 * N + n]);
    out[6] += fl[10 * N + n] > 0.0 ? 1.0 : 0.0;
    out[7] += 0.5 * rho *
              (fl[2 * N + n] * fl[2 * N + n] + fl[3 * N + n] * fl[3 * N + n] + fl[4 * N + n] * fl[4 * N + n]);
  }
  free(fl);
}

/* Laplace readout (extended Young-Laplace relation with pi = 0 for an isolated
 * droplet): dp = cs2 (<rho>_{phi > cut} - <rho>_{phi < -cut}). */
double orc_laplace(orc_sim* s, double cut) {
  double* fl = (double*)malloc(sizeof(double) * NFIELD * s->N);
  orc_fields(s, fl);
  const int64_t N = s->N;
  double si = 0, so = 0;
  int64_t ni = 0, no = 0;
  for (int64_t n = 0; n < N; ++n) {
    if (s->solid[n]) continue;
    double ph = fl[n], r = fl[N + n];
    if (ph > cut) {
      si += r;
      ++ni;
    } else if (ph < -cut) {
      so += r;
      ++no;
    }
  }
  free(fl);
  if (ni == 0 || no == 0) return NAN;
  return (si / ni - so / no) / 3.0;
}

/* Droplet count: connected components of fluid nodes with phi > 0,
 * 6-connected, periodic on open axes (plain flood fill). */
int32_t orc_droplet_count(orc_sim* s) {
  double* fl = (double*)malloc(sizeof(double) * NFIELD * s->N);
  orc_fields(s, fl);
  const int64_t N = s->N;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  uint8_t* seen = (uint8_t*)calloc(N, 1);
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * N);
  int32_t count = 0;
  const int dirs[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  for (int64_t n0 = 0; n0 < N; ++n0) {
    if (seen[n0] || s->solid[n0] || !(fl[n0] > 0.0)) continue;
    ++count;
    int64_t top = 0;
    stack[top++] = n0;
    seen[n0] = 1;
    while (top) {
      int64_t n = stack[--top];
      int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
      for (int d = 0; d < 6; ++d) {
        int v[3] = {x + dirs[d][0], y + dirs[d][1], z + dirs[d][2]};
        int nn3[3] = {nx, ny, nz};
        int ok = 1;
        for (int a = 0; a < 3; ++a) {
          if (axis_wall(s, a)) {
            if (v[a] < 0 || v[a] >= nn3[a]) ok = 0;
          } else {
            v[a] = wrap(v[a], nn3[a], 0);
          }
        }
        if (!ok) continue;
        int64_t m = nid(s, v[0], v[1], v[2]);
        if (seen[m] || s->solid[m] || !(fl[m] > 0.0)) continue;
        seen[m] = 1;
        stack[top++] = m;
      }
    }
  }
  free(stack);
  free(seen);
  free(fl);
  return count;
}

/* Regularised reconstruction (Sec. IV.C, Eqs. distnoneq, eq:llb-pull):
 * f_i = f^eq_i(rho, u) + w_i/(2 cs2^2) (c_i c_i - cs2 I):Pi^neq, with the
 * reading Pi^neq = -rho cs2 tau_bar (grad u + grad u^T), gradients by the
 * isotropic stencil (solid neighbour -> the node's own value), and the colour
 * split f^A = (rhoA/rho) f with rhoA = rho (1+phi)/2.  Sets the oracle state. */
void orc_reconstruct(orc_sim* s, const double* phi, const double* rho, const double* u /* [3][N] */) {
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const int64_t N = s->N;
  const int wx = axis_wall(s, 0), wy = axis_wall(s, 1), wz = axis_wall(s, 2);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t n = nid(s, x, y, z);
        if (s->solid[n]) {
          for (int i = 0; i < Q; ++i) s->f[0][i * N + n] = s->f[1][i * N + n] = 0.0;
          continue;
        }
        double du[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}; /* du[b][a] = d_a u_b */
        for (int i = 1; i < Q; ++i) {
          int xx = wrap(x + LC[i][0], nx, wx), yy = wrap(y + LC[i][1], ny, wy), zz = wrap(z + LC[i][2], nz, wz);
          int64_t m = nid(s, xx, yy, zz);
          int64_t src = s->solid[m] ? n : m;
          for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) du[b][a] += 3.0 * LW[i] * LC[i][a] * u[b * N + src];
        }
        double r = rho[n];
        double ra = r * (1.0 + phi[n]) / 2.0, rb = r * (1.0 - phi[n]) / 2.0;
        double tau = orc_tau_bar(s->p.tau_a, s->p.tau_b, ra, rb);
        double Pi[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) Pi[a][b] = -r * (1.0 / 3.0) * tau * (du[b][a] + du[a][b]);
        double uu[3] = {u[n], u[N + n], u[2 * N + n]};
        double feq[Q];
        orc_feq(r, uu, feq);
        for (int i = 0; i < Q; ++i) {
          double contr = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              contr += (LC[i][a] * LC[i][b] - (a == b ? 1.0 / 3.0 : 0.0)) * Pi[a][b];
          double fi = feq[i] + LW[i] / (2.0 / 9.0) * contr;
          s->f[0][i * N + n] = ra / r * fi;
          s->f[1][i * N + n] = rb / r * fi;
        }
      }
  s->t = 0;
}
