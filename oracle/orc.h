/* CPU oracle for the multigrid compact gas-kinetic scheme (CGKS) of arXiv 2402.02075.
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, slow FP64 code is the reference the CUDA path is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never calls it.  It shares no source with the CUDA path.  Built with
 * -O2 -ffp-contract=off (no FMA contraction, no fast-math).
 *
 * Every function follows the paper's definitions in the order the paper states them; where the
 * paper is silent or garbled the reading used is stated beside the code.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#define ORC_MAXNF 6      /* faces per cell (hexahedron) */
#define ORC_MAXGP 4      /* Gauss points per face (quadrilateral) */

typedef struct {
  double gamma, mach, reynolds, prandtl, aoa[2], cfl_fine, cfl_coarse, eps_inviscid, c_press,
      weno_eps, skew_min, sutherland, correction_relax;
  int32_t n_levels, pre, post, coarse_steps, passes_per_level, viscous, dt_mode, precision;
  int32_t coarse_smoother; /* 0 forward Euler, 1 LU-SGS (Sec. 4.3) */
  int32_t compression_factor; /* 1 the CF of Sec. 3.3, 0 alpha = 1 */
  int32_t prolongation;    /* 0 injection, 1 injection smoothed over face neighbours */
  uint64_t agglo_seed;
} orc_params;

/* one level of the mesh hierarchy as seen by a first-order (KFVS) solver and the coarsening */
typedef struct {
  int64_t nc, nf;         /* cells, faces (interior, then periodic, then boundary) */
  int64_t n_int, n_per;   /* interior non-periodic faces come first, then periodic */
  double *vol, *ctr;      /* [nc], [nc][3] */
  int32_t *fL, *fR;       /* [nf]; fR = -1 on boundary faces */
  int32_t *ftag, *ftagR;  /* interior -1 / periodic side tag of L / boundary BC tag; ftagR: tag of R side */
  double *Sn, *area, *amom, *shift; /* [nf][3] area vector (outward from L), [nf] area,
                                       [nf][3] area-weighted face centre, [nf][3] R->L translation */
  int32_t *c2f_ptr, *c2f;  /* cell -> incident faces (ascending face id) */
  int32_t *fine2coarse;    /* map from the next finer level ([nc_finer]), NULL on the fine level */
  int64_t nc_finer;
} orc_level;

typedef struct {
  /* fine mesh */
  int64_t n_nodes, nc, nf, n_int, n_per, n_bnd;
  int8_t *ctype;                 /* 4 tet, 5 prism, 6 hex, 7 pyramid (orc_nfaces: number of faces) */
  double *vol, *ctr, *m2;        /* [nc], [nc][3], [nc][6] central second-moment averages xx,yy,zz,xy,yz,xz */
  /* geometry of the coarsening (orc_mesh.c canon_face): [nc], [nc][3], [nf][3], [nf], [nf][3] */
  double *cvol, *cctr, *cSn, *carea, *camom;
  int32_t *fL, *fR, *ftag, *ftagR, *fngp;
  double *shift;                 /* [nf][3] */
  double *gx, *gA;               /* [nf][4][3] Gauss points and area vectors dA_k (|dA_k| = weight) */
  int32_t *cf;                   /* [nc][6] face id of each local face */
  int8_t *cside;                 /* [nc][6] 0: the cell is L of that face, 1: the cell is R */
  /* multigrid hierarchy */
  int n_levels;
  orc_level lev[8];
} orc_mesh;

/* linear algebra (orc_linalg.c) */
typedef struct {
  int m, n;
  double V[24 * 9];  /* Householder vectors, column k in V[k*m ...] */
  double tau[9];
  double R[9 * 9];   /* upper triangle, row-major n x n */
} orc_qr;
int orc_qr_factor(int m, int n, const double* A /* column-major m x n */, orc_qr* f);
void orc_qr_qt(const orc_qr* f, double* b);  /* b <- Q^T b, length m */
void orc_qr_q(const orc_qr* f, double* b);   /* b <- Q b,   length m */
int orc_ge_solve(int n, const double* A /* row-major */, const double* b, double* x);

/* gas kinetics (orc_gks.c) */
typedef struct { double rho, U, V, W, lam; } orc_maxw;
typedef struct { double rho, mu[9], mv[7], mw[7], mxi[3]; } orc_mom;
void orc_moments(const orc_maxw* g, double K, int space /* 0 full, +1 u>0, -1 u<0 */, orc_mom* m);
double orc_mom_term(const orc_mom* m, int ku, int kv, int kw, const double* s, int alpha);
int orc_prim_from_cons(const double W[5], double gamma, orc_maxw* g);
void orc_frame(const double n[3], double t1[3], double t2[3]);
void orc_time_integrals(double dt, double tau, double tau_n, double q[5]);
typedef struct {
  double gamma, K, mu, prandtl, eps_inviscid, c_press, sutherland;
  int viscous;
  double Winf[5];
} orc_phys;
/* dynamic viscosity at t = T/T_inf = gamma p / rho: constant mu_inf, or Sutherland's law
   mu_inf t^(3/2) (1 + s)/(t + s) with s = S/T_inf */
double orc_viscosity(const orc_phys* ph, double t);
int orc_gks_point(const orc_phys* ph, const double WL[5], const double GL[15], const double WR[5],
                  const double GR[15], const double n[3], double dt, double F[5], double Wt[5]);
int orc_kfvs_point(const orc_phys* ph, const double WL[5], const double WR[5], const double n[3], double F[5]);
double orc_cf_alpha(const orc_phys* ph, const double WL[5], const double WR[5], const double n[3]);
int orc_bc_ghost(const orc_phys* ph, int tag, const double n[3], const double W[5], const double G[15],
                 double Wg[5], double Gg[15]);
int orc_slope(const orc_maxw* g, double K, const double dW[5], double s[5]);

/* implicit coarse smoother (orc_lusgs.c) */
int orc_level_colors(const orc_level* L, int32_t* color);
int orc_lusgs_step(const orc_params* P, const orc_level* L, const int32_t* color, int ncol, double* W,
                   const double* RHS, const double* dt, int64_t* skipped);

/* mesh (orc_mesh.c) */
int orc_nfaces(int t);
int orc_mesh_build(orc_mesh* M, int64_t n_nodes, const double* xyz, int64_t n_cells, const int8_t* ctype,
                   const int64_t* cell_ptr, const int32_t* cell_nodes, int64_t n_bfaces,
                   const int64_t* bface_ptr, const int32_t* bface_nodes, const int32_t* bface_tag,
                   int64_t n_periodic, const int32_t* periodic_pairs, char* err);
void orc_mesh_free(orc_mesh* M);
void orc_face_centre(const orc_mesh* M, int64_t f, double xc[3], double Sn[3], double* area);

#endif
