/* Flat entry points of the oracle for the Python test harness (ctypes).  TEST INFRASTRUCTURE ONLY.
 * Field arrays crossing this interface are component-major ([5][N], [15][N]) like the library's. */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

typedef struct orc_solver orc_solver;
orc_solver* orc_solver_new(orc_mesh* M, const orc_params* P, char* err);
const orc_params* orc_solver_params(const orc_solver* S);
void orc_solver_delete(orc_solver* S);
int orc_solver_run(orc_solver* S, int multigrid, int n, double* hist);
int orc_solver_reconstruct(orc_solver* S, double* rc, int mode);
int orc_residual_fine(orc_solver* S, const double* W, const double* G, const double* alpha_prev, double* Res,
                      double* Gnew, double* anew, double* dt_out);
int orc_residual_kfvs(orc_solver* S, int lev, const double* W, double* Res);
void orc_solver_dt_level(orc_solver* S, int l, const double* W, double* dt);
double* orc_solver_W(orc_solver* S);
double* orc_solver_G(orc_solver* S);
double* orc_solver_alpha(orc_solver* S);
int64_t orc_solver_skipped(orc_solver* S);
uint64_t orc_splitmix64(uint64_t x);
uint64_t orc_face_hash(uint64_t nl, uint64_t nr, uint64_t nf);

typedef struct {
  orc_mesh* M;
  orc_solver* S;
} handle;

void* orc_mesh_new(int64_t n_nodes, const double* xyz, int64_t n_cells, const int8_t* ctype, const int64_t* cell_ptr,
                   const int32_t* cell_nodes, int64_t n_bfaces, const int64_t* bface_ptr, const int32_t* bface_nodes,
                   const int32_t* bface_tag, int64_t n_periodic, const int32_t* pairs, char* err) {
  orc_mesh* M = calloc(1, sizeof(orc_mesh));
  if (orc_mesh_build(M, n_nodes, xyz, n_cells, ctype, cell_ptr, cell_nodes, n_bfaces, bface_ptr, bface_nodes, bface_tag,
                     n_periodic, pairs, err)) {
    free(M);
    return NULL;
  }
  return M;
}

void orc_mesh_delete(void* m) {
  if (!m) return;
  orc_mesh_free((orc_mesh*)m);
  free(m);
}

void orc_mesh_counts(void* m, int64_t* out) {
  orc_mesh* M = m;
  out[0] = M->nc;
  out[1] = M->nf;
  out[2] = M->n_int;
  out[3] = M->n_per;
  out[4] = M->n_bnd;
}

void orc_mesh_cells(void* m, double* vol, double* ctr, double* m2) {
  orc_mesh* M = m;
  memcpy(vol, M->vol, sizeof(double) * M->nc);
  memcpy(ctr, M->ctr, sizeof(double) * 3 * M->nc);
  memcpy(m2, M->m2, sizeof(double) * 6 * M->nc);
}

void orc_mesh_coarsening_geometry(void* m, double* vol, double* ctr, double* Sn, double* area) {
  orc_mesh* M = m;
  memcpy(vol, M->cvol, sizeof(double) * M->nc);
  memcpy(ctr, M->cctr, sizeof(double) * 3 * M->nc);
  memcpy(Sn, M->cSn, sizeof(double) * 3 * M->nf);
  memcpy(area, M->carea, sizeof(double) * M->nf);
}

void orc_mesh_faces(void* m, int32_t* fL, int32_t* fR, int32_t* ftag, int32_t* fngp, double* gx, double* gA,
                    double* shift, int32_t* cf, int8_t* cside) {
  orc_mesh* M = m;
  memcpy(fL, M->fL, sizeof(int32_t) * M->nf);
  memcpy(fR, M->fR, sizeof(int32_t) * M->nf);
  memcpy(ftag, M->ftag, sizeof(int32_t) * M->nf);
  memcpy(fngp, M->fngp, sizeof(int32_t) * M->nf);
  memcpy(gx, M->gx, sizeof(double) * 12 * M->nf);
  memcpy(gA, M->gA, sizeof(double) * 12 * M->nf);
  memcpy(shift, M->shift, sizeof(double) * 3 * M->nf);
  memcpy(cf, M->cf, sizeof(int32_t) * 6 * M->nc);
  memcpy(cside, M->cside, 6 * M->nc);
}

void* orc_new(void* mesh, const orc_params* P, char* err) {
  handle* h = calloc(1, sizeof(handle));
  h->M = mesh;
  h->S = orc_solver_new(h->M, P, err);
  if (!h->S) {
    free(h);
    return NULL;
  }
  return h;
}

void orc_delete(void* hp) {
  handle* h = hp;
  if (!h) return;
  orc_solver_delete(h->S);
  free(h);
}

void orc_set_state(void* hp, const double* W, const double* G, const double* alpha) {
  handle* h = hp;
  int64_t n = h->M->nc;
  double *w = orc_solver_W(h->S), *g = orc_solver_G(h->S), *a = orc_solver_alpha(h->S);
  for (int64_t i = 0; i < n; ++i) {
    for (int q = 0; q < 5; ++q) w[5 * i + q] = W[q * n + i];
    for (int j = 0; j < 15; ++j) g[15 * i + j] = G ? G[j * n + i] : 0.0;
    a[i] = alpha ? alpha[i] : 1.0;
  }
}

void orc_get_state(void* hp, double* W, double* G, double* alpha) {
  handle* h = hp;
  int64_t n = h->M->nc;
  double *w = orc_solver_W(h->S), *g = orc_solver_G(h->S), *a = orc_solver_alpha(h->S);
  for (int64_t i = 0; i < n; ++i) {
    if (W)
      for (int q = 0; q < 5; ++q) W[q * n + i] = w[5 * i + q];
    if (G)
      for (int j = 0; j < 15; ++j) G[j * n + i] = g[15 * i + j];
    if (alpha) alpha[i] = a[i];
  }
}

/* fine CGKS residual at the current state; no update */
int orc_residual(void* hp, double* res, double* Gnew, double* anew, double* dt, double* norm) {
  handle* h = hp;
  int64_t n = h->M->nc;
  double* r = malloc(sizeof(double) * 5 * n);
  double* g = malloc(sizeof(double) * 15 * n);
  int rc = orc_residual_fine(h->S, orc_solver_W(h->S), orc_solver_G(h->S), orc_solver_alpha(h->S), r, g, anew, dt);
  if (!rc) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (res)
        for (int q = 0; q < 5; ++q) res[q * n + i] = r[5 * i + q];
      if (Gnew)
        for (int j = 0; j < 15; ++j) Gnew[j * n + i] = g[15 * i + j];
      double x = r[5 * i] / h->M->vol[i];
      s += x * x;
    }
    if (norm) *norm = sqrt(s / (double)n);
  }
  free(r);
  free(g);
  return rc;
}

int orc_run(void* hp, int multigrid, int n, double* hist) {
  handle* h = hp;
  return orc_solver_run(h->S, multigrid, n, hist);
}

int64_t orc_skipped(void* hp) { return orc_solver_skipped(((handle*)hp)->S); }

int orc_reconstruct(void* hp, double* rc, int mode) {
  handle* h = hp;
  return orc_solver_reconstruct(h->S, rc, mode);
}

int orc_level_counts(void* hp, int lev, int64_t* out) {
  handle* h = hp;
  if (lev < 0 || lev >= h->M->n_levels) return -1;
  const orc_level* L = &h->M->lev[lev];
  out[0] = L->nc;
  out[1] = L->nf;
  out[2] = L->n_int;
  out[3] = L->n_per;
  return 0;
}

int orc_level_data(void* hp, int lev, int32_t* map, double* vol, double* ctr, int32_t* fL, int32_t* fR, int32_t* ftag,
                   double* Sn, double* area) {
  handle* h = hp;
  if (lev < 0 || lev >= h->M->n_levels) return -1;
  const orc_level* L = &h->M->lev[lev];
  if (map && L->fine2coarse) memcpy(map, L->fine2coarse, sizeof(int32_t) * L->nc_finer);
  if (vol) memcpy(vol, L->vol, sizeof(double) * L->nc);
  if (ctr) memcpy(ctr, L->ctr, sizeof(double) * 3 * L->nc);
  if (fL) memcpy(fL, L->fL, sizeof(int32_t) * L->nf);
  if (fR) memcpy(fR, L->fR, sizeof(int32_t) * L->nf);
  if (ftag) memcpy(ftag, L->ftag, sizeof(int32_t) * L->nf);
  if (Sn) memcpy(Sn, L->Sn, sizeof(double) * 3 * L->nf);
  if (area) memcpy(area, L->area, sizeof(double) * L->nf);
  return 0;
}

int orc_colors(void* hp, int lev, int32_t* colors) {
  handle* h = hp;
  if (lev < 0 || lev >= h->M->n_levels) return -1;
  return orc_level_colors(&h->M->lev[lev], colors);
}

/* one LU-SGS step on level lev: Wout = W + dU for the defect RHS and time steps dt (SoA arrays) */
int orc_lusgs(void* hp, int lev, const double* W, const double* RHS, const double* dt, double* Wout,
              int64_t* skipped) {
  handle* h = hp;
  if (lev < 0 || lev >= h->M->n_levels) return -1;
  const orc_level* L = &h->M->lev[lev];
  int64_t n = L->nc;
  double* w = malloc(sizeof(double) * 5 * n);
  double* r = malloc(sizeof(double) * 5 * n);
  int32_t* col = malloc(sizeof(int32_t) * n);
  for (int64_t i = 0; i < n; ++i)
    for (int q = 0; q < 5; ++q) {
      w[5 * i + q] = W[q * n + i];
      r[5 * i + q] = RHS[q * n + i];
    }
  int ncol = orc_level_colors(L, col);
  *skipped = 0;
  int rc = orc_lusgs_step(orc_solver_params(h->S), L, col, ncol, w, r, dt, skipped);
  if (!rc)
    for (int64_t i = 0; i < n; ++i)
      for (int q = 0; q < 5; ++q) Wout[q * n + i] = w[5 * i + q];
  free(w);
  free(r);
  free(col);
  return rc;
}

int orc_kfvs_residual(void* hp, int lev, const double* W, double* res) {
  handle* h = hp;
  if (lev < 0 || lev >= h->M->n_levels) return -1;
  int64_t n = h->M->lev[lev].nc;
  double* w = malloc(sizeof(double) * 5 * n);
  double* r = malloc(sizeof(double) * 5 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int q = 0; q < 5; ++q) w[5 * i + q] = W[q * n + i];
  int rc = orc_residual_kfvs(h->S, lev, w, r);
  if (!rc)
    for (int64_t i = 0; i < n; ++i)
      for (int q = 0; q < 5; ++q) res[q * n + i] = r[5 * i + q];
  free(w);
  free(r);
  return rc;
}

int orc_level_dt(void* hp, int lev, const double* W, double* dt) {
  handle* h = hp;
  if (lev < 0 || lev >= h->M->n_levels) return -1;
  int64_t n = h->M->lev[lev].nc;
  double* w = malloc(sizeof(double) * 5 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int q = 0; q < 5; ++q) w[5 * i + q] = W[q * n + i];
  orc_solver_dt_level(h->S, lev, w, dt);
  free(w);
  return 0;
}

/* quadrature points and weights of every cell (tensor Gauss rule of n1d points per direction on the
   same iso-parametric maps as the geometry), for exact cell averages of analytic fields */
int orc_mesh_qpoints(void* m, const int8_t* ctype, const int64_t* cell_ptr, const int32_t* cell_nodes,
                     const double* xyz, int n1d, double* pts, double* wts);

/* ---- point-wise pins ------------------------------------------------------------------------ */
static void phys_of(const orc_params* P, orc_phys* ph) {
  memset(ph, 0, sizeof(*ph));
  double g = P->gamma;
  ph->gamma = g;
  ph->K = (5.0 - 3.0 * g) / (g - 1.0);
  ph->prandtl = P->prandtl;
  ph->eps_inviscid = P->eps_inviscid;
  ph->c_press = P->c_press;
  ph->viscous = P->viscous;
  ph->mu = P->viscous ? P->mach / P->reynolds : 0.0;
  ph->sutherland = P->sutherland;
  double a = P->aoa[0] * M_PI / 180.0, b = P->aoa[1] * M_PI / 180.0;
  double u[3] = {P->mach * cos(a) * cos(b), P->mach * sin(b), P->mach * sin(a) * cos(b)};
  ph->Winf[0] = 1.0;
  for (int d = 0; d < 3; ++d) ph->Winf[1 + d] = u[d];
  ph->Winf[4] = 1.0 / g / (g - 1.0) + 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

void orc_pt_moments(const double* gp, double K, int space, double* out) {
  orc_maxw g = {gp[0], gp[1], gp[2], gp[3], gp[4]};
  orc_mom m;
  orc_moments(&g, K, space, &m);
  memcpy(out, m.mu, 9 * sizeof(double));
  memcpy(out + 9, m.mv, 7 * sizeof(double));
  memcpy(out + 16, m.mw, 7 * sizeof(double));
  memcpy(out + 23, m.mxi, 3 * sizeof(double));
}

/* int u^ku v^kv w^kw (s . psi) psi_alpha g over the full (space 0) or half (+1 u > 0, -1 u < 0) space:
 * the building block of every moment of the gas-kinetic flux (s NULL: s . psi := 1) */
double orc_pt_mom_term(const double* gp, double K, int space, int ku, int kv, int kw, const double* s, int alpha) {
  orc_maxw g = {gp[0], gp[1], gp[2], gp[3], gp[4]};
  orc_mom m;
  orc_moments(&g, K, space, &m);
  return orc_mom_term(&m, ku, kv, kw, s, alpha);
}

int orc_pt_slope(const double* gp, double K, const double* dW, double* s) {
  orc_maxw g = {gp[0], gp[1], gp[2], gp[3], gp[4]};
  return orc_slope(&g, K, dW, s);
}

void orc_pt_time(double dt, double tau, double tn, double* q) { orc_time_integrals(dt, tau, tn, q); }

int orc_pt_gks(const orc_params* P, const double* WL, const double* GL, const double* WR, const double* GR,
               const double* n, double dt, double* F, double* Wt) {
  orc_phys ph;
  phys_of(P, &ph);
  return orc_gks_point(&ph, WL, GL, WR, GR, n, dt, F, Wt);
}

int orc_pt_kfvs(const orc_params* P, const double* WL, const double* WR, const double* n, double* F) {
  orc_phys ph;
  phys_of(P, &ph);
  return orc_kfvs_point(&ph, WL, WR, n, F);
}

double orc_pt_cf(const orc_params* P, const double* WL, const double* WR, const double* n) {
  orc_phys ph;
  phys_of(P, &ph);
  return orc_cf_alpha(&ph, WL, WR, n);
}

int orc_pt_ghost(const orc_params* P, int tag, const double* n, const double* W, const double* G, double* Wg,
                 double* Gg) {
  orc_phys ph;
  phys_of(P, &ph);
  return orc_bc_ghost(&ph, tag, n, W, G, Wg, Gg);
}

void orc_pt_frame(const double* n, double* t1, double* t2) { orc_frame(n, t1, t2); }
uint64_t orc_pt_hash(uint64_t nl, uint64_t nr, uint64_t nf) { return orc_face_hash(nl, nr, nf); }
uint64_t orc_pt_splitmix64(uint64_t x) { return orc_splitmix64(x); }

int orc_solver_term_scales(orc_solver* S, double* fabs_out, double* gabs_out);
int orc_term_scales(void* hp, double* fabs_out, double* gabs_out) {
  return orc_solver_term_scales(((handle*)hp)->S, fabs_out, gabs_out);
}
