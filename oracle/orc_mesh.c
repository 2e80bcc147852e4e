/* Oracle mesh topology and geometry (Sec. 2.2 of the paper): mixed tet/prism/hex cells with linear
 * (iso-parametric, trilinear/bilinear) elements; 3 Gauss points per triangular face and 4 per
 * quadrilateral face.  TEST INFRASTRUCTURE ONLY.
 *
 * Readings (the paper gives no formulas here):
 *  - triangle rule: barycentric (2/3,1/6,1/6) and permutations, weight 1/3 of the area each;
 *  - quadrilateral rule: 2x2 Gauss-Legendre (+-1/sqrt(3)) on the bilinear map; each Gauss point
 *    carries the area vector dA_k = (x_s x x_t)(s_k,t_k) (weight 1), so the normal is per point and
 *    sum_k dA_k is the exact area vector of the bilinear patch;
 *  - volume moments to second order: hexahedra by 3x3x3 Gauss on the trilinear map, prisms by a
 *    collapsed (Duffy) 3x3x3 Gauss rule, tetrahedra by the closed forms (exact in every case);
 *  - interior faces are oriented from the lower cell id (L) to the higher (R) and ordered by (L, R);
 *    periodic faces follow in pair order (L = owner of the first face of the pair, its geometry is
 *    used, R is moved onto it by shift = mean(nodes a) - mean(nodes b)); boundary faces last, in
 *    boundary-face order.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

static const int FTET[4][4] = {{0, 2, 1, -1}, {0, 1, 3, -1}, {1, 2, 3, -1}, {0, 3, 2, -1}};
static const int FPRI[5][4] = {{0, 2, 1, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
static const int FHEX[6][4] = {{0, 3, 2, 1}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
/* pyramid (type 7): base 0..3 counter-clockwise seen from the apex 4 */
static const int FPYR[5][4] = {{0, 3, 2, 1}, {0, 1, 4, -1}, {1, 2, 4, -1}, {2, 3, 4, -1}, {3, 0, 4, -1}};

/* faces of a cell type: 4 tetrahedron, 5 prism, 6 hexahedron, 7 pyramid (5) */
int orc_nfaces(int t) { return t == 7 ? 5 : t; }

static int local_face(int t, int lf, const int32_t* cn, int32_t out[4]) {
  const int* f = t == 4 ? FTET[lf] : (t == 5 ? FPRI[lf] : (t == 7 ? FPYR[lf] : FHEX[lf]));
  int nv = f[3] < 0 ? 3 : 4;
  for (int i = 0; i < nv; ++i) out[i] = cn[f[i]];
  return nv;
}

typedef struct {
  int32_t key[4];
  int32_t cell, lf;
} cfrec;

static int cmp_key(const int32_t* a, const int32_t* b) {
  for (int i = 0; i < 4; ++i)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}
static int cmp_cfrec(const void* pa, const void* pb) {
  const cfrec* a = pa;
  const cfrec* b = pb;
  int c = cmp_key(a->key, b->key);
  if (c) return c;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  return a->lf < b->lf ? -1 : (a->lf > b->lf);
}
static void make_key(const int32_t* nodes, int nv, int32_t key[4]) {
  for (int i = 0; i < 4; ++i) key[i] = i < nv ? nodes[i] : INT32_MAX;
  for (int i = 1; i < nv; ++i)
    for (int j = i; j > 0 && key[j - 1] > key[j]; --j) {
      int32_t t = key[j];
      key[j] = key[j - 1];
      key[j - 1] = t;
    }
}

typedef struct {
  int32_t L, R, lfL;
} ipair;
static int cmp_ipair(const void* pa, const void* pb) {
  const ipair* a = pa;
  const ipair* b = pb;
  if (a->L != b->L) return a->L < b->L ? -1 : 1;
  return a->R < b->R ? -1 : (a->R > b->R);
}

static void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Gauss points and area vectors of a face given its nodes in outward order */
static void face_gp(const double* P, int nv, double* gx, double* gA) {
  if (nv == 3) {
    double e1[3], e2[3], A[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = P[3 + d] - P[d];
      e2[d] = P[6 + d] - P[d];
    }
    cross(e1, e2, A);
    for (int k = 0; k < 3; ++k) {
      for (int d = 0; d < 3; ++d) {
        gx[3 * k + d] = (2.0 / 3.0) * P[3 * k + d] + (1.0 / 6.0) * P[3 * ((k + 1) % 3) + d] +
                        (1.0 / 6.0) * P[3 * ((k + 2) % 3) + d];
        gA[3 * k + d] = 0.5 * A[d] / 3.0;
      }
    }
    for (int d = 0; d < 3; ++d) gx[9 + d] = gA[9 + d] = 0.0;
  } else {
    const double g = 1.0 / sqrt(3.0);
    const double S[4] = {-g, g, g, -g}, T[4] = {-g, -g, g, g};
    for (int k = 0; k < 4; ++k) {
      double s = S[k], t = T[k];
      double N[4] = {0.25 * (1 - s) * (1 - t), 0.25 * (1 + s) * (1 - t), 0.25 * (1 + s) * (1 + t),
                     0.25 * (1 - s) * (1 + t)};
      double Ns[4] = {-0.25 * (1 - t), 0.25 * (1 - t), 0.25 * (1 + t), -0.25 * (1 + t)};
      double Nt[4] = {-0.25 * (1 - s), -0.25 * (1 + s), 0.25 * (1 + s), 0.25 * (1 - s)};
      double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
      for (int d = 0; d < 3; ++d) {
        gx[3 * k + d] = 0.0;
        for (int i = 0; i < 4; ++i) {
          gx[3 * k + d] += N[i] * P[3 * i + d];
          xs[d] += Ns[i] * P[3 * i + d];
          xt[d] += Nt[i] * P[3 * i + d];
        }
      }
      cross(xs, xt, gA + 3 * k);
    }
  }
}

/* Geometry of the coarsening.  The agglomeration compares a skewness measure with a limit, so its
   inputs are defined by one formula with a fixed order of operations (this file is compiled without
   floating-point contraction): a face of nodes P_0..P_{n-1} (its left cell's local order) has area
   vector 1/2 (P_1 - P_0) x (P_2 - P_0) (triangle) or 1/2 (P_2 - P_0) x (P_3 - P_1) (quadrilateral,
   exact for a bilinear face), centre the node mean and area the length of the area vector; a cell
   has centre the node mean and volume 1/3 sum over its faces (own local order, outward) of
   centre . area vector (the divergence theorem for flat faces). */
static void canon_face(const double* P, int nv, double S[3], double X[3]) {
  double e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = nv == 3 ? P[3 + d] - P[d] : P[6 + d] - P[d];
    e2[d] = nv == 3 ? P[6 + d] - P[d] : P[9 + d] - P[3 + d];
  }
  S[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
  S[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
  S[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
  for (int d = 0; d < 3; ++d) {
    double a = P[d];
    for (int i = 1; i < nv; ++i) a = a + P[3 * i + d];
    X[d] = a / (double)nv;
  }
}

static double det3(const double a[3], const double b[3], const double c[3]) {
  double x[3];
  cross(b, c, x);
  return a[0] * x[0] + a[1] * x[1] + a[2] * x[2];
}

/* volume, centroid and central second-moment averages of one cell */
static void cell_geom(int t, const double* X, double* vol, double c[3], double m2[6]) {
  if (t == 7) { /* pyramid: the hexahedron map with its top face collapsed onto the apex */
    double H[24];
    for (int i = 0; i < 4; ++i)
      for (int d = 0; d < 3; ++d) {
        H[3 * i + d] = X[3 * i + d];
        H[3 * (i + 4) + d] = X[12 + d];
      }
    cell_geom(6, H, vol, c, m2);
    return;
  }
  if (t == 4) {
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = X[3 + d] - X[d];
      e2[d] = X[6 + d] - X[d];
      e3[d] = X[9 + d] - X[d];
    }
    *vol = det3(e1, e2, e3) / 6.0;
    for (int d = 0; d < 3; ++d) c[d] = 0.25 * (X[d] + X[3 + d] + X[6 + d] + X[9 + d]);
    for (int q = 0; q < 6; ++q) m2[q] = 0.0;
    for (int i = 0; i < 4; ++i) {
      double y[3] = {X[3 * i] - c[0], X[3 * i + 1] - c[1], X[3 * i + 2] - c[2]};
      m2[0] += y[0] * y[0];
      m2[1] += y[1] * y[1];
      m2[2] += y[2] * y[2];
      m2[3] += y[0] * y[1];
      m2[4] += y[1] * y[2];
      m2[5] += y[0] * y[2];
    }
    for (int q = 0; q < 6; ++q) m2[q] /= 20.0;
    return;
  }
  /* quadrature points and weights (weights include |det J|) */
  double qx[27][3], qw[27];
  const double g = sqrt(0.6);
  const double p3[3] = {-g, 0.0, g}, w3[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  int nq = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int e = 0; e < 3; ++e) {
        double x[3] = {0, 0, 0}, j1[3] = {0, 0, 0}, j2[3] = {0, 0, 0}, j3[3] = {0, 0, 0}, w;
        if (t == 6) {
          double xi = p3[a], et = p3[b], ze = p3[e];
          static const int sg[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                       {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
          for (int i = 0; i < 8; ++i) {
            double fx = 1 + sg[i][0] * xi, fy = 1 + sg[i][1] * et, fz = 1 + sg[i][2] * ze;
            double N = 0.125 * fx * fy * fz;
            double dNx = 0.125 * sg[i][0] * fy * fz, dNy = 0.125 * fx * sg[i][1] * fz,
                   dNz = 0.125 * fx * fy * sg[i][2];
            for (int d = 0; d < 3; ++d) {
              x[d] += N * X[3 * i + d];
              j1[d] += dNx * X[3 * i + d];
              j2[d] += dNy * X[3 * i + d];
              j3[d] += dNz * X[3 * i + d];
            }
          }
          w = w3[a] * w3[b] * w3[e] * det3(j1, j2, j3);
        } else { /* prism: r = u, s = v (1 - u) on the unit square, zeta in [-1, 1] */
          double u = 0.5 * (1.0 + p3[a]), v = 0.5 * (1.0 + p3[b]), ze = p3[e];
          double r = u, s = v * (1.0 - u);
          double L[3] = {1.0 - r - s, r, s};
          double dLr[3] = {-1.0, 1.0, 0.0}, dLs[3] = {-1.0, 0.0, 1.0};
          for (int i = 0; i < 3; ++i)
            for (int d = 0; d < 3; ++d) {
              double bot = X[3 * i + d], top = X[3 * (i + 3) + d];
              double col = 0.5 * (1.0 - ze) * bot + 0.5 * (1.0 + ze) * top;
              x[d] += L[i] * col;
              j1[d] += dLr[i] * col;
              j2[d] += dLs[i] * col;
              j3[d] += L[i] * 0.5 * (top - bot);
            }
          w = (0.5 * w3[a]) * (0.5 * w3[b]) * (1.0 - u) * w3[e] * det3(j1, j2, j3);
        }
        qx[nq][0] = x[0];
        qx[nq][1] = x[1];
        qx[nq][2] = x[2];
        qw[nq++] = w;
      }
  double V = 0, m[3] = {0, 0, 0};
  for (int q = 0; q < nq; ++q) {
    V += qw[q];
    for (int d = 0; d < 3; ++d) m[d] += qw[q] * qx[q][d];
  }
  *vol = V;
  for (int d = 0; d < 3; ++d) c[d] = m[d] / V;
  for (int q = 0; q < 6; ++q) m2[q] = 0.0;
  for (int q = 0; q < nq; ++q) {
    double y[3] = {qx[q][0] - c[0], qx[q][1] - c[1], qx[q][2] - c[2]};
    m2[0] += qw[q] * y[0] * y[0];
    m2[1] += qw[q] * y[1] * y[1];
    m2[2] += qw[q] * y[2] * y[2];
    m2[3] += qw[q] * y[0] * y[1];
    m2[4] += qw[q] * y[1] * y[2];
    m2[5] += qw[q] * y[0] * y[2];
  }
  for (int q = 0; q < 6; ++q) m2[q] /= V;
}

void orc_face_centre(const orc_mesh* M, int64_t f, double xc[3], double Sn[3], double* area) {
  double a = 0.0;
  for (int d = 0; d < 3; ++d) xc[d] = Sn[d] = 0.0;
  for (int k = 0; k < M->fngp[f]; ++k) {
    const double* A = M->gA + 12 * f + 3 * k;
    const double* x = M->gx + 12 * f + 3 * k;
    double w = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    a += w;
    for (int d = 0; d < 3; ++d) {
      xc[d] += w * x[d];
      Sn[d] += A[d];
    }
  }
  for (int d = 0; d < 3; ++d) xc[d] /= a;
  *area = a;
}

#define FAIL(...)                                 \
  do {                                            \
    if (err) snprintf(err, 256, __VA_ARGS__);     \
    rc = -1;                                      \
    goto done;                                    \
  } while (0)

int orc_mesh_build(orc_mesh* M, int64_t n_nodes, const double* xyz, int64_t n_cells, const int8_t* ctype,
                   const int64_t* cell_ptr, const int32_t* cell_nodes, int64_t n_bfaces,
                   const int64_t* bface_ptr, const int32_t* bface_nodes, const int32_t* bface_tag,
                   int64_t n_periodic, const int32_t* periodic_pairs, char* err) {
  int rc = 0;
  cfrec *recs = NULL, *brecs = NULL;
  ipair* ip = NULL;
  int32_t *bmatch = NULL, *bused = NULL, *bperiodic = NULL;
  memset(M, 0, sizeof(*M));
  M->n_nodes = n_nodes;
  M->nc = n_cells;
  int64_t nrec = 0;
  for (int64_t c = 0; c < n_cells; ++c) {
    int t = ctype[c];
    int64_t cnt = cell_ptr[c + 1] - cell_ptr[c];
    if (!((t == 4 && cnt == 4) || (t == 5 && cnt == 6) || (t == 6 && cnt == 8) || (t == 7 && cnt == 5)))
      FAIL("cell %lld: bad type/node count", (long long)c);
    for (int64_t q = cell_ptr[c]; q < cell_ptr[c + 1]; ++q)
      if (cell_nodes[q] < 0 || cell_nodes[q] >= n_nodes) FAIL("cell %lld: node out of range", (long long)c);
    nrec += orc_nfaces(t);
  }
  recs = malloc(sizeof(cfrec) * (nrec ? nrec : 1));
  {
    int64_t r = 0;
    for (int64_t c = 0; c < n_cells; ++c)
      for (int lf = 0; lf < orc_nfaces(ctype[c]); ++lf) {
        int32_t nodes[4];
        int nv = local_face(ctype[c], lf, cell_nodes + cell_ptr[c], nodes);
        make_key(nodes, nv, recs[r].key);
        recs[r].cell = (int32_t)c;
        recs[r].lf = lf;
        ++r;
      }
  }
  qsort(recs, nrec, sizeof(cfrec), cmp_cfrec);
  /* boundary records */
  brecs = malloc(sizeof(cfrec) * (n_bfaces ? n_bfaces : 1));
  for (int64_t b = 0; b < n_bfaces; ++b) {
    int nv = (int)(bface_ptr[b + 1] - bface_ptr[b]);
    if (nv != 3 && nv != 4) FAIL("boundary face %lld: %d nodes", (long long)b, nv);
    make_key(bface_nodes + bface_ptr[b], nv, brecs[b].key);
    brecs[b].cell = (int32_t)b;
    brecs[b].lf = 0;
  }
  qsort(brecs, n_bfaces, sizeof(cfrec), cmp_cfrec);
  bmatch = malloc(sizeof(int32_t) * 2 * (n_bfaces ? n_bfaces : 1)); /* owner cell, local face */
  for (int64_t b = 0; b < 2 * n_bfaces; ++b) bmatch[b] = -1;
  ip = malloc(sizeof(ipair) * (nrec / 2 + 1));
  int64_t n_int = 0;
  for (int64_t r = 0; r < nrec;) {
    int64_t s = r + 1;
    while (s < nrec && cmp_key(recs[s].key, recs[r].key) == 0) ++s;
    if (s - r == 2) {
      ip[n_int].L = recs[r].cell;
      ip[n_int].R = recs[r + 1].cell;
      ip[n_int].lfL = recs[r].lf;
      if (ip[n_int].L == ip[n_int].R) FAIL("cell %d faces itself", recs[r].cell);
      ++n_int;
    } else if (s - r == 1) {
      /* find the boundary face with this key */
      int64_t lo = 0, hi = n_bfaces - 1, found = -1;
      while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int c = cmp_key(brecs[mid].key, recs[r].key);
        if (c == 0) {
          found = mid;
          break;
        }
        if (c < 0)
          lo = mid + 1;
        else
          hi = mid - 1;
      }
      if (found < 0) FAIL("cell %d local face %d is on no boundary face", recs[r].cell, recs[r].lf);
      int32_t b = brecs[found].cell;
      if (bmatch[2 * b] >= 0) FAIL("boundary face %d matched twice", b);
      bmatch[2 * b] = recs[r].cell;
      bmatch[2 * b + 1] = recs[r].lf;
    } else {
      FAIL("a face is shared by %lld cells", (long long)(s - r));
    }
    r = s;
  }
  for (int64_t b = 0; b < n_bfaces; ++b)
    if (bmatch[2 * b] < 0) FAIL("boundary face %lld matches no cell face", (long long)b);
  qsort(ip, n_int, sizeof(ipair), cmp_ipair);
  for (int64_t i = 1; i < n_int; ++i)
    if (ip[i].L == ip[i - 1].L && ip[i].R == ip[i - 1].R) FAIL("cells %d,%d share two faces", ip[i].L, ip[i].R);
  /* periodic pairs */
  bperiodic = calloc(n_bfaces ? n_bfaces : 1, sizeof(int32_t));
  for (int64_t p = 0; p < n_periodic; ++p) {
    int32_t a = periodic_pairs[2 * p], b = periodic_pairs[2 * p + 1];
    if (a < 0 || b < 0 || a >= n_bfaces || b >= n_bfaces || a == b) FAIL("periodic pair %lld invalid", (long long)p);
    if (bface_tag[a] < 100 || bface_tag[b] < 100) FAIL("periodic pair %lld: tags must be >= 100", (long long)p);
    if (bperiodic[a] || bperiodic[b]) FAIL("periodic pair %lld reuses a face", (long long)p);
    if (bface_ptr[a + 1] - bface_ptr[a] != bface_ptr[b + 1] - bface_ptr[b]) FAIL("periodic pair %lld: shapes differ", (long long)p);
    bperiodic[a] = bperiodic[b] = 1;
  }
  int64_t n_bnd = 0;
  for (int64_t b = 0; b < n_bfaces; ++b) {
    if (bface_tag[b] >= 100 && !bperiodic[b]) FAIL("periodic-tagged boundary face %lld has no pair", (long long)b);
    if (bface_tag[b] < 1 || (bface_tag[b] > 5 && bface_tag[b] < 100)) FAIL("boundary face %lld: unknown tag", (long long)b);
    if (!bperiodic[b]) ++n_bnd;
  }
  M->n_int = n_int;
  M->n_per = n_periodic;
  M->n_bnd = n_bnd;
  M->nf = n_int + n_periodic + n_bnd;
  int64_t nf = M->nf;
  M->ctype = malloc(n_cells);
  memcpy(M->ctype, ctype, n_cells);
  M->vol = malloc(sizeof(double) * n_cells);
  M->ctr = malloc(sizeof(double) * 3 * n_cells);
  M->m2 = malloc(sizeof(double) * 6 * n_cells);
  M->fL = malloc(sizeof(int32_t) * nf);
  M->fR = malloc(sizeof(int32_t) * nf);
  M->ftag = malloc(sizeof(int32_t) * nf);
  M->ftagR = malloc(sizeof(int32_t) * nf);
  M->fngp = malloc(sizeof(int32_t) * nf);
  M->shift = calloc(3 * nf, sizeof(double));
  M->gx = calloc(12 * nf, sizeof(double));
  M->gA = calloc(12 * nf, sizeof(double));
  M->cf = malloc(sizeof(int32_t) * 6 * n_cells);
  M->cside = malloc(6 * n_cells);
  for (int64_t i = 0; i < 6 * n_cells; ++i) {
    M->cf[i] = -1;
    M->cside[i] = 0;
  }
  for (int64_t c = 0; c < n_cells; ++c) {
    double X[24];
    int nn = (int)(cell_ptr[c + 1] - cell_ptr[c]);
    for (int i = 0; i < nn; ++i)
      for (int d = 0; d < 3; ++d) X[3 * i + d] = xyz[3 * (int64_t)cell_nodes[cell_ptr[c] + i] + d];
    cell_geom(ctype[c], X, M->vol + c, M->ctr + 3 * c, M->m2 + 6 * c);
    if (!(M->vol[c] > 0.0)) FAIL("cell %lld has non-positive volume", (long long)c);
  }
  /* helper to fill a face's geometry from (cell, local face) */
#define FACE_GEOM(F, C, LF)                                                      \
  do {                                                                           \
    int32_t nodes_[4];                                                           \
    int nv_ = local_face(ctype[C], LF, cell_nodes + cell_ptr[C], nodes_);        \
    double P_[12];                                                               \
    for (int i_ = 0; i_ < nv_; ++i_)                                             \
      for (int d_ = 0; d_ < 3; ++d_) P_[3 * i_ + d_] = xyz[3 * (int64_t)nodes_[i_] + d_]; \
    face_gp(P_, nv_, M->gx + 12 * (F), M->gA + 12 * (F));                        \
    M->fngp[F] = nv_;                                                            \
  } while (0)
  /* the local face index of cell C that corresponds to a record: found through recs */
  for (int64_t f = 0; f < n_int; ++f) {
    M->fL[f] = ip[f].L;
    M->fR[f] = ip[f].R;
    M->ftag[f] = -1;
    M->ftagR[f] = -1;
    FACE_GEOM(f, ip[f].L, ip[f].lfL);
  }
  /* cell -> face maps for interior faces: walk the records again */
  for (int64_t r = 0; r < nrec;) {
    int64_t s = r + 1;
    while (s < nrec && cmp_key(recs[s].key, recs[r].key) == 0) ++s;
    if (s - r == 2) {
      int32_t L = recs[r].cell, R = recs[r + 1].cell;
      /* binary search (L, R) in ip */
      int64_t lo = 0, hi = n_int - 1, f = -1;
      while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (ip[mid].L == L && ip[mid].R == R) {
          f = mid;
          break;
        }
        if (ip[mid].L < L || (ip[mid].L == L && ip[mid].R < R))
          lo = mid + 1;
        else
          hi = mid - 1;
      }
      M->cf[6 * L + recs[r].lf] = (int32_t)f;
      M->cside[6 * L + recs[r].lf] = 0;
      M->cf[6 * R + recs[r + 1].lf] = (int32_t)f;
      M->cside[6 * R + recs[r + 1].lf] = 1;
    }
    r = s;
  }
  for (int64_t p = 0; p < n_periodic; ++p) {
    int64_t f = n_int + p;
    int32_t a = periodic_pairs[2 * p], b = periodic_pairs[2 * p + 1];
    int32_t ca = bmatch[2 * a], la = bmatch[2 * a + 1], cb = bmatch[2 * b], lb = bmatch[2 * b + 1];
    M->fL[f] = ca;
    M->fR[f] = cb;
    M->ftag[f] = bface_tag[a];
    M->ftagR[f] = bface_tag[b];
    FACE_GEOM(f, ca, la);
    double ma[3] = {0, 0, 0}, mb[3] = {0, 0, 0};
    int nv = (int)(bface_ptr[a + 1] - bface_ptr[a]);
    for (int i = 0; i < nv; ++i)
      for (int d = 0; d < 3; ++d) {
        ma[d] += xyz[3 * (int64_t)bface_nodes[bface_ptr[a] + i] + d];
        mb[d] += xyz[3 * (int64_t)bface_nodes[bface_ptr[b] + i] + d];
      }
    for (int d = 0; d < 3; ++d) M->shift[3 * f + d] = ma[d] / nv - mb[d] / nv;
    M->cf[6 * ca + la] = (int32_t)f;
    M->cside[6 * ca + la] = 0;
    M->cf[6 * cb + lb] = (int32_t)f;
    M->cside[6 * cb + lb] = 1;
  }
  {
    int64_t f = n_int + n_periodic;
    for (int64_t b = 0; b < n_bfaces; ++b) {
      if (bperiodic[b]) continue;
      int32_t c = bmatch[2 * b], lf = bmatch[2 * b + 1];
      M->fL[f] = c;
      M->fR[f] = -1;
      M->ftag[f] = bface_tag[b];
      M->ftagR[f] = -1;
      FACE_GEOM(f, c, lf);
      M->cf[6 * c + lf] = (int32_t)f;
      M->cside[6 * c + lf] = 0;
      ++f;
    }
  }
  for (int64_t c = 0; c < n_cells; ++c)
    for (int lf = 0; lf < orc_nfaces(ctype[c]); ++lf)
      if (M->cf[6 * c + lf] < 0) FAIL("cell %lld local face %d unassigned", (long long)c, lf);
  /* geometry of the coarsening */
  M->cvol = malloc(sizeof(double) * n_cells);
  M->cctr = malloc(sizeof(double) * 3 * n_cells);
  M->cSn = malloc(sizeof(double) * 3 * (nf ? nf : 1));
  M->carea = malloc(sizeof(double) * (nf ? nf : 1));
  M->camom = malloc(sizeof(double) * 3 * (nf ? nf : 1));
  for (int64_t c = 0; c < n_cells; ++c) {
    int nn = (int)(cell_ptr[c + 1] - cell_ptr[c]);
    for (int d = 0; d < 3; ++d) {
      double a = xyz[3 * (int64_t)cell_nodes[cell_ptr[c]] + d];
      for (int i = 1; i < nn; ++i) a = a + xyz[3 * (int64_t)cell_nodes[cell_ptr[c] + i] + d];
      M->cctr[3 * c + d] = a / (double)nn;
    }
    double v = 0.0;
    for (int lf = 0; lf < orc_nfaces(ctype[c]); ++lf) {
      int32_t nodes[4];
      int nv = local_face(ctype[c], lf, cell_nodes + cell_ptr[c], nodes);
      double P[12], S[3], X[3];
      for (int i = 0; i < nv; ++i)
        for (int d = 0; d < 3; ++d) P[3 * i + d] = xyz[3 * (int64_t)nodes[i] + d];
      canon_face(P, nv, S, X);
      v = v + (X[0] * S[0] + X[1] * S[1] + X[2] * S[2]);
      if (M->cside[6 * c + lf] == 0) { /* the face seen from its left cell */
        int32_t f = M->cf[6 * c + lf];
        double a = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
        M->carea[f] = a;
        for (int d = 0; d < 3; ++d) {
          M->cSn[3 * f + d] = S[d];
          M->camom[3 * f + d] = a * X[d];
        }
      }
    }
    M->cvol[c] = v / 3.0;
  }
done:
  free(recs);
  free(brecs);
  free(ip);
  free(bmatch);
  free(bused);
  free(bperiodic);
  if (rc) orc_mesh_free(M);
  return rc;
}

static void level_free(orc_level* L) {
  free(L->vol);
  free(L->ctr);
  free(L->fL);
  free(L->fR);
  free(L->ftag);
  free(L->ftagR);
  free(L->Sn);
  free(L->area);
  free(L->amom);
  free(L->shift);
  free(L->c2f_ptr);
  free(L->c2f);
  free(L->fine2coarse);
  memset(L, 0, sizeof(*L));
}

void orc_mesh_free(orc_mesh* M) {
  free(M->ctype);
  free(M->vol);
  free(M->ctr);
  free(M->m2);
  free(M->fL);
  free(M->fR);
  free(M->ftag);
  free(M->ftagR);
  free(M->fngp);
  free(M->cvol);
  free(M->cctr);
  free(M->cSn);
  free(M->carea);
  free(M->camom);
  free(M->shift);
  free(M->gx);
  free(M->gA);
  free(M->cf);
  free(M->cside);
  for (int l = 0; l < 8; ++l) level_free(&M->lev[l]);
  memset(M, 0, sizeof(*M));
}

void orc_level_free(orc_level* L) { level_free(L); }

/* Gauss-Legendre rule on [-1, 1] by Newton iteration on P_n */
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* tensor Gauss points (n1d per direction) and weights (|det J| included) of every cell on the same
   iso-parametric maps as the geometry; used by the tests for exact cell averages of smooth fields */
int orc_mesh_qpoints(void* mp, const int8_t* ctype, const int64_t* cell_ptr, const int32_t* cell_nodes,
                     const double* xyz, int n1d, double* pts, double* wts) {
  orc_mesh* M = mp;
  double gx[16], gw[16];
  if (n1d < 1 || n1d > 16) return -1;
  gauss_legendre(n1d, gx, gw);
  const int nq = n1d * n1d * n1d;
  for (int64_t c = 0; c < M->nc; ++c) {
    double X[24];
    int nn = (int)(cell_ptr[c + 1] - cell_ptr[c]);
    for (int i = 0; i < nn; ++i)
      for (int d = 0; d < 3; ++d) X[3 * i + d] = xyz[3 * (int64_t)cell_nodes[cell_ptr[c] + i] + d];
    if (ctype[c] == 7)
      for (int i = 5; i < 8; ++i)
        for (int d = 0; d < 3; ++d) X[3 * i + d] = X[12 + d];
    int q = 0;
    for (int a = 0; a < n1d; ++a)
      for (int b = 0; b < n1d; ++b)
        for (int e = 0; e < n1d; ++e, ++q) {
          double x[3] = {0, 0, 0}, j1[3] = {0, 0, 0}, j2[3] = {0, 0, 0}, j3[3] = {0, 0, 0}, w;
          if (ctype[c] == 6 || ctype[c] == 7) {
            double xi = gx[a], et = gx[b], ze = gx[e];
            static const int sg[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                         {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
            for (int i = 0; i < 8; ++i) {
              double fx = 1 + sg[i][0] * xi, fy = 1 + sg[i][1] * et, fz = 1 + sg[i][2] * ze;
              for (int d = 0; d < 3; ++d) {
                x[d] += 0.125 * fx * fy * fz * X[3 * i + d];
                j1[d] += 0.125 * sg[i][0] * fy * fz * X[3 * i + d];
                j2[d] += 0.125 * fx * sg[i][1] * fz * X[3 * i + d];
                j3[d] += 0.125 * fx * fy * sg[i][2] * X[3 * i + d];
              }
            }
            w = gw[a] * gw[b] * gw[e] * det3(j1, j2, j3);
          } else if (ctype[c] == 5) {
            double u = 0.5 * (1.0 + gx[a]), v = 0.5 * (1.0 + gx[b]), ze = gx[e];
            double r = u, s = v * (1.0 - u);
            double L[3] = {1.0 - r - s, r, s}, dLr[3] = {-1.0, 1.0, 0.0}, dLs[3] = {-1.0, 0.0, 1.0};
            for (int i = 0; i < 3; ++i)
              for (int d = 0; d < 3; ++d) {
                double bot = X[3 * i + d], top = X[3 * (i + 3) + d];
                double col = 0.5 * (1.0 - ze) * bot + 0.5 * (1.0 + ze) * top;
                x[d] += L[i] * col;
                j1[d] += dLr[i] * col;
                j2[d] += dLs[i] * col;
                j3[d] += L[i] * 0.5 * (top - bot);
              }
            w = (0.5 * gw[a]) * (0.5 * gw[b]) * (1.0 - u) * gw[e] * det3(j1, j2, j3);
          } else {
            double u = 0.5 * (1.0 + gx[a]), v = 0.5 * (1.0 + gx[b]), t = 0.5 * (1.0 + gx[e]);
            double r = u, s = v * (1.0 - u), tt = t * (1.0 - u) * (1.0 - v);
            double e1[3], e2[3], e3[3];
            for (int d = 0; d < 3; ++d) {
              e1[d] = X[3 + d] - X[d];
              e2[d] = X[6 + d] - X[d];
              e3[d] = X[9 + d] - X[d];
              x[d] = X[d] + r * e1[d] + s * e2[d] + tt * e3[d];
            }
            w = (0.5 * gw[a]) * (0.5 * gw[b]) * (0.5 * gw[e]) * (1.0 - u) * (1.0 - u) * (1.0 - v) * det3(e1, e2, e3);
          }
          for (int d = 0; d < 3; ++d) pts[3 * ((int64_t)c * nq + q) + d] = x[d];
          wts[(int64_t)c * nq + q] = w;
        }
  }
  return 0;
}
