/* Oracle mesh coarsening (Sec. 4.1 of the paper, Algorithm 1).  TEST INFRASTRUCTURE ONLY.
 *
 * One coarsening pass over a level:
 *   1. hash of every interior face, h_f = [23 (N_l + N_r) + N_l N_r] mod N_f (Eq. hash value), with
 *      N_f the number of interior faces of the level and N_l, N_r the cell labels;
 *   2. faces are visited in ascending face order and selected when their hash value is not yet in
 *      the table (first one wins);
 *   3. each selected face is confirmed when the skewness test holds (Eqs. virtual center and
 *      skewness factor);
 *   4. confirmed faces merge their two cells.
 * Readings (paper silent/garbled):
 *  - boundary and periodic faces are never candidates;
 *  - cell labels are the cell ids (seed 0, the paper's formula); a seed s > 0 relabels cell N as
 *    splitmix64(N xor s) >> 33 (31 bits, so the hash stays inside 64 bits);
 *  - skewness: for every face of L or R that is not between them, with d = face centre - C_c and
 *    S n its area vector, sin(alpha) = |d . n| / |d|; the merge is confirmed when
 *    (d . S n)^2 >= skew_min^2 |d|^2 |S n|^2 holds for all of them (IEEE operations in this order,
 *    no FMA); the measure is pinned by a hand-built pair, the limit skew_min (0.2 by default) is
 *    not given by the paper (parity unpinned);
 *  - merging is a pairwise matching: confirmed faces in ascending order merge their cells only when
 *    both are still unmatched in this pass;
 *  - coarse cells are numbered in the order of their smallest member; coarse volume V_a + V_b and
 *    centroid (V_a C_a + V_b C_b)/(V_a + V_b), singletons copied;
 *  - coarse faces: one per (coarse L < coarse R, periodic side) with the summed oriented area vectors
 *    in ascending fine face order; boundary faces one per (coarse cell, tag);
 *  - passes_per_level passes make one multigrid level.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t orc_face_hash(uint64_t nl, uint64_t nr, uint64_t nf) { return (23ULL * (nl + nr) + nl * nr) % nf; }

static uint64_t label(int64_t c, uint64_t seed) {
  if (seed == 0) return (uint64_t)c;
  return orc_splitmix64((uint64_t)c ^ seed) >> 33;
}

void orc_level_free(orc_level* L);

static void build_c2f(orc_level* L) {
  L->c2f_ptr = calloc(L->nc + 1, sizeof(int32_t));
  for (int64_t f = 0; f < L->nf; ++f) {
    L->c2f_ptr[L->fL[f] + 1]++;
    if (L->fR[f] >= 0 && L->fR[f] != L->fL[f]) L->c2f_ptr[L->fR[f] + 1]++;
  }
  for (int64_t c = 0; c < L->nc; ++c) L->c2f_ptr[c + 1] += L->c2f_ptr[c];
  L->c2f = malloc(sizeof(int32_t) * (L->c2f_ptr[L->nc] ? L->c2f_ptr[L->nc] : 1));
  int32_t* fill = calloc(L->nc, sizeof(int32_t));
  for (int64_t f = 0; f < L->nf; ++f) {
    int32_t a = L->fL[f], b = L->fR[f];
    L->c2f[L->c2f_ptr[a] + fill[a]++] = (int32_t)f;
    if (b >= 0 && b != a) L->c2f[L->c2f_ptr[b] + fill[b]++] = (int32_t)f;
  }
  free(fill);
}

static void level_alloc(orc_level* L, int64_t nc, int64_t nf) {
  L->nc = nc;
  L->nf = nf;
  L->vol = malloc(sizeof(double) * nc);
  L->ctr = malloc(sizeof(double) * 3 * nc);
  L->fL = malloc(sizeof(int32_t) * (nf ? nf : 1));
  L->fR = malloc(sizeof(int32_t) * (nf ? nf : 1));
  L->ftag = malloc(sizeof(int32_t) * (nf ? nf : 1));
  L->ftagR = malloc(sizeof(int32_t) * (nf ? nf : 1));
  L->Sn = malloc(sizeof(double) * 3 * (nf ? nf : 1));
  L->area = malloc(sizeof(double) * (nf ? nf : 1));
  L->amom = malloc(sizeof(double) * 3 * (nf ? nf : 1));
  L->shift = malloc(sizeof(double) * 3 * (nf ? nf : 1));
}

/* the fine mesh as a level */
static void fine_level(const orc_mesh* M, orc_level* L) {
  memset(L, 0, sizeof(*L));
  level_alloc(L, M->nc, M->nf);
  memcpy(L->vol, M->vol, sizeof(double) * M->nc);
  memcpy(L->ctr, M->ctr, sizeof(double) * 3 * M->nc);
  for (int64_t f = 0; f < M->nf; ++f) {
    L->fL[f] = M->fL[f];
    L->fR[f] = M->fR[f];
    L->ftag[f] = M->ftag[f];
    L->ftagR[f] = M->ftagR[f];
    double a = 0.0, S[3] = {0, 0, 0}, m[3] = {0, 0, 0};
    for (int k = 0; k < M->fngp[f]; ++k) {
      const double* dA = M->gA + 12 * f + 3 * k;
      const double* x = M->gx + 12 * f + 3 * k;
      double w = sqrt(dA[0] * dA[0] + dA[1] * dA[1] + dA[2] * dA[2]);
      a += w;
      for (int d = 0; d < 3; ++d) {
        S[d] += dA[d];
        m[d] += w * x[d];
      }
    }
    L->area[f] = a;
    for (int d = 0; d < 3; ++d) {
      L->Sn[3 * f + d] = S[d];
      L->amom[3 * f + d] = m[d];
      L->shift[3 * f + d] = M->shift[3 * f + d];
    }
  }
  L->n_int = M->n_int;
  L->n_per = M->n_per;
  build_c2f(L);
}

typedef struct {
  int32_t a, b, tag; /* interior/periodic: (cL, cR, side tag of cL); boundary: (c, INT32_MAX, tag) */
  int64_t g;         /* source face */
  int32_t flip;
} crec;
static int cmp_crec(const void* pa, const void* pb) {
  const crec* x = pa;
  const crec* y = pb;
  if (x->b == INT32_MAX) {
    if (y->b != INT32_MAX) return 1;
  } else if (y->b == INT32_MAX)
    return -1;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  if (x->tag != y->tag) return x->tag < y->tag ? -1 : 1;
  return x->g < y->g ? -1 : (x->g > y->g);
}

static int skew_ok(const orc_level* L, int32_t a, int32_t b, double kmin) {
  double Va = L->vol[a], Vb = L->vol[b], Cc[3];
  for (int d = 0; d < 3; ++d) Cc[d] = (Va * L->ctr[3 * a + d] + Vb * L->ctr[3 * b + d]) / (Va + Vb);
  const int32_t cells[2] = {a, b};
  for (int side = 0; side < 2; ++side) {
    int32_t x = cells[side];
    for (int32_t k = L->c2f_ptr[x]; k < L->c2f_ptr[x + 1]; ++k) {
      int32_t g = L->c2f[k];
      int32_t gl = L->fL[g], gr = L->fR[g];
      int inL = gl == a || gl == b, inR = gr == a || gr == b;
      if (inL && inR) continue; /* a face between the two merging cells */
      /* faces of b already seen from a? a face between x and a third cell appears once per x */
      int asR = (gr == x) && (gl != x);
      double xg[3], d[3];
      for (int e = 0; e < 3; ++e) {
        xg[e] = L->amom[3 * g + e] / L->area[g];
        if (asR) xg[e] = xg[e] - L->shift[3 * g + e];
        d[e] = xg[e] - Cc[e];
      }
      const double* S = L->Sn + 3 * g;
      double dn = (d[0] * S[0] + d[1] * S[1]) + d[2] * S[2];
      double dd = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
      double ss = (S[0] * S[0] + S[1] * S[1]) + S[2] * S[2];
      double lhs = dn * dn;
      double rhs = ((kmin * kmin) * dd) * ss;
      if (!(lhs >= rhs)) return 0;
    }
  }
  return 1;
}

/* one coarsening pass: cur -> out, map [cur.nc] */
static int coarsen_pass(const orc_level* cur, uint64_t seed, double kmin, orc_level* out, int32_t* map) {
  const int64_t nc = cur->nc, nf = cur->nf;
  int64_t Nf = 0;
  for (int64_t f = 0; f < nf; ++f)
    if (cur->fR[f] >= 0 && cur->ftag[f] == -1) ++Nf;
  int32_t* partner = malloc(sizeof(int32_t) * nc);
  for (int64_t c = 0; c < nc; ++c) partner[c] = -1;
  if (Nf > 0) {
    /* first loop: the collection V_d of faces whose hash value is new to the table */
    unsigned char* seen = calloc(Nf, 1);
    int64_t* Vd = malloc(sizeof(int64_t) * Nf);
    int64_t nd = 0;
    for (int64_t f = 0; f < nf; ++f) {
      if (!(cur->fR[f] >= 0 && cur->ftag[f] == -1)) continue;
      uint64_t h = orc_face_hash(label(cur->fL[f], seed), label(cur->fR[f], seed), (uint64_t)Nf);
      if (seen[h]) continue;
      seen[h] = 1;
      Vd[nd++] = f;
    }
    /* second loop: skewness confirmation, then the merge of the two cells */
    for (int64_t i = 0; i < nd; ++i) {
      int32_t a = cur->fL[Vd[i]], b = cur->fR[Vd[i]];
      if (!skew_ok(cur, a, b, kmin)) continue;
      if (partner[a] < 0 && partner[b] < 0) {
        partner[a] = b;
        partner[b] = a;
      }
    }
    free(Vd);
    free(seen);
  }
  int64_t m = 0;
  for (int64_t c = 0; c < nc; ++c)
    if (partner[c] < 0 || c < partner[c]) map[c] = (int32_t)m++;
  for (int64_t c = 0; c < nc; ++c)
    if (partner[c] >= 0 && c > partner[c]) map[c] = map[partner[c]];
  /* coarse faces */
  crec* recs = malloc(sizeof(crec) * (nf ? nf : 1));
  int64_t nr = 0;
  for (int64_t g = 0; g < nf; ++g) {
    int32_t cl = map[cur->fL[g]];
    if (cur->fR[g] < 0) {
      recs[nr].a = cl;
      recs[nr].b = INT32_MAX;
      recs[nr].tag = cur->ftag[g];
      recs[nr].g = g;
      recs[nr].flip = 0;
      ++nr;
      continue;
    }
    int32_t cr = map[cur->fR[g]];
    if (cur->ftag[g] == -1 && cl == cr) continue;
    int flip = cl > cr;
    recs[nr].a = flip ? cr : cl;
    recs[nr].b = flip ? cl : cr;
    recs[nr].tag = flip ? cur->ftagR[g] : cur->ftag[g];
    recs[nr].g = g;
    recs[nr].flip = flip;
    ++nr;
  }
  qsort(recs, nr, sizeof(crec), cmp_crec);
  int64_t ncf = 0;
  for (int64_t r = 0; r < nr; ++r)
    if (r == 0 || recs[r].a != recs[r - 1].a || recs[r].b != recs[r - 1].b || recs[r].tag != recs[r - 1].tag) ++ncf;
  memset(out, 0, sizeof(*out));
  level_alloc(out, m, ncf);
  /* coarse cells */
  for (int64_t c = 0; c < nc; ++c) {
    if (partner[c] >= 0 && c > partner[c]) continue;
    int32_t k = map[c];
    if (partner[c] < 0) {
      out->vol[k] = cur->vol[c];
      for (int d = 0; d < 3; ++d) out->ctr[3 * k + d] = cur->ctr[3 * c + d];
    } else {
      int32_t b = partner[c];
      double Va = cur->vol[c], Vb = cur->vol[b];
      out->vol[k] = Va + Vb;
      for (int d = 0; d < 3; ++d) out->ctr[3 * k + d] = (Va * cur->ctr[3 * c + d] + Vb * cur->ctr[3 * b + d]) / (Va + Vb);
    }
  }
  int64_t j = -1;
  out->n_int = 0;
  out->n_per = 0;
  for (int64_t r = 0; r < nr; ++r) {
    const crec* q = &recs[r];
    if (r == 0 || q->a != recs[r - 1].a || q->b != recs[r - 1].b || q->tag != recs[r - 1].tag) {
      ++j;
      out->fL[j] = q->a;
      out->fR[j] = q->b == INT32_MAX ? -1 : q->b;
      out->ftag[j] = q->tag;
      out->ftagR[j] = q->b == INT32_MAX ? -1 : (q->flip ? cur->ftag[q->g] : cur->ftagR[q->g]);
      out->area[j] = 0.0;
      for (int d = 0; d < 3; ++d) {
        out->Sn[3 * j + d] = 0.0;
        out->amom[3 * j + d] = 0.0;
        out->shift[3 * j + d] = q->flip ? -cur->shift[3 * q->g + d] : cur->shift[3 * q->g + d];
      }
      if (q->b != INT32_MAX) {
        if (q->tag == -1)
          out->n_int++;
        else
          out->n_per++;
      }
    }
    double sg = q->flip ? -1.0 : 1.0;
    out->area[j] += cur->area[q->g];
    for (int d = 0; d < 3; ++d) {
      out->Sn[3 * j + d] += sg * cur->Sn[3 * q->g + d];
      double mom = cur->amom[3 * q->g + d];
      if (q->flip) mom = mom - cur->area[q->g] * cur->shift[3 * q->g + d];
      out->amom[3 * j + d] += mom;
    }
  }
  build_c2f(out);
  free(recs);
  free(partner);
  return 0;
}

static void level_copy(const orc_level* a, orc_level* b) {
  memset(b, 0, sizeof(*b));
  level_alloc(b, a->nc, a->nf);
  memcpy(b->vol, a->vol, sizeof(double) * a->nc);
  memcpy(b->ctr, a->ctr, sizeof(double) * 3 * a->nc);
  memcpy(b->fL, a->fL, sizeof(int32_t) * a->nf);
  memcpy(b->fR, a->fR, sizeof(int32_t) * a->nf);
  memcpy(b->ftag, a->ftag, sizeof(int32_t) * a->nf);
  memcpy(b->ftagR, a->ftagR, sizeof(int32_t) * a->nf);
  memcpy(b->Sn, a->Sn, sizeof(double) * 3 * a->nf);
  memcpy(b->area, a->area, sizeof(double) * a->nf);
  memcpy(b->amom, a->amom, sizeof(double) * 3 * a->nf);
  memcpy(b->shift, a->shift, sizeof(double) * 3 * a->nf);
  b->n_int = a->n_int;
  b->n_per = a->n_per;
  build_c2f(b);
}

int orc_build_levels(orc_mesh* M, const orc_params* P, char* err) {
  int nl = P->n_levels < 1 ? 1 : P->n_levels;
  if (nl > 8) {
    if (err) snprintf(err, 256, "at most 8 levels");
    return -1;
  }
  for (int l = 0; l < 8; ++l) orc_level_free(&M->lev[l]);
  fine_level(M, &M->lev[0]);
  for (int l = 1; l < nl; ++l) {
    orc_level cur, nxt;
    level_copy(&M->lev[l - 1], &cur);
    if (l == 1) { /* level 1 is built from the coarsening's own geometry of the fine level */
      memcpy(cur.vol, M->cvol, sizeof(double) * M->nc);
      memcpy(cur.ctr, M->cctr, sizeof(double) * 3 * M->nc);
      memcpy(cur.Sn, M->cSn, sizeof(double) * 3 * M->nf);
      memcpy(cur.area, M->carea, sizeof(double) * M->nf);
      memcpy(cur.amom, M->camom, sizeof(double) * 3 * M->nf);
    }
    int32_t* comp = malloc(sizeof(int32_t) * cur.nc);
    for (int64_t i = 0; i < cur.nc; ++i) comp[i] = (int32_t)i;
    for (int p = 0; p < P->passes_per_level; ++p) {
      int32_t* map = malloc(sizeof(int32_t) * cur.nc);
      coarsen_pass(&cur, P->agglo_seed, P->skew_min, &nxt, map);
      for (int64_t i = 0; i < M->lev[l - 1].nc; ++i) comp[i] = map[comp[i]];
      orc_level_free(&cur);
      cur = nxt;
      free(map);
    }
    M->lev[l] = cur;
    M->lev[l].fine2coarse = comp;
    M->lev[l].nc_finer = M->lev[l - 1].nc;
  }
  M->n_levels = nl;
  return 0;
}
