// Fine-mesh setup on the device (Sec. 2.2 and 3 of the paper):
//  - face matching by a hash table keyed on the sorted node ids of every cell face;
//  - face numbering: interior faces ordered by (left, right) cell with left < right, periodic faces
//    in pair order, boundary faces in boundary-face order (prefix sums, no global sort);
//  - Gauss points on linear (iso-parametric) faces: 3 per triangle (barycentric 2/3,1/6,1/6, weight
//    1/3), 4 per quadrilateral (2x2 Gauss-Legendre on the bilinear map, per-point area vector);
//  - cell volume, centroid and central second moments by tensor Gauss rules on the iso-parametric
//    maps (collapsed coordinates for prisms and tetrahedra);
//  - per-cell operators of the HWENO reconstruction: the constrained least-squares p^2 (Sec. 3.1)
//    as a 9 x (4 N_f) linear map of the stencil data, Green-Gauss weights (Sec. 3.2),
//    least-squares gradient weights and the constants of the smoothness indicators (Sec. 3.4).
#include <cstdio>

#include "internal.cuh"
#include "recon_ops.cuh"

// local faces of each cell type, outward orientation (VTK-like node numbering)
// (type 4 tetrahedron, 5 prism, 6 hexahedron, 7 pyramid: base 0..3 counter-clockwise seen from apex 4)
__constant__ int8_t c_lface[4][6][4] = {
    {{0, 2, 1, -1}, {0, 1, 3, -1}, {1, 2, 3, -1}, {0, 3, 2, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}},
    {{0, 2, 1, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}, {-1, -1, -1, -1}},
    {{0, 3, 2, 1}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}},
    {{0, 3, 2, 1}, {0, 1, 4, -1}, {1, 2, 4, -1}, {2, 3, 4, -1}, {3, 0, 4, -1}, {-1, -1, -1, -1}}};

__device__ __forceinline__ int lface_nv(int t, int lf) { return c_lface[t - 4][lf][3] < 0 ? 3 : 4; }
__host__ __device__ __forceinline__ int cell_nnodes(int t) { return t == 4 ? 4 : (t == 5 ? 6 : (t == 7 ? 5 : 8)); }

// ---- geometry of the coarsening ------------------------------------------------------------------
// The agglomeration decides merges by comparing a skewness measure with a limit, so its geometric
// inputs are defined by one formula evaluated with a fixed sequence of correctly rounded operations
// (no contraction into FMA): the same values on every machine and in any independent implementation
// of the formula.  A face of nodes P_0..P_{n-1} (the left cell's local order): area vector
// 1/2 (P_1 - P_0) x (P_2 - P_0) for a triangle, 1/2 (P_2 - P_0) x (P_3 - P_1) for a quadrilateral
// (both exact for flat triangles and bilinear quadrilaterals), centre the node mean, area the length
// of the area vector.  A cell: centre the node mean, volume 1/3 sum over its faces (own local order,
// outward) of centre . area vector.
__device__ __forceinline__ void canon_face(const double P[4][3], int nv, double S[3], double X[3]) {
  double e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = nv == 3 ? __dsub_rn(P[1][d], P[0][d]) : __dsub_rn(P[2][d], P[0][d]);
    e2[d] = nv == 3 ? __dsub_rn(P[2][d], P[0][d]) : __dsub_rn(P[3][d], P[1][d]);
  }
  S[0] = __dmul_rn(0.5, __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1])));
  S[1] = __dmul_rn(0.5, __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2])));
  S[2] = __dmul_rn(0.5, __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0])));
  for (int d = 0; d < 3; ++d) {
    double a = P[0][d];
    for (int i = 1; i < nv; ++i) a = __dadd_rn(a, P[i][d]);
    X[d] = __ddiv_rn(a, (double)nv);
  }
}

__global__ void k_canon_faces(int64_t nf, const int32_t* fL, const int32_t* flf, const int8_t* ctype,
                              const int64_t* cptr, const int32_t* cn, const double* xyz, double* Sn, double* area,
                              double* amom) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int64_t c = fL[f];
  const int t = ctype[c], lf = flf[f], nv = lface_nv(t, lf);
  double P[4][3], S[3], X[3];
  for (int i = 0; i < nv; ++i) {
    const int64_t node = cn[cptr[c] + c_lface[t - 4][lf][i]];
    for (int d = 0; d < 3; ++d) P[i][d] = xyz[3 * node + d];
  }
  canon_face(P, nv, S, X);
  const double a = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(S[0], S[0]), __dmul_rn(S[1], S[1])), __dmul_rn(S[2], S[2])));
  area[f] = a;
  for (int d = 0; d < 3; ++d) {
    Sn[d * nf + f] = S[d];
    amom[d * nf + f] = __dmul_rn(a, X[d]);
  }
}

__global__ void k_canon_cells(int64_t nc, const int8_t* ctype, const int64_t* cptr, const int32_t* cn,
                              const double* xyz, double* vol, double* ctr) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int t = ctype[c];
  const int nn = cell_nnodes(t);
  for (int d = 0; d < 3; ++d) {
    double a = xyz[3 * (int64_t)cn[cptr[c]] + d];
    for (int i = 1; i < nn; ++i) a = __dadd_rn(a, xyz[3 * (int64_t)cn[cptr[c] + i] + d]);
    ctr[d * nc + c] = __ddiv_rn(a, (double)nn);
  }
  double v = 0.0;
  for (int lf = 0; lf < cell_nfaces(t); ++lf) {
    const int nv = lface_nv(t, lf);
    double P[4][3], S[3], X[3];
    for (int i = 0; i < nv; ++i) {
      const int64_t node = cn[cptr[c] + c_lface[t - 4][lf][i]];
      for (int d = 0; d < 3; ++d) P[i][d] = xyz[3 * node + d];
    }
    canon_face(P, nv, S, X);
    v = __dadd_rn(v, __dadd_rn(__dadd_rn(__dmul_rn(X[0], S[0]), __dmul_rn(X[1], S[1])), __dmul_rn(X[2], S[2])));
  }
  vol[c] = __ddiv_rn(v, 3.0);
}

struct Key4 {
  int32_t v[4];
};

__device__ __forceinline__ Key4 sorted_key(const int32_t* nodes, int nv) {
  Key4 k;
#pragma unroll
  for (int i = 0; i < 4; ++i) k.v[i] = i < nv ? nodes[i] : INT32_MAX;
#pragma unroll
  for (int i = 1; i < 4; ++i)
#pragma unroll
    for (int j = i; j > 0; --j)
      if (k.v[j - 1] > k.v[j]) {
        int32_t t = k.v[j];
        k.v[j] = k.v[j - 1];
        k.v[j - 1] = t;
      }
  return k;
}

__device__ __forceinline__ Key4 cell_face_key(const int8_t* ctype, const int64_t* cptr, const int32_t* cn, int64_t c,
                                              int lf) {
  const int t = ctype[c];
  int32_t nodes[4];
  const int nv = lface_nv(t, lf);
  for (int i = 0; i < nv; ++i) nodes[i] = cn[cptr[c] + c_lface[t - 4][lf][i]];
  return sorted_key(nodes, nv);
}

__device__ __forceinline__ uint64_t key_hash(const Key4& k) {
  uint64_t h = 0x9E3779B97F4A7C15ULL;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h ^= (uint64_t)(uint32_t)k.v[i] + 0x9E3779B97F4A7C15ULL + (h << 6) + (h >> 2);
    h *= 0xBF58476D1CE4E5B9ULL;
  }
  return h ^ (h >> 31);
}

__device__ __forceinline__ bool key_eq(const Key4& a, const Key4& b) {
  return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2] && a.v[3] == b.v[3];
}

__global__ void k_validate_cells(int64_t nc, const int8_t* ctype, const int64_t* cptr, const int32_t* cn,
                                 int64_t n_nodes, DevErr* err) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int t = ctype[c];
  const int64_t cnt = cptr[c + 1] - cptr[c];
  if (!((t == 4 && cnt == 4) || (t == 5 && cnt == 6) || (t == 6 && cnt == 8) || (t == 7 && cnt == 5))) {
    set_err(err, CGKS_EMESH, (int)c, 1);
    return;
  }
  for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q)
    if (cn[q] < 0 || cn[q] >= n_nodes) set_err(err, CGKS_EMESH, (int)c, 2);
}

// insert every cell face; the second arrival of a key records both partners
__global__ void k_insert_faces(int64_t nc, const int8_t* ctype, const int64_t* cptr, const int32_t* cn,
                               unsigned long long* slots, uint64_t mask, int64_t* partner, DevErr* err) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nc * 6) return;
  const int64_t c = r / 6;
  const int lf = (int)(r % 6);
  if (lf >= cell_nfaces(ctype[c])) return;
  const Key4 k = cell_face_key(ctype, cptr, cn, c, lf);
  uint64_t h = key_hash(k) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
    const unsigned long long prev = atomicCAS(&slots[h], 0ULL, (unsigned long long)(r + 1));
    if (prev == 0ULL) return;
    const int64_t o = (int64_t)prev - 1;
    if (key_eq(cell_face_key(ctype, cptr, cn, o / 6, (int)(o % 6)), k)) {
      if (o / 6 == c) {
        set_err(err, CGKS_EMESH, (int)c, 3);
        return;
      }
      if (atomicCAS((unsigned long long*)&partner[o], (unsigned long long)-1LL, (unsigned long long)r) !=
          (unsigned long long)-1LL) {
        set_err(err, CGKS_EMESH, (int)c, 4);  // a face shared by three cells
        return;
      }
      partner[r] = o;
      return;
    }
  }
  set_err(err, CGKS_EMESH, (int)c, 5);
}

__global__ void k_match_bfaces(int64_t nb, const int64_t* bptr, const int32_t* bnodes, const int8_t* ctype,
                               const int64_t* cptr, const int32_t* cn, const unsigned long long* slots, uint64_t mask,
                               const int64_t* partner, int32_t* bnd_of, int64_t* bowner, DevErr* err) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int nv = (int)(bptr[b + 1] - bptr[b]);
  if (nv != 3 && nv != 4) {
    set_err(err, CGKS_EMESH, (int)b, 10);
    return;
  }
  int32_t nodes[4];
  for (int i = 0; i < nv; ++i) nodes[i] = bnodes[bptr[b] + i];
  const Key4 k = sorted_key(nodes, nv);
  uint64_t h = key_hash(k) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
    const unsigned long long s = slots[h];
    if (s == 0ULL) break;
    const int64_t o = (int64_t)s - 1;
    if (key_eq(cell_face_key(ctype, cptr, cn, o / 6, (int)(o % 6)), k)) {
      if (partner[o] >= 0) {
        set_err(err, CGKS_EMESH, (int)b, 11);  // boundary face on an interior face
        return;
      }
      if (atomicCAS(&bnd_of[o], -1, (int32_t)b) != -1) {
        set_err(err, CGKS_EMESH, (int)b, 12);
        return;
      }
      bowner[b] = o;
      return;
    }
  }
  set_err(err, CGKS_EMESH, (int)b, 13);  // boundary face matches no cell face
}

__global__ void k_check_records(int64_t nc, const int8_t* ctype, const int64_t* partner, const int32_t* bnd_of,
                                DevErr* err) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nc * 6) return;
  if ((int)(r % 6) >= cell_nfaces(ctype[r / 6])) return;
  if (partner[r] < 0 && bnd_of[r] < 0) set_err(err, CGKS_EMESH, (int)(r / 6), 20);
}

__global__ void k_periodic_pairs(int64_t np, const int32_t* pairs, int64_t nb, const int32_t* btag, const int64_t* bptr,
                                 int32_t* bcount, DevErr* err) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int32_t a = pairs[2 * p], b = pairs[2 * p + 1];
  if (a < 0 || b < 0 || a >= nb || b >= nb || a == b) {
    set_err(err, CGKS_EINVAL, (int)p, 30);
    return;
  }
  if (btag[a] < 100 || btag[b] < 100 || bptr[a + 1] - bptr[a] != bptr[b + 1] - bptr[b]) {
    set_err(err, CGKS_EINVAL, (int)p, 31);
    return;
  }
  atomicAdd(&bcount[a], 1);
  atomicAdd(&bcount[b], 1);
}

__global__ void k_check_bfaces(int64_t nb, const int32_t* btag, const int32_t* bcount, int32_t* nonper, DevErr* err) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int t = btag[b];
  const bool per = t >= 100;
  if (!per && (t < 1 || t > 5)) set_err(err, CGKS_EINVAL, (int)b, 32);
  if (bcount[b] != (per ? 1 : 0)) set_err(err, CGKS_EINVAL, (int)b, 33);
  nonper[b] = per ? 0 : 1;
}

__global__ void k_count_owned(int64_t nc, const int8_t* ctype, const int64_t* partner, int32_t* cnt) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int n = 0;
  for (int lf = 0; lf < cell_nfaces(ctype[c]); ++lf) {
    const int64_t o = partner[c * 6 + lf];
    if (o >= 0 && o / 6 > c) ++n;
  }
  cnt[c] = n;
}

__global__ void k_write_interior(int64_t nc, const int8_t* ctype, const int64_t* partner, const int32_t* off,
                                 int32_t* fL, int32_t* fR, int32_t* ftag, int32_t* ftagR, int32_t* flf, int32_t* cf,
                                 int8_t* cside) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int64_t nbr[6];
  int lfs[6], n = 0;
  for (int lf = 0; lf < cell_nfaces(ctype[c]); ++lf) {
    const int64_t o = partner[c * 6 + lf];
    if (o >= 0 && o / 6 > c) {
      int j = n++;
      while (j > 0 && nbr[j - 1] / 6 > o / 6) {
        nbr[j] = nbr[j - 1];
        lfs[j] = lfs[j - 1];
        --j;
      }
      nbr[j] = o;
      lfs[j] = lf;
    }
  }
  for (int k = 0; k < n; ++k) {
    const int32_t f = off[c] + k;
    const int64_t o = nbr[k];
    fL[f] = (int32_t)c;
    fR[f] = (int32_t)(o / 6);
    ftag[f] = -1;
    ftagR[f] = -1;
    flf[f] = lfs[k];
    cf[(int64_t)lfs[k] * nc + c] = f;
    cside[(int64_t)lfs[k] * nc + c] = 0;
    cf[(o % 6) * nc + o / 6] = f;
    cside[(o % 6) * nc + o / 6] = 1;
  }
}

__global__ void k_write_periodic(int64_t np, int64_t n_int, const int32_t* pairs, const int64_t* bowner,
                                 const int32_t* btag, const int64_t* bptr, const int32_t* bnodes, const double* xyz,
                                 int64_t nc, int32_t* fL, int32_t* fR, int32_t* ftag, int32_t* ftagR, int32_t* flf,
                                 double* fshift, int64_t nf, int32_t* cf, int8_t* cside) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int32_t a = pairs[2 * p], b = pairs[2 * p + 1];
  const int64_t ra = bowner[a], rb = bowner[b];
  const int64_t f = n_int + p;
  fL[f] = (int32_t)(ra / 6);
  fR[f] = (int32_t)(rb / 6);
  ftag[f] = btag[a];
  ftagR[f] = btag[b];
  flf[f] = (int32_t)(ra % 6);
  const int nv = (int)(bptr[a + 1] - bptr[a]);
  for (int d = 0; d < 3; ++d) {
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < nv; ++i) {
      sa += xyz[3 * (int64_t)bnodes[bptr[a] + i] + d];
      sb += xyz[3 * (int64_t)bnodes[bptr[b] + i] + d];
    }
    fshift[d * nf + f] = sa / nv - sb / nv;
  }
  cf[(ra % 6) * nc + ra / 6] = (int32_t)f;
  cside[(ra % 6) * nc + ra / 6] = 0;
  cf[(rb % 6) * nc + rb / 6] = (int32_t)f;
  cside[(rb % 6) * nc + rb / 6] = 1;
}

__global__ void k_write_boundary(int64_t nb, int64_t base, const int32_t* nonper, const int32_t* rank,
                                 const int64_t* bowner, const int32_t* btag, int64_t nc, int32_t* fL, int32_t* fR,
                                 int32_t* ftag, int32_t* ftagR, int32_t* flf, int32_t* cf, int8_t* cside) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb || !nonper[b]) return;
  const int64_t f = base + rank[b];
  const int64_t r = bowner[b];
  fL[f] = (int32_t)(r / 6);
  fR[f] = -1;
  ftag[f] = btag[b];
  ftagR[f] = -1;
  flf[f] = (int32_t)(r % 6);
  cf[(r % 6) * nc + r / 6] = (int32_t)f;
  cside[(r % 6) * nc + r / 6] = 0;
}

__global__ void k_gp_count(int64_t nf, const int32_t* fL, const int32_t* flf, const int8_t* ctype, int32_t* cnt) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  cnt[f] = lface_nv(ctype[fL[f]], flf[f]);
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Gauss points and their area vectors (outward from the left cell) of every face; also the
// face's area vector, area, area-weighted centre and unit mean normal
__global__ void k_face_geom(int64_t nf, const int32_t* fL, const int32_t* flf, const int8_t* ctype,
                            const int64_t* cptr, const int32_t* cn, const double* xyz, const int32_t* gp_ptr,
                            int64_t ngp, int32_t* gp_face, double* gx, double* gA, double* Sn, double* area,
                            double* amom, double* fctr, double* fnrm) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int64_t c = fL[f];
  const int t = ctype[c], lf = flf[f];
  const int nv = lface_nv(t, lf);
  double P[4][3];
  for (int i = 0; i < nv; ++i) {
    const int64_t node = cn[cptr[c] + c_lface[t - 4][lf][i]];
    for (int d = 0; d < 3; ++d) P[i][d] = xyz[3 * node + d];
  }
  double X[4][3], A[4][3];
  if (nv == 3) {
    double e1[3], e2[3], n[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = P[1][d] - P[0][d];
      e2[d] = P[2][d] - P[0][d];
    }
    cross3(e1, e2, n);
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) {
        X[k][d] = (P[k][d] * 4.0 + P[(k + 1) % 3][d] + P[(k + 2) % 3][d]) / 6.0;
        A[k][d] = n[d] / 6.0;
      }
  } else {
    const double g = 0.57735026918962576451;  // 1/sqrt(3)
    const double sk[4] = {-g, g, g, -g}, tk[4] = {-g, -g, g, g};
    for (int k = 0; k < 4; ++k) {
      const double s = sk[k], tt = tk[k];
      double xs[3], xt[3];
      for (int d = 0; d < 3; ++d) {
        const double a = P[0][d], b = P[1][d], cc = P[2][d], e = P[3][d];
        X[k][d] = 0.25 * ((1 - s) * (1 - tt) * a + (1 + s) * (1 - tt) * b + (1 + s) * (1 + tt) * cc + (1 - s) * (1 + tt) * e);
        xs[d] = 0.25 * ((1 - tt) * (b - a) + (1 + tt) * (cc - e));
        xt[d] = 0.25 * ((1 - s) * (e - a) + (1 + s) * (cc - b));
      }
      cross3(xs, xt, A[k]);
    }
  }
  const int64_t g0 = gp_ptr[f];
  double S[3] = {0, 0, 0}, ar = 0.0, m[3] = {0, 0, 0};
  for (int k = 0; k < nv; ++k) {
    gp_face[g0 + k] = (int32_t)f;
    const double w = sqrt(A[k][0] * A[k][0] + A[k][1] * A[k][1] + A[k][2] * A[k][2]);
    ar += w;
    for (int d = 0; d < 3; ++d) {
      gx[d * ngp + g0 + k] = X[k][d];
      gA[d * ngp + g0 + k] = A[k][d];
      S[d] += A[k][d];
      m[d] += w * X[k][d];
    }
  }
  const double sn = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  area[f] = ar;
  for (int d = 0; d < 3; ++d) {
    Sn[d * nf + f] = S[d];
    amom[d * nf + f] = m[d];
    fctr[d * nf + f] = m[d] / ar;
    fnrm[d * nf + f] = S[d] / sn;
  }
}

__device__ __forceinline__ double det3(const double a[3], const double b[3], const double c[3]) {
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

// volume moments by tensor Gauss rules (3 points per direction) on the iso-parametric maps;
// prisms and tetrahedra through collapsed (Duffy) coordinates on the unit cube
__global__ void k_cell_geom(int64_t nc, const int8_t* ctype, const int64_t* cptr, const int32_t* cn, const double* xyz,
                            double* vol, double* ctr, double* m2, DevErr* err) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int t = ctype[c];
  double X[8][3];
  const int nn = cell_nnodes(t);
  for (int i = 0; i < nn; ++i)
    for (int d = 0; d < 3; ++d) X[i][d] = xyz[3 * (int64_t)cn[cptr[c] + i] + d];
  if (t == 7) {  // pyramid: the hexahedron map with its top face collapsed onto the apex
    for (int i = 5; i < 8; ++i)
      for (int d = 0; d < 3; ++d) X[i][d] = X[4][d];
    t = 6;
  }
  const double q = 0.7745966692414833770;  // sqrt(3/5)
  const double xg[3] = {-q, 0.0, q}, wg[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  double V = 0.0, M1[3] = {0, 0, 0}, M2[6] = {0, 0, 0, 0, 0, 0};
  double px[27][3], pw[27];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int e = 0; e < 3; ++e) {
        double x[3], J0[3], J1[3], J2[3], w;
        if (t == 6) {
          const double r = xg[a], s = xg[b], u = xg[e];
          for (int d = 0; d < 3; ++d) {
            double v[8];
            for (int i = 0; i < 8; ++i) v[i] = X[i][d];
            // trilinear map in the reference cube [-1,1]^3
            const double c00 = (1 - r) * v[0] + (1 + r) * v[1], c10 = (1 - r) * v[3] + (1 + r) * v[2];
            const double c01 = (1 - r) * v[4] + (1 + r) * v[5], c11 = (1 - r) * v[7] + (1 + r) * v[6];
            const double c0 = (1 - s) * c00 + (1 + s) * c10, c1 = (1 - s) * c01 + (1 + s) * c11;
            x[d] = 0.125 * ((1 - u) * c0 + (1 + u) * c1);
            J2[d] = 0.125 * (c1 - c0);
            J1[d] = 0.125 * ((1 - u) * (c10 - c00) + (1 + u) * (c11 - c01));
            const double d00 = v[1] - v[0], d10 = v[2] - v[3], d01 = v[5] - v[4], d11 = v[6] - v[7];
            J0[d] = 0.125 * ((1 - u) * ((1 - s) * d00 + (1 + s) * d10) + (1 + u) * ((1 - s) * d01 + (1 + s) * d11));
          }
          w = wg[a] * wg[b] * wg[e] * det3(J0, J1, J2);
        } else if (t == 5) {
          const double ua = 0.5 * (1 + xg[a]), vb = 0.5 * (1 + xg[b]), z = xg[e];
          const double r = ua, s = vb * (1 - ua);
          for (int d = 0; d < 3; ++d) {
            const double b0 = X[0][d], b1 = X[1][d], b2 = X[2][d], t0 = X[3][d], t1 = X[4][d], t2 = X[5][d];
            const double l0 = 0.5 * (1 - z), l1 = 0.5 * (1 + z);
            const double c0 = l0 * b0 + l1 * t0, c1 = l0 * b1 + l1 * t1, c2 = l0 * b2 + l1 * t2;
            x[d] = (1 - r - s) * c0 + r * c1 + s * c2;
            J0[d] = c1 - c0;
            J1[d] = c2 - c0;
            J2[d] = 0.5 * ((1 - r - s) * (t0 - b0) + r * (t1 - b1) + s * (t2 - b2));
          }
          w = 0.25 * wg[a] * wg[b] * wg[e] * (1 - ua) * det3(J0, J1, J2);
        } else {
          const double ua = 0.5 * (1 + xg[a]), vb = 0.5 * (1 + xg[b]), wc = 0.5 * (1 + xg[e]);
          const double r = ua, s = vb * (1 - ua), tt = wc * (1 - ua) * (1 - vb);
          for (int d = 0; d < 3; ++d) {
            J0[d] = X[1][d] - X[0][d];
            J1[d] = X[2][d] - X[0][d];
            J2[d] = X[3][d] - X[0][d];
            x[d] = X[0][d] + r * J0[d] + s * J1[d] + tt * J2[d];
          }
          w = 0.125 * wg[a] * wg[b] * wg[e] * (1 - ua) * (1 - ua) * (1 - vb) * det3(J0, J1, J2);
        }
        const int k = (a * 3 + b) * 3 + e;
        pw[k] = w;
        for (int d = 0; d < 3; ++d) px[k][d] = x[d];
        V += w;
        for (int d = 0; d < 3; ++d) M1[d] += w * x[d];
      }
  double cc[3];
  for (int d = 0; d < 3; ++d) cc[d] = M1[d] / V;
  for (int k = 0; k < 27; ++k) {
    const double y0 = px[k][0] - cc[0], y1 = px[k][1] - cc[1], y2 = px[k][2] - cc[2];
    M2[0] += pw[k] * y0 * y0;
    M2[1] += pw[k] * y1 * y1;
    M2[2] += pw[k] * y2 * y2;
    M2[3] += pw[k] * y0 * y1;
    M2[4] += pw[k] * y1 * y2;
    M2[5] += pw[k] * y0 * y2;
  }
  if (!(V > 0.0)) set_err(err, CGKS_EMESH, (int)c, 40);
  vol[c] = V;
  for (int d = 0; d < 3; ++d) ctr[d * nc + c] = cc[d];
  for (int j = 0; j < 6; ++j) m2[j * nc + c] = M2[j] / V;
}

// cell -> faces CSR with ascending face ids (the deterministic gather order)
__global__ void k_fill_c2f(int64_t nc, const int8_t* ctype, const int32_t* cf, const int32_t* ptr, int32_t* c2f) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int32_t v[6];
  const int n = cell_nfaces(ctype[c]);
  for (int m = 0; m < n; ++m) {
    int32_t f = cf[(int64_t)m * nc + c];
    int j = m;
    while (j > 0 && v[j - 1] > f) {
      v[j] = v[j - 1];
      --j;
    }
    v[j] = f;
  }
  for (int m = 0; m < n; ++m) c2f[ptr[c] + m] = v[m];
}

__global__ void k_types_to_int(int64_t nc, const int8_t* ctype, int32_t* out) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c < nc) out[c] = cell_nfaces(ctype[c]);
}

__global__ void __launch_bounds__(64) k_recon_ops(ROArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) recon_ops_body(i, a);
}

// ---- host orchestration ------------------------------------------------------------------------

static cgks_status upload(cgks_ctx* ctx, std::vector<void*>& tmp, const void* host, size_t bytes, void** dev) {
  CKS(dev_alloc(ctx, tmp, dev, bytes ? bytes : 1));
  if (bytes) CK(cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return CGKS_OK;
}

cgks_status build_fine_mesh(cgks_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_cells, const int8_t* ctype,
                            const int64_t* cell_ptr, const int32_t* cell_nodes, int64_t n_bfaces,
                            const int64_t* bface_ptr, const int32_t* bface_nodes, const int32_t* bface_tag,
                            const int32_t* periodic_pairs, int64_t n_periodic) {
  std::vector<void*> tmp;
  struct Guard {
    std::vector<void*>& t;
    ~Guard() { free_list(t); }
  } guard{tmp};
  cudaStream_t st = ctx->stream;
  Fine& F = ctx->F;
  auto& M = ctx->mesh_allocs;
  const int B = 256;
  const int64_t nc = n_cells, nb = n_bfaces, np = n_periodic;
  double* d_xyz;
  int8_t* d_ct;
  int64_t *d_cptr, *d_bptr;
  int32_t *d_cn, *d_bn, *d_btag, *d_pairs;
  CKS(upload(ctx, tmp, xyz, sizeof(double) * 3 * n_nodes, (void**)&d_xyz));
  CKS(upload(ctx, tmp, ctype, nc, (void**)&d_ct));
  CKS(upload(ctx, tmp, cell_ptr, sizeof(int64_t) * (nc + 1), (void**)&d_cptr));
  CKS(upload(ctx, tmp, cell_nodes, sizeof(int32_t) * cell_ptr[nc], (void**)&d_cn));
  CKS(upload(ctx, tmp, bface_ptr, sizeof(int64_t) * (nb + 1), (void**)&d_bptr));
  CKS(upload(ctx, tmp, bface_nodes, sizeof(int32_t) * bface_ptr[nb], (void**)&d_bn));
  CKS(upload(ctx, tmp, bface_tag, sizeof(int32_t) * nb, (void**)&d_btag));
  CKS(upload(ctx, tmp, periodic_pairs, sizeof(int32_t) * 2 * np, (void**)&d_pairs));
  CK(cudaMemsetAsync(ctx->derr, 0, sizeof(DevErr), st));
  k_validate_cells<<<grid_for(nc, B), B, 0, st>>>(nc, d_ct, d_cptr, d_cn, n_nodes, ctx->derr);
  CKS(check_device_error(ctx, "cell validation"));
  // hash table of cell faces
  uint64_t cap = 1024;
  while (cap < (uint64_t)(nc * 6) * 2) cap <<= 1;
  unsigned long long* slots;
  int64_t* partner;
  int32_t* bnd_of;
  int64_t* bowner;
  CKS(dalloc(ctx, tmp, &slots, cap));
  CKS(dalloc(ctx, tmp, &partner, nc * 6));
  CKS(dalloc(ctx, tmp, &bnd_of, nc * 6));
  CKS(dalloc(ctx, tmp, &bowner, nb));
  CK(cudaMemsetAsync(partner, 0xFF, sizeof(int64_t) * nc * 6, st));
  CK(cudaMemsetAsync(bnd_of, 0xFF, sizeof(int32_t) * nc * 6, st));
  k_insert_faces<<<grid_for(nc * 6, B), B, 0, st>>>(nc, d_ct, d_cptr, d_cn, slots, cap - 1, partner, ctx->derr);
  k_match_bfaces<<<grid_for(nb, B), B, 0, st>>>(nb, d_bptr, d_bn, d_ct, d_cptr, d_cn, slots, cap - 1, partner, bnd_of,
                                                bowner, ctx->derr);
  k_check_records<<<grid_for(nc * 6, B), B, 0, st>>>(nc, d_ct, partner, bnd_of, ctx->derr);
  int32_t *bcount, *nonper, *brank;
  CKS(dalloc(ctx, tmp, &bcount, nb));
  CKS(dalloc(ctx, tmp, &nonper, nb));
  CKS(dalloc(ctx, tmp, &brank, nb));
  if (np) k_periodic_pairs<<<grid_for(np, B), B, 0, st>>>(np, d_pairs, nb, d_btag, d_bptr, bcount, ctx->derr);
  if (nb) k_check_bfaces<<<grid_for(nb, B), B, 0, st>>>(nb, d_btag, bcount, nonper, ctx->derr);
  CKS(check_device_error(ctx, "face matching"));
  // numbering
  int32_t *cnt, *off;
  CKS(dalloc(ctx, tmp, &cnt, nc));
  CKS(dalloc(ctx, tmp, &off, nc));
  k_count_owned<<<grid_for(nc, B), B, 0, st>>>(nc, d_ct, partner, cnt);
  int64_t n_int = 0, n_bnd = 0;
  CKS(scan_exclusive(ctx, cnt, off, nc, &n_int));
  CKS(scan_exclusive(ctx, nonper, brank, nb, &n_bnd));
  const int64_t nf = n_int + np + n_bnd;
  F.nc = nc;
  F.nf = nf;
  F.n_int = n_int;
  F.n_per = np;
  F.n_bnd = n_bnd;
  CKS(dalloc(ctx, M, &F.ctype, nc));
  CK(cudaMemcpyAsync(F.ctype, d_ct, nc, cudaMemcpyDeviceToDevice, st));
  CKS(dalloc(ctx, M, &F.fL, nf));
  CKS(dalloc(ctx, M, &F.fR, nf));
  CKS(dalloc(ctx, M, &F.ftag, nf));
  CKS(dalloc(ctx, M, &F.ftagR, nf));
  CKS(dalloc(ctx, M, &F.flf, nf));
  CKS(dalloc(ctx, M, &F.fshift, 3 * nf));
  CKS(dalloc(ctx, M, &F.cf, 6 * nc));
  CKS(dalloc(ctx, M, &F.cside, 6 * nc));
  k_write_interior<<<grid_for(nc, B), B, 0, st>>>(nc, d_ct, partner, off, F.fL, F.fR, F.ftag, F.ftagR, F.flf, F.cf,
                                                  F.cside);
  if (np)
    k_write_periodic<<<grid_for(np, B), B, 0, st>>>(np, n_int, d_pairs, bowner, d_btag, d_bptr, d_bn, d_xyz, nc, F.fL,
                                                    F.fR, F.ftag, F.ftagR, F.flf, F.fshift, nf, F.cf, F.cside);
  if (nb)
    k_write_boundary<<<grid_for(nb, B), B, 0, st>>>(nb, n_int + np, nonper, brank, bowner, d_btag, nc, F.fL, F.fR,
                                                    F.ftag, F.ftagR, F.flf, F.cf, F.cside);
  // Gauss points
  int32_t* gcnt;
  CKS(dalloc(ctx, tmp, &gcnt, nf));
  CKS(dalloc(ctx, M, &F.gp_ptr, nf + 1));
  k_gp_count<<<grid_for(nf, B), B, 0, st>>>(nf, F.fL, F.flf, d_ct, gcnt);
  int64_t ngp = 0;
  CKS(scan_exclusive(ctx, gcnt, F.gp_ptr, nf, &ngp));
  int32_t ngp32 = (int32_t)ngp;
  CK(cudaMemcpyAsync(F.gp_ptr + nf, &ngp32, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  F.ngp = ngp;
  Level L0;
  L0.nc = nc;
  L0.nf = nf;
  L0.n_int = n_int;
  L0.n_per = np;
  CKS(dalloc(ctx, M, &F.gp_face, ngp));
  CKS(dalloc(ctx, M, &F.gp_x, 3 * ngp));
  CKS(dalloc(ctx, M, &F.gp_A, 3 * ngp));
  CKS(dalloc(ctx, M, &F.fctr, 3 * nf));
  CKS(dalloc(ctx, M, &F.fnrm, 3 * nf));
  CKS(dalloc(ctx, M, &L0.Sn, 3 * nf));
  CKS(dalloc(ctx, M, &L0.area, nf));
  CKS(dalloc(ctx, M, &L0.amom, 3 * nf));
  k_face_geom<<<grid_for(nf, B), B, 0, st>>>(nf, F.fL, F.flf, d_ct, d_cptr, d_cn, d_xyz, F.gp_ptr, ngp, F.gp_face,
                                             F.gp_x, F.gp_A, L0.Sn, L0.area, L0.amom, F.fctr, F.fnrm);
  // cell geometry
  CKS(dalloc(ctx, M, &F.vol, nc));
  CKS(dalloc(ctx, M, &F.ctr, 3 * nc));
  CKS(dalloc(ctx, M, &F.m2, 6 * nc));
  k_cell_geom<<<grid_for(nc, 128), 128, 0, st>>>(nc, d_ct, d_cptr, d_cn, d_xyz, F.vol, F.ctr, F.m2, ctx->derr);
  // cell -> face CSR
  int32_t* tcnt;
  CKS(dalloc(ctx, tmp, &tcnt, nc));
  CKS(dalloc(ctx, M, &F.c2f_ptr, nc + 1));
  k_types_to_int<<<grid_for(nc, B), B, 0, st>>>(nc, d_ct, tcnt);
  int64_t nlinks = 0;
  CKS(scan_exclusive(ctx, tcnt, F.c2f_ptr, nc, &nlinks));
  int32_t nl32 = (int32_t)nlinks;
  CK(cudaMemcpyAsync(F.c2f_ptr + nc, &nl32, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CKS(dalloc(ctx, M, &F.c2f, nlinks));
  k_fill_c2f<<<grid_for(nc, B), B, 0, st>>>(nc, d_ct, F.cf, F.c2f_ptr, F.c2f);
  CKS(check_device_error(ctx, "geometry"));
  // reconstruction operators
  CKS(dalloc(ctx, M, &F.Kop, (size_t)CGKS_KOP * nc));
  CKS(dalloc(ctx, M, &F.ggw, 18 * nc));
  CKS(dalloc(ctx, M, &F.lsw, 18 * nc));
  CKS(dalloc(ctx, M, &F.aux, CGKS_AUX * nc));
  CKS(dalloc(ctx, M, &F.dtw, 24 * nc));
  ROArgs ro{nc, nf, d_ct, F.cf, F.cside, F.fL, F.fR, F.vol, F.ctr, F.m2, L0.Sn, L0.area, F.fshift, F.fctr, F.fnrm,
            F.Kop, F.ggw, F.lsw, F.aux, F.dtw, ctx->derr};
  k_recon_ops<<<grid_for(nc, 64), 64, 0, st>>>(ro);
  CKS(check_device_error(ctx, "reconstruction operators"));
  // level 0 view
  L0.vol = F.vol;
  L0.ctr = F.ctr;
  L0.fL = F.fL;
  L0.fR = F.fR;
  L0.ftag = F.ftag;
  L0.ftagR = F.ftagR;
  L0.shift = F.fshift;
  L0.c2f_ptr = F.c2f_ptr;
  L0.c2f = F.c2f;
  ctx->L.clear();
  ctx->L.push_back(L0);
  // level 0 as seen by the coarsening: same topology, geometry of the coarsening
  Level Lc = L0;
  CKS(dalloc(ctx, M, &Lc.vol, nc));
  CKS(dalloc(ctx, M, &Lc.ctr, 3 * nc));
  CKS(dalloc(ctx, M, &Lc.Sn, 3 * nf));
  CKS(dalloc(ctx, M, &Lc.area, nf));
  CKS(dalloc(ctx, M, &Lc.amom, 3 * nf));
  k_canon_faces<<<grid_for(nf, B), B, 0, st>>>(nf, F.fL, F.flf, d_ct, d_cptr, d_cn, d_xyz, Lc.Sn, Lc.area, Lc.amom);
  k_canon_cells<<<grid_for(nc, 128), 128, 0, st>>>(nc, d_ct, d_cptr, d_cn, d_xyz, Lc.vol, Lc.ctr);
  CK(cudaGetLastError());
  ctx->L0c = Lc;
  CK(cudaStreamSynchronize(st));
  return CGKS_OK;
}
