// Mesh coarsening on the device (Sec. 4.1 of the paper, Algorithm 1), bit-exact with the sequential
// definition:
//   hash      h_f = [23 (N_l + N_r) + N_l N_r] mod N_f over the interior faces (uint64);
//   selection the first face (lowest id) of every hash value: atomicMin per bucket, which does not
//             depend on thread order;
//   skewness  virtual centre C_c = (V_l C_l + V_r C_r)/(V_l + V_r); every face of L or R not between
//             them must satisfy (d . S n)^2 >= skew_min^2 |d|^2 |S n|^2, d = face centre - C_c,
//             evaluated with explicitly rounded IEEE operations (no FMA contraction);
//   merging   greedy pairwise matching in ascending face order, computed by locally-dominant rounds
//             (a confirmed face whose two cells are unmatched merges when it is the smallest such
//             face at both cells), which selects exactly the faces of the sequential greedy pass;
//   numbering coarse cells in the order of their smallest member; coarse faces one per
//             (coarse L < coarse R, periodic side tag) ordered lexicographically, boundary faces one
//             per (coarse cell, tag) after them; area vectors summed in ascending fine-face order.
#include "internal.cuh"

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t cell_label(int64_t c, uint64_t seed) {
  return seed == 0 ? (uint64_t)c : splitmix64_dev((uint64_t)c ^ seed) >> 33;
}

__device__ __forceinline__ bool is_candidate(const int32_t* fR, const int32_t* ftag, int64_t f) {
  return fR[f] >= 0 && ftag[f] == -1;
}

__global__ void k_count_candidates(int64_t nf, const int32_t* fR, const int32_t* ftag, unsigned long long* count) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f < nf && is_candidate(fR, ftag, f)) atomicAdd(count, 1ULL);
}

__device__ __forceinline__ uint64_t face_hash(const int32_t* fL, const int32_t* fR, int64_t f, uint64_t seed, uint64_t nfc) {
  const uint64_t a = cell_label(fL[f], seed), b = cell_label(fR[f], seed);
  return (23ULL * (a + b) + a * b) % nfc;
}

__global__ void k_bucket_min(int64_t nf, const int32_t* fL, const int32_t* fR, const int32_t* ftag, uint64_t seed,
                             uint64_t nfc, int32_t* bucket) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf || !is_candidate(fR, ftag, f)) return;
  atomicMin(&bucket[face_hash(fL, fR, f, seed, nfc)], (int32_t)f);
}

__device__ bool skew_confirmed(const Level& P, int32_t a, int32_t b, double kmin2) {
  const int64_t nc = P.nc, nf = P.nf;
  const double Va = P.vol[a], Vb = P.vol[b];
  const double Vs = __dadd_rn(Va, Vb);
  double Cc[3];
#pragma unroll
  for (int e = 0; e < 3; ++e)
    Cc[e] = __ddiv_rn(__dadd_rn(__dmul_rn(Va, P.ctr[e * nc + a]), __dmul_rn(Vb, P.ctr[e * nc + b])), Vs);
  const int32_t cells[2] = {a, b};
  for (int side = 0; side < 2; ++side) {
    const int32_t x = cells[side];
    for (int32_t k = P.c2f_ptr[x]; k < P.c2f_ptr[x + 1]; ++k) {
      const int64_t g = P.c2f[k];
      const int32_t gl = P.fL[g], gr = P.fR[g];
      const bool inL = gl == a || gl == b, inR = gr == a || gr == b;
      if (inL && inR) continue;
      const bool asR = gr == x && gl != x;
      double d[3], S[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        double xg = __ddiv_rn(P.amom[e * nf + g], P.area[g]);
        if (asR) xg = __dsub_rn(xg, P.shift[e * nf + g]);
        d[e] = __dsub_rn(xg, Cc[e]);
        S[e] = P.Sn[e * nf + g];
      }
      const double dn = __dadd_rn(__dadd_rn(__dmul_rn(d[0], S[0]), __dmul_rn(d[1], S[1])), __dmul_rn(d[2], S[2]));
      const double dd = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
      const double ss = __dadd_rn(__dadd_rn(__dmul_rn(S[0], S[0]), __dmul_rn(S[1], S[1])), __dmul_rn(S[2], S[2]));
      const double lhs = __dmul_rn(dn, dn);
      const double rhs = __dmul_rn(__dmul_rn(kmin2, dd), ss);
      if (!(lhs >= rhs)) return false;
    }
  }
  return true;
}

__global__ void k_select_confirm(Level P, uint64_t seed, uint64_t nfc, const int32_t* bucket, double kmin2,
                                 int8_t* conf) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= P.nf) return;
  int8_t ok = 0;
  if (is_candidate(P.fR, P.ftag, f) && bucket[face_hash(P.fL, P.fR, f, seed, nfc)] == (int32_t)f)
    ok = skew_confirmed(P, P.fL[f], P.fR[f], kmin2) ? 1 : 0;
  conf[f] = ok;
}

// smallest confirmed face of each unmatched cell whose other cell is unmatched
__global__ void k_best_face(Level P, const int8_t* conf, const int32_t* partner, int32_t* best) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= P.nc) return;
  int32_t b = INT32_MAX;
  if (partner[c] < 0)
    for (int32_t k = P.c2f_ptr[c]; k < P.c2f_ptr[c + 1]; ++k) {
      const int32_t g = P.c2f[k];
      if (!conf[g]) continue;
      const int32_t o = P.fL[g] == c ? P.fR[g] : P.fL[g];
      if (partner[o] < 0 && g < b) b = g;
    }
  best[c] = b;
}

__global__ void k_match_round(Level P, const int8_t* conf, const int32_t* best, int32_t* partner,
                              unsigned long long* matched) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= P.nf || !conf[f]) return;
  const int32_t a = P.fL[f], b = P.fR[f];
  if (best[a] == (int32_t)f && best[b] == (int32_t)f) {
    partner[a] = b;
    partner[b] = a;
    atomicAdd(matched, 1ULL);
  }
}

__global__ void k_rep_flag(int64_t nc, const int32_t* partner, int32_t* rep) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c < nc) rep[c] = (partner[c] < 0 || c < partner[c]) ? 1 : 0;
}

__global__ void k_map_cells(int64_t nc, const int32_t* partner, const int32_t* rep, const int32_t* cid, int32_t* map) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  map[c] = rep[c] ? cid[c] : cid[partner[c]];
}

__global__ void k_coarse_cells(Level P, const int32_t* partner, const int32_t* rep, const int32_t* cid, int64_t ncc,
                               double* vol, double* ctr) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= P.nc || !rep[c]) return;
  const int64_t k = cid[c], nc = P.nc;
  const int32_t b = partner[c];
  if (b < 0) {
    vol[k] = P.vol[c];
#pragma unroll
    for (int e = 0; e < 3; ++e) ctr[e * ncc + k] = P.ctr[e * nc + c];
    return;
  }
  const double Va = P.vol[c], Vb = P.vol[b], Vs = __dadd_rn(Va, Vb);
  vol[k] = Vs;
#pragma unroll
  for (int e = 0; e < 3; ++e)
    ctr[e * ncc + k] = __ddiv_rn(__dadd_rn(__dmul_rn(Va, P.ctr[e * nc + c]), __dmul_rn(Vb, P.ctr[e * nc + b])), Vs);
}

struct CRec {
  int32_t r, tag;  // r: coarse right cell (INT32_MAX for boundary faces); tag: periodic side / BC tag
  int32_t g, flip;
};

__device__ __forceinline__ bool crec_less(const CRec& x, const CRec& y) {
  if (x.r != y.r) return x.r < y.r;
  if (x.tag != y.tag) return x.tag < y.tag;
  return x.g < y.g;
}

// records of the faces owned by coarse cell k (k = coarse left cell), sorted; returns count or -1
__device__ int coarse_records(const Level& P, int64_t k, int32_t a, int32_t b, const int32_t* map, CRec* rec) {
  int n = 0;
  const int32_t mem[2] = {a, b};
  for (int s = 0; s < (b >= 0 ? 2 : 1); ++s) {
    const int32_t x = mem[s];
    for (int32_t j = P.c2f_ptr[x]; j < P.c2f_ptr[x + 1]; ++j) {
      const int32_t g = P.c2f[j];
      const int32_t gl = P.fL[g], gr = P.fR[g];
      CRec q;
      q.g = g;
      if (gr < 0) {
        q.r = INT32_MAX;
        q.tag = P.ftag[g];
        q.flip = 0;
      } else {
        const int32_t cl = map[gl], cr = map[gr];
        if (P.ftag[g] == -1 && cl == cr) continue;  // internal to the coarse cell
        const int flip = cl > cr;
        if ((flip ? cr : cl) != k) continue;         // owned by the other coarse cell
        if ((flip ? gr : gl) != x) continue;         // emitted once, from the new left member
        q.r = flip ? cl : cr;
        q.tag = flip ? P.ftagR[g] : P.ftag[g];
        q.flip = flip;
      }
      if (n >= CGKS_AGG_CAP) return -1;
      int i = n++;
      while (i > 0 && crec_less(q, rec[i - 1])) {
        rec[i] = rec[i - 1];
        --i;
      }
      rec[i] = q;
    }
  }
  return n;
}

__global__ void k_coarse_face_count(Level P, const int32_t* partner, const int32_t* rep, const int32_t* cid,
                                    const int32_t* map, int32_t* nint, int32_t* nbnd, DevErr* err) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= P.nc || !rep[c]) return;
  CRec rec[CGKS_AGG_CAP];
  const int64_t k = cid[c];
  const int n = coarse_records(P, k, (int32_t)c, partner[c], map, rec);
  if (n < 0) {
    set_err(err, CGKS_EMESH, (int)c, 60);
    nint[k] = nbnd[k] = 0;
    return;
  }
  int ni = 0, nb = 0;
  for (int i = 0; i < n; ++i)
    if (i == 0 || rec[i].r != rec[i - 1].r || rec[i].tag != rec[i - 1].tag) {
      if (rec[i].r == INT32_MAX)
        ++nb;
      else
        ++ni;
    }
  nint[k] = ni;
  nbnd[k] = nb;
}

__global__ void k_coarse_face_write(Level P, const int32_t* partner, const int32_t* rep, const int32_t* cid,
                                    const int32_t* map, const int32_t* oint, const int32_t* obnd, int64_t n_int_tot,
                                    Level Q) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= P.nc || !rep[c]) return;
  CRec rec[CGKS_AGG_CAP];
  const int64_t k = cid[c];
  const int n = coarse_records(P, k, (int32_t)c, partner[c], map, rec);
  if (n < 0) return;
  const int64_t nfP = P.nf, nfQ = Q.nf;
  int64_t fi = oint[k] - 1, fb = n_int_tot + obnd[k] - 1, f = -1;
  for (int i = 0; i < n; ++i) {
    const CRec& q = rec[i];
    const int64_t g = q.g;
    if (i == 0 || q.r != rec[i - 1].r || q.tag != rec[i - 1].tag) {
      f = q.r == INT32_MAX ? ++fb : ++fi;
      Q.fL[f] = (int32_t)k;
      Q.fR[f] = q.r == INT32_MAX ? -1 : q.r;
      Q.ftag[f] = q.tag;
      Q.ftagR[f] = q.r == INT32_MAX ? -1 : (q.flip ? P.ftag[g] : P.ftagR[g]);
      Q.area[f] = 0.0;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        Q.Sn[e * nfQ + f] = 0.0;
        Q.amom[e * nfQ + f] = 0.0;
        Q.shift[e * nfQ + f] = q.flip ? -P.shift[e * nfP + g] : P.shift[e * nfP + g];
      }
    }
    const double sg = q.flip ? -1.0 : 1.0;
    Q.area[f] = __dadd_rn(Q.area[f], P.area[g]);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      Q.Sn[e * nfQ + f] = __dadd_rn(Q.Sn[e * nfQ + f], sg * P.Sn[e * nfP + g]);
      double mom = P.amom[e * nfP + g];
      if (q.flip) mom = __dsub_rn(mom, __dmul_rn(P.area[g], P.shift[e * nfP + g]));
      Q.amom[e * nfQ + f] = __dadd_rn(Q.amom[e * nfQ + f], mom);
    }
  }
}

// cell -> face lists: degrees, then filling (order fixed afterwards by a per-cell sort)
__global__ void k_degree(int64_t nf, const int32_t* fL, const int32_t* fR, int32_t* deg) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  atomicAdd(&deg[fL[f]], 1);
  if (fR[f] >= 0 && fR[f] != fL[f]) atomicAdd(&deg[fR[f]], 1);
}

__global__ void k_fill_links(int64_t nf, const int32_t* fL, const int32_t* fR, const int32_t* ptr, int32_t* cursor,
                             int32_t* c2f) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  c2f[ptr[fL[f]] + atomicAdd(&cursor[fL[f]], 1)] = (int32_t)f;
  if (fR[f] >= 0 && fR[f] != fL[f]) c2f[ptr[fR[f]] + atomicAdd(&cursor[fR[f]], 1)] = (int32_t)f;
}

__global__ void k_sort_segments(int64_t n, const int32_t* ptr, int32_t* v) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int32_t i = ptr[c] + 1; i < ptr[c + 1]; ++i) {
    const int32_t x = v[i];
    int32_t j = i;
    while (j > ptr[c] && v[j - 1] > x) {
      v[j] = v[j - 1];
      --j;
    }
    v[j] = x;
  }
}

__global__ void k_iota(int64_t n, int32_t* v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = (int32_t)i;
}

__global__ void k_compose(int64_t n, const int32_t* map, int32_t* comp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) comp[i] = map[comp[i]];
}

__global__ void k_member_count(int64_t n, const int32_t* f2c, int32_t* cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[f2c[i]], 1);
}

__global__ void k_member_fill(int64_t n, const int32_t* f2c, const int32_t* ptr, int32_t* cursor, int32_t* agg) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) agg[ptr[f2c[i]] + atomicAdd(&cursor[f2c[i]], 1)] = (int32_t)i;
}

static cgks_status read_count(cgks_ctx* ctx, int64_t* out) {
  CK(cudaMemcpyAsync(ctx->h_count, ctx->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *out = *ctx->h_count;
  return CGKS_OK;
}

// CSR (ptr, list) of `n` rows from a per-row count array; ptr gets n + 1 entries
static cgks_status csr_from_counts(cgks_ctx* ctx, std::vector<void*>& M, int32_t* cnt, int64_t n, int32_t** ptr,
                                   int64_t* total) {
  CKS(dalloc(ctx, M, ptr, n + 1));
  CKS(scan_exclusive(ctx, cnt, *ptr, n, total));
  const int32_t t32 = (int32_t)*total;
  CK(cudaMemcpyAsync(*ptr + n, &t32, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

static cgks_status build_c2f(cgks_ctx* ctx, std::vector<void*>& M, std::vector<void*>& tmp, Level& Q) {
  cudaStream_t st = ctx->stream;
  int32_t *deg, *cur;
  CKS(dalloc(ctx, tmp, &deg, Q.nc));
  CKS(dalloc(ctx, tmp, &cur, Q.nc));
  k_degree<<<grid_for(Q.nf, 256), 256, 0, st>>>(Q.nf, Q.fL, Q.fR, deg);
  int64_t tot = 0;
  CKS(csr_from_counts(ctx, M, deg, Q.nc, &Q.c2f_ptr, &tot));
  CKS(dalloc(ctx, M, &Q.c2f, tot));
  k_fill_links<<<grid_for(Q.nf, 256), 256, 0, st>>>(Q.nf, Q.fL, Q.fR, Q.c2f_ptr, cur, Q.c2f);
  k_sort_segments<<<grid_for(Q.nc, 128), 128, 0, st>>>(Q.nc, Q.c2f_ptr, Q.c2f);
  CK(cudaGetLastError());
  return CGKS_OK;
}

// one coarsening pass P -> Q with map[P.nc]
static cgks_status coarsen_pass(cgks_ctx* ctx, const Level& P, Level& Q, int32_t* map) {
  std::vector<void*> tmp;
  struct Guard {
    std::vector<void*>& t;
    ~Guard() { free_list(t); }
  } guard{tmp};
  auto& M = ctx->mesh_allocs;
  cudaStream_t st = ctx->stream;
  const int B = 256;
  const uint64_t seed = ctx->P.agglo_seed;
  CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(int64_t), st));
  k_count_candidates<<<grid_for(P.nf, B), B, 0, st>>>(P.nf, P.fR, P.ftag, (unsigned long long*)ctx->d_count);
  int64_t nfc = 0;
  CKS(read_count(ctx, &nfc));
  int8_t* conf;
  int32_t *partner, *best, *rep, *cid;
  CKS(dalloc(ctx, tmp, &conf, P.nf));
  CKS(dalloc(ctx, tmp, &partner, P.nc));
  CKS(dalloc(ctx, tmp, &best, P.nc));
  CKS(dalloc(ctx, tmp, &rep, P.nc));
  CKS(dalloc(ctx, tmp, &cid, P.nc));
  CK(cudaMemsetAsync(partner, 0xFF, sizeof(int32_t) * P.nc, st));
  if (nfc > 0) {
    int32_t* bucket;
    CKS(dalloc(ctx, tmp, &bucket, nfc));
    CK(cudaMemsetAsync(bucket, 0x7F, sizeof(int32_t) * nfc, st));
    k_bucket_min<<<grid_for(P.nf, B), B, 0, st>>>(P.nf, P.fL, P.fR, P.ftag, seed, (uint64_t)nfc, bucket);
    const double kmin2 = ctx->P.skew_min * ctx->P.skew_min;
    k_select_confirm<<<grid_for(P.nf, B), B, 0, st>>>(P, seed, (uint64_t)nfc, bucket, kmin2, conf);
    for (int64_t round = 0; round <= P.nf; ++round) {
      k_best_face<<<grid_for(P.nc, B), B, 0, st>>>(P, conf, partner, best);
      CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(int64_t), st));
      k_match_round<<<grid_for(P.nf, B), B, 0, st>>>(P, conf, best, partner, (unsigned long long*)ctx->d_count);
      int64_t matched = 0;
      CKS(read_count(ctx, &matched));
      if (matched == 0) break;
    }
  } else {
    CK(cudaMemsetAsync(conf, 0, P.nf, st));
  }
  k_rep_flag<<<grid_for(P.nc, B), B, 0, st>>>(P.nc, partner, rep);
  int64_t ncc = 0;
  CKS(scan_exclusive(ctx, rep, cid, P.nc, &ncc));
  k_map_cells<<<grid_for(P.nc, B), B, 0, st>>>(P.nc, partner, rep, cid, map);
  Q = Level();
  Q.nc = ncc;
  CKS(dalloc(ctx, M, &Q.vol, ncc));
  CKS(dalloc(ctx, M, &Q.ctr, 3 * ncc));
  k_coarse_cells<<<grid_for(P.nc, B), B, 0, st>>>(P, partner, rep, cid, ncc, Q.vol, Q.ctr);
  int32_t *nint, *nbnd, *oint, *obnd;
  CKS(dalloc(ctx, tmp, &nint, ncc));
  CKS(dalloc(ctx, tmp, &nbnd, ncc));
  CKS(dalloc(ctx, tmp, &oint, ncc));
  CKS(dalloc(ctx, tmp, &obnd, ncc));
  k_coarse_face_count<<<grid_for(P.nc, 64), 64, 0, st>>>(P, partner, rep, cid, map, nint, nbnd, ctx->derr);
  CKS(check_device_error(ctx, "coarse faces"));
  int64_t ti = 0, tb = 0;
  CKS(scan_exclusive(ctx, nint, oint, ncc, &ti));
  CKS(scan_exclusive(ctx, nbnd, obnd, ncc, &tb));
  Q.nf = ti + tb;
  CKS(dalloc(ctx, M, &Q.fL, Q.nf));
  CKS(dalloc(ctx, M, &Q.fR, Q.nf));
  CKS(dalloc(ctx, M, &Q.ftag, Q.nf));
  CKS(dalloc(ctx, M, &Q.ftagR, Q.nf));
  CKS(dalloc(ctx, M, &Q.Sn, 3 * Q.nf));
  CKS(dalloc(ctx, M, &Q.area, Q.nf));
  CKS(dalloc(ctx, M, &Q.amom, 3 * Q.nf));
  CKS(dalloc(ctx, M, &Q.shift, 3 * Q.nf));
  k_coarse_face_write<<<grid_for(P.nc, 64), 64, 0, st>>>(P, partner, rep, cid, map, oint, obnd, ti, Q);
  CKS(build_c2f(ctx, M, tmp, Q));
  CK(cudaStreamSynchronize(st));
  CKS(check_device_error(ctx, "coarsening pass"));
  return CGKS_OK;
}

// unit normal and length of each face's (summed) area vector, once per level for the KFVS face flux
// and the coarse time step
__global__ void k_face_normals(int64_t nf, const double* __restrict__ Sn, double* __restrict__ nS) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const double S[3] = {Sn[f], Sn[nf + f], Sn[2 * nf + f]};
  const double s = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) nS[d * nf + f] = s > 0.0 ? S[d] / s : 0.0;
  nS[3 * nf + f] = s;
}

cgks_status build_levels(cgks_ctx* ctx) {
  auto& M = ctx->mesh_allocs;
  cudaStream_t st = ctx->stream;
  const int nl = ctx->P.n_levels < 1 ? 1 : ctx->P.n_levels;
  if (nl > 8) return cgks_fail(ctx, CGKS_EINVAL, "at most 8 multigrid levels");
  ctx->L.resize(1);
  for (int l = 1; l < nl; ++l) {
    // level 1 is built from the coarsening's own geometry of level 0 (identical in any implementation)
    const Level& prev = l == 1 ? ctx->L0c : ctx->L[l - 1];
    int32_t* comp;
    CKS(dalloc(ctx, M, &comp, prev.nc));
    k_iota<<<grid_for(prev.nc, 256), 256, 0, st>>>(prev.nc, comp);
    Level cur = prev;
    for (int p = 0; p < ctx->P.passes_per_level; ++p) {
      Level nxt;
      int32_t* map;
      CKS(dalloc(ctx, M, &map, cur.nc));
      CKS(coarsen_pass(ctx, cur, nxt, map));
      k_compose<<<grid_for(prev.nc, 256), 256, 0, st>>>(prev.nc, map, comp);
      cur = nxt;
    }
    cur.f2c = comp;
    cur.nc_finer = prev.nc;
    std::vector<void*> tmp;
    int32_t *cnt, *cursor;
    CKS(dalloc(ctx, tmp, &cnt, cur.nc));
    CKS(dalloc(ctx, tmp, &cursor, cur.nc));
    k_member_count<<<grid_for(prev.nc, 256), 256, 0, st>>>(prev.nc, comp, cnt);
    int64_t tot = 0;
    CKS(csr_from_counts(ctx, M, cnt, cur.nc, &cur.agg_ptr, &tot));
    CKS(dalloc(ctx, M, &cur.agg, tot));
    k_member_fill<<<grid_for(prev.nc, 256), 256, 0, st>>>(prev.nc, comp, cur.agg_ptr, cursor, cur.agg);
    k_sort_segments<<<grid_for(cur.nc, 128), 128, 0, st>>>(cur.nc, cur.agg_ptr, cur.agg);
    CK(cudaStreamSynchronize(st));
    free_list(tmp);
    ctx->L.push_back(cur);
  }
  for (Level& L : ctx->L) {
    CKS(dalloc(ctx, M, &L.nS, 4 * L.nf));
    k_face_normals<<<grid_for(L.nf, 256), 256, 0, st>>>(L.nf, L.Sn, L.nS);
  }
  ctx->C.assign(ctx->L.size(), CoarseBuf());
  for (size_t l = 1; l < ctx->L.size(); ++l) {
    CoarseBuf& B = ctx->C[l];
    const int64_t n = ctx->L[l].nc;
    CKS(dalloc(ctx, M, &B.W, 5 * n));
    CKS(dalloc(ctx, M, &B.W0, 5 * n));
    CKS(dalloc(ctx, M, &B.Rs, 5 * n));
    CKS(dalloc(ctx, M, &B.F, 5 * n));
    CKS(dalloc(ctx, M, &B.R, 5 * n));
    CKS(dalloc(ctx, M, &B.dt, n));
    CKS(dalloc(ctx, M, &B.ff, 5 * ctx->L[l].nf));
    CKS(dalloc(ctx, M, &B.ff32, 5 * ctx->L[l].nf));
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}
