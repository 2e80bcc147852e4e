// C ABI of libcgks (include/cgks.h): context, mesh upload, state, residual, explicit steps,
// V-cycles, steady solve; plus the allocation, scan and error plumbing shared by the kernels.
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "internal.cuh"

static thread_local std::string g_create_error;

cgks_status cgks_fail(cgks_ctx* c, cgks_status s, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return s;
}

cgks_status dev_alloc(cgks_ctx* ctx, std::vector<void*>& list, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cgks_fail(ctx, CGKS_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " +
                                           cudaGetErrorString(e));
  }
  list.push_back(*p);
  e = cudaMemsetAsync(*p, 0, bytes, ctx->stream);
  if (e != cudaSuccess) return cgks_fail(ctx, CGKS_ECUDA, cudaGetErrorString(e));
  return CGKS_OK;
}

void free_list(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

Phys make_phys(const cgks_params& P) {
  Phys ph{};
  ph.gamma = P.gamma;
  ph.K = (5.0 - 3.0 * P.gamma) / (P.gamma - 1.0);
  ph.mu = P.viscous ? P.mach / P.reynolds : 0.0;
  ph.prandtl = P.prandtl;
  ph.eps_inviscid = P.eps_inviscid;
  ph.c_press = P.c_press;
  ph.suth = P.sutherland;
  ph.cf = P.compression_factor;
  ph.weno_eps = P.weno_eps;
  ph.cfl_fine = P.cfl_fine;
  ph.cfl_coarse = P.cfl_coarse;
  ph.viscous = P.viscous;
  ph.dt_mode = P.dt_mode;
  const double a = P.aoa[0] * M_PI / 180.0, b = P.aoa[1] * M_PI / 180.0;
  const double u[3] = {P.mach * cos(a) * cos(b), P.mach * sin(b), P.mach * sin(a) * cos(b)};
  ph.Winf[0] = 1.0;
  for (int d = 0; d < 3; ++d) ph.Winf[1 + d] = u[d];
  ph.Winf[4] = 1.0 / P.gamma / (P.gamma - 1.0) + 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  return ph;
}

cgks_status check_device_error(cgks_ctx* ctx, const char* where) {
  CK(cudaMemcpyAsync(ctx->h_err, ctx->derr, sizeof(DevErr), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const DevErr e = *ctx->h_err;
  if (e.code) {
    CK(cudaMemsetAsync(ctx->derr, 0, sizeof(DevErr), ctx->stream));
    const char* what = e.code == CGKS_ENAN ? "non-physical or non-finite state" : "invalid input";
    return cgks_fail(ctx, (cgks_status)e.code, std::string(where) + ": " + what + " at index " +
                                                     std::to_string(e.index) + " (check " + std::to_string(e.detail) + ")");
  }
  return CGKS_OK;
}

// ---- exclusive scan of int32 ------------------------------------------------------------------

#define SCAN_THREADS 256
#define SCAN_ITEMS 4
#define SCAN_TILE (SCAN_THREADS * SCAN_ITEMS)

__device__ int32_t block_exclusive_scan(int32_t v, int32_t* sh, int32_t* total) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {
    const int32_t x = t >= off ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += x;
    __syncthreads();
  }
  const int32_t incl = sh[t];
  if (total) *total = sh[SCAN_THREADS - 1];
  __syncthreads();
  return incl - v;
}

__global__ void k_scan_tiles(const int32_t* in, int32_t* out, int64_t n, int32_t* tile_sum) {
  __shared__ int32_t sh[SCAN_THREADS];
  __shared__ int32_t tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS], s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int32_t run = block_exclusive_scan(s, sh, &tot);
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// scan of the tile sums by one block, chunk per thread; writes the grand total
__global__ void k_scan_tile_sums(int32_t* tile_sum, int64_t ntiles, int64_t* total) {
  __shared__ int32_t sh[SCAN_THREADS];
  __shared__ int32_t tot;
  const int64_t chunk = (ntiles + SCAN_THREADS - 1) / SCAN_THREADS;
  const int64_t b = threadIdx.x * chunk, e = b + chunk < ntiles ? b + chunk : ntiles;
  int32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += tile_sum[i];
  int32_t run = block_exclusive_scan(s, sh, &tot);
  for (int64_t i = b; i < e; ++i) {
    const int32_t x = tile_sum[i];
    tile_sum[i] = run;
    run += x;
  }
  if (threadIdx.x == 0) *total = tot;
}

__global__ void k_scan_add(int32_t* out, int64_t n, const int32_t* tile_sum) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_sum[i / SCAN_TILE];
}

cgks_status scan_exclusive(cgks_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, int64_t* total) {
  cudaStream_t st = ctx->stream;
  if (n == 0) {
    if (total) *total = 0;
    return CGKS_OK;
  }
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  std::vector<void*> tmp;
  int32_t* ts;
  int64_t* dtot;
  CKS(dalloc(ctx, tmp, &ts, ntiles));
  CKS(dalloc(ctx, tmp, &dtot, 1));
  k_scan_tiles<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, out, n, ts);
  k_scan_tile_sums<<<1, SCAN_THREADS, 0, st>>>(ts, ntiles, dtot);
  k_scan_add<<<grid_for(n, 256), 256, 0, st>>>(out, n, ts);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && total) {
    e = cudaMemcpyAsync(ctx->h_count, dtot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *total = *ctx->h_count;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  free_list(tmp);
  if (e != cudaSuccess) return cgks_fail(ctx, CGKS_ECUDA, std::string("scan: ") + cudaGetErrorString(e));
  return CGKS_OK;
}

// ---- kernel timing ---------------------------------------------------------------------------

static cudaEvent_t take_event(cgks_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(cgks_ctx* ctx, int kind, double units, double bytes) : c(ctx), k(kind) {
  if (!c->prof) return;
  cudaEvent_t e0 = take_event(c);
  e1 = take_event(c);
  cudaEventRecord(e0, c->stream);
  c->prof_ev[k].push_back({e0, e1, units, bytes});
}

ProfScope::~ProfScope() {
  if (e1) cudaEventRecord(e1, c->stream);
}

static void release_events(cgks_ctx* c) {
  for (auto& v : c->prof_ev) {
    for (auto& p : v) {
      c->ev_pool.push_back(p.e0);
      c->ev_pool.push_back(p.e1);
    }
    v.clear();
  }
}

// ---- C ABI --------------------------------------------------------------------------------------

extern "C" {

cgks_status cgks_profile(cgks_ctx* ctx, int enable) {
  if (!ctx) return CGKS_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  release_events(ctx);
  ctx->prof = enable != 0;
  return CGKS_OK;
}

cgks_status cgks_kernel_stats(cgks_ctx* ctx, int which, double* ms, int64_t* launches, double* units,
                              double* bytes) {
  if (!ctx) return CGKS_EINVAL;
  if (which < 0 || which >= PK_COUNT) return cgks_fail(ctx, CGKS_EINVAL, "kernel id out of range");
  CK(cudaStreamSynchronize(ctx->stream));
  double total = 0.0, u = 0.0, b = 0.0;
  for (auto& p : ctx->prof_ev[which]) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p.e0, p.e1));
    total += t;
    u += p.units;
    b += p.bytes;
  }
  if (ms) *ms = total;
  if (launches) *launches = (int64_t)ctx->prof_ev[which].size();
  if (units) *units = u;
  if (bytes) *bytes = b;
  return CGKS_OK;
}

cgks_status cgks_default_params(cgks_params* p) {
  if (!p) return CGKS_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->gamma = 1.4;
  p->mach = 0.2;
  p->reynolds = 1e4;
  p->prandtl = 1.0;
  p->cfl_fine = 0.5;
  p->cfl_coarse = 0.9;
  p->eps_inviscid = 0.01;
  p->c_press = 1.0;
  p->weno_eps = 1e-5;
  p->skew_min = 0.2;
  p->correction_relax = 1.0;
  p->compression_factor = 1;
  p->n_levels = 3;
  p->pre = 1;
  p->post = 0;
  p->coarse_steps = 2;
  p->passes_per_level = 2;
  return CGKS_OK;
}

static cgks_status check_params(cgks_ctx* ctx, const cgks_params* p) {
  if (!p) return cgks_fail(ctx, CGKS_EINVAL, "params is NULL");
  if (!(p->gamma > 1.0) || !(p->gamma < 5.0 / 3.0 + 1e-12)) return cgks_fail(ctx, CGKS_EINVAL, "gamma must be in (1, 5/3]");
  if (!(p->mach >= 0.0) || !(p->cfl_fine > 0.0) || !(p->cfl_coarse > 0.0)) return cgks_fail(ctx, CGKS_EINVAL, "mach/cfl");
  if (p->viscous && !(p->reynolds > 0.0)) return cgks_fail(ctx, CGKS_EINVAL, "reynolds must be positive");
  if (!(p->prandtl > 0.0) || !(p->weno_eps > 0.0)) return cgks_fail(ctx, CGKS_EINVAL, "prandtl/weno_eps");
  if (!(p->sutherland >= 0.0)) return cgks_fail(ctx, CGKS_EINVAL, "sutherland must be >= 0");
  if (p->n_levels < 1 || p->n_levels > 8 || p->passes_per_level < 0 || p->coarse_steps < 0 || p->pre < 0 || p->post < 0)
    return cgks_fail(ctx, CGKS_EINVAL, "multigrid counts out of range");
  if (p->precision != 0 && p->precision != 1) return cgks_fail(ctx, CGKS_EINVAL, "precision must be 0 or 1");
  if (!(p->correction_relax > 0.0) || !(p->correction_relax <= 1.0))
    return cgks_fail(ctx, CGKS_EINVAL, "correction_relax must be in (0, 1]");
  if (p->coarse_smoother != 0 && p->coarse_smoother != 1)
    return cgks_fail(ctx, CGKS_EINVAL, "coarse_smoother must be 0 or 1");
  if (p->compression_factor != 0 && p->compression_factor != 1)
    return cgks_fail(ctx, CGKS_EINVAL, "compression_factor must be 0 or 1");
  if (p->prolongation != 0 && p->prolongation != 1) return cgks_fail(ctx, CGKS_EINVAL, "prolongation must be 0 or 1");
  if (p->adjoint_recompute != 0 && p->adjoint_recompute != 1)
    return cgks_fail(ctx, CGKS_EINVAL, "adjoint_recompute must be 0 or 1");
  return CGKS_OK;
}

cgks_status cgks_create(const cgks_params* params, void* cuda_stream, cgks_ctx** out) {
  if (!out) return cgks_fail(nullptr, CGKS_EINVAL, "out is NULL");
  *out = nullptr;
  cgks_ctx* ctx = new (std::nothrow) cgks_ctx();
  if (!ctx) return cgks_fail(nullptr, CGKS_ENOMEM, "host allocation");
  cgks_status s = check_params(ctx, params);
  if (s != CGKS_OK) {
    g_create_error = ctx->err;
    delete ctx;
    return s;
  }
  ctx->P = *params;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_err, sizeof(DevErr));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_count, sizeof(int64_t));
  if (e != cudaSuccess) {
    g_create_error = std::string("cgks_create: ") + cudaGetErrorString(e);
    delete ctx;
    return CGKS_ECUDA;
  }
  if ((s = dalloc(ctx, ctx->ctx_allocs, &ctx->derr, 1)) != CGKS_OK ||
      (s = dalloc(ctx, ctx->ctx_allocs, &ctx->d_count, 1)) != CGKS_OK ||
      (s = dalloc(ctx, ctx->ctx_allocs, &ctx->d_skipped, 1)) != CGKS_OK ||
      (s = dalloc(ctx, ctx->ctx_allocs, &ctx->nrm_part, 1024)) != CGKS_OK ||
      (s = dalloc(ctx, ctx->ctx_allocs, &ctx->nrm, 1)) != CGKS_OK) {
    g_create_error = ctx->err;
    cgks_destroy(ctx);
    return s;
  }
  *out = ctx;
  return CGKS_OK;
}

cgks_status cgks_destroy(cgks_ctx* ctx) {
  if (!ctx) return CGKS_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  release_events(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->gstream) {
    cudaStreamSynchronize(ctx->gstream);
    cudaStreamDestroy(ctx->gstream);
  }
  for (cudaEvent_t e : ctx->gev)
    if (e) cudaEventDestroy(e);
  free_list(ctx->mesh_allocs);
  free_list(ctx->ctx_allocs);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  if (ctx->h_count) cudaFreeHost(ctx->h_count);
  if (ctx->h_nrm) cudaFreeHost(ctx->h_nrm);
  delete ctx;
  return CGKS_OK;
}

cgks_status cgks_set_params(cgks_ctx* ctx, const cgks_params* params) {
  if (!ctx) return CGKS_EINVAL;
  CKS(check_params(ctx, params));
  ctx->P = *params;
  return CGKS_OK;
}

cgks_status cgks_mesh_upload(cgks_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_cells, const int8_t* cell_type,
                             const int64_t* cell_ptr, const int32_t* cell_nodes, int64_t n_bfaces,
                             const int64_t* bface_ptr, const int32_t* bface_nodes, const int32_t* bface_tag,
                             const int32_t* periodic_pairs, int64_t n_periodic) {
  if (!ctx) return CGKS_EINVAL;
  if (n_nodes <= 0 || n_cells <= 0 || n_bfaces < 0 || n_periodic < 0 || !xyz || !cell_type || !cell_ptr || !cell_nodes ||
      (n_bfaces && (!bface_ptr || !bface_nodes || !bface_tag)) || (n_periodic && !periodic_pairs))
    return cgks_fail(ctx, CGKS_EINVAL, "cgks_mesh_upload: null pointer or non-positive size");
  if (n_cells * 6 >= (int64_t)INT32_MAX) return cgks_fail(ctx, CGKS_EINVAL, "too many cells for 32-bit indices");
  if (cell_ptr[0] != 0) return cgks_fail(ctx, CGKS_EMESH, "cell_ptr[0] must be 0");
  for (int64_t c = 0; c < n_cells; ++c)
    if (cell_ptr[c + 1] < cell_ptr[c]) return cgks_fail(ctx, CGKS_EMESH, "cell_ptr not monotone");
  if (n_bfaces) {
    if (bface_ptr[0] != 0) return cgks_fail(ctx, CGKS_EMESH, "bface_ptr[0] must be 0");
    for (int64_t b = 0; b < n_bfaces; ++b)
      if (bface_ptr[b + 1] < bface_ptr[b]) return cgks_fail(ctx, CGKS_EMESH, "bface_ptr not monotone");
  }
  CK(cudaStreamSynchronize(ctx->stream));
  free_list(ctx->mesh_allocs);
  // the adjoint's arrays were in mesh_allocs
  ctx->Jp = ctx->Jr = ctx->adt = ctx->pbar = ctx->aself = ctx->arec = ctx->avec = ctx->apart = ctx->akry = nullptr;
  ctx->ajc = ctx->acb = ctx->aWG = nullptr;
  ctx->lin_recompute = false;
  ctx->F = Fine();
  ctx->L.clear();
  ctx->C.clear();
  ctx->has_mesh = ctx->has_state = false;
  static const int64_t empty64 = 0;
  ctx->linearized = false;
  ctx->h_xyz.assign(xyz, xyz + 3 * n_nodes);
  ctx->h_ctype.assign(cell_type, cell_type + n_cells);
  ctx->h_cptr.assign(cell_ptr, cell_ptr + n_cells + 1);
  ctx->h_cnodes.assign(cell_nodes, cell_nodes + cell_ptr[n_cells]);
  ctx->h_bptr.assign(n_bfaces ? bface_ptr : nullptr, n_bfaces ? bface_ptr + n_bfaces + 1 : nullptr);
  ctx->h_bnodes.assign(n_bfaces ? bface_nodes : nullptr, n_bfaces ? bface_nodes + bface_ptr[n_bfaces] : nullptr);
  ctx->h_btag.assign(n_bfaces ? bface_tag : nullptr, n_bfaces ? bface_tag + n_bfaces : nullptr);
  ctx->h_pairs.assign(n_periodic ? periodic_pairs : nullptr, n_periodic ? periodic_pairs + 2 * n_periodic : nullptr);
  CKS(build_fine_mesh(ctx, n_nodes, xyz, n_cells, cell_type, cell_ptr, cell_nodes, n_bfaces,
                      n_bfaces ? bface_ptr : &empty64, bface_nodes, bface_tag, periodic_pairs, n_periodic));
  {  // Gauss points seen from the cells: tet 4 x 3, prism 2 x 3 + 3 x 4, hex 6 x 4, pyramid 4 + 4 x 3
    int64_t s = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
      const int t = cell_type[c];
      s += t == 4 ? 12 : t == 5 ? 18 : t == 6 ? 24 : 16;
    }
    ctx->F.gp_sides = s;
  }
  CKS(build_levels(ctx));
  const Fine& F = ctx->F;
  auto& M = ctx->mesh_allocs;
  CKS(dalloc(ctx, M, &ctx->W, 5 * F.nc));
  CKS(dalloc(ctx, M, &ctx->G, 15 * F.nc));
  CKS(dalloc(ctx, M, &ctx->alpha, F.nc));
  CKS(dalloc(ctx, M, &ctx->rc, (size_t)CGKS_RC * F.nc));
  CKS(dalloc(ctx, M, &ctx->dt, F.nc));
  CKS(dalloc(ctx, M, &ctx->res, 5 * F.nc));
  CKS(dalloc(ctx, M, &ctx->gpr, (size_t)CGKS_GPR * F.ngp));
  CKS(dalloc(ctx, M, &ctx->ffl, 5 * F.nf));
  CKS(dalloc(ctx, M, &ctx->ffl32, 5 * F.nf));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->has_mesh = true;
  return CGKS_OK;
}

#define NEED_MESH()                                                                   \
  do {                                                                                \
    if (!ctx) return CGKS_EINVAL;                                                     \
    if (!ctx->has_mesh) return cgks_fail(ctx, CGKS_EINVAL, "no mesh uploaded");       \
  } while (0)
#define NEED_STATE()                                                                  \
  do {                                                                                \
    NEED_MESH();                                                                      \
    if (!ctx->has_state) return cgks_fail(ctx, CGKS_EINVAL, "state not initialised"); \
  } while (0)

cgks_status cgks_level_info(cgks_ctx* ctx, int level, int64_t* n_cells, int64_t* n_faces) {
  NEED_MESH();
  if (level < 0 || level >= (int)ctx->L.size()) return cgks_fail(ctx, CGKS_EINVAL, "level out of range");
  if (n_cells) *n_cells = ctx->L[level].nc;
  if (n_faces) *n_faces = ctx->L[level].nf;
  return CGKS_OK;
}

cgks_status cgks_coarse_map(cgks_ctx* ctx, int level, int32_t* fine_to_coarse) {
  NEED_MESH();
  if (level < 1 || level >= (int)ctx->L.size() || !fine_to_coarse)
    return cgks_fail(ctx, CGKS_EINVAL, "cgks_coarse_map: level must be in [1, n_levels) and output non-NULL");
  const Level& L = ctx->L[level];
  CK(cudaMemcpyAsync(fine_to_coarse, L.f2c, sizeof(int32_t) * L.nc_finer, cudaMemcpyDefault, ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_level_geometry(cgks_ctx* ctx, int level, double* vol, double* ctr, int32_t* face_left,
                                int32_t* face_right, int32_t* face_tag, double* area_vec) {
  NEED_MESH();
  if (level < 0 || level >= (int)ctx->L.size()) return cgks_fail(ctx, CGKS_EINVAL, "level out of range");
  const Level& L = ctx->L[level];
  cudaStream_t st = ctx->stream;
  if (vol) CK(cudaMemcpyAsync(vol, L.vol, sizeof(double) * L.nc, cudaMemcpyDefault, st));
  if (ctr) CK(cudaMemcpyAsync(ctr, L.ctr, sizeof(double) * 3 * L.nc, cudaMemcpyDefault, st));
  if (face_left) CK(cudaMemcpyAsync(face_left, L.fL, sizeof(int32_t) * L.nf, cudaMemcpyDefault, st));
  if (face_right) CK(cudaMemcpyAsync(face_right, L.fR, sizeof(int32_t) * L.nf, cudaMemcpyDefault, st));
  if (face_tag) CK(cudaMemcpyAsync(face_tag, L.ftag, sizeof(int32_t) * L.nf, cudaMemcpyDefault, st));
  if (area_vec) CK(cudaMemcpyAsync(area_vec, L.Sn, sizeof(double) * 3 * L.nf, cudaMemcpyDefault, st));
  return CGKS_OK;
}

cgks_status cgks_fine_moments(cgks_ctx* ctx, double* m2) {
  NEED_MESH();
  if (!m2) return cgks_fail(ctx, CGKS_EINVAL, "m2 is NULL");
  CK(cudaMemcpyAsync(m2, ctx->F.m2, sizeof(double) * 6 * ctx->F.nc, cudaMemcpyDefault, ctx->stream));
  return CGKS_OK;
}

__global__ void k_fill(int64_t n, double v, double* x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

cgks_status cgks_state_init(cgks_ctx* ctx, const double* W, const double* gradW, const double* alpha) {
  NEED_MESH();
  if (!W) return cgks_fail(ctx, CGKS_EINVAL, "W is NULL");
  const int64_t n = ctx->F.nc;
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->W, W, sizeof(double) * 5 * n, cudaMemcpyDefault, st));
  if (gradW)
    CK(cudaMemcpyAsync(ctx->G, gradW, sizeof(double) * 15 * n, cudaMemcpyDefault, st));
  else
    CK(cudaMemsetAsync(ctx->G, 0, sizeof(double) * 15 * n, st));
  if (alpha)
    CK(cudaMemcpyAsync(ctx->alpha, alpha, sizeof(double) * n, cudaMemcpyDefault, st));
  else
    k_fill<<<grid_for(n, 256), 256, 0, st>>>(n, 1.0, ctx->alpha);
  CK(cudaMemsetAsync(ctx->d_skipped, 0, sizeof(int64_t), st));
  CK(cudaGetLastError());
  ctx->has_state = true;
  ctx->iters = 0;
  ctx->r1 = 0.0;
  return CGKS_OK;
}

cgks_status cgks_state_get(cgks_ctx* ctx, double* W, double* gradW, double* alpha) {
  NEED_STATE();
  const int64_t n = ctx->F.nc;
  cudaStream_t st = ctx->stream;
  if (W) CK(cudaMemcpyAsync(W, ctx->W, sizeof(double) * 5 * n, cudaMemcpyDefault, st));
  if (gradW) CK(cudaMemcpyAsync(gradW, ctx->G, sizeof(double) * 15 * n, cudaMemcpyDefault, st));
  if (alpha) CK(cudaMemcpyAsync(alpha, ctx->alpha, sizeof(double) * n, cudaMemcpyDefault, st));
  return CGKS_OK;
}

static cgks_status read_norm(cgks_ctx* ctx, const double* dev, double* host, int n) {
  CK(cudaMemcpyAsync(host, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_residual(cgks_ctx* ctx, int order, double* res, double* gradW_new, double* alpha_new, double* dt,
                          double* norm) {
  NEED_STATE();
  const Fine& F = ctx->F;
  cudaStream_t st = ctx->stream;
  if (order == 3) {
    CKS(fine_fluxes(ctx, ctx->W, ctx->G, ctx->alpha));
    CKS(fine_gather(ctx, ctx->W, nullptr, ctx->res, gradW_new, alpha_new, 0));
    if (dt) CK(cudaMemcpyAsync(dt, ctx->dt, sizeof(double) * F.nc, cudaMemcpyDefault, st));
  } else if (order == 1) {
    CKS(kfvs_residual(ctx, 0, ctx->W, ctx->res));
    if (gradW_new || alpha_new) return cgks_fail(ctx, CGKS_EINVAL, "order 1 has no gradient outputs");
    if (dt) CKS(coarse_dt(ctx, 0, ctx->W, dt));
  } else {
    return cgks_fail(ctx, CGKS_EINVAL, "order must be 1 or 3");
  }
  if (res) CK(cudaMemcpyAsync(res, ctx->res, sizeof(double) * 5 * F.nc, cudaMemcpyDefault, st));
  if (norm) {
    CKS(density_norm(ctx, ctx->res, F.vol, F.nc, ctx->nrm));
    CKS(read_norm(ctx, ctx->nrm, norm, 1));
  }
  return check_device_error(ctx, "cgks_residual");
}

cgks_status cgks_kfvs_residual(cgks_ctx* ctx, int level, const double* W, double* res) {
  NEED_MESH();
  if (level < 0 || level >= (int)ctx->L.size() || !W || !res)
    return cgks_fail(ctx, CGKS_EINVAL, "cgks_kfvs_residual: bad level or NULL array");
  CKS(kfvs_residual(ctx, level, W, res));
  return check_device_error(ctx, "cgks_kfvs_residual");
}

cgks_status cgks_kfvs_jvp(cgks_ctx* ctx, int level, const double* W0, const double* dW, double* out) {
  NEED_MESH();
  if (level < 0 || level >= (int)ctx->L.size() || !W0 || !dW || !out)
    return cgks_fail(ctx, CGKS_EINVAL, "cgks_kfvs_jvp: bad level or NULL array");
  CKS(kfvs_jvp(ctx, level, W0, dW, 0, out));
  return check_device_error(ctx, "cgks_kfvs_jvp");
}

static cgks_status run_iterations(cgks_ctx* ctx, int n, double* norm_hist, bool multigrid, const char* name) {
  NEED_STATE();
  if (n < 0) return cgks_fail(ctx, CGKS_EINVAL, "negative iteration count");
  std::vector<void*> tmp;
  double* hist = nullptr;
  if (norm_hist && n > 0) CKS(dalloc(ctx, tmp, &hist, n));
  cgks_status s = CGKS_OK;
  for (int k = 0; k < n && s == CGKS_OK; ++k) s = multigrid ? vcycle_once(ctx, hist ? hist + k : nullptr)
                                                            : step_once(ctx, hist ? hist + k : nullptr);
  if (s == CGKS_OK && hist) s = read_norm(ctx, hist, norm_hist, n);
  free_list(tmp);
  CKS(s);
  ctx->iters += n;
  return check_device_error(ctx, name);
}

cgks_status cgks_step(cgks_ctx* ctx, int n_steps, double* norm_hist) {
  return run_iterations(ctx, n_steps, norm_hist, false, "cgks_step");
}

cgks_status cgks_vcycle(cgks_ctx* ctx, int n_cycles, double* norm_hist) {
  return run_iterations(ctx, n_cycles, norm_hist, true, "cgks_vcycle");
}

// one chunk of n iterations (V-cycles or single-grid steps) enqueued eagerly, the density norm of
// iteration k into hist[k]
static cgks_status enqueue_chunk(cgks_ctx* ctx, bool multigrid, int n, double* hist) {
  for (int k = 0; k < n; ++k) CKS(multigrid ? vcycle_once(ctx, hist + k) : step_once(ctx, hist + k));
  return CGKS_OK;
}

// the same chunk captured once into a CUDA graph (the iterations are launch sequences of fixed shape,
// so small meshes pay one graph launch instead of tens of kernel launches per iteration).  Capture
// and replay run on a private non-blocking stream, ordered after and before the context stream by
// events (the context stream may be the legacy default stream, which cannot be captured).
static cgks_status graph_stream(cgks_ctx* ctx) {
  if (!ctx->gstream) CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
  for (cudaEvent_t& e : ctx->gev)
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return CGKS_OK;
}

// false when capture is not possible; the caller then runs the chunk eagerly
static bool capture_chunk(cgks_ctx* ctx, bool multigrid, int n, double* hist, cudaGraphExec_t* exec) {
  if (graph_stream(ctx) != CGKS_OK) {
    ctx->err.clear();
    return false;
  }
  cudaStream_t user = ctx->stream, gs = ctx->gstream;
  if (cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ctx->stream = gs;
  const cgks_status s = enqueue_chunk(ctx, multigrid, n, hist);
  ctx->stream = user;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(gs, &graph);
  bool ok = s == CGKS_OK && e == cudaSuccess && graph;
  if (ok) ok = cudaGraphInstantiate(exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    *exec = nullptr;
    cudaGetLastError();
    ctx->err.clear();
  }
  return ok;
}

// one replay of the captured chunk, after the work already queued on the context stream and before
// whatever is queued on it next
static cgks_status replay_chunk(cgks_ctx* ctx, cudaGraphExec_t exec) {
  CK(cudaEventRecord(ctx->gev[0], ctx->stream));
  CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
  CK(cudaGraphLaunch(exec, ctx->gstream));
  CK(cudaEventRecord(ctx->gev[1], ctx->gstream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0));
  return CGKS_OK;
}

cgks_status cgks_steady_solve(cgks_ctx* ctx, int multigrid, double drop, int64_t max_iters, int64_t* iters_done,
                              double* final_drop, double* seconds) {
  NEED_STATE();
  if (!(drop > 0.0) || max_iters < 1) return cgks_fail(ctx, CGKS_EINVAL, "drop must be > 0 and max_iters >= 1");
  const int check_every = 10;
  std::vector<void*> tmp;
  double* hist;
  CKS(dalloc(ctx, tmp, &hist, check_every));
  std::vector<double> h(check_every);
  const auto t0 = std::chrono::steady_clock::now();
  double r0 = 0.0, ratio = 1.0;
  int64_t it = 0;
  cgks_status s = CGKS_OK;
  // the first chunk runs eagerly (it builds whatever is built on first use); full chunks after it
  // replay one captured graph, unless kernel timing is on (it records events around each launch)
  cudaGraphExec_t exec = nullptr;
  bool try_graph = !ctx->prof;
  while (it < max_iters && s == CGKS_OK) {
    const int n = (int)std::min<int64_t>(check_every, max_iters - it);
    if (it > 0 && n == check_every && try_graph && !exec) try_graph = capture_chunk(ctx, multigrid != 0, n, hist, &exec);
    if (exec && n == check_every) {
      s = replay_chunk(ctx, exec);
    } else {
      s = enqueue_chunk(ctx, multigrid != 0, n, hist);
    }
    if (s != CGKS_OK) break;
    s = read_norm(ctx, hist, h.data(), n);
    if (s != CGKS_OK) break;
    s = check_device_error(ctx, "cgks_steady_solve");
    if (s != CGKS_OK) break;
    if (it == 0) r0 = h[0];
    it += n;
    ratio = r0 > 0.0 ? h[n - 1] / r0 : 0.0;
    if (ratio <= drop) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  free_list(tmp);
  CKS(s);
  ctx->iters += it;
  if (iters_done) *iters_done = it;
  if (final_drop) *final_drop = ratio;
  if (seconds) *seconds = sec;
  if (ratio > drop) return cgks_fail(ctx, CGKS_ENOTCONV, "steady solve: max_iters reached before the drop");
  return CGKS_OK;
}

cgks_status cgks_coarse_colors(cgks_ctx* ctx, int level, int32_t* colors, int32_t* n_colors) {
  NEED_MESH();
  if (level < 1 || level >= (int)ctx->L.size()) return cgks_fail(ctx, CGKS_EINVAL, "cgks_coarse_colors: bad level");
  return lusgs_color_count(ctx, level, colors, n_colors);
}

cgks_status cgks_skipped_updates(cgks_ctx* ctx, int64_t* count) {
  NEED_STATE();
  if (!count) return cgks_fail(ctx, CGKS_EINVAL, "count is NULL");
  CK(cudaMemcpyAsync(ctx->h_count, ctx->d_skipped, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *count = *ctx->h_count;
  return CGKS_OK;
}


__global__ void k_fma_chain(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

cgks_status cgks_fp64_peak(double* tflops) {
  if (!tflops) return cgks_fail(nullptr, CGKS_EINVAL, "tflops is NULL");
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cgks_fail(nullptr, CGKS_ECUDA, "no CUDA device");
  const int blocks = nsm * 4, threads = 256, iters = 8192;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * threads) != cudaSuccess) return cgks_fail(nullptr, CGKS_ENOMEM, "cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) k_fma_chain<<<blocks, threads>>>(d, iters, 0.999999, 1e-7);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma_chain<<<blocks, threads>>>(d, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return cgks_fail(nullptr, CGKS_ECUDA, cudaGetErrorString(e));
  *tflops = 2.0 * blocks * threads * (double)iters * 8.0 / (best * 1e-3) / 1e12;
  return CGKS_OK;
}

const char* cgks_last_error(const cgks_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
