// Discrete adjoint of the steady compact scheme (an extension of the paper's method: its steady
// problem of Sec. 2.4 and 4 differentiated, not a step the paper takes).
//
// The steady problem has u = (W [5][N], grad W [15][N]) as unknowns and
//   F(u) = ( Res(W, G), Gnew(W, G) - G ) = 0,
// Res the residual of the explicit update and Gnew the Gauss-Green gradient (compression factor
// off).  The chain of one evaluation is  (W, G) -> reconstruction (coefficients rc, time step dt)
// per cell -> gas-kinetic flux per Gauss point (inputs: W and grad W of both sides at the point, dt
// of the face) -> fixed-order sums per cell.  cgks_linearize forms the Jacobian of each link by
// forward-mode duals (the residual's own code on Dual<double>, exact to round-off) and keeps it:
//   Jp [41 x 10][ngp]   per Gauss point
//   Jr [2,220][nc]      per cell: own slot 20 inputs x (50 coefficients, dt); each of up to 6
//                       neighbour slots 5 variables x 4 inputs x 10 coefficients (block diagonal)
// so a transposed product is three memory-bound passes over stored matrices instead of a
// reverse sweep through the flux (about 3.4 kFLOP of FP64 per point).  The transposed product runs
// the chain backwards:
//   k_vjp_points  per point: cotangents of (flux, interface state) from those of (Res, Gnew) of
//                 its two cells, times Jp^T -> cotangents of the point inputs
//   k_vjp_coef    per cell: cotangents of its 50 coefficients and dt from its faces' points
//                 (the transposed evaluation of the polynomial and its gradient)
//   k_vjp_slots   per cell and row group: those times Jr^T -> cotangents of its own (W, G) and one
//                 record per neighbour (32 cells x 16 groups per block, the cells' cotangents in
//                 shared memory)
//   k_vjp_cells   per cell: own part plus the records its neighbours wrote for it
// All sums run in a fixed order (no atomics), so results are reproducible bit for bit.
#include <algorithm>
#include <vector>

#include "adjoint.cuh"

// ---- forward-mode linearisation ----------------------------------------------------------------

__global__ void __launch_bounds__(128) k_point_jac(PointArgs a, double* Jp) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < a.ngp) point_jacobian_body(g, a, Jp);
}

__global__ void __launch_bounds__(128) k_recon_jac(ReconArgs a, double* Jr) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) recon_jacobian_body(i, a, Jr);
}

// ---- transposed product ------------------------------------------------------------------------


__global__ void __launch_bounds__(128) k_vjp_points(VjpArgs a) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < a.ngp) vjp_point_body(g, a);
}

__global__ void __launch_bounds__(128) k_vjp_coef(VjpArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) vjp_coef_body(i, a);
}

// 32 cells x 16 row groups per block: the tile's 51 x 32 cotangents staged in shared memory once,
// every row of the stored matrix read by a warp of 32 consecutive cells
__global__ void __launch_bounds__(512) k_vjp_slots(VjpArgs a) {
  __shared__ double cbs[CGKS_RJ_OUT][32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t i = blockIdx.x * (int64_t)32 + tx;
  for (int o = ty; o < CGKS_RJ_OUT; o += 16) cbs[o][tx] = i < a.nc ? a.cbuf[(int64_t)o * a.nc + i] : 0.0;
  __syncthreads();
  if (i >= a.nc) return;
  for (int g = ty; g < 20 + 6 * 5; g += 16) vjp_slot_body(i, g, a, &cbs[0][tx], 32);
}

// the reconstruction's transposed product recomputed per cell (adjoint_recompute 1), in place of
// k_vjp_slots
__global__ void __launch_bounds__(128) k_vjp_recon(ReconArgs ra, VjpArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) vjp_recon_body(i, ra, a, a.cbuf + i, a.nc);
}

__global__ void __launch_bounds__(128) k_vjp_cells(VjpArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) vjp_cell_body(i, a);
}

// ---- functional, adjoint iteration, reductions ---------------------------------------------------

// wall force J = sum over wall faces (tags 1, 2) of p(W_L) S_comp (S the face's area vector, outward
// from the cell): per-cell share jc and dJ/dW
__global__ void k_wall_force(int64_t nc, int64_t ngp, const int8_t* ctype, const int32_t* cf, const int32_t* fR,
                             const int32_t* ftag, const int32_t* gp_ptr, const double* gp_A, const double* W,
                             double gamma, int comp, double* jc, double* dJdW) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int nt = ctype[i] == 7 ? 5 : ctype[i];
  double S = 0.0;
  for (int m = 0; m < nt; ++m) {
    const int64_t f = cf[(int64_t)m * nc + i];
    if (fR[f] >= 0 || (ftag[f] != 1 && ftag[f] != 2)) continue;
    for (int64_t g = gp_ptr[f]; g < gp_ptr[f + 1]; ++g) S += gp_A[comp * ngp + g];
  }
  const double w0 = W[i], u[3] = {W[nc + i] / w0, W[2 * nc + i] / w0, W[3 * nc + i] / w0};
  const double k2 = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double p = (gamma - 1.0) * (W[4 * nc + i] - w0 * k2);
  jc[i] = p * S;
  if (dJdW) {
    const double dp[5] = {k2, -u[0], -u[1], -u[2], 1.0};
#pragma unroll
    for (int q = 0; q < 5; ++q) dJdW[q * nc + i] = (gamma - 1.0) * dp[q] * S;
  }
}

// v = P mu with P = diag(dt/|Omega|) on the W rows (identity on the G rows, not copied)
__global__ void k_adj_scale(int64_t nc, const double* mu, const double* dt, const double* vol, double* v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const double h = dt[i] / vol[i];
#pragma unroll
  for (int q = 0; q < 5; ++q) v[q * nc + i] = h * mu[q * nc + i];
}

// delta = (F_u)^T P mu + g (the G rows of F_u carry -I); mu += delta; d2[i] = |delta_i|^2
__global__ void k_adj_update(int64_t nc, const double* wbar, const double* g, double* mu, double* d2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 20; ++c) {
    const int64_t k = (int64_t)c * nc + i;
    const double d = wbar[k] + (g ? g[k] : 0.0) - (c >= 5 ? mu[k] : 0.0);
    mu[k] += d;
    s += d * d;
  }
  d2[i] = s;
}

// d2[i] = sum over the 20 rows of x[c][i]^2
__global__ void k_sq_rows(int64_t nc, const double* x, double* d2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s = 0.0;
  for (int c = 0; c < 20; ++c) s += x[(int64_t)c * nc + i] * x[(int64_t)c * nc + i];
  d2[i] = s;
}

// lambda = P mu
__global__ void k_adj_lambda(int64_t nc, const double* mu, const double* dt, const double* vol, double* lam) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const double h = dt[i] / vol[i];
#pragma unroll
  for (int c = 0; c < 20; ++c) lam[(int64_t)c * nc + i] = (c < 5 ? h : 1.0) * mu[(int64_t)c * nc + i];
}

// x[i] = sum_c a[c][i] (b+[c][i] - b-[c][i]) over the 20 rows
__global__ void k_adj_dot_rows(int64_t nc, const double* a, const double* bp, const double* bm, double* x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s = 0.0;
  for (int c = 0; c < 20; ++c) s += a[(int64_t)c * nc + i] * (bp[(int64_t)c * nc + i] - bm[(int64_t)c * nc + i]);
  x[i] = s;
}

// GMRES helpers over [20][nc] vectors: y = a x + b y; per-cell dot products d[i] = sum_c x y;
// y = wbar - (0 on the W rows, x on the G rows) (the -I of Gnew - G)
__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) y[k] = a * x[k] + b * y[k];
}

__global__ void k_dot_rows(int64_t nc, const double* x, const double* y, double* d) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s = 0.0;
  for (int c = 0; c < 20; ++c) s += x[(int64_t)c * nc + i] * y[(int64_t)c * nc + i];
  d[i] = s;
}

__global__ void k_mv_finish(int64_t nc, const double* wbar, const double* x, double* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  for (int c = 0; c < 20; ++c) {
    const int64_t k = (int64_t)c * nc + i;
    y[k] = wbar[k] - (c >= 5 ? x[k] : 0.0);
  }
}

// fixed-order sum: 304 block partials over a grid-stride loop, then one block
__global__ void k_sum_partial(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double s[256];
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) v += x[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_sum_final(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < nparts; ++k) v += part[k];
    *out = v;
  }
}

static constexpr int kSumParts = 304;

static cgks_status device_sum(cgks_ctx* ctx, const double* x, int64_t n, double* host_out) {
  k_sum_partial<<<kSumParts, 256, 0, ctx->stream>>>(n, x, ctx->apart);
  k_sum_final<<<1, 32, 0, ctx->stream>>>(kSumParts, ctx->apart, ctx->apart + kSumParts);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(host_out, ctx->apart + kSumParts, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

static constexpr int kGmresM = 30;  // Krylov vectors per restart

// the functional's per-cell shares and the reduction partials (small: the wall force needs no more)
static cgks_status small_buffers(cgks_ctx* ctx) {
  if (ctx->ajc) return CGKS_OK;
  CKS(dalloc(ctx, ctx->mesh_allocs, &ctx->apart, kSumParts + 1));
  CKS(dalloc(ctx, ctx->mesh_allocs, &ctx->ajc, ctx->F.nc));
  return CGKS_OK;
}

static cgks_status adjoint_buffers(cgks_ctx* ctx) {
  CKS(small_buffers(ctx));
  if (ctx->pbar) return CGKS_OK;
  const Fine& F = ctx->F;
  auto& M = ctx->mesh_allocs;
  CKS(dalloc(ctx, M, &ctx->Jp, (size_t)CGKS_PJ_IN * CGKS_PJ_OUT * F.ngp));
  CKS(dalloc(ctx, M, &ctx->adt, F.nc));
  CKS(dalloc(ctx, M, &ctx->pbar, (size_t)CGKS_PB * F.ngp));
  CKS(dalloc(ctx, M, &ctx->aself, (size_t)20 * F.nc));
  CKS(dalloc(ctx, M, &ctx->arec, (size_t)20 * 2 * F.nf));
  CKS(dalloc(ctx, M, &ctx->acb, (size_t)CGKS_RJ_OUT * F.nc));
  // work vectors: mu, v, wbar, g, lambda, F+, F- (20 rows each) and one row of per-cell scalars
  CKS(dalloc(ctx, M, &ctx->avec, (size_t)(7 * 20 + 1) * F.nc));
  return CGKS_OK;
}

// the reconstruction's inputs at the linearisation point (adjoint_recompute 1): the copy of (W, grad W,
// alpha) that cgks_linearize keeps
static ReconArgs lin_recon_args(cgks_ctx* ctx) {
  const Fine& F = ctx->F;
  const int64_t nc = F.nc;
  return ReconArgs{F.nc, F.nf, F.ctype, F.cf, F.fL, F.fR, F.ftag, F.cside, F.fnrm, F.Kop, F.ggw, F.lsw, F.aux, F.dtw,
                   F.vol, ctx->aWG, ctx->aWG + 5 * nc, ctx->aWG + 20 * nc, nullptr, nullptr, make_phys(ctx->P), ctx->derr};
}

static cgks_status run_vjp(cgks_ctx* ctx, const double* rbar, const double* gbar, double* out) {
  const Fine& F = ctx->F;
  VjpArgs va{F.nc, F.nf, F.ngp, F.ctype, F.cside, F.cf, F.fL, F.fR, F.gp_face, F.gp_ptr, F.gp_x, F.gp_A, F.fshift,
             F.ctr, F.vol, ctx->adt, ctx->Jp, ctx->Jr, rbar, gbar, ctx->pbar, ctx->aself, ctx->arec, ctx->acb, out};
  k_vjp_points<<<grid_for(F.ngp, 128), 128, 0, ctx->stream>>>(va);
  k_vjp_coef<<<grid_for(F.nc, 128), 128, 0, ctx->stream>>>(va);
  if (ctx->lin_recompute)
    k_vjp_recon<<<grid_for(F.nc, 128), 128, 0, ctx->stream>>>(lin_recon_args(ctx), va);
  else
    k_vjp_slots<<<grid_for(F.nc, 32), dim3(32, 16), 0, ctx->stream>>>(va);
  k_vjp_cells<<<grid_for(F.nc, 128), 128, 0, ctx->stream>>>(va);
  CK(cudaGetLastError());
  return CGKS_OK;
}

static cgks_status adjoint_supported(cgks_ctx* ctx, const char* where) {
  if (!ctx) return CGKS_EINVAL;
  if (!ctx->has_mesh || !ctx->has_state) return cgks_fail(ctx, CGKS_EINVAL, std::string(where) + ": no mesh or state");
  if (ctx->P.compression_factor != 0)
    return cgks_fail(ctx, CGKS_EUNSUPPORTED, std::string(where) + ": the adjoint needs compression_factor = 0");
  if (ctx->P.dt_mode != 0)
    return cgks_fail(ctx, CGKS_EUNSUPPORTED, std::string(where) + ": the adjoint needs local time steps (dt_mode 0)");
  return CGKS_OK;
}

// ---- C ABI --------------------------------------------------------------------------------------

cgks_status cgks_linearize(cgks_ctx* ctx) {
  CKS(adjoint_supported(ctx, "cgks_linearize"));
  CKS(adjoint_buffers(ctx));
  const Fine& F = ctx->F;
  const Phys ph = make_phys(ctx->P);
  CKS(fine_fluxes(ctx, ctx->W, ctx->G, ctx->alpha));  // coefficients and time steps at the state
  ReconArgs ra{F.nc, F.nf, F.ctype, F.cf, F.fL, F.fR, F.ftag, F.cside, F.fnrm, F.Kop, F.ggw, F.lsw, F.aux, F.dtw,
               F.vol, ctx->W, ctx->G, ctx->alpha, ctx->rc, ctx->dt, ph, ctx->derr};
  ctx->lin_recompute = ctx->P.adjoint_recompute != 0;
  if (ctx->lin_recompute) {
    // keep the state; the reconstruction's transposed product is recomputed from it in every product
    if (!ctx->aWG) CKS(dalloc(ctx, ctx->mesh_allocs, &ctx->aWG, (size_t)21 * F.nc));
    CK(cudaMemcpyAsync(ctx->aWG, ctx->W, sizeof(double) * 5 * F.nc, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->aWG + 5 * F.nc, ctx->G, sizeof(double) * 15 * F.nc, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->aWG + 20 * F.nc, ctx->alpha, sizeof(double) * F.nc, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    if (!ctx->Jr) CKS(dalloc(ctx, ctx->mesh_allocs, &ctx->Jr, (size_t)CGKS_RJ_ROWS * F.nc));
    k_recon_jac<<<grid_for(F.nc, 128), 128, 0, ctx->stream>>>(ra, ctx->Jr);
  }
  PointArgs pa{F.ngp, F.nf, F.nc, F.gp_face, F.fL, F.fR, F.ftag, F.gp_x, F.gp_A, F.fshift, F.ctr, ctx->rc,
               ctx->dt, ctx->gpr, ph, ctx->derr};
  k_point_jac<<<grid_for(F.ngp, 128), 128, 0, ctx->stream>>>(pa, ctx->Jp);
  CK(cudaMemcpyAsync(ctx->adt, ctx->dt, sizeof(double) * F.nc, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaGetLastError());
  CKS(check_device_error(ctx, "cgks_linearize"));
  ctx->linearized = true;
  return CGKS_OK;
}

cgks_status cgks_residual_vjp(cgks_ctx* ctx, const double* res_bar, const double* grad_bar, double* W_bar,
                              double* G_bar) {
  if (!ctx) return CGKS_EINVAL;
  if (!ctx->linearized) return cgks_fail(ctx, CGKS_EINVAL, "cgks_residual_vjp: call cgks_linearize first");
  if (!res_bar || !grad_bar || !W_bar || !G_bar) return cgks_fail(ctx, CGKS_EINVAL, "cgks_residual_vjp: NULL array");
  const int64_t nc = ctx->F.nc;
  double* out = ctx->avec + 2 * 20 * nc;  // wbar
  CKS(run_vjp(ctx, res_bar, grad_bar, out));
  CK(cudaMemcpyAsync(W_bar, out, sizeof(double) * 5 * nc, cudaMemcpyDefault, ctx->stream));
  CK(cudaMemcpyAsync(G_bar, out + 5 * nc, sizeof(double) * 15 * nc, cudaMemcpyDefault, ctx->stream));
  return check_device_error(ctx, "cgks_residual_vjp");
}

cgks_status cgks_wall_force(cgks_ctx* ctx, int component, double* J, double* dJ_dW) {
  if (!ctx) return CGKS_EINVAL;
  if (!ctx->has_mesh || !ctx->has_state) return cgks_fail(ctx, CGKS_EINVAL, "cgks_wall_force: no mesh or state");
  if (component < 0 || component > 2 || !J) return cgks_fail(ctx, CGKS_EINVAL, "cgks_wall_force: bad arguments");
  CKS(small_buffers(ctx));
  const Fine& F = ctx->F;
  double* jc = ctx->ajc;
  k_wall_force<<<grid_for(F.nc, 128), 128, 0, ctx->stream>>>(F.nc, F.ngp, F.ctype, F.cf, F.fR, F.ftag, F.gp_ptr, F.gp_A,
                                                             ctx->W, ctx->P.gamma, component, jc, dJ_dW);
  CK(cudaGetLastError());
  CKS(device_sum(ctx, jc, F.nc, J));
  return check_device_error(ctx, "cgks_wall_force");
}

// M x = (dF/du)^T P x: the operator of the adjoint system in the variable mu (lambda = P mu)
static cgks_status adjoint_matvec(cgks_ctx* ctx, const double* x, double* y) {
  const Fine& F = ctx->F;
  const int64_t nc = F.nc;
  double *v = ctx->avec + 20 * nc, *wbar = v + 20 * nc;
  k_adj_scale<<<grid_for(nc, 128), 128, 0, ctx->stream>>>(nc, x, ctx->adt, F.vol, v);
  CKS(run_vjp(ctx, v, x + 5 * nc, wbar));
  k_mv_finish<<<grid_for(nc, 128), 128, 0, ctx->stream>>>(nc, wbar, x, y);
  CK(cudaGetLastError());
  return CGKS_OK;
}

static cgks_status dot(cgks_ctx* ctx, const double* x, const double* y, double* out) {
  const int64_t nc = ctx->F.nc;
  double* d = ctx->avec + 7 * 20 * nc;
  k_dot_rows<<<grid_for(nc, 128), 128, 0, ctx->stream>>>(nc, x, y, d);
  return device_sum(ctx, d, nc, out);
}

// restarted GMRES(kGmresM) on M mu = -g (modified Gram-Schmidt Arnoldi, Givens rotations); the
// residual it reports is that of the adjoint system, |M mu + g| / |g|
static cgks_status gmres(cgks_ctx* ctx, double* mu, const double* g, double gn, int64_t max_iters, double tol,
                         int64_t* it_out, double* rel_out) {
  const int64_t nc = ctx->F.nc, n = 20 * nc;
  cudaStream_t st = ctx->stream;
  double* V = ctx->akry;
  const int m = kGmresM;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), sv(m + 1), yv(m);
  int64_t it = 0;
  double rel = 1.0;
  bool first = true;
  const unsigned gb = grid_for(n, 256);
  for (;;) {
    // true residual r = -g - M mu into V_0
    if (first) {
      k_axpby<<<gb, 256, 0, st>>>(n, -1.0, g, 0.0, V);
    } else {
      CKS(adjoint_matvec(ctx, mu, V));
      ++it;
      k_axpby<<<gb, 256, 0, st>>>(n, -1.0, g, -1.0, V);
    }
    first = false;
    double b2 = 0.0;
    CKS(dot(ctx, V, V, &b2));
    const double beta = sqrt(b2);
    rel = beta / gn;
    if (!(rel <= 1e300)) return cgks_fail(ctx, CGKS_ENAN, "cgks_adjoint_solve: GMRES diverged");
    if (rel <= tol || it >= max_iters) break;
    k_axpby<<<gb, 256, 0, st>>>(n, 0.0, V, 1.0 / beta, V);
    std::fill(sv.begin(), sv.end(), 0.0);
    sv[0] = beta;
    int k = 0;
    for (int j = 0; j < m && it < max_iters; ++j) {
      double* vj = V + (int64_t)j * n;
      double* w = V + (int64_t)(j + 1) * n;
      CKS(adjoint_matvec(ctx, vj, w));
      ++it;
      for (int i = 0; i <= j; ++i) {
        double h = 0.0;
        CKS(dot(ctx, w, V + (int64_t)i * n, &h));
        H[i * m + j] = h;
        k_axpby<<<gb, 256, 0, st>>>(n, -h, V + (int64_t)i * n, 1.0, w);
      }
      double w2 = 0.0;
      CKS(dot(ctx, w, w, &w2));
      const double hn = sqrt(w2);
      H[(j + 1) * m + j] = hn;
      if (hn > 0.0) k_axpby<<<gb, 256, 0, st>>>(n, 0.0, w, 1.0 / hn, w);
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = den > 0.0 ? H[j * m + j] / den : 1.0;
      sn[j] = den > 0.0 ? H[(j + 1) * m + j] / den : 0.0;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      sv[j + 1] = -sn[j] * sv[j];
      sv[j] = cs[j] * sv[j];
      k = j + 1;
      if (fabs(sv[j + 1]) <= tol * gn || hn == 0.0) break;
    }
    // mu += V y with H y = s (upper triangular)
    for (int i = k - 1; i >= 0; --i) {
      double t = sv[i];
      for (int l = i + 1; l < k; ++l) t -= H[i * m + l] * yv[l];
      yv[i] = H[i * m + i] != 0.0 ? t / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < k; ++i) k_axpby<<<gb, 256, 0, st>>>(n, yv[i], V + (int64_t)i * n, 1.0, mu);
    CK(cudaGetLastError());
  }
  *it_out = it;
  *rel_out = rel;
  return CGKS_OK;
}

cgks_status cgks_adjoint_solve(cgks_ctx* ctx, const double* dJ_du, int method, int64_t max_iters, double tol,
                               double* lambda, int64_t* iters, double* rel_res) {
  if (!ctx) return CGKS_EINVAL;
  if (!ctx->linearized) return cgks_fail(ctx, CGKS_EINVAL, "cgks_adjoint_solve: call cgks_linearize first");
  if (!dJ_du || !lambda || max_iters < 1 || !(tol > 0.0) || (method != 0 && method != 1))
    return cgks_fail(ctx, CGKS_EINVAL, "cgks_adjoint_solve: bad arguments");
  const Fine& F = ctx->F;
  const int64_t nc = F.nc;
  cudaStream_t st = ctx->stream;
  double *mu = ctx->avec, *v = mu + 20 * nc, *wbar = v + 20 * nc, *g = wbar + 20 * nc, *d2 = ctx->avec + 7 * 20 * nc;
  CK(cudaMemcpyAsync(g, dJ_du, sizeof(double) * 20 * nc, cudaMemcpyDefault, st));
  CK(cudaMemsetAsync(mu, 0, sizeof(double) * 20 * nc, st));
  // |g|^2
  double g2 = 0.0;
  k_sq_rows<<<grid_for(nc, 128), 128, 0, st>>>(nc, g, d2);
  CKS(device_sum(ctx, d2, nc, &g2));
  const double gn = sqrt(g2);
  int64_t it = 0;
  double rel = 1.0;
  if (!(gn > 0.0)) {
    rel = 0.0;
  } else if (method == 1) {
    if (!ctx->akry) CKS(dalloc(ctx, ctx->mesh_allocs, &ctx->akry, (size_t)(kGmresM + 1) * 20 * nc));
    CKS(gmres(ctx, mu, g, gn, max_iters, tol, &it, &rel));
  } else {
    const int check = 25;
    while (it < max_iters) {
      k_adj_scale<<<grid_for(nc, 128), 128, 0, st>>>(nc, mu, ctx->adt, F.vol, v);
      CKS(run_vjp(ctx, v, mu + 5 * nc, wbar));
      k_adj_update<<<grid_for(nc, 128), 128, 0, st>>>(nc, wbar, g, mu, d2);
      ++it;
      if (it % check == 0 || it == max_iters) {
        double r2 = 0.0;
        CKS(device_sum(ctx, d2, nc, &r2));
        rel = sqrt(r2) / gn;
        if (!(rel <= 1e300)) return cgks_fail(ctx, CGKS_ENAN, "cgks_adjoint_solve: the iteration diverged");
        if (rel <= tol) break;
      }
    }
  }
  k_adj_lambda<<<grid_for(nc, 128), 128, 0, st>>>(nc, mu, ctx->adt, F.vol, v);
  CK(cudaMemcpyAsync(lambda, v, sizeof(double) * 20 * nc, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  if (iters) *iters = it;
  if (rel_res) *rel_res = rel;
  CKS(check_device_error(ctx, "cgks_adjoint_solve"));
  return rel <= tol ? CGKS_OK : cgks_fail(ctx, CGKS_ENOTCONV, "cgks_adjoint_solve: tolerance not reached");
}

// F(u) = (Res, Gnew) of the fine residual at the current state into out [20][nc] (the -G of the
// steady problem cancels in the differences it is used for)
static cgks_status fine_F(cgks_ctx* ctx, double* out) {
  const int64_t nc = ctx->F.nc;
  CKS(fine_fluxes(ctx, ctx->W, ctx->G, ctx->alpha));
  CKS(fine_gather(ctx, ctx->W, nullptr, out, out + 5 * nc, nullptr, 0));
  return CGKS_OK;
}

// lambda . (F+ - F-) / (2 h) with F+- the residual of a context whose mesh is ctx's with the nodes
// moved by +-h field (shape derivative at the frozen state), plus the change of J
static cgks_status shape_partial(cgks_ctx* ctx, int component, const double* field, double h, const double* lam,
                                 double* out) {
  const int64_t nc = ctx->F.nc, nn = (int64_t)ctx->h_xyz.size() / 3;
  double* Fpm[2] = {ctx->avec + 5 * 20 * nc, ctx->avec + 6 * 20 * nc};
  double J[2] = {0.0, 0.0};
  cgks_params P1 = ctx->P;
  P1.n_levels = 1;
  std::vector<double> xyz(ctx->h_xyz.size());
  for (int s = 0; s < 2; ++s) {
    const double e = s == 0 ? h : -h;
    for (size_t k = 0; k < xyz.size(); ++k) xyz[k] = ctx->h_xyz[k] + e * field[k];
    cgks_ctx* t = nullptr;
    CKS(cgks_create(&P1, ctx->stream, &t));
    const int64_t nb = (int64_t)ctx->h_btag.size(), np = (int64_t)ctx->h_pairs.size() / 2;
    cgks_status r = cgks_mesh_upload(t, nn, xyz.data(), nc, ctx->h_ctype.data(), ctx->h_cptr.data(), ctx->h_cnodes.data(),
                                     nb, nb ? ctx->h_bptr.data() : nullptr, nb ? ctx->h_bnodes.data() : nullptr,
                                     nb ? ctx->h_btag.data() : nullptr, np ? ctx->h_pairs.data() : nullptr, np);
    if (r == CGKS_OK) r = cgks_state_init(t, ctx->W, ctx->G, ctx->alpha);
    if (r == CGKS_OK) r = fine_F(t, Fpm[s]);
    if (r == CGKS_OK) r = cgks_wall_force(t, component, &J[s], nullptr);
    if (r == CGKS_OK) {
      cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
      if (e2 != cudaSuccess) r = cgks_fail(ctx, CGKS_ECUDA, cudaGetErrorString(e2));
    }
    if (r != CGKS_OK) {
      std::string msg = std::string("shape derivative: ") + t->err;
      cgks_destroy(t);
      return cgks_fail(ctx, r, msg);
    }
    cgks_destroy(t);
  }
  double* x = ctx->avec + 7 * 20 * nc;
  k_adj_dot_rows<<<grid_for(nc, 128), 128, 0, ctx->stream>>>(nc, lam, Fpm[0], Fpm[1], x);
  CK(cudaGetLastError());
  double dot = 0.0;
  CKS(device_sum(ctx, x, nc, &dot));
  *out = (J[0] - J[1]) / (2.0 * h) + dot / (2.0 * h);
  return CGKS_OK;
}

cgks_status cgks_adjoint(cgks_ctx* ctx, int component, const double* node_modes, int n_modes, double h_mode,
                         double h_mach, int method, int64_t max_iters, double tol, double* dJ_dmodes,
                         double* dJ_dmach, int64_t* iters, double* rel_res) {
  CKS(adjoint_supported(ctx, "cgks_adjoint"));
  if (component < 0 || component > 2 || n_modes < 0 || (n_modes && (!node_modes || !dJ_dmodes || !(h_mode > 0.0))) ||
      !dJ_dmach || !(h_mach > 0.0))
    return cgks_fail(ctx, CGKS_EINVAL, "cgks_adjoint: bad arguments");
  const int64_t nc = ctx->F.nc;
  cudaStream_t st = ctx->stream;
  CKS(adjoint_buffers(ctx));
  // dJ/du at the current state (W rows from the wall cells; G rows zero)
  double* dJdu = ctx->avec + 4 * 20 * nc;  // the lambda slot doubles as dJ/du until the solve
  CK(cudaMemsetAsync(dJdu, 0, sizeof(double) * 20 * nc, st));
  double J = 0.0;
  CKS(cgks_wall_force(ctx, component, &J, dJdu));
  CKS(cgks_linearize(ctx));
  double* lam_d = dJdu;  // the solve copies dJ/du out before it writes lambda here
  CKS(cgks_adjoint_solve(ctx, dJdu, method, max_iters, tol, lam_d, iters, rel_res));
  // Mach: the free stream (boundary states, viscosity) moves, the flow state stays
  double* Fpm[2] = {ctx->avec + 5 * 20 * nc, ctx->avec + 6 * 20 * nc};
  const cgks_params P0 = ctx->P;
  for (int s = 0; s < 2; ++s) {
    ctx->P.mach = P0.mach + (s == 0 ? h_mach : -h_mach);
    cgks_status r = fine_F(ctx, Fpm[s]);
    if (r != CGKS_OK) {
      ctx->P = P0;
      return r;
    }
  }
  ctx->P = P0;
  double* x = ctx->avec + 7 * 20 * nc;
  k_adj_dot_rows<<<grid_for(nc, 128), 128, 0, st>>>(nc, lam_d, Fpm[0], Fpm[1], x);
  CK(cudaGetLastError());
  double dot = 0.0;
  CKS(device_sum(ctx, x, nc, &dot));
  *dJ_dmach = dot / (2.0 * h_mach);
  // node displacement modes
  const size_t nn3 = ctx->h_xyz.size();
  for (int m = 0; m < n_modes; ++m) {
    CKS(shape_partial(ctx, component, node_modes + (size_t)m * nn3, h_mode, lam_d, &dJ_dmodes[m]));
  }
  // leave the fine work arrays as a residual evaluation at the state would
  CKS(fine_fluxes(ctx, ctx->W, ctx->G, ctx->alpha));
  return check_device_error(ctx, "cgks_adjoint");
}
