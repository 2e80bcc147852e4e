// Kernels of the fine-level CGKS residual (bodies in fine.cuh) and their host launchers.
#include "fine.cuh"

__global__ void __launch_bounds__(128) k_reconstruct(ReconArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) reconstruct_body(i, a);
}

__global__ void __launch_bounds__(128) k_gks_points(PointArgs a) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < a.ngp) gks_point_body(g, a);
}

__global__ void __launch_bounds__(128) k_gather(GatherArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) gather_body(i, a);
}

// global minimum time step (dt_mode 1): fixed-order two-stage reduction, then broadcast
__global__ void k_min_partial(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double s[256];
  double v = 1e300;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v = fmin(v, x[i]);
  s[threadIdx.x] = v;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_min_broadcast(int64_t n, int nparts, const double* __restrict__ part, double* __restrict__ x) {
  __shared__ double mn;
  if (threadIdx.x == 0) {
    double v = 1e300;
    for (int k = 0; k < nparts; ++k) v = fmin(v, part[k]);
    mn = v;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = mn;
}

cgks_status global_min_dt(cgks_ctx* ctx, double* dt, int64_t n) {
  const int parts = 304;
  k_min_partial<<<parts, 256, 0, ctx->stream>>>(n, dt, ctx->nrm_part);
  k_min_broadcast<<<parts, 256, 0, ctx->stream>>>(n, parts, ctx->nrm_part, dt);
  CK(cudaGetLastError());
  return CGKS_OK;
}

cgks_status fine_fluxes(cgks_ctx* ctx, const double* W, const double* G, const double* alpha) {
  const Fine& F = ctx->F;
  const Phys ph = make_phys(ctx->P);
  ReconArgs ra{F.nc, F.nf, F.ctype, F.cf, F.fL, F.fR, F.ftag, F.cside, F.fnrm, F.Kop, F.ggw, F.lsw, F.aux, F.dtw,
               F.vol, W, G, alpha, ctx->rc, ctx->dt, ph, ctx->derr};
  {
    ProfScope ps(ctx, 1);
    k_reconstruct<<<grid_for(F.nc, 128), 128, 0, ctx->stream>>>(ra);
  }
  if (ctx->P.dt_mode == 1) CKS(global_min_dt(ctx, ctx->dt, F.nc));
  PointArgs pa{F.ngp, F.nf, F.nc, F.gp_face, F.fL, F.fR, F.ftag, F.gp_x, F.gp_A, F.fshift, F.ctr, ctx->rc,
               ctx->dt, ctx->gpF, ctx->gpW, ctx->gpa, ph, ctx->derr};
  {
    ProfScope ps(ctx, 0);
    k_gks_points<<<grid_for(F.ngp, 128), 128, 0, ctx->stream>>>(pa);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

cgks_status fine_gather(cgks_ctx* ctx, const double* W_in, double* W_out, double* res, double* G_out,
                        double* alpha_out, int update) {
  const Fine& F = ctx->F;
  GatherArgs ga{F.nc, F.ngp, F.ctype, F.cside, F.cf, F.gp_ptr, F.gp_A, ctx->gpF, ctx->gpW, ctx->gpa, F.vol,
                ctx->dt, W_in, W_out, res, G_out, alpha_out, update, ctx->P.gamma, ctx->derr};
  {
    ProfScope ps(ctx, 2);
    k_gather<<<grid_for(F.nc, 128), 128, 0, ctx->stream>>>(ga);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}
