// Kernels of the fine-level CGKS residual (bodies in fine.cuh) and their host launchers.
#include "fine.cuh"

__global__ void __launch_bounds__(128, 4) k_reconstruct(ReconArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc) reconstruct_body(i, a);
}

template <bool STATE>
__global__ void __launch_bounds__(128) k_gks_points(PointArgs a) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < a.ngp) gks_point_body<STATE>(g, a);
}

// ---- gather: per cell, fixed-order sums of its faces' Gauss-point records ----------------------
//
// One thread per cell, 32 cells per warp.  The records of a face are contiguous (3 or 4 records of
// 112 bytes), so for each local-face slot the warp copies the 32 faces' records into shared memory
// with 16-byte cp.async copies, lanes of one copy instruction covering one face's contiguous bytes
// (coalesced), and each thread then sums its own face from shared memory in ascending point order
// (gather_face, the same arithmetic and order as gather_body).  The copies of slot m + 1 are in
// flight while slot m is summed (two buffers per warp).  GRAD false (residual only): the first three
// chunks of each record (the flux) are copied.

#define GATHER_WARPS 2                      // warps per block
#define GATHER_FACE_DOUBLES (4 * CGKS_GPR)  // room for the records of one face: 448 bytes
#define GATHER_SMEM (GATHER_WARPS * 2 * 32 * GATHER_FACE_DOUBLES * (int)sizeof(double))

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <bool GRAD>
__global__ void __launch_bounds__(32 * GATHER_WARPS) k_gather(GatherArgs a) {
  constexpr int CH = GRAD ? CGKS_GPR / 2 : 3;  // 16-byte chunks copied per record
  extern __shared__ __align__(16) double gsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nc = a.nc;
  const int64_t i = ((int64_t)blockIdx.x * GATHER_WARPS + w) * 32 + lane;
  const bool valid = i < nc;
  const int nt = valid ? (a.ctype[i] == 7 ? 5 : a.ctype[i]) : 0;  // pyramids (type 7) have 5 faces
  const int nmax = __reduce_max_sync(0xffffffffu, nt);
  double* const buf0 = gsm + (size_t)(2 * w) * 32 * GATHER_FACE_DOUBLES;  // buffers of slots 0, 2, 4
  double* const buf1 = buf0 + 32 * GATHER_FACE_DOUBLES;                    // and of slots 1, 3, 5
  // face slot m of this lane's cell: first record, number of records, side sign
  auto slot = [&](int m, int64_t& g0, int& ng, bool& sg) {
    g0 = 0;
    ng = 0;
    sg = false;
    if (m < nt) {
      const int64_t f = a.cf[(int64_t)m * nc + i];
      sg = a.cside[(int64_t)m * nc + i] != 0;
      g0 = a.gp_ptr[f];
      ng = (int)(a.gp_ptr[f + 1] - g0);
    }
  };
  // the 32 faces of one slot into buffer b: chunk c of record k of face j by lane k CH + c, each to
  // its offset within the face's records (lanes 0 .. CH ng - 1; CH ng <= 28)
  const int rk = lane / CH, rc = lane - rk * CH;
  const int off = CGKS_GPR * rk + 2 * rc;
  auto issue = [&](double* b, int64_t g0, int ng) {
    for (int j = 0; j < 32; ++j) {
      const int64_t gj = __shfl_sync(0xffffffffu, g0, j);
      const int nj = __shfl_sync(0xffffffffu, ng, j);
      if (rk < nj) cp_async16(b + j * GATHER_FACE_DOUBLES + off, a.gpr + CGKS_GPR * gj + off);
    }
    cp_async_commit();
  };
  GatherAcc c;
  gather_init(c);
  int64_t g0;
  int ng;
  bool sg;
  slot(0, g0, ng, sg);
  if (nmax > 0) issue(buf0, g0, ng);
  for (int m = 0; m < nmax; ++m) {
    int64_t g1 = 0;
    int n1 = 0;
    bool s1 = false;
    if (m + 1 < nmax) {
      slot(m + 1, g1, n1, s1);
      issue((m & 1) ? buf0 : buf1, g1, n1);
    } else {
      cp_async_commit();  // an empty group keeps "all but the newest group" meaning slot m
    }
    cp_async_wait_one();
    __syncwarp();
    if (ng > 0) gather_face<GRAD>(((m & 1) ? buf1 : buf0) + lane * GATHER_FACE_DOUBLES, ng, sg, c);
    __syncwarp();  // every lane is done with buffer m & 1 before slot m + 2 is copied into it
    g0 = g1;
    ng = n1;
    sg = s1;
  }
  if (valid) gather_store(i, a, c);
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

cgks_status fine_fluxes(cgks_ctx* ctx, const double* W, const double* G, const double* alpha, bool state) {
  const Fine& F = ctx->F;
  const Phys ph = make_phys(ctx->P);
  ReconArgs ra{F.nc, F.nf, F.ctype, F.cf, F.fL, F.fR, F.ftag, F.cside, F.fnrm, F.Kop, F.ggw, F.lsw, F.aux, F.dtw,
               F.vol, W, G, alpha, ctx->rc, ctx->dt, ph, ctx->derr};
  const double slots = (double)(F.nf + F.n_int + F.n_per);
  {
    ProfScope ps(ctx, PK_RECON, (double)F.nc, F.nc * (306.0 * 8 + 1 + 51.0 * 8) + slots * 5 + F.nf * 36.0);
    const int b = spread_block(F.nc, 128, ctx->n_sm);
    k_reconstruct<<<grid_for(F.nc, b), b, 0, ctx->stream>>>(ra);
  }
  if (ctx->P.dt_mode == 1) CKS(global_min_dt(ctx, ctx->dt, F.nc));
  PointArgs pa{F.ngp, F.nf, F.nc, F.gp_face, F.fL, F.fR, F.ftag, F.gp_x, F.gp_A, F.fshift, F.ctr, ctx->rc,
               ctx->dt, ctx->gpr, ph, ctx->derr};
  {
    ProfScope ps(ctx, state ? PK_POINTS : PK_POINTS_FLUX, (double)F.ngp,
                 F.ngp * (52.0 + (state ? 8.0 * CGKS_GPR : 40.0)) + F.nf * 36.0 + F.nc * 432.0);
    const int b = spread_block(F.ngp, 128, ctx->n_sm);
    if (state)
      k_gks_points<true><<<grid_for(F.ngp, b), b, 0, ctx->stream>>>(pa);
    else
      k_gks_points<false><<<grid_for(F.ngp, b), b, 0, ctx->stream>>>(pa);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

cgks_status fine_gather(cgks_ctx* ctx, const double* W_in, double* W_out, double* res, double* G_out,
                        double* alpha_out, int update) {
  const Fine& F = ctx->F;
  GatherArgs ga{F.nc, F.ngp, F.ctype, F.cside, F.cf, F.gp_ptr, ctx->gpr, F.vol,
                ctx->dt, W_in, W_out, res, G_out, alpha_out, update, ctx->P.gamma, ctx->derr};
  {
    // the residual alone (no gradient, compression factor or update): only the records' fluxes are read
    const bool grad = G_out || alpha_out || update;
    const double per_cell = 1 + 8 + (update ? 88 : 0) + (res ? 40 : 0) + (G_out ? 120 : 0) + (alpha_out ? 8 : 0);
    ProfScope ps(ctx, grad ? PK_GATHER : PK_GATHER_RES, (double)F.gp_sides,
                 F.nc * per_cell + (F.nf + F.n_int + F.n_per) * 5.0 + F.nf * 4.0 + F.ngp * (grad ? 8.0 * CGKS_GPR : 40.0));
    static bool smem_set = false;  // the kernel's dynamic shared memory exceeds the 48 KiB default
    if (!smem_set) {
      CK(cudaFuncSetAttribute(k_gather<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, GATHER_SMEM));
      CK(cudaFuncSetAttribute(k_gather<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, GATHER_SMEM));
      smem_set = true;
    }
    const int64_t per_block = 32 * GATHER_WARPS;
    const unsigned nb = (unsigned)((F.nc + per_block - 1) / per_block);
    if (grad)
      k_gather<true><<<nb, 32 * GATHER_WARPS, GATHER_SMEM, ctx->stream>>>(ga);
    else
      k_gather<false><<<nb, 32 * GATHER_WARPS, GATHER_SMEM, ctx->stream>>>(ga);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}
