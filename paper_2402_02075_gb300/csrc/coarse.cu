// Coarse levels of the V-cycle (Sec. 4.2 of the paper): first-order KFVS residual, local time
// steps, FAS forcing and forward-Euler smoothing, volume-weighted state restriction, summed
// residual restriction, injection correction, and the residual norm.  All sums run in a fixed
// order (no floating-point atomics), so results are bitwise reproducible.
#include "internal.cuh"
#include "kinetic.cuh"

// KFVS face fluxes x area (FP64)
__global__ void k_kfvs_faces(int64_t nf, const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                             const int32_t* __restrict__ ftag, const double* __restrict__ nS, int64_t nc,
                             const double* __restrict__ W, double* __restrict__ ff, Phys ph, DevErr* err) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const double s = nS[3 * nf + f];
  if (s == 0.0) {  // a coarse face whose summed area vectors cancel carries no flux
#pragma unroll
    for (int q = 0; q < 5; ++q) ff[q * nf + f] = 0.0;
    return;
  }
  const double n[3] = {nS[f], nS[nf + f], nS[2 * nf + f]};
  const int64_t L = fL[f], R = fR[f];
  double WL[5], WR[5], F[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) WL[q] = W[q * nc + L];
  if (R >= 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) WR[q] = W[q * nc + R];
  } else if (!bc_ghost<double>(ftag[f], n, WL, nullptr, WR, nullptr, ph.gamma, ph.Winf)) {
    set_err(err, CGKS_ENAN, (int)L, 20);
  }
  if (!kfvs_flux<double>(WL, WR, n, ph.K, ph.gamma - 1.0, F)) set_err(err, CGKS_ENAN, (int)L, 21);
#pragma unroll
  for (int q = 0; q < 5; ++q) ff[q * nf + f] = s * F[q];
}

// Directional derivative of the KFVS face fluxes x area at the state W0 in the direction dW, in
// FP32 forward mode: dW = X - W0 when x_is_state, else X.  The boundary ghost state is
// differentiated with the cell state it is built from.
__global__ void k_kfvs_jvp_faces(int64_t nf, const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                                 const int32_t* __restrict__ ftag, const double* __restrict__ Sn, int64_t nc,
                                 const double* __restrict__ W0, const double* __restrict__ X, int x_is_state,
                                 float* __restrict__ ff, Phys ph, DevErr* err) {
  using D = Dual<float>;
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const float S[3] = {float(Sn[f]), float(Sn[nf + f]), float(Sn[2 * nf + f])};
  const float s = sqrtf(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  if (s == 0.0f) {  // no net area, no flux
#pragma unroll
    for (int q = 0; q < 5; ++q) ff[q * nf + f] = 0.0f;
    return;
  }
  const D n[3] = {D(S[0] / s), D(S[1] / s), D(S[2] / s)};
  const int64_t L = fL[f], R = fR[f];
  D WL[5], WR[5], F[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double w = W0[q * nc + L], x = X[q * nc + L];
    WL[q] = D(float(w), float(x_is_state ? x - w : x));
  }
  if (R >= 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double w = W0[q * nc + R], x = X[q * nc + R];
      WR[q] = D(float(w), float(x_is_state ? x - w : x));
    }
  } else if (!bc_ghost<D>(ftag[f], n, WL, nullptr, WR, nullptr, D(ph.gamma), ph.Winf)) {
    set_err(err, CGKS_ENAN, (int)L, 23);
  }
  if (!kfvs_flux<D>(WL, WR, n, D(ph.K), D(ph.gamma - 1.0), F)) set_err(err, CGKS_ENAN, (int)L, 24);
#pragma unroll
  for (int q = 0; q < 5; ++q) ff[q * nf + f] = s * F[q].d;
}

// res = -(sum of outward face fluxes), summed in FP64 in ascending face order
template <typename T>
__global__ void k_kfvs_gather(int64_t nc, int64_t nf, const int32_t* __restrict__ ptr, const int32_t* __restrict__ c2f,
                              const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                              const T* __restrict__ ff, double* __restrict__ res) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double r[5] = {0, 0, 0, 0, 0};
  for (int32_t k = ptr[c]; k < ptr[c + 1]; ++k) {
    const int64_t f = c2f[k];
    const int32_t a = fL[f], b = fR[f];
    if (a == b) continue;  // a cell's periodic image of itself: the two sides cancel
    const double s = a == c ? 1.0 : -1.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) r[q] -= s * (double)ff[q * nf + f];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) res[q * nc + c] = r[q];
}

// local time step CFL |Omega| / sum_p A_p (|u . n_p| + c): A_p the area of the coarse face (the sum
// of its fine faces' areas), n_p the direction of its summed area vector (nS; zero, so no |u . n|
// term, when that vector cancels)
__global__ void k_coarse_dt(int64_t nc, int64_t nf, const int32_t* __restrict__ ptr, const int32_t* __restrict__ c2f,
                            const double* __restrict__ nS, const double* __restrict__ area,
                            const double* __restrict__ vol, const double* __restrict__ W,
                            double* __restrict__ dt, double gamma, double cfl) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double r = 1.0 / W[c];
  const double u[3] = {W[nc + c] * r, W[2 * nc + c] * r, W[3 * nc + c] * r};
  const double p = (gamma - 1.0) * (W[4 * nc + c] - 0.5 * W[c] * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  const double snd = sqrt(gamma * p * r);
  double s = 0.0;
  for (int32_t k = ptr[c]; k < ptr[c + 1]; ++k) {
    const int64_t f = c2f[k];
    const double un = fabs(u[0] * nS[f] + u[1] * nS[nf + f] + u[2] * nS[2 * nf + f]);
    s += area[f] * (un + snd);
  }
  dt[c] = cfl * vol[c] / s;
}

// F = Rs - R  (FAS forcing term)
__global__ void k_forcing(int64_t n5, const double* __restrict__ Rs, const double* __restrict__ R, double* __restrict__ F) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n5) F[j] = Rs[j] - R[j];
}

// W += dt / V (R + F); an update that would make rho or p non-positive is skipped for that cell
// (counted), a non-finite one is an error
__global__ void k_fe_update(int64_t nc, const double* __restrict__ dt, const double* __restrict__ vol,
                            const double* __restrict__ R, const double* __restrict__ F, double* __restrict__ W,
                            double gamma, unsigned long long* skipped, DevErr* err) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double h = dt[c] / vol[c];
  double w[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) w[q] = W[q * nc + c] + h * (R[q * nc + c] + F[q * nc + c]);
  const double p = (gamma - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
  if (!(isfinite(w[0]) && isfinite(w[1]) && isfinite(w[2]) && isfinite(w[3]) && isfinite(w[4]))) {
    set_err(err, CGKS_ENAN, (int)c, 22);
  } else if (w[0] > 0.0 && p > 0.0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) W[q * nc + c] = w[q];
  } else {
    atomicAdd(skipped, 1ULL);
  }
}

// coarse state = sum V_i W_i / V_c and coarse defect = sum (R_i [+ F_i]) over the finer cells of
// each coarse cell, in ascending finer-cell order
__global__ void k_restrict(int64_t ncc, int64_t ncf, const int32_t* __restrict__ aptr, const int32_t* __restrict__ agg,
                           const double* __restrict__ vf, const double* __restrict__ vc, const double* __restrict__ Wf,
                           const double* __restrict__ Rf, const double* __restrict__ Ff, double* __restrict__ Wc,
                           double* __restrict__ Rc) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncc) return;
  double w[5] = {0, 0, 0, 0, 0}, r[5] = {0, 0, 0, 0, 0};
  for (int32_t k = aptr[c]; k < aptr[c + 1]; ++k) {
    const int64_t i = agg[k];
    const double v = vf[i];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      w[q] += v * Wf[q * ncf + i];
      r[q] += Ff ? Rf[q * ncf + i] + Ff[q * ncf + i] : Rf[q * ncf + i];
    }
  }
  const double rv = 1.0 / vc[c];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    Wc[q * ncc + c] = w[q] * rv;
    Rc[q * ncc + c] = r[q];
  }
}

// W_f += r (W_c - W_c^0) (injection, r = correction_relax); a correction that would make rho or p
// non-positive is skipped
__global__ void k_prolong(int64_t ncf, int64_t ncc, const int32_t* __restrict__ f2c, const double* __restrict__ Wc,
                          const double* __restrict__ Wc0, double* __restrict__ Wf, double gamma, double relax,
                          unsigned long long* skipped) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ncf) return;
  const int64_t c = f2c[i];
  double w[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) w[q] = Wf[q * ncf + i] + relax * (Wc[q * ncc + c] - Wc0[q * ncc + c]);
  const double p = (gamma - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
  if (w[0] > 0.0 && p > 0.0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) Wf[q * ncf + i] = w[q];
  } else {
    atomicAdd(skipped, 1ULL);
  }
}

// prolongation 1: cell i of the receiving level takes the volume-weighted mean of the injected
// corrections of itself and its face neighbours (in ascending face order), then W += relax x that
__global__ void k_prolong_smooth(int64_t ncf, int64_t ncc, const int32_t* __restrict__ ptr,
                                 const int32_t* __restrict__ c2f, const int32_t* __restrict__ fL,
                                 const int32_t* __restrict__ fR, const double* __restrict__ vol,
                                 const int32_t* __restrict__ f2c, const double* __restrict__ Wc,
                                 const double* __restrict__ Wc0, double* __restrict__ Wf, double gamma, double relax,
                                 unsigned long long* skipped) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ncf) return;
  double acc[5], sv = vol[i];
  {
    const int64_t c = f2c[i];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = vol[i] * (Wc[q * ncc + c] - Wc0[q * ncc + c]);
  }
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
    const int64_t f = c2f[k];
    const int32_t a = fL[f], b = fR[f];
    if (b < 0 || a == b) continue;
    const int64_t j = a == i ? b : a;
    const int64_t c = f2c[j];
    const double v = vol[j];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] += v * (Wc[q * ncc + c] - Wc0[q * ncc + c]);
    sv += v;
  }
  double w[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) w[q] = Wf[q * ncf + i] + relax * (acc[q] / sv);
  const double p = (gamma - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
  if (w[0] > 0.0 && p > 0.0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) Wf[q * ncf + i] = w[q];
  } else {
    atomicAdd(skipped, 1ULL);
  }
}

static void prolong(cgks_ctx* ctx, int lev_fine, const int32_t* f2c, int64_t ncc, const double* Wc,
                    const double* Wc0, double* Wf) {
  const Level& L = ctx->L[lev_fine];
  cudaStream_t st = ctx->stream;
  ProfScope ps(ctx, PK_PROLONG, (double)L.nc,
               L.nc * 84.0 + ncc * 80.0 +
                   (ctx->P.prolongation == 1 ? (L.nf + L.n_int + L.n_per) * 4.0 + L.nf * 8.0 + L.nc * 12.0 : 0.0));
  if (ctx->P.prolongation == 1)
    k_prolong_smooth<<<grid_for(L.nc, 256), 256, 0, st>>>(L.nc, ncc, L.c2f_ptr, L.c2f, L.fL, L.fR, L.vol, f2c, Wc, Wc0,
                                                           Wf, ctx->P.gamma, ctx->P.correction_relax,
                                                           (unsigned long long*)ctx->d_skipped);
  else
    k_prolong<<<grid_for(L.nc, 256), 256, 0, st>>>(L.nc, ncc, f2c, Wc, Wc0, Wf, ctx->P.gamma, ctx->P.correction_relax,
                                                   (unsigned long long*)ctx->d_skipped);
}

// sqrt(mean (res_rho / V)^2): per-block partial sums, then one thread adds them in block order
__global__ void k_norm_partial(int64_t n, const double* __restrict__ res, const double* __restrict__ vol,
                               double* __restrict__ part) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = res[i] / vol[i];
    acc += x * x;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_norm_final(int nparts, int64_t n, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < nparts; ++k) s += part[k];
  *out = sqrt(s / (double)n);
}

cgks_status density_norm(cgks_ctx* ctx, const double* res, const double* vol, int64_t n, double* out_dev) {
  const int parts = 304;
  ProfScope ps(ctx, PK_NORM, (double)n, n * 16.0);
  k_norm_partial<<<parts, 256, 0, ctx->stream>>>(n, res, vol, ctx->nrm_part);
  k_norm_final<<<1, 32, 0, ctx->stream>>>(parts, n, ctx->nrm_part, out_dev);
  CK(cudaGetLastError());
  return CGKS_OK;
}

cgks_status global_min_dt(cgks_ctx* ctx, double* dt, int64_t n);

// KFVS residual of level `lev` (FP64)
cgks_status kfvs_residual(cgks_ctx* ctx, int lev, const double* W, double* res) {
  const Level& L = ctx->L[lev];
  const Phys ph = make_phys(ctx->P);
  double* ff = lev == 0 ? ctx->ffl : ctx->C[lev].ff;
  const double entries = (double)(L.nf + L.n_int + L.n_per);
  {
    ProfScope ps(ctx, PK_KFVS_FACES, (double)L.nf, L.nf * 84.0 + L.nc * 40.0);
    const int b = spread_block(L.nf, 256, ctx->n_sm);
    k_kfvs_faces<<<grid_for(L.nf, b), b, 0, ctx->stream>>>(L.nf, L.fL, L.fR, L.ftag, L.nS, L.nc, W, ff, ph, ctx->derr);
  }
  {
    ProfScope ps(ctx, PK_KFVS_GATHER, (double)L.nc, L.nc * 44.0 + entries * 4.0 + L.nf * 48.0);
    k_kfvs_gather<double><<<grid_for(L.nc, 256), 256, 0, ctx->stream>>>(L.nc, L.nf, L.c2f_ptr, L.c2f, L.fL, L.fR, ff,
                                                                         res);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

cgks_status kfvs_jvp(cgks_ctx* ctx, int lev, const double* W0, const double* X, int x_is_state, double* res) {
  const Level& L = ctx->L[lev];
  const Phys ph = make_phys(ctx->P);
  float* ff = lev == 0 ? ctx->ffl32 : ctx->C[lev].ff32;
  const double entries = (double)(L.nf + L.n_int + L.n_per);
  {
    ProfScope ps(ctx, PK_KFVS_JVP, (double)L.nf, L.nf * 56.0 + L.nc * 80.0);
    k_kfvs_jvp_faces<<<grid_for(L.nf, 256), 256, 0, ctx->stream>>>(L.nf, L.fL, L.fR, L.ftag, L.Sn, L.nc, W0, X,
                                                                    x_is_state, ff, ph, ctx->derr);
  }
  {
    ProfScope ps(ctx, PK_KFVS_GATHER, (double)L.nc, L.nc * 44.0 + entries * 4.0 + L.nf * 28.0);
    k_kfvs_gather<float><<<grid_for(L.nc, 256), 256, 0, ctx->stream>>>(L.nc, L.nf, L.c2f_ptr, L.c2f, L.fL, L.fR, ff,
                                                                        res);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

cgks_status coarse_dt(cgks_ctx* ctx, int lev, const double* W, double* dt) {
  const Level& L = ctx->L[lev];
  {
    ProfScope ps(ctx, PK_COARSE_DT, (double)L.nc, L.nc * 60.0 + (L.nf + L.n_int + L.n_per) * 4.0 + L.nf * 32.0);
    const int b = spread_block(L.nc, 256, ctx->n_sm);
    k_coarse_dt<<<grid_for(L.nc, b), b, 0, ctx->stream>>>(L.nc, L.nf, L.c2f_ptr, L.c2f, L.nS, L.area, L.vol, W, dt,
                                                          ctx->P.gamma, ctx->P.cfl_coarse);
  }
  if (ctx->P.dt_mode == 1) CKS(global_min_dt(ctx, dt, L.nc));
  CK(cudaGetLastError());
  return CGKS_OK;
}

// coarse-level FAS smoothing on level l with the restricted state already in C[l].W (and W0) and
// the restricted defect in C[l].Rs, then recursion to the next level and correction
// coarse-level residual at the current state B.W into B.R, the defect being B.R + B.F:
// FP64 FAS: R = Res(W), F = Res* - Res(W^0);  precision 1 (defect correction): R = J(W^0)(W - W^0)
// in FP32 forward mode, F = Res*, so the defect is linear in the correction W - W^0 and FP32 only
// perturbs it relative to its own size
static cgks_status coarse_residual(cgks_ctx* ctx, int l) {
  CoarseBuf& B = ctx->C[l];
  if (ctx->P.precision == 1) return kfvs_jvp(ctx, l, B.W0, B.W, 1, B.R);
  return kfvs_residual(ctx, l, B.W, B.R);
}

static cgks_status coarse_smooth(cgks_ctx* ctx, int l) {
  const Level& L = ctx->L[l];
  CoarseBuf& B = ctx->C[l];
  CKS(coarse_dt(ctx, l, B.W, B.dt));
  if (ctx->P.coarse_smoother == 1) return lusgs_step(ctx, l);
  {
    ProfScope ps(ctx, PK_FE_UPDATE, (double)L.nc, L.nc * 176.0);
    k_fe_update<<<grid_for(L.nc, 256), 256, 0, ctx->stream>>>(L.nc, B.dt, L.vol, B.R, B.F, B.W, ctx->P.gamma,
                                                               (unsigned long long*)ctx->d_skipped, ctx->derr);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

// coarse level l of the V-cycle, entered with W = W^0 (the restricted state) and Res* (the
// restricted defect)
static cgks_status coarse_cycle(cgks_ctx* ctx, int l) {
  const Level& L = ctx->L[l];
  CoarseBuf& B = ctx->C[l];
  cudaStream_t st = ctx->stream;
  const int64_t n5 = 5 * L.nc;
  // the residual at W = W^0 serves the forcing and the first step
  if (ctx->P.precision == 1) {
    CK(cudaMemcpyAsync(B.F, B.Rs, sizeof(double) * n5, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(B.R, 0, sizeof(double) * n5, st));
  } else {
    CKS(kfvs_residual(ctx, l, B.W, B.R));
    ProfScope ps(ctx, PK_FORCING, (double)L.nc, n5 * 24.0);
    k_forcing<<<grid_for(n5, 256), 256, 0, st>>>(n5, B.Rs, B.R, B.F);
  }
  for (int s = 0; s < ctx->P.coarse_steps; ++s) {
    if (s > 0) CKS(coarse_residual(ctx, l));
    CKS(coarse_smooth(ctx, l));
  }
  if (l + 1 < (int)ctx->L.size()) {
    const Level& Cn = ctx->L[l + 1];
    CoarseBuf& N = ctx->C[l + 1];
    CKS(coarse_residual(ctx, l));
    {
      ProfScope ps(ctx, PK_RESTRICT, (double)L.nc, L.nc * 132.0 + Cn.nc * 92.0);
      k_restrict<<<grid_for(Cn.nc, 256), 256, 0, st>>>(Cn.nc, L.nc, Cn.agg_ptr, Cn.agg, L.vol, Cn.vol, B.W, B.R, B.F,
                                                       N.W, N.Rs);
    }
    CK(cudaMemcpyAsync(N.W0, N.W, sizeof(double) * 5 * Cn.nc, cudaMemcpyDeviceToDevice, st));
    CKS(coarse_cycle(ctx, l + 1));
    prolong(ctx, l, Cn.f2c, Cn.nc, N.W, N.W0, B.W);
    for (int s = 0; s < ctx->P.post; ++s) {
      CKS(coarse_residual(ctx, l));
      CKS(coarse_smooth(ctx, l));
    }
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

// one explicit CGKS step of the fine level (Eq. smo); norm of the residual before the step
cgks_status step_once(cgks_ctx* ctx, double* norm_dev) {
  CKS(fine_fluxes(ctx, ctx->W, ctx->G, ctx->alpha));
  // the gather reads only the Gauss-point records, so W, gradW and alpha are updated in place
  CKS(fine_gather(ctx, ctx->W, ctx->W, ctx->res, ctx->G, ctx->alpha, 1));
  if (norm_dev) CKS(density_norm(ctx, ctx->res, ctx->F.vol, ctx->F.nc, norm_dev));
  return CGKS_OK;
}

// one V-cycle (Sec. 4.2)
cgks_status vcycle_once(cgks_ctx* ctx, double* norm_dev) {
  cudaStream_t st = ctx->stream;
  const int pre = ctx->P.pre > 0 ? ctx->P.pre : 1;
  for (int s = 0; s < pre; ++s) CKS(step_once(ctx, s == 0 ? norm_dev : nullptr));
  if (ctx->L.size() <= 1) return CGKS_OK;
  const Fine& F = ctx->F;
  const Level& C1 = ctx->L[1];
  CoarseBuf& B1 = ctx->C[1];
  // defect at the smoothed state (the residual alone: no interface state, gradient or compression
  // factor is formed)
  CKS(fine_fluxes(ctx, ctx->W, ctx->G, ctx->alpha, false));
  CKS(fine_gather(ctx, ctx->W, nullptr, ctx->res, nullptr, nullptr, 0));
  {
    ProfScope ps(ctx, PK_RESTRICT, (double)F.nc, F.nc * 92.0 + C1.nc * 92.0);
    k_restrict<<<grid_for(C1.nc, 256), 256, 0, st>>>(C1.nc, F.nc, C1.agg_ptr, C1.agg, ctx->L0c.vol, C1.vol, ctx->W,
                                                     ctx->res, nullptr, B1.W, B1.Rs);
  }
  CK(cudaMemcpyAsync(B1.W0, B1.W, sizeof(double) * 5 * C1.nc, cudaMemcpyDeviceToDevice, st));
  CKS(coarse_cycle(ctx, 1));
  prolong(ctx, 0, C1.f2c, C1.nc, B1.W, B1.W0, ctx->W);
  for (int s = 0; s < ctx->P.post; ++s) CKS(step_once(ctx, nullptr));
  CK(cudaGetLastError());
  return CGKS_OK;
}
