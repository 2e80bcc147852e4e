// Implicit coarse-level smoother of Sec. 4.3 (backward Euler with the first-order Lax-Friedrichs
// Jacobian splitting, matrix-free symmetric Gauss-Seidel: LU-SGS) on the agglomerated levels.
//
// One step solves, for the increments dU,
//   (|Omega_i|/dt_i + 1/2 sum_p lambda_p S_p) dU_i
//       + sum_p 1/2 [F_n(U_p + dU_p) - F_n(U_p) - lambda_p dU_p] S_p = Res_i + F_i
// (n out of cell i, F_n the Euler flux through the face, lambda_p = max(|U.n| + c) of the two cells,
// S_p the length of the face's summed area vector) with one forward and one backward Gauss-Seidel
// sweep.  The sweep order is colour-major: Jones-Plassmann rounds on priorities
// (splitmix64(id), id) give every cell a colour shared by none of its neighbours, so each colour is
// one parallel launch and the result equals the sequential sweep in (colour, id) order.  Ghost
// neighbours keep dU = 0, faces whose area vectors cancel and a cell's periodic face with itself are
// skipped, and an increment that would make rho or p non-positive is not applied (counted).
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 (Steele, Lea, Flood 2014)
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t other_cell(const int32_t* fL, const int32_t* fR, int64_t f, int64_t i) {
  const int32_t a = fL[f], b = fR[f];
  if (b < 0 || a == b) return -1;
  return a == i ? b : a;
}

// an uncoloured cell whose priority beats every uncoloured neighbour's is selected this round
__global__ void k_jpl_select(int64_t nc, const int32_t* __restrict__ ptr, const int32_t* __restrict__ c2f,
                             const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                             const int32_t* __restrict__ color, int8_t* __restrict__ sel) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  int8_t top = color[i] < 0;
  const uint64_t pi = mix64((uint64_t)i);
  for (int32_t k = ptr[i]; k < ptr[i + 1] && top; ++k) {
    const int64_t j = other_cell(fL, fR, c2f[k], i);
    if (j < 0 || color[j] >= 0) continue;
    const uint64_t pj = mix64((uint64_t)j);
    if (pj > pi || (pj == pi && j > i)) top = 0;
  }
  sel[i] = top;
}

// selected cells take the smallest colour none of their (earlier-coloured) neighbours has; two
// selected cells are never neighbours, so the assignments of one round are independent
__global__ void k_jpl_assign(int64_t nc, const int32_t* __restrict__ ptr, const int32_t* __restrict__ c2f,
                             const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                             const int8_t* __restrict__ sel, int32_t* __restrict__ color,
                             unsigned long long* left) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  if (!sel[i]) {
    if (color[i] < 0) atomicAdd(left, 1ULL);
    return;
  }
  for (int32_t c = 0;; ++c) {
    bool used = false;
    for (int32_t k = ptr[i]; k < ptr[i + 1] && !used; ++k) {
      const int64_t j = other_cell(fL, fR, c2f[k], i);
      used = j >= 0 && color[j] == c;
    }
    if (!used) {
      color[i] = c;
      return;
    }
  }
}

__device__ __forceinline__ void euler_flux_n(const double W[5], const double n[3], double g, double F[5]) {
  const double rho = W[0], r = 1.0 / rho;
  const double u[3] = {W[1] * r, W[2] * r, W[3] * r};
  const double p = (g - 1.0) * (W[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  F[0] = rho * un;
#pragma unroll
  for (int d = 0; d < 3; ++d) F[1 + d] = W[1 + d] * un + p * n[d];
  F[4] = (W[4] + p) * un;
}

__device__ __forceinline__ double wave_speed(const double* W, int64_t nc, int64_t i, const double n[3], double g) {
  const double rho = W[i], r = 1.0 / rho;
  const double u[3] = {W[nc + i] * r, W[2 * nc + i] * r, W[3 * nc + i] * r};
  const double p = (g - 1.0) * (W[4 * nc + i] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  return fabs(u[0] * n[0] + u[1] * n[1] + u[2] * n[2]) + sqrt(g * p * r);
}

// lambda of every face: max over its cells of |U.n| + c (the cell's own on boundary faces)
__global__ void k_lusgs_lambda(int64_t nf, const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                               const double* __restrict__ Sn, int64_t nc, const double* __restrict__ W, double g,
                               double* __restrict__ lam) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const double S[3] = {Sn[f], Sn[nf + f], Sn[2 * nf + f]};
  const double s = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  if (s == 0.0) {
    lam[f] = 0.0;
    return;
  }
  const double n[3] = {S[0] / s, S[1] / s, S[2] / s};
  const int32_t a = fL[f], b = fR[f];
  const double la = wave_speed(W, nc, a, n, g);
  lam[f] = b >= 0 ? fmax(la, wave_speed(W, nc, b, n, g)) : la;
}

// D_i = |Omega_i| / dt_i + 1/2 sum_p lambda_p S_p, in ascending face order
__global__ void k_lusgs_diag(int64_t nc, int64_t nf, const int32_t* __restrict__ ptr, const int32_t* __restrict__ c2f,
                             const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                             const double* __restrict__ Sn, const double* __restrict__ lam,
                             const double* __restrict__ vol, const double* __restrict__ dt, double* __restrict__ D) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s = 0.0;
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
    const int64_t f = c2f[k];
    if (fL[f] == fR[f]) continue;
    const double S[3] = {Sn[f], Sn[nf + f], Sn[2 * nf + f]};
    s += lam[f] * sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  }
  D[i] = vol[i] / dt[i] + 0.5 * s;
}

struct SweepArgs {
  int64_t nc, nf;
  const int32_t *ptr, *c2f, *fL, *fR, *color, *cells;
  const double *Sn, *lam, *W, *R, *F, *D;
  double* dU;
  double gamma;
};

// forward (FWD) or backward sweep over the cells of colour k: neighbours of a lower (forward) or
// higher (backward) colour contribute 1/2 [F_n(U_j + dU_j) - F_n(U_j) - lambda dU_j] S
template <bool FWD>
__global__ void k_lusgs_sweep(SweepArgs a, int64_t count, int32_t k) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t nc = a.nc, nf = a.nf, i = a.cells[t];
  double acc[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) acc[q] = FWD ? a.R[q * nc + i] + a.F[q * nc + i] : 0.0;
  for (int32_t e = a.ptr[i]; e < a.ptr[i + 1]; ++e) {
    const int64_t f = a.c2f[e];
    const int64_t j = other_cell(a.fL, a.fR, f, i);
    if (j < 0) continue;
    if (FWD ? a.color[j] >= k : a.color[j] <= k) continue;
    const double S[3] = {a.Sn[f], a.Sn[nf + f], a.Sn[2 * nf + f]};
    const double s = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    if (s == 0.0) continue;
    const double sg = a.fL[f] == i ? 1.0 : -1.0;
    const double n[3] = {sg * (S[0] / s), sg * (S[1] / s), sg * (S[2] / s)};
    double Wj[5], Wp[5], dUj[5], Fp[5], F0[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      Wj[q] = a.W[q * nc + j];
      dUj[q] = a.dU[q * nc + j];
      Wp[q] = Wj[q] + dUj[q];
    }
    euler_flux_n(Wp, n, a.gamma, Fp);
    euler_flux_n(Wj, n, a.gamma, F0);
    const double lam = a.lam[f];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double o = 0.5 * ((Fp[q] - F0[q]) - lam * dUj[q]) * s;
      acc[q] = FWD ? acc[q] - o : acc[q] + o;
    }
  }
  const double Di = a.D[i];
#pragma unroll
  for (int q = 0; q < 5; ++q) a.dU[q * nc + i] = FWD ? acc[q] / Di : a.dU[q * nc + i] - acc[q] / Di;
}

// W += dU, skipping (and counting) cells whose rho or p would not stay positive
__global__ void k_lusgs_apply(int64_t nc, const double* __restrict__ dU, double* __restrict__ W, double g,
                              unsigned long long* skipped, DevErr* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double w[5];
  bool fin = true;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    w[q] = W[q * nc + i] + dU[q * nc + i];
    fin = fin && isfinite(w[q]);
  }
  if (!fin) {
    set_err(err, CGKS_ENAN, (int)i, 25);
    return;
  }
  const double p = (g - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
  if (w[0] > 0.0 && p > 0.0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) W[q * nc + i] = w[q];
  } else {
    atomicAdd(skipped, 1ULL);
  }
}

}  // namespace

// colours and the colour-major cell order of level l (built once per mesh)
cgks_status lusgs_colors(cgks_ctx* ctx, int l) {
  CoarseBuf& B = ctx->C[l];
  if (B.color) return CGKS_OK;
  const Level& L = ctx->L[l];
  cudaStream_t st = ctx->stream;
  auto& M = ctx->mesh_allocs;
  int8_t* sel = nullptr;
  CKS(dalloc(ctx, M, &B.color, L.nc));
  CKS(dalloc(ctx, M, &B.order, L.nc));
  CKS(dalloc(ctx, M, &B.lam, L.nf));
  CKS(dalloc(ctx, M, &B.Dg, L.nc));
  CKS(dalloc(ctx, M, &B.dU, 5 * L.nc));
  std::vector<void*> tmp;
  cgks_status s = dalloc(ctx, tmp, &sel, L.nc);
  if (s != CGKS_OK) {
    free_list(tmp);
    return s;
  }
  std::vector<int32_t> minus1(L.nc, -1);
  cudaError_t e = cudaMemcpyAsync(B.color, minus1.data(), sizeof(int32_t) * L.nc, cudaMemcpyHostToDevice, st);
  // each round colours at least the uncoloured cell of highest priority, so nc rounds bound it
  int64_t left = L.nc;
  for (int64_t round = 0; e == cudaSuccess && left > 0 && round <= L.nc; ++round) {
    k_jpl_select<<<grid_for(L.nc, 256), 256, 0, st>>>(L.nc, L.c2f_ptr, L.c2f, L.fL, L.fR, B.color, sel);
    e = cudaMemsetAsync(ctx->d_count, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) break;
    k_jpl_assign<<<grid_for(L.nc, 256), 256, 0, st>>>(L.nc, L.c2f_ptr, L.c2f, L.fL, L.fR, sel, B.color,
                                                      (unsigned long long*)ctx->d_count);
    e = cudaMemcpyAsync(ctx->h_count, ctx->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) left = *ctx->h_count;
  }
  free_list(tmp);
  CK(e);
  if (left > 0) return cgks_fail(ctx, CGKS_EINVAL, "LU-SGS colouring did not finish");
  // colour-major order, ascending cell id within a colour (counting sort on the host)
  std::vector<int32_t> col(L.nc), order(L.nc);
  CK(cudaMemcpyAsync(col.data(), B.color, sizeof(int32_t) * L.nc, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int32_t ncol = 0;
  for (int32_t c : col) ncol = std::max(ncol, c + 1);
  B.coff.assign(ncol + 1, 0);
  for (int32_t c : col) ++B.coff[c + 1];
  for (int32_t c = 0; c < ncol; ++c) B.coff[c + 1] += B.coff[c];
  std::vector<int64_t> pos(B.coff.begin(), B.coff.end() - 1);
  for (int64_t i = 0; i < L.nc; ++i) order[pos[col[i]]++] = (int32_t)i;
  CK(cudaMemcpyAsync(B.order, order.data(), sizeof(int32_t) * L.nc, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return CGKS_OK;
}

// one LU-SGS step on level l for the defect B.R + B.F with the time steps in B.dt
cgks_status lusgs_step(cgks_ctx* ctx, int l) {
  CKS(lusgs_colors(ctx, l));
  const Level& L = ctx->L[l];
  CoarseBuf& B = ctx->C[l];
  cudaStream_t st = ctx->stream;
  const double g = ctx->P.gamma;
  k_lusgs_lambda<<<grid_for(L.nf, 256), 256, 0, st>>>(L.nf, L.fL, L.fR, L.Sn, L.nc, B.W, g, B.lam);
  k_lusgs_diag<<<grid_for(L.nc, 256), 256, 0, st>>>(L.nc, L.nf, L.c2f_ptr, L.c2f, L.fL, L.fR, L.Sn, B.lam, L.vol,
                                                     B.dt, B.Dg);
  SweepArgs a{L.nc, L.nf, L.c2f_ptr, L.c2f, L.fL, L.fR, B.color, B.order, L.Sn, B.lam, B.W, B.R, B.F, B.Dg, B.dU, g};
  const int32_t ncol = (int32_t)B.coff.size() - 1;
  for (int32_t k = 0; k < ncol; ++k) {
    const int64_t cnt = B.coff[k + 1] - B.coff[k];
    SweepArgs ak = a;
    ak.cells = B.order + B.coff[k];
    k_lusgs_sweep<true><<<grid_for(cnt, 128), 128, 0, st>>>(ak, cnt, k);
  }
  for (int32_t k = ncol - 1; k >= 0; --k) {
    const int64_t cnt = B.coff[k + 1] - B.coff[k];
    SweepArgs ak = a;
    ak.cells = B.order + B.coff[k];
    k_lusgs_sweep<false><<<grid_for(cnt, 128), 128, 0, st>>>(ak, cnt, k);
  }
  k_lusgs_apply<<<grid_for(L.nc, 256), 256, 0, st>>>(L.nc, B.dU, B.W, g, (unsigned long long*)ctx->d_skipped,
                                                      ctx->derr);
  CK(cudaGetLastError());
  return CGKS_OK;
}

cgks_status lusgs_color_count(cgks_ctx* ctx, int l, int32_t* colors, int32_t* n_colors) {
  CKS(lusgs_colors(ctx, l));
  const CoarseBuf& B = ctx->C[l];
  if (colors)
    CK(cudaMemcpyAsync(colors, B.color, sizeof(int32_t) * ctx->L[l].nc, cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (n_colors) *n_colors = (int32_t)B.coff.size() - 1;
  return CGKS_OK;
}
