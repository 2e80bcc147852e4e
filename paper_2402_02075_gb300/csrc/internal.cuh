// Internal declarations of libcgks: device buffers of the mesh hierarchy and the solver state,
// launch helpers and error plumbing.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cgks.h"

#define CGKS_MAXNF 6          // faces of a hexahedron
#define CGKS_KOP 216          // reconstruction operator entries per cell: 9 x (4 * 6)
#define CGKS_RC 50            // reconstruction coefficients per cell: 5 variables x 10
#define CGKS_GPR 14           // Gauss-point record: flux x weight (5), interface state (5), area vector (3), alpha
#define CGKS_AUX 8            // per-cell constants of the smoothness indicators
#define CGKS_AGG_CAP 256      // records per coarse cell while building coarse faces
#define HD __host__ __device__ __forceinline__

// device error word: [0] code (cgks_status), [1] cell or face index, [2] detail
struct DevErr {
  int32_t code, index, detail, pad;
};

__host__ __device__ __forceinline__ void set_err(DevErr* e, int code, int index, int detail = 0) {
#ifdef __CUDA_ARCH__
  if (atomicCAS(&e->code, 0, code) == 0) {
#else
  if (e->code == 0) {
    e->code = code;
#endif
    e->index = index;
    e->detail = detail;
  }
}

// constants of the physical model passed by value to the kernels
struct Phys {
  double gamma, K, mu, prandtl, eps_inviscid, c_press, weno_eps, cfl_fine, cfl_coarse, suth;
  int viscous, dt_mode, cf;
  double Winf[5];
};

// one level of the multigrid hierarchy as used by the first-order solver and by the coarsening
struct Level {
  int64_t nc = 0, nf = 0, n_int = 0, n_per = 0;
  double *vol = nullptr, *ctr = nullptr;                          // [nc], [3][nc]
  int32_t *fL = nullptr, *fR = nullptr, *ftag = nullptr, *ftagR = nullptr;  // [nf]
  double *Sn = nullptr, *area = nullptr, *amom = nullptr, *shift = nullptr;  // [3][nf],[nf],[3][nf],[3][nf]
  double* nS = nullptr;  // [4][nf] unit normal S/|S| (0 where the summed area vectors cancel), |S|
  int32_t *c2f_ptr = nullptr, *c2f = nullptr;                    // cell -> faces, ascending ids
  int32_t *f2c = nullptr;                                        // finer cell -> this level's cell
  int64_t nc_finer = 0;
  int32_t *agg_ptr = nullptr, *agg = nullptr;                    // this level's cell -> finer cells
};

// the fine mesh with its Gauss points and reconstruction operators
struct Fine {
  int64_t nc = 0, nf = 0, n_int = 0, n_per = 0, n_bnd = 0, ngp = 0;
  int64_t gp_sides = 0;  // Gauss points summed over every cell's faces (interior points counted twice)
  int8_t* ctype = nullptr;
  double *vol = nullptr, *ctr = nullptr, *m2 = nullptr;          // [nc], [3][nc], [6][nc]
  int32_t *fL = nullptr, *fR = nullptr, *ftag = nullptr, *ftagR = nullptr, *flf = nullptr;
  int32_t *gp_ptr = nullptr, *gp_face = nullptr;                 // [nf + 1], [ngp]
  double *gp_x = nullptr, *gp_A = nullptr;                       // [3][ngp] point, area vector
  double *fshift = nullptr, *fnrm = nullptr, *fctr = nullptr;    // [3][nf] each
  int32_t *cf = nullptr;                                         // [6][nc] face of each local face
  int8_t* cside = nullptr;                                       // [6][nc] 0: cell is L, 1: R
  int32_t *c2f_ptr = nullptr, *c2f = nullptr;                    // cell -> faces (ascending)
  double *Kop = nullptr;                                         // [216][nc] p^2 operator
  double *ggw = nullptr;                                         // [18][nc] outward S n / (2|Omega|)
  double *lsw = nullptr;                                         // [18][nc] least-squares gradient weights
  double *aux = nullptr;                                         // [8][nc] |Omega|^(2/3), |Omega|^(4/3), m2
  double *dtw = nullptr;                                         // [24][nc] time-step weights per local face
};

struct CoarseBuf {  // per coarse level work arrays
  double *W = nullptr, *W0 = nullptr, *Rs = nullptr, *F = nullptr, *R = nullptr, *dt = nullptr, *ff = nullptr;
  float* ff32 = nullptr;  // FP32 directional derivatives of the face fluxes (precision 1)
  // LU-SGS smoother (coarse_smoother 1): colours, colour-major cell order and its offsets,
  // per-face lambda, diagonal, increments
  int32_t *color = nullptr, *order = nullptr;
  std::vector<int64_t> coff;
  double *lam = nullptr, *Dg = nullptr, *dU = nullptr;
};

// kernel kinds timed by cgks_profile (ids of cgks_kernel_stats)
enum ProfKind {
  PK_POINTS = 0,   // k_gks_points: Gauss points
  PK_RECON,        // k_reconstruct: cells
  PK_GATHER,       // k_gather: cells
  PK_KFVS_FACES,   // k_kfvs_faces: faces of a coarse level
  PK_KFVS_GATHER,  // k_kfvs_gather (FP64 and FP32 face fluxes): cells
  PK_COARSE_DT,    // k_coarse_dt: cells
  PK_FORCING,      // k_forcing: cells
  PK_FE_UPDATE,    // k_fe_update: cells
  PK_RESTRICT,     // k_restrict: cells of the finer level
  PK_PROLONG,      // k_prolong / k_prolong_smooth: cells of the finer level
  PK_KFVS_JVP,     // k_kfvs_jvp_faces: faces
  PK_NORM,         // k_norm_partial + k_norm_final: cells
  PK_POINTS_FLUX,  // k_gks_points<false> (the flux alone, the V-cycle's defect): Gauss points
  PK_GATHER_RES,   // k_gather<false> (the residual alone): Gauss points seen from cells
  PK_COUNT
};

struct ProfRec {
  cudaEvent_t e0, e1;
  double units, bytes;
};

struct cgks_ctx {
  cgks_params P{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 152;  // streaming multiprocessors of the device
  std::string err;
  bool has_mesh = false, has_state = false;
  Fine F;
  std::vector<Level> L;  // L[0] is the fine level seen as a first-order mesh
  Level L0c;             // L[0] with the geometry of the coarsening (input of level 1, restriction weights)
  std::vector<CoarseBuf> C;
  // fine state and work arrays
  double *W = nullptr, *G = nullptr, *alpha = nullptr;
  double *rc = nullptr, *dt = nullptr, *res = nullptr;
  double* gpr = nullptr;            // [ngp][CGKS_GPR] Gauss-point records (112 bytes, 16-byte aligned)
  double *W1 = nullptr;             // copy of W used by the V-cycle
  double *ffl = nullptr;            // first-order face fluxes of level 0
  float* ffl32 = nullptr;           // their FP32 directional derivatives
  double *nrm_part = nullptr, *nrm = nullptr, *h_nrm = nullptr;
  DevErr* derr = nullptr;
  DevErr* h_err = nullptr;
  int64_t* d_count = nullptr;
  int64_t* h_count = nullptr;
  int64_t* d_skipped = nullptr;     // coarse updates and corrections skipped by the positivity rule
  double r1 = 0.0;
  int64_t iters = 0;
  // adjoint: the stored linearisation at the state of the last cgks_linearize, its time steps,
  // and the work arrays of the transposed products (in mesh_allocs)
  double *Jp = nullptr, *Jr = nullptr, *adt = nullptr;
  double* aWG = nullptr;       // [21][nc] (W, grad W, alpha) at cgks_linearize (adjoint_recompute 1)
  bool lin_recompute = false;  // the last cgks_linearize stored no reconstruction linearisation
  double *pbar = nullptr, *aself = nullptr, *arec = nullptr, *avec = nullptr, *apart = nullptr, *akry = nullptr;
  double* ajc = nullptr;  // per-cell shares of the wall force
  double* acb = nullptr;  // per-cell coefficient cotangents of a transposed product
  bool linearized = false;
  // host copy of the uploaded mesh (shape derivatives re-upload it with displaced nodes)
  std::vector<double> h_xyz;
  std::vector<int8_t> h_ctype;
  std::vector<int64_t> h_cptr, h_bptr;
  std::vector<int32_t> h_cnodes, h_bnodes, h_btag, h_pairs;
  std::vector<void*> mesh_allocs;   // freed on re-upload / destroy
  std::vector<void*> ctx_allocs;    // freed on destroy
  // kernel timing (cgks_profile): event pairs per kernel kind, with the units and the algorithmic
  // bytes of each recorded launch
  bool prof = false;
  std::vector<ProfRec> prof_ev[PK_COUNT];
  std::vector<cudaEvent_t> ev_pool;
  // private non-blocking stream and ordering events of the graph-replayed steady-solve chunks
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
};

// event pair recorded around one launch of kernel kind k when profiling is enabled; units are the
// cells, faces or Gauss points the launch processes, bytes its compulsory DRAM traffic (every input
// read once, every output written once)
struct ProfScope {
  cgks_ctx* c;
  int k;
  cudaEvent_t e1 = nullptr;
  ProfScope(cgks_ctx* ctx, int kind, double units, double bytes);
  ~ProfScope();
};

// ---- error helpers (host) ---------------------------------------------------------------------
cgks_status cgks_fail(cgks_ctx* c, cgks_status s, const std::string& msg);
#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return cgks_fail(ctx, CGKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define CKS(expr)                         \
  do {                                    \
    cgks_status s_ = (expr);              \
    if (s_ != CGKS_OK) return s_;         \
  } while (0)

// device allocation recorded in `list` (zero-filled)
cgks_status dev_alloc(cgks_ctx* ctx, std::vector<void*>& list, void** p, size_t bytes);
template <typename T>
cgks_status dalloc(cgks_ctx* ctx, std::vector<void*>& list, T** p, size_t count) {
  return dev_alloc(ctx, list, reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}
void free_list(std::vector<void*>& list);

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// block size of a launch of n long FP64-bound threads: `max_block` when the launch fills every SM,
// else smaller blocks (a multiple of the warp, at least one) so that the threads spread over all the
// SMs: an SM issues 2 FP64 operations per clock, so a few blocks queued on a few SMs of a small
// mesh would take as long as a full wave
inline int spread_block(int64_t n, int max_block, int n_sm) {
  const int64_t per_sm = (n + n_sm - 1) / n_sm;
  if (per_sm >= max_block) return max_block;
  const int64_t b = ((per_sm + 31) / 32) * 32;
  return (int)(b < 32 ? 32 : b);
}

// exclusive prefix sum of n int32 values (device), total returned through *total (host) when
// non-null (synchronises).  Uses ctx scratch allocated on demand.
cgks_status scan_exclusive(cgks_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, int64_t* total);

// entry points between translation units
cgks_status build_fine_mesh(cgks_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_cells, const int8_t* ctype,
                            const int64_t* cell_ptr, const int32_t* cell_nodes, int64_t n_bfaces,
                            const int64_t* bface_ptr, const int32_t* bface_nodes, const int32_t* bface_tag,
                            const int32_t* periodic_pairs, int64_t n_periodic);
cgks_status build_levels(cgks_ctx* ctx);
Phys make_phys(const cgks_params& P);
cgks_status check_device_error(cgks_ctx* ctx, const char* where);

// fine CGKS residual: reconstruct + Gauss-point fluxes; then either a gather into outputs or an
// explicit update of (W, G, alpha)
// state false: the Gauss-point fluxes alone (no interface state, area or compression factor in the
// records), for a residual-only gather
cgks_status fine_fluxes(cgks_ctx* ctx, const double* W, const double* G, const double* alpha, bool state = true);
cgks_status fine_gather(cgks_ctx* ctx, const double* W_in, double* W_out, double* res, double* G_out,
                        double* alpha_out, int update);
cgks_status density_norm(cgks_ctx* ctx, const double* res, const double* vol, int64_t n, double* out_dev);

// first-order (KFVS) residual of a level; res may equal nullptr when only the face fluxes are needed
cgks_status kfvs_residual(cgks_ctx* ctx, int lev, const double* W, double* res);
// res = J(W0) dW, J the Jacobian of the KFVS residual of level `lev`, in FP32 forward mode with FP64
// sums; dW = X - W0 when x_is_state, else X
cgks_status kfvs_jvp(cgks_ctx* ctx, int lev, const double* W0, const double* X, int x_is_state, double* res);
cgks_status coarse_dt(cgks_ctx* ctx, int lev, const double* W, double* dt);
cgks_status vcycle_once(cgks_ctx* ctx, double* norm_dev);
// LU-SGS step on coarse level l for the defect C[l].R + C[l].F with the time steps in C[l].dt
cgks_status lusgs_step(cgks_ctx* ctx, int l);
cgks_status lusgs_color_count(cgks_ctx* ctx, int l, int32_t* colors, int32_t* n_colors);
cgks_status step_once(cgks_ctx* ctx, double* norm_dev);
