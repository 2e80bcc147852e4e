/* cgks.h - C ABI of libcgks, a GB300 (sm_103a) implementation of the multigrid compact gas-kinetic
 * scheme (CGKS) for steady flows on 3D mixed hexahedral/prismatic/pyramidal/tetrahedral meshes
 * (H. Liu, X. Ji, Y. Mao, Y. Ding, K. Xu, arXiv:2402.02075).
 *
 * Conventions shared by every entry point
 *  - Every call returns a cgks_status; CGKS_OK is 0.  On any other value cgks_last_error() gives a
 *    one-line message.  No C++ exception crosses this boundary.
 *  - Array arguments are DEVICE pointers (memory of the current CUDA device) unless the comment says
 *    "host".  The caller owns every pointer it passes; the library copies what it keeps.
 *  - Field arrays are component-major: W is double[5][N] (rho, rho u, rho v, rho w, rho E), the
 *    cell-averaged gradient gradW is double[15][N] with row 3*q + d = d(W_q)/dx_d.
 *  - Work is enqueued on the CUDA stream given to cgks_create (stream order); calls return after
 *    enqueueing, except those with host outputs, which synchronise that stream before returning.
 *  - Non-dimensionalisation: free stream rho = 1, p = 1/gamma (unit sound speed), |U| = mach along
 *    the angles aoa; viscosity mu = mach / reynolds (reference length 1), constant.
 *  - Boundary-face tags: 1 slip wall, 2 no-slip adiabatic wall, 3 farfield (Riemann invariants),
 *    4 supersonic inflow, 5 supersonic outflow (extrapolation), >= 100 periodic side.
 */
#ifndef CGKS_H
#define CGKS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CGKS_OK = 0,
  CGKS_EINVAL = 1,       /* bad argument (null pointer, size, level out of range, state not set) */
  CGKS_ENOMEM = 2,       /* device allocation failed */
  CGKS_ECUDA = 3,        /* a CUDA call failed; the message carries cudaGetErrorString */
  CGKS_EMESH = 4,        /* inconsistent mesh (unmatched face, bad cell type, non-positive volume) */
  CGKS_ENAN = 5,         /* non-finite value or rho <= 0 / p <= 0 in a state; message names the cell */
  CGKS_ENOTCONV = 6,     /* steady solve reached max_iters before the requested drop */
  CGKS_ETIMEOUT = 7,     /* reserved for bounded device-side waits (none are used) */
  CGKS_EUNSUPPORTED = 8  /* entry point or option not available in this build */
} cgks_status;

typedef struct cgks_ctx cgks_ctx; /* opaque, owned by the library */

/* Solver parameters.  Defaults (cgks_default_params) are the paper's constants where it gives them
 * and documented readings where it does not. */
typedef struct {
  double gamma;        /* ratio of specific heats, internal degrees K = (5 - 3 gamma)/(gamma - 1) (Sec. 2.1) */
  double mach;         /* free-stream Mach number */
  double reynolds;     /* Reynolds number (reference length 1); used when viscous != 0 */
  double prandtl;      /* Prandtl number; the BGK model has Pr = 1, other values correct the heat flux */
  double aoa[2];       /* degrees: angle of attack (x-z plane) and sideslip of the free stream */
  double cfl_fine;     /* CFL number of the fine-level local time step */
  double cfl_coarse;   /* CFL number of the coarse-level (KFVS) local time step (0.9) */
  double eps_inviscid; /* epsilon in tau_n = eps dt + C |p_l - p_r|/(p_l + p_r) dt (Sec. 2.3, 0.01) */
  double c_press;      /* C of the pressure-jump term of tau_n (Sec. 2.3, 1) */
  double weno_eps;     /* epsilon of the non-linear WENO weights (Sec. 3.4, 1e-5) */
  double skew_min;     /* skewness limit of the coarsening (Sec. 4.1; no value given, 0.2) */
  double sutherland;   /* Sutherland constant over the free-stream temperature, S/T_inf (0.383 for air
                          at 288 K): mu = mu_inf t^(3/2) (1 + s)/(t + s), t = T/T_inf; 0 (the default)
                          keeps mu constant */
  double correction_relax; /* factor on the injected coarse correction W += r (W_c - W_c^0); Sec. 4.2
                              injects the plain correction (1, the default) */
  int32_t n_levels;    /* multigrid levels including the fine one (Sec. 4.2 uses 3) */
  int32_t pre;         /* fine pre-smoothing steps per V-cycle (Sec. 4.2: 1) */
  int32_t post;        /* post-smoothing steps per level (Sec. 4.2: 0) */
  int32_t coarse_steps;     /* forward-Euler KFVS steps per coarse level and cycle (2) */
  int32_t passes_per_level; /* pairwise coarsening passes per multigrid level (2) */
  int32_t viscous;     /* 0 Euler, 1 Navier-Stokes (tau = mu/p) */
  int32_t dt_mode;     /* 0 local time steps, 1 one global (minimum) time step per level */
  int32_t precision;   /* 0 FP64 on every level (FAS coarse equations); 1 mixed: the coarse levels smooth
                          the correction W - W^0 with the FP32 linearised KFVS operator (defect
                          correction, cgks_kfvs_jvp); the fine level, the defect, its restriction,
                          the states, updates and correction stay FP64 */
  int32_t coarse_smoother; /* 0 forward Euler (Sec. 4.2); 1 LU-SGS, the implicit variant of Sec. 4.3 */
  int32_t compression_factor; /* 1 (default): the gradient compression factor of Sec. 3.3; 0: alpha = 1
                                 (no compression), which the adjoint needs: the factor's |p_l - p_r|
                                 terms have no derivative where the jump vanishes */
  int32_t prolongation;    /* 0 injection (Sec. 4.2); 1 injection smoothed once over face neighbours: a
                              cell receives the volume-weighted mean of its own and its neighbours'
                              injected corrections (not in the paper) */
  int32_t adjoint_recompute; /* transposed products of the adjoint (not in the paper): 0 (default) read
                                the reconstruction's linearisation that cgks_linearize stores (2,220
                                doubles per cell); 1 store nothing for the reconstruction and recompute
                                its transposed product in every product (reverse mode through the WENO
                                reconstruction of each cell, from the state at cgks_linearize) */
  uint64_t agglo_seed; /* 0: the paper's hash on cell ids; s > 0 relabels cell N as splitmix64(N ^ s) >> 33 */
} cgks_params;

/* Fills *p with the defaults listed above (gamma 1.4, mach 0.2, reynolds 1e4, prandtl 1, aoa 0,
 * cfl 0.5/0.5, eps 0.01, C 1, weno 1e-5, skew 0.2, 3 levels, pre 1, post 0, 1 coarse step,
 * 2 passes, inviscid, local time steps, FP64, forward-Euler coarse smoother, seed 0).  Host pointer. */
cgks_status cgks_default_params(cgks_params* p);

/* Creates a context on the current CUDA device.  params: host pointer, copied.  stream: a
 * cudaStream_t (NULL = legacy default stream) on which all work of this context is enqueued. */
cgks_status cgks_create(const cgks_params* params, void* cuda_stream, cgks_ctx** out);

/* Frees every device and host buffer of the context.  NULL is accepted. */
cgks_status cgks_destroy(cgks_ctx* ctx);

/* Replaces the parameters (host pointer).  Options that shape the multigrid hierarchy
 * (n_levels, passes_per_level, skew_min, agglo_seed) take effect at the next cgks_mesh_upload. */
cgks_status cgks_set_params(cgks_ctx* ctx, const cgks_params* params);

/* Uploads the fine mesh (all HOST pointers, copied) and builds on the device: faces and their
 * Gauss points (3 per triangle, 4 per quadrilateral, Sec. 2.2), cell volume moments, the
 * reconstruction operators (Sec. 3) and the coarse levels by hash agglomeration (Sec. 4.1).
 *   xyz         double[n_nodes][3]
 *   cell_type   int8[n_cells]: 4 tetrahedron, 5 prism, 6 hexahedron, 7 pyramid; nodes in VTK
 *               order (pyramid: base 0..3 counter-clockwise seen from the apex, apex 4)
 *   cell_ptr    int64[n_cells + 1] offsets into cell_nodes (4, 6, 8 or 5 nodes per cell)
 *   cell_nodes  int32 node ids
 *   bface_ptr   int64[n_bfaces + 1], bface_nodes int32 (3 or 4 nodes, any order), bface_tag int32
 *   periodic_pairs int32[n_periodic][2] boundary-face ids (nullable when n_periodic == 0); the
 *               second face of a pair is the translate of the first.
 * Cell ids are the upload order; the hash of Sec. 4.1 uses them.  Errors: CGKS_EMESH (a cell face
 * matched by no cell and no boundary face, a face shared by three cells, bad type, non-positive
 * volume), CGKS_EINVAL, CGKS_ENOMEM.  Synchronises the stream.  Replaces any earlier mesh. */
cgks_status cgks_mesh_upload(cgks_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_cells,
                             const int8_t* cell_type, const int64_t* cell_ptr, const int32_t* cell_nodes,
                             int64_t n_bfaces, const int64_t* bface_ptr, const int32_t* bface_nodes,
                             const int32_t* bface_tag, const int32_t* periodic_pairs, int64_t n_periodic);

/* Sizes of multigrid level `level` (0 = fine).  Host outputs, nullable. */
cgks_status cgks_level_info(cgks_ctx* ctx, int level, int64_t* n_cells, int64_t* n_faces);

/* Map from the cells of level-1 to the cells of `level` (level >= 1): int32[n_cells(level-1)],
 * device pointer written by the library. */
cgks_status cgks_coarse_map(cgks_ctx* ctx, int level, int32_t* fine_to_coarse);

/* Geometry of a level, device outputs (each nullable): cell volumes double[n], centroids
 * double[3][n]; faces: left/right cell int32[nf] (right = -1 on boundary faces), tag int32[nf]
 * (-1 interior, BC tag on boundary faces, side tag of the left cell on periodic faces), area
 * vectors double[3][nf] (outward from the left cell, summed over the agglomerated fine faces). */
cgks_status cgks_level_geometry(cgks_ctx* ctx, int level, double* vol, double* ctr, int32_t* face_left,
                                int32_t* face_right, int32_t* face_tag, double* area_vec);

/* Fine-level central second-moment averages double[6][N] (xx, yy, zz, xy, yz, xz). Device output. */
cgks_status cgks_fine_moments(cgks_ctx* ctx, double* m2);

/* Sets the fine state: W double[5][N]; gradW double[15][N] or NULL (zero gradients); alpha (the
 * compression factor used by the next Green-Gauss sub-stencil, Sec. 3.3) double[N] or NULL (1).
 * Device pointers, copied.  Resets the residual-drop reference. */
cgks_status cgks_state_init(cgks_ctx* ctx, const double* W, const double* gradW, const double* alpha);

/* Copies the fine state out (device pointers, each nullable). */
cgks_status cgks_state_get(cgks_ctx* ctx, double* W, double* gradW, double* alpha);

/* One fine residual evaluation at the current state, no update.
 *   order 3: CGKS (HWENO reconstruction + gas-kinetic flux, Sec. 2-3); order 1: first-order KFVS.
 *   res      double[5][N] = -(sum of outward face fluxes) of every cell (device, nullable)
 *   gradW_new double[15][N] the Gauss-Green gradients at t + dt times the compression factor
 *            (Sec. 2.4, 3.3; order 3 only; device, nullable)
 *   alpha_new double[N] the compression factor (order 3 only; device, nullable)
 *   dt       double[N] local time steps used by the faces (device, nullable)
 *   norm     host double: sqrt(mean over cells of (res_rho / |Omega|)^2) (nullable; synchronises) */
cgks_status cgks_residual(cgks_ctx* ctx, int order, double* res, double* gradW_new, double* alpha_new,
                          double* dt, double* norm);

/* First-order KFVS residual of level `level` for the state W double[5][n_level] (device in/out). */
cgks_status cgks_kfvs_residual(cgks_ctx* ctx, int level, const double* W, double* res);

/* Directional derivative out = J(W0) dW of the KFVS residual of level `level` (the Jacobian of
 * cgks_kfvs_residual at W0, boundary ghost states included), evaluated in FP32 forward mode with
 * FP64 sums over each cell's faces.  This is the coarse-level operator of the mixed-precision
 * V-cycle (precision 1): the coarse equations of Sec. 4.2 in defect-correction form.  W0, dW, out:
 * device double[5][n_level]; out may not alias W0 or dW.  CGKS_ENAN if W0 is not a physical state. */
cgks_status cgks_kfvs_jvp(cgks_ctx* ctx, int level, const double* W0, const double* dW, double* out);

/* n_steps explicit single-grid CGKS steps (Eq. smo).  norm_hist: host double[n_steps] of the
 * residual norm before each step (nullable; synchronises).  CGKS_ENAN if a state becomes
 * non-physical (checked at the end of the call). */
cgks_status cgks_step(cgks_ctx* ctx, int n_steps, double* norm_hist);

/* n_cycles V-cycles (Sec. 4.2): pre-smoothing CGKS step(s), defect at the new state, FAS coarse
 * levels with KFVS forward-Euler smoothing, injection correction.  norm_hist as in cgks_step. */
cgks_status cgks_vcycle(cgks_ctx* ctx, int n_cycles, double* norm_hist);

/* Iterates cgks_vcycle (multigrid != 0) or cgks_step until the residual norm falls below
 * drop x (first norm) or max_iters iterations.  Host outputs (nullable): iterations done, final
 * norm ratio, wall seconds.  The norm is read every `check_every` = 10 iterations.  After the first
 * 10 iterations, which run eagerly, each further chunk of 10 replays one CUDA graph (the same
 * kernels in the same order: the results are those of eager launches), on a private stream of the
 * context ordered after and before the context stream by events; not while kernel timing
 * (cgks_profile) is on.
 * CGKS_ENOTCONV when max_iters is reached first. */
cgks_status cgks_steady_solve(cgks_ctx* ctx, int multigrid, double drop, int64_t max_iters, int64_t* iters_done,
                              double* final_drop, double* seconds);

/* Colours of the LU-SGS sweep order of coarse level `level` (>= 1): Jones-Plassmann rounds on
 * priorities (splitmix64(cell id), cell id), each cell taking the smallest colour none of its
 * face neighbours has; the sweeps visit colour 0, 1, ... forward and back.  colors: int32[n_level]
 * (host or device, nullable); n_colors: host, nullable.  Built on first use; synchronises. */
cgks_status cgks_coarse_colors(cgks_ctx* ctx, int level, int32_t* colors, int32_t* n_colors);

/* Number of cell updates skipped by the positivity rule since the last cgks_state_init: coarse
 * forward-Euler updates and fine/coarse injection corrections that would have made rho or p
 * non-positive leave that cell unchanged (Sec. 4.2 gives no rule; skipping keeps the cycle going
 * through the start-up transient).  Synchronises. */
cgks_status cgks_skipped_updates(cgks_ctx* ctx, int64_t* count);

/* ---- Discrete adjoint of the steady problem (an extension: the paper solves, it does not
 * differentiate).  The steady compact scheme (Sec. 2.4, 4) has u = (W [5][N], grad W [15][N]) as
 * unknowns and F(u) = (Res(W, G), Gnew(W, G) - G) = 0, with Res the residual of the explicit update
 * and Gnew the Gauss-Green gradient.  For a functional J(u, beta) and parameters beta (the free-stream
 * Mach number, node displacement modes) the adjoint gives dJ/dbeta = dJ/dbeta|_u + lambda^T
 * dF/dbeta|_u with (dF/du)^T lambda = -(dJ/du)^T.  All calls need compression_factor = 0 (the
 * factor's pressure-jump terms are not differentiable where the jump vanishes) and dt_mode = 0
 * (CGKS_EUNSUPPORTED otherwise).  Vectors of 20 rows are [20][N]: the 5 rows of W then the 15 of
 * grad W, in the layouts of cgks_state_init. */

/* Forms and stores the linearisation of (Res, Gnew) at the current state by forward-mode duals
 * (41 x 10 doubles per Gauss point, 2,220 per cell; device memory owned by the context, freed with
 * the mesh).  Errors: CGKS_EINVAL (no state), CGKS_ENOMEM, CGKS_EUNSUPPORTED. */
cgks_status cgks_linearize(cgks_ctx* ctx);

/* Transposed product with the stored linearisation: (W_bar, G_bar) = (d(Res, Gnew)/d(W, G))^T
 * (res_bar, grad_bar).  res_bar [5][N], grad_bar [15][N] in; W_bar [5][N], G_bar [15][N] out (device
 * or pinned host, caller-owned).  Errors: CGKS_EINVAL (NULL array, no linearisation). */
cgks_status cgks_residual_vjp(cgks_ctx* ctx, const double* res_bar, const double* grad_bar, double* W_bar,
                              double* G_bar);

/* Wall force J = sum over wall faces (tags 1, 2) of p(W) S_component, p the pressure of the wall
 * cell's average and S the face's area vector (outward from the cell).  J: host scalar out;
 * dJ_dW: NULLable device [5][N] out (dJ/dW, zero away from the wall).  Synchronises. */
cgks_status cgks_wall_force(cgks_ctx* ctx, int component, double* J, double* dJ_dW);

/* Solves (dF/du)^T lambda = -dJ_du with the stored linearisation, in the variable mu with
 * lambda = P mu, P the local time steps over the volumes on the W rows (identity on the G rows):
 *   method 0: the transposed pseudo-time iteration of the explicit scheme, mu <- mu + (dF/du)^T P mu
 *             + dJ_du (its iteration matrix is the transpose of the scheme's, so it converges where
 *             the scheme does; the residual is checked every 25 iterations);
 *   method 1: restarted GMRES(30) on (dF/du)^T P mu = -dJ_du (30 Krylov vectors of [20][N] held on
 *             the device, allocated on first use, freed with the mesh); fewer products than method
 *             0 on small cases, but restarted GMRES can stagnate (it did on an 18,432-cell ramp).
 * dJ_du [20][N] in, lambda [20][N] out (device).  Stops when |(dF/du)^T lambda + dJ_du| <= tol
 * |dJ_du| or after max_iters transposed products; iters and rel_res (NULLable host) report the
 * count and the ratio.  Errors: CGKS_EINVAL (bad method), CGKS_ENOTCONV (tolerance not reached;
 * lambda holds the last iterate), CGKS_ENAN (divergence). */
cgks_status cgks_adjoint_solve(cgks_ctx* ctx, const double* dJ_du, int method, int64_t max_iters, double tol,
                               double* lambda, int64_t* iters, double* rel_res);

/* Gradient of the wall force (component 0..2) at the current (steady) state with respect to the
 * free-stream Mach number and to n_modes node displacement modes: node_modes host
 * [n_modes][n_nodes][3] (the upload's node order; NULL when n_modes == 0), dJ_dmodes host [n_modes]
 * out, dJ_dmach host out.  Linearises, solves the adjoint (method, max_iters, tol as
 * cgks_adjoint_solve),
 * and takes the parameter partials dF/dbeta, dJ/dbeta at the frozen state by central differences of
 * the residual with steps h_mach and h_mode (for a mode: the mesh re-uploaded with its nodes moved,
 * into a one-level context on the same stream).  Synchronises. */
cgks_status cgks_adjoint(cgks_ctx* ctx, int component, const double* node_modes, int n_modes, double h_mode,
                         double h_mach, int method, int64_t max_iters, double tol, double* dJ_dmodes,
                         double* dJ_dmach, int64_t* iters, double* rel_res);

/* Measured FP64 fused-multiply-add throughput of the current device in TFLOP/s (host output),
 * from a register-resident FMA chain kernel; the roofline denominator of the FP64-bound kernels. */
cgks_status cgks_fp64_peak(double* tflops);

/* Kernel timing for roofline measurement.  cgks_profile(ctx, 1) records CUDA events on the
 * context stream around every launch of the kernels of the cycle until cgks_profile(ctx, 0), with
 * the units each launch processes and its algorithmic DRAM bytes (every input read once, every
 * output written once; the per-unit formulas are those of the kernels' documentation).  Kernel ids
 * (`which`):
 *   0 Gauss-point gas-kinetic flux (units: Gauss points)   1 reconstruction (cells)
 *   2 fine gather / update (Gauss points seen from cells)  3 coarse KFVS face fluxes (faces)
 *   4 coarse KFVS gather (cells)                           5 coarse local time step (cells)
 *   6 FAS forcing (cells)                                  7 coarse forward-Euler update (cells)
 *   8 restriction (cells of the finer level)               9 prolongation (cells of the finer level)
 *  10 FP32 KFVS directional derivative (faces)            11 residual norm (cells)
 *  12 Gauss-point flux alone, for the V-cycle's defect     13 fine gather of the residual alone
 *     (Gauss points)                                          (Gauss points seen from cells)
 * cgks_kernel_stats synchronises the stream and returns (host outputs, each nullable) the summed
 * device time in milliseconds, the number of launches, the summed units and the summed algorithmic
 * bytes of kernel `which` recorded since profiling was enabled; an id outside 0..13 is CGKS_EINVAL. */
cgks_status cgks_profile(cgks_ctx* ctx, int enable);
cgks_status cgks_kernel_stats(cgks_ctx* ctx, int which, double* ms, int64_t* launches, double* units,
                              double* bytes);

/* Density-residual norm sqrt(mean_i (res_rho[i] / vol[i])^2) (the quantity cgks_residual reports)
 * for callers that cannot let the library allocate device memory: applications that hand each
 * component a fixed, accounted slice of GPU memory from their own pool, and loops that cannot absorb
 * the device-wide synchronisation an allocation or free may cause.  The paper has no counterpart.
 *   res_rho, vol  device double[n] (the density row of a residual and the cell volumes)
 *   norm          device double, written on `cuda_stream` (cudaStream_t; NULL = legacy stream)
 * Nothing is allocated: the partial sums live in a 512 KiB array inside the loaded module, so
 * n may be at most 67,108,864 (65,536 tiles of 1,024 cells); larger n returns CGKS_EINVAL.  The
 * first call on each device looks up that array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array: calls whose GPU work
 * overlaps (other streams, other host threads) race and may return wrong norms; serialise them.
 * Each call overwrites the partial sums it uses, so no clearing is needed between calls.  The
 * looked-up address is kept per device index for the life of the process: after cudaDeviceReset,
 * or when the device is used through a context other than its primary one, it no longer names the
 * array, so do not call this entry point after either.  The result equals cgks_residual's norm to
 * round-off (about 1e-15 relative), not bit for bit: the partial sums are grouped differently.  No
 * context is involved: on failure cgks_last_error(NULL) gives the message. */
cgks_status cgks_density_norm_noalloc(const double* res_rho, const double* vol, int64_t n, void* cuda_stream,
                                      double* norm);

/* Text of the last error of ctx (or of the last failed cgks_create when ctx is NULL). */
const char* cgks_last_error(const cgks_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
