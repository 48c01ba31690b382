/*
 * tt_iga.h -- C ABI of the TT-IGA library: a tensor-train isogeometric solver
 * for the 3D Poisson problem -Laplace(u) = f with homogeneous Dirichlet data
 * on a single-patch spline geometry, running on one NVIDIA GB300 (sm_103a).
 *
 * Method (arXiv 2509.13224):
 *   geometry coefficients R = det J J^{-1} J^{-T} (Eq. Rxi) and the source
 *   f det J sampled at tensor Gauss points are compressed into TT cores by
 *   TT-cross (Section 4.1.2, 4.2.1, 4.2.2); each core is contracted per
 *   direction with the univariate basis factors a_ij^(d) into the cores of a
 *   TT-matrix stiffness K and a TT load vector F (Section 4.2.1-4.2.2); the
 *   sum over (i, j) is recompressed by TT rounding (Section 4.2.1, global
 *   assembly); the Dirichlet rows/columns are removed (Section 4.3); and the
 *   system K u = F is solved by an AMEn TT solver (Section 4.1.2).
 *
 * Conventions shared by every call:
 *   - Return value: 0 (TT_IGA_OK) on success, a negative tt_iga_status on
 *     failure; tt_iga_last_error(ctx) then holds a one-line message.
 *   - Every call runs on the context's CUDA stream.  Device inputs must be
 *     ready when the call is made.  Calls that return host values (ranks,
 *     statistics, norms, host buffers) and the kernel-level entry points
 *     synchronise that stream before returning.
 *   - Opaque handles (tt_iga_geom, tt_iga_system, tt_iga_solution) are owned by
 *     the library and released with the matching *_destroy call; they must not
 *     outlive their context.
 *   - Pointers documented as "device" must be device (or managed) memory of the
 *     context's device; "host" pointers are ordinary host memory.  Arrays are
 *     dense, row-major (last index fastest) unless stated.
 *   - Direction d = 1, 2, 3 is parametric coordinate xi_d.  The flattened
 *     global index of a multi-index (i1, i2, i3) is g = i1 + n1 (i2 + n2 i3)
 *     (i1 fastest).  For the annulus geometry xi_1 is radial, xi_2 angular and
 *     xi_3 axial.
 *   - TT cores of a tensor with mode sizes n_k are stored as
 *     G_k[r_{k-1}][n_k][r_k] with r_0 = r_3 = 1 (Section 4.1.1).  TT-matrix
 *     cores are band-stored as M_k[r_{k-1}][n_k][2p+1][r_k]: entry (i, j) of
 *     mode k is at band slot o = j - i + p; slots with j outside [0, n_k) hold 0.
 *   - All arithmetic is FP64 unless a call says otherwise.
 */
#ifndef TT_IGA_H
#define TT_IGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_IGA_OK = 0,
  TT_IGA_ERR_ARG = -1,           /* invalid argument (null pointer, size, enum) */
  TT_IGA_ERR_OOM = -2,           /* device allocation failed */
  TT_IGA_ERR_CUDA = -3,          /* a CUDA runtime call or kernel launch failed */
  TT_IGA_ERR_NOT_CONVERGED = -4, /* iteration cap reached; a partial result is still returned */
  TT_IGA_ERR_TIMEOUT = -5,       /* a bounded device-side wait ran out */
  TT_IGA_ERR_TOO_LARGE = -6,     /* a size exceeds a documented limit */
  TT_IGA_ERR_BAD_GEOMETRY = -7,  /* det J <= 0 somewhere on the quadrature grid */
  TT_IGA_ERR_STATE = -8          /* handle used with the wrong context or in the wrong state */
} tt_iga_status;

typedef struct tt_iga_ctx tt_iga_ctx;
typedef struct tt_iga_geom tt_iga_geom;
typedef struct tt_iga_system tt_iga_system;
typedef struct tt_iga_solution tt_iga_solution;

/* ---------------------------------------------------------------- context */

typedef struct {
  void *stream;  /* cudaStream_t to run on (cudaStreamLegacy = (void*)1 is accepted); NULL: the
                  * library creates its own non-blocking stream */
  int device;    /* CUDA device ordinal */
  /* Optional device allocator (both or neither).  NULL: stream-ordered
   * cudaMallocAsync / cudaFreeAsync on the context stream.  Returned pointers
   * must be 256-byte aligned, as cudaMalloc's are (bulk copies into shared
   * memory need 16); a misaligned pointer is handed back to free_fn and the
   * call fails with TT_IGA_ERR_ARG. */
  void *(*alloc_fn)(size_t bytes, void *stream, void *user);
  void (*free_fn)(void *ptr, void *stream, void *user);
  void *alloc_user;
} tt_iga_ctx_opts;

/* Create a context.  o may be NULL (device 0, own stream, default allocator). */
int tt_iga_ctx_create(tt_iga_ctx **ctx, const tt_iga_ctx_opts *o);
/* Synchronise and destroy; releases everything the context still owns. */
void tt_iga_ctx_destroy(tt_iga_ctx *ctx);
/* Message of the last failing call on ctx ("" if none).  Valid until the next call. */
const char *tt_iga_last_error(const tt_iga_ctx *ctx);
/* Bytes currently held by the context's device allocations. */
int tt_iga_ctx_memory(const tt_iga_ctx *ctx, size_t *bytes_in_use, size_t *bytes_peak);
/* Number of CUDA kernels the library has launched in this process (all contexts). */
unsigned long long tt_iga_launch_count(void);
/* Limit the context's cooperative kernels (the fused local PCG, one grid-wide
 * launch per AMEn local solve) to max_sms SMs' worth of CTAs (0: the whole
 * GPU, the default).  Several contexts solving at once (batch lanes, serving
 * lanes) can then run their local solves side by side instead of queueing for
 * the whole GPU; other kernels are not limited.  A smaller grid changes the
 * order of the PCG's partial sums, so results can differ in the last bits. */
int tt_iga_ctx_set_sm_limit(tt_iga_ctx *ctx, int max_sms);

/* Live timing of one kernel family on the context stream, for roofline
 * reporting: every launch of the family is bracketed by a CUDA event pair.
 * family: 0 off, 1 band stage of the AMEn local matvec, 2 FP64 GEMM,
 * 3 Householder QR panel, 6 fused local PCG.  Enabling resets the record. */
int tt_iga_profile_enable(tt_iga_ctx *ctx, int family);
/* Synchronise and return the summed event time (ms), the number of timed
 * launches and their summed algorithmic FLOPs. */
int tt_iga_profile_read(tt_iga_ctx *ctx, double *ms_total, long long *launches, double *flops_total);

/* --------------------------------------------------------------- geometry */

enum { TT_IGA_GEOM_BOX = 0, TT_IGA_GEOM_ANNULUS = 1, TT_IGA_GEOM_NURBS = 2 };

/* Geometry and discretisation (Section 3.3, Section 2).
 *  ANNULUS: quarter annulus of radii r_in < r_out and height `height`: radial
 *    degree-1 B-spline, angular quadratic NURBS quarter arc (weights 1,
 *    sqrt(2)/2, 1), axial degree-1 B-spline, composed with a twist about z by
 *    angle twist*zeta and a radial swell 1 + swell*sin(pi zeta), zeta = z/height.
 *  BOX: [0,lx] x [0,ly] x [0,lz].
 * Discretisation: open uniform knots with n[d] B-splines of degree p per
 * direction (n[d] >= p+2 so that interior unknowns exist), nq Gauss points
 * per element (0: p+1).  The coefficient fields R_ij are compressed by TT-cross
 * to relative accuracy cross_tol with TT ranks capped at max_rank (0: 64);
 * seed drives the random fibre and validation samples. */
typedef struct {
  int kind;
  double r_in, r_out, height, twist, swell;
  double lx, ly, lz;
  int p;
  int n[3];
  int nq;
  double cross_tol;
  int max_rank;
  uint64_t seed;
} tt_iga_geom_desc;

/* Build the 1D tables of every direction and the TT cores of the six unique
 * entries of R (Section 4.2.1, R_ij^TT) on the device.  ERR_BAD_GEOMETRY if a
 * sampled det J <= 0; ERR_NOT_CONVERGED if the cross did not validate within
 * max_rank (the handle is still returned). */
int tt_iga_geometry(tt_iga_ctx *ctx, const tt_iga_geom_desc *g, tt_iga_geom **out);

#define TT_IGA_NURBS_MAX_DEGREE 4
#define TT_IGA_NURBS_MAX_CP 64

/* A single-patch trivariate NURBS volume (Section 2.2):
 *   x(xi) = sum_a w_a P_a N_a(xi) / sum_a w_a N_a(xi),  N_a = N_a1(xi_1) N_a2(xi_2) N_a3(xi_3),
 * with degree deg[d] (1 .. TT_IGA_NURBS_MAX_DEGREE) and ncp[d] control points
 * (deg[d] + 1 .. TT_IGA_NURBS_MAX_CP) per direction, open knot vectors knots[d]
 * of ncp[d] + deg[d] + 1 nondecreasing values starting with deg[d] + 1 zeros and
 * ending with deg[d] + 1 ones, control points ctrl[(i3 ncp[1] + i2) ncp[0] + i1][3]
 * and positive weights weights[(i3 ncp[1] + i2) ncp[0] + i1] (xi_1 fastest).
 * Host pointers, read during tt_iga_geometry_nurbs only.  The solution space is
 * the one of tt_iga_geom_desc (degree p, n[d] functions on open uniform knots),
 * independent of the patch's own knots: the patch is the exact geometry. */
typedef struct {
  int deg[3];
  int ncp[3];
  const double *knots[3];
  const double *ctrl;
  const double *weights;
} tt_iga_nurbs_patch;

/* tt_iga_geometry for a NURBS patch: g supplies the discretisation (p, n, nq,
 * cross_tol, max_rank, seed) and g->kind must be TT_IGA_GEOM_NURBS.  Systems on
 * this geometry take CONSTANT right-hand sides (the manufactured solutions are
 * defined for the annulus and the box).  ERR_ARG on a malformed patch. */
int tt_iga_geometry_nurbs(tt_iga_ctx *ctx, const tt_iga_geom_desc *g, const tt_iga_nurbs_patch *patch,
                          tt_iga_geom **out);
void tt_iga_geom_destroy(tt_iga_geom *g);
/* TT ranks (r1, r2) of field f = 0..5 in the order R11, R12, R13, R22, R23, R33
 * (rank 0 marks a field that is zero to the cross tolerance), plus the
 * validated maximum relative sample error of each field. */
int tt_iga_geom_ranks(const tt_iga_geom *g, int ranks[6][2], double max_rel_err[6]);

/* ------------------------------------------------------------ right-hand side */

enum { TT_IGA_RHS_MANUFACTURED = 0, TT_IGA_RHS_CONSTANT = 1, TT_IGA_RHS_RING_LOG = 2 };
#define TT_IGA_MAX_MODES 8

/* Source term.  MANUFACTURED: f = -Laplace(u) of the bubble solution of the
 * geometry (annulus: (rho^2 - r_in^2)(r_out^2 - rho^2) x' y' zeta (1 - zeta) in
 * the coordinates with twist and swell undone; box: sin(pi x/lx) sin(pi y/ly)
 * sin(pi z/lz)) times 1 + sum_k a[k] sin(b[k] . x + c[k]); the Laplacian is
 * taken exactly on the device by hyper-dual arithmetic.  CONSTANT: f = value.
 * RING_LOG: f = value (0 for the ring problem of Section 4.3); on the annulus
 * without twist and swell, with value 0, zero flux on the four faces of
 * directions 1 and 2, and on each radial face (xi_1 = 0: rho = r_in, xi_1 = 1:
 * rho = r_out) either Dirichlet data or a flux, at least one of them Dirichlet,
 * the exact solution is u = A + B ln(rho / r_in): Dirichlet data u_in, u_out on
 * both gives A = u_in, B = (u_out - u_in) / ln(r_out / r_in); a flux q on the
 * outer face gives B = q r_out, on the inner face B = -q r_in (outward normal
 * -rho), and the Dirichlet face fixes A.  tt_iga_l2_error compares against it,
 * with the data taken from the solution's boundary conditions. */
typedef struct {
  int kind;
  int n_modes; /* 0 .. TT_IGA_MAX_MODES */
  double a[TT_IGA_MAX_MODES];
  double b[TT_IGA_MAX_MODES][3];
  double c[TT_IGA_MAX_MODES];
  double value;
} tt_iga_rhs_desc;

/* --------------------------------------------------------------- assembly */

/* Assemble the restricted TT system (Sections 4.2-4.3): K^TT = sum_ij K_ij^TT
 * from the R_ij cores by per-direction quadrature contraction, rounded to
 * relative accuracy round_tol (Oseledets QR + SVD rounding, FP64), and one TT
 * load vector per right-hand side (f det J by TT-cross to cross_tol, then the
 * per-direction contraction with N_d).  Boundary functions 0 and n_d - 1 of
 * every direction are dropped (homogeneous Dirichlet data), so the unknowns
 * per direction are n_d - 2.  rhs points to n_rhs descriptors (n_rhs >= 1). */
int tt_iga_assemble(tt_iga_ctx *ctx, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int n_rhs,
                    double round_tol, tt_iga_system **out);

/* Boundary conditions (Section 4.3).  Face f = 2 d + side of parametric
 * direction d = 0, 1, 2 (side 0: xi_d = 0, side 1: xi_d = 1; for the annulus
 * d = 0 is the radial direction).  dirichlet[f] != 0: u = value[f] on the face
 * (constant data), imposed by dropping the basis function that is
 * interpolatory there and moving the data to the right-hand side,
 * F <- F - K g with g the lift carrying the data on the dropped functions;
 * dirichlet[f] == 0: natural condition with the constant outward normal flux
 * du/dn = flux[f] (0: zero flux), which adds the face's part of the surface
 * load vector f_s (Section 3.3; the boundary term of the weak form of Section
 * 3.2), int_face flux[f] N_a dGamma, to every right-hand side; the area density
 * |dx/dxi_e x dx/dxi_f| of the face (e, f its tangential directions) is a
 * TT-cross of its own, contracted with the same per-direction Gauss rules as
 * the volume load.  Nonzero values are accepted on the faces of one direction
 * only, and the faces of the other two directions must then be natural; at
 * least one face must be Dirichlet (otherwise K is singular); a nonzero flux
 * is accepted on natural faces only; values and fluxes must be finite.
 * Violations return TT_IGA_ERR_ARG. */
typedef struct {
  int dirichlet[6];
  double value[6];
  double flux[6];
} tt_iga_bc_desc;

/* tt_iga_assemble with boundary conditions bc (tt_iga_assemble is the case of
 * six homogeneous Dirichlet faces).  The unknowns of direction d are the basis
 * functions lo_d .. n_d - 1 - hi_d, lo_d / hi_d = 1 when face 2d / 2d+1 is
 * Dirichlet, so the mode sizes are n_d - lo_d - hi_d; the solution, its
 * evaluation and its L2 error include the lift. */
int tt_iga_assemble_bc(tt_iga_ctx *ctx, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int n_rhs,
                       double round_tol, const tt_iga_bc_desc *bc, tt_iga_system **out);
void tt_iga_system_destroy(tt_iga_system *s);
/* Operator TT ranks (R1, R2), load ranks of right-hand side k, and mode sizes. */
int tt_iga_system_info(const tt_iga_system *s, int op_ranks[2], int n_rhs_max, int (*rhs_ranks)[2],
                       int modes[3]);

/* ------------------------------------------------------------------ solve */

enum { TT_IGA_FP64 = 0, TT_IGA_MIXED_FP32 = 1, TT_IGA_MIXED_TF32 = 2 };

/* AMEn options (Section 4.1.2).  tol: target relative residual
 * ||F - K u||_2 / ||F||_2.  precision FP64: every operator application,
 * inner product, residual and update in FP64 (the band block-Jacobi
 * preconditioner of the local PCG is factorised and applied in FP32; it
 * shapes the iteration only).  MIXED_FP32: the local PCG runs in FP32 on the
 * CUDA cores inside FP64 iterative refinement of each local system;
 * interfaces, residuals and QR/SVD truncation stay FP64.  MIXED_TF32: as
 * MIXED_FP32, with the two dense contractions of each local operator
 * application (the right-interface stage p PhiR^T and the left-interface stage
 * PhiL T2) on the tensor cores: tcgen05 kind::tf32 MMAs with FP32
 * accumulators in tensor memory, each operand split into TF32 high and low
 * parts and three products summed (3xTF32, about FP32 accuracy); the banded
 * operator stage and the preconditioner stay on CUDA cores.  A local system
 * whose operands do not fit the kernel's shared-memory and tensor-memory budget
 * is solved on CUDA cores (stats.local_matvecs_tensor counts the applications
 * that used the tensor cores).  Zero fields take the defaults in brackets. */
typedef struct {
  double tol;       /* [1e-8] */
  int precision;    /* [TT_IGA_FP64] */
  int max_sweeps;   /* [30] */
  int kickrank;     /* [4] residual enrichment columns per step; negative disables */
  int max_rank;     /* [256] */
  int local_maxit;  /* [500] local PCG iteration cap */
  int rhs_index;    /* which right-hand side of the system to solve [0] */
  int verbose;      /* print one line per sweep to stderr */
  double local_rtol; /* inexact local solves: each AMEn local system is solved until its residual is
                        below max(the bound that tol implies, local_rtol x its initial residual);
                        negative: the bound alone (every local system to full accuracy) [-1] */
} tt_iga_solve_opts;

typedef struct {
  int sweeps;
  int ranks[2];
  double rel_residual;      /* exact ||F - K u|| / ||F|| (see tt_iga_residual), or -1 if it could not
                               be computed: converged then rests on the local residuals */
  double local_residual;    /* largest relative local residual of the last sweep */
  long long local_matvecs;  /* local operator applications (all precisions) */
  long long local_matvecs_fp64;
  double ms_total;          /* device time of the solve (CUDA events) */
  int converged;
  long long local_matvecs_tensor;  /* local operator applications on the tensor cores (MIXED_TF32) */
} tt_iga_stats;

/* Solve K u = F for right-hand side opts->rhs_index.  On ERR_NOT_CONVERGED the
 * last iterate is returned in *out.  st may be NULL. */
int tt_iga_solve(tt_iga_ctx *ctx, const tt_iga_system *s, const tt_iga_solve_opts *opts,
                 tt_iga_solution **out, tt_iga_stats *st);
void tt_iga_solution_destroy(tt_iga_solution *u);
/* TT ranks of the solution. */
int tt_iga_solution_ranks(const tt_iga_solution *u, int ranks[2]);
/* Exact relative residual ||F - K u||_2 / ||F||_2 of u against right-hand side k,
 * computed in TT arithmetic with orthogonal projections (FP64) while the TT rank
 * of F - K u stays within 256; above that, for problems of at most 2^22
 * unknowns, by expanding F and K u to dense vectors on the device.
 * TT_IGA_ERR_TOO_LARGE when neither applies. */
int tt_iga_residual(tt_iga_ctx *ctx, const tt_iga_system *s, const tt_iga_solution *u, int k,
                    double *rel_residual);

/* tt_iga_solve started from the iterate u0 instead of a random rank-2 TT
 * (AMEn of Section 4.1.2 with a given initial guess): a solution of a nearby
 * problem, or one rebuilt from exported cores by tt_iga_import_cores, so that
 * a solve can resume from a checkpoint.  u0's mode sizes (and block layout)
 * must equal those of s; its ranks are kept as the starting ranks (1..256).
 * The result is a new handle; u0 is not modified.  Return codes as
 * tt_iga_solve, plus TT_IGA_ERR_STATE when a handle belongs to another
 * context. */
int tt_iga_solve_from(tt_iga_ctx *ctx, const tt_iga_system *s, const tt_iga_solve_opts *opts, const tt_iga_solution *u0,
                      tt_iga_solution **out, tt_iga_stats *st);

/* Several right-hand sides as one block-TT solve (AMEn of Section 4.1.2 on the
 * block system).  tt_iga_system_stack builds the block system of all n_rhs
 * right-hand sides of s: the right-hand-side index k is merged into TT mode
 * `mode` (0, 1 or 2; index i_d + m_d k, so that mode's size becomes n_rhs m_d),
 * the operator is I (x) K (that core of K repeated on the diagonal blocks of
 * the merged mode, no coupling across blocks) and its single load holds
 * F_k / ||F_k|| in block k (TT ranks added,
 * then rounded to relative accuracy eps; 0: 1e-14).  scales (host, n_rhs
 * doubles, may be NULL) receives ||F_k||.  A solution of the block system
 * (tt_iga_solve with rhs_index 0) is sliced by tt_iga_solution_unstack: block
 * k times scale, the solution of right-hand side k of s, rounded to 1e-14
 * relative accuracy (so its TT ranks are its own numerical ranks, not the block
 * solution's, which span every right-hand side).  tt_iga_eval and tt_iga_l2_error reject block solutions.
 * TT_IGA_ERR_ARG for a mode outside 0..2, a system that is already a block
 * system, a zero right-hand side, a block index outside 0..n_rhs-1 or a
 * non-finite scale.  The new handles belong to the caller (release with
 * tt_iga_system_destroy / tt_iga_solution_destroy). */
int tt_iga_system_stack(tt_iga_ctx *ctx, const tt_iga_system *s, int mode, double eps, tt_iga_system **out,
                        double *scales);
int tt_iga_solution_unstack(tt_iga_ctx *ctx, const tt_iga_solution *ub, int k, double scale,
                            tt_iga_solution **out);
/* Every right-hand side of s by one block-TT solve: stack, solve the block
 * system to relative residual opts->tol / sqrt(n_rhs) (the block residual is
 * the root mean square of the per-right-hand-side relative residuals, so each
 * of them meets opts->tol), unstack.  out (host array of n_rhs handles)
 * receives the solutions, also on ERR_NOT_CONVERGED; rel_res (host, n_rhs, may
 * be NULL) the exact per-right-hand-side relative residuals (-1 where the TT
 * rank of F_k - K u_k would exceed 256); st the block solve's statistics.
 * mode: the TT mode that carries the right-hand-side index (0, 1, 2; -1: 1,
 * the middle mode, whose two neighbouring ranks then span the unions of the
 * solutions' outer-mode subspaces).  opts->rhs_index is ignored. */
int tt_iga_solve_block(tt_iga_ctx *ctx, const tt_iga_system *s, const tt_iga_solve_opts *opts, int mode,
                       tt_iga_solution **out, tt_iga_stats *st, double *rel_res);

/* Copy the solution's TT cores to host memory: out receives core 1
 * [1][m1][r1], core 2 [r1][m2][r2] and core 3 [r2][m3][1] back to back (FP64);
 * modes[3] (m_d = n_d - 2 with six Dirichlet faces, n_d - lo_d - hi_d in
 * general, see tt_iga_assemble_bc) and ranks[4] are filled.  ERR_TOO_LARGE if cap (in
 * doubles) is too small; pass out = NULL to query the sizes only. */
int tt_iga_solution_cores(tt_iga_ctx *ctx, const tt_iga_solution *u, double *out, size_t cap, int modes[3],
                          int ranks[4]);

/* The inverse of tt_iga_solution_cores: a solution of system s rebuilt from
 * host TT cores in the TT format of Section 4.1.1 (core 1 [1][m1][r1], core 2
 * [r1][m2][r2], core 3 [r2][m3][1] back to back, FP64; host pointer, read
 * during the call only).  modes[3] must equal the system's mode sizes (the
 * unknowns per direction) and ranks[4] = {1, r1, r2, 1} with 1 <= r1, r2 <=
 * 256; the solution takes the system's degree, boundary layout (lift) and
 * block layout.  A solution exported, imported and evaluated gives the same
 * values.  TT_IGA_ERR_ARG for mismatched sizes or a non-finite core entry. */
int tt_iga_import_cores(tt_iga_ctx *ctx, const tt_iga_system *s, const double *cores, const int modes[3],
                        const int ranks[4], tt_iga_solution **out);

/* ------------------------------------------------------------ evaluation */

/* u_h(xi) = sum_a u_a N_a(xi) at m parametric points xi[m][3] in [0,1]^3.
 * xi and u_out are device pointers (FP64). */
int tt_iga_eval(tt_iga_ctx *ctx, const tt_iga_solution *u, int m, const double *xi, double *u_out);
/* Relative L2 error sqrt(int (u_h - u)^2) / sqrt(int u^2) over the mapped
 * domain (Eq. L2norm, with p+3 Gauss points per element) against the exact
 * solution of rhs: the manufactured solution (kind MANUFACTURED), or the log
 * solution of the ring problem (kind RING_LOG: annulus without twist and swell,
 * data on the radial faces only, taken from u's boundary conditions). */
int tt_iga_l2_error(tt_iga_ctx *ctx, const tt_iga_geom *g, const tt_iga_solution *u,
                    const tt_iga_rhs_desc *rhs, double *rel_l2);

/* Relative L2 difference of two solutions on the mapped domain of g (Eq.
 * L2norm applied to u_h - v_h):
 *   sqrt( int (u_h - v_h)^2 dOmega / int v_h^2 dOmega ),
 * with the Gauss rule of the discretisation (nq points per element and
 * direction) and det J by TT-cross to g's cross tolerance.  Computed in TT
 * arithmetic: the mass matrix int N_a N_b det J is assembled per direction
 * like the stiffness (Section 4.2.1, selector (N, N) in every direction), and
 * w = u - v is rounded (QR + SVD, Section 4.2.1) before w^T M w is formed, so
 * the difference of two nearly equal solutions is resolved to about 1e-15 of
 * ||v||.  u and v must share g's discretisation and boundary layout and carry
 * no Dirichlet lift (TT_IGA_ERR_ARG otherwise). */
int tt_iga_l2_diff(tt_iga_ctx *ctx, const tt_iga_geom *g, const tt_iga_solution *u, const tt_iga_solution *v,
                   double *rel_l2);

/* ------------------------------------------------------------ batching */

/* How an instance's right-hand sides are solved: BLOCK, one block-TT solve of
 * all of them (tt_iga_solve_block, right-hand-side index in the middle TT
 * mode; each meets opts.tol); EACH, one AMEn solve per right-hand side. */
enum { TT_IGA_RHS_BLOCK = 0, TT_IGA_RHS_EACH = 1 };

/* One instance of a batch: geometry and discretisation, its right-hand sides
 * (host array of n_rhs descriptors, 1..8), the assembly rounding tolerance,
 * the solve options (rhs_index is ignored: every right-hand side is solved)
 * and rhs_solve (TT_IGA_RHS_BLOCK or TT_IGA_RHS_EACH; a single right-hand
 * side is always solved by tt_iga_solve). */
typedef struct {
  tt_iga_geom_desc geom;
  int n_rhs;
  const tt_iga_rhs_desc *rhs;
  double round_tol;
  tt_iga_solve_opts opts;
  int rhs_solve;
  /* Optional (NULL: none): host buffer of cores_cap doubles that receives the
   * solution of every right-hand side k = 0 .. n_rhs-1 as TT cores in the layout
   * of tt_iga_solution_cores, back to back; the result's rhs_ranks give their
   * ranks.  TT_IGA_ERR_TOO_LARGE when they do not fit. */
  double *cores_out;
  size_t cores_cap;
} tt_iga_batch_item;

typedef struct {
  int status;                /* tt_iga_status of this instance */
  int ranks[2];              /* solution ranks of its last right-hand side (BLOCK: of all) */
  int sweeps;                /* AMEn sweeps summed over its solves */
  double rel_residual_max;   /* worst exact relative residual over its right-hand sides
                                (-1 where one was skipped for its TT rank) */
  long long dofs;            /* n1 n2 n3 times the number of right-hand sides */
  double ms_geometry, ms_assemble, ms_solve;  /* host wall clock per phase */
  double t_start_ms, t_end_ms;                /* start / end relative to the batch start */
  int rhs_ranks[8][2];                        /* solution ranks per right-hand side (with cores_out) */
} tt_iga_batch_result;

/* Solve `count` independent instances on `device` with `lanes` concurrent
 * contexts (each its own stream and host thread, 1..64) fed from a work queue,
 * largest instance first.  sm_per_lane: the SM budget of each lane's
 * cooperative kernels (tt_iga_ctx_set_sm_limit): -1 an equal share, the SM
 * count divided by the number of lanes, so that the lanes' local PCG kernels
 * run side by side; 0 the whole GPU for every lane (independent solves that
 * queue for the SMs); > 0 that many SMs.  results[count] (host) receives one
 * record per instance in input order; *wall_ms (may be NULL) the batch wall
 * time.  With more than one lane, each lane runs the parts of a call
 * sequentially on its own stream (a single context runs the coefficient fields
 * and the operator and loads on helper streams and host threads instead): the
 * lanes already overlap, and extra host threads would compete with them for
 * the CPU.  Many lanes want as many hardware work queues
 * (CUDA_DEVICE_MAX_CONNECTIONS, set before CUDA starts; the default is 8).
 * Returns TT_IGA_OK or the first failing instance's status.  Results do
 * not depend on the lane count or the SM budget beyond the grid sizes of the
 * local PCG, whose reductions are summed in a fixed order per grid. */
int tt_iga_batch_solve(int device, int count, const tt_iga_batch_item *items, int lanes, int sm_per_lane,
                       tt_iga_batch_result *results, double *wall_ms);
/* Autotuner: run the batch once for every pair of lane count (lane_candidates)
 * and SM budget per lane (share_candidates, as sm_per_lane above; none given:
 * -1) and report the fastest pair (*best_lanes, *best_sm_per_lane, may be
 * NULL) and its wall time (*best_ms, may be NULL); results hold the last run. */
int tt_iga_batch_autotune(int device, int count, const tt_iga_batch_item *items, const int *lane_candidates,
                          int n_lane_candidates, const int *share_candidates, int n_share_candidates,
                          tt_iga_batch_result *results, int *best_lanes, int *best_sm_per_lane, double *best_ms);

/* ----------------------------------------------------- dense test hooks */

/* Dense restricted operator (N x N, N = prod(n_d - 2), host, row g = i1 + ...).
 * ERR_TOO_LARGE if N > 4096 or cap < N*N. */
int tt_iga_densify_operator(tt_iga_ctx *ctx, const tt_iga_system *s, double *out, size_t cap);
/* Dense restricted load vector k / solution (N entries, host). ERR_TOO_LARGE if N > 2^22. */
int tt_iga_densify_rhs(tt_iga_ctx *ctx, const tt_iga_system *s, int k, double *out, size_t cap);
int tt_iga_densify_solution(tt_iga_ctx *ctx, const tt_iga_solution *u, double *out, size_t cap);
/* Entries of the restricted operator / load / solution at m multi-indices
 * (host int arrays rows[m][3], cols[m][3], 0-based restricted indices) into host out[m]. */
int tt_iga_operator_entries(tt_iga_ctx *ctx, const tt_iga_system *s, int m, const int *rows,
                            const int *cols, double *out);
int tt_iga_vector_entries(tt_iga_ctx *ctx, const tt_iga_system *s, const tt_iga_solution *u, int k,
                          int m, const int *idx, double *out);

/* ------------------------------------------------- kernel-level entry points */

/* 1D tables (Section 2.1): Q = (n - p) * nq Gauss points of the open uniform
 * knot vector, ordered element by element.  Device outputs: pts[Q], wts[Q],
 * N[Q][p+1], dN[Q][p+1] (value / derivative of basis e + k at point q of
 * element e).  p <= 7, nq <= 8. */
int tt_iga_basis_tables(tt_iga_ctx *ctx, int n, int p, int nq, double *pts, double *wts, double *N,
                        double *dN);

/* Point evaluator (Section 3.3, Eq. Rxi): for m grid points given by device
 * int32 idx[m][3] into the Gauss grids of g, writes device out[m][8] =
 * (R11, R12, R13, R22, R23, R33, det J, f det J) with f from rhs (may be NULL:
 * f = 0).  *bad_geometry (host) is set to the number of points with det J <= 0. */
int tt_iga_geom_points(tt_iga_ctx *ctx, const tt_iga_geom *g, const tt_iga_rhs_desc *rhs, int m,
                       const int *idx, double *out, long long *bad_geometry);

/* Per-direction quadrature contraction (Section 4.2.1):
 *   M[a][o][b] with b index = beta: M[alpha][i][o][beta] = sum_q w_q G[alpha][q][beta] A[i][q] B[i+o-p][q]
 * for a coefficient core G[r0][Q][r1] (device), with A, B chosen by
 * test_deriv / trial_deriv (0: N, 1: N') from the tables of tt_iga_basis_tables
 * for (n, p, nq).  Output M[r0][n][2p+1][r1] (device, fully overwritten). */
int tt_iga_stiffness_core(tt_iga_ctx *ctx, int n, int p, int nq, const double *wts, const double *N,
                          const double *dN, const double *G, int r0, int r1, int test_deriv,
                          int trial_deriv, double *M);
/* Load contraction (Section 4.2.2): F[alpha][i][beta] = sum_q w_q G[alpha][q][beta] N_i(q). */
int tt_iga_load_core(tt_iga_ctx *ctx, int n, int p, int nq, const double *wts, const double *N,
                     const double *G, int r0, int r1, double *F);

/* TT rounding (Oseledets 2011, the recompression used after each summation in
 * Section 4.2.1): right-to-left QR orthogonalisation then left-to-right
 * truncated SVD with threshold eps ||X||_F / sqrt(d - 1), FP64.
 * Input: d = 3 cores (device) of mode sizes nm[3] (n_k, or n_k (2p+1) for
 * band-stored TT-matrices) and ranks r[4] (r[0] = r[3] = 1, r1, r2 <= 256).
 * Output: the rounded cores are written to out_cores[k] (device, caller-owned,
 * each with room for at least r[k] nm[k] r[k+1] doubles -- rounding never
 * raises a rank) and their ranks to out_r[4] (host).  out_cores may alias
 * cores.  max_rank caps the result (0: none). */
int tt_iga_round(tt_iga_ctx *ctx, const int nm[3], const int r[4], const double *const cores[3],
                 double eps, int max_rank, double *const out_cores[3], int out_r[4]);

/* Dense FP64 GEMM used by the rank-by-rank contractions of the local systems:
 * C = alpha op(A) op(B) + beta C, row-major, op(X) = X or X^T (ta, tb).
 * op(A) is m x k with element (i, l) at A[i*lda + l] (ta = 0) or A[l*lda + i]
 * (ta = 1); likewise B (k x n) and C (m x n, ldc).  All device pointers. */
int tt_iga_gemm_f64(tt_iga_ctx *ctx, int ta, int tb, int m, int n, int k, double alpha, const double *A, int lda,
                    const double *B, int ldb, double beta, double *C, int ldc);

/* Tall-skinny Householder QR, FP64: A (device, m x k row-major, lda >= k)
 * = Q R with Q (device, m x k, ld k) orthonormal columns and R (device, k x k
 * upper triangular).  k <= 256.  Q may alias A only if lda == k. */
int tt_iga_qr(tt_iga_ctx *ctx, int m, int k, const double *A, int lda, double *Q, double *R);
/* Block-band preconditioner of an AMEn local system (Section 4.1.2, local
 * solves): solves B z = r once, where B is the symmetric part of
 * sum_{g,d} PhiL[:, g, :] (x) A[g, :, :, d] (x) PhiR[:, d, :] over the unknowns
 * x[a][i][c] (index (a n + i) rr + c), with the FP32 factor the AMEn local PCG
 * uses for interface blocks m = rl rr <= 8 (odd-even reduction of the
 * block-tridiagonal super-row form).  PhiL (device, rl x Rl x rl), A (device,
 * band-stored operator core [Rl][n][2p+1][Rr], slot o = j - i + p), PhiR
 * (device, rr x Rr x rr), r and z (device, rl n rr).  B must be symmetric
 * positive definite; the result is B^{-1} r to FP32 accuracy.  Returns
 * TT_IGA_ERR_TOO_LARGE when m > 8, n > 1024 or p > 7.  A test entry point: the
 * solver applies the same factor inside its PCG. */
int tt_iga_blockband_solve(tt_iga_ctx *ctx, int rl, int rr, int Rl, int Rr, int n, int p, const double *PhiL,
                           const double *A, const double *PhiR, const double *r, double *z);
/* SVD of a small square matrix A (device, k x k): A = U diag(s) V^T by
 * one-sided Jacobi on the rows of A, FP64, singular values descending.
 * U, s, V row-major device buffers (k x k, k, k x k).  U has orthonormal
 * columns to FP64 precision; column j of V has unit norm (zero when s_j = 0)
 * and is orthogonal to the others to about eps s_0 / s_j.  k <= 256. */
int tt_iga_svd_small(tt_iga_ctx *ctx, int k, const double *A, double *U, double *s, double *V);
/* Allocation-free SVD.  The paper has no counterpart: this is a library
 * service for callers that cannot allocate device memory.  Such callers are,
 * for example, a serving process that reserved all of the GPU's memory for its
 * own pools at start-up and forbids any further cudaMalloc, code whose
 * allocator is not reachable from where it runs (a plug-in handed only a
 * stream and buffers), and code on a latency budget that an allocation, or
 * its failure under memory pressure, would break.
 *
 * Same factorisation as tt_iga_svd_small (A = U diag(s) V^T by one-sided
 * Jacobi, FP64, singular values descending).  It takes no context (creating
 * one allocates) and runs on `stream` (a cudaStream_t; NULL is the legacy
 * default stream).  A, U, s, V are caller-owned device buffers as in
 * tt_iga_svd_small; info (device int, may be NULL) receives 0 when the Jacobi
 * sweeps converged and 1 when they had not after 60 sweeps (the factors are
 * then those of the last sweep).  Outputs are valid once `stream` has been
 * synchronised.
 *
 * Scratch: a fixed 1 MiB array inside the library (two 256 x 256 FP64 panels),
 * which every GPU that loads the library holds until the process exits.  No
 * cudaMalloc, cudaFree or allocating library routine is called.
 * Limit: k <= 256; larger k returns TT_IGA_ERR_TOO_LARGE and launches nothing.
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress, no allocation) and caches it; make
 * that first call before any stream capture.  A cudaDeviceReset invalidates
 * the cached address, so do not call this entry point after one.
 * All calls share the array and every call overwrites it before reading it:
 * calls whose kernels can overlap on the GPU (different streams with no
 * ordering between them) race on it and must not be issued.
 * Returns TT_IGA_OK once the kernel is enqueued, TT_IGA_ERR_ARG for a null
 * buffer, TT_IGA_ERR_CUDA when the launch itself fails (its own return code;
 * an error left by other work is neither reported nor cleared).  No message is
 * recorded (there is no context). */
int tt_iga_svd_small_noalloc(void *stream, int k, const double *A, double *U, double *s, double *V, int *info);
/* Maximum-volume row selection (Goreinov et al. 2010) of a tall matrix U
 * (device, m x r): device outputs rows[r] (int32) and B = U U[rows,:]^{-1}
 * (device, m x r).  Stops when max |B| <= 1 + delta or after maxit swaps. */
int tt_iga_maxvol(tt_iga_ctx *ctx, int m, int r, const double *U, double delta, int maxit, int *rows,
                  double *B);

#ifdef __cplusplus
}
#endif
#endif /* TT_IGA_H */
