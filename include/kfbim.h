/*
 * kfbim.h - C ABI of the GB300 kernel-free boundary integral (KFBI) solver for
 * the 3D Stokes interior Dirichlet problem (arXiv 2303.04992).
 *
 * Problem (Sec. 2, Eq. SP):  -mu Lap u + grad p = f,  div u = 0 in Omega,
 * u = g on Gamma = dOmega.  Omega is embedded in the cube B = [lo, hi]^3 with
 * an N^3 MAC grid (Sec. 4.2).  The solution is u = G_v f - M_v phi with the
 * density phi solving the second-kind BIE 1/2 phi - M_v phi = g - G_v f
 * (Eq. BIE-S), solved by GMRES from phi = 0 (Alg. 1 step 3).  Every integral is
 * evaluated by solving the unified interface problem IUS-1..5 on the grid
 * (Sec. 4): corrected MAC scheme (Eq. MAC), Schur-complement CG with an FFT
 * Poisson solver (Eq. linearS1, items i-iii), and ten-node quadratic trace
 * interpolation (Sec. 4.4).
 *
 * Conventions
 *  - Every pointer named *_dev is CUDA device memory owned by the caller; every
 *    *_host pointer is host memory owned by the caller.  The library owns its
 *    context, tables and workspace (allocated in kfbim_setup, freed in
 *    kfbim_destroy).
 *  - Work is enqueued on the caller's `stream` (a cudaStream_t, NULL = legacy
 *    default stream).  Calls that iterate to a tolerance synchronise that stream
 *    to read one convergence scalar per iteration.
 *  - Grid fields are N^3 doubles in C order [k][j][i] (i = x fastest).  Face
 *    field u^(c) holds at (i,j,k) the value at face index i (c = 1), j (c = 2)
 *    or k (c = 3) along its normal axis, at lo + index*h, and at cell-centre
 *    coordinates lo + (index + 1/2) h across it; face index 0 is the wall and
 *    is returned as 0.  The pressure field p holds cell centres.
 *  - Control points: the intersections of Gamma with the grid lines of u^(c)'s
 *    own grid (Sec. 3), ordered by component c, line axis, line, position.
 *    The "primary" points (line most normal to Gamma) carry the density
 *    unknowns and the BIE equations; density vectors are ordered like the
 *    primary points.
 *  - Devices: a context belongs to the CUDA device that was current at
 *    kfbim_setup.  Every call runs there, whichever device the calling thread
 *    has current, and gives the thread its device back; `stream` must belong
 *    to the context's device.
 *  - Threads: calls on different contexts may run at the same time from
 *    different host threads, on one device or several (each context owns its
 *    workspace; the kernel shared-memory limits the library raises are kept
 *    per device under a lock).  Calls on one context must not overlap.  The
 *    kernel_launches statistic counts the launches of the call's own thread.
 *  - CUDA graphs: iterative loops (the Schur CG) run as captured CUDA graphs,
 *    the CG as one graph with a device-side loop (a conditional node).  With
 *    the environment variable KFBIM_CUDA_GRAPHS=0 at kfbim_setup the kernels
 *    are launched one by one instead (same results; kernel profilers cannot
 *    profile kernels inside graphs with conditional nodes).
 *  - Return value: KFBIM_OK or a negative kfbim_status; kfbim_last_error()
 *    returns the message of the last failure on that context.  Invalid inputs
 *    are reported, never aborted on.  On KFBIM_E_NOCONV the outputs still hold
 *    the last iterate.
 */
#ifndef KFBIM_H
#define KFBIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kfbim_ctx kfbim_ctx;

typedef enum {
  KFBIM_OK = 0,
  KFBIM_E_INVALID = -1,   /* bad argument (null pointer, size, option) */
  KFBIM_E_GEOMETRY = -2,  /* interface not resolved by the grid */
  KFBIM_E_NOCONV = -3,    /* GMRES or CG iteration cap reached */
  KFBIM_E_NONFINITE = -4, /* NaN/Inf in an input or a residual */
  KFBIM_E_CUDA = -5,      /* CUDA runtime error */
  KFBIM_E_OOM = -6        /* device or host allocation failed */
} kfbim_status;

typedef enum {
  KFBIM_SPHERE = 0,
  KFBIM_ELLIPSOID = 1,
  KFBIM_STAR = 2,
  KFBIM_TORUS = 3,
  KFBIM_CALLBACK = 4
} kfbim_geometry_kind;

/* CALLBACK level set: F(x, user) returns F at x; derivs(x, g, H, user) writes
 * the gradient g[3] and the Hessian H[9] (row-major) at x. */
typedef double (*kfbim_level_fn)(const double x[3], void* user);
typedef void (*kfbim_level_derivs_fn)(const double x[3], double g[3], double H[9], void* user);

/* Analytic interface, Omega = {F <= 0}.
 *   SPHERE:    params[0] = radius.
 *   ELLIPSOID: params[0..2] = semi-axes; rot = row-major 3x3 rotation Q, the
 *              body frame is xi = Q^T (x - center).
 *   STAR:      r(theta, phi) = params[0] + params[1] sin(params[2] theta)
 *              cos(params[3] phi), theta polar angle from +z, phi azimuth.
 *   TORUS:     (params[1] - sqrt(x^2 + y^2))^2 + z^2 = params[0]^2 about the
 *              z axis through center: tube radius params[0] < axis distance
 *              params[1] (Example 5.3).
 *   CALLBACK:  any level set supplied by the caller through F and derivs (both
 *              non-null; center, rot and params are ignored).  They are called
 *              only from the thread running kfbim_setup / kfbim_setup_host,
 *              during that call, and must return finite values; the gradient
 *              must not vanish on Gamma (a control point where it does, or
 *              where it is not finite, gives E_GEOMETRY).  The tables are built
 *              once, so the device path never calls them. */
typedef struct {
  int kind;
  double center[3];
  double rot[9];
  double params[8];
  kfbim_level_fn F;              /* CALLBACK only, else ignored */
  kfbim_level_derivs_fn derivs;  /* CALLBACK only, else ignored */
  void* user;                    /* CALLBACK only: passed to F and derivs */
} kfbim_geometry;

typedef struct {
  int N;          /* cells per axis: a power of two with 16 <= N <= 256, or 96 */
  double lo, hi;  /* box [lo, hi]^3 */
} kfbim_grid;

typedef enum {
  KFBIM_FP64 = 0,       /* every step in FP64 */
  KFBIM_MIXED = 1,      /* FP32 transforms and Schur CG inside FP64 iterative
                           refinement of the corrected MAC system; jumps,
                           corrections, traces, residuals and GMRES stay FP64 */
  KFBIM_FP32 = 2,       /* the grid solve in FP32 only: one FP32 Schur CG (to
                           inner_tol) and FP32 transforms, no FP64 refinement;
                           jumps, corrections, traces and GMRES stay FP64.  The
                           matvec is accurate to about 1e-6 relative, so
                           gmres_tol should not be below about 1e-6.  A forward
                           mode for large grids (such as a 256^3 forward solve) */
  KFBIM_MIXED_TF32 = 3  /* MIXED with every FP32 transform on the tensor cores
                           (3xTF32 transform-matrix GEMMs, transforms = TENSOR);
                           N = 128 only, else E_INVALID */
} kfbim_precision;

typedef enum {
  KFBIM_STOKES = 0,  /* -mu Lap u + grad p = f, div u = 0 (Eq. SP) */
  KFBIM_NAVIER = 1   /* -mu Lap u - (lambda + mu) grad div u = f (Eq. Navier), solved
                        in the unified form -mu Lap u + grad p = f, div u + c p = 0,
                        c = 1/(lambda + mu), with the elastic interface traction */
} kfbim_pde;

typedef struct {
  double mu;          /* viscosity, or Lame mu (> 0) */
  int precision;      /* kfbim_precision */
  double gmres_tol;   /* relative l2 residual, e.g. 1e-10 */
  int gmres_max;      /* <= 200 */
  double cg_tol;      /* FP64 Schur CG relative residual, e.g. 1e-14 */
  int cg_max;
  double refine_tol;  /* MIXED: relative residual of the FP64 system; the
                         solution error it leaves grows like N^2 (condition
                         number of the MAC system).  With 1e-11, MIXED solves
                         agree with FP64 solves to about 6e-9 (density) at
                         N = 128 and 2.4e-8 at N = 256 */
  int refine_max;     /* MIXED: refinement sweeps cap */
  double inner_tol;   /* MIXED: FP32 CG relative residual per sweep */
  int pde;            /* kfbim_pde */
  double lambda;      /* Lame lambda (NAVIER; lambda + mu > 0, lambda >= 0) */
  int transforms;     /* kfbim_transforms: kernels of the FP32 (MIXED) axis passes */
  double relax;       /* MIXED: inexact GMRES.  The grid solve of the matvec taken
                         at GMRES relative residual r stops its refinement at
                         max(refine_tol, min(1e-4, relax * gmres_tol / r)): later
                         Krylov vectors enter the solution with coefficients of
                         size about r, so their matvecs may be that much less
                         accurate.  0 keeps refine_tol for every matvec.  Default
                         0.1 (at 128^3 about a third fewer FP32 correction solves,
                         density still within 1e-8 of the FP64 oracle) */
} kfbim_options;

/* Kernels of the FP32 transforms of MIXED contexts.
 * The Schur CG (Sec. 4.2, the dominant cost) runs, for N = 32, 64 and 128, as
 * four kernels per iteration: the transforms along z of the CG direction, one
 * CTA per (x, y) plane for the rest of the three spectral terms in shared
 * memory, the inverse transforms along z with the first dot product, and the
 * vector update (the "slab" iteration).  The other FP32 transforms (Schur
 * right-hand side, velocity recovery) run as one-axis passes: four-step FFT
 * passes on the CUDA cores, or, for N = 128, a dense 3xTF32
 * transform-matrix GEMM on the tensor cores (tcgen05).  FP64 passes are
 * always FFT passes. */
typedef enum {
  KFBIM_XF_AUTO = 0,    /* slab CG; one-axis passes timed at setup, the faster of the
                           FFT and tensor-core forms per stage kind */
  KFBIM_XF_FFT = 1,     /* slab CG; FFT one-axis passes */
  KFBIM_XF_TENSOR = 2,  /* tensor-core passes where N = 128, CG included (one-axis stages) */
  KFBIM_XF_STAGED = 3   /* FFT one-axis passes everywhere, CG included (five staged
                           launches per Schur apply, three CG vector kernels) */
} kfbim_transforms;

typedef struct {
  int gmres_iters;
  int interface_solves;
  int cg_iters;        /* total over all interface solves */
  int refine_sweeps;   /* total (MIXED) */
  double gmres_residual;
  int64_t kernel_launches; /* CUDA kernels launched by the call */
} kfbim_stats;

/* Fills *opt with the defaults (Stokes, mu 1, FP64, gmres 1e-10/200,
 * cg 1e-14/2000, refine 1e-11/8, inner 3e-6, lambda 0, transforms AUTO). */
void kfbim_default_options(kfbim_options* opt);

/* Alg. 1 step 1: grids, sides, intersections, frames, control points and all
 * jump / correction / interpolation tables; uploads them to the current CUDA
 * device.  Host work only, plus device allocations.  Errors: E_INVALID,
 * E_GEOMETRY (interface within 3h of the wall, double crossings, too few fit
 * neighbours), E_OOM, E_CUDA.  On error *ctx is NULL. */
int kfbim_setup(const kfbim_geometry* geom, const kfbim_grid* grid,
                const kfbim_options* opt, kfbim_ctx** ctx);

/* kfbim_setup with its device work (table uploads, workspace clears) ordered
 * on `stream` (a cudaStream_t of the current device) instead of the legacy
 * default stream, so that it does not serialise with other streams of the
 * caller; the call synchronises `stream` before returning (the host tables
 * are released afterwards).  Same arguments and errors as kfbim_setup. */
int kfbim_setup_async(const kfbim_geometry* geom, const kfbim_grid* grid,
                      const kfbim_options* opt, void* stream, kfbim_ctx** ctx);

/* Device memory for a context from the caller instead of cudaMalloc, e.g.
 * a framework's caching allocator that owns the device heap.  alloc returns
 * `bytes` of device memory on the current device (the context's), at least
 * 256-byte aligned (else setup fails with E_INVALID), or NULL when it cannot
 * (E_OOM); free gets back every block, with its size, from kfbim_destroy,
 * after the device has been synchronised.  Both are called on the thread of
 * the library call: alloc during setup and, for workspace allocated on first
 * use (kfbim_solve_batch, kfbim_solve_host), during that call.  Pinned host
 * buffers and streams still come from the CUDA runtime. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, size_t bytes, void* user);
  void* user;
} kfbim_allocator;

/* kfbim_setup_async with an optional allocator (NULL: cudaMalloc).  The
 * allocator struct is copied; its user pointer must stay valid until
 * kfbim_destroy. */
int kfbim_setup_ex(const kfbim_geometry* geom, const kfbim_grid* grid, const kfbim_options* opt,
                   void* stream, const kfbim_allocator* alloc, kfbim_ctx** ctx);

/* Host-only variant of kfbim_setup: builds the control points and every table
 * on the host and touches no GPU (for inspection and host-side tests).  The
 * returned context supports kfbim_sizes, kfbim_points, kfbim_sides,
 * kfbim_table_sizes and kfbim_destroy; solver calls on it return
 * KFBIM_E_INVALID. */
int kfbim_setup_host(const kfbim_geometry* geom, const kfbim_grid* grid,
                     const kfbim_options* opt, kfbim_ctx** ctx);

/* Releases every device and host resource of ctx (synchronises the device
 * when ctx owns device memory). */
int kfbim_destroy(kfbim_ctx* ctx);
const char* kfbim_last_error(const kfbim_ctx* ctx);

/* Sizes: all control points, primary points (density unknowns), N. */
int kfbim_sizes(const kfbim_ctx* ctx, int64_t* n_points, int64_t* n_primary, int* N);

/* Sizes of the sparse tables: surface-fit entries, correction rows (RHS
 * targets at irregular nodes) and correction entries; each nullable. */
int kfbim_table_sizes(const kfbim_ctx* ctx, int64_t* fit_nnz, int64_t* corr_rows,
                      int64_t* corr_nnz);

/* Control-point data (host, each nullable): xyz [n_points*3], comp (1..3),
 * axis (0..2), primary flag (0/1). */
int kfbim_points(const kfbim_ctx* ctx, double* xyz_host, int32_t* comp_host,
                 int32_t* axis_host, int32_t* primary_host);

/* The control points of component comp (1..3) that carry density unknowns
 * (Sec. 3: the intersections of Gamma with the grid lines of u^(comp)'s own
 * grid, the primary ones, Alg. 1 step 1), in the order of the comp-th block of
 * every density and boundary-data vector: g_dev of kfbim_solve is
 * [g^(1) at control_points(1) | g^(2) at control_points(2) | g^(3) at
 * control_points(3)].  *n receives the count; xyz_host [n*3] and normal_host
 * [n*3] (outward unit normals, Sec. 2) are filled when non-null (query the
 * count first with both null).  Host memory; works on host-only contexts. */
int kfbim_control_points(const kfbim_ctx* ctx, int comp, int64_t* n, double* xyz_host,
                         double* normal_host);

/* The points where the forcing f^+ is needed for the jump conditions (Sec. 4.3:
 * [[f]] enters the second-order jumps at every control point, primary or not):
 * all n_points control points in the canonical order of fpts_dev.  *n receives
 * n_points; xyz_host [n*3] is filled when non-null.  Host memory. */
int kfbim_jump_points(const kfbim_ctx* ctx, int64_t* n, double* xyz_host);

/* Outward unit normal grad F / |grad F| at every control point (Sec. 2),
 * normal_host [n_points*3] in the order of kfbim_points; host memory. */
int kfbim_normals(const kfbim_ctx* ctx, double* normal_host);

/* Side of every node of grid c (0 = cells, 1..3 = faces of u^(c)), 1 = Omega;
 * N^3 bytes in field layout. */
int kfbim_sides(const kfbim_ctx* ctx, int c, uint8_t* side_host);

/* One GMRES matvec (Prop. DBI): out = (1/2 I - M_v) phi at the primary points.
 * phi_dev, out_dev: n_primary doubles (may not alias). */
int kfbim_apply(kfbim_ctx* ctx, const double* phi_dev, double* out_dev, void* stream);

/* Full solve (Alg. 1 steps 2-3 and the final interior fields).
 *   g_dev      [n_primary]     Dirichlet data at the primary points.
 *   fpts_dev   [3*n_points]    f at every control point, component-blocked
 *                              (f^(1) for all points, then f^(2), f^(3));
 *                              nullable (then f = 0).
 *   fgrid_dev  [3*N^3]         f^(c) at the nodes of face grid c; nullable.
 *                              Values outside Omega are ignored (f~ = 0 there).
 *   phi_dev    [n_primary]     out: density.
 *   u_dev      [3*N^3]         out, nullable: interface-problem velocity; its
 *                              values at Omega nodes are u_h.
 *   p_dev      [N^3]           out, nullable: pressure (cells).  Stokes: gauge
 *                              mean(p) = mu * mean(g_cells) of the augmented
 *                              system with gamma = 1, alpha = mu N^3.  Navier:
 *                              p = -(lambda + mu) div u, no gauge.
 *   stats      nullable. */
int kfbim_solve(kfbim_ctx* ctx, const double* g_dev, const double* fpts_dev,
                const double* fgrid_dev, double* phi_dev, double* u_dev, double* p_dev,
                kfbim_stats* stats, void* stream);

/* kfbim_solve with host buffers: copies inputs to the device, solves and
 * copies phi (and u, p when non-null) back; same shapes as kfbim_solve. */
int kfbim_solve_host(kfbim_ctx* ctx, const double* g_host, const double* fpts_host,
                     const double* fgrid_host, double* phi_host, double* u_host,
                     double* p_host, kfbim_stats* stats, void* stream);

/* Adjoint (gradients with respect to the boundary data; not in the paper,
 * which solves forward problems only).  With A the GMRES matvec of
 * kfbim_apply and U the linear map from the density to the interface-solve
 * velocity (the u_dev of kfbim_solve), a solve computes u = U A^-1 (g - G_v f)
 * + (terms in f), so for a loss L(u) the gradient with respect to g is
 * dL/dg = A^-T U^T dL/du.
 * kfbim_apply_adjoint: out = A^T lam, lam_dev and out_dev n_primary doubles
 *   (may not alias): the transposed trace, transposed grid solve (the forward
 *   corrected MAC solve of (w, 0) with the pressure negated: K^T = S K S for
 *   S = diag(I, -I)), transposed corrections and transposed jump map.
 * kfbim_solve_adjoint: gbar = A^-T U^T ubar by GMRES on A^T (same tolerance
 *   and cap as kfbim_solve).  ubar_dev [3*N^3]: dL/du on the three face grids
 *   (wall-face entries ignored); gbar_dev [n_primary]: dL/dg at the primary
 *   points.  stats nullable.  Errors as kfbim_solve.  The transposed tables
 *   are built by kfbim_setup (device memory about a third of the forward
 *   tables). */
int kfbim_apply_adjoint(kfbim_ctx* ctx, const double* lam_dev, double* out_dev, void* stream);
int kfbim_solve_adjoint(kfbim_ctx* ctx, const double* ubar_dev, double* gbar_dev,
                        kfbim_stats* stats, void* stream);

/* Largest batch accepted by kfbim_solve_batch. */
#define KFBIM_BATCH_MAX 64

/* B independent solves (Alg. 1 steps 2-3) on the geometry and grid of ctx,
 * for B sets of boundary data and forcing.  The paper solves one problem at
 * a time; this is the many-right-hand-side form of the same solve.  Every
 * array holds the B instances back to back, each with the shape kfbim_solve
 * gives it: g_dev [B*n_primary], fpts_dev [B*3*n_points] (nullable),
 * fgrid_dev [B*3*N^3] (nullable), phi_dev [B*n_primary], u_dev [B*3*N^3]
 * (nullable), p_dev [B*N^3] (nullable), stats [B] (nullable; kernel_launches
 * is the count of the whole call).  Instance b's result equals that of
 * kfbim_solve on instance b up to rounding order (the same GMRES, refinement
 * and CG iteration per instance).
 * MIXED contexts run the instances in lockstep: every FFT stage is one launch
 * for all instances still iterating, each Schur CG of the batch (N = 32, 64,
 * 128) is one launch of a CUDA graph whose conditional while loop runs the
 * three slab kernels of every instance until all are done, and GMRES reads
 * its host scalars once per iteration for the whole batch.  FP64 contexts solve the instances one
 * after another.  The first call with a larger B than before allocates the
 * per-instance workspace (about 20 N^3 doubles-worth plus the Krylov basis of
 * gmres_max + 1 vectors per instance); it is kept until kfbim_destroy.
 * Errors: KFBIM_E_INVALID for B outside 1..KFBIM_BATCH_MAX or a null g/phi;
 * KFBIM_E_NONFINITE if any instance meets NaN/Inf; KFBIM_E_NOCONV if any
 * instance hit the GMRES cap (its stats entry says which). */
int kfbim_solve_batch(kfbim_ctx* ctx, int B, const double* g_dev, const double* fpts_dev,
                      const double* fgrid_dev, double* phi_dev, double* u_dev, double* p_dev,
                      kfbim_stats* stats, void* stream);

/* Per-kernel timing of the FFT transform passes (the dominant kernels).
 * enable = 1 starts (and zeroes) the counters, 0 stops them, -1 reads them:
 * total device milliseconds between CUDA events recorded around each launch,
 * the number of launches and the algorithmic bytes they move (N^3 values read
 * and written per pass, read-modify-write when accumulating), split into the
 * FP64 and the FP32 passes.  Output pointers are host memory, nullable.
 * Reading synchronises the device. */
int kfbim_profile(kfbim_ctx* ctx, int enable, double* ms64, int64_t* launches64,
                  double* bytes64, double* ms32, int64_t* launches32, double* bytes32);

/* Kernel classes of kfbim_profile_kernels. */
typedef enum {
  KFBIM_KCLASS_TRANSFORM_FP64 = 0,  /* one-axis transform passes, FP64 */
  KFBIM_KCLASS_TRANSFORM_FP32 = 1,  /* one-axis transform passes, FP32 (FFT or tensor core) */
  KFBIM_KCLASS_CG_ZFWD = 2,         /* slab CG: the previous iteration's x, r update, d = r + beta d,
                                       z transforms (9 N^3 floats) */
  KFBIM_KCLASS_CG_XY = 3,           /* slab CG: xy planes of the three terms (4 N^3 floats) */
  KFBIM_KCLASS_CG_ZINV = 4,         /* slab CG: inverse z transforms, d.q, r.r, r.q, q.q (5 N^3 floats) */
  KFBIM_KCLASS_CG_UPDATE = 5,       /* slab CG: the x update still pending when a run stops
                                       (3 N^3 floats, once per CG run) */
  KFBIM_KCLASS_CG_VECTOR = 6,       /* staged CG: the three vector kernels (14 N^3 values) */
  KFBIM_KCLASS_MAC_RESIDUAL = 7,    /* MIXED refinement: FP64 MAC residual (12 N^3 doubles) */
  KFBIM_KCLASS_JUMPS = 8,           /* jump evaluation (fit rows, jump maps, jumps) */
  KFBIM_KCLASS_COUNT = 9
} kfbim_kernel_class;

/* Per-class totals of the timing started by kfbim_profile(ctx, 1, ...):
 * for k < n, ms[k] device milliseconds between CUDA events recorded on the
 * call's stream around each launch group of class k, launches[k] kernels and
 * bytes[k] algorithmic bytes (the values the class's kernels must read and
 * write, counted once).  Classes >= KFBIM_KCLASS_COUNT read 0.  Output arrays
 * are host memory, nullable.  While timing is on, the Schur CG runs without
 * CUDA graphs.  Synchronises the device. */
int kfbim_profile_kernels(kfbim_ctx* ctx, int n, double* ms, int64_t* launches, double* bytes);

/* Stage entry points (same kernels as the solve path, exposed for parity tests).
 * kfbim_jumps: jump values at every control point (Sec. 4.3), layout
 *   J_dev[12 * n_points] slot-major: slot s of point y at s*n_points + y with
 *   slots [u^(c)], [grad u^(c)] (3), [Hess u^(c)] (11,22,33,23,13,12),
 *   [p], [d_a p] (a = the point's line axis). fpts_dev nullable.
 * kfbim_interface: the unified interface solve IUS-1..5 on the grid for
 *   density phi and forcing (fpts, fgrid nullable); writes u (3 N^3), p (N^3).
 * kfbim_trace: u^+ at the primary points from face fields u and jumps J. */
int kfbim_jumps(kfbim_ctx* ctx, const double* phi_dev, const double* fpts_dev,
                double* J_dev, void* stream);
int kfbim_interface(kfbim_ctx* ctx, const double* phi_dev, const double* fpts_dev,
                    const double* fgrid_dev, double* u_dev, double* p_dev, void* stream);
int kfbim_trace(kfbim_ctx* ctx, const double* u_dev, const double* J_dev,
                double* out_dev, void* stream);

/* Boundary pressure p^+ at every control point (Sec. 4.4, last paragraph:
 * the stress needs no derivative of p, so a linear rule suffices), e.g. for
 * the traction -p n + mu (grad u + grad u^T) n on Gamma.  Trilinear
 * interpolation over the eight cell centres around the point; cells in
 * Omega^c contribute p + [p], the jump of slot 10 of J at the point.
 *   p_dev [N^3] cell pressure (u_dev/p_dev of kfbim_solve or kfbim_interface);
 *   J_dev [12*n_points] the jumps of the same density (kfbim_jumps);
 *   out_dev [n_points], canonical point order.  First-order accurate next to
 *   the interface (zeroth-order jump correction). */
int kfbim_pressure_trace(kfbim_ctx* ctx, const double* p_dev, const double* J_dev,
                         double* out_dev, void* stream);

/* One FP32 axis pass (test entry point of the transform kernels): out = W . T in
 * along axis (0 x, 1 y, 2 z) of an N^3 field, T = transform `type` (1 DCT-II,
 * 2 its inverse, 3 DST-II, 4 its inverse, 5 DST-I, 6 its inverse; conventions
 * in transforms.cuh), W the spectral weight `wmode` (0 none, 1 Schur, 2 Poisson,
 * 3 Schur RHS; component wc = 0..2) or 1.  backend: KFBIM_XF_FFT or
 * KFBIM_XF_TENSOR (E_INVALID unless N = 128 and MIXED).  in_dev, out_dev: N^3
 * floats (may alias). */
int kfbim_transform_f32(kfbim_ctx* ctx, int type, int axis, int wmode, int wc,
                        const float* in_dev, float* out_dev, int backend, void* stream);

/* The kernel each kind of FP32 stage runs on (0 FFT, 1 tensor core) for a
 * plain stage (one transform per job) and a fused stage (transform, weight,
 * transform), and the autotuner's timings in ms per three-job stage: plain
 * FFT, plain tensor core, fused FFT, fused tensor core (zeros when the
 * autotuner did not run).  Host pointers, nullable. */
int kfbim_transforms_info(const kfbim_ctx* ctx, int* plain, int* fused, float* tune_ms4);

/* FFT Poisson solve -Delta_h u = r on face grid c (1..3) with the box
 * conditions of Sec. 4.2 (DST-I across the normal axis, DST-II along the
 * others): r_dev, u_dev N^3 doubles (wall face ignored / written 0). */
int kfbim_poisson(kfbim_ctx* ctx, int c, const double* r_dev, double* u_dev, void* stream);

/* Schur operator of item ii): q = (1/mu) G^T (-Delta_h)^{-1} G d + sum(d)/alpha,
 * alpha = mu N^3 (Stokes), or + c d (Navier); d_dev, q_dev N^3 doubles (cells). */
int kfbim_schur_apply(kfbim_ctx* ctx, const double* d_dev, double* q_dev, void* stream);

/* The FP32 Schur operator of the slab CG iteration (test entry point of its
 * kernels; MIXED contexts with N = 32, 64 or 128 and transforms AUTO or FFT,
 * else E_INVALID): q = (1/mu) sum_c G_c^T (-Delta_c)^{-1} G_c d (+ c d for
 * Navier), without the rank-one term of kfbim_schur_apply; d_dev, q_dev N^3
 * floats (cells, must not alias).  Synchronises the stream. */
int kfbim_schur_apply_f32(kfbim_ctx* ctx, const float* d_dev, float* q_dev, void* stream);

/* Allocation-free variant of kfbim_poisson, for callers that may not allocate
 * device memory: code that runs under a memory manager owning the whole device
 * heap (a caching allocator that reserved HBM up front, or a host application
 * that hands its plug-ins only buffers it allocated itself), and loops where
 * cudaMalloc's implicit device synchronisation is not acceptable.  The paper has
 * no counterpart: it is a deployment convenience around the FFT Poisson solve.
 *
 * Solves -Delta_h u = r on face grid c (1..3) of an N^3 grid on [lo, hi]^3,
 * N a power of two with 16 <= N <= 64; r_dev and u_dev are caller-owned N^3
 * doubles in the layout of kfbim_poisson (must not alias).  No context, no
 * cudaMalloc/cudaFree and no allocating library routine: the scratch (two N^3
 * fields) and the transform tables live in file-scope static device arrays of
 * 4 MiB + 2 KiB, which every GPU that loads the library holds until exit.
 * Outside a stream capture every call looks up the arrays' device addresses
 * (cudaGetSymbolAddress, no allocation); under capture the addresses of the
 * last call on that device are used, so make a first call on each device
 * before any stream capture (a first call under capture returns
 * KFBIM_E_INVALID).
 * All calls share the arrays: calls that overlap on the GPU (different
 * streams, or several host threads on one device) race and corrupt each
 * other's results; calls on one stream are ordered and each call rewrites the
 * whole scratch and tables before reading them, so nothing from a previous
 * call leaks into the next.
 * Errors: KFBIM_E_INVALID for a bad argument or N > 64 (a message names the
 * limit on stderr), KFBIM_E_CUDA if the symbols cannot be resolved or one of
 * this call's launches fails (an error left pending by earlier, unrelated work
 * is neither reported nor cleared). */
int kfbim_poisson_noalloc(int c, int N, double lo, double hi, const double* r_dev,
                          double* u_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KFBIM_H */
