/*
 * gd.h -- C ABI of the GB300 gradient-domain multigrid solver (libgd.so).
 *
 * Method: Kazhdan et al., "Gradient-Domain Processing for Large EM Image
 * Stacks".  Two gradient-domain steps on a registered image stack:
 *
 *   anisotropic diffusion along z (Sec. 3.1, Eq. anisotropic_diffusion):
 *       (bx Kx + by Ky + bz Kz) I1 = (bx Kx + by Ky) I0
 *   screened Poisson per slice (Sec. 3.1, Eq. screened_poisson):
 *       (alpha + Kx + Ky) I2 = alpha I1 + (Kx + Ky) I0
 *
 * both instances of the general screened anisotropic system of Sec. 4,
 *       (alpha - div W grad) I = alpha I0 - div W G,
 * discretised by default with the 6-point "Constant" stencil of Sec. 4.2:
 * face-adjacent neighbours have coefficient -1 and, with homogeneous Neumann
 * boundaries, the diagonal is the number of existing neighbours, i.e. along
 * one axis K_n = tridiag(-1, [1, 2, ..., 2, 1], -1).  Unit voxel spacing on all
 * axes.  The singular AD system (alpha = 0) is solved with mean(I1) =
 * mean(I0).  The Hybrid and Linear discretisations of Sec. 4.2 are chosen at
 * gd_stack_create; batches of independent slices of different sizes have
 * their own handle (gd_batch_*, below).
 *
 * Solver: V-cycle multigrid (Sec. 4.1) with red-black Gauss-Seidel
 * relaxation, residual + down-sampling by summing children, up-sampling by
 * replication (Constant transfers, Sec. 4.2) and a direct (fast
 * diagonalisation) solve at the coarsest level; FP32 kernels with the
 * fine-level iterate kept as an unevaluated float pair and its residual
 * re-evaluated every cycle (iterative refinement), so the relative residual can
 * go below what an FP32 array can represent.
 *
 * ----------------------------------------------------------------------------
 * Conventions for every entry point
 *
 * Arrays: float32, contiguous, [nz][ny][nx] with x fastest (element
 *   (i,j,k) at ((k*ny + j)*nx + i)), nx*ny*nz elements.  Pointers may be
 *   device pointers (cudaMalloc / torch CUDA tensors) or host pointers
 *   (pinned or pageable); host arrays are copied to internal device buffers
 *   on the stack's stream and results copied back before the call returns.
 *   The caller owns every array it passes; the library never frees them.
 * Streams: all work is enqueued on the stream given to gd_stack_create.
 *   Calls return after the result is complete (they read the residual norm
 *   back every cycle).
 * Status: every function returns a gd_status; a gd_report passed in gets
 *   the same value in .status.  On GD_ERR_NOT_CONVERGED the output holds the
 *   last iterate.  On GD_ERR_INVALID_ARG / GD_ERR_UNSUPPORTED nothing is
 *   written.  GD_ERR_CUDA means a CUDA call failed; gd_last_error() says
 *   which.
 * Threads: one stack must not be used from two threads at once; distinct
 *   stacks are independent.
 */
#ifndef GD_H
#define GD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gd_stack gd_stack; /* opaque: sizes, stream, MG hierarchy and workspace */

typedef enum {
  GD_OK = 0,
  GD_ERR_INVALID_ARG = 1,  /* null pointer, bad size, negative / NaN weight, ... */
  GD_ERR_UNSUPPORTED = 2,  /* valid but not implemented (boundary, discretisation, precision) */
  GD_ERR_OOM = 3,          /* device or host allocation failed */
  GD_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  GD_ERR_NOT_CONVERGED = 5,/* max_cycles reached, or residual stalled, above rel_tol */
  GD_ERR_DIVERGED = 6,     /* residual became non-finite or grew by > 1e3 */
  GD_ERR_TIMEOUT = 7       /* a kernel gave up a bounded wait for its own asynchronous copies */
} gd_status;

enum { GD_BC_NEUMANN = 0 };                                     /* reading of Sec. 3-4: natural BC */
enum { GD_DISC_CONSTANT = 0, GD_DISC_HYBRID = 1, GD_DISC_LINEAR = 2 }; /* Sec. 4.2 */
enum { GD_PREC_FP32 = 0, GD_PREC_MIXED = 1 };
enum { GD_SYSTEM_AD = 0, GD_SYSTEM_SP = 1 };

/* Weights of the general system of Sec. 4: alpha = screening weight, W =
 * Diag(beta_x, beta_y, beta_z) (Sec. 3.1: all >= 0). */
typedef struct {
  double alpha, beta_x, beta_y, beta_z;
} gd_weights;

/* Solve control.  A V(nu1,nu2) cycle is repeated until the relative residual
 * ||b - A x||_2 / ||b||_2 (Table 1 caption: residual over the initial
 * constraints, b being the full right-hand side) is <= rel_tol or
 * max_cycles cycles have run.  coarsest_xy: x and y are not coarsened below
 * this many cells (the coarsest level then has coarsest_xy..2*coarsest_xy-1
 * cells along them); 0 means 16. */
typedef struct {
  int max_cycles;
  double rel_tol;
  int nu1, nu2;
  int coarsest_xy;
  int flags; /* GD_FLAG_* */
} gd_solve_ctl;

/* also evaluate the relative residual of the float32 output as stored
 * (one extra pass); reported in gd_report.rel_residual_out */
#define GD_FLAG_REPORT_OUTPUT_RESIDUAL 1

#define GD_HISTORY 64
typedef struct {
  int status;
  int cycles;               /* V-cycles run */
  int levels;               /* multigrid levels in the hierarchy used */
  double rel_residual;      /* ||b - A x|| / ||b|| of the solver's iterate (float pair) */
  double rel_residual_out;  /* same for the float32 output as stored (NaN unless flagged) */
  double rho_per_cycle;     /* geometric-mean residual reduction per cycle */
  double rhs_norm;          /* ||b||_2 */
  double history[GD_HISTORY]; /* relative residual before cycle 1 and after cycle c (c < 64) */
} gd_report;

/*
 * gd_stack_create -- sizes and stream of one stack; allocates nothing on the
 * device yet (the hierarchy is built on the first solve and reused while the
 * weights keep the same coarsening plan).
 *   nx, ny >= 2, nz >= 1:  stack size (voxels) -- Sec. 3.1, slices along z
 *   bc:   GD_BC_NEUMANN only (others: GD_ERR_UNSUPPORTED)
 *   disc: the discretisation of Sec. 4.2:
 *         GD_DISC_CONSTANT -- 6-point operator, piecewise-constant transfers,
 *           re-discretised 6-point coarse operators (the fast path);
 *         GD_DISC_HYBRID -- the same 6-point fine operator (same answers),
 *           first-order B-spline transfers (1/2, 1, 1/2) and Galerkin
 *           27-point coarse operators, eight-colour Gauss-Seidel on them;
 *         GD_DISC_LINEAR -- trilinear finite elements: the fine operator is
 *           27-point (1D stiffness K_n and P1 mass (1/6) tridiag(1, [2, 4,
 *           ..., 4, 2], 1) per axis; an axis of one node, and z for the
 *           per-slice step, keep mass 1), the right-hand sides are the same
 *           operators applied to I0 and I1, the residual of the float-pair
 *           iterate is evaluated in compensated float arithmetic (exact
 *           integer-scaled factors, TwoSum); B-spline transfers, Galerkin
 *           levels.  gd_vcycle, gd_residual and gd_smooth evaluate the
 *           6-point operator and return GD_ERR_UNSUPPORTED on such a stack.
 *         Hybrid and Linear need prec = GD_PREC_FP32 (else GD_ERR_UNSUPPORTED).
 *   prec: GD_PREC_FP32, or GD_PREC_MIXED: the correction solves of
 *         gd_diffuse_z / gd_screened_poisson_slices store every multigrid level
 *         between the fine and the coarsest (corrections, constraints, sweep
 *         arrays) as bfloat16 with float32 arithmetic -- the paper's 16-bit
 *         storage of intermediate solutions and constraints (Sec. 4.1, "Disk
 *         I/O").  The fine level, the coarsest solve, the iterate, the outer
 *         residual and the output stay float32 (float pair), so the tolerance
 *         is reached the same way.  A hierarchy with a level whose x extent is
 *         not a multiple of 8 (or with fewer than three levels) keeps float32
 *         throughout.  gd_vcycle, gd_residual and gd_smooth always use
 *         float32.
 *   cuda_stream: a cudaStream_t, or NULL for the legacy default stream
 * If the environment variable GD_DISABLE_TMA is set (and not "0") when the
 * stack is created, the stack runs only the plain kernels (no TMA pipeline,
 * no fused transfers); results are the same up to rounding.  The V-cycle of a
 * solve is captured once as a CUDA graph and replayed (on the stack's
 * stream); GD_DISABLE_GRAPHS set at creation launches every kernel directly
 * instead (identical results).
 */
int gd_stack_create(gd_stack **out, int nx, int ny, int nz, int bc, int disc, int prec,
                    void *cuda_stream);

/*
 * gd_diffuse_z -- anisotropic diffusion, Sec. 3.1 Eq. (anisotropic_diffusion):
 * solves (bx Kx + by Ky + bz Kz) I1 = (bx Kx + by Ky) I0 with mean(I1) =
 * mean(I0).  w.alpha is ignored (AD has no screening term); needs
 * beta_x, beta_y >= 0, beta_z > 0.
 *   I0 (in), I1 (out): stack arrays; I1 must not alias I0.
 *   x0 (in, nullable): initial guess (default zero: from I0 the residual
 *     is the removed inter-slice variation, several times the right-hand
 *     side on EM stacks); may alias I1.
 */
int gd_diffuse_z(gd_stack *s, const float *I0, float *I1, gd_weights w, const gd_solve_ctl *ctl,
                 const float *x0, gd_report *rep);

/*
 * gd_screened_poisson_slices -- screened Poisson per slice, Sec. 3.1
 * Eq. (screened_poisson): (alpha + Kx + Ky) I2 = alpha I1 + (Kx + Ky) I0 on
 * every slice; the slices are independent systems solved together.
 *   I0, I1 (in), I2 (out): stack arrays; I2 must alias neither input.
 *   alpha > 0: screening weight (the paper uses 0.01).
 *   x0 (in, nullable): initial guess (default I0, whose residual is
 *     alpha (I1 - I0): small against the right-hand side when the screening
 *     weight is small); may alias I2.
 */
int gd_screened_poisson_slices(gd_stack *s, const float *I0, const float *I1, float *I2,
                               double alpha, const gd_solve_ctl *ctl, const float *x0,
                               gd_report *rep);

/*
 * gd_screened_poisson -- the general system of Sec. 4 with an explicit
 * right-hand side: (alpha + bx Kx + by Ky + bz Kz) x = b, solved like the two
 * steps above (float-pair refinement over float32 V(nu1,nu2)-cycles) to
 * ||b - A x|| <= rel_tol ||b||.  Needs alpha > 0 (the system is then
 * nonsingular) and beta_* >= 0; beta_z == 0 makes the slices independent.
 *   b (in), x (out): stack arrays; x must not alias b.
 *   x0 (in, nullable): initial guess (default zero); may alias x.
 */
int gd_screened_poisson(gd_stack *s, gd_weights w, const float *b, float *x, const gd_solve_ctl *ctl,
                        const float *x0, gd_report *rep);

/*
 * gd_ad_then_sp -- the paper's two steps in one call (Sec. 3.1: AD, then SP
 * on the result): gd_diffuse_z(I0 -> I1) followed by
 * gd_screened_poisson_slices(I0, I1 -> I2), with I0 copied to the device once
 * (when it is a host array) and I1 kept on the device.
 *   I0 (in), I2 (out): stack arrays (device or host), distinct;
 *   w_ad: the AD weights (as gd_diffuse_z); alpha > 0: the SP weight;
 *   ctl_ad, ctl_sp (nullable): the two solves' controls;
 *   I1 (out, nullable): receives the AD result when given (device arrays
 *     are used in place of the stack's buffer);
 *   rep_ad, rep_sp (nullable): the two reports.
 * Returns the first error, else GD_ERR_NOT_CONVERGED if either solve
 * stopped short of its tolerance, else GD_OK.
 */
int gd_ad_then_sp(gd_stack *s, const float *I0, float *I2, gd_weights w_ad, double alpha,
                  const gd_solve_ctl *ctl_ad, const gd_solve_ctl *ctl_sp, float *I1, gd_report *rep_ad,
                  gd_report *rep_sp);

/*
 * gd_npr_rhs -- right-hand side of the NPR gradient filter of Sec. 7 (after
 * Bhat et al. 2010, Sec. 6.2): b = alpha I0 - div(W V) with the target
 * gradients V = lambda (1 - exp(-|grad I0|^2 / (2 sigma^2))) grad I0, for
 * gd_screened_poisson with the same weights (the paper's video example:
 * alpha = 0.001, W = Diag(1, 1, 0.1), lambda = 1.25, sigma = 5).
 * Gradients are forward differences on voxel faces, none leaving the
 * domain; the face p -> p + e_d is modulated by the norm of the
 * forward-difference vector at its lower voxel p.
 *   I0 (in), b (out): stack arrays (device or host), b must not alias I0.
 *   w: alpha and the gradient weights W; sigma > 0.
 */
int gd_npr_rhs(gd_stack *s, const float *I0, float *b, gd_weights w, double lambda, double sigma);

/*
 * gd_vcycle -- ncycles plain float32 V-cycles (Sec. 4.1) on A x = b with an
 * explicit right-hand side, A = alpha + bx Kx + by Ky + bz Kz (Sec. 4 general
 * form).  system: GD_SYSTEM_AD (3D coupling, needs bz > 0) or GD_SYSTEM_SP
 * (independent slices, needs bz == 0 and alpha > 0).  x is updated in place
 * (initial guess in, iterate out); no refinement, no mean fix.  The report
 * gives the relative residual before and after (history[0], history[1]).
 */
int gd_vcycle(gd_stack *s, int system, gd_weights w, const float *b, float *x, int ncycles,
              gd_report *rep);

/* gd_destroy -- frees the stack and its device memory (NULL is a no-op). */
int gd_destroy(gd_stack *s);

/*
 * gd_residual -- relative residual ||b - A x|| / ||b|| (FP64 accumulation) of a
 * float32 x for the AD system (I1 ignored; w.alpha ignored) or the SP system
 * (w.alpha > 0 used, W fixed to Diag(1,1,0)), with b assembled from I0 (and
 * I1) as in Sec. 3.1.  Writes *rel (host double).
 */
int gd_residual(gd_stack *s, int system, gd_weights w, const float *I0, const float *I1,
                const float *x, double *rel);

/*
 * gd_smooth -- nsweeps red-black Gauss-Seidel sweeps (Sec. 4.1 multi-colour
 * relaxation: red = (i+j+k) even first, then black) of the fine-level system
 * A x = b, A = alpha + bx Kx + by Ky + bz Kz, x updated in place.
 */
int gd_smooth(gd_stack *s, gd_weights w, const float *b, float *x, int nsweeps);

/* Per-kernel event timing, for measurement.  When enabled, the stack records
 * a CUDA event pair around each launch of its kernels (on its stream).
 * gd_profile_query(s, k, name, len, &launches, &ms, &bytes) returns kernel
 * class k's totals since the last reset (GD_ERR_INVALID_ARG past the last
 * class); bytes is the algorithmic bytes moved by those launches. */
int gd_profile_enable(gd_stack *s, int on);
int gd_profile_reset(gd_stack *s);
int gd_profile_query(gd_stack *s, int k, char *name, int name_len, long long *launches,
                     double *ms, double *bytes);

/*
 * gd_smooth_noalloc -- the red-black relaxation of gd_smooth for callers that
 * must not allocate device memory: plug-ins whose host application owns the
 * whole device pool, and latency-bound loops that cannot afford the implicit
 * synchronisation of cudaMalloc / cudaFree.  gd_smooth allocates the second
 * array of its out-of-place sweep on every call; this entry point uses a
 * fixed scratch array compiled into the library instead (every GPU that
 * loads the library holds its GD_NOALLOC_MAX_VOXELS floats, 16 MB, until the
 * process exits).  The paper has no counterpart: it is an interface for such
 * callers, not a step of the method.
 *   nx, ny >= 2, nz >= 1, nx*ny*nz <= GD_NOALLOC_MAX_VOXELS (else
 *     GD_ERR_INVALID_ARG, nothing launched);
 *   w: weights of A = alpha + bx Kx + by Ky + bz Kz (as gd_smooth);
 *   b (in), x (in/out): device arrays of the current device only (host
 *     arrays would need staging buffers, i.e. allocations; another GPU's
 *     arrays are not addressable from this one's kernels): GD_ERR_INVALID_ARG;
 *     b and x must not overlap (GD_ERR_INVALID_ARG);
 *   cuda_stream: a cudaStream_t or NULL; returns after the sweeps complete.
 * It allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current.  The address is kept for
 * the life of the process, so it assumes the device's context is not reset in
 * between.  All calls on a device share the one scratch
 * array, which keeps the last call's contents (each call overwrites what it
 * reads): calls that overlap on the GPU (other streams, other threads) race.
 */
#define GD_NOALLOC_MAX_VOXELS (4 * 1024 * 1024)
int gd_smooth_noalloc(int nx, int ny, int nz, gd_weights w, const float *b, float *x, int nsweeps,
                      void *cuda_stream);

/*
 * ---- Batched screened Poisson on slices of different sizes ----
 *
 * The screened Poisson step of Sec. 3.1 (Eq. screened_poisson), solved on
 * independent 2D slices: slice s (nx_s x ny_s cells, weight alpha_s > 0)
 * solves (alpha_s + Kx + Ky) I2 = alpha_s I1 + (Kx + Ky) I0 with the 6-point
 * "Constant" stencil of Sec. 4.2 (Neumann boundary).  The slices decouple
 * (the step has no z term), so one multigrid V-cycle (Sec. 4.1) runs over
 * all of them at once: each slice has its own 2D hierarchy (the stack
 * solver's coarsening rule), every kernel is one launch over the tiles of
 * all slices at a depth, each slice's coarsest level is solved exactly, and
 * the cycle is replayed from a CUDA graph.
 *
 * Array layout: one packed float32 array per quantity; slice s occupies
 * elements [off_s, off_s + nx_s ny_s), x fastest, off_s = sum over t < s of
 * nx_t ny_t (gd_batch_offset).  Device pointers are used in place; host
 * pointers are staged through buffers the batch allocates on first use.
 */
typedef struct gd_batch gd_batch;

/*
 * gd_batch_create -- plans the hierarchies and allocates the packed levels.
 *   nslices >= 1; nx[s], ny[s] in [1, 2^20]; alpha[s] finite and > 0 (the
 *     arrays are copied);
 *   coarsest_xy: an axis is not halved below this many cells (0 means 16);
 *   stream: a cudaStream_t (NULL: the legacy default stream).
 * GD_ERR_UNSUPPORTED if a slice's coarsest level would hold more than 4096
 * cells (aspect ratios above about 256:1); GD_ERR_OOM on allocation failure.
 * On failure *out is NULL and gd_batch_last_error(NULL) holds the reason.
 */
int gd_batch_create(gd_batch **out, int nslices, const int *nx, const int *ny, const double *alpha,
                    int coarsest_xy, void *stream);

/*
 * gd_batch_screened_poisson -- V(nu1, nu2) cycles until every slice's
 * relative residual ||b_s - A_s x_s|| / ||b_s|| is <= ctl->rel_tol, or
 * ctl->max_cycles cycles.  The iterate is float32 (its rounding bounds the
 * attainable relative residual near 1e-6); nu1 + nu2 must be even;
 * ctl->coarsest_xy must be 0 or the batch's.
 *   I0, I1 (in), I2 (out): packed arrays of gd_batch_voxels() floats;
 *   x0 (in, nullable): initial guess (default I0);
 *   rep (out, nullable): status, cycles, levels (deepest hierarchy),
 *     rel_residual (max over slices), rhs_norm (over all slices), history
 *     (max relative residual before cycle 1 and after each cycle);
 *   slice_rel (out, nullable): [nslices] final relative residual per slice.
 * Returns GD_ERR_NOT_CONVERGED (I2 still written) when the tolerance is not
 * met, GD_ERR_DIVERGED when a residual is not finite.
 */
int gd_batch_screened_poisson(gd_batch *b, const float *I0, const float *I1, float *I2,
                              const gd_solve_ctl *ctl, const float *x0, gd_report *rep,
                              double *slice_rel);

/*
 * gd_batch_tune -- picks the rows per work item of the batch's kernels (32,
 * 64, 128 or 256; 64 until tuned) by timing two V(2,2) cycles with each, and
 * keeps the fastest.  Overwrites the batch's internal buffers only; call it
 * between solves.  chunk_out (nullable) receives the choice.
 */
int gd_batch_tune(gd_batch *b, int *chunk_out);

long long gd_batch_voxels(const gd_batch *b);            /* total cells, -1 for NULL */
long long gd_batch_offset(const gd_batch *b, int slice); /* off_s, -1 if out of range */
int gd_batch_levels(const gd_batch *b);                  /* depth of the deepest hierarchy */
/* Algorithmic device-memory bytes of one V(nu1, nu2) cycle with its outer
 * pass, and of the once-per-solve passes (input, first outer pass, output):
 * each pass's arrays read and written once. */
int gd_batch_traffic(const gd_batch *b, int nu1, int nu2, double *per_cycle, double *per_solve);
/* Algorithmic bytes of the last gd_batch_screened_poisson: the once-per-solve
 * passes plus each cycle over the slices still iterating in it (-1 for NULL). */
double gd_batch_last_traffic(const gd_batch *b);
long long gd_batch_launch_count(const gd_batch *b);      /* kernel launches since creation */
const char *gd_batch_last_error(const gd_batch *b);
int gd_batch_destroy(gd_batch *b);

/*
 * gd_selftest_wait -- failure-detection self-test: one CTA waits on an
 * mbarrier that nothing arrives at, with the same bounded try_wait (500 ns
 * suspend hint per poll) the TMA kernels use, for `polls` polls (1 ..
 * 2^24).  Returns GD_ERR_TIMEOUT when the wait gave up (the expected
 * outcome; the kernel returns normally and the context stays usable),
 * GD_OK if it completed, GD_ERR_CUDA on a launch error.  Runs on the legacy
 * default stream of the current device.
 */
int gd_selftest_wait(unsigned polls);

/* Fault injection for tests (host side): with the environment variable
 * GD_FAIL_ALLOC_AFTER=N set when a stack is created, that stack's
 * allocations after the first N fail with GD_ERR_OOM. */

/* Number of kernel launches the stack has enqueued since creation. */
long long gd_launch_count(gd_stack *s);

/*
 * Level inspection (the Constant discretisation), for measuring what the
 * mixed-precision mode's 16-bit storage does to each level (Sec. 4.1 "Disk
 * I/O" stores intermediate levels in 16 bits).  They describe the hierarchy
 * of the stack's last solve or gd_vcycle call.
 *   gd_level_count: levels (0 before any solve).
 *   gd_level_info: info[10] = {nx, ny, nz, sx, sy, sz, lx, ly, lz, bytes per
 *     value (4 float32, 2 bfloat16)} -- the level's size and, per axis, the
 *     children counts of its cells (s, and l for the last one) -- and
 *     weights[4] = {wx, wy, wz, wm}: the level's operator is
 *     wx Kx(x)My(x)Mz + wy Mx(x)Ky(x)Mz + wz Mx(x)My(x)Kz + wm Mx(x)My(x)Mz with
 *     K the 1D Neumann Laplacian and M_d = diag(children counts).
 *   gd_level_fetch: copies level `level` (>= 1; level 0 is the caller's
 *     array) -- which = 0: its correction x after the last cycle's
 *     post-smoothing, 1: its right-hand side b -- into dst (nx*ny*nz floats,
 *     device or host), widening bfloat16 to float32; synchronises the stream.
 * GD_ERR_UNSUPPORTED for the Hybrid and Linear discretisations.
 */
int gd_level_count(gd_stack *s);
int gd_level_info(gd_stack *s, int level, int *info, double *weights);
int gd_level_fetch(gd_stack *s, int level, int which, float *dst);

const char *gd_status_string(int status);
const char *gd_last_error(gd_stack *s);
int gd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GD_H */
