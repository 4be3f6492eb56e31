/*
 * parametrix.h -- C ABI of the GB300 (sm_103a) parametrix surface-PDE library.
 *
 * The library discretises and solves  div_G(a grad_G u) = f  on a closed
 * surface G with the parametrix integral-equation method of Goodwill and
 * O'Neil ("A parametrix method for elliptic surface PDEs"):
 *   - parametrix K(x, x') = log|x - x'| / (2 pi a(x'))           (Sec. 4.2, eq. diff_param)
 *   - remainder  R(x, x') = (a(x)/a(x')) [ q^2/pi - H(x) q/pi ]
 *                           + grad_G a(x) . r / (2 pi a(x') |r|^2),
 *     r = x - x', q = n(x).r/|r|^2                  (Thm. parametrix, eq. explicit_remainder, c = 0)
 *   - second-kind equation  sigma + R[sigma] = f,  u = K[sigma]  (Thm. second_kind, eq. IE)
 *   - Nystrom discretisation with smooth, singular (polar) and nearly
 *     singular (adaptive) quadrature                              (Sec. 6.1)
 *
 * Surface discretisation (the input of pm_surface_create): npatch
 * quadrilateral patches, each the image of [-1,1]^2, with p x p nodes at the
 * tensor product of the ascending p-point Gauss-Legendre nodes.  Node
 * numbering is patch-major: global index  P*p*p + i*p + j  for node (u_i, v_j)
 * of patch P (i along u, j along v).  N = npatch*p*p.  All array arguments
 * are row-major, node-major (e.g. nodes[3*k + c]).
 *
 * Conventions for every call:
 *   - Every function returns a pm_status; nothing aborts, traps or prints.
 *     pm_last_error() returns a message for the calling thread's last error.
 *   - The caller owns all arrays it passes.  Inputs are copied during the
 *     call; the library never keeps a caller pointer.
 *   - Host pointers must be valid for the sizes stated; device pointers
 *     (on_device = 1) must be device memory on the context's device.
 *   - A NULL stream means the CUDA legacy default stream.  Calls with host
 *     buffers synchronise the stream before returning; calls with device
 *     buffers are asynchronous on the stream.
 *   - Handles are not thread-safe: one thread at a time per surface.
 */
#ifndef PARAMETRIX_H
#define PARAMETRIX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pm_ctx pm_ctx;          /* one CUDA device                        */
typedef struct pm_surface pm_surface;  /* geometry + near field + coefficient    */

typedef enum {
    PM_OK = 0,
    PM_ERR_INVALID_ARG = 1,       /* bad size, NULL, non-finite or inconsistent input */
    PM_ERR_OOM = 2,               /* device or host allocation failed               */
    PM_ERR_CUDA = 3,              /* a CUDA runtime call failed                     */
    PM_ERR_NOT_CONVERGED = 4,     /* pm_solve: tolerance not reached in maxit       */
    PM_ERR_BREAKDOWN = 5,         /* pm_solve: Krylov breakdown                     */
    PM_ERR_RHS_NOT_MEAN_ZERO = 6, /* pm_solve: f has a non-zero mean (Thm. LBsolvable) */
    PM_ERR_TIMEOUT = 7,           /* a bounded device wait ran out                  */
    PM_ERR_INTERNAL = 8,          /* a device-side check failed (recorded, not trapped) */
    PM_ERR_NO_COEFF = 9           /* the surface has no coefficient yet             */
} pm_status;

typedef enum {
    PM_PREC_FP64 = 0,     /* float64 smooth sums and float64 near-field values      */
    PM_PREC_FP32 = 1,     /* float32 smooth sums with compensated (TwoSum) tile
                             accumulation, float32 near-field values               */
    PM_PREC_FP32_TC = 2,  /* reserved for the tensor-core FMM far field            */
    PM_PREC_FF = 3,       /* float-float (FP32-pair, ~48-bit) smooth sums on the FP32
                             pipe, float64 near-field values: float64-class accuracy
                             (~1e-13 relative) at a fraction of GB300's float64 cost */
    PM_PREC_FMM = 4       /* float32 Chebyshev kernel-interpolation FMM for the smooth
                             sums (far field by 8x8x8-point box expansions, adjacent
                             leaves exact), float32 near-field values; large surfaces */
} pm_precision;

/* Quadrature and solver options (pm_default_opts fills the defaults). */
typedef struct {
    double near_factor;     /* target is near a patch if |x - c_P| < near_factor * rho_P
                               (c_P, rho_P: centroid and radius of the 4 corner images);
                               Sec. 6.1.2 uses 1.5                                     */
    double theta_tol;       /* self rule: absolute tolerance of the adaptive theta panels
                               on int L(theta)^2 (Sec. 6.1.1 criterion); 1e-14          */
    double theta_max_width; /* self rule: largest theta panel (radians); 0 (default) =
                               pi/16 for p <= 10, pi/24 for p = 11                       */
    double near_eta;        /* near rule: split a sub-square while the target is within
                               2*near_eta*(its corner radius) of its centre; 1.0       */
    int near_max_depth;     /* near rule: deepest subdivision level; 12                 */
    int near_max_leaves;    /* near rule: leaf budget per (target, patch), <= 512; 512 */
    int gmres_restart;      /* pm_solve: Krylov subspace size per cycle; 50             */
    int max_refine;         /* pm_solve: iterative-refinement steps; 8                  */
    double inner_tol;       /* pm_solve: relative tolerance of each inner float32 GMRES; 1e-6 */
    double mean_tol;        /* pm_solve: |sum w f| / (sqrt(sum w) ||f||_w) above which f
                               is rejected as not mean zero; 1e-8                       */
    int residual_prec;      /* pm_solve: precision of true residuals and of u = K~ sigma
                               (PM_PREC_FF or PM_PREC_FP64; default PM_PREC_FF).
                               PM_PREC_FP32: a float32 or FMM solve takes both in its own
                               operator precision -- GMRES (float64 basis) to tol on the
                               float32 / FMM operator, no float-float refinement; u then
                               carries that operator's error (~1e-5 relative)            */
    int fmm_depth;          /* PM_PREC_FMM: octree depth (2..8); 0 = chosen by a cost model */
    int batch_rhs;          /* nrhs > 1: 1 = batched kernels and lockstep GMRES over all
                               right-hand sides (default), 0 = one right-hand side at a time */
    int direct_tpt;         /* float32 smooth sums: targets per thread (1, 2 or 4); 0 = auto */
    int direct_blocks_per_sm; /* float32 smooth sums: source splits chosen so the grid holds
                               about this many blocks per SM (1..16); 0 = auto          */
    int direct_symmetric;   /* float-float smooth sums: 1 = evaluate each
                               unordered node pair once (tile pairs; row and column sums
                               from the shared pair geometry) where the (N/128) x N
                               partial slices fit in 1 GiB, else one-sided sums (default);
                               0 = one-sided sums always                                */
    int residual_update;    /* pm_solve with float32/FMM applies: after a correction d, take
                               r - A32 d as the next residual when 1e-5 |d| (the float32
                               operator's error bound on d) is below 0.1 tol |f|, instead of
                               recomputing f - A sigma in residual_prec; 1 (default) or 0 */
    int fmm_tensor_m2l;     /* PM_PREC_FMM far field: 1 = M2L as one operator GEMM per offset
                               class (16 classes of the 316 V-list offsets under the cube's
                               signed axis permutations) on the float16 tensor cores (the
                               library's own tcgen05 kernel), float32 operands scaled by
                               powers of two and split in two float16 parts (three
                               products), float32 accumulation; operators ~0.25 GB per
                               context, built once (default); 0 = M2L evaluated directly
                               on the float32 pipe                                        */
} pm_opts;

void pm_default_opts(pm_opts* opts);

/* Create a context on CUDA device `device`.  *out is NULL on failure. */
pm_status pm_ctx_create(int device, pm_ctx** out);
void pm_ctx_destroy(pm_ctx* ctx);

/*
 * Create a surface and build its near field (Sec. 6.1).
 *   nodes     [N*3]  positions y(u_i, v_j)
 *   normals   [N*3]  outward unit normals
 *   tangents  [N*6]  (dy/du, dy/dv) with respect to the [-1,1]^2 patch coordinates
 *   curvature [N]    mean curvature H = (1/2) div_G n (outward n: H = 1/R on a sphere)
 *   weights   [N]    smooth-rule weights w = omega_i omega_j |y_u x y_v| (Gauss weights
 *                    omega); checked against the tangents to 1e-8 relative
 *   opts      NULL for the defaults
 * The near field is built once here, in float64, as coefficient-independent
 * quadrature weights (self: polar rule of eq. radial_int; near: adaptive
 * subdivision of Sec. 6.1.2).  Requires 2 <= p <= 11 and npatch >= 1.
 * PM_ERR_INVALID_ARG for bad sizes, NULL arrays or non-finite/inconsistent values.
 */
pm_status pm_surface_create(pm_ctx* ctx, int npatch, int p,
                            const double* nodes, const double* normals,
                            const double* tangents, const double* curvature,
                            const double* weights, const pm_opts* opts,
                            pm_surface** out);
void pm_surface_destroy(pm_surface* s);

/*
 * A second surface on src's geometry: it shares src's nodes, normals, near-field
 * structure and quadrature weights (read-only once built; nothing is recomputed
 * or copied) and has its own coefficient, sum buffers, solver state and FMM tree.
 * Options and knobs are copied from src.  Call pm_surface_set_coeff on it before
 * applying or solving.  The shared buffers are freed with the last surface that
 * uses them, so src may be destroyed first.  PM_ERR_INVALID_ARG for NULL
 * arguments; PM_ERR_OOM / PM_ERR_CUDA if its own buffers cannot be allocated.
 */
pm_status pm_surface_clone(const pm_surface* src, pm_surface** out);

/*
 * Change the float32 smooth-sum launch shape of an existing surface (the
 * autotuner's knobs; no quadrature is recomputed).  direct_tpt in {0,1,2,4},
 * direct_blocks_per_sm in 0..16 (0 = automatic choice).
 */
pm_status pm_surface_tune(pm_surface* s, int direct_tpt, int direct_blocks_per_sm);

/*
 * Launch-shape knobs of a surface's applies: the autotuner's search space.
 * 0 in any field selects the built-in choice.  None changes a result beyond
 * float32 summation order; none recomputes quadrature.
 */
typedef struct {
    int direct_tpt;           /* float32 sums, one right-hand side: targets per thread, 1/2/4 (2) */
    int direct_blocks_per_sm; /* float32 sums, one right-hand side: source splits chosen for
                                 about this many blocks per SM, 1..16 (12)                  */
    int batch_rhs_per_block;  /* batched float32 sums: right-hand sides per block, 8/16/32 (16) */
    int batch_blocks_per_sm;  /* batched float32 sums: blocks aimed at per SM, 1..16 (8)     */
    int fmm_depth;            /* PM_PREC_FMM: octree depth 2..8 (cost model); a change drops
                                 the surface's tree, rebuilt at the next FMM apply          */
    int fmm_streams;          /* PM_PREC_FMM: 1 = every kernel of an apply on the caller's
                                 stream, one after another; 2 = the far field (P2M, M2M,
                                 M2L, L2L) on a second stream of the highest priority, beside
                                 the adjacent-leaf P2P on the caller's stream (2)           */
} pm_knobs;

/* Set (all fields, validated first: PM_ERR_INVALID_ARG leaves the surface
 * unchanged) or read the surface's knobs.  Setting synchronises the device; no
 * other call may use the surface meanwhile (applies, solves, server requests). */
pm_status pm_surface_set_knobs(pm_surface* s, const pm_knobs* k);
pm_status pm_surface_get_knobs(const pm_surface* s, pm_knobs* k);

typedef struct {
    pm_knobs best;        /* fastest configuration found; now set on the surface      */
    double best_ms;       /* its time per remainder apply (median of the repetitions)  */
    double default_ms;    /* time per apply with the built-in choice (a candidate too) */
    int candidates;       /* configurations timed                                     */
} pm_tune_result;

/*
 * Autotuner: times remainder applies (smooth sums + near field) of nrhs
 * right-hand sides in precision prec for every candidate launch shape and keeps
 * the fastest.  prec = PM_PREC_FP32, nrhs = 1: direct_tpt x direct_blocks_per_sm
 * ({1,2,4} x {4,8,12,16}); PM_PREC_FP32, nrhs > 1: batch_rhs_per_block x
 * batch_blocks_per_sm ({8,16,32} x {4,8,12,16}); PM_PREC_FMM (nrhs = 1): the
 * cost model's depth and its two neighbours (depths whose leaves exceed the
 * P2P limit are skipped).  Each candidate: one warm-up apply, then reps
 * (1..100) applies timed with CUDA events on a private stream; the median
 * counts.  The input is a fixed smooth density, allocated and freed here.
 * Requires pm_surface_set_coeff; no other call may use the surface meanwhile.
 * On an error the knobs in force before the call are restored.  out may not be
 * NULL.
 */
pm_status pm_surface_autotune(pm_surface* s, int nrhs, pm_precision prec, int reps,
                              pm_tune_result* out);

/* Device name (NUL-terminated, truncated to len - 1 bytes) and SM count of the
 * context's GPU; either pointer may be NULL.  Keys autotuner caches. */
pm_status pm_ctx_info(const pm_ctx* ctx, char* name, int len, int* num_sms);

/*
 * FMM tree statistics (builds the tree on first use): stats[0] = adjacent-leaf
 * source/target pairs evaluated exactly, stats[1] = far-field box pairs
 * (V lists), stats[2] = depth, stats[3] = number of boxes.
 */
pm_status pm_surface_fmm_stats(pm_surface* s, double stats[4]);

/*
 * Stored float-float smooth-sum matrices (Sec. 6.1, the smooth part of the
 * Nystrom discretisation of eq. explicit_remainder and eq. diff_param).  which:
 * bit 0 = the remainder kernel, bit 1 = the parametrix kernel, 0 = release both.
 * Each stored kernel is evaluated once at every ordered pair (i, j != i) in the
 * float-float arithmetic of the PM_PREC_FF sums and kept in device memory in 6
 * bytes: the high float and a 16-bit code of the low word, which restores the
 * entry to within 2^-40 of its magnitude.  The remainder matrix takes N x ld
 * entries (ld = N rounded up to 128); the parametrix matrix, which is symmetric,
 * takes the upper triangle of 128 x 128 tiles on surfaces that use the symmetric
 * float-float sums (opts.direct_symmetric, N >= 256), else N x ld entries: 58 GB
 * and 29 GB at N = 98,304.  Every later PM_PREC_FF apply of a stored kernel
 * (solves' refinement residuals and representation included) reads the matrix
 * instead of evaluating the pairs; results agree with the unstored sums to about
 * 2^-40 relative.  pm_surface_set_coeff re-evaluates the stored
 * remainder matrix (it carries the coefficient); the parametrix matrix depends
 * on the geometry only.  Clones do not inherit stored matrices; a c != 0
 * coefficient (pm_surface_set_coeff_c) releases them; pm_surface_destroy frees them.
 * Requires pm_surface_set_coeff.  Refused with PM_ERR_OOM, storing nothing, when
 * the matrices would not fit in the free device memory less a margin of
 * max(1 GiB, 2 % of the device); any matrix stored before the call is released
 * first.  Synchronises the device; no other call may use the surface meanwhile.
 * PM_ERR_INVALID_ARG for a NULL surface, which outside 0..3 or a c != 0 surface.
 */
pm_status pm_surface_store_ff(pm_surface* s, int which);

/* The kernels currently stored by pm_surface_store_ff (same bits; 0 for NULL). */
int pm_surface_stored_ff(const pm_surface* s);


/* Number of nodes N and near-field blocks (target, near patch) of a surface. */
pm_status pm_surface_info(const pm_surface* s, int* N, int* nblocks);

/*
 * Set the coefficient a (> 0) of div_G(a grad_G u) = f (Sec. 4.2).
 *   a      [N]    host array, every value finite and > 0
 *   grad_a [N*3]  host array of the surface gradient grad_G a at the nodes, or
 *                 NULL to compute it by spectral differentiation of the patch
 *                 interpolant of a (eq. gradg)
 * Combines the stored quadrature weights into the near-field corrections of
 * R and K; no quadrature is recomputed.
 * Advection (Sec. 4.3, eq. adv_remainder): for div_G(a grad_G u) + b . grad_G u = f
 * with a tangential field b, pass grad_a = grad_G a + b.  The advection term
 * b . grad_G K of the remainder has the form of its grad_G a term, so every apply
 * and solve then uses R_b.  For b with non-zero surface divergence the range is no
 * longer the mean-zero functions: solve with PM_SOLVE_PROJECT_RHS (the rank-one
 * term still selects the solution; u is returned with zero mean).
 */
pm_status pm_surface_set_coeff(pm_surface* s, const double* a, const double* grad_a);

/*
 * Apply the discretised remainder operator: out = R~ sigma (Sec. 6.1, eq. IEsum).
 * R~ sigma_i = sum_{j != i} w_j R(x_i, x_j) sigma_j + sum_{near k} C_ik sigma_k.
 * The identity and the rank-one term of the solve are NOT included.
 *   sigma, out  [nrhs*N] float64, right-hand side r at offset r*N
 *   on_device   1: device pointers (asynchronous on stream); 0: host pointers
 * PM_ERR_NO_COEFF before pm_surface_set_coeff.
 */
pm_status pm_apply_R(pm_surface* s, const double* sigma, double* out, int nrhs,
                     pm_precision prec, int on_device, void* stream);

/* out = K~ sigma, the discretised parametrix operator including 1/a(x')
 * (eq. representation); same conventions as pm_apply_R. */
pm_status pm_apply_K(pm_surface* s, const double* sigma, double* out, int nrhs,
                     pm_precision prec, int on_device, void* stream);

/* Parts of an apply, for testing and profiling; same conventions. */
enum {
    PM_PART_SMOOTH_R = 0,   /* sum_{j != i} w_j R(x_i, x_j) sigma_j only        */
    PM_PART_SMOOTH_K = 1,   /* sum_{j != i} w_j K(x_i, x_j) sigma_j only        */
    PM_PART_NEAR_R = 2,     /* sum_{near k} C^R_ik sigma_k only                 */
    PM_PART_NEAR_K = 3      /* sum_{near k} C^K_ik sigma_k only                 */
};
pm_status pm_apply_part(pm_surface* s, int part, const double* sigma, double* out,
                        int nrhs, pm_precision prec, int on_device, void* stream);

/*
 * Copy the near field to host arrays: row_ptr [N+1], blk_patch [nblocks]
 * (block b of row i covers patch blk_patch[b]; the target's own patch is the
 * first block of its row), corr_R / corr_K [nblocks*p*p] float64 corrections
 * C_ik = W_ik / a_k - w_k F(x_i, x_k) (k != i), C_ii = W_ii / a_i.
 * Any output pointer may be NULL.  corr_* need pm_surface_set_coeff first.
 */
pm_status pm_surface_get_near(const pm_surface* s, int* row_ptr, int* blk_patch,
                              double* corr_R, double* corr_K);

/* Flags of pm_solve. */
#define PM_SOLVE_PROJECT_RHS 1u    /* subtract the mean of f instead of rejecting it */
#define PM_SOLVE_DEVICE_PTRS 2u    /* f, u, sigma_out are device pointers            */
#define PM_SOLVE_INITIAL_GUESS 4u  /* sigma_out holds the starting density on entry  */

typedef struct {
    int iterations;          /* total inner GMRES iterations                         */
    int refinements;         /* outer refinement steps (true-residual evaluations)   */
    double residual;         /* final true relative residual ||f - A sigma|| / ||f|| */
    double removed_mean;     /* mean subtracted from f (PM_SOLVE_PROJECT_RHS)         */
    double seconds;          /* wall time of the call                                */
    int residual_updates;    /* residuals taken as r - A32 d (opts.residual_update)   */
} pm_solve_info;

/*
 * Solve div_G(a grad_G u) = f for the mean-zero u (Thm. LBsolvable, Thm. second_kind):
 * (I + R~ + 1 w^T) sigma = f by GMRES with a float64 Krylov basis and operator
 * applies in `prec` (PM_PREC_FP32, PM_PREC_FF or PM_PREC_FP64), iterative
 * refinement on true residuals in opts.residual_prec until ||f - A sigma||/||f||
 * <= tol, then u = K~ sigma (in opts.residual_prec) minus its weighted mean.
 *   f, u       [nrhs*N]  (host, or device with PM_SOLVE_DEVICE_PTRS)
 *   sigma_out  [nrhs*N] or NULL
 *   info       [nrhs] or NULL
 * With nrhs > 1 (and opts.batch_rhs) all right-hand sides are solved together:
 * batched multi-RHS smooth sums and lockstep GMRES; info[r].iterations then
 * counts the lockstep Arnoldi steps of the whole batch.
 * PM_SOLVE_INITIAL_GUESS (warm start, e.g. resuming a solve from a saved density):
 * sigma_out, required, holds a starting sigma per right-hand side on entry; the
 * solve begins from its true residual f - A sigma (0 iterations when that already
 * meets tol) and overwrites sigma_out with the final sigma.  Right-hand sides are
 * then solved one at a time.
 * PM_ERR_RHS_NOT_MEAN_ZERO if f is not mean zero and PM_SOLVE_PROJECT_RHS is not set;
 * PM_ERR_NOT_CONVERGED if tol is not met within maxit inner iterations.
 */
pm_status pm_solve(pm_surface* s, const double* f, double* u, int nrhs, double tol,
                   int maxit, pm_precision prec, unsigned flags, double* sigma_out,
                   pm_solve_info* info, void* stream);

/*
 * Open-surface boundary-value problems (Sec. 5): div_Gamma(a grad_Gamma u) = f on an
 * open surface Gamma with, on its boundary gamma, Neumann data nu . grad_Gamma u =
 * f_gamma (kind = PM_BVP_NEUMANN, Sec. 5.2, eq. NeuBVPsystem) or Dirichlet data
 * u = f_gamma (kind = PM_BVP_DIRICHLET, Sec. 5.3, eq. DirBVPsystem; a constant, as the
 * paper's compactness theorem for T_gamma requires).  s is a surface built by
 * pm_surface_create from Gamma's quadrilateral patches (its nodes interior to the
 * patches) with pm_surface_set_coeff done (c = 0); it must outlive the handle.  gamma
 * is ncurves closed curves; curve c is given at M[c] >= 2 edge nodes, the points at
 * t_k = 2 pi (k + 1/2) / M[c] of a 2 pi-periodic parameter t, and at F[c] M[c]
 * oversampled points t_j = 2 pi j / (F[c] M[c]) (Sec. 6.1.4's Fourier oversampling),
 * curve after curve.  Me = sum M[c] edge nodes (at most 4,096), Fo = sum F[c] M[c]
 * oversampled points, sum F[c] M[c]^2 (the interpolation matrices) at most 2^26.
 * Host arrays, copied by the call:
 *   edge_x [Me][3], edge_d1 [Me][3] = dgamma/dt, edge_d2 [Me][3] = d2gamma/dt2,
 *   edge_nu [Me][3] the unit binormal (tangent to Gamma, normal to gamma, pointing away
 *   from Gamma), edge_a [Me] = a > 0 at the node, edge_patch [Me] the patch whose
 *   edge holds the node and edge_uv [Me][2] the node's reference coordinates there
 *   (one of them -1 or +1; nodes should avoid patch corners);
 *   over_x [Fo][3], over_nu [Fo][3] (binormal), over_speed [Fo] = |dgamma/dt|,
 *   over_a [Fo] = a at the oversampled points.
 * The systems take sigma at the surface's N nodes and mu at the Me edge nodes:
 *   Neumann:   sigma + R~ sigma + R_gamma mu = f,
 *              -mu/(2a) + K'_Gamma sigma + K'_gamma mu + sum_k w_k mu_k = f_gamma,
 *              u = K~ sigma + K_gamma mu  (the rank-one term, w_k the trapezoid
 *              weights, removes the Neumann null space: u is unique up to a constant);
 *   Dirichlet: sigma + R~ sigma + T_gamma mu = f,  +mu/(2a) + K~ sigma + N_gamma mu = f_gamma,
 *              u = K~ sigma + N_gamma mu,
 * all in float64.  Creation computes the surface quadrature of every edge node on the
 * device, with s's coefficient built in: after a later pm_surface_set_coeff(_c) on s,
 * pm_bvp_apply and pm_bvp_solve refuse the handle (PM_ERR_INVALID_ARG); create a new
 * one.  PM_ERR_INVALID_ARG for NULL arguments, an unknown kind, bad sizes, an edge
 * node not on an edge of its patch or a non-constant a for Dirichlet; PM_ERR_NO_COEFF
 * without a coefficient.
 */
#define PM_BVP_NEUMANN 0
#define PM_BVP_DIRICHLET 1
typedef struct pm_bvp pm_bvp;
pm_status pm_bvp_create(pm_surface* s, int kind, int ncurves, const int* M, const int* F,
                        const double* edge_x, const double* edge_d1, const double* edge_d2,
                        const double* edge_nu, const double* edge_a, const int* edge_patch,
                        const double* edge_uv, const double* over_x, const double* over_nu,
                        const double* over_speed, const double* over_a, pm_bvp** out);
void pm_bvp_destroy(pm_bvp* b);

/* The system's operator on host arrays sigma [N], mu [Me] (rank-one term included):
 * out_s [N] the surface rows, out_e [Me] the edge rows. */
pm_status pm_bvp_apply(pm_bvp* b, const double* sigma, const double* mu, double* out_s,
                       double* out_e);

/* Solve for f [N], f_gamma [Me] (host) by restarted GMRES (opts.gmres_restart,
 * at most maxit iterations) to relative residual tol, then u [N] = K~ sigma +
 * K_gamma mu; sigma [N] and mu [Me] are written when not NULL.  info as for pm_solve
 * (refinements 0).  PM_ERR_NOT_CONVERGED (u, sigma, mu still written) when tol is
 * not reached. */
pm_status pm_bvp_solve(pm_bvp* b, const double* f, const double* f_gamma, double tol,
                       int maxit, double* u, double* sigma, double* mu, pm_solve_info* info);

/*
 * Solve several operators' systems together (the batched form across operators):
 * ops[k] u_k,r = f_k,r for r < nrhs[k], k < nops, as one lockstep GMRES over all
 * sum(nrhs) right-hand sides, with the float32 operator applies of every instance in
 * the same launches (one persistent smooth-sum launch over a work list of (instance,
 * target tile, right-hand-side group, source chunk) items, one near-field launch) and
 * each GMRES cycle replayed as one CUDA graph.  The operators may differ in geometry,
 * size and coefficient; each must appear once (give it several right-hand sides
 * instead), belong to one context and have its coefficient set.  f[k], u[k]: [nrhs[k]
 * * N_k] row-major per right-hand side, host arrays (device arrays with
 * PM_SOLVE_DEVICE_PTRS).  prec must be PM_PREC_FP32; solver options (restart length,
 * refinements, inner tolerance, residual update, mean tolerance and residual
 * precision: float-float refinement, or the float32 operator itself with
 * residual_prec = PM_PREC_FP32) are those of ops[0].  info (nullable) receives
 * sum(nrhs) entries in instance order; iterations count the lockstep Arnoldi steps.
 * The launch shape (right-hand sides per block, blocks per SM) is ops[0]'s batched
 * knobs (pm_surface_set_knobs / pm_surface_autotune).  One multi-instance solve runs
 * at a time per context (its workspace is the context's).  Errors as pm_solve, plus
 * PM_ERR_INVALID_ARG for a repeated operator, another context or another precision.
 */
pm_status pm_solve_multi(pm_surface* const* ops, int nops, const int* nrhs,
                         const double* const* f, double* const* u, double tol, int maxit,
                         pm_precision prec, unsigned flags, pm_solve_info* info, void* stream);

/*
 * Per-phase kernel timing.  While enabled, the library records a pair of CUDA
 * events on the launching stream around every launch of each phase; reading
 * synchronises on those events and returns the summed milliseconds and the
 * launch count since the last reset (reset = 1 clears them).  With
 * phase = PM_PHASE_COUNT, *ms is 0 and *launches is the number of kernels the
 * library launched for this surface since the last reset (counted whether or
 * not timing is enabled).  The two FMM phases time single kernels that also lie
 * inside the DIRECT_R / DIRECT_K phase of the same apply.
 */
enum {
    PM_PHASE_PREP = 0,        /* source strengths s = w sigma / a          */
    PM_PHASE_DIRECT_R = 1,    /* smooth remainder sum                      */
    PM_PHASE_DIRECT_K = 2,    /* smooth parametrix sum                     */
    PM_PHASE_NEAR = 3,        /* near-field correction + split reduction   */
    PM_PHASE_SOLVE_VEC = 4,   /* GMRES vector kernels                      */
    PM_PHASE_DIRECT64 = 5,    /* float64 or float-float smooth remainder sum */
    PM_PHASE_FMM_M2L = 6,     /* FMM M2L tensor-core GEMM (inside DIRECT_R/K) */
    PM_PHASE_FMM_P2P = 7,     /* FMM adjacent-leaf exact sums (inside DIRECT_R/K) */
    PM_PHASE_DIRECT64_K = 8,  /* float64 or float-float smooth parametrix sum */
    PM_PHASE_COUNT = 9
};
pm_status pm_profile_enable(pm_surface* s, int enable);
pm_status pm_profile_read(pm_surface* s, int phase, double* ms, int* launches, int reset);

/*
 * Diagnostic: the library's float-float natural logarithm (Tang's table
 * method) of x = xh + xl for n host values, written to out (host, float64).
 */
pm_status pm_selftest_fflog(pm_surface* s, const float* xh, const float* xl, int n,
                            double* out);

/*
 * Self-test of the FMM's M2L offset classes (host code only, no device call):
 * for the 343 box offsets d = (dx, dy, dz) in [-3, 3]^3, entry
 * k = ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3) of cls[343] receives the class
 * (0..15) of a V-list offset (max |d_i| in {2, 3}) or -1, and sym[343] the
 * signed axis permutation g with d = g d_c: bits 0-1, 2-3, 4-5 = pi(0..2),
 * bit 6 + a set where s_a = -1, (g v)_a = s_a v_pi(a).  canon[48] receives the
 * 16 canonical offsets d_c (x >= y >= z >= 0) as (x, y, z) triples.
 * PM_ERR_INVALID_ARG for NULL arrays.
 */
pm_status pm_selftest_fmm_classes(int* cls, int* sym, int* canon);

/*
 * Self-test of the tensor-core GEMM that carries the FMM's M2L (Sec. 6.2: the
 * far field as one dense operator product per offset class), on sm_103a
 * tcgen05 MMAs with float32 accumulators in tensor memory and TMA-staged
 * operand tiles:  C[j * rows + r] = sum_k A[r * K + k] * B[j * K + k]  for
 * r < rows, j < ncols.  Host arrays: A [rows * K] and B [ncols * K] hold
 * float16 (bf16 = 0) or bfloat16 (bf16 = 1) bit patterns, K-major; C
 * [ncols * rows] float32 receives the product (column j's rows contiguous).
 * The library allocates and frees the device copies.  reps > 0 runs the
 * product reps more times and writes the mean device time of one launch (ms)
 * to *ms.  PM_ERR_INVALID_ARG unless rows is a positive multiple of 128, K of
 * 64 and ncols >= 1 (or for NULL arrays, or reps > 0 with ms NULL);
 * PM_ERR_TIMEOUT if a bounded wait inside the kernel ran out (the kernel then
 * returns early and C is not valid); PM_ERR_CUDA for a failed CUDA call.
 */
pm_status pm_selftest_tc_gemm(pm_ctx* ctx, const unsigned short* A, const unsigned short* B,
                              float* C, int rows, int K, int ncols, int bf16, int reps,
                              double* ms);

/*
 * Self-test of the library's planar Green's function for c != 0 (host code only,
 * no device call; the same functions are compiled for the device).  Sec. 4.2,
 * eq. diff_param: with q = c/a (real, non-zero) and g = a G the Green's function
 * of Delta_2 + q, writes for each of the n radii r[i] > 0 (host, float64)
 * out[6 i .. 6 i + 5] = Re g, Im g, Re g', Im g', Re g'', Im g'' (host, float64),
 * g = -(i/4) H0(sqrt(q) r) for q > 0 and -K0(sqrt(-q) r) / (2 pi) for q < 0
 * (unit source strength: 2 pi r g' -> 1 as r -> 0).  PM_ERR_INVALID_ARG for NULL
 * arrays, n < 0, q zero or not finite, or a radius that is not finite and positive.
 */
pm_status pm_selftest_green(const double* r, int n, double q, double* out);

/*
 * The same in float32 (the evaluation the per-pair smooth sums use): r and out
 * are host float32 arrays, out[6 i .. 6 i + 5] as above.  Same errors.
 */
pm_status pm_selftest_green_f32(const float* r, int n, float q, float* out);

/*
 * Self-test of the float32 per-pair arithmetic of the c != 0 smooth sums (host code
 * only): for real c != 0, out[4 i .. 4 i + 3] = Re, Im of
 * sum_{j != i} a_j R(x_i, x_j) s_j and of sum_{j != i} a_j K(x_i, x_j) s_j
 * (eq. explicit_remainder with its c terms, eq. diff_param), each pair in float32,
 * summed in float64.  Host arrays: x, n, gb [N*3] (gb = grad_G a, plus b for
 * advection), H, a, c [N] float32; s [N*2] float32 complex (s_j = w_j sigma_j / a_j);
 * out [N*4] float64.  O(N^2).  PM_ERR_INVALID_ARG for NULL arrays, N < 0, a <= 0, or
 * c zero or not finite.
 */
pm_status pm_selftest_smooth_c_f32(int N, const float* x, const float* n, const float* H,
                                   const float* a, const float* gb, const float* c,
                                   const float* s, double* out);

/*
 * Device float32 smooth sums for real c != 0 (Sec. 6.1.3 smooth rule with the
 * kernels of eq. explicit_remainder and eq. diff_param): the same quantities as
 * pm_selftest_smooth_c_f32, from DEVICE arrays in the same layouts, each target's
 * sum compensated (TwoSum per 128 sources) and written to out [N*4] (device,
 * float64) on the given stream (NULL: the default stream).  Requires a > 0 and
 * c != 0 at every node (c = 0 is the library's c = 0 path) and distinct node
 * positions.  Asynchronous; PM_ERR_INVALID_ARG for NULL arrays or N outside
 * 1..2^26, PM_ERR_CUDA if the launch fails.  Its per-pair arithmetic is the
 * host-tested pair function above.
 */
pm_status pm_smooth_c_f32(int N, const float* x, const float* n, const float* H,
                          const float* a, const float* gb, const float* c, const float* s,
                          double* out, void* stream);

/*
 * Consistency check of a built surface (the library's substitute for a memory
 * checker): on the device, every index the apply kernels follow is verified
 * against the array it addresses (near-field row pointers and block patch/row
 * indices, own patch first, the per-patch near-field unions, the self-rule theta
 * plan), and the stored geometry, weight sets and corrections (float64 and
 * float32, complex for c != 0) are scanned for NaN and Inf.  Failed checks are
 * recorded in a device word (first failure kept); nothing traps.  Synchronises.
 * PM_OK, PM_ERR_INTERNAL with the failed check and index in pm_last_error(),
 * PM_ERR_INVALID_ARG for NULL, PM_ERR_CUDA if a launch fails.  A library built
 * with -DPM_BOUNDS_CHECK runs it before every pm_apply_R/K/part and scans each
 * result for non-finite values.
 */
pm_status pm_surface_check(pm_surface* s);

/*
 * Triangle patches (Sec. 6.1): a closed surface of npatch curved triangles over the
 * reference simplex T0 = {u, v >= 0, u + v <= 1}, each sampled at the same order-p
 * rule of nt = p (p + 1) / 2 nodes (the paper's Vioreanu-Rokhlin nodes, or any
 * unisolvent set inside T0 with positive weights), 2 <= p <= 8.
 *   ref [nt][3]: the rule's (u, v, w) on T0 (host, copied);
 *   nodes, normals [N][3], tangents [N][6] = (y_u, y_v), curvature [N] and weights [N]
 *   as in pm_surface_create, N = npatch * nt, node k of patch P at row P * nt + k;
 *   the weights must equal w_k |y_u x y_v| (relative 1e-8).
 * The patch geometry, surface element and density are interpolated from the nodes
 * in the polynomials of total degree <= p - 1 (Koornwinder basis, Sec. 6.1.2); the
 * near-field rules are the polar self rule about the target's node (theta split at
 * T0's vertex directions, Sec. 6.1.1) and midpoint subdivision of T0 into four
 * triangles with a 16 x 16 collapsed Gauss rule (Sec. 6.1.2).  The result is a
 * pm_surface like any other: pm_surface_set_coeff, the applies, pm_solve,
 * pm_solve_multi, pm_surface_clone and the server accept it (grad_a = NULL
 * differentiates a's interpolant); pm_surface_set_coeff_c refuses it.
 * PM_ERR_INVALID_ARG for NULL arrays, p or npatch out of range, nodes outside T0,
 * a non-unisolvent node set, weights or normals inconsistent with the tangents.
 */
pm_status pm_surface_create_tri(pm_ctx* ctx, int npatch, int p, const double* ref,
                                const double* nodes, const double* normals,
                                const double* tangents, const double* curvature,
                                const double* weights, const pm_opts* opts, pm_surface** out);

/*
 * Host self-test of the triangle basis (no GPU): for the rule ref [nt][3] of order p,
 * l [npts][nt] = the Lagrange basis of the nodes at the points (u[q], v[q]), and
 * Du, Dv [nt][nt] = d l_k / du, d l_k / dv at node j (row j).  PM_ERR_INVALID_ARG as
 * pm_surface_create_tri for the rule, or for NULL outputs.
 */
pm_status pm_selftest_tri_basis(int p, const double* ref, int npts, const double* u,
                                const double* v, double* l, double* Du, double* Dv);

/*
 * Host self-test (no GPU) of the library's float64 g, g', g'' for complex q = c/a
 * (as pm_selftest_green; the branch arg q in (-pi/2, 3pi/2], K0 and K1 at complex
 * argument by their series and a deformed integration contour): out [n][6] =
 * (re, im) of g, g', g''.  q_im = 0 is pm_selftest_green.  PM_ERR_INVALID_ARG for
 * NULL arrays, n < 0, r <= 0 or not finite, q zero or not finite.
 */
pm_status pm_selftest_green_c(const double* r, int n, double q_re, double q_im, double* out);

/*
 * Helmholtz and modified-Helmholtz surface problems, div_G(a grad_G u) + c u = f
 * with c real or complex (Sec. 4.2; Thm. second_kind with the parametrix of eq.
 * diff_param and the remainder of eq. explicit_remainder).  With q = c/a the
 * kernels use g(r; k) = -(i/4) H0(k r), k^2 = q on the branch arg q in
 * (-pi/2, 3pi/2] (real q < 0: -K0(sqrt(-q) r)/(2 pi); complex q: K0, K1 at complex
 * argument), and log(r)/(2 pi) where q = 0 exactly; the source's q enters through
 * k(y) (at the nodes in the smooth rule, interpolated on the patch in the singular
 * and near rules).  There is no null space: sigma + R~ sigma = f and
 * u = K~ sigma, with no rank-one term and no mean condition on f or u.
 *
 * pm_surface_set_coeff_c: a [N] > 0, grad_a [N][3] or NULL (spectral, as in
 * pm_surface_set_coeff), c [N][2] complex (re, im) and finite (host arrays, copied).  It sets a
 * as pm_surface_set_coeff does and, when some c is non-zero, builds the complex
 * float64 near-field corrections of the c != 0 operators (Sec. 6.1.1 polar rule
 * with dyadically graded radial panels, Sec. 6.1.2 subdivision; synchronises).
 * The surface is then in c mode: pm_apply_R/K/part, pm_solve, pm_solve_multi,
 * the server and the autotuner refuse it (PM_ERR_INVALID_ARG) until
 * pm_surface_set_coeff is called again.  All c == 0 is pm_surface_set_coeff.
 * PM_ERR_INVALID_ARG for NULL a or c, non-finite c (and what pm_surface_set_coeff
 * rejects), PM_ERR_INTERNAL if a near-field leaf budget is exceeded.
 */
pm_status pm_surface_set_coeff_c(pm_surface* s, const double* a, const double* grad_a,
                                 const double* c);

/*
 * One apply of a c-mode surface in float64: out = R~ sigma (which_K = 0) or
 * out = K~ sigma (which_K = 1).  sigma and out are complex [N][2] (re, im
 * interleaved), host arrays (synchronous) or, with on_device = 1, device
 * arrays (asynchronous on the stream; NULL: the default stream).
 * PM_ERR_NO_COEFF if the surface is not in c mode, PM_ERR_INVALID_ARG for NULL
 * arrays or which_K outside {0, 1}.
 */
pm_status pm_apply_c(pm_surface* s, int which_K, const double* sigma, double* out,
                     int on_device, void* stream);

/*
 * Solve of a c-mode surface: GMRES(opts.gmres_restart) in complex float64 on
 * sigma + R~ sigma = f from sigma = 0 until the true residual |f - A sigma| is at
 * most tol |f| (checked after each restart cycle) or maxit Arnoldi steps, then
 * u = K~ sigma.  f, u and sigma_out (nullable) are complex [N][2] host arrays;
 * info (nullable): iterations, restart cycles (in .refinements), the final
 * relative residual, removed_mean = 0.  PM_ERR_NOT_CONVERGED (u and info still
 * written) when the tolerance is not met; PM_ERR_NO_COEFF if the surface is not
 * in c mode; PM_ERR_INVALID_ARG for NULL f or u, tol <= 0 or maxit < 1.
 */
pm_status pm_solve_c(pm_surface* s, const double* f, double* u, double tol, int maxit,
                     double* sigma_out, pm_solve_info* info);

/*
 * Serving: continuous batching of solve requests over many operators.
 *
 * A request names its operator either as a caller's pm_surface whose coefficient
 * is set (pm_server_submit) or as a description (pm_server_submit_desc): the
 * geometry arrays of pm_surface_create and the coefficient of
 * pm_surface_set_coeff, keyed by caller ids of the geometry and of the
 * coefficient.  The server builds a described operator itself on a worker the
 * first time it is needed (near-field build for a new geometry id; a clone that
 * shares the near-field weights for a new coefficient id on a built geometry)
 * and keeps it resident for later requests with the same ids; it is destroyed
 * with the server.
 *
 * pm_server_create starts n_workers threads, each with its own CUDA stream.  A
 * worker takes the operator whose oldest waiting request arrived first among the
 * operators no other worker is serving; builds it if needed; otherwise admits up
 * to max_batch of that operator's waiting requests of one precision (in arrival
 * order) and solves them together (batched applies, lockstep GMRES, float-float
 * refinement; see pm_solve).  Requests arriving meanwhile join later batches, so
 * work on different operators overlaps on the device.
 *
 * Memory admission: every build and batch reserves the device bytes it will
 * newly allocate, from a model of the library's allocations (operator arrays,
 * near field; Krylov and batched workspaces an operator does not already hold;
 * the FMM tree), and is admitted only while the reservations in flight plus its
 * own stay within hbm_budget_bytes and, measured by cudaMemGetInfo at admission,
 * within the device's free memory less a margin of max(256 MiB, 2% of the
 * device).  With nothing else in flight the oldest work is admitted regardless
 * of the free-memory reading; if its allocation then fails the request ends with
 * PM_ERR_OOM and the server continues.
 *   hbm_budget_bytes  cap on the bytes the server may reserve at once
 *   max_batch         right-hand sides per batch (1 = one request at a time)
 * pm_server_submit copies f (host, [N]) and returns a ticket; prec is the solve's
 * operator precision (FP64, FP32, FF or FMM; PM_ERR_INVALID_ARG otherwise), and a
 * batch only joins requests of one operator and one precision; PM_ERR_OOM if one
 * request's modelled workspace alone exceeds the budget.  Operators handed to a
 * server must not be used by the caller until every request on them has been
 * waited for.  pm_server_wait blocks until the ticket is done (timeout_ms < 0: no
 * limit; PM_ERR_TIMEOUT otherwise, the ticket stays valid), copies u (host, [N])
 * and the solve info, reports the submit-to-finish latency, releases the ticket
 * and returns the solve's status; on failure pm_last_error() on the waiting
 * thread holds the worker's message.  One thread at a time may wait on a ticket:
 * a second concurrent pm_server_wait on it returns PM_ERR_INVALID_ARG.
 */
typedef struct pm_server pm_server;
pm_status pm_server_create(pm_ctx* ctx, size_t hbm_budget_bytes, int max_batch, int n_workers,
                           pm_server** out);
void pm_server_destroy(pm_server* sv);
pm_status pm_server_submit(pm_server* sv, pm_surface* op, const double* f, double tol,
                           pm_precision prec, unsigned long long* ticket);

/* An operator described by its arrays (host, copied at submit when the ids are new;
 * the arrays of a request whose ids the server already knows are not read).
 * geometry_id names one geometry (the same npatch, p and arrays every time);
 * coeff_id one coefficient on it.  Arrays as pm_surface_create (nodes, normals
 * [N*3], tangents [N*6], curvature, weights [N]) and pm_surface_set_coeff
 * (a [N] > 0, grad_a [N*3] or NULL); opts NULL for the defaults. */
typedef struct {
    unsigned long long geometry_id, coeff_id;
    int npatch, p;
    const double *nodes, *normals, *tangents, *curvature, *weights;
    const double *a, *grad_a;
    const pm_opts* opts;
} pm_operator_desc;

/* Submit a request on a described operator.  PM_ERR_INVALID_ARG for NULL arrays
 * of a new operator, p outside 2..11, or a geometry id seen before with another
 * node count; PM_ERR_OOM if the operator's modelled size exceeds the budget.  A
 * build that fails ends every request on that operator with the build's status
 * and message. */
pm_status pm_server_submit_desc(pm_server* sv, const pm_operator_desc* desc, const double* f,
                                double tol, pm_precision prec, unsigned long long* ticket);
pm_status pm_server_poll(pm_server* sv, unsigned long long ticket, int* done);
pm_status pm_server_wait(pm_server* sv, unsigned long long ticket, double* u,
                         pm_solve_info* info, double* latency_s, int timeout_ms);

/* Times of one request (seconds): submit to finish; the part spent building its
 * operator while it waited (near field or clone; 0 if the operator was resident);
 * the solve of its batch; the rest, waiting in the queue. */
typedef struct {
    double latency_s, build_s, solve_s, queue_s;
} pm_request_times;
pm_status pm_server_wait_ex(pm_server* sv, unsigned long long ticket, double* u,
                            pm_solve_info* info, pm_request_times* times, int timeout_ms);
pm_status pm_server_stats(pm_server* sv, long long* batches, long long* solved,
                          long long* max_batch, size_t* bytes_in_use);
/* Change the batch limit and the number of workers that take new work (1 ..
 * n_workers of pm_server_create; the others idle) for batches formed from now
 * on; the operators the server holds stay resident.  PM_ERR_INVALID_ARG outside
 * those ranges. */
pm_status pm_server_configure(pm_server* sv, int max_batch, int active_workers);
/* Operator builds so far, bytes reserved now, the free-memory margin, operators known. */
pm_status pm_server_stats_ex(pm_server* sv, long long* builds, size_t* reserved_bytes,
                             size_t* margin_bytes, int* operators);

/*
 * Smooth remainder sum without any allocation.
 *
 * Some callers cannot call cudaMalloc: code whose device memory is owned
 * entirely by another allocator (a framework's caching pool or a fixed arena,
 * where a side allocation can fail or fragment it), latency-critical loops
 * where cudaMalloc/cudaFree would synchronise the device, and callers that
 * may not create a pm_surface at all (creating one allocates).  This entry
 * point computes, with the same float32 compensated kernel as
 * pm_apply_part(PM_PART_SMOOTH_R, PM_PREC_FP32),
 *   out[i] = sum_{j != i} s[j] [ (a_i/pi) q^2 - (a_i H_i/pi) q + grad_a_i . r/(2 pi |r|^2) ],
 *   r = x_i - x_j, q = n_i . r / |r|^2,
 * i.e. the smooth remainder sum for strengths s[j] = w_j sigma_j / a_j supplied
 * by the caller.  It has no counterpart in the paper (an interface addition).
 *   N                   1 <= N <= 32768 (larger N is rejected with PM_ERR_INVALID_ARG)
 *   x, n, grad_a [N*3]  device float32 positions, unit normals, grad_G a
 *   H, a, s      [N]    device float32 mean curvature, coefficient (> 0), strengths
 *   out          [N]    device float64 result
 *   stream              cudaStream_t (NULL: legacy default stream); asynchronous
 * Scratch: the packed sources/targets and per-split partial sums live in one
 * file-scope device array of 4 MiB that every GPU loading the library holds
 * until the process exits.  Each call made outside stream capture looks up that
 * array's device address in the current context (cudaGetSymbolAddress, which
 * allocates nothing) and remembers it for the device; a call made while the
 * stream is being captured uses the address remembered from the last
 * uncaptured call on that device, so make one call on each device before any
 * stream capture (otherwise the captured call returns PM_ERR_INVALID_ARG).
 * Every call overwrites the parts it reads, so nothing must be cleared between
 * calls, but all calls share the one array: calls that overlap on the GPU
 * (different streams, or different host threads, on the same device) race and
 * corrupt each other's results.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  Requires distinct node positions;
 * the j = i term is an exact zero for any finite strength.
 */
pm_status pm_smooth_remainder_f32_noalloc(int N, const float* x, const float* n,
                                          const float* H, const float* a,
                                          const float* grad_a, const float* s,
                                          double* out, void* stream);

const char* pm_status_str(pm_status st);
const char* pm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PARAMETRIX_H */
