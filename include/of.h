/*
 * of.h -- C ABI of the GB300 optical-flow solver.
 *
 * The library solves, for a batch of frame pairs, the P1 finite-element
 * system of the Horn-Schunck optical-flow model with an illumination unknown
 * (Gilliocq-Hirtz & Belhachmi, arXiv 1508.02977):
 *
 *   -div(Lambda grad U) + A U = F  in Omega,  dU/dn = 0 on dOmega
 *                                     (Section 1, Eq. eqpro1illu)
 *   U = (u1, u2, m),  Lambda = (alpha, alpha, lambda),
 *   A = g g^T,  F = -ft g,  g = (f_x, f_y, -f)   (Eq. OF2, Eq. BW2, rho = 0)
 *
 * discretised by P1 elements on the pixel grid, two triangles per pixel
 * square (Section 2.2, Eq. discret-form, Fig. sch-mesh), with a per-element
 * regularisation alpha adapted by the indicator of Section 2.3 (Eq. errind).
 *
 * Discretisation conventions shared by every entry point:
 *  - one node per pixel centre; node (x, y), 0 <= x < W, 0 <= y < H;
 *  - square (x, y), x < W-1, y < H-1, split along (x,y)->(x+1,y+1):
 *      t = 0: (x,y) (x+1,y) (x+1,y+1)      t = 1: (x,y) (x,y+1) (x+1,y+1);
 *  - per element K: g_K = (d/dx, d/dy of the P1 interpolant of frame 2,
 *    -mean of frame 1 over the 3 vertices), ft_K = mean of (f2 - f1);
 *  - m is delta m = M - 1 of the illumination law f2(x+u) = M f1(x)
 *    (Eq. deltam).
 *
 * Layouts (all row-major, row pitch in elements, pitch >= row length):
 *  - frame  [H][pitch]                    (f1, f2, dL/df1, dL/df2)
 *  - alpha  [H-1][W-1][2] contiguous      (element (x,y,t) at (y*(W-1)+x)*2+t)
 *  - vector [3][H][W] contiguous planes   (U, dL/dU; u1, u2, m)
 *
 * Pointers: unless stated otherwise an array argument may be a device
 * pointer or a host pointer (pinned host memory gives asynchronous copies);
 * the library tells them apart through unified addressing.  All work is
 * ordered on the stream given to of_create; an input must stay valid until
 * that stream has passed the call, an output is valid once it has (the
 * entry points that return host-side results synchronise the stream
 * themselves and say so).  Arrays stay owned by the caller; the library owns
 * only its own workspace, released by of_destroy.
 *
 * Errors: every entry point returns an of_status; no entry point aborts,
 * traps or prints.  of_last_error gives a message for the last non-OK status
 * of a handle.  A CUDA error inside a call returns OF_ERR_CUDA.  A build of
 * the library compiled with -DOF_BOUNDS_CHECK checks the device indices of
 * its kernels against their buffers; a violation skips the access, sets a
 * bit of the device error word, and the entry point returns OF_ERR_CUDA
 * ("a device index check failed").
 */
#ifndef OF_H_
#define OF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct of_ctx *of_handle;

typedef enum {
    OF_OK = 0,
    OF_ERR_ARG = 1,            /* invalid argument (null handle, bad size, pair out of range) */
    OF_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    OF_ERR_OOM = 3,            /* device allocation failed */
    OF_ERR_STATE = 4,          /* call out of order (e.g. of_solve before of_set_frames) */
    OF_ERR_NOT_CONVERGED = 5,  /* iteration cap reached; the best iterate is written */
    OF_ERR_BREAKDOWN = 6,      /* non-finite or non-positive CG scalar (singular/indefinite data) */
    OF_ERR_TIMEOUT = 7         /* a bounded device wait ran out */
} of_status;

typedef enum { OF_F32 = 0, OF_F64 = 1 } of_dtype;

typedef enum {
    OF_PREC_FP64 = 0,   /* every step in FP64 (frames, alpha and vectors stored in FP64) */
    OF_PREC_MIXED = 1   /* FP32 inner PCG + Schwarz sweeps; FP64 residual, dots, refinement */
} of_precision;

typedef enum {
    OF_PC_SCHWARZ = 0,  /* overlapping Schwarz, symmetric variant, as the PCG preconditioner */
    OF_PC_JACOBI = 1    /* node-block Jacobi (3x3 blocks); no subdomains */
} of_preconditioner;

typedef enum {
    OF_MODEL_ILLUMINATION = 0,  /* (u1, u2, m): brightness change m, Eq. OF2 and Eq. eqpro1illu */
    OF_MODEL_CONSTANT = 1       /* brightness constancy (Horn and Schunck, Eq. BW without m): the
                                   illumination column of the data term is dropped; m stays 0 */
} of_model;

/* Grid options.  A field left at 0 takes the default in brackets. */
typedef struct {
    int tile_x, tile_y;      /* owned subdomain tile in nodes, multiples of 4 [32 x 32] */
    int overlap;             /* extension of each subdomain on interior sides, nodes (0: none) */
    int sweeps;              /* symmetric 3-colour block SOR sweeps per local solve [1] */
    of_precision precision;  /* [OF_PREC_FP64] */
    double lambda;           /* regularisation of m (Eq. BW2) [1.0] */
    of_preconditioner preconditioner;  /* [OF_PC_SCHWARZ] */
    double omega;            /* relaxation factor of the local sweeps, 0 < omega < 2 [1.0: block
                                Gauss-Seidel]; any such value keeps the preconditioner symmetric
                                positive definite (the colour order is a palindrome) */
    double sigma;            /* K_sigma pre-smoothing of the frames (Section 1), standard deviation
                                in pixels, 0 <= sigma <= 16 [0: frames used as given]; sampled
                                Gaussian of radius ceil(3 sigma) along x then y, each pass normalised
                                over the taps inside the image */
    of_model model;          /* [OF_MODEL_ILLUMINATION] */
    int coarse;              /* two-level preconditioner: spacing in nodes of a coarse grid (nodes at
                                0, s, 2s, ... and W-1, likewise in y) whose bilinear hat functions add
                                the correction R0^T (R0 A R0^T)^{-1} R0 r to the Schwarz sweeps; at most
                                8192 coarse unknowns per pair and 74 coarse nodes across (FP64: 51)
                                [0: one-level] */
    double rho;              /* K_rho integration scale of the data term (Section 1: the matrix A_rho and
                                vector F), 0 <= rho <= 16 [0: A = g g^T, F = -ft g per element]: each
                                product g_c g_d and -ft g_c is smoothed over the lattice of its triangle
                                family (t = 0 and t = 1 separately) by the sampled Gaussian of sigma's
                                form, normalised inside the lattice.  The operator uses A_rho exactly; the
                                Schwarz (and coarse) preconditioner is built from the unsmoothed g g^T */
    int schwarz;             /* method of of_solve [0]:
                                0: PCG preconditioned by the symmetric restricted overlapping Schwarz
                                   method (the options above);
                                1: the paper's Schwarz method as a stationary iteration (Section 3.2,
                                   Eq. schwarz): each subdomain solves its extended problem with Dirichlet
                                   data from the previous global iterate outside it, and every node takes the
                                   value of the subdomain that owns it (restricted additive Schwarz),
                                     U^k = U^{k-1} + sum_i R~_i^T A_i^{-1} R_i (b - A U^{k-1}),
                                   with A_i^{-1} approximated by `sweeps` (here up to 4096) symmetric block
                                   SOR sweeps from zero (exact as the sweeps grow).  of_solve iterates until
                                   ||b - A U|| <= rtol ||b|| or max_inner iterations; inner_iters counts the
                                   iterations and of_get_schwarz_history gives ||U^k - U^{k-1}||_2 of each.
                                   Needs the Schwarz preconditioner settings, coarse = 0 and rho = 0 */
    double lambda_min;       /* 0: lambda constant, as the paper keeps it (Section 2.3) [0]; > 0: lambda per
                                element (Section 1: Lambda piecewise constant), initialised to `lambda`, set by
                                of_set_lambda, and adapted by of_adapt_alpha with the rule of alpha (the same
                                eta_K) and this threshold (<= lambda).  The operator, the residual and the
                                indicator use the per-element lambda (Lambda_e = max of the two sides); the
                                Schwarz preconditioner keeps the constant `lambda`; needs rho = 0; the
                                adaptation-pass VJP is not provided with it */
    int half_sweeps;         /* mixed path, PCG: local sweeps of the Schwarz preconditioner in packed FP16
                                arithmetic, two nodes per instruction [0]: 0 = wherever the tile allows
                                (sweeps >= 1, extended tile height 2 HP with HP a multiple of 3, at most
                                384 node pairs per colour), 1 = required (OF_ERR_ARG where not allowed),
                                -1 = FP32 sweeps.  The right-hand side of each local solve is scaled by its
                                first Jacobi step's largest entry, the diagonal blocks and the residual
                                update stay FP32, and r.z is formed in FP32 */
} of_grid_opts;

/* Solve options.  A field left at 0 takes the default in brackets. */
typedef struct {
    double rtol;       /* stop when ||b - A U||_2 <= rtol ||b||_2 [1e-6]; the residual is formed in
                          FP64 (FP64 path) or double-float arithmetic (mixed path, ~48 bits) */
    int max_outer;     /* refinement passes (mixed) [20] */
    int max_inner;     /* PCG iterations per pass (mixed) or in total (FP64) [2000] */
    int warm_start;    /* 1: start from the U passed in; 0: start from U = 0 */
    double inner_rtol; /* mixed: a pass asks the inner PCG to bring its starting residual down to
                          pass_frac times the outer tolerance, but by no more than this factor
                          [5e-7] */
    int host_loop;     /* 1: drive the inner PCG loop from the host (launch by launch, polling
                          convergence); 0: one CUDA graph per pass whose while-node the device
                          ends [0] */
    double pass_frac;  /* mixed: the fraction of the outer tolerance a refinement pass aims at, in
                          (0, 1] [0.5]; a smaller fraction leaves the final residual further below
                          rtol, which bounds the flow error more tightly at the cost of iterations */
} of_solve_opts;

/* Per-pair result of of_solve / of_adjoint (host memory, written on return). */
typedef struct {
    int status;           /* of_status of this pair */
    int outer_iters;      /* FP64 residual evaluations after the first */
    int inner_iters;      /* PCG iterations in total */
    double rel_residual;  /* final ||b - A U||_2 / ||b||_2, FP64, from the device */
    float ms;             /* device time of the whole call (same for every pair) */
} of_solve_info;

/* Creates a handle bound to `device` and `cuda_stream` (a cudaStream_t, may
 * be NULL for the legacy default stream).  *h receives the handle. */
of_status of_create(of_handle *h, int device, void *cuda_stream);

/* Declares a batch of `batch` frame pairs, pair p of W[p] x H[p] nodes
 * (W, H >= 2; host arrays), and allocates the device workspace for them.
 * Frames, alpha and solutions of earlier setups are discarded.  Returns
 * OF_ERR_ARG for bad sizes or options (the earlier setup then stays as it
 * was), OF_ERR_OOM if the workspace does not fit (the handle then holds no
 * grid: later calls return OF_ERR_STATE until a setup succeeds). */
of_status of_setup_grid(of_handle h, int batch, const int32_t *W, const int32_t *H, const of_grid_opts *o);

/* Copies the two frames of pair `pair` ([H][pitch], dtype dt, pitch >=
 * W) into the workspace, converting to the storage precision (FP32 for
 * OF_PREC_MIXED, FP64 for OF_PREC_FP64), and smooths them with K_sigma when
 * the grid options give sigma > 0: the stored frames are f = K_sigma * I of
 * Section 1. */
of_status of_set_frames(of_handle h, int pair, const void *f1, const void *f2, of_dtype dt, int64_t row_pitch_elems);

/* Copies the stored (smoothed) frames f(., t), f(., t+1) of pair `pair` out
 * as dense [H][W] arrays of dtype dt (host or device).  Returns OF_ERR_STATE
 * before of_set_frames. */
of_status of_get_frames(of_handle h, int pair, void *f1, void *f2, of_dtype dt);

/* Copies the element data of pair `pair` out as 18 dense [H-1][W-1] planes
 * (dtype dt, host or device): plane t * 9 + k holds, for triangle family t,
 * the entries 00, 01, 02, 11, 12, 22 of A_rho (k = 0..5) and F (k = 6..8).
 * Returns OF_ERR_STATE when rho = 0 (no element data is stored) or before
 * of_set_frames. */
of_status of_get_element_data(of_handle h, int pair, void *out, of_dtype dt);

/* Sets the per-element alpha of pair `pair` from `alpha` ([H-1][W-1][2],
 * dtype dt), or, if alpha is NULL, to the constant alpha_const (> 0). */
of_status of_set_alpha(of_handle h, int pair, const void *alpha, double alpha_const, of_dtype dt);

/* Copies the current per-element alpha of a pair out ([H-1][W-1][2]). */
of_status of_get_alpha(of_handle h, int pair, void *alpha, of_dtype dt);

/* Per-element lambda (grid option lambda_min > 0, Section 1): sets that of
 * pair `pair` from `lam` ([H-1][W-1][2], dtype dt) or, if lam is NULL, to the
 * constant lam_const (> 0); of_get_lambda copies it out.  OF_ERR_STATE on a
 * grid with a constant lambda. */
of_status of_set_lambda(of_handle h, int pair, const void *lam, double lam_const, of_dtype dt);
of_status of_get_lambda(of_handle h, int pair, void *lam, of_dtype dt);

/* Solves A U = b for every pair (Section 2.2, Eq. discret-form): PCG with
 * the overlapping Schwarz preconditioner of Section 3.2 (Eq. schwarz, one
 * subdomain per CTA), in FP64 or in FP32 with FP64 iterative refinement.
 * U[p] ([3][H][W], dtype dt) receives the solution; with warm_start it is
 * also the initial guess.  info (host, `batch` entries, may be NULL)
 * receives per-pair results.  Synchronises the stream.  Returns the worst
 * per-pair status (OF_ERR_NOT_CONVERGED / OF_ERR_BREAKDOWN) or OF_OK. */
of_status of_solve(of_handle h, const of_solve_opts *o, void *const *U, of_dtype dt, of_solve_info *info);

/* ||U^k - U^{k-1}||_2 of every iteration of the last of_solve of pair
 * `pair` on a grid with schwarz = 1 (Section 3.2, Eq. schwarz), into hist
 * (host, at least `cap` entries; the first min(cap, n) are written); *n
 * receives the number of iterations.  OF_ERR_STATE if the last of_solve was
 * not such a solve. */
of_status of_get_schwarz_history(of_handle h, int pair, double *hist, int cap, int *n);

/* Error indicator eta_K of Section 2.3 (Eq. errind) for the last solution
 * of every pair, then the alpha update of Section 2.3:
 *   alpha_K <- max(alpha_K / (1 + kappa max(eta_K / ||eta||_inf - eta_thr, 0)), alpha_th)
 * (no change for a pair whose eta is identically 0).  Requires a previous
 * of_solve.  eta (optional, per pair [H-1][W-1][2], dtype dt, may be NULL)
 * receives eta_K before the update. */
of_status of_adapt_alpha(of_handle h, double kappa, double eta_thr, double alpha_th, void *const *eta, of_dtype dt);

/* Vector-jacobian product of one adaptation pass (Section 2.3): the map
 * (alpha, U, f1, f2) -> alpha_new = update(alpha, eta(U, alpha, f)) of
 * of_adapt_alpha, linearised at the current alpha and the solution of the
 * last of_solve (which must belong to it; alpha is not changed).  Given
 * dLdalpha_new[p] ([H-1][W-1][2]) it writes dLdalpha[p] (same shape, the
 * part through the update and the indicator), dLdU[p] ([3][H][W]) and, if
 * not NULL, dLdf2[p], dLdf1[p] ([H][W]; w.r.t. the images given to
 * of_set_frames when sigma > 0).  The flat branches of the update pass
 * nothing, max(eta) passes its derivative to the first element attaining
 * it, and Lambda_e = max of the two sides of an edge passes half to each
 * at a tie.  Chained with of_adjoint (dL/dU of the pass as its input), this
 * differentiates a loss through any number of passes from per-pass
 * checkpoints of alpha and U.  With rho > 0 the indicator's interior
 * residual is F - A_rho U_h, and its frame derivatives go back through the
 * element data (K_rho^T, then the products), as in of_adjoint.  Device
 * arrays only.  Synchronises the stream. */
of_status of_adapt_alpha_vjp(of_handle h, double kappa, double eta_thr, double alpha_th,
                             void *const *dLdalpha_new, void *const *dLdalpha, void *const *dLdU,
                             void *const *dLdf2, void *const *dLdf1, of_dtype dt);

/* Gradients of a scalar loss L(U) through the solve (implicit
 * differentiation of A(theta) U = b(theta)): solves A Lam = dL/dU (A is
 * symmetric, so the adjoint system is the same operator) with the options
 * of the last of_solve, then forms per element
 *   dL/dalpha_K = -|K| sum_{c=u1,u2} grad Lam_c . grad U_c
 * and, through g_K and ft_K, dL/df2 and dL/df1 at the nodes (with rho > 0
 * through the K_rho element tensors: dE/dA_rho and dE/dF per element, K_rho
 * transposed, then the products back to g_K and ft_K; with sigma > 0 the
 * frame gradients are w.r.t. the images given to of_set_frames).  dLdU[p] is
 * [3][H][W]; dLdalpha[p] is [H-1][W-1][2]; dLdf2[p], dLdf1[p] are [H][W]
 * (row pitch W); any output array list may be NULL.  Requires a previous
 * of_solve (its U is the linearisation point).  Synchronises the stream. */
of_status of_adjoint(of_handle h, void *const *dLdU, void *const *dLdalpha, void *const *dLdf2,
                     void *const *dLdf1, of_dtype dt, of_solve_info *info);

/* q = A p for one pair with the operator of Section 2.2 applied matrix-free
 * (p, q: [3][H][W], dtype dt; FP64 handles apply in FP64, mixed handles in
 * FP32).  The load vector b of the same system is written to b if b is not
 * NULL. */
of_status of_apply(of_handle h, int pair, const void *p, void *q, void *b, of_dtype dt);

/* z = M^{-1} r with the Schwarz preconditioner of the handle (symmetric
 * restricted overlapping Schwarz, Section 3.2, local solves by symmetric
 * block Gauss-Seidel sweeps) for one pair; r, z: [3][H][W]. */
of_status of_precondition(of_handle h, int pair, const void *r, void *z, of_dtype dt);

/* FP64 relative residual ||b - A U||_2 / ||b||_2 of a pair for a given U
 * ([3][H][W], dtype dt), computed on the device in FP64.  Synchronises. */
of_status of_residual(of_handle h, int pair, const void *U, of_dtype dt, double *rel_residual);

/* Kernel counts and timing of the solve path, for measurement.  Every kernel
 * launch of of_solve / of_adjoint / of_adapt_alpha is counted (inside the
 * inner-loop CUDA graph, from the iteration count); with profiling on, the
 * inner loop is launched kernel by kernel instead of as the graph and the
 * launches of the three solve kernels are bracketed by CUDA events on the
 * handle's stream.  Totals accumulate until read.  Index 0: PCG apply (p, d,
 * q and p.q), 1: Schwarz preconditioner (r, z, r.r, r.z), 2: FP64 residual /
 * refinement, 3: every other kernel (copies, element records, indicator,
 * alpha update, adjoint gradients; counted, not timed). */
typedef struct {
    int launches[4];
    double ms[4];
} of_profile;

/* Turns kernel timing on (1) or off (0); either call clears the totals. */
of_status of_set_profiling(of_handle h, int on);

/* Copies the accumulated totals out and clears them. */
of_status of_get_profile(of_handle h, of_profile *out);

/* FP64 residual r = b - A U of one frame pair without a handle and without
 * any device allocation.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory (a frame-budgeted render or
 * capture loop where allocator calls may synchronise or fail, a plug-in whose
 * host application owns every allocation).  The caller passes every input and
 * output; the library's only scratch is a fixed static device array of
 * 512 KB (block partial sums and an arrival counter) that every GPU which
 * loads the library holds until the process exits.
 *   f1, f2 [H][W], alpha [H-1][W-1][2], U [3][H][W]: FP64 device arrays;
 *   r (optional, NULL = not written) [3][H][W] FP64 device array;
 *   norms: FP64 device array of 3: ||b - A U||/||b||, ||b - A U||^2, ||b||^2.
 * Limit: ceil(W/124) * ceil(H/32) <= 32768 thread blocks (every frame up to
 * 8192 x 8192 nodes fits); larger frames return OF_ERR_ARG, as do bad sizes
 * or null inputs.  The first call on a device (the current one) looks up the
 * device address of the scratch array, and so does the first call after a
 * reset of that device (a new context); make those calls before any stream
 * capture.  All calls share the scratch and it keeps the last call's
 * contents (the counter that must start at zero is cleared by every call):
 * calls that overlap on the GPU (other streams, other host threads) race.
 * Work is enqueued on cuda_stream (NULL: legacy default stream); the outputs
 * are valid once the stream has passed the call. */
of_status of_residual_noalloc(int W, int H, const double *f1, const double *f2, const double *alpha,
                              double lambda, const double *U, double *r, double *norms, void *cuda_stream);

/* Upper bound of every device wait (the preconditioner's TMA staging
 * barriers), in SM clock cycles [4e9, about 2 s].  A wait that runs out sets a
 * device error word; the kernel stops staging, still completes, and the call
 * returns OF_ERR_TIMEOUT with the handle usable.  cycles <= 0 restores the
 * default. */
of_status of_set_wait_limit(of_handle h, int64_t cycles);

/* Test hook for that failure path; no counterpart in the paper.  With
 * extra_bytes > 0 (a multiple of 16, at most 4096) every staging barrier of
 * the preconditioner expects that many bytes more than its copies deliver:
 * the copies complete, the barrier never does, and each wait runs out after
 * the wait limit.  0 turns it off. */
of_status of_debug_starve_staging(of_handle h, int extra_bytes);

/* Test hook for the allocation failure path; no counterpart in the paper.
 * With bytes > 0 the handle's device allocations fail (as out of memory)
 * once they would hold more than `bytes` in all, so that OF_ERR_OOM can be
 * provoked without exhausting the GPU.  0 removes the limit.  OF_ERR_ARG for
 * bytes < 0. */
of_status of_set_alloc_limit(of_handle h, int64_t bytes);

/* Releases the workspace and the handle (NULL is accepted). */
of_status of_destroy(of_handle h);

/* Message for the last non-OK status of h (or of a failed of_create when h
 * is NULL); never NULL. */
const char *of_last_error(of_handle h);

#ifdef __cplusplus
}
#endif
#endif /* OF_H_ */
