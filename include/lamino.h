/*
 * lamino.h - C ABI of the B300 laminography library (liblamino.so).
 *
 * The library computes the Fourier-based laminographic forward operator L,
 * its adjoint, the total-variation pieces and ADMM-TV reconstruction of
 * Ma et al., "mLR: Scalable Laminography Reconstruction based on
 * Memoization" (SC'25): Eq. 1 (objective), Section 2 (operator shapes and
 * Algorithm 1, LSP), Algorithm 2 and Section 4.2 (operation cancellation
 * and the fused subtraction).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Sizes.  n = n1 = n2 (lateral, x and y), nz = n0 (z, the rotation axis),
 *   det_h = h and det_w = w (detector rows and columns), n_theta = T.  Each of
 *   n, nz, h, w must be even, of the form 2^a 3^b 5^c and in [8, 2048], n
 *   also a multiple of 8; 1 <= T <= 65536.
 * Layouts (row-major, last index fastest):
 *   volume u       real      [n][nz][n]   = u[x][z][y]
 *   data d, d_hat  complex   [T][h][w]    = d[theta][v][u]   (interleaved re, im)
 *   gradient field real      [3][n][nz][n] (component 0: x, 1: z, 2: y)
 * Precision.  A plan is created for LAM_F32 (float / float2 arrays) or
 *   LAM_F64 (double / double2 arrays); every array passed to it uses that type.
 * Geometry.  theta[k] is the k-th rotation angle in radians; phi is the beam's
 *   elevation above the sample plane in radians, 0 <= phi < pi/2 (phi = 0 is
 *   tomography about z).  Slice frequencies are
 *     xi = (ku/w) (cos th, sin th, 0) + (kv/h) (sin phi sin th, -sin phi cos th, cos phi),
 *   ku in [-w/2, w/2), kv in [-h/2, h/2); coordinates are centred.
 * Alignment.  Arrays are aligned to their element type (complex arrays to
 *   the complex element: 8 bytes FP32, 16 bytes FP64); a real volume u passed
 *   to a forward call must start on a two-element boundary (8 / 16 bytes), or
 *   the call returns LAM_EINVAL.
 * Pointers.  Every array argument is a device pointer owned by the caller
 *   (reconstruct() alone also accepts host pointers).  Nothing on the
 *   operator or ADMM path allocates: scratch comes from the caller's
 *   workspace (lam_workspace_bytes) and ADMM state (admm_state_bytes).
 *   The plan owns only its geometry tables (allocated by lam_plan_create).
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are asynchronous on it; a call returns once its kernels
 *   are enqueued.
 * Errors.  Every call returns LAM_OK or a negative lam_status; arguments are
 *   checked on the host before anything is enqueued (a failed check enqueues
 *   nothing).  lam_last_error() gives a message for the calling thread.
 *   Device-side conditions (non-finite ADMM scalars) set a status word in the
 *   ADMM state that admm_status() reads.  No C++ exception crosses the ABI.
 */
#ifndef LAMINO_H
#define LAMINO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LAM_OK = 0,
    LAM_EINVAL = -1,       /* bad argument (size, pointer, angle, precision) */
    LAM_ENOMEM = -2,       /* plan tables could not be allocated */
    LAM_ECUDA = -3,        /* a CUDA call or kernel launch failed */
    LAM_ETIMEOUT = -4,     /* reserved: a bounded device wait gave up */
    LAM_ENAN = -5,         /* non-finite value in an ADMM reduction */
    LAM_EUNSUPPORTED = -6, /* size or option outside what the kernels support */
    LAM_EBOUNDS = -7       /* an index check of a LAM_BOUNDS_CHECK build failed */
} lam_status;

typedef enum { LAM_F32 = 0, LAM_F64 = 1 } lam_prec;

typedef struct lam_plan lam_plan;

/* Create a plan for one geometry.  oversample must be 2 (the padded grids
 * are 2nz, 2n, 2n); half_width m in [2, 8] sets 2m Gaussian taps per
 * dimension.  theta is a host array of n_theta angles (copied).  The plan
 * uploads its FP64-computed tables (deapodisation, z-gather weights,
 * per-angle slice coordinates, twiddles) to the current device. */
lam_status lam_plan_create(lam_plan** out, int n, int nz, int det_h, int det_w, int n_theta,
                           const double* theta, double phi, int oversample, int half_width,
                           int prec);
lam_status lam_plan_destroy(lam_plan* plan);

/* Plan options (lam_plan_set_option).
 * LAM_OPT_ADJOINT_SPREAD (default LAM_SPREAD_TILES) chooses how the adjoint
 *   spreads slice values onto the padded planes, tile by tile in shared memory:
 *   LAM_SPREAD_TILES   every warp sums into its own tile with plain loads and
 *                      stores (no atomics), tiles added in a fixed order:
 *                      bitwise reproducible run to run; the fastest.
 *   LAM_SPREAD_ATOMIC  floating-point shared-memory atomic adds; rounding
 *                      depends on scheduling (not reproducible bit for bit).
 *   LAM_SPREAD_EXACT   64-bit fixed-point atomic adds: every cell is the exact
 *                      sum of its products rounded to one fixed grid (step
 *                      ~ 2^-61 x a bound on the cell sums, an absolute error
 *                      per product); reproducible.
 *   LAM_SPREAD_HALO    per-warp tiles extended by a halo: each slice point is
 *                      visited once (by the tile of its window origin); the
 *                      halos are summed in a second pass; reproducible.
 *   LAM_SPREAD_TILES_EXACT  the tile spread with 64-bit fixed-point cells
 *                      (as LAM_SPREAD_EXACT, integer read-add-writes instead of
 *                      atomics): exact sums of the rounded products,
 *                      reproducible; the exact centre jobs use it too.
 *   LAM_SPREAD_TILES2  the tile spread with one slice point per half-warp,
 *                      each half-warp summing into a tile of its own (two
 *                      tiles per warp, added in a fixed order): reproducible.
 *   LAM_SPREAD_SWEEP   row sweep: a warp sorts its slice points by the x
 *                      origin of their windows and sweeps a 64 x 8 band of the
 *                      plane with the window rows held in registers (no
 *                      shared-memory read-add-write per tap); the order of
 *                      every sum follows from the input: reproducible.
 * LAM_OPT_FAST_ADJOINT: value != 0 selects LAM_SPREAD_ATOMIC, 0 the default.
 * LAM_OPT_LSP_FORM (default 2) is the LSP form that ADMM states initialised
 *   afterwards use: 2 = Algorithm 2 (operation cancellation: the LSP works on
 *   d_hat = F_2D d with F*_2D / F_2D cancelled, the residual carried by
 *   linearity: one L_hat and one L_hat^H per CG step); 1 = Algorithm 1 (the
 *   plain form: each CG step forms r = L u - d with the full L, applies the
 *   full L^H, and applies L to the direction: two L and one L^H).  Both give
 *   the same iterates up to rounding; the option exists for the comparison.
 * LAM_OPT_Z_THREADS, LAM_OPT_PLANE_FFT_THREADS (256 or 512) are the threads
 *   per block of the z-stage kernels and of the plane row / column FFT
 *   kernels.  The columns, rows or lines per block are picked again to fit;
 *   256 lets two blocks share an SM.  Results do not depend on either.
 * LAM_OPT_RESIDUAL (default LAM_RESID_COMPENSATED for FP32 plans, 0 for FP64)
 *   is how ADMM states initialised afterwards keep the Algorithm 2 residual
 *   r = L_hat u - d_hat, a combination of:
 *   LAM_RESID_REFRESH      evaluate r afresh (one extra L_hat with the fused
 *                          subtraction) at the start of every LSP instead of
 *                          carrying it across LSPs by linearity;
 *   LAM_RESID_COMPENSATED  carry the updates r += gamma L_hat p in a
 *                          compensated (hi + lo) pair (FP32 states hold the lo
 *                          part; FP64 states ignore this bit).
 *   Batched ADMM accepts LAM_RESID_COMPENSATED only.
 * LAM_OPT_EXACT_CENTRE_JOBS (value >= 0; default 3 for FP32 plans, the planes
 *   with |kv - h/2| <= 2, and 0 for FP64) is the number of plane jobs nearest
 *   the centre plane kv = h/2 (the paired adjoint treats planes kv and h - kv
 *   as one job, centre first) whose tile spread (LAM_SPREAD_TILES) accumulates
 *   in exact fixed point (as LAM_SPREAD_TILES_EXACT) instead of FP32.  Near the
 *   centre every slice line passes close to the origin, so the cells there sum
 *   thousands of nearly equal products, which FP32 running sums round
 *   systematically; these few jobs carry most of the energy of L^H applied to
 *   smooth data.  0 = none.
 * LAM_OPT_MEMO_TAU (default 0: off; else tau * 10000 in [1, 9999]) makes ADMM
 *   states initialised afterwards (Algorithm 2 form; size them with
 *   admm_state_bytes after setting it) memoize F*_u2D per plane job
 *   (Sections 4.1, 4.4, 4.5): each job has a one-item cache of (key, value),
 *   key = K = min(1024, T w) slice values per plane at fixed pseudo-random
 *   positions, value = the job's u1 plane.  When the cosine similarity
 *   (Eq. cs) of this call's key and the cached key exceeds tau, the job's
 *   spread and inverse plane FFTs are skipped and its plane is the cached one
 *   times <key, cached key> / |cached key|^2 (F*_u2D is linear); otherwise the
 *   computed plane and its key replace the item.  An approximation: results
 *   depend on tau.  Scalars LAM_SC_MEMO_HITS / LAM_SC_MEMO_LOOKUPS count jobs.
 * Setting an option invalidates ADMM graphs captured with the plan. */
enum {
    LAM_OPT_FAST_ADJOINT = 1,
    LAM_OPT_ADJOINT_SPREAD = 2,
    LAM_OPT_LSP_FORM = 3,
    LAM_OPT_Z_THREADS = 4,
    LAM_OPT_PLANE_FFT_THREADS = 5,
    LAM_OPT_RESIDUAL = 6,
    LAM_OPT_EXACT_CENTRE_JOBS = 7,
    LAM_OPT_MEMO_TAU = 8
};
enum { LAM_RESID_REFRESH = 1, LAM_RESID_COMPENSATED = 2 };
enum {
    LAM_SPREAD_TILES = 0,
    LAM_SPREAD_ATOMIC = 1,
    LAM_SPREAD_EXACT = 2,
    LAM_SPREAD_HALO = 3,
    LAM_SPREAD_TILES_EXACT = 4,
    LAM_SPREAD_TILES2 = 5,
    LAM_SPREAD_SWEEP = 6
};
lam_status lam_plan_set_option(lam_plan* plan, int option, int value);

/* Autotuner (a set-up call; synchronises `stream`, not under capture): times
 * L_hat + L_hat^H (mean of `reps` after one warm-up) for candidate launch
 * shapes by coordinate descent: gather tile side (16 / 32 / 64, dividing
 * 2n), rows and columns per plane-FFT block and columns per z-stage block
 * (the plan's choice and its halvings), keeping the fastest in the plan.
 * u, d_hat: device buffers of the plan's volume and data shapes (scratch,
 * overwritten); ws: the workspace.  *seconds (if not NULL) receives the best
 * pair time.  Results do not depend on the shapes.  ADMM graphs captured with
 * the plan are invalidated.  Batches read the shapes at lam_batch_create. */
lam_status lam_plan_autotune(lam_plan* plan, void* u, void* d_hat, void* ws, int reps, double* seconds,
                             void* stream);

/* Index checks.  A library built with LAM_BOUNDS_CHECK defined checks the
 * table- and geometry-derived indices of the z-stage transpose (each cell's
 * kv range against its weight row), the 2D gather (the tap window against the
 * staged tile, the output index) and the 2D spread (the input index) before
 * each access.  An index out of range skips that access and records the
 * first failing site in the plan's device error word: nothing traps and
 * nothing is accessed out of range.  Other builds compile the checks away.
 * lam_plan_status reads the word (synchronises `stream`): LAM_OK, or
 * LAM_EBOUNDS with the site named in lam_last_error(); it clears the word.
 * lam_bounds_checked() is 1 in a LAM_BOUNDS_CHECK build, 0 otherwise. */
lam_status lam_plan_status(const lam_plan* plan, void* stream);
int lam_bounds_checked(void);

/* Bytes of device scratch the operator calls need (ws argument).  The
 * workspace holds the z-transformed volume u1[h][n][n] (complex) and a batch
 * of padded planes.  Alignment: 256 bytes. */
size_t lam_workspace_bytes(const lam_plan* plan);

/* Bytes of the workspace prefix that lam_forward_hat, lam_adjoint_hat,
 * lam_forward and tv_smooth use (everything but the data-space buffer that
 * lam_adjoint and the Algorithm 1 ADMM form need at the end).  A buffer of
 * this size serves those calls; the others need lam_workspace_bytes. */
size_t lam_workspace_bytes_hat(const lam_plan* plan);

/* L (Section 2, Algorithm 1 forward pass: F*_2D F_u2D F_u1D):
 *   d[th][v][u] = 1/(h w) sum_{kv,ku} u^(xi(th,kv,ku)) exp(+2 pi i (ku s/w + kv t/h)),
 * u^ evaluated by the Gaussian USFFT (oversampling 2, half-width m).
 * u: real [n][nz][n] (read); d: complex [T][h][w] (written). */
lam_status lam_forward(const lam_plan* plan, const void* u, void* d, void* ws, void* stream);

/* Re L^H (the transpose of lam_forward under Re<.,.>; F*_u1D F*_u2D F_2D/(hw)).
 * d: complex [T][h][w] (read); u: real [n][nz][n] (written). */
lam_status lam_adjoint(const lam_plan* plan, const void* d, void* u, void* ws, void* stream);

/* L-hat = F_u2D F_u1D (Algorithm 2 forward pass, no F*_2D).  If sub is not
 * NULL the output is L-hat u - sub (the subtraction fused into F_u2D,
 * Section 4.2).  u real [n][nz][n]; d_hat, sub complex [T][h][w]. */
lam_status lam_forward_hat(const lam_plan* plan, const void* u, void* d_hat, const void* sub,
                           void* ws, void* stream);

/* Re L-hat^H = Re F*_u1D F*_u2D (Algorithm 2 adjoint pass, no F_2D).
 * d_hat complex [T][h][w] (read); u real [n][nz][n] (written). */
lam_status lam_adjoint_hat(const lam_plan* plan, const void* d_hat, void* u, void* ws, void* stream);

/* FBP-style single-pass reconstruction: L^H of ramp-filtered data,
 *   u = Re L_hat^H (W . F_2D d),  W(ku) = pi cos(phi) |ku| / (T w^2 h),
 * with |ku| read as 1/4 at ku = 0.  W is the inverse density of the slice
 * points in frequency space: in the plane xi_z = (kv/h) cos(phi) the T lines
 * of plane kv lie tangent to the circle of radius |kv| sin(phi)/h, which makes
 * the density T w h / (pi cos(phi) |ku|/w) per unit volume; so L_hat^H W L_hat
 * approximates the identity on band-limited volumes outside the missing cone
 * (frequencies within phi of the z axis, which no slice reaches).  Not part of
 * the paper's method (which is iterative); a one-pass baseline.
 * d: complex [T][h][w] (read); u: real [n][nz][n] (written); ws: the full
 * workspace (lam_workspace_bytes: the filtered spectrum uses its data-space
 * buffer). */
lam_status lam_fbp(const lam_plan* plan, const void* d, void* u, void* ws, void* stream);

/* Per-angle centred 2D DFT on the h x w grid (Section 4.2):
 *   inverse = 0: F_2D, out = sum in exp(-2 pi i (ku s/w + kv t/h))   (unnormalised)
 *   inverse = 1: F*_2D, out = 1/(h w) sum in exp(+2 pi i (...))
 * in, out complex [T][h][w]; in == out is allowed. */
lam_status lam_fft2d(const lam_plan* plan, const void* in, void* out, int inverse, void* stream);

/* Forward-difference gradient with a zero difference at the last index.
 * u real [n][nz][n] (read); g real [3][n][nz][n] (written). */
lam_status tv_grad(const lam_plan* plan, const void* u, void* g, void* stream);

/* div = -grad^T (exact negative transpose of tv_grad).
 * g real [3][n][nz][n] (read); u real [n][nz][n] (written). */
lam_status tv_div(const lam_plan* plan, const void* g, void* u, void* stream);

/* Smoothed isotropic TV (the alpha ||u||_TV term of Eq. 1 with |.| replaced
 * by sqrt(|.|^2 + eps^2)), for gradient-based use and autograd:
 *   value = sum_voxels sqrt(|grad u|^2 + eps^2)            (written to *value,
 *           host memory, if value != NULL; synchronises `stream`)
 *   grad  = -div(grad u / sqrt(|grad u|^2 + eps^2))       (if grad != NULL)
 * u real [n][nz][n] (read); grad real [n][nz][n] (written); eps > 0.  Uses
 * the reduction scratch at the end of ws. */
lam_status tv_smooth(const lam_plan* plan, const void* u, double eps, void* grad, double* value, void* ws,
                     void* stream);

/* ---------------------------------------------------------------------------
 * ADMM-TV (Section 2: LSP, RSP, multiplier and penalty updates; LSP in the
 * Algorithm 2 form).  The state is one caller-allocated device buffer; the
 * library lays it out (u, psi, lambda, CG vectors, d_hat, residual, FP64
 * scalars and an iteration history) and never allocates.
 * ------------------------------------------------------------------------- */

/* Scalars readable with admm_read_scalars (indices into the returned array). */
enum {
    LAM_SC_RHO = 0,        /* current penalty rho */
    LAM_SC_ALPHA = 1,      /* TV weight alpha */
    LAM_SC_OBJECTIVE = 2,  /* 1/2 ||L u - d||^2 + alpha TV(u) after the last step */
    LAM_SC_RESID_R = 3,    /* primal residual r = ||grad u - psi|| */
    LAM_SC_RESID_S = 4,    /* dual residual s = rho ||div(psi - psi_old)|| */
    LAM_SC_ITER = 5,       /* outer iterations done */
    LAM_SC_DATA2 = 6,      /* ||L u - d||^2 */
    LAM_SC_TV = 7,         /* TV(u) */
    LAM_SC_STATUS = 8,     /* 0, or LAM_ENAN once a reduction was non-finite */
    LAM_SC_MEMO_HITS = 9,  /* plane jobs served from the memoization cache (LAM_OPT_MEMO_TAU) */
    LAM_SC_MEMO_LOOKUPS = 10, /* plane jobs looked up */
    LAM_NSCALARS = 16
};

/* Bytes of the ADMM state buffer (256-byte aligned pieces). */
lam_status admm_state_bytes(const lam_plan* plan, size_t* bytes);

/* Initialise: u = psi = lambda = 0, rho, alpha, d_hat = F_2D d, residual =
 * -d_hat.  adapt_rho != 0 enables residual balancing (mu = 10, factor 2).
 * d: complex [T][h][w] device array (read).  n_inner >= 1 CG steps per LSP. */
lam_status admm_init(const lam_plan* plan, void* state, const void* d, double alpha, double rho,
                     int n_inner, int adapt_rho, void* ws, void* stream);

/* One outer ADMM iteration: LSP (n_inner CG steps, 1 L-hat and 1 L-hat^H
 * each), RSP shrinkage, multiplier update, residuals, penalty update and the
 * objective.  All scalars stay on the device; no host synchronisation. */
lam_status admm_step(const lam_plan* plan, void* state, void* ws, void* stream);

/* iters outer iterations.  use_graph != 0 captures one iteration into a CUDA
 * graph (on first use for this (state, ws) pair; cached in the plan) and
 * replays it; `stream` must then not be the legacy default stream. */
lam_status admm_run(const lam_plan* plan, void* state, void* ws, int iters, int use_graph,
                    void* stream);

/* Device pointer to the volume u inside the state (real [n][nz][n]). */
void* admm_u(const lam_plan* plan, void* state);

/* Copy LAM_NSCALARS doubles to host memory (synchronises `stream`). */
lam_status admm_read_scalars(const lam_plan* plan, const void* state, double* out, void* stream);

/* Copy the history of the first `count` outer iterations to host memory as
 * [count][4] doubles (objective, rho used, r, s); synchronises `stream`.
 * The history holds up to 4096 iterations. */
lam_status admm_read_history(const lam_plan* plan, const void* state, int count, double* out,
                             void* stream);

/* LAM_OK, or the status word of the state (LAM_ENAN); synchronises. */
lam_status admm_status(const lam_plan* plan, const void* state, void* stream);

/* One-call reconstruction (FP32): iters outer ADMM-TV iterations with 4 CG
 * steps each from real data [n_theta][det_h][det_w] (host or device memory),
 * alpha, rho (adaptive).  Allocates and frees its own plan, workspace and
 * state; u_out (host or device) receives u[n][nz][n].  Synchronous. */
lam_status reconstruct(const float* data, const double* theta, double phi, int n, int nz,
                       int det_h, int det_w, int n_theta, int iters, double alpha, double rho,
                       float* u_out);

/* ---------------------------------------------------------------------------
 * Batches: several reconstructions of uneven sizes run together.  Every
 * plane-stage operator step (z transform, row and column FFTs, gather,
 * spread) is one persistent launch over a work list that concatenates all
 * problems' blocks, instead of one launch per problem (Section 4.2's
 * batching of the per-chunk work, across problems).
 * ------------------------------------------------------------------------- */
typedef struct lam_batch lam_batch;

/* Binds up to 32 plans (same precision and half-width, plans on the current
 * device, n a multiple of 16) to their workspaces (ws[i] of
 * lam_workspace_bytes(plans[i]) bytes, holding all of the plan's plane jobs:
 * the default when the padded planes of the h/2 + 1 jobs need at most 8 GiB in
 * FP32, 1 GiB in FP64).  Allocates one small device
 * table; the batch does not own the plans or workspaces, which must outlive
 * it.  The batched adjoint always uses the tile spread (LAM_SPREAD_TILES),
 * with each plan's LAM_OPT_EXACT_CENTRE_JOBS centre jobs spread exactly by
 * launches of their own; the option is read at lam_batch_create. */
lam_status lam_batch_create(lam_batch** out, const lam_plan* const* plans, void* const* ws, int count);
lam_status lam_batch_destroy(lam_batch* batch);

/* L_hat / L_hat^H / L / L^H of every problem i of the batch: u[i] and d[i]
 * as in the single-plan calls (device arrays of plan i's shapes).  Results
 * are bitwise equal to the single-plan calls.  The full L and L^H run F*_2D /
 * F_2D per problem around the batched stages. */
lam_status lam_forward_hat_batched(const lam_batch* batch, const void* const* u, void* const* d_hat, void* stream);
lam_status lam_adjoint_hat_batched(const lam_batch* batch, const void* const* d_hat, void* const* u, void* stream);
lam_status lam_forward_batched(const lam_batch* batch, const void* const* u, void* const* d, void* stream);
lam_status lam_adjoint_batched(const lam_batch* batch, const void* const* d, void* const* u, void* stream);

/* `iters` ADMM outer iterations of every problem: states[i] initialised with
 * admm_init on plan i.  By default the problems run concurrently on side
 * streams (lam_batch_set_streams).  In the persistent mode (streams = 0, all
 * states with the same n_inner, Algorithm 2 form, no memoization or residual
 * refresh) the operators run batched and the elementwise steps per problem
 * in admm_step's order.  Either way each state evolves bitwise as under
 * admm_step.  use_graph != 0 captures
 * one outer iteration of the whole batch as a CUDA graph (re-captured when
 * the states change) and replays it; it needs a non-default stream. */
lam_status admm_run_batched(lam_batch* batch, void* const* states, int iters, int use_graph, void* stream);

/* Concurrent mode of admm_run_batched.  streams = 0: the persistent batched
 * stages above.  streams >= 1 (lam_batch_create sets min(count, 8) unless two
 * problems share a workspace): every problem runs its own
 * outer iteration (admm_step's kernels and options: either LSP form,
 * memoization, residual options) with problem i on the batch's side stream
 * i mod streams; the side streams fork from and join to the caller's stream
 * (one graph with use_graph), so small problems overlap on the GPU.  Each
 * state evolves bitwise as under admm_step.  Creates the side streams and
 * events (released by lam_batch_destroy or the next call); drops a captured
 * graph.  LAM_EINVAL if two problems share a workspace or the current device
 * is not the batch's. */
lam_status lam_batch_set_streams(lam_batch* batch, int streams);

/* Thread-local message for the last non-OK status returned on this thread. */
const char* lam_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LAMINO_H */
