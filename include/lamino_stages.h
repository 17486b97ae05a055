/*
 * lamino_stages.h - per-stage entry points of liblamino.so, for stage-level
 * parity tests and profiling.  Same conventions as lamino.h; u1 is the
 * z-transformed volume stored plane-major as complex [h][n][n]
 * (u1[kv][x][y]), the layout the plane stage reads.
 */
#ifndef LAMINO_STAGES_H
#define LAMINO_STAGES_H

#include "lamino.h"

#ifdef __cplusplus
extern "C" {
#endif

/* F_u1D (Section 2): u real [n][nz][n] -> u1 complex [h][n][n]. */
lam_status lamx_u1d_fwd(const lam_plan* plan, const void* u, void* u1, void* stream);

/* Re F*_u1D (transpose of lamx_u1d_fwd, real part): u1 -> u. */
lam_status lamx_u1d_adj(const lam_plan* plan, const void* u1, void* u, void* stream);

/* F_u2D (Section 2): u1 complex [h][n][n] -> d_hat complex [T][h][w]; if sub
 * is not NULL the output is F_u2D u1 - sub (Section 4.2's fused
 * subtraction).  Uses the plane part of ws.  Every plane is transformed on
 * its own (u1 need not be the transform of a real volume). */
lam_status lamx_u2d_fwd(const lam_plan* plan, const void* u1, void* d_hat, const void* sub, void* ws,
                        void* stream);

/* F*_u2D (transpose of lamx_u2d_fwd): d_hat -> u1.  Uses the plane part of ws. */
lam_status lamx_u2d_adj(const lam_plan* plan, const void* d_hat, void* u1, void* ws, void* stream);

/* lamx_u2d_fwd without a workspace; it allocates nothing.  (The paper has no
 * counterpart: this serves callers that cannot provide device memory, such
 * as code running inside a device allocator's hooks or a process whose
 * memory is all owned by another pool.)  Same arguments and result as
 * lamx_u2d_fwd minus ws.  The padded planes live in one static 8 MiB device
 * array inside the library, so one padded (2n)^2 plane must fit: n <= 512 in
 * FP32, n <= 256 in FP64; larger plans get LAM_EUNSUPPORTED with nothing
 * launched.  Planes are processed in batches of as many as fit.  The first
 * call on each device looks the array's address up once
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The current device must be the plan's (else LAM_EINVAL).  Nothing in the
 * array needs to start at zero.  There is one array per device, so calls
 * that overlap in time (several streams, threads or plans) race and give
 * wrong results: order them on one stream or synchronise between them. */
lam_status lamx_u2d_fwd_static(const lam_plan* plan, const void* u1, void* d_hat, const void* sub, void* stream);

/* The adjoint spread alone (the first kernel of F*_u2D, the type-1 Gaussian
 * spread of Section 2's F_u2D transpose): the slice values of d_hat
 * ([n_theta][h][w], plan precision) of the Hermitian plane jobs
 * j0 .. j0 + nb - 1 are spread onto the padded planes of the workspace's
 * plane batch, with the plan's spread variant.  Requires
 * 0 <= j0, 1 <= nb, j0 + nb <= the number of plane jobs, and nb <= the
 * planes per batch (LAM_EINVAL otherwise).  For timing the dominant kernel
 * of L_hat^H on its own; the workspace planes are overwritten. */
lam_status lamx_spread(const lam_plan* plan, const void* d_hat, void* ws, int j0, int nb, void* stream);

/* Plane jobs per launch of the L_hat / L_hat^H plane stages (the batch size
 * those calls use); 0 for a NULL plan. */
int lamx_jobs_per_batch(const lam_plan* plan);

/* Data planes (kv rows of d_hat) that plane jobs j0 .. j0 + nb - 1 cover: 2
 * for a job with a conjugate-mirror plane, else 1; -1 for a NULL plan or a
 * range outside the plan's jobs. */
int lamx_job_planes(const lam_plan* plan, int j0, int nb);

/* Launch shapes chosen by the plan, for diagnostics: out[0..count) receives
 * TY (z forward), TY (z transpose), rows per block, columns per block,
 * scatter tile side, tile images, planes per batch, jmin, jmax, the
 * number of plane jobs the full operators run (h/2 + 1 when every plane
 * pairs with its conjugate mirror), the gather tile side, the threads per
 * block of the z stage and of the plane FFTs, and the adjoint spread (its
 * LAM_SPREAD_* value). */
lam_status lamx_plan_info(const lam_plan* plan, int* out, int count);

/* Batch diagnostics: out[2 s], out[2 s + 1] = work items and persistent grid
 * of batched stage s (z forward, row FFT, column FFT, gather, spread, column
 * FFT^H, row FFT^H, z transpose); out[16] = kernel nodes of the captured
 * ADMM graph (0 before the first graph run). */
lam_status lamx_batch_info(const lam_batch* batch, int* out, int count);

/* The forward's plane FFTs alone: planes j0 .. j0 + nb - 1 of u1 (complex
 * [h][n][n]) deapodised, padded to 2n x 2n and transformed (rows, then
 * columns) into P (complex [nb][2n][2n], device).  For timing against
 * library FFTs. */
lam_status lamx_plane_ffts(const lam_plan* plan, const void* u1, void* P, int j0, int nb, void* stream);

/* FP32 FMA throughput of the current device (eight independent FMA chains
 * per thread, 8 blocks of 256 threads per SM; CUDA-event timed, synchronises
 * `stream`): *flops_per_s = 2 x FMAs / s.  sink: a device buffer of
 * sink_floats >= 8 x SM-count floats (never written in practice). */
lam_status lamx_fma_peak(void* sink, int sink_floats, double* flops_per_s, void* stream);

/* Kernel nodes in the CUDA graph admm_run captured for this state (one outer
 * iteration); 0 before the first graph run. */
lam_status lamx_admm_graph_kernels(const lam_plan* plan, void* state, size_t* count);

/* Byte offsets of the pieces of an ADMM state buffer of this plan, in this
 * order (up to `count` of them): FP64 scalars, history, reduction partials,
 * reduction counter, u, du, G_lsp (L_hat^H r), G, G_prev, p, e = grad u - psi
 * [3], lambda [3], dpsi [3], d_hat, r, L_hat p, r_lo, total bytes.  Volumes are
 * real [n][nz][n] of the plan's precision, data arrays complex [T][h][w].
 * For tools that inspect, convert or checkpoint a state; host only. */
lam_status lamx_admm_layout(const lam_plan* plan, size_t* out, int count);

/* Self-test of the index checks (LAM_BOUNDS_CHECK builds; LAM_EUNSUPPORTED
 * otherwise): one checked device write of 1 into element `index` of the
 * plan's 64-int self-test scratch.  An index outside [0, 64) is caught by the
 * check itself (never written), and lam_plan_status then reports LAM_EBOUNDS
 * at the self-test site.  Asynchronous on `stream`. */
lam_status lamx_bounds_selftest(const lam_plan* plan, int index, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LAMINO_STAGES_H */
