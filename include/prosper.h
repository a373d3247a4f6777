/*
 * prosper.h -- C ABI of libprosper, a GB300 (sm_103a) implementation of the
 * data-parallel E-step of ProSper's truncated-posterior EM (Expectation
 * Truncation) and of the closed-form M-steps around it.
 *
 * Paper: G. Exarchakis et al., "ProSper -- A Python Library for Probabilistic
 * Sparse Coding with Non-Standard Priors and Superpositions" (arXiv 1908.06843).
 *   Eq. 1-2        generative model template p(s|Theta), p(y|s,Theta) = p(y; f(Theta,s))
 *   Table 1        models: BSC (linear, binary), TSC (linear, ternary), DSC (linear,
 *                  discrete), GSC (linear, spike-and-slab), MCA (max)
 *   Sec. 2         EM with truncated posteriors
 *   Sec. 3         BSC_ET(D, H, Hprime, gamma); Model.step; Model.inference -> res["s"], res["p"]
 *
 * Conventions for every entry point
 *   - All array arguments are DEVICE pointers unless a name ends in _host.
 *     The caller allocates and owns them; the library never frees them.
 *   - Dictionaries are stored transposed: W is H x D row-major, row h is the
 *     dictionary element W_h (column h of the paper's D x H matrix).
 *   - Y is N x D row-major FP32.
 *   - Calls are ordered on the given CUDA stream (cudaStream_t passed as
 *     void*; NULL = legacy default stream) and return before the GPU work
 *     finishes unless stated otherwise.  Results are valid after the stream
 *     is synchronised.
 *   - Return value: PROSPER_OK (0) or a negative PROSPER_E* code; the message
 *     of the last failure on the calling thread is prosper_last_error().
 *     No C++ exception crosses this interface.
 *   - A context is not thread-safe: one host thread (or external locking)
 *     per context.  Two contexts may be used concurrently on different streams.
 */
#ifndef PROSPER_H
#define PROSPER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PROSPER_OK         0
#define PROSPER_EINVAL    -1  /* bad argument: sizes, limits, NULL pointer, wrong model fields */
#define PROSPER_ENOMEM    -2  /* device or pinned-host allocation failed */
#define PROSPER_ECUDA     -3  /* a CUDA runtime call or kernel launch failed */
#define PROSPER_ENONFINITE -4 /* non-finite value detected (input data or M-step result) */
#define PROSPER_ETIMEOUT  -5  /* serving: the request did not finish within the wait limit */
#define PROSPER_EBUSY     -6  /* serving: admission refused (request larger than the memory budget) */
#define PROSPER_ESTATE    -7  /* wrong call order (e.g. serve_submit before serve_start) */

/* Models of Table 1 that this library implements. */
#define PROSPER_BSC 0  /* binary sparse coding: linear f = W s, s in {0,1}^H, Bernoulli(pi) prior */
#define PROSPER_MCA 1  /* maximal causes analysis: f_d = max_h W_dh s_h, W >= 0 */
#define PROSPER_GSC 2  /* Gaussian sparse coding: s_h = b_h z_h, b ~ Bernoulli(pi), z_h ~ N(mu_h, psi_h) */
#define PROSPER_TSC 3  /* ternary sparse coding: linear f = W s, s in {-1,0,1}^H, zero-mean categorical
                          prior p(s_h = -1) = p(s_h = 1) = pi/2 */
#define PROSPER_DSC 4  /* discrete sparse coding: linear f = W s, s_h in {0, phi_1 .. phi_m} (m <= 3 values
                          fixed by prosper_init_dsc), categorical prior p(s_h = phi_v) = theta[TH_DSC_P + v] */
#define PROSPER_MMCA 5 /* max-magnitude causes: f_d = W_dh* with h* the active unit of largest |W_dh|
                          (the lower h on a tie), signed W, binary latents, Bernoulli(pi) prior */

/* Precision of the BSC preselection projection W^T y (other models: FP32 only). */
#define PROSPER_FP32          0  /* FP32 SIMT projection; exact top-H' of the FP32 scores */
#define PROSPER_BF16_RESCORE  1  /* BF16 tensor-core (tcgen05) projection of the unit-norm rows
                                    W_h/||W_h|| for the selection only, ranked on the score
                                    rounded to 15 mantissa bits (ties to the lower h); the H'
                                    selected projections are recomputed in FP32 */

/* Limits (prosper_init returns PROSPER_EINVAL outside them).
 *   all models: 0 <= gamma <= Hprime <= H, H <= 256, D <= 1024.
 *   BSC:     1 <= Hprime <= 16, |K| <= 4096 states per point; for Hprime > 10 also
 *            gamma <= 8 (those use the table-driven state kernel).
 *   TSC/DSC: 1 <= Hprime <= 16, gamma <= 8, |K| = sum_{k<=gamma} C(Hprime,k) m^k <= 4096.
 *   MCA/MMCA: 1 <= Hprime <= 16, |K| <= 1024, D <= 256.
 *   GSC:     1 <= Hprime <= 10, gamma <= 3, H <= 32, D <= 256, and the E-step's
 *            shared memory (dictionary, Gram matrix, per-warp slots, about
 *            4 (H D + H^2 + 8 (H D + 32 N_s + 3 H + 8 |K| + 64 + D)) bytes with
 *            N_s = 2 Hprime + Hprime (Hprime + 1)/2) within 227 KB; e.g.
 *            D = 64, H = 32, Hprime = 8, gamma = 3 uses 163 KB.
 * PROSPER_BF16_RESCORE (BSC only) additionally needs D % 64 == 0, D <= 256,
 * H % 64 == 0 and 2 H D + 256 D + 28 KB <= 227 KB (the BF16 dictionary, one
 * operand tile and the candidate buffers stay in shared memory), e.g. D = H = 256. */
#define PROSPER_MAX_HPRIME 16
#define PROSPER_MAX_STATES 4096

/* theta[] layout (device doubles, PROSPER_THETA_LEN of them). */
#define PROSPER_TH_PI    0   /* prior activation probability pi                   */
#define PROSPER_TH_SIGMA 1   /* observation noise standard deviation sigma         */
#define PROSPER_TH_RHO   2   /* MCA: exponent rho of the smoothed max in the M-step */
#define PROSPER_TH_T     3   /* posterior temperature T of deterministic annealing
                                (Sec. 3, LinearAnnealing): every E-step uses
                                q_n(s) ~ p(s, y_n)^(1/T) on K_n and reports
                                log Z_n = T log sum_{s in K_n} p(s, y_n)^(1/T);
                                a value <= 0 is read as T = 1 (no annealing).
                                The M-step does not read or change it. */
#define PROSPER_TH_DSC_P 4   /* DSC: prior probabilities of the m nonzero values, theta[4 .. 4+m-1]
                                (p(s_h = 0) = 1 - their sum); the M-step updates them and sets
                                theta[TH_PI] to their sum.  Other models read 4 doubles only. */
#define PROSPER_THETA_LEN 8

/* scal[] layout of the scalar sufficient statistics (device doubles). */
#define PROSPER_SC_F      0  /* F = sum_n log sum_{s in K_n} p(s, y_n | Theta) (truncated log-likelihood, nats) */
#define PROSPER_SC_S1     1  /* sum_n <|s|>_n  (expected number of active units)                         */
#define PROSPER_SC_YY     2  /* sum_n y_n^T y_n                                                          */
#define PROSPER_SC_N      3  /* number of points accumulated                                             */
#define PROSPER_SC_MCA_R2 4  /* MCA: sum_n <||y_n - f(s)||^2>  (hard max, current W)                     */
#define PROSPER_SC_DSC0   5  /* TSC/DSC: scal[5 + v] = sum_n sum_h <[s_h = phi_{v+1}]> (value counts)    */
#define PROSPER_SC_LEN    8

typedef struct prosper_ctx prosper_ctx;

/* Model parameters Theta (Eq. 1-2).  All device pointers. */
typedef struct {
    float  *W;      /* H x D row-major FP32; read by E-step/encode, overwritten by M-step */
    double *theta;  /* pi, sigma, rho, T (+ DSC value probabilities): see PROSPER_TH_*    */
    float  *mu;     /* GSC: H slab means (NULL for BSC/MCA)                               */
    float  *psi;    /* GSC: H slab variances (NULL for BSC/MCA)                           */
} prosper_params;

/* Sufficient statistics accumulated by prosper_estep (all device, FP64,
 * overwritten -- not accumulated -- by each call). */
typedef struct {
    double *At;    /* H x D: sum_n <s>_n y_n^T, the transpose of A = sum_n y_n <s>_n^T */
    double *B;     /* H x H: sum_n <s s^T>_n (full symmetric matrix)                  */
    double *scal;  /* PROSPER_SC_LEN scalars (layout above)                            */
    double *gsc;   /* GSC: 3H = [sum <b_h>, sum <s_h>, sum <s_h^2>]; NULL otherwise     */
    double *mca;   /* MCA/MMCA: 2 H D = [sum <A_dh> y_dn (H x D), sum <A_dh> (H x D)]; else NULL */
} prosper_stats;

/* Create a context for one model and approximation (Sec. 3: BSC_ET(D, H,
 * Hprime, gamma)).  The context owns the per-iteration constants (Gram matrix
 * W^T W, 1/||W_h||, BF16 dictionary copy, GSC subset tables) and scratch for up
 * to max_points points per call (larger calls are processed in pieces).
 * precision: PROSPER_FP32 or PROSPER_BF16_RESCORE (BSC only).
 * Errors: PROSPER_EINVAL on limits above, PROSPER_ENOMEM, PROSPER_ECUDA. */
int prosper_init(prosper_ctx **out, int model, int D, int H, int Hprime, int gamma,
                 int precision, int64_t max_points);

/* Context for DSC (Table 1, row DSC: linear superposition, discrete latents,
 * categorical prior) with the m (1..3) nonzero latent values values_host[0..m-1]
 * (host array, distinct and nonzero; copied).  The state set holds every pattern
 * of at most gamma nonzero units among the Hprime candidates, each taking one of
 * the m values; the preselection score is sign(phi) W_h^T y/||W_h|| maximised
 * over the values (|W_h^T y|/||W_h|| when the values have both signs).
 * FP32 only; otherwise as prosper_init. */
int prosper_init_dsc(prosper_ctx **out, int D, int H, int Hprime, int gamma, int m,
                     const float *values_host, int64_t max_points);

/* Release the context and everything it allocated.  NULL is accepted. */
int prosper_destroy(prosper_ctx *ctx);

/* Truncated E-step over N points (Sec. 2; Eq. 1-2 with Table 1's model):
 * for each point the top-Hprime latents by the model's selection score are
 * preselected, every binary state with at most gamma active units among them
 * is evaluated, the posterior over that set is normalised, and the
 * sufficient statistics are summed into *out (overwritten).
 * Y: device N x D FP32.  N >= 0 (N = 0 gives zero statistics).
 * Selection scores: BSC W_h^T y/||W_h||; TSC |W_h^T y|/||W_h||; DSC see
 * prosper_init_dsc; MCA sum_d W_dh y_d / sum_d W_dh; MMCA sum_d W_dh y_d /
 * sum_d |W_dh|; GSC the singleton log-joint log p(e_h, y).  Exact score ties
 * go to the lower h. */
int prosper_estep(prosper_ctx *ctx, const prosper_params *p, const float *Y, int64_t N,
                  prosper_stats *out, void *stream);

/* ET's data-point cut (a variant of the truncated E-step from the ET
 * literature the paper builds on; BSC and TSC contexts).  While on, every
 * prosper_estep runs two passes: the first computes each point's
 * log sum_{K_n} p(s, y_n); the statistics (At, B, scal including F and the
 * count scal[PROSPER_SC_N]) are then summed over the points whose FP32 log Z
 * reaches the N_cut-th largest value, N_cut = floor(N P_pi(|s| <= gamma))
 * (at least 1; ties at the threshold are all kept).  prosper_mstep then
 * multiplies the new pi by H pi / E_pi[|s| : |s| <= gamma] at the current pi
 * (the kept points favour few causes); pass it N = scal[PROSPER_SC_N].
 * The first pass allocates one float per point on the first call that needs
 * more room.  Not available with prosper_estep_host.  PROSPER_EINVAL for the
 * other models. */
int prosper_set_data_cut(prosper_ctx *ctx, int on);

/* Closed-form M-step ("Model.step", Sec. 3) from statistics of N points:
 * BSC/TSC/DSC/GSC W = A B^{-1} (FP64, blocked Cholesky of B), pi = sum<|s|>/(N H)
 * (TSC: p(+-1) = pi/2; DSC: theta[TH_DSC_P + v] = scal[SC_DSC0 + v]/(N H)),
 * sigma^2 = (sum y^T y - 2 tr(W^T A) + tr(W^T W B))/(N D) with the new W;
 * GSC also mu_h, psi_h; MCA the rho-smoothed-max update of W (clamped >= 1e-6;
 * MMCA: the same update on |W| without the clamp),
 * pi as BSC, sigma^2 = sum<||y - f||^2>/(N D).  A unit with B_hh <= 1e-9 N
 * keeps its parameters.  Overwrites p->W, p->theta (and mu, psi) on device. */
int prosper_mstep(prosper_ctx *ctx, const prosper_stats *st, int64_t N, prosper_params *p,
                  void *stream);

/* Encoding with fixed Theta ("Model.inference", Sec. 3: res["s"], res["p"]).
 * Per point n (all outputs device, may be NULL to skip):
 *   sel     N x Hprime int16: the preselected latents, ascending
 *   s_mean  N x Hprime float: posterior means <s_h> of those latents
 *   map_idx N x gamma  int16: most probable state in K_n (active latents ascending, -1 padded)
 *   map_p   N float: its approximate posterior probability q_n(MAP)
 *   logZ    N float: log sum_{s in K_n} p(s, y_n | Theta)
 * MAP ties go to the state with fewer active units, then the lexicographically
 * smaller sorted list of local indices. */
int prosper_encode(prosper_ctx *ctx, const prosper_params *p, const float *Y, int64_t N,
                   int16_t *sel, float *s_mean, int16_t *map_idx, float *map_p, float *logZ,
                   void *stream);

/* prosper_encode for the discrete-latent models (TSC, DSC), which also writes
 * map_val (N x gamma float, may be NULL): the value of each unit listed in
 * map_idx (0 where map_idx is -1).  s_mean then holds the signed posterior means
 * <s_h>.  PROSPER_EINVAL for the other models (their MAP units all take the
 * value 1). */
int prosper_encode_values(prosper_ctx *ctx, const prosper_params *p, const float *Y, int64_t N,
                          int16_t *sel, float *s_mean, int16_t *map_idx, float *map_val,
                          float *map_p, float *logZ, void *stream);

/* BSC encoding without any device allocation (the paper has no counterpart:
 * this serves callers that cannot call cudaMalloc when they encode -- code
 * past a fixed start-up phase that must never allocate, a process whose
 * device memory belongs to a framework's caching allocator, or code that must
 * not synchronise the device, which cudaMalloc/cudaFree may do).
 * Same results and output layouts as prosper_encode on a PROSPER_BSC,
 * PROSPER_FP32 context with these D, H, Hprime, gamma, but no context: the
 * scratch lives in a fixed ~1.06 MB device array inside the library that
 * every GPU loading it holds until exit.  Limits: D <= 256, H <= 256,
 * 1 <= Hprime <= 10, gamma <= Hprime, N <= 4096 per call; larger sizes return
 * PROSPER_EINVAL.  W (H x D), theta, Y (N x D) and the outputs are device
 * pointers.  All calls share the array: calls whose GPU work overlaps race,
 * so issue them on one stream.  The first call on each device looks up the
 * array's device address; make it before any stream capture.  Non-finite
 * input is not reported here (there is no context status word): such a point
 * gets a non-finite log Z. */
int prosper_encode_noalloc(int D, int H, int Hprime, int gamma, const float *W,
                           const double *theta, const float *Y, int64_t N, int16_t *sel,
                           float *s_mean, int16_t *map_idx, float *map_p, float *logZ,
                           void *stream);

/* Same E-step as prosper_estep with Y and the statistics in HOST memory:
 * Y_host (N x D) is copied to the device in equal pieces of at most 32,768
 * points, overlapped with the kernels of the previous pieces (page-locked
 * Y_host lets the copies run asynchronously; pageable memory works but the
 * copies then stall the host), the statistics are copied back into host
 * arrays At_host (H x D), B_host (H x H), scal_host (PROSPER_SC_LEN) (each may
 * be NULL), and the call returns after the stream has finished.  p (W, theta,
 * mu, psi) stays on the device. */
int prosper_estep_host(prosper_ctx *ctx, const prosper_params *p, const float *Y_host,
                       int64_t N, double *At_host, double *B_host, double *scal_host,
                       void *stream);

/* Kernel tracing (measurement aid, not part of the method).  While enabled,
 * every kernel the context launches is bracketed by CUDA events recorded on
 * its stream.  prosper_trace_read synchronises the device, writes up to max
 * distinct kernel names (each a NUL-terminated string in a 48-byte slot of
 * names), their summed device time in ms and their launch counts, clears the
 * record, and returns the number of distinct kernels (or a negative error). */
int prosper_trace_enable(prosper_ctx *ctx, int on);
int prosper_trace_read(prosper_ctx *ctx, int max, char *names, double *total_ms, int *launches);

/* Failure detection: synchronise the stream, read and clear the context's
 * device status word and report what the kernels flagged since the last call:
 * PROSPER_ENONFINITE (non-finite y^T y of an input point, or an M-step
 * matrix that is not positive definite), PROSPER_ETIMEOUT (a tensor-core
 * pipeline wait that gave up after its time limit; the kernel then returned
 * without touching its outputs further), else PROSPER_OK. */
int prosper_status(prosper_ctx *ctx, void *stream);

/* Message of the last failure on the calling thread ("" if none). */
const char *prosper_last_error(void);

/* ------------------------------------------------------------------------
 * Encoding service with continuous batching (Sec. 3 "inference" as a
 * service).  A host scheduler thread owned by the context takes submitted
 * requests (1 .. 4096 patches each), packs waiting requests into the next
 * free device slot as soon as one is free (a slot holds up to slot_points
 * points), and runs prosper_encode on that slot's stream; several slots are
 * in flight at once, so requests that arrive while others run are admitted
 * as slots free up and their work overlaps on the device.  W, its Gram
 * matrix and the state tables stay resident.  The per-point results do not
 * depend on which batch or slot a point lands in.
 * ---------------------------------------------------------------------- */

/* Start the service.  n_slots device slots of slot_points points each
 * (memory budget = n_slots * slot_points * (D*4 + per-point outputs) bytes).
 * p is copied (device pointers must stay valid until prosper_serve_stop). */
int prosper_serve_start(prosper_ctx *ctx, const prosper_params *p, int n_slots,
                        int slot_points);

/* Submit n points (host N x D FP32, copied before return).  *ticket receives
 * the request id.  PROSPER_EBUSY if n > slot_points (never admissible). */
int prosper_serve_submit(prosper_ctx *ctx, const float *Y_host, int n, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: forever) for a ticket and copy its results to
 * host arrays (layouts as prosper_encode; each may be NULL).  Returns
 * PROSPER_ETIMEOUT if not finished in time (the ticket stays valid).
 * t_submit_ns / t_done_ns (may be NULL) receive the submit time and the time
 * the scheduler saw the slot's completion, CLOCK_MONOTONIC nanoseconds. */
int prosper_serve_wait(prosper_ctx *ctx, uint64_t ticket, int timeout_ms,
                       int16_t *sel_host, float *s_mean_host, int16_t *map_idx_host,
                       float *map_p_host, float *logZ_host,
                       int64_t *t_submit_ns, int64_t *t_done_ns);

/* Open-loop load generator for measuring the service (a measurement aid, not
 * part of the method).  A submitter thread submits request i (sizes[i] points
 * of the host pool Y_pool_host (pool_points x D), starting at row offsets[i])
 * at arrival_ns[i] nanoseconds after the start, whatever happened to earlier
 * requests; the calling thread polls every outstanding ticket without blocking
 * and copies each finished request's outputs to host memory, as a client
 * would.  Per request (host arrays of n_req): t_submit_ns (just before
 * prosper_serve_submit), t_observed_ns (the client saw the results) and, if
 * t_done_ns is not NULL, the scheduler's completion time; all CLOCK_MONOTONIC.
 * Returns after every request finished, or with the first error. */
int prosper_serve_loadgen(prosper_ctx *ctx, const float *Y_pool_host, int64_t pool_points,
                          int n_req, const int32_t *sizes, const int64_t *offsets,
                          const int64_t *arrival_ns, int64_t *t_submit_ns,
                          int64_t *t_observed_ns, int64_t *t_done_ns);

/* Stop the scheduler thread after the queued work finished; frees the slots. */
int prosper_serve_stop(prosper_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PROSPER_H */
