// internal.cuh -- shared declarations of libprosper's CUDA translation units.
// Nothing here is part of the public C ABI (include/prosper.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/prosper.h"

namespace prosper {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);

// Raise `func`'s dynamic shared-memory limit on the CURRENT device to at least
// `bytes`.  cudaFuncSetAttribute applies to one device only, so the value set
// is remembered per (device, kernel) under a lock; every launcher that needs
// more than 48 KB calls this before each launch (a map lookup when nothing
// changes).  Returns PROSPER_OK or PROSPER_ECUDA (with set_error).
int ensure_smem_attr(const void *func, size_t bytes);

// |K| = sum_{k <= gamma} C(Hp, k) m^k: states with at most gamma nonzero units
// among Hp candidates, each taking one of m values (m = 1: binary latents).
int num_states(int Hp, int gamma, int m = 1);

// the linear-superposition models (BSC, TSC, DSC) share the projection,
// preselection and sum y<s>^T kernels
inline bool linear_model(int model) {
    return model == PROSPER_BSC || model == PROSPER_TSC || model == PROSPER_DSC;
}
// the max-superposition models (MCA, MMCA) share the MCA kernels
inline bool max_model(int model) { return model == PROSPER_MCA || model == PROSPER_MMCA; }

#define PROSPER_CUDA_TRY(expr)                                                     \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            ::prosper::set_error("%s failed: %s (%s:%d)", #expr,                   \
                                 cudaGetErrorString(_e), __FILE__, __LINE__);      \
            return PROSPER_ECUDA;                                                  \
        }                                                                          \
    } while (0)

#define PROSPER_LAUNCH_CHECK()                                                     \
    do {                                                                           \
        cudaError_t _e = cudaGetLastError();                                       \
        if (_e != cudaSuccess) {                                                   \
            ::prosper::set_error("kernel launch failed: %s (%s:%d)",               \
                                 cudaGetErrorString(_e), __FILE__, __LINE__);      \
            return PROSPER_ECUDA;                                                  \
        }                                                                          \
    } while (0)

// Per-point scratch rows are padded to this many entries (Hprime <= 16).
constexpr int SEL_STRIDE = 16;
// Hprime range of the register-resident BSC state kernel (k_bsc_states); above
// it BSC uses the table-driven kernel of dsc.cu.
constexpr int BSC_REG_MAX_HPRIME = 10;

// Status word bits written by kernels (ctx->d_status).
constexpr unsigned ST_NONFINITE = 1u;     // a data point had a non-finite y^T y
constexpr unsigned ST_TC_TIMEOUT = 2u;    // a bounded pipeline wait (mbarrier) gave up
constexpr unsigned ST_CHOL_FAIL = 4u;     // M-step matrix not positive definite

struct ServeState;  // serve.cu
struct TraceState;  // api.cu

// Kernel tracing (prosper_trace_enable): CUDA events recorded around every
// kernel launch on the launching stream.  TraceScope is a no-op when off.
struct TraceScope {
    prosper_ctx *c;
    cudaStream_t s;
    bool on;
    size_t idx;   // this scope's record
    TraceScope(prosper_ctx *ctx, const char *name, cudaStream_t stream, int kernels = 1);
    ~TraceScope();
};

}  // namespace prosper

struct prosper_ctx {
    int model, D, H, Hp, gamma, precision;
    int nK;                 // |K| = sum_{k<=gamma} C(Hp, k)
    int64_t chunk;          // points per internal piece (scratch capacity)
    int device, num_sms;

    // per-iteration constants (rebuilt from W by every estep/encode call)
    float *G = nullptr;       // H x H Gram matrix W^T W (FP32)
    float *rnorm = nullptr;   // H: 1/||W_h|| (0 for a zero row)
    float *Wd = nullptr;      // D x H: W in the paper's layout (FP32 SIMT projection operand)
    uint16_t *Wb = nullptr;   // BF16 copy of W in the tcgen05 shared-memory image layout
    float *mca_logW = nullptr;  // MCA: H x D log W_dh
    float *gsc_tab = nullptr;   // GSC: per active subset {logdet, M_b^-1 packed} (8 floats)
    int gsc_nsub = 0;
    void *dsc_tab = nullptr;    // table-driven state kernel: nK packed states (uint2 each)
    int dsc_m = 1;              // nonzero latent values: 1 (binary), 2 (TSC), 1..3 (DSC)
    float dsc_vals[3] = {1.f, 0.f, 0.f};   // the nonzero values phi_1 .. phi_m
    int score_mode = 0;         // preselection score: 0 signed, 1 magnitude, 2 negated

    // ET data-point cut (prosper_set_data_cut)
    int cut = 0;                // 1: statistics from the N_cut best-explained points
    float *cut_logz = nullptr;  // per-point log Z of the first pass (cut_cap floats)
    int64_t cut_cap = 0;
    unsigned *cut_hist = nullptr;     // 2 x 65536 radix-select histograms
    long long *cut_state = nullptr;   // N_cut, upper bin, count above it
    float *cut_thr = nullptr;         // the N_cut-th largest log Z
    int64_t cut_n0 = 0;         // first point of the E-step piece being launched

    // per-piece scratch
    int32_t *sel = nullptr;   // chunk x SEL_STRIDE selected latents (ascending)
    float *selp = nullptr;    // chunk x SEL_STRIDE FP32 projections of the selected latents
    float *yy = nullptr;      // chunk x 2: y^T y as an unevaluated sum hi + lo
    float *es = nullptr;      // chunk x SEL_STRIDE posterior means <s> of the selected latents
    float *apart = nullptr;   // num_sms x H x D FP32 partials of sum y<s>^T (tensor-core path)
    int apart_pieces = 0;     // tensor-core launches since the E-step began (partials pending)

    // M-step workspace (FP64)
    double *mB = nullptr;     // Hq x Hq (Hq = H rounded up to 32): B and its trailing updates
    double *mX = nullptr;     // Hq x D: At and its trailing updates
    double *mI = nullptr;     // Hq x Hq: identity and its trailing updates
    double *mP = nullptr;     // Hq x 32: the current panel of the Cholesky factor
    double *mY = nullptr;     // Hq x D: L^-1 At
    double *mZ = nullptr;     // Hq x Hq: L^-1
    double *mW = nullptr;     // H x D: the new W^T in FP64
    double *mpart = nullptr;  // per-CTA partials of tr(W^T A) and tr(W^T W B)

    unsigned *d_status = nullptr;  // device status word (ST_* bits)
    int tc_test_no_commit_ms = 0;  // failure-detection test hook (environment, off by default)
    int astat_simt = 0;            // 1: use the SIMT kernel for sum y<s>^T (PROSPER_ASTAT_SIMT=1)

    // host-staging for prosper_estep_host
    float *h_stage = nullptr;
    float *d_stage = nullptr;
    int64_t stage_points = 0;
    cudaStream_t h_copy = nullptr;            // copy stream of prosper_estep_host
    cudaEvent_t h_copied[3] = {}, h_used[3] = {}, h_start = nullptr;

    prosper::ServeState *serve = nullptr;
    prosper::TraceState *trace = nullptr;
    double *d_hstats = nullptr;   // device statistics of prosper_estep_host
};

namespace prosper {

// ------------------------------------------------------------ launchers
// All launchers return PROSPER_OK or PROSPER_ECUDA (with set_error).
int launch_bsc_prep(prosper_ctx *c, const float *W, cudaStream_t s);
int launch_bsc_proj_f32(prosper_ctx *c, const float *Y, int64_t N, cudaStream_t s);
int launch_bsc_proj_bf16(prosper_ctx *c, const float *Y, const float *W, int64_t N,
                         cudaStream_t s);
size_t bf16_smem_bytes(int D, int H);
int launch_bsc_states(prosper_ctx *c, const double *theta, int64_t N, int64_t n_offset,
                      prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                      float *mapp_out, float *logz_out, cudaStream_t s);
// table-driven warp-per-point state kernel (dsc.cu): TSC, DSC and BSC with Hprime > 10
int dsc_build_table(prosper_ctx *c);
size_t dsc_smem_bytes(int Hp, int m);
int launch_dsc_states(prosper_ctx *c, const double *theta, int64_t N, int64_t n_offset,
                      prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                      float *mapv_out, float *mapp_out, float *logz_out, cudaStream_t s);
// BSC/TSC/DSC: projection + preselection of a piece of n points, then its
// states (k_bsc_states for BSC with Hprime <= 10, else the table kernel)
int launch_linear_proj(prosper_ctx *c, const float *Y, const float *W, int64_t n, cudaStream_t s);
// ET data-point cut (cut.cu): buffers for N points, and the threshold of the
// N_cut-th largest log Z in c->cut_logz[0 .. N) into c->cut_thr
int cut_reserve(prosper_ctx *c, int64_t N);
int launch_cut_select(prosper_ctx *c, const double *theta, int64_t N, cudaStream_t s);
int launch_linear_states(prosper_ctx *c, const double *theta, int64_t N, int64_t n_offset,
                         prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                         float *mapv_out, float *mapp_out, float *logz_out, cudaStream_t s);
int launch_astat(prosper_ctx *c, const float *Y, int64_t N, double *At, cudaStream_t s);
int launch_astat_tc(prosper_ctx *c, const float *Y, int64_t N, cudaStream_t s);
int finish_astat_tc(prosper_ctx *c, double *At, cudaStream_t s);
bool astat_tc_ok(int D, int H);
int launch_symmetrize(prosper_ctx *c, double *B, cudaStream_t s);

int launch_mca_prep(prosper_ctx *c, const float *W, cudaStream_t s);
int launch_mca_estep(prosper_ctx *c, const float *W, const double *theta, const float *Y,
                     int64_t N, prosper_stats *st, int16_t *sel_out, float *smean_out,
                     int16_t *map_out, float *mapp_out, float *logz_out, cudaStream_t s);

int launch_gsc_prep(prosper_ctx *c, const prosper_params *p, cudaStream_t s);
size_t gsc_smem_bytes(int D, int H, int Hp, int nK);   // shared memory of the GSC E-step kernel
int launch_gsc_estep(prosper_ctx *c, const prosper_params *p, const float *Y, int64_t N,
                     prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                     float *mapp_out, float *logz_out, cudaStream_t s);

int mstep_hq(int H);
int mstep_nparts(int H, int D);
int launch_mstep(prosper_ctx *c, const prosper_stats *st, int64_t N, prosper_params *p,
                 cudaStream_t s);

// number of BSC projection-kernel tiles per persistent CTA etc. live in the .cu files

}  // namespace prosper
