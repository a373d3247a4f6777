// api.cu -- the C ABI of include/prosper.h: argument checks, context memory,
// and the order in which the E-step / M-step / encode kernels are issued.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <string>
#include <vector>

namespace prosper {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int ensure_smem_attr(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> done;
    int dev = 0;
    PROSPER_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = done[std::make_pair(dev, func)];
    if (bytes > cur) {
        PROSPER_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        cur = bytes;
    }
    return PROSPER_OK;
}

struct TraceRec {
    const char *name;
    cudaEvent_t a, b;
    int kernels;
};
struct TraceState {
    bool on = false;
    std::vector<TraceRec> recs;
};

TraceScope::TraceScope(prosper_ctx *ctx, const char *name, cudaStream_t stream, int kernels)
    : c(ctx), s(stream), on(ctx && ctx->trace && ctx->trace->on), idx(0) {
    if (!on) return;
    TraceRec r{name, nullptr, nullptr, kernels};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, s);
    idx = c->trace->recs.size();
    c->trace->recs.push_back(r);
}

TraceScope::~TraceScope() {
    if (on) cudaEventRecord(c->trace->recs[idx].b, s);
}

int num_states(int Hp, int gamma, int m) {
    double c = 0.0, b = 1.0, mk = 1.0;
    for (int k = 0; k <= gamma && k <= Hp; ++k) {
        c += b * mk;
        b = b * (Hp - k) / (k + 1);
        mk *= m;
    }
    return (int)(c + 0.5);
}

template <class T>
static int dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return PROSPER_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu bytes) failed: %s", count * sizeof(T), cudaGetErrorString(e));
        cudaGetLastError();
        return PROSPER_ENOMEM;
    }
    return PROSPER_OK;
}

static int check_params(const prosper_ctx *c, const prosper_params *p) {
    if (!p || !p->W || !p->theta) {
        set_error("params: W and theta must be device pointers");
        return PROSPER_EINVAL;
    }
    if (c->model == PROSPER_GSC && (!p->mu || !p->psi)) {
        set_error("params: GSC needs mu and psi");
        return PROSPER_EINVAL;
    }
    return PROSPER_OK;
}

static int check_stats(const prosper_ctx *c, const prosper_stats *st) {
    if (!st || !st->At || !st->B || !st->scal) {
        set_error("stats: At, B and scal must be device pointers");
        return PROSPER_EINVAL;
    }
    if (c->model == PROSPER_GSC && !st->gsc) {
        set_error("stats: GSC needs gsc[3H]");
        return PROSPER_EINVAL;
    }
    if (max_model(c->model) && !st->mca) {
        set_error("stats: MCA needs mca[2HD]");
        return PROSPER_EINVAL;
    }
    return PROSPER_OK;
}

// ---------------------------------------------------------------- E-step
static int estep_begin(prosper_ctx *c, const prosper_params *p, prosper_stats *st,
                       cudaStream_t s) {
    const size_t H = c->H, D = c->D;
    c->apart_pieces = 0;
    PROSPER_CUDA_TRY(cudaMemsetAsync(st->At, 0, sizeof(double) * H * D, s));
    PROSPER_CUDA_TRY(cudaMemsetAsync(st->B, 0, sizeof(double) * H * H, s));
    PROSPER_CUDA_TRY(cudaMemsetAsync(st->scal, 0, sizeof(double) * PROSPER_SC_LEN, s));
    if (c->model == PROSPER_GSC)
        PROSPER_CUDA_TRY(cudaMemsetAsync(st->gsc, 0, sizeof(double) * 3 * H, s));
    if (max_model(c->model))
        PROSPER_CUDA_TRY(cudaMemsetAsync(st->mca, 0, sizeof(double) * 2 * H * D, s));
    if (linear_model(c->model)) return launch_bsc_prep(c, p->W, s);
    if (max_model(c->model)) return launch_mca_prep(c, p->W, s);
    return launch_gsc_prep(c, p, s);
}

static int estep_piece(prosper_ctx *c, const prosper_params *p, const float *Y, int64_t n,
                       prosper_stats *st, cudaStream_t s) {
    int rc;
    if (linear_model(c->model)) {
        rc = launch_linear_proj(c, Y, p->W, n, s);
        if (rc) return rc;
        rc = launch_linear_states(c, p->theta, n, 0, st, nullptr, nullptr, nullptr, nullptr, nullptr,
                                  nullptr, s);
        if (rc) return rc;
        return launch_astat(c, Y, n, st->At, s);
    }
    if (max_model(c->model))
        return launch_mca_estep(c, p->W, p->theta, Y, n, st, nullptr, nullptr, nullptr, nullptr,
                                nullptr, s);
    return launch_gsc_estep(c, p, Y, n, st, nullptr, nullptr, nullptr, nullptr, nullptr, s);
}

static int estep_end(prosper_ctx *c, prosper_stats *st, cudaStream_t s) {
    int rc = finish_astat_tc(c, st->At, s);
    if (rc) return rc;
    return launch_symmetrize(c, st->B, s);
}

}  // namespace prosper

using namespace prosper;

extern "C" {

const char *prosper_last_error(void) { return g_err; }

static int init_common(prosper_ctx **out, int model, int D, int H, int Hprime, int gamma,
                       int precision, int64_t max_points, int m, const float *vals) {
    if (!out) { set_error("out is NULL"); return PROSPER_EINVAL; }
    *out = nullptr;
    if (D < 1 || D > 1024) { set_error("D=%d outside [1, 1024]", D); return PROSPER_EINVAL; }
    if (H < 1 || H > 256) { set_error("H=%d outside [1, 256]", H); return PROSPER_EINVAL; }
    const int hp_max = model == PROSPER_GSC ? BSC_REG_MAX_HPRIME : PROSPER_MAX_HPRIME;
    if (Hprime < 1 || Hprime > hp_max || Hprime > H) {
        set_error("Hprime=%d outside [1, min(H, %d)]", Hprime, hp_max);
        return PROSPER_EINVAL;
    }
    if (gamma < 0 || gamma > Hprime) { set_error("gamma=%d outside [0, Hprime]", gamma); return PROSPER_EINVAL; }
    const int nK = num_states(Hprime, gamma, m);
    if (model == PROSPER_GSC && gamma > 3) { set_error("GSC: gamma=%d > 3", gamma); return PROSPER_EINVAL; }
    if (model == PROSPER_GSC && H > 32) { set_error("GSC: H=%d > 32", H); return PROSPER_EINVAL; }
    if ((model == PROSPER_GSC || max_model(model)) && D > 256) {
        set_error("MCA/MMCA/GSC: D=%d > 256", D);
        return PROSPER_EINVAL;
    }
    if (model == PROSPER_GSC && gsc_smem_bytes(D, H, Hprime, nK) > 227 * 1024) {
        set_error("GSC: D=%d, H=%d, Hprime=%d, gamma=%d need %zu bytes of shared memory per CTA (> 227 KB)",
                  D, H, Hprime, gamma, gsc_smem_bytes(D, H, Hprime, nK));
        return PROSPER_EINVAL;
    }
    if (max_model(model) && nK > 1024) {
        set_error("MCA/MMCA: %d states per point > 1024", nK);
        return PROSPER_EINVAL;
    }
    // the table-driven state kernel (TSC, DSC, BSC above Hprime 10) packs at
    // most 8 nonzero units per state
    const bool table = model == PROSPER_TSC || model == PROSPER_DSC ||
                       (model == PROSPER_BSC && Hprime > BSC_REG_MAX_HPRIME);
    if (linear_model(model) && nK > PROSPER_MAX_STATES) {
        set_error("%d states per point > %d", nK, PROSPER_MAX_STATES);
        return PROSPER_EINVAL;
    }
    if (table && gamma > 8) {
        set_error("gamma=%d > 8 (discrete latents, or BSC with Hprime > %d)", gamma, BSC_REG_MAX_HPRIME);
        return PROSPER_EINVAL;
    }
    if (precision != PROSPER_FP32 && precision != PROSPER_BF16_RESCORE) {
        set_error("unknown precision %d", precision);
        return PROSPER_EINVAL;
    }
    if (precision == PROSPER_BF16_RESCORE &&
        (model != PROSPER_BSC || D % 64 != 0 || H % 64 != 0 || D > 256 || bf16_smem_bytes(D, H) > 227 * 1024)) {
        set_error("BF16_RESCORE needs BSC, D %% 64 == 0, D <= 256, H %% 64 == 0 and the BF16 dictionary, "
                  "one operand tile and the candidate buffers within 227 KB of shared memory");
        return PROSPER_EINVAL;
    }
    if (max_points <= 0) max_points = 1 << 20;
    // PROSPER_TEST_TC_NO_COMMIT_MS=<ms> (tests only): the BF16 projection kernel
    // skips its MMA chain and gives up waiting after <ms>, exercising the
    // timeout path that prosper_status reports
    int test_ms = 0;
    if (const char *e = getenv("PROSPER_TEST_TC_NO_COMMIT_MS")) test_ms = atoi(e);

    prosper_ctx *c = new (std::nothrow) prosper_ctx();
    if (!c) { set_error("host allocation failed"); return PROSPER_ENOMEM; }
    c->model = model; c->D = D; c->H = H; c->Hp = Hprime; c->gamma = gamma;
    c->precision = precision;
    c->nK = nK;
    c->dsc_m = m;
    bool pos = false, neg = false;
    for (int v = 0; v < m; ++v) {
        c->dsc_vals[v] = vals[v];
        pos |= vals[v] > 0.f;
        neg |= vals[v] < 0.f;
    }
    // preselection score: signed normalised projection; magnitude when the
    // latent values have both signs; negated when they are all negative
    c->score_mode = (pos && neg) ? 1 : (neg ? 2 : 0);
    c->chunk = max_points;
    c->tc_test_no_commit_ms = (test_ms > 0 && test_ms <= 2000) ? test_ms : 0;
    if (const char *e = getenv("PROSPER_ASTAT_SIMT")) c->astat_simt = atoi(e) != 0;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(e));
        delete c;
        return PROSPER_ECUDA;
    }
    int rc = PROSPER_OK;
    const size_t ch = (size_t)c->chunk;
#define ALLOC(ptr, n) do { if (!rc) rc = dev_alloc(&(ptr), (n)); } while (0)
    ALLOC(c->d_status, 1);
    if (linear_model(model) || model == PROSPER_GSC) {
        ALLOC(c->G, (size_t)H * H);
        ALLOC(c->rnorm, (size_t)H);
        const size_t Hq = (size_t)mstep_hq(H);
        ALLOC(c->mB, Hq * Hq);
        ALLOC(c->mX, Hq * D);
        ALLOC(c->mI, Hq * Hq);
        ALLOC(c->mP, Hq * 32);
        ALLOC(c->mY, Hq * D);
        ALLOC(c->mZ, Hq * Hq);
        ALLOC(c->mW, (size_t)H * D);
        ALLOC(c->mpart, (size_t)mstep_nparts(H, D));
    }
    if (linear_model(model)) {
        if (precision == PROSPER_FP32) ALLOC(c->Wd, (size_t)D * H);
        else ALLOC(c->Wb, (size_t)H * D);
        ALLOC(c->sel, ch * SEL_STRIDE);
        ALLOC(c->selp, ch * SEL_STRIDE);
        ALLOC(c->es, ch * SEL_STRIDE);
        if (astat_tc_ok(D, H)) ALLOC(c->apart, (size_t)c->num_sms * H * D);
        ALLOC(c->yy, ch * 2);
    }
    if (max_model(model)) ALLOC(c->mca_logW, (size_t)H * D);
    if (model == PROSPER_GSC) {
        int nsub = 0;              // nonempty subsets of at most gamma of the H latents
        double b = 1.0;
        for (int k = 0; k <= gamma; ++k) {
            if (k > 0) nsub += (int)(b + 0.5);
            b = b * (H - k) / (k + 1);
        }
        c->gsc_nsub = nsub;
        ALLOC(c->gsc_tab, (size_t)nsub * 8);
    }
#undef ALLOC
    if (!rc && table) rc = dsc_build_table(c);
    if (!rc && cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess) rc = PROSPER_ECUDA;
    if (rc) {
        prosper_destroy(c);
        return rc;
    }
    *out = c;
    return PROSPER_OK;
}

int prosper_init(prosper_ctx **out, int model, int D, int H, int Hprime, int gamma,
                 int precision, int64_t max_points) {
    if (out) *out = nullptr;
    if (model < PROSPER_BSC || model > PROSPER_MMCA || model == PROSPER_DSC) {
        set_error(model == PROSPER_DSC ? "DSC contexts are created by prosper_init_dsc"
                                       : "unknown model %d", model);
        return PROSPER_EINVAL;
    }
    static const float kBinary[1] = {1.f}, kTernary[2] = {-1.f, 1.f};
    if (model == PROSPER_TSC)
        return init_common(out, model, D, H, Hprime, gamma, precision, max_points, 2, kTernary);
    return init_common(out, model, D, H, Hprime, gamma, precision, max_points, 1, kBinary);
}

int prosper_init_dsc(prosper_ctx **out, int D, int H, int Hprime, int gamma, int m,
                     const float *values_host, int64_t max_points) {
    if (out) *out = nullptr;
    if (m < 1 || m > 3 || !values_host) { set_error("DSC: m=%d outside [1, 3] or no values", m); return PROSPER_EINVAL; }
    for (int v = 0; v < m; ++v) {
        if (!(values_host[v] != 0.f) || !std::isfinite(values_host[v])) {
            set_error("DSC: value %d is zero or not finite", v);
            return PROSPER_EINVAL;
        }
        for (int u = 0; u < v; ++u)
            if (values_host[u] == values_host[v]) { set_error("DSC: values %d and %d are equal", u, v); return PROSPER_EINVAL; }
    }
    return init_common(out, PROSPER_DSC, D, H, Hprime, gamma, PROSPER_FP32, max_points, m, values_host);
}

int prosper_status(prosper_ctx *c, void *stream) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned st = 0;
    PROSPER_CUDA_TRY(cudaMemcpyAsync(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PROSPER_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        PROSPER_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s));
        PROSPER_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (st & ST_TC_TIMEOUT) { set_error("a tensor-core pipeline wait gave up"); return PROSPER_ETIMEOUT; }
    if (st & ST_NONFINITE) { set_error("non-finite value in the input or a result"); return PROSPER_ENONFINITE; }
    if (st & ST_CHOL_FAIL) { set_error("M-step matrix not positive definite"); return PROSPER_ENONFINITE; }
    return PROSPER_OK;
}

int prosper_trace_enable(prosper_ctx *c, int on) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    if (!c->trace) c->trace = new TraceState();
    c->trace->on = on != 0;
    return PROSPER_OK;
}

int prosper_trace_read(prosper_ctx *c, int max, char *names, double *total_ms, int *launches) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    if (!c->trace) return 0;
    PROSPER_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<std::string> order;
    std::map<std::string, std::pair<double, int>> acc;
    for (auto &r : c->trace->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        auto it = acc.find(r.name);
        if (it == acc.end()) { order.push_back(r.name); acc[r.name] = {ms, r.kernels}; }
        else { it->second.first += ms; it->second.second += r.kernels; }
    }
    c->trace->recs.clear();
    int k = 0;
    for (auto &nm : order) {
        if (k >= max) break;
        if (names) { strncpy(names + 48 * k, nm.c_str(), 47); names[48 * k + 47] = 0; }
        if (total_ms) total_ms[k] = acc[nm].first;
        if (launches) launches[k] = acc[nm].second;
        ++k;
    }
    return k;
}

int prosper_destroy(prosper_ctx *c) {
    if (!c) return PROSPER_OK;
    if (c->serve) prosper_serve_stop(c);
    if (c->trace) {
        for (auto &r : c->trace->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        delete c->trace;
    }
    cudaFree(c->d_hstats);
    cudaFree(c->G); cudaFree(c->rnorm); cudaFree(c->Wd); cudaFree(c->Wb);
    cudaFree(c->mca_logW); cudaFree(c->gsc_tab); cudaFree(c->dsc_tab);
    cudaFree(c->cut_logz); cudaFree(c->cut_hist); cudaFree(c->cut_state); cudaFree(c->cut_thr);
    cudaFree(c->sel); cudaFree(c->selp); cudaFree(c->yy); cudaFree(c->es); cudaFree(c->apart);
    if (c->h_copy) {
        cudaStreamSynchronize(c->h_copy);
        for (int i = 0; i < 3; ++i) { cudaEventDestroy(c->h_copied[i]); cudaEventDestroy(c->h_used[i]); }
        cudaEventDestroy(c->h_start);
        cudaStreamDestroy(c->h_copy);
    }
    cudaFree(c->mB); cudaFree(c->mX); cudaFree(c->mI); cudaFree(c->mP); cudaFree(c->mY); cudaFree(c->mZ); cudaFree(c->mW); cudaFree(c->mpart); cudaFree(c->d_status);
    cudaFree(c->d_stage);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    delete c;
    return PROSPER_OK;
}

int prosper_estep(prosper_ctx *c, const prosper_params *p, const float *Y, int64_t N,
                  prosper_stats *st, void *stream) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    int rc = check_params(c, p);
    if (!rc) rc = check_stats(c, st);
    if (rc) return rc;
    if (N < 0 || (N > 0 && !Y)) { set_error("bad Y/N"); return PROSPER_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = estep_begin(c, p, st, s))) return rc;
    if (c->cut && N > 0) {
        // data cut: a first pass stores every point's log Z, the threshold of
        // the N_cut best-explained points follows, and the second pass sums
        // the statistics of the points that reach it
        if ((rc = cut_reserve(c, N))) return rc;
        for (int64_t n0 = 0; n0 < N; n0 += c->chunk) {
            const int64_t n = std::min<int64_t>(c->chunk, N - n0);
            if ((rc = launch_linear_proj(c, Y + n0 * c->D, p->W, n, s))) return rc;
            rc = launch_linear_states(c, p->theta, n, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                                      nullptr, c->cut_logz + n0, s);
            if (rc) return rc;
        }
        if ((rc = launch_cut_select(c, p->theta, N, s))) return rc;
    }
    for (int64_t n0 = 0; n0 < N; n0 += c->chunk) {
        const int64_t n = std::min<int64_t>(c->chunk, N - n0);
        c->cut_n0 = n0;
        if ((rc = estep_piece(c, p, Y + n0 * c->D, n, st, s))) return rc;
    }
    return estep_end(c, st, s);
}

int prosper_set_data_cut(prosper_ctx *c, int on) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    if (on && c->model != PROSPER_BSC && c->model != PROSPER_TSC) {
        set_error("data cut: BSC and TSC contexts only");
        return PROSPER_EINVAL;
    }
    c->cut = on ? 1 : 0;
    return PROSPER_OK;
}

int prosper_mstep(prosper_ctx *c, const prosper_stats *st, int64_t N, prosper_params *p,
                  void *stream) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    int rc = check_params(c, p);
    if (!rc) rc = check_stats(c, st);
    if (rc) return rc;
    if (N <= 0) { set_error("mstep needs N > 0"); return PROSPER_EINVAL; }
    return launch_mstep(c, st, N, p, (cudaStream_t)stream);
}

static int encode_impl(prosper_ctx *c, const prosper_params *p, const float *Y, int64_t N,
                       int16_t *sel, float *s_mean, int16_t *map_idx, float *map_val, float *map_p,
                       float *logZ, void *stream) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    int rc = check_params(c, p);
    if (rc) return rc;
    if (N < 0 || (N > 0 && !Y)) { set_error("bad Y/N"); return PROSPER_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) return PROSPER_OK;
    if (linear_model(c->model)) {
        if ((rc = launch_bsc_prep(c, p->W, s))) return rc;
        for (int64_t n0 = 0; n0 < N; n0 += c->chunk) {
            const int64_t n = std::min<int64_t>(c->chunk, N - n0);
            const float *Yp = Y + n0 * c->D;
            if ((rc = launch_linear_proj(c, Yp, p->W, n, s))) return rc;
            rc = launch_linear_states(c, p->theta, n, n0, nullptr, sel, s_mean, map_idx, map_val,
                                      map_p, logZ, s);
            if (rc) return rc;
        }
        return PROSPER_OK;
    }
    if (max_model(c->model)) {
        if ((rc = launch_mca_prep(c, p->W, s))) return rc;
        return launch_mca_estep(c, p->W, p->theta, Y, N, nullptr, sel, s_mean, map_idx, map_p,
                                logZ, s);
    }
    if ((rc = launch_gsc_prep(c, p, s))) return rc;
    return launch_gsc_estep(c, p, Y, N, nullptr, sel, s_mean, map_idx, map_p, logZ, s);
}

int prosper_encode(prosper_ctx *c, const prosper_params *p, const float *Y, int64_t N,
                   int16_t *sel, float *s_mean, int16_t *map_idx, float *map_p, float *logZ,
                   void *stream) {
    return encode_impl(c, p, Y, N, sel, s_mean, map_idx, nullptr, map_p, logZ, stream);
}

int prosper_encode_values(prosper_ctx *c, const prosper_params *p, const float *Y, int64_t N,
                          int16_t *sel, float *s_mean, int16_t *map_idx, float *map_val,
                          float *map_p, float *logZ, void *stream) {
    if (c && c->model != PROSPER_TSC && c->model != PROSPER_DSC) {
        set_error("encode_values: TSC or DSC contexts only");
        return PROSPER_EINVAL;
    }
    return encode_impl(c, p, Y, N, sel, s_mean, map_idx, map_val, map_p, logZ, stream);
}

int prosper_estep_host(prosper_ctx *c, const prosper_params *p, const float *Y_host, int64_t N,
                       double *At_host, double *B_host, double *scal_host, void *stream) {
    if (!c) { set_error("ctx is NULL"); return PROSPER_EINVAL; }
    int rc = check_params(c, p);
    if (rc) return rc;
    if (N < 0 || (N > 0 && !Y_host)) { set_error("bad Y/N"); return PROSPER_EINVAL; }
    if (c->cut) { set_error("estep_host: the data cut needs the device E-step"); return PROSPER_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    // pieces of 32,768 points (32 MB at D = 256) through NSTAGE device staging
    // buffers: the host link (about 210 GB/s on this part) moves a piece in
    // ~160 us, longer than its E-step work, so the copies run back to back
    // (smaller pieces leave the kernels too little work to fill the GPU)
    constexpr int NSTAGE = 3;
    const int64_t cap = std::min<int64_t>(c->chunk, 32768);
    // equal pieces (multiples of 128 points): the work left after the last copy
    // is then one piece's E-step, not a full piece plus a remainder
    const int64_t npieces = N > 0 ? (N + cap - 1) / cap : 1;
    const int64_t piece = std::min<int64_t>(cap, ((N + npieces - 1) / npieces + 127) / 128 * 128);
    const size_t H = c->H, D = c->D;
    if (!c->d_stage) {
        size_t bytes = sizeof(float) * NSTAGE * (size_t)cap * D;
        PROSPER_CUDA_TRY(cudaMalloc(&c->d_stage, bytes));
        c->stage_points = cap;
    }
    if (!c->h_copy) {
        PROSPER_CUDA_TRY(cudaStreamCreateWithFlags(&c->h_copy, cudaStreamNonBlocking));
        for (int i = 0; i < NSTAGE; ++i) {
            PROSPER_CUDA_TRY(cudaEventCreateWithFlags(&c->h_copied[i], cudaEventDisableTiming));
            PROSPER_CUDA_TRY(cudaEventCreateWithFlags(&c->h_used[i], cudaEventDisableTiming));
        }
        PROSPER_CUDA_TRY(cudaEventCreateWithFlags(&c->h_start, cudaEventDisableTiming));
    }
    const size_t need = H * D + H * H + PROSPER_SC_LEN + 3 * H + 2 * H * D;
    if (!c->d_hstats) PROSPER_CUDA_TRY(cudaMalloc(&c->d_hstats, sizeof(double) * need));
    prosper_stats st;
    st.At = c->d_hstats;
    st.B = st.At + H * D;
    st.scal = st.B + H * H;
    st.gsc = st.scal + PROSPER_SC_LEN;
    st.mca = st.gsc + 3 * H;
    cudaStream_t cs = c->h_copy;
    // the copy stream starts after the work queued on s before this call (the
    // staging buffers are then free), in parallel with the E-step's prologue
    cudaEventRecord(c->h_start, s);
    cudaStreamWaitEvent(cs, c->h_start, 0);
    if ((rc = estep_begin(c, p, &st, s))) return rc;
    int k = 0;
    for (int64_t n0 = 0; n0 < N && !rc; n0 += piece, ++k) {
        const int64_t n = std::min<int64_t>(piece, N - n0);
        const int b = k % NSTAGE;
        float *buf = c->d_stage + (size_t)b * cap * D;
        if (k >= NSTAGE) cudaStreamWaitEvent(cs, c->h_used[b], 0);
        if (cudaMemcpyAsync(buf, Y_host + n0 * D, sizeof(float) * n * D, cudaMemcpyHostToDevice,
                            cs) != cudaSuccess) {
            set_error("H2D copy failed");
            rc = PROSPER_ECUDA;
            break;
        }
        cudaEventRecord(c->h_copied[b], cs);
        cudaStreamWaitEvent(s, c->h_copied[b], 0);
        rc = estep_piece(c, p, buf, n, &st, s);
        cudaEventRecord(c->h_used[b], s);
    }
    if (!rc) rc = estep_end(c, &st, s);
    if (!rc) {
        if (At_host) cudaMemcpyAsync(At_host, st.At, sizeof(double) * H * D, cudaMemcpyDeviceToHost, s);
        if (B_host) cudaMemcpyAsync(B_host, st.B, sizeof(double) * H * H, cudaMemcpyDeviceToHost, s);
        if (scal_host)
            cudaMemcpyAsync(scal_host, st.scal, sizeof(double) * PROSPER_SC_LEN, cudaMemcpyDeviceToHost, s);
    }
    unsigned status = 0;
    cudaMemcpyAsync(&status, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaStreamSynchronize(cs);
    if (rc) return rc;
    if (e != cudaSuccess) { set_error("stream failed: %s", cudaGetErrorString(e)); return PROSPER_ECUDA; }
    if (status & ST_NONFINITE) {
        cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s);
        cudaStreamSynchronize(s);
        set_error("non-finite value in the input data");
        return PROSPER_ENONFINITE;
    }
    return PROSPER_OK;
}

}  // extern "C"
