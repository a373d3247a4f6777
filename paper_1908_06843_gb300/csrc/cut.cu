// cut.cu -- ET's data-point cut on the GPU: the threshold log Z of the N_cut
// best-explained points.
//
// Reading (the paper names truncated posteriors, Sec. 2, and defers ET's
// details to its references): N_cut = floor(N P_pi(|s| <= gamma)) with
// P_pi(|s| <= gamma) = sum_{k <= gamma} C(H,k) pi^k (1 - pi)^(H - k), the
// expected number of points generated by at most gamma causes (at least 1).
// The E-step's statistics then use the points whose log sum_{K_n} p(s, y_n)
// (as the FP32 value the encode path reports) reaches the N_cut-th largest
// value; every point tied with it is kept.
//
// The N_cut-th largest value is found by radix selection on order-preserving
// 32-bit keys: a histogram of the upper 16 bits, a scan from the top to the
// bin where the count reaches N_cut, a histogram of the lower 16 bits inside
// that bin and a second scan.  Integer counts only, so the threshold does not
// depend on timing.
#include "internal.cuh"

#include <cmath>

namespace prosper {
namespace {

constexpr int kBins = 65536;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ unsigned order_key(float x) {
    const unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_value(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// N_cut from the current pi (theta), in FP64; state[0] = target count
__global__ void k_cut_count(const double *__restrict__ theta, int64_t N, int H, int gamma,
                            long long *__restrict__ state) {
    const double pi = theta[PROSPER_TH_PI];
    double P = 1.0;
    if (gamma < H) {
        double w = 1.0, sw = 0.0;     // C(H,k) (pi/(1-pi))^k
        for (int k = 0; k <= gamma; ++k) {
            sw += w;
            w *= (double)(H - k) / (k + 1) * pi / (1.0 - pi);
        }
        P = sw * exp(H * log1p(-pi));
    }
    long long n = (long long)floor((double)N * P);
    state[0] = n < 1 ? 1 : (n > N ? N : n);
}

__global__ void k_cut_hist(const float *__restrict__ logz, int64_t N, int pass,
                           const long long *__restrict__ state, unsigned *__restrict__ hist) {
    const unsigned hi = pass ? (unsigned)state[1] : 0u;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = order_key(logz[n]);
        if (pass == 0) atomicAdd(&hist[k >> 16], 1u);
        else if ((k >> 16) == hi) atomicAdd(&hist[k & 0xFFFFu], 1u);
    }
}

// One block: the bin (scanning from the top) where the running count reaches
// the target.  pass 0: target = N_cut, writes state[1] = upper bin and
// state[2] = the count above it; pass 1: target = N_cut - state[2], writes the
// threshold value.
__global__ void __launch_bounds__(kScanThreads) k_cut_scan(const unsigned *__restrict__ hist, int pass,
                                                          long long *__restrict__ state,
                                                          float *__restrict__ thr) {
    __shared__ long long part[kScanThreads];
    const int t = threadIdx.x;
    constexpr int per = kBins / kScanThreads;          // 64 bins, taken from the top
    const int top = kBins - 1 - per * t;               // this thread's highest bin
    long long s = 0;
    for (int i = 0; i < per; ++i) s += hist[top - i];
    part[t] = s;
    __syncthreads();
    // exclusive prefix (in descending bin order) by a plain two-level sum
    __shared__ long long chunk[32];
    if (t < 32) {
        long long c = 0;
        for (int i = 0; i < 32; ++i) c += part[32 * t + i];
        chunk[t] = c;
    }
    __syncthreads();
    long long before = 0;
    for (int i = 0; i < t / 32; ++i) before += chunk[i];
    for (int i = 32 * (t / 32); i < t; ++i) before += part[i];
    const long long target = pass ? state[0] - state[2] : state[0];
    if (before < target && before + s >= target) {
        long long run = before;
        for (int i = 0; i < per; ++i) {
            const long long h = hist[top - i];
            if (run + h >= target) {
                if (pass == 0) {
                    state[1] = top - i;
                    state[2] = run;
                } else {
                    *thr = key_value(((unsigned)state[1] << 16) | (unsigned)(top - i));
                }
                break;
            }
            run += h;
        }
    }
}

}  // namespace

int launch_cut_select(prosper_ctx *c, const double *theta, int64_t N, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    TraceScope tr(c, "cut_select", s, 5);
    PROSPER_CUDA_TRY(cudaMemsetAsync(c->cut_hist, 0, sizeof(unsigned) * 2 * kBins, s));
    k_cut_count<<<1, 1, 0, s>>>(theta, N, c->H, c->gamma, c->cut_state);
    PROSPER_LAUNCH_CHECK();
    const int grid = (int)std::min<int64_t>((N + 255) / 256, 4 * (int64_t)c->num_sms);
    k_cut_hist<<<grid, 256, 0, s>>>(c->cut_logz, N, 0, c->cut_state, c->cut_hist);
    PROSPER_LAUNCH_CHECK();
    k_cut_scan<<<1, kScanThreads, 0, s>>>(c->cut_hist, 0, c->cut_state, c->cut_thr);
    PROSPER_LAUNCH_CHECK();
    k_cut_hist<<<grid, 256, 0, s>>>(c->cut_logz, N, 1, c->cut_state, c->cut_hist + kBins);
    PROSPER_LAUNCH_CHECK();
    k_cut_scan<<<1, kScanThreads, 0, s>>>(c->cut_hist + kBins, 1, c->cut_state, c->cut_thr);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

int cut_reserve(prosper_ctx *c, int64_t N) {
    if (!c->cut_hist) {
        if (cudaMalloc(&c->cut_hist, sizeof(unsigned) * 2 * kBins) != cudaSuccess ||
            cudaMalloc(&c->cut_state, sizeof(long long) * 4) != cudaSuccess ||
            cudaMalloc(&c->cut_thr, sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            set_error("data cut: allocation failed");
            return PROSPER_ENOMEM;
        }
    }
    if (c->cut_cap < N) {
        cudaFree(c->cut_logz);
        c->cut_logz = nullptr;
        if (cudaMalloc(&c->cut_logz, sizeof(float) * (size_t)N) != cudaSuccess) {
            cudaGetLastError();
            c->cut_cap = 0;
            set_error("data cut: cudaMalloc of %lld log Z values failed", (long long)N);
            return PROSPER_ENOMEM;
        }
        c->cut_cap = N;
    }
    return PROSPER_OK;
}

}  // namespace prosper
