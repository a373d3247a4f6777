// noalloc.cu -- prosper_encode_noalloc: BSC encoding (the FP32 form of
// prosper_encode) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they encode: code
// that runs after a fixed start-up phase and must never allocate again (a
// real-time serving loop, or a process whose device memory is entirely
// handed to a framework's caching allocator), and code that must not
// synchronise the device (cudaMalloc and cudaFree may do so implicitly).
// This entry point therefore needs no context and allocates nothing: its
// scratch (the Gram matrix, 1/||W_h||, the transposed dictionary and the
// per-point candidate lists) lives in one file-scope __device__ array of fixed
// size, which every GPU that loads this library holds until the process exits.
//
// Limits (rejected with PROSPER_EINVAL): D <= 256, H <= 256,
// 1 <= Hprime <= 10, 0 <= gamma <= Hprime, N <= 4096 points per call.
//
// The array is shared by every call on a device and keeps the last call's
// contents; everything a call reads is written by that call first, except the
// status word, which each call clears.  Calls whose GPU work overlaps (on two
// streams, or from two host threads) race on the array and give undefined
// results: issue them on one stream or serialise them.
//
// Non-finite input is not reported on this path (there is no context whose
// status word a caller could read): a point whose y holds NaN or Inf gets a
// non-finite log Z, which the caller can test.
//
// The first call on each device looks up the device address of the array
// (cudaGetSymbolAddress, with that device current); make that first call
// before any stream capture begins.
#include "internal.cuh"

#include <mutex>

namespace prosper {
namespace {

constexpr int NA_D = 256, NA_H = 256, NA_N = 4096;
constexpr size_t align64(size_t n) { return (n + 63) & ~(size_t)63; }   // 256-byte units
constexpr size_t OFF_G = 0;                                             // H x H
constexpr size_t OFF_RN = OFF_G + align64((size_t)NA_H * NA_H);         // H
constexpr size_t OFF_WD = OFF_RN + align64(NA_H);                       // D x H
constexpr size_t OFF_SEL = OFF_WD + align64((size_t)NA_D * NA_H);       // N x 16 int32
constexpr size_t OFF_SELP = OFF_SEL + align64((size_t)NA_N * SEL_STRIDE);   // N x 16
constexpr size_t OFF_YY = OFF_SELP + align64((size_t)NA_N * SEL_STRIDE);    // N x 2
constexpr size_t OFF_ST = OFF_YY + align64((size_t)NA_N * 2);              // status word
constexpr size_t NA_FLOATS = OFF_ST + 64;                                   // ~1.06 MB

static __device__ __align__(256) float g_noalloc_scratch[NA_FLOATS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float *g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Per-device set-up: the device address of the scratch array (host code only
// sees a host-side stand-in under its name).
int scratch_for_current_device(float **out, int *num_sms, int *device) {
    int dev = 0;
    PROSPER_CUDA_TRY(cudaGetDevice(&dev));
    *device = dev;
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond %d", dev, kMaxDevices);
        return PROSPER_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the encode scratch failed: %s", cudaGetErrorString(e));
            return PROSPER_ECUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            set_error("cudaDeviceGetAttribute failed: %s", cudaGetErrorString(e));
            return PROSPER_ECUDA;
        }
        g_num_sms[dev] = sms;
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    *num_sms = g_num_sms[dev];
    return PROSPER_OK;
}

}  // namespace
}  // namespace prosper

using namespace prosper;

extern "C" int prosper_encode_noalloc(int D, int H, int Hprime, int gamma, const float *W,
                                      const double *theta, const float *Y, int64_t N,
                                      int16_t *sel, float *s_mean, int16_t *map_idx,
                                      float *map_p, float *logZ, void *stream) {
    if (D < 1 || D > NA_D || H < 1 || H > NA_H) {
        set_error("encode_noalloc: D=%d, H=%d outside [1, %d] x [1, %d]", D, H, NA_D, NA_H);
        return PROSPER_EINVAL;
    }
    if (Hprime < 1 || Hprime > BSC_REG_MAX_HPRIME || Hprime > H || gamma < 0 || gamma > Hprime) {
        set_error("encode_noalloc: Hprime=%d, gamma=%d outside the limits", Hprime, gamma);
        return PROSPER_EINVAL;
    }
    if (N < 0 || N > NA_N) {
        set_error("encode_noalloc: N=%lld outside [0, %d] points per call", (long long)N, NA_N);
        return PROSPER_EINVAL;
    }
    if (!W || !theta || (N > 0 && !Y)) {
        set_error("encode_noalloc: W, theta and Y must be device pointers");
        return PROSPER_EINVAL;
    }
    if (N == 0) return PROSPER_OK;
    float *base = nullptr;
    int sms = 0;
    int dev = 0;
    int rc = scratch_for_current_device(&base, &sms, &dev);
    if (rc) return rc;

    // a context on the host stack whose scratch pointers all point into the
    // array; value-initialised, so every member not set here is zero / null
    prosper_ctx c{};
    c.model = PROSPER_BSC; c.D = D; c.H = H; c.Hp = Hprime; c.gamma = gamma;
    c.precision = PROSPER_FP32;
    c.nK = num_states(Hprime, gamma);
    c.chunk = NA_N;
    c.device = dev;
    c.num_sms = sms;
    c.G = base + OFF_G;
    c.rnorm = base + OFF_RN;
    c.Wd = base + OFF_WD;
    c.sel = reinterpret_cast<int32_t *>(base + OFF_SEL);
    c.selp = base + OFF_SELP;
    c.yy = base + OFF_YY;
    c.d_status = reinterpret_cast<unsigned *>(base + OFF_ST);
    cudaStream_t s = (cudaStream_t)stream;
    PROSPER_CUDA_TRY(cudaMemsetAsync(c.d_status, 0, sizeof(unsigned), s));
    if ((rc = launch_bsc_prep(&c, W, s))) return rc;
    if ((rc = launch_bsc_proj_f32(&c, Y, N, s))) return rc;
    return launch_bsc_states(&c, theta, N, 0, nullptr, sel, s_mean, map_idx, map_p, logZ, s);
}
