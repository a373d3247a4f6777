// mstep.cu -- closed-form M-steps in FP64 ("Model.step", paper Sec. 3; the
// prior and noise parameters are learned together with W, Sec. 1).
//
// BSC, GSC:  W = A B^{-1}   <=>   Wt = B^{-1} At  (Wt = W^T is H x D)
//            solved with a right-looking Cholesky factorisation of B
//            (Golub & Van Loan, Alg. 4.2.1 in outer-product form) and two
//            triangular solves per column of At;
//            pi = sum<|s|>/(N H);
//            sigma^2 = (sum y^T y - 2 tr(W^T A) + tr(W^T W B))/(N D) with the new W;
//            GSC: mu_h = sum<s_h>/sum<b_h>,
//                 psi_h = (sum<s_h^2> - 2 mu_h sum<s_h> + mu_h^2 sum<b_h>)/sum<b_h>.
// MCA:       W_dh = sum<A_dh> y_d / sum<A_dh> (kept if the denominator is 0,
//            clamped >= 1e-6), pi as BSC, sigma^2 = sum<||y - f||^2>/(N D).
// A unit with B_hh <= 1e-9 N (never active) keeps its W_h (its row and column
// of B are zero, so the system decouples exactly); the active block gets a
// ridge of 1e-9 tr(B)/H on the diagonal.
#include "internal.cuh"

namespace prosper {
namespace {

// msc[] slots
constexpr int MS_TRB = 0, MS_T1 = 1, MS_T2 = 2;

__global__ void k_trace(const double *__restrict__ B, int H, double *msc) {
    __shared__ double red[32];
    double s = 0.0;
    for (int h = threadIdx.x; h < H; h += blockDim.x) s += B[(size_t)h * H + h];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) { msc[MS_TRB] = s; msc[MS_T1] = 0.0; msc[MS_T2] = 0.0; }
    }
}

// mB = B (active block, + ridge) or identity; mX = At (active rows) or old W rows.
__global__ void k_build(const double *__restrict__ B, const double *__restrict__ At,
                        const float *__restrict__ W, int H, int D, double Ntot,
                        const double *__restrict__ msc, double *__restrict__ mB,
                        double *__restrict__ mX) {
    const double thr = 1e-9 * Ntot;
    const double ridge = 1e-9 * msc[MS_TRB] / H;
    const int64_t total = (int64_t)H * H + (int64_t)H * D;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < (int64_t)H * H) {
            int i = (int)(idx / H), j = (int)(idx % H);
            bool ai = B[(size_t)i * H + i] > thr, aj = B[(size_t)j * H + j] > thr;
            double v;
            if (ai && aj) v = B[idx] + (i == j ? ridge : 0.0);
            else v = (i == j) ? 1.0 : 0.0;
            mB[idx] = v;
        } else {
            int64_t k = idx - (int64_t)H * H;
            int h = (int)(k / D);
            bool ah = B[(size_t)h * H + h] > thr;
            mX[k] = ah ? At[k] : (double)W[k];
        }
    }
}

// In-place lower Cholesky factor of mB (H x H), one CTA.  Writes zeros above
// the diagonal.  Sets ST_CHOL_FAIL if a pivot is not positive.
__global__ void __launch_bounds__(1024) k_cholesky(double *A, int H, unsigned *status) {
    __shared__ double piv;
    __shared__ int fail;
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < H; ++j) {
        if (threadIdx.x == 0) {
            double d = A[(size_t)j * H + j];
            if (!(d > 0.0)) { fail = 1; d = 1.0; }
            piv = sqrt(d);
            A[(size_t)j * H + j] = piv;
        }
        __syncthreads();
        const double inv = 1.0 / piv;
        for (int i = j + 1 + threadIdx.x; i < H; i += blockDim.x) A[(size_t)i * H + j] *= inv;
        __syncthreads();
        // trailing update of the lower triangle: A[i][k] -= A[i][j] A[k][j], j < k <= i
        const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = j + 1 + wid; i < H; i += nw) {
            const double lij = A[(size_t)i * H + j];
            for (int k = j + 1 + lane; k <= i; k += 32) A[(size_t)i * H + k] -= lij * A[(size_t)k * H + j];
        }
        __syncthreads();
    }
    for (int64_t t = threadIdx.x; t < (int64_t)H * H; t += blockDim.x) {
        int i = (int)(t / H), k = (int)(t % H);
        if (k > i) A[t] = 0.0;
    }
    if (threadIdx.x == 0 && fail) atomicOr(status, ST_CHOL_FAIL);
}

// Solve L L^T x = mX[:, d] for one column d per CTA; writes the FP64 result
// back into mX and the FP32 copy into W.
__global__ void __launch_bounds__(256) k_cholsolve(const double *__restrict__ L, double *mX,
                                                   float *W, int H, int D) {
    extern __shared__ double x[];
    const int d = blockIdx.x;
    for (int h = threadIdx.x; h < H; h += blockDim.x) x[h] = mX[(size_t)h * D + d];
    __syncthreads();
    for (int i = 0; i < H; ++i) {                     // L v = b
        if (threadIdx.x == 0) x[i] /= L[(size_t)i * H + i];
        __syncthreads();
        const double xi = x[i];
        for (int k = i + 1 + threadIdx.x; k < H; k += blockDim.x) x[k] -= L[(size_t)k * H + i] * xi;
        __syncthreads();
    }
    for (int i = H - 1; i >= 0; --i) {                // L^T x = v
        if (threadIdx.x == 0) x[i] /= L[(size_t)i * H + i];
        __syncthreads();
        const double xi = x[i];
        for (int k = threadIdx.x; k < i; k += blockDim.x) x[k] -= L[(size_t)i * H + k] * xi;
        __syncthreads();
    }
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        mX[(size_t)h * D + d] = x[h];
        W[(size_t)h * D + d] = (float)x[h];
    }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// t1 = sum Wn . At, t2 = sum_h sum_d Wn[h][d] (B Wn)[h][d]  (original B).
// One CTA per row h.
__global__ void __launch_bounds__(256) k_traces(const double *__restrict__ Wn,
                                                const double *__restrict__ At,
                                                const double *__restrict__ B, int H, int D,
                                                double *msc) {
    __shared__ double red[32];
    const int h = blockIdx.x;
    double t1 = 0.0, t2 = 0.0;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const double w = Wn[(size_t)h * D + d];
        t1 += w * At[(size_t)h * D + d];
        double bw = 0.0;
        for (int k = 0; k < H; ++k) bw += B[(size_t)h * H + k] * Wn[(size_t)k * D + d];
        t2 += w * bw;
    }
    double s1 = block_sum(t1, red);
    double s2 = block_sum(t2, red);
    if (threadIdx.x == 0) {
        atomicAdd(msc + MS_T1, s1);
        atomicAdd(msc + MS_T2, s2);
    }
}

__global__ void k_theta(const double *__restrict__ scal, const double *__restrict__ msc,
                        const double *__restrict__ gsc, double *theta, float *mu, float *psi,
                        int H, int D, double Ntot, int model, unsigned *status) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        theta[PROSPER_TH_PI] = scal[PROSPER_SC_S1] / (Ntot * H);
        double s2;
        if (model == PROSPER_MCA) s2 = scal[PROSPER_SC_MCA_R2] / (Ntot * D);
        else s2 = (scal[PROSPER_SC_YY] - 2.0 * msc[MS_T1] + msc[MS_T2]) / (Ntot * D);
        theta[PROSPER_TH_SIGMA] = sqrt(s2 > 0.0 ? s2 : 0.0);
        if (!isfinite(s2) || !isfinite(theta[PROSPER_TH_PI])) atomicOr(status, ST_NONFINITE);
    }
    if (model == PROSPER_GSC) {
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x) {
            double sb = gsc[h], ss = gsc[H + h], ss2 = gsc[2 * H + h];
            if (!(sb > 1e-9 * Ntot)) continue;
            double m = ss / sb;
            double v = (ss2 - 2.0 * m * ss + m * m * sb) / sb;
            mu[h] = (float)m;
            psi[h] = (float)(v > 1e-8 ? v : 1e-8);
        }
    }
}

__global__ void k_mca_w(const double *__restrict__ mca, float *W, int H, int D) {
    const int64_t HD = (int64_t)H * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < HD;
         i += (int64_t)gridDim.x * blockDim.x) {
        double num = mca[i], den = mca[HD + i];
        if (den > 0.0) {
            double w = num / den;
            W[i] = (float)(w < 1e-6 ? 1e-6 : w);
        }
    }
}

}  // namespace

int launch_mstep(prosper_ctx *c, const prosper_stats *st, int64_t N, prosper_params *p,
                 cudaStream_t s) {
    const int H = c->H, D = c->D;
    const double Ntot = (double)N;
    TraceScope tr(c, "mstep", s, c->model == PROSPER_MCA ? 2 : 6);
    if (c->model == PROSPER_MCA) {
        k_mca_w<<<c->num_sms * 4, 256, 0, s>>>(st->mca, p->W, H, D);
        PROSPER_LAUNCH_CHECK();
        k_theta<<<1, 32, 0, s>>>(st->scal, c->msc, nullptr, p->theta, nullptr, nullptr, H, D, Ntot,
                                 c->model, c->d_status);
        PROSPER_LAUNCH_CHECK();
        return PROSPER_OK;
    }
    k_trace<<<1, 256, 0, s>>>(st->B, H, c->msc);
    PROSPER_LAUNCH_CHECK();
    k_build<<<c->num_sms * 4, 256, 0, s>>>(st->B, st->At, p->W, H, D, Ntot, c->msc, c->mB, c->mX);
    PROSPER_LAUNCH_CHECK();
    k_cholesky<<<1, 1024, 0, s>>>(c->mB, H, c->d_status);
    PROSPER_LAUNCH_CHECK();
    k_cholsolve<<<D, 256, sizeof(double) * H, s>>>(c->mB, c->mX, p->W, H, D);
    PROSPER_LAUNCH_CHECK();
    k_traces<<<H, 256, 0, s>>>(c->mX, st->At, st->B, H, D, c->msc);
    PROSPER_LAUNCH_CHECK();
    k_theta<<<1, 256, 0, s>>>(st->scal, c->msc, st->gsc, p->theta, p->mu, p->psi, H, D, Ntot,
                              c->model, c->d_status);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

}  // namespace prosper
