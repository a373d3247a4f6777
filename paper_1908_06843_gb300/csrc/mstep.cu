// mstep.cu -- closed-form M-steps in FP64 ("Model.step", paper Sec. 3; the
// prior and noise parameters are learned together with W, Sec. 1).
//
// BSC, GSC:  W = A B^{-1}   <=>   Wt = B^{-1} At  (Wt = W^T is H x D);
//            pi = sum<|s|>/(N H);
//            sigma^2 = (sum y^T y - 2 tr(W^T A) + tr(W^T W B))/(N D) with the new W;
//            GSC: mu_h = sum<s_h>/sum<b_h>,
//                 psi_h = (sum<s_h^2> - 2 mu_h sum<s_h> + mu_h^2 sum<b_h>)/sum<b_h>.
// MCA:       W_dh = sum<A_dh> y_d / sum<A_dh> (kept if the denominator is 0,
//            clamped >= 1e-6), pi as BSC, sigma^2 = sum<||y - f||^2>/(N D).
// A unit with B_hh <= 1e-9 N (never active) keeps its W_h (its row and column
// of B are zero, so the system decouples exactly); the active block gets a
// ridge of 1e-9 tr(B)/H on the diagonal.
//
// The solve is spread over the whole GPU, because FP64 arithmetic is scarce
// on this part (a few FP64 FMAs per clock per SM): a blocked right-looking
// Cholesky factorisation (block 32; Golub & Van Loan, Matrix Computations,
// Sec. 4.2) of the system augmented by [At | I], so the forward substitution
// yields L^-1 At and L^-1 in the same pass, followed by one parallel product
// Wt = (L^-1)^T (L^-1 At).  tr(W^T W B) uses the symmetry of W W^T.  All
// reductions write per-CTA partials that one CTA adds in a fixed order, so the
// result does not depend on scheduling.
#include "internal.cuh"

namespace prosper {
namespace {

constexpr int MB = 32;    // Cholesky block (rows/columns)
constexpr int MT = 16;    // trailing-update output tile
constexpr int NT = 256;   // threads per CTA of every M-step kernel

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

// Builds the augmented system [mB | mX | mI] of order Hq = H rounded up to MB:
//   mB = B on the active block (+ ridge 1e-9 tr(B)/H), identity elsewhere
//        (inactive units and the padding rows/columns);
//   mX = At on active rows, the old W on inactive rows, 0 on padding rows;
//   mI = identity.
// Every CTA forms tr(B) itself (H loads), so no separate launch is needed.
__global__ void __launch_bounds__(NT) k_build(const double *__restrict__ B,
                                              const double *__restrict__ At,
                                              const float *__restrict__ W, int H, int Hq, int D,
                                              double Ntot, double *__restrict__ mB,
                                              double *__restrict__ mX, double *__restrict__ mI) {
    __shared__ double red[NT / 32];
    double tr = 0.0;
    for (int h = threadIdx.x; h < H; h += NT) tr += B[(size_t)h * H + h];
    tr = block_sum(tr, red);
    __shared__ double ridge_s;
    if (threadIdx.x == 0) ridge_s = 1e-9 * tr / H;
    __syncthreads();
    const double ridge = ridge_s, thr = 1e-9 * Ntot;
    const int64_t nB = (int64_t)Hq * Hq, nX = (int64_t)Hq * D;
    for (int64_t idx = (int64_t)blockIdx.x * NT + threadIdx.x; idx < 2 * nB + nX;
         idx += (int64_t)gridDim.x * NT) {
        if (idx < nB) {
            const int i = (int)(idx / Hq), j = (int)(idx % Hq);
            double v = (i == j) ? 1.0 : 0.0;
            if (i < H && j < H && B[(size_t)i * H + i] > thr && B[(size_t)j * H + j] > thr)
                v = B[(size_t)i * H + j] + (i == j ? ridge : 0.0);
            mB[idx] = v;
        } else if (idx < 2 * nB) {
            const int64_t e = idx - nB;
            mI[e] = (e / Hq == e % Hq) ? 1.0 : 0.0;
        } else {
            const int64_t e = idx - 2 * nB;
            const int h = (int)(e / D);
            double v = 0.0;
            if (h < H) v = (B[(size_t)h * H + h] > thr) ? At[e] : (double)W[e];
            mX[e] = v;
        }
    }
}

// Step k of the blocked right-looking Cholesky factorisation B = L L^T
// (Golub & Van Loan, Alg. 4.2.4 with block size MB), carried along the
// right-hand sides [mX | mI] so that the forward substitution happens in the
// same pass.  Every CTA factors the diagonal block A_kk in shared memory, then
//   CTA b <  nrow : L_ik = A_ik L_kk^-T for row block i = k + 1 + b (into mB);
//   CTA b >= nrow : Y_k = L_kk^-1 R_k for one 32-column tile of mX, or of the
//                   identity block columns j <= k of mI (the others are still
//                   zero in row block k).
// CTA 0 reports a non-positive pivot (the pivot is then taken as 1).
__global__ void __launch_bounds__(NT) k_panel(double *__restrict__ mB, double *__restrict__ mX,
                                              double *__restrict__ mI, int Hq, int D, int k,
                                              int nrow, int ncolx, unsigned *status) {
    __shared__ double L[MB][MB + 1];
    __shared__ double T[MB][MB + 1];
    __shared__ double invd[MB];
    __shared__ int fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = k * MB;
    for (int e = tid; e < MB * MB; e += NT) L[e / MB][e % MB] = mB[(size_t)(k0 + e / MB) * Hq + k0 + e % MB];
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int t = 0; t < MB; ++t) {
        if (tid == 0) {
            double d = L[t][t];
            if (!(d > 0.0)) { fail = 1; d = 1.0; }
            d = sqrt(d);
            L[t][t] = d;
            invd[t] = 1.0 / d;
        }
        __syncthreads();
        if (tid > t && tid < MB) L[tid][t] *= invd[t];
        __syncthreads();
        for (int e = tid; e < MB * MB; e += NT) {
            const int r = e / MB, c = e % MB;
            if (c > t && c <= r) L[r][c] -= L[r][t] * L[c][t];
        }
        __syncthreads();
    }
    const int b = blockIdx.x;
    const bool rowrole = b < nrow;
    double *R;
    int ld, r0, c0, ncols;
    if (rowrole) {
        R = mB; ld = Hq; r0 = k0 + MB * (b + 1); c0 = k0; ncols = MB;
    } else if (b - nrow < ncolx) {
        R = mX; ld = D; r0 = k0; c0 = (b - nrow) * MB; ncols = min(MB, D - c0);
    } else {
        R = mI; ld = Hq; r0 = k0; c0 = (b - nrow - ncolx) * MB; ncols = MB;
    }
    for (int e = tid; e < MB * MB; e += NT) {
        const int r = e / MB, c = e % MB;
        T[r][c] = c < ncols ? R[(size_t)(r0 + r) * ld + c0 + c] : 0.0;
    }
    __syncthreads();
    // both roles are a forward substitution along a 32-vector held one entry
    // per lane: x_t = a_t / L_tt, then a_u -= L_ut x_t for u > t
    //   row role   : the vector is row v of A_ik   (X L_kk^T = A_ik)
    //   column role: the vector is column v of R_k (L_kk Y = R_k)
    for (int v = warp; v < MB; v += NT / 32) {
        double a = rowrole ? T[v][lane] : T[lane][v];
        for (int t = 0; t < MB; ++t) {
            const double xt = __shfl_sync(0xffffffffu, a, t) * invd[t];
            if (lane == t) a = xt;
            else if (lane > t) a -= L[lane][t] * xt;
        }
        if (rowrole) T[v][lane] = a;
        else T[lane][v] = a;
    }
    __syncthreads();
    for (int e = tid; e < MB * MB; e += NT) {
        const int r = e / MB, c = e % MB;
        if (c < ncols) R[(size_t)(r0 + r) * ld + c0 + c] = T[r][c];
    }
    if (b == 0 && tid == 0 && fail) atomicOr(status, ST_CHOL_FAIL);
}

// Trailing update of step k on MT x MT tiles:
//   tiles [0, nbt)      : A_ij -= L_ik L_jk^T, lower tiles of the rows/columns > k
//   tiles [nbt, grid)   : R_i  -= L_ik Y_k for the row blocks i > k, over the
//                         16-column tiles of mX and of mI's block columns <= k.
__global__ void __launch_bounds__(NT) k_update(double *__restrict__ mB, double *__restrict__ mX,
                                               double *__restrict__ mI, int Hq, int D, int k,
                                               int nbt, int nxt, int nrt) {
    __shared__ double As[MT][MB + 1];
    __shared__ double Bs[MB][MT + 1];
    const int tid = threadIdx.x;
    const int k0 = k * MB, base = k0 + MB;
    int x = blockIdx.x, row0, col0, ld, ncols;
    double *out;
    bool lower_tile;
    if (x < nbt) {
        int si = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
        while ((si + 1) * (si + 2) / 2 <= x) ++si;
        while (si * (si + 1) / 2 > x) --si;
        const int sj = x - si * (si + 1) / 2;
        row0 = base + si * MT;
        col0 = base + sj * MT;
        out = mB; ld = Hq; ncols = MT; lower_tile = true;
    } else {
        x -= nbt;
        const int si = x / nrt, ct = x % nrt;
        row0 = base + si * MT;
        if (ct < nxt) { out = mX; ld = D; col0 = ct * MT; ncols = min(MT, D - col0); }
        else { out = mI; ld = Hq; col0 = (ct - nxt) * MT; ncols = MT; }
        lower_tile = false;
    }
    for (int e = tid; e < MT * MB; e += NT) {
        const int r = e / MB, t = e % MB;
        As[r][t] = mB[(size_t)(row0 + r) * Hq + k0 + t];
    }
    for (int e = tid; e < MB * MT; e += NT) {
        if (lower_tile) {
            const int c = e / MB, t = e % MB;   // row c of L_jk
            Bs[t][c] = mB[(size_t)(col0 + c) * Hq + k0 + t];
        } else {
            const int t = e / MT, c = e % MT;   // row t of Y_k
            Bs[t][c] = c < ncols ? out[(size_t)(k0 + t) * ld + col0 + c] : 0.0;
        }
    }
    __syncthreads();
    const int r = tid / MT, c = tid % MT;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < MB; ++t) acc += As[r][t] * Bs[t][c];
    if (c < ncols) out[(size_t)(row0 + r) * ld + col0 + c] -= acc;
}

// Back substitution with the explicit inverse: after the forward pass mI holds
// L^-1 (lower triangular) and mX holds L^-1 X, so W^T = L^-T (L^-1 X):
//   Wn[i][d] = sum_{t >= i} Linv[t][i] Y[t][d]      (8 x 32 tile per CTA)
// Writes Wn in FP64 (mW, H x D) and FP32 (W), and the CTA's share of
// t1 = sum Wn . At into part[blockIdx.x].  CTAs with more rows above the
// diagonal come first (largest work first).
__global__ void __launch_bounds__(NT) k_backsub(const double *__restrict__ mI,
                                                const double *__restrict__ mX,
                                                const double *__restrict__ At, int H, int Hq,
                                                int D, int nct, double *__restrict__ mW,
                                                float *__restrict__ W, double *__restrict__ part) {
    __shared__ double Ls[MB][8 + 1];
    __shared__ double Ys[MB][MB + 1];
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    const int i0 = (blockIdx.x / nct) * 8, d0 = (blockIdx.x % nct) * MB;
    const int r = tid >> 5, dcol = d0 + lane;
    double acc = 0.0;
    for (int t0 = i0; t0 < Hq; t0 += MB) {
        {
            const int t = tid >> 3, rr = tid & 7;
            Ls[t][rr] = (t0 + t < Hq) ? mI[(size_t)(t0 + t) * Hq + i0 + rr] : 0.0;
        }
        for (int e = tid; e < MB * MB; e += NT) {
            const int t = e / MB, c = e % MB;
            Ys[t][c] = (t0 + t < Hq && d0 + c < D) ? mX[(size_t)(t0 + t) * D + d0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < MB; ++t) acc += Ls[t][r] * Ys[t][lane];
        __syncthreads();
    }
    const int h = i0 + r;
    double t1 = 0.0;
    if (h < H && dcol < D) {
        const size_t o = (size_t)h * D + dcol;
        mW[o] = acc;
        W[o] = (float)acc;
        t1 = acc * At[o];
    }
    t1 = block_sum(t1, red);
    if (tid == 0) part[blockIdx.x] = t1;
}

// t2 = sum_{h,k} B_hk (Wn Wn^T)_hk over the lower MT x MT tile pairs of
// (h, k) (off-diagonal pairs count twice) and 64-wide chunks of d; one
// partial per CTA into part[blockIdx.x].
__global__ void __launch_bounds__(NT) k_t2(const double *__restrict__ mW,
                                           const double *__restrict__ B, int H, int D,
                                           int nchunk, double *__restrict__ part) {
    __shared__ double Wh[MT][64 + 1];
    __shared__ double Wk[MT][64 + 1];
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;
    const int p = blockIdx.x / nchunk, ch = blockIdx.x % nchunk;
    int tb = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while ((tb + 1) * (tb + 2) / 2 <= p) ++tb;
    while (tb * (tb + 1) / 2 > p) --tb;
    const int sb = p - tb * (tb + 1) / 2;
    const int dc = ch * 64;
    for (int e = tid; e < MT * 64; e += NT) {
        const int r = e / 64, d = e % 64;
        const int hh = tb * MT + r, kk = sb * MT + r;
        Wh[r][d] = (hh < H && dc + d < D) ? mW[(size_t)hh * D + dc + d] : 0.0;
        Wk[r][d] = (kk < H && dc + d < D) ? mW[(size_t)kk * D + dc + d] : 0.0;
    }
    __syncthreads();
    const int r = tid / MT, c = tid % MT;
    double g = 0.0;
#pragma unroll 16
    for (int d = 0; d < 64; ++d) g += Wh[r][d] * Wk[c][d];
    const int h = tb * MT + r, kk = sb * MT + c;
    double v = 0.0;
    if (h < H && kk < H) v = g * B[(size_t)h * H + kk] * (tb == sb ? 1.0 : 2.0);
    v = block_sum(v, red);
    if (tid == 0) part[blockIdx.x] = v;
}

// pi, sigma (and GSC mu, psi).  t1, t2 are the sums of the partials written by
// k_backsub (n1 values) and k_t2 (n2 values), added in a fixed order.
__global__ void __launch_bounds__(NT) k_theta(const double *__restrict__ scal,
                                              const double *__restrict__ part, int n1, int n2,
                                              const double *__restrict__ gsc, double *theta,
                                              float *mu, float *psi, int H, int D, double Ntot,
                                              int model, unsigned *status) {
    __shared__ double red[NT / 32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n1; i += NT) a += part[i];
    for (int i = threadIdx.x; i < n2; i += NT) b += part[n1 + i];
    const double t1 = block_sum(a, red);
    const double t2 = block_sum(b, red);
    if (threadIdx.x == 0) {
        theta[PROSPER_TH_PI] = scal[PROSPER_SC_S1] / (Ntot * H);
        double s2;
        if (model == PROSPER_MCA) s2 = scal[PROSPER_SC_MCA_R2] / (Ntot * D);
        else s2 = (scal[PROSPER_SC_YY] - 2.0 * t1 + t2) / (Ntot * D);
        theta[PROSPER_TH_SIGMA] = sqrt(s2 > 0.0 ? s2 : 0.0);
        if (!isfinite(s2) || !isfinite(theta[PROSPER_TH_PI])) atomicOr(status, ST_NONFINITE);
    }
    if (model == PROSPER_GSC) {
        for (int h = threadIdx.x; h < H; h += NT) {
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

int mstep_hq(int H) { return (H + MB - 1) / MB * MB; }

int mstep_nparts(int H, int D) {
    const int Hq = mstep_hq(H), nT = (H + MT - 1) / MT;
    return (Hq / 8) * ((D + MB - 1) / MB) + nT * (nT + 1) / 2 * ((D + 63) / 64);
}

int launch_mstep(prosper_ctx *c, const prosper_stats *st, int64_t N, prosper_params *p,
                 cudaStream_t s) {
    const int H = c->H, D = c->D;
    const double Ntot = (double)N;
    if (c->model == PROSPER_MCA) {
        TraceScope tr(c, "mstep", s, 2);
        k_mca_w<<<c->num_sms * 4, 256, 0, s>>>(st->mca, p->W, H, D);
        PROSPER_LAUNCH_CHECK();
        k_theta<<<1, NT, 0, s>>>(st->scal, c->mpart, 0, 0, nullptr, p->theta, nullptr, nullptr, H, D,
                                 Ntot, c->model, c->d_status);
        PROSPER_LAUNCH_CHECK();
        return PROSPER_OK;
    }
    const int Hq = mstep_hq(H), NB = Hq / MB;
    const int nxt16 = (D + MT - 1) / MT, ncolx = (D + MB - 1) / MB;
    const int nct = (D + MB - 1) / MB, n1 = (Hq / 8) * nct;
    const int nT = (H + MT - 1) / MT, nchunk = (D + 63) / 64, n2 = nT * (nT + 1) / 2 * nchunk;
    TraceScope tr(c, "mstep", s, 4 + 2 * NB - 1);
    const int64_t nbuild = 2 * (int64_t)Hq * Hq + (int64_t)Hq * D;
    k_build<<<(int)std::min<int64_t>((nbuild + NT - 1) / NT, 4 * c->num_sms), NT, 0, s>>>(
        st->B, st->At, p->W, H, Hq, D, Ntot, c->mB, c->mX, c->mI);
    PROSPER_LAUNCH_CHECK();
    for (int k = 0; k < NB; ++k) {
        const int m = NB - 1 - k;                 // row blocks below the diagonal block
        k_panel<<<m + ncolx + (k + 1), NT, 0, s>>>(c->mB, c->mX, c->mI, Hq, D, k, m, ncolx,
                                                   c->d_status);
        PROSPER_LAUNCH_CHECK();
        if (m == 0) continue;
        const int nbt = m * (2 * m + 1);          // lower 16x16 tiles of the trailing block
        const int nrt = nxt16 + 2 * (k + 1);      // 16-column tiles of [mX | mI(:, <= k)]
        k_update<<<nbt + 2 * m * nrt, NT, 0, s>>>(c->mB, c->mX, c->mI, Hq, D, k, nbt, nxt16, nrt);
        PROSPER_LAUNCH_CHECK();
    }
    k_backsub<<<n1, NT, 0, s>>>(c->mI, c->mX, st->At, H, Hq, D, nct, c->mW, p->W, c->mpart);
    PROSPER_LAUNCH_CHECK();
    k_t2<<<n2, NT, 0, s>>>(c->mW, st->B, H, D, nchunk, c->mpart + n1);
    PROSPER_LAUNCH_CHECK();
    k_theta<<<1, NT, 0, s>>>(st->scal, c->mpart, n1, n2, st->gsc, p->theta, p->mu, p->psi, H, D,
                             Ntot, c->model, c->d_status);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

}  // namespace prosper
