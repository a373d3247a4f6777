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

__device__ __forceinline__ bool unit_active(const double *__restrict__ B, int H, int h, double thr) {
    return h < H && B[(size_t)h * H + h] > thr;
}

// Builds the augmented system [mB | mX | mI] of order Hq = H rounded up to MB:
//   mB = B on the active block (+ ridge 1e-9 tr(B)/H), identity elsewhere
//        (inactive units and the padding rows/columns);
//   mX = At on active rows, the old W on inactive rows, 0 on padding rows;
//   mI = identity;  mZ (the factor's inverse, filled block by block) = 0.
// Every CTA forms tr(B) itself (H loads), so no separate launch is needed.
__global__ void __launch_bounds__(NT) k_build(const double *__restrict__ B,
                                              const double *__restrict__ At,
                                              const float *__restrict__ W, int H, int Hq, int D,
                                              double Ntot, double *__restrict__ mB,
                                              double *__restrict__ mX, double *__restrict__ mI,
                                              double *__restrict__ mZ) {
    __shared__ double red[NT / 32];
    __shared__ double ridge_s;
    double tr = 0.0;
    for (int h = threadIdx.x; h < H; h += NT) tr += B[(size_t)h * H + h];
    tr = block_sum(tr, red);
    if (threadIdx.x == 0) ridge_s = 1e-9 * tr / H;
    __syncthreads();
    const double ridge = ridge_s, thr = 1e-9 * Ntot;
    const int64_t nB = (int64_t)Hq * Hq, nX = (int64_t)Hq * D;
    for (int64_t idx = (int64_t)blockIdx.x * NT + threadIdx.x; idx < 2 * nB + nX;
         idx += (int64_t)gridDim.x * NT) {
        if (idx < nB) {
            const int i = (int)(idx / Hq), j = (int)(idx % Hq);
            double v = (i == j) ? 1.0 : 0.0;
            if (unit_active(B, H, i, thr) && unit_active(B, H, j, thr))
                v = B[(size_t)i * H + j] + (i == j ? ridge : 0.0);
            mB[idx] = v;
        } else if (idx < 2 * nB) {
            const int64_t e = idx - nB;
            mI[e] = (e / Hq == e % Hq) ? 1.0 : 0.0;
            mZ[e] = 0.0;
        } else {
            const int64_t e = idx - 2 * nB;
            const int h = (int)(e / D);
            double v = 0.0;
            if (h < H) v = unit_active(B, H, h, thr) ? At[e] : (double)W[e];
            mX[e] = v;
        }
    }
}

// 1/sqrt(d) to about 1e-13 relative: single-precision estimate refined by one
// Newton-Raphson step for the reciprocal square root, y <- y (3 - d y^2)/2,
// in FP64.  Outside the single-precision range the FP64 library routine is used.
__device__ __forceinline__ double rsqrt_pivot(double d) {
    if (!(d > 1e-30 && d < 1e30)) return rsqrt(d);
    const double y = (double)rsqrtf((float)d);
    const double e = fma(-(d * y), y, 1.0);
    return fma(0.5 * y, e, y);
}

// Step k of the blocked right-looking Cholesky factorisation B = L L^T
// (Golub & Van Loan, Matrix Computations, Sec. 4.2; block MB), carried along
// the right-hand sides [mX | mI] so that the forward substitution happens in
// the same pass.
//
// Every CTA factors the diagonal block A_kk in shared memory together with its
// inverse Z = L_kk^-1 (right-looking: pivot t scales column t of A and row t
// of Z by 1/sqrt(pivot), then the trailing triangle and the rows of Z below t
// take the rank-1 update; the updates of one pivot are packed over all warps).
// Then CTA pair (2 q, 2 q + 1) forms one 32 x 32 output tile as a product with Z:
//   q <  nrow : panel  P_i = A_ik Z^T           for row block i = k + 1 + q
//   q >= nrow : Y_k    = Z R_k                 for a 32-column tile of mX, or of
//               the identity block columns j <= k of mI (the others are still
//               zero in row block k); Y goes to mY / mZ.
// Each CTA of a pair takes 16 of the 32 output columns (or rows), in pairs
// (e, 31 - e) so that every warp does the same number of multiply-adds.
// Outputs go to buffers this launch does not read.  CTA 0 reports a
// non-positive pivot (the pivot is then taken as 1).
__global__ void __launch_bounds__(NT) k_panel(const double *__restrict__ mB,
                                              const double *__restrict__ mX,
                                              const double *__restrict__ mI, double *__restrict__ P,
                                              double *__restrict__ mY, double *__restrict__ mZ,
                                              int Hq, int D, int k, int nrow, int ncolx,
                                              unsigned *status) {
    __shared__ double A[MB][MB + 1];
    __shared__ double Z[MB][MB + 1];
    __shared__ double T[MB][MB + 1];
    __shared__ uint8_t tri_u[MB * (MB + 1) / 2], tri_c[MB * (MB + 1) / 2];
    __shared__ int fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = k * MB;
    const int q = blockIdx.x >> 1, half = blockIdx.x & 1;
    const bool rowrole = q < nrow;
    const double *R;
    int ld, r0, c0, ncols;
    if (rowrole) {
        R = mB; ld = Hq; r0 = k0 + MB * (q + 1); c0 = k0; ncols = MB;
    } else if (q - nrow < ncolx) {
        R = mX; ld = D; r0 = k0; c0 = (q - nrow) * MB; ncols = min(MB, D - c0);
    } else {
        R = mI; ld = Hq; r0 = k0; c0 = (q - nrow - ncolx) * MB; ncols = MB;
    }
    for (int e = tid; e < MB * MB; e += NT) {
        const int r = e / MB, c = e % MB;
        A[r][c] = mB[(size_t)(k0 + r) * Hq + k0 + c];
        Z[r][c] = (r == c) ? 1.0 : 0.0;
        T[r][c] = c < ncols ? R[(size_t)(r0 + r) * ld + c0 + c] : 0.0;
    }
    // lower-triangle entries (u, c), c <= u, listed from column MB-1 down to 0:
    // those with c > t are exactly the first (MB-1-t)(MB-t)/2
    for (int e = tid; e < MB * (MB + 1) / 2; e += NT) {
        int m = 0;
        while ((m + 1) * (m + 2) / 2 <= e) ++m;
        const int c = MB - 1 - m;
        tri_c[e] = (uint8_t)c;
        tri_u[e] = (uint8_t)(c + e - m * (m + 1) / 2);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int t = 0; t < MB; ++t) {
        if (warp == 0) {
            double d = A[t][t];
            const bool bad = !(d > 0.0);
            if (bad) d = 1.0;
            const double r = rsqrt_pivot(d);
            if (lane > t) A[lane][t] *= r;
            else Z[t][lane] *= r;
            if (lane == 0 && bad) fail = 1;
        }
        __syncthreads();
        const int n = MB - 1 - t, ntri = n * (n + 1) / 2, tot = ntri + n * (t + 1);
        for (int e = tid; e < tot; e += NT) {
            if (e < ntri) {
                const int u = tri_u[e], c = tri_c[e];
                A[u][c] -= A[u][t] * A[c][t];
            } else {
                const int e2 = e - ntri, u = t + 1 + e2 / (t + 1), j = e2 % (t + 1);
                Z[u][j] -= A[u][t] * Z[t][j];
            }
        }
        __syncthreads();
    }
    // row role  : P[r][e] = sum_{t <= e} A_ik[r][t] Z[e][t]     (lane = r)
    // column role: Y[e][c] = sum_{t <= e} Z[e][t] R_k[t][c]     (lane = c)
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        const int e0 = half * 8 + warp, e = pass ? MB - 1 - e0 : e0;
        double acc = 0.0;
        if (rowrole) {
            for (int t = 0; t <= e; ++t) acc += T[lane][t] * Z[e][t];
            P[(size_t)(r0 + lane) * MB + e] = acc;
        } else {
            for (int t = 0; t <= e; ++t) acc += Z[e][t] * T[t][lane];
            if (lane < ncols) {
                if (R == mX) mY[(size_t)(k0 + e) * D + c0 + lane] = acc;
                else mZ[(size_t)(k0 + e) * Hq + c0 + lane] = acc;
            }
        }
    }
    if (blockIdx.x == 0 && tid == 0 && fail) atomicOr(status, ST_CHOL_FAIL);
}

// Trailing update of step k on MT x MT tiles:
//   tiles [0, nbt)    : A_ij -= P_i P_j^T, the lower tiles of the rows/columns > k
//   tiles [nbt, grid) : R_i  -= P_i Y_k  for the row blocks i > k, over the
//                       16-column tiles of mX and of mI's block columns <= k.
__global__ void __launch_bounds__(NT) k_update(double *__restrict__ mB, double *__restrict__ mX,
                                               double *__restrict__ mI,
                                               const double *__restrict__ P,
                                               const double *__restrict__ mY,
                                               const double *__restrict__ mZ, int Hq, int D, int k,
                                               int nbt, int nxt, int nrt) {
    __shared__ double As[MT][MB + 1];
    __shared__ double Bs[MB][MT + 1];
    const int tid = threadIdx.x;
    const int k0 = k * MB, base = k0 + MB;
    int x = blockIdx.x, row0, col0, ld, ncols;
    double *out;
    const double *src = nullptr;
    if (x < nbt) {
        int si = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
        while ((si + 1) * (si + 2) / 2 <= x) ++si;
        while (si * (si + 1) / 2 > x) --si;
        const int sj = x - si * (si + 1) / 2;
        row0 = base + si * MT;
        col0 = base + sj * MT;
        out = mB; ld = Hq; ncols = MT;
    } else {
        x -= nbt;
        const int si = x / nrt, ct = x % nrt;
        row0 = base + si * MT;
        if (ct < nxt) { out = mX; src = mY; ld = D; col0 = ct * MT; ncols = min(MT, D - col0); }
        else { out = mI; src = mZ; ld = Hq; col0 = (ct - nxt) * MT; ncols = MT; }
    }
    for (int e = tid; e < MT * MB; e += NT) {
        const int r = e / MB, t = e % MB;
        As[r][t] = P[(size_t)(row0 + r) * MB + t];
        if (src == nullptr) Bs[t][r] = P[(size_t)(col0 + r) * MB + t];
    }
    if (src != nullptr)
        for (int e = tid; e < MB * MT; e += NT) {
            const int t = e / MT, c = e % MT;
            Bs[t][c] = c < ncols ? src[(size_t)(k0 + t) * ld + col0 + c] : 0.0;
        }
    __syncthreads();
    const int r = tid / MT, c = tid % MT;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < MB; ++t) acc += As[r][t] * Bs[t][c];
    if (c < ncols) out[(size_t)(row0 + r) * ld + col0 + c] -= acc;
}

// Back substitution with the explicit inverse: mZ holds L^-1 (lower
// triangular) and mY holds L^-1 X, so W^T = L^-T (L^-1 X):
//   Wn[i][d] = sum_{t >= i} Linv[t][i] Y[t][d]
// One CTA takes the 8-row tiles p and nti-1-p (equal work) of one 32-column
// tile.  Writes Wn in FP64 (mW, H x D) and FP32 (W), and three partials:
//   part[3b]   = sum over active rows of Wn . At
//   part[3b+1] = sum over inactive rows of Wn . At
//   part[3b+2] = sum over active rows of Wn . Wn
__global__ void __launch_bounds__(NT) k_backsub(const double *__restrict__ mZ,
                                                const double *__restrict__ mY,
                                                const double *__restrict__ At,
                                                const double *__restrict__ B, int H, int Hq,
                                                int D, int nct, double Ntot,
                                                double *__restrict__ mW, float *__restrict__ W,
                                                double *__restrict__ part) {
    __shared__ double Ls[MB][8 + 1];
    __shared__ double Ys[MB][MB + 1];
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, r = tid >> 5;
    const int nti = Hq / 8, p = blockIdx.x / nct, d0 = (blockIdx.x % nct) * MB;
    const int dcol = d0 + lane;
    const double thr = 1e-9 * Ntot;
    double pa = 0.0, pi = 0.0, qa = 0.0;
    for (int which = 0; which < 2; ++which) {
        const int i0 = (which ? nti - 1 - p : p) * 8;
        double acc = 0.0;
        for (int t0 = i0; t0 < Hq; t0 += MB) {
            {
                const int t = tid >> 3, rr = tid & 7;
                Ls[t][rr] = (t0 + t < Hq) ? mZ[(size_t)(t0 + t) * Hq + i0 + rr] : 0.0;
            }
            for (int e = tid; e < MB * MB; e += NT) {
                const int t = e / MB, c = e % MB;
                Ys[t][c] = (t0 + t < Hq && d0 + c < D) ? mY[(size_t)(t0 + t) * D + d0 + c] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < MB; ++t) acc += Ls[t][r] * Ys[t][lane];
            __syncthreads();
        }
        const int h = i0 + r;
        if (h < H && dcol < D) {
            const size_t o = (size_t)h * D + dcol;
            mW[o] = acc;
            W[o] = (float)acc;
            if (unit_active(B, H, h, thr)) { pa += acc * At[o]; qa += acc * acc; }
            else pi += acc * At[o];
        }
    }
    pa = block_sum(pa, red);
    pi = block_sum(pi, red);
    qa = block_sum(qa, red);
    if (tid == 0) {
        part[3 * blockIdx.x] = pa;
        part[3 * blockIdx.x + 1] = pi;
        part[3 * blockIdx.x + 2] = qa;
    }
}

// tr(W^T W B) = sum_{h,k} B_hk (Wn Wn^T)_hk.  On the active block the solve
// gives B_aa Wn_a = At_a - ridge Wn_a, so that part equals
//   sum_a Wn_a . At_a - ridge sum_a ||Wn_a||^2
// (from the k_backsub partials).  This kernel adds the pairs that involve a
// never-active unit i: CTA (i, 32-row block of h) writes
//   sum_h B_hi (Wn_h . Wn_i) (2 if h is active, else 1),
// and 0 when i is active.
__global__ void __launch_bounds__(NT) k_t2_inactive(const double *__restrict__ mW,
                                                    const double *__restrict__ B, int H, int D,
                                                    double Ntot, double *__restrict__ part) {
    __shared__ double red[NT / 32];
    const int i = blockIdx.x / ((H + 31) / 32), hb = blockIdx.x % ((H + 31) / 32);
    const double thr = 1e-9 * Ntot;
    if (unit_active(B, H, i, thr)) {
        if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v = 0.0;
    for (int hh = warp; hh < 32; hh += NT / 32) {
        const int h = hb * 32 + hh;
        if (h >= H) break;
        double g = 0.0;
        for (int d = lane; d < D; d += 32) g += mW[(size_t)h * D + d] * mW[(size_t)i * D + d];
        v += g * B[(size_t)h * H + i] * (unit_active(B, H, h, thr) ? 2.0 : 1.0);
    }
    v = block_sum(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// pi, sigma (and GSC mu, psi).  t1 = tr(W^T A) and t2 = tr(W^T W B) from the
// partials of k_backsub (n1 triples) and k_t2_inactive (n2 values), added in a
// fixed order.
__global__ void __launch_bounds__(NT) k_theta(const double *__restrict__ scal,
                                              const double *__restrict__ part, int n1, int n2,
                                              const double *__restrict__ B,
                                              const double *__restrict__ gsc, double *theta,
                                              float *mu, float *psi, int H, int D, double Ntot,
                                              int model, int nvals, int cut_gamma,
                                              unsigned *status) {
    __shared__ double red[NT / 32];
    double pa = 0.0, pi = 0.0, qa = 0.0, x = 0.0, tr = 0.0;
    for (int i = threadIdx.x; i < n1; i += NT) {
        pa += part[3 * i]; pi += part[3 * i + 1]; qa += part[3 * i + 2];
    }
    for (int i = threadIdx.x; i < n2; i += NT) x += part[3 * n1 + i];
    if (B != nullptr)
        for (int h = threadIdx.x; h < H; h += NT) tr += B[(size_t)h * H + h];
    pa = block_sum(pa, red);
    pi = block_sum(pi, red);
    qa = block_sum(qa, red);
    x = block_sum(x, red);
    tr = block_sum(tr, red);
    if (threadIdx.x == 0) {
        const double pi_old = theta[PROSPER_TH_PI];
        theta[PROSPER_TH_PI] = scal[PROSPER_SC_S1] / (Ntot * H);
        if (cut_gamma >= 0 && cut_gamma < H) {
            // data cut: the kept points favour few causes; scale by
            // H pi / E_pi[|s| : |s| <= gamma] at the current pi
            double w = 1.0, sw = 0.0, skw = 0.0;
            for (int k = 0; k <= cut_gamma; ++k) {
                sw += w;
                skw += k * w;
                w *= (double)(H - k) / (k + 1) * pi_old / (1.0 - pi_old);
            }
            const double mean = skw / sw;
            if (mean > 0.0) theta[PROSPER_TH_PI] *= H * pi_old / mean;
        }
        double s2;
        if (model == PROSPER_MCA || model == PROSPER_MMCA) {
            s2 = scal[PROSPER_SC_MCA_R2] / (Ntot * D);
        } else {
            const double ridge = 1e-9 * tr / H;
            const double t1 = pa + pi, t2 = pa - ridge * qa + x;
            s2 = (scal[PROSPER_SC_YY] - 2.0 * t1 + t2) / (Ntot * D);
        }
        theta[PROSPER_TH_SIGMA] = sqrt(s2 > 0.0 ? s2 : 0.0);
        if (!isfinite(s2) || !isfinite(theta[PROSPER_TH_PI])) atomicOr(status, ST_NONFINITE);
        // DSC: each nonzero value's probability is its expected frequency (the
        // categorical argmax of Q); TSC keeps p(+-1) = pi/2 through pi alone
        if (model == PROSPER_DSC)
            for (int v = 0; v < nvals; ++v)
                theta[PROSPER_TH_DSC_P + v] = scal[PROSPER_SC_DSC0 + v] / (Ntot * H);
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

// W_dh = sum<A_dh> y_d / sum<A_dh> (kept where the denominator is 0); MCA
// clamps W >= 1e-6 (its powers need W > 0), MMCA's W is signed
__global__ void k_mca_w(const double *__restrict__ mca, float *W, int H, int D, int clamp) {
    const int64_t HD = (int64_t)H * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < HD;
         i += (int64_t)gridDim.x * blockDim.x) {
        double num = mca[i], den = mca[HD + i];
        if (den > 0.0) {
            double w = num / den;
            W[i] = (float)((clamp && w < 1e-6) ? 1e-6 : w);
        }
    }
}

}  // namespace

int mstep_hq(int H) { return (H + MB - 1) / MB * MB; }

static int mstep_n1(int H, int D) { return (mstep_hq(H) / 16) * ((D + MB - 1) / MB); }
static int mstep_n2(int H) { return H * ((H + 31) / 32); }

int mstep_nparts(int H, int D) { return 3 * mstep_n1(H, D) + mstep_n2(H); }

int launch_mstep(prosper_ctx *c, const prosper_stats *st, int64_t N, prosper_params *p,
                 cudaStream_t s) {
    const int H = c->H, D = c->D;
    const double Ntot = (double)N;
    if (c->model == PROSPER_MCA || c->model == PROSPER_MMCA) {
        TraceScope tr(c, "mstep", s, 2);
        k_mca_w<<<c->num_sms * 4, 256, 0, s>>>(st->mca, p->W, H, D, c->model == PROSPER_MCA);
        PROSPER_LAUNCH_CHECK();
        k_theta<<<1, NT, 0, s>>>(st->scal, nullptr, 0, 0, nullptr, nullptr, p->theta, nullptr,
                                 nullptr, H, D, Ntot, c->model, 0, -1, c->d_status);
        PROSPER_LAUNCH_CHECK();
        return PROSPER_OK;
    }
    const int Hq = mstep_hq(H), NB = Hq / MB;
    const int nxt16 = (D + MT - 1) / MT, ncolx = (D + MB - 1) / MB;
    const int n1 = mstep_n1(H, D), n2 = mstep_n2(H);
    TraceScope tr(c, "mstep", s, 2 * NB + 3);
    const int64_t nbuild = 2 * (int64_t)Hq * Hq + (int64_t)Hq * D;
    k_build<<<(int)std::min<int64_t>((nbuild + NT - 1) / NT, 4 * c->num_sms), NT, 0, s>>>(
        st->B, st->At, p->W, H, Hq, D, Ntot, c->mB, c->mX, c->mI, c->mZ);
    PROSPER_LAUNCH_CHECK();
    for (int k = 0; k < NB; ++k) {
        const int m = NB - 1 - k;                 // row blocks below the diagonal block
        k_panel<<<2 * (m + ncolx + k + 1), NT, 0, s>>>(c->mB, c->mX, c->mI, c->mP, c->mY, c->mZ,
                                                       Hq, D, k, m, ncolx, c->d_status);
        PROSPER_LAUNCH_CHECK();
        if (m == 0) continue;
        const int nbt = m * (2 * m + 1);          // lower 16x16 tiles of the trailing block
        const int nrt = nxt16 + 2 * (k + 1);      // 16-column tiles of [mX | mI(:, <= k)]
        k_update<<<nbt + 2 * m * nrt, NT, 0, s>>>(c->mB, c->mX, c->mI, c->mP, c->mY, c->mZ, Hq, D,
                                                  k, nbt, nxt16, nrt);
        PROSPER_LAUNCH_CHECK();
    }
    k_backsub<<<n1, NT, 0, s>>>(c->mZ, c->mY, st->At, st->B, H, Hq, D, (D + MB - 1) / MB, Ntot,
                                c->mW, p->W, c->mpart);
    PROSPER_LAUNCH_CHECK();
    k_t2_inactive<<<n2, NT, 0, s>>>(c->mW, st->B, H, D, Ntot, c->mpart + 3 * n1);
    PROSPER_LAUNCH_CHECK();
    k_theta<<<1, NT, 0, s>>>(st->scal, c->mpart, n1, n2, st->B, st->gsc, p->theta, p->mu, p->psi,
                             H, D, Ntot, c->model, c->dsc_m, c->cut ? c->gamma : -1, c->d_status);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

}  // namespace prosper
