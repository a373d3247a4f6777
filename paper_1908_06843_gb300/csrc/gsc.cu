// gsc.cu -- Gaussian Sparse Coding (Table 1, row GSC: linear superposition,
// Gaussian noise, spike-and-slab prior s_h = b_h z_h, b_h ~ Bernoulli(pi),
// z_h ~ N(mu_h, psi_h)) truncated E-step.
//
// For an active set b (k = |b| units) the data are Gaussian given b:
//   y | b ~ N(W_b mu_b, C_b),  C_b = sigma^2 I + W_b Psi_b W_b^T.
// With M_b = Psi_b^-1 + G_bb / sigma^2 (G = W^T W), Woodbury and the matrix
// determinant lemma give, relative to the empty state,
//   l(b) - l(0) = k log(pi/(1-pi)) - (log|Psi_b| + log|M_b|)/2
//                 - (r_b / sigma^2 - u_b^T M_b^-1 u_b / sigma^4)/2,
//   u_b = p_b - G_bb mu_b,  r_b = -2 mu_b^T p_b + mu_b^T G_bb mu_b,  p = W^T y,
// and the slab posterior is N(kappa_b, M_b^-1), kappa_b = M_b^-1 (p_b/sigma^2 + Psi_b^-1 mu_b).
// log|Psi_b| + log|M_b| and M_b^-1 do not depend on y: k_gsc_table computes
// them in FP64 for every subset of at most gamma (<= 3) latents once per call
// (row-a0 constants); the per-state arithmetic is FP32.
// Preselection score (reading): the singleton log-joint l(e_h).
// The E-step kernel and its launch templates are in gsc_estep.cuh.
#include "gsc_estep.cuh"

namespace prosper {
namespace {

// One thread per nonempty subset of at most gamma latents: FP64 Cholesky of
// M_b, log|Psi_b| + log|M_b| and M_b^-1 (packed upper triangle).
__global__ void k_gsc_table(const float *__restrict__ G, const float *__restrict__ psi,
                            const double *__restrict__ theta, int H, int gamma, int nsub,
                            float *__restrict__ tab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsub) return;
    const double sigma = theta[PROSPER_TH_SIGMA];
    const double is2 = 1.0 / (sigma * sigma);
    // size class and colex rank
    int k = 1;
    int64_t r = t;
    while (k < gamma && r >= binom_small(H, k)) { r -= binom_small(H, k); ++k; }
    int b[3] = {0, 0, 0};
    for (int i = k - 1; i >= 0; --i) {
        int c = i;
        while (binom_small(c + 1, i + 1) <= r) ++c;
        b[i] = c;
        r -= binom_small(c, i + 1);
    }
    double M[3][3], L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double logpsi = 0.0;
    for (int i = 0; i < k; ++i) {
        logpsi += log((double)psi[b[i]]);
        for (int j = 0; j < k; ++j)
            M[i][j] = (i == j ? 1.0 / (double)psi[b[i]] : 0.0) + is2 * (double)G[(size_t)b[i] * H + b[j]];
    }
    double logdetM = 0.0;
    for (int j = 0; j < k; ++j) {
        double d = M[j][j];
        for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q];
        d = d > 0.0 ? d : 1e-300;
        L[j][j] = sqrt(d);
        logdetM += 2.0 * log(L[j][j]);
        for (int i = j + 1; i < k; ++i) {
            double s = M[i][j];
            for (int q = 0; q < j; ++q) s -= L[i][q] * L[j][q];
            L[i][j] = s / L[j][j];
        }
    }
    double Mi[3][3];
    for (int c = 0; c < k; ++c) {          // solve M x = e_c
        double x[3];
        for (int i = 0; i < k; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int q = 0; q < i; ++q) s -= L[i][q] * x[q];
            x[i] = s / L[i][i];
        }
        for (int i = k - 1; i >= 0; --i) {
            double s = x[i];
            for (int q = i + 1; q < k; ++q) s -= L[q][i] * x[q];
            x[i] = s / L[i][i];
        }
        for (int i = 0; i < k; ++i) Mi[i][c] = x[i];
    }
    float *o = tab + (size_t)t * TAB;
    o[0] = (float)(logpsi + logdetM);
    o[1] = (float)Mi[0][0];
    o[2] = k > 1 ? (float)Mi[0][1] : 0.f;
    o[3] = k > 2 ? (float)Mi[0][2] : 0.f;
    o[4] = k > 1 ? (float)Mi[1][1] : 0.f;
    o[5] = k > 2 ? (float)Mi[1][2] : 0.f;
    o[6] = k > 2 ? (float)Mi[2][2] : 0.f;
    o[7] = 0.f;
}

}  // namespace

size_t gsc_smem_hp(int D, int H, int Hp, int nK) {
    const size_t slots = 2 * (size_t)Hp + (size_t)Hp * (Hp + 1) / 2;   // Slots<Hp>::N
    size_t f = (size_t)H * D + (size_t)H * H + ((nK + 3) & ~3) + 2 * (size_t)((H + 3) & ~3);
    f += (size_t)GW * (slots * 32 + 64 + 3 * H + H * D);
    f += (size_t)GW * D;                 // per-warp y buffers
    f += (size_t)GW * nK * TAB + 4;      // per-warp subset-table rows (+ alignment slack)
    return f * sizeof(float);
}

size_t gsc_smem_bytes(int D, int H, int Hp, int nK) { return gsc_smem_hp(D, H, Hp, nK); }

int launch_gsc_prep(prosper_ctx *c, const prosper_params *p, cudaStream_t s) {
    int rc = launch_bsc_prep(c, p->W, s);     // G = W^T W (and 1/||W_h||)
    if (rc) return rc;
    TraceScope tr(c, "gsc_table", s);
    k_gsc_table<<<(c->gsc_nsub + 127) / 128, 128, 0, s>>>(c->G, p->psi, p->theta, c->H, c->gamma,
                                                          c->gsc_nsub, c->gsc_tab);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

int launch_gsc_estep(prosper_ctx *c, const prosper_params *p, const float *Y, int64_t N,
                     prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                     float *mapp_out, float *logz_out, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    if (c->H > 32) {
        set_error("GSC: H=%d > 32", c->H);
        return PROSPER_EINVAL;
    }
    GscArgs A;
    A.W = p->W; A.Y = Y; A.mu = p->mu; A.psi = p->psi; A.G = c->G; A.tab = c->gsc_tab;
    A.theta = p->theta; A.N = N; A.D = c->D; A.H = c->H; A.Hp = c->Hp; A.gamma = c->gamma;
    A.nK = c->nK;
    A.At = st ? st->At : nullptr; A.B = st ? st->B : nullptr;
    A.scal = st ? st->scal : nullptr; A.gsc = st ? st->gsc : nullptr;
    A.sel_out = sel_out; A.map_out = map_out; A.smean_out = smean_out; A.mapp_out = mapp_out;
    A.logz_out = logz_out;
    const bool enc = (st == nullptr);
    const int64_t warps = (N + 3) / 4;
    const int grid = (int)std::min<int64_t>((warps + GW - 1) / GW, (int64_t)c->num_sms);
    TraceScope tr(c, enc ? "gsc_encode" : "gsc_estep", s);
    if (c->Hp <= 3) return gsc_launch_1_3(c->Hp, A, enc, grid, s);
    if (c->Hp <= 6) return gsc_launch_4_6(c->Hp, A, enc, grid, s);
    if (c->Hp <= 8) return gsc_launch_7_8(c->Hp, A, enc, grid, s);
    return gsc_launch_9_10(c->Hp, A, enc, grid, s);
}

}  // namespace prosper
