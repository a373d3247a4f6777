// gsc_estep.cuh -- the GSC E-step kernel k_gsc_estep (the method is described
// in gsc.cu) and its launch templates.  gsc_e1.cu .. gsc_e4.cu each
// instantiate it for a range of Hprime, so that the 80 instantiations
// (Hprime x pixel blocks x encode/E-step) compile in parallel.
#pragma once
#include "internal.cuh"
#include "topk.cuh"

#include <cmath>

namespace prosper {

struct GscArgs {
    const float *W, *Y, *mu, *psi, *G, *tab;
    const double *theta;
    int64_t N;
    int D, H, Hp, gamma, nK;
    double *At, *B, *scal, *gsc;
    int16_t *sel_out, *map_out;
    float *smean_out, *mapp_out, *logz_out;
};

// shared-memory bytes of one GSC E-step CTA (gsc.cu)
size_t gsc_smem_hp(int D, int H, int Hp, int nK);
// the launches for Hprime 1..3, 4..6, 7..8 and 9..10 (gsc_e1.cu .. gsc_e4.cu)
int gsc_launch_1_3(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s);
int gsc_launch_4_6(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s);
int gsc_launch_7_8(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s);
int gsc_launch_9_10(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s);

namespace {

constexpr int GW = 8;   // warps per CTA
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2Pi = 1.8378770664093454836;
constexpr int TAB = 8;  // floats per subset: logdet, Minv 00 01 02 11 12 22, pad

__host__ __device__ inline int64_t binom_small(int n, int k) {
    if (k < 0 || n < k) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}
// C(n, k) for k <= 3 without division loops (64-bit integer division is a
// long software sequence on the GPU; this runs for every state of every point)
__device__ __forceinline__ int binom3(int n, int k) {
    if (n < k) return 0;
    return k == 0 ? 1 : k == 1 ? n : k == 2 ? n * (n - 1) / 2 : n * (n - 1) * (n - 2) / 6;
}
// first index of the size-k block (blocks ordered by size, colex inside)
__host__ __device__ inline int64_t sub_offset(int H, int k) {
    int64_t o = 0;
    for (int j = 1; j < k; ++j) o += binom_small(H, j);
    return o;
}

__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// acc (hi, lo) += v with Knuth's TwoSum (hi + lo carries about 48 bits)
__device__ __forceinline__ void two_sum_acc(float2 &acc, float v) {
    const float s = acc.x + v;
    const float bb = s - acc.x;
    acc.y += (acc.x - (s - bb)) + (v - bb);
    acc.x = s;
}
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// per-lane accumulator slots: <b_j> (HP), <s_j> (HP), <s_i s_j> (i <= j)
template <int HP>
struct Slots {
    static constexpr int NB = 0, NS = HP, NP = 2 * HP;
    static constexpr int N = 2 * HP + HP * (HP + 1) / 2;
    __device__ static int pair(int i, int j) { return NP + i * HP - i * (i - 1) / 2 + (j - i); }
};

template <int HP, int DK, bool ENCODE>
__global__ void __launch_bounds__(GW * 32, 1) k_gsc_estep(GscArgs A) {
    using S = Slots<HP>;
    extern __shared__ __align__(16) float sm[];
    const int D = A.D, H = A.H, gamma = A.gamma, nK = A.nK;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *Ws = sm;                                  // D x H (transposed: lane h reads row d)
    float *Gs = Ws + H * D;                          // H x H
    unsigned *Ks = reinterpret_cast<unsigned *>(Gs + H * H);   // nK canonical masks
    float *mus = reinterpret_cast<float *>(Ks + ((nK + 3) & ~3));   // mu (H)
    float *mpr = mus + ((H + 3) & ~3);                                // mu / psi (H)
    float *wbase = mpr + ((H + 3) & ~3);
    float *acc = wbase + warp * (S::N * 32 + 64 + 3 * H + H * D);   // per warp
    unsigned *scratch = reinterpret_cast<unsigned *>(acc + S::N * 32);
    float *gpart = acc + S::N * 32 + 64;             // 3H
    float *apart = gpart + 3 * H;                    // H x D

    for (int i = tid; i < H * D; i += GW * 32) Ws[(i % D) * H + i / D] = A.W[i];
    float *ysm = wbase + (size_t)GW * (S::N * 32 + 64 + 3 * H + H * D) + (size_t)warp * D;   // per warp
    // per warp: the subset-table row of each state, read from global memory in
    // the log-joint pass and reused by the moment pass (same lane, same state)
    float *trow = reinterpret_cast<float *>(
                      (reinterpret_cast<uintptr_t>(wbase + (size_t)GW * (S::N * 32 + 64 + 3 * H + H * D + D)) + 15) &
                      ~static_cast<uintptr_t>(15)) +
                  (size_t)warp * nK * TAB;   // 16-byte aligned (float4 stores)
    for (int h = tid; h < H; h += GW * 32) {
        mus[h] = A.mu[h];
        mpr[h] = A.mu[h] / A.psi[h];
    }
    for (int i = tid; i < H * H; i += GW * 32) Gs[i] = A.G[i];
    if (tid == 0) {   // canonical state masks: by size, then lexicographic
        int n = 0;
        for (int k = 0; k <= gamma; ++k) {
            // enumerate combinations of size k in lexicographic order
            int idx[HP + 1];
            for (int i = 0; i < k; ++i) idx[i] = i;
            for (;;) {
                unsigned m = 0;
                for (int i = 0; i < k; ++i) m |= 1u << idx[i];
                Ks[n++] = m;
                int i = k - 1;
                while (i >= 0 && idx[i] == HP - k + i) --i;
                if (i < 0) break;
                ++idx[i];
                for (int j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
            }
        }
    }
    if (!ENCODE)
        for (int i = lane; i < 3 * H + H * D; i += 32) gpart[i] = 0.f;
    __syncthreads();

    const double pi = A.theta[PROSPER_TH_PI], sigma = A.theta[PROSPER_TH_SIGMA];
    // deterministic annealing: log-joints divided by T (theta[3]; <= 0 reads as 1)
    const double Tth = A.theta[PROSPER_TH_T];
    const double T = Tth > 0.0 ? Tth : 1.0;
    const float L2E = (float)(1.4426950408889634 / T);
    const float lpi = (float)log(pi / (1.0 - pi));
    const float is2 = (float)(1.0 / (sigma * sigma));
    const float is4 = is2 * is2;
    const double logp00 = H * log(1.0 - pi) - 0.5 * D * (kLog2Pi + log(sigma * sigma));
    const double i2s2 = 0.5 / (sigma * sigma);
    // per-warp sums of F, sum<|s|> and y^T y as FP32 pairs (hi + lo, Knuth's
    // TwoSum): FP64 adds are ~65x slower than FP32 ones on this part
    float2 accF = make_float2(0.f, 0.f), accS1 = accF, accYY = accF;
    int accN = 0;

    const int64_t gw = (int64_t)blockIdx.x * GW + warp, nw = (int64_t)gridDim.x * GW;
    for (int64_t n = gw; n < A.N; n += nw) {
        float y[DK];
#pragma unroll
        for (int k = 0; k < DK; ++k) {
            const int d = lane + 32 * k;
            y[k] = d < D ? A.Y[n * D + d] : 0.f;
        }
        float yy = 0.f;
#pragma unroll
        for (int k = 0; k < DK; ++k) yy = fmaf(y[k], y[k], yy);
        yy = wsum(yy);
        // projections p_h: lane h forms W_h . y from the transposed dictionary
        // and the point's y staged in this warp's shared buffer (H <= 32)
#pragma unroll
        for (int k = 0; k < DK; ++k) {
            const int d = lane + 32 * k;
            if (d < D) ysm[d] = y[k];
        }
        __syncwarp();
        float ph = 0.f;
        if (lane < H) {
            float p0 = 0.f, p1 = 0.f;
            int d = 0;
            for (; d + 1 < D; d += 2) {
                p0 = fmaf(Ws[d * H + lane], ysm[d], p0);
                p1 = fmaf(Ws[(d + 1) * H + lane], ysm[d + 1], p1);
            }
            if (d < D) p0 = fmaf(Ws[d * H + lane], ysm[d], p0);
            ph = p0 + p1;
        }
        __syncwarp();
        // singleton log-joint (terms common to all h dropped) as the selection score
        unsigned key[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) key[j] = 0u;
        if (lane < H) {
            const float g = Gs[lane * H + lane], m_ = A.mu[lane], ps = A.psi[lane];
            const float Mh = 1.f / ps + g * is2;
            const float u = ph - g * m_;
            const float sc = -0.5f * (logf(ps) + logf(Mh)) - 0.5f * ((-2.f * m_ * ph + m_ * m_ * g) * is2 -
                                                                      u * u * is4 / Mh);
            key[0] = score_key(sc);
        }
        const int myh = warp_topk(key, A.Hp, lane, scratch);
        __syncwarp();
        const int rank = topk_rank(myh, A.Hp, lane);
        int I[HP];
        float pI[HP];
#pragma unroll
        for (int j = 0; j < HP; ++j) {
            const unsigned ball = __ballot_sync(0xffffffffu, lane < HP && rank == j);
            I[j] = __shfl_sync(0xffffffffu, myh, __ffs(ball) - 1);
            pI[j] = __shfl_sync(0xffffffffu, ph, I[j]);
        }
        // ---- states: lane v takes states v, v + 32, ...
        float lv[8];            // nK <= 1 + 10 + 45 + 120 = 176 states -> <= 6 per lane
        float m = -INFINITY;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int v = lane + 32 * r;
            lv[r] = -INFINITY;
            if (v < nK) {
                const unsigned mk = Ks[v];
                const int k = __popc(mk);
                float l = 0.f;
                if (k > 0) {
                    int bl[3] = {0, 0, 0}, bg[3] = {0, 0, 0};
                    int q = 0;
#pragma unroll
                    for (int j = 0; j < HP; ++j)
                        if (((mk >> j) & 1u) && q < 3) { bl[q] = j; bg[q] = I[j]; ++q; }
                    int rk = (k > 1 ? H : 0) + (k > 2 ? H * (H - 1) / 2 : 0);   // first index of the size-k block
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        if (i < k) rk += binom3(bg[i], i + 1);
                    const float4 *t4 = reinterpret_cast<const float4 *>(A.tab + rk * TAB);
                    const float4 ta = __ldg(t4), tb = __ldg(t4 + 1);
                    reinterpret_cast<float4 *>(trow + v * TAB)[0] = ta;
                    reinterpret_cast<float4 *>(trow + v * TAB)[1] = tb;
                    const float t[7] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z};
                    float mi[3][3];
                    mi[0][0] = t[1]; mi[0][1] = mi[1][0] = t[2]; mi[0][2] = mi[2][0] = t[3];
                    mi[1][1] = t[4]; mi[1][2] = mi[2][1] = t[5]; mi[2][2] = t[6];
                    float p[3], mu[3], u[3], rr = 0.f;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        float pv = 0.f;
#pragma unroll
                        for (int j = 0; j < HP; ++j) pv = (j == bl[i]) ? pI[j] : pv;
                        p[i] = (i < k) ? pv : 0.f;
                        mu[i] = (i < k) ? mus[bg[i]] : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        float gm = 0.f;
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            if (i < k && j < k) gm = fmaf(Gs[bg[i] * H + bg[j]], mu[j], gm);
                        u[i] = p[i] - gm;
                        rr = fmaf(mu[i], gm - 2.f * p[i], rr);
                    }
                    float quad = 0.f;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            if (i < k && j < k) quad = fmaf(u[i] * mi[i][j], u[j], quad);
                    l = (float)k * lpi - 0.5f * t[0] - 0.5f * (rr * is2 - quad * is4);
                }
                lv[r] = l * L2E;
                m = fmaxf(m, lv[r]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        // ---- posterior moments into lane-private slots
#pragma unroll 4
        for (int o = 0; o < S::N; ++o) acc[o * 32 + lane] = 0.f;
        float Z = 0.f;
        int best = 0x7fffffff;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int v = lane + 32 * r;
            if (v >= nK) continue;
            const unsigned mk = Ks[v];
            const int k = __popc(mk);
            const float e = fast_ex2(lv[r] - m);
            Z += e;
            const int key_ = (k << 16) + 0xFFFF - (int)(__brev(mk) >> (32 - HP));
            best = (lv[r] == m) ? min(best, key_) : best;
            if (k == 0 || e == 0.f) continue;
            int bl[3] = {0, 0, 0}, bg[3] = {0, 0, 0};
            int q = 0;
#pragma unroll
            for (int j = 0; j < HP; ++j)
                if (((mk >> j) & 1u) && q < 3) { bl[q] = j; bg[q] = I[j]; ++q; }
            const float *t = trow + v * TAB;     // stored by this lane in the log-joint pass
            float mi[3][3];
            mi[0][0] = t[1]; mi[0][1] = mi[1][0] = t[2]; mi[0][2] = mi[2][0] = t[3];
            mi[1][1] = t[4]; mi[1][2] = mi[2][1] = t[5]; mi[2][2] = t[6];
            float w[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float pv = 0.f;
#pragma unroll
                for (int j = 0; j < HP; ++j) pv = (j == bl[i]) ? pI[j] : pv;
                w[i] = (i < k) ? pv * is2 + mpr[bg[i]] : 0.f;
            }
            float kap[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (i < k && j < k) s = fmaf(mi[i][j], w[j], s);
                kap[i] = s;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i >= k) break;
                acc[(S::NB + bl[i]) * 32 + lane] += e;
                acc[(S::NS + bl[i]) * 32 + lane] += e * kap[i];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (j < i || j >= k) continue;
                    acc[S::pair(bl[i], bl[j]) * 32 + lane] += e * (mi[i][j] + kap[i] * kap[j]);
                }
            }
        }
        Z = wsum(Z);
        best = (int)__reduce_min_sync(0xffffffffu, (unsigned)best);
        __syncwarp();
        const float invZ = 1.f / Z;
        // column sums of the lane-private slots: lane o (and o + 32, ...) owns output o
        for (int o = lane; o < S::N; o += 32) {
            float s = 0.f;
#pragma unroll 8
            for (int l2 = 0; l2 < 32; ++l2) s += acc[o * 32 + l2];
            acc[o * 32] = s * invZ;         // slot o, column 0 now holds the normalised value
        }
        __syncwarp();
        const double logZ = ((double)m + (double)log2f(Z)) * (kLn2 * T) + logp00 - (double)yy * i2s2;
        if (ENCODE) {
            if (lane == 0) {
                if (A.sel_out)
                    for (int j = 0; j < HP; ++j) A.sel_out[n * HP + j] = (int16_t)I[j];
                if (A.smean_out)
                    for (int j = 0; j < HP; ++j) A.smean_out[n * HP + j] = acc[(S::NS + j) * 32];
                if (A.map_out) {
                    const unsigned rm = 0xFFFFu - (unsigned)(best & 0xFFFF);
                    int k = 0;
                    for (int j = 0; j < HP; ++j)
                        if (((rm >> (HP - 1 - j)) & 1u) && k < gamma) A.map_out[n * gamma + k++] = (int16_t)I[j];
                    for (; k < gamma; ++k) A.map_out[n * gamma + k] = (int16_t)-1;
                }
                if (A.mapp_out) A.mapp_out[n] = invZ;
                if (A.logz_out) A.logz_out[n] = (float)logZ;
            }
            __syncwarp();
            continue;
        }
        // statistics: B (FP64 atomics on the upper triangle), At and the GSC
        // sums in warp-private shared partials
        for (int o = lane; o < HP * (HP + 1) / 2; o += 32) {
            int i = 0, rem = o;
            while (rem >= HP - i) { rem -= HP - i; ++i; }
            const int j = i + rem;
            const float v = acc[S::pair(i, j) * 32];
            if (v != 0.f) atomicAdd(A.B + (size_t)I[i < HP ? i : 0] * H + I[j < HP ? j : 0], (double)v);
        }
        float s1 = 0.f;
#pragma unroll
        for (int j = 0; j < HP; ++j) {
            const float eb = acc[(S::NB + j) * 32], es = acc[(S::NS + j) * 32];
            const float ess = acc[S::pair(j, j) * 32];
            s1 += eb;
            const int h = I[j];
            if (lane == 0) {
                gpart[h] += eb;
                gpart[H + h] += es;
                gpart[2 * H + h] += ess;
            }
#pragma unroll
            for (int k = 0; k < DK; ++k) {
                const int d = lane + 32 * k;
                if (d < D) apart[h * D + d] = fmaf(es, y[k], apart[h * D + d]);
            }
        }
        __syncwarp();
        if (lane == 0) {
            const float fh = (float)logZ;
            two_sum_acc(accF, fh);
            two_sum_acc(accF, (float)(logZ - (double)fh));
            two_sum_acc(accS1, s1);
            two_sum_acc(accYY, yy);
            ++accN;
        }
    }
    if (ENCODE) return;
    if (lane == 0) {
        atomicAdd(A.scal + PROSPER_SC_F, (double)accF.x + (double)accF.y);
        atomicAdd(A.scal + PROSPER_SC_S1, (double)accS1.x + (double)accS1.y);
        atomicAdd(A.scal + PROSPER_SC_YY, (double)accYY.x + (double)accYY.y);
        atomicAdd(A.scal + PROSPER_SC_N, (double)accN);
    }
    __syncthreads();
    const int stride = S::N * 32 + 64 + 3 * H + H * D;
    for (int i = tid; i < 3 * H + H * D; i += GW * 32) {
        float s = 0.f;
        for (int w = 0; w < GW; ++w) s += wbase[(size_t)w * stride + S::N * 32 + 64 + i];
        if (s == 0.f) continue;
        if (i < 3 * H) atomicAdd(A.gsc + i, (double)s);
        else atomicAdd(A.At + (i - 3 * H), (double)s);
    }
}

template <int HP>
size_t gsc_smem(int D, int H, int nK) {
    static_assert(Slots<HP>::N == 2 * HP + HP * (HP + 1) / 2, "slot count");
    return gsc_smem_hp(D, H, HP, nK);
}

template <int HP, int DK>
int gsc_launch2(GscArgs &A, bool enc, int grid, cudaStream_t s) {
    const size_t smem = gsc_smem<HP>(A.D, A.H, A.nK);
    if (smem > 227 * 1024) {
        set_error("GSC: shared memory %zu bytes exceeds the limit (reduce D or H)", smem);
        return PROSPER_EINVAL;
    }
    if (int rc = ensure_smem_attr(enc ? (const void *)k_gsc_estep<HP, DK, true>
                                      : (const void *)k_gsc_estep<HP, DK, false>, smem))
        return rc;
    if (enc) k_gsc_estep<HP, DK, true><<<grid, GW * 32, smem, s>>>(A);
    else k_gsc_estep<HP, DK, false><<<grid, GW * 32, smem, s>>>(A);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

template <int HP>
int gsc_launch(GscArgs &A, bool enc, int grid, cudaStream_t s) {
    const int dk = (A.D + 31) / 32;
    if (dk <= 1) return gsc_launch2<HP, 1>(A, enc, grid, s);
    if (dk <= 2) return gsc_launch2<HP, 2>(A, enc, grid, s);
    if (dk <= 4) return gsc_launch2<HP, 4>(A, enc, grid, s);
    if (dk <= 8) return gsc_launch2<HP, 8>(A, enc, grid, s);
    set_error("GSC: D=%d > 256", A.D);
    return PROSPER_EINVAL;
}

}  // namespace
}  // namespace prosper
