// mca.cu -- Maximal Causes Analysis (Table 1, row MCA: max superposition,
// Gaussian noise, binary latents, Bernoulli prior) truncated E-step, and its
// signed variant MMCA (Table 1, row MMCA: per pixel the active component of
// largest magnitude, f_d = W_dh* with h* = argmax_{h in s} |W_dh|, the first
// in unit order on a tie; scores, logs and smoothed maxima on |W|).
//
// One warp per data point; lane l owns the pixels d = l + 32 k (k < DK).
//   1. Preselection score S_h = sum_d W_dh y_d / sum_d W_dh (reading: the paper
//      names Hprime but not the score), top-H' with ties to the lower h.
//   2. The states with <= gamma active units among the H' candidates are
//      visited depth-first; the superposition f_d(s) = max_{h in s} W_dh is
//      carried down the tree (one max per pixel per state) and
//      l(s) = |s| log(pi/(1-pi)) - (||y - f(s)||^2 - ||y||^2) / (2 sigma^2)
//      is formed with one warp reduction per state.
//   3. Log-sum-exp, posterior means, the MAP state (canonically first maximum),
//      E||y - f||^2 (hard max, for the sigma update) and, for every state whose
//      weight 2^(l - m) is nonzero in FP32, the rho-smoothed-max factors
//      A_dh(s) = s_h (W_dh / Wbar_d(s))^(rho-1), Wbar_d(s) = (sum_{h in s} W_dh^rho)^(1/rho),
//      evaluated as exp2 of log2 differences with Wbar scaled by the max.
//      sum_n <A_dh> y_d and sum_n <A_dh> are kept per warp in shared memory
//      (no atomics) and added to the FP64 statistics once per CTA.
#include "internal.cuh"
#include "topk.cuh"

#include <cmath>

namespace prosper {
namespace {

constexpr int MW = 8;          // warps per CTA
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2Pi = 1.8378770664093454836;

struct McaArgs {
    const float *W;        // H x D
    const float *Y;        // N x D
    const double *theta;
    int64_t N;
    int D, H, Hp, gamma, nK;   // nK = number of states per point
    int mm;                // 1: MMCA (magnitude max, signed W)
    double *mca;           // 2 H D (estep) or NULL
    double *scal;
    int16_t *sel_out, *map_out;
    float *smean_out, *mapp_out, *logz_out;
};

__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float fast_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// one step of the superposition carried down the state tree: MCA max(f, w);
// MMCA the value of larger magnitude (f, the earlier unit, on a tie)
__device__ __forceinline__ float smax(float f, float w, int mm) {
    return mm ? (fabsf(w) > fabsf(f) ? w : f) : fmaxf(f, w);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// shared layout: W (H x D), log2 W (H x D), W transposed (D x H), 1/sum_d W_dh (H), per warp
// { l[KW], mask[KW], 32 x 33 partial sums } (KW = max(nK, D, 64) rounded to 4) and,
// with SMEM_STATS, per warp sum<A>y and sum<A> (H x D each)
// acc (hi, lo) += v with Knuth's TwoSum (hi + lo carries about 48 bits)
__device__ __forceinline__ void two_sum_acc(float2 &acc, float v) {
    const float s = acc.x + v;
    const float bb = s - acc.x;
    acc.y += (acc.x - (s - bb)) + (v - bb);
    acc.x = s;
}

constexpr int KMAX = 1024;

// HPM: register arrays sized for Hprime <= HPM (10 or 16)
template <int DK, bool ENCODE, bool SMEM_STATS, int HPM>
__global__ void __launch_bounds__(MW * 32, 1) k_mca_estep(McaArgs A) {
    extern __shared__ __align__(16) float sm[];
    const int D = A.D, H = A.H, Hp = A.Hp, gamma = A.gamma;
    float *Ws = sm;
    float *Ls = Ws + H * D;
    float *WsT = Ls + H * D;             // D x H: lane h reads row d (preselection)
    float *Rc = WsT + H * D;
    float *wl = Rc + ((H + 3) & ~3);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int KW = (max(max(A.nK, D), 64) + 3) & ~3;
    const int WSTR = 2 * KW + 32 * 33;
    float *ell = wl + warp * WSTR;
    unsigned *msk = reinterpret_cast<unsigned *>(ell + KW);
    float *part = ell + 2 * KW;                                   // 32 x 33 partial sums
    float *Ay = wl + MW * WSTR + (size_t)warp * 2 * H * D;        // SMEM_STATS only
    float *Aa = Ay + H * D;

    for (int i = tid; i < H * D; i += MW * 32) {
        const float w = A.W[i];
        Ws[i] = w;
        WsT[(i % D) * H + i / D] = w;
        const float aw = A.mm ? fabsf(w) : w;
        Ls[i] = aw > 0.f ? log2f(aw) : -INFINITY;
    }
    for (int h = tid; h < H; h += MW * 32) {
        float s = 0.f;
        for (int d = 0; d < D; ++d) s += A.mm ? fabsf(A.W[(size_t)h * D + d]) : A.W[(size_t)h * D + d];
        Rc[h] = s > 0.f ? 1.f / s : 0.f;
    }
    if (SMEM_STATS)
        for (int i = lane; i < 2 * H * D; i += 32) Ay[i] = 0.f;
    __syncthreads();

    const double pi = A.theta[PROSPER_TH_PI], sigma = A.theta[PROSPER_TH_SIGMA];
    const float rho = (float)A.theta[PROSPER_TH_RHO];
    // deterministic annealing: log-joints divided by T (theta[3]; <= 0 reads as 1)
    const double Tth = A.theta[PROSPER_TH_T];
    const double T = Tth > 0.0 ? Tth : 1.0;
    const float lpi = (float)(log(pi / (1.0 - pi)) * 1.4426950408889634 / T);
    const float ih = (float)(1.4426950408889634 / (2.0 * sigma * sigma * T));   // log2e / (2 sigma^2 T)
    const double logp00 = H * log(1.0 - pi) - 0.5 * D * (kLog2Pi + log(sigma * sigma));
    const double i2s2 = 0.5 / (sigma * sigma);

    // per-warp sums as FP32 pairs (hi + lo, Knuth's TwoSum): FP64 adds are
    // ~65x slower than FP32 ones on this part
    float2 accF = make_float2(0.f, 0.f), accS1 = accF, accYY = accF, accR2 = accF;
    int accN = 0;
    const int64_t gw = (int64_t)blockIdx.x * MW + warp, nw = (int64_t)gridDim.x * MW;
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
        yy = warp_sum(yy);
        // ---- preselection: lane h gets sum_d W_dh y_d (H <= 256: 8 per lane) from
        //      the transposed dictionary and the point's y staged in the warp's
        //      state buffer (free until pass 1)
#pragma unroll
        for (int k = 0; k < DK; ++k) {
            const int d = lane + 32 * k;
            if (d < D) ell[d] = y[k];
        }
        __syncwarp();
        unsigned key[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int h = lane + 32 * j;
            key[j] = 0u;
            if (h < H) {
                float p0 = 0.f, p1 = 0.f;
                int d = 0;
                for (; d + 1 < D; d += 2) {
                    p0 = fmaf(WsT[d * H + h], ell[d], p0);
                    p1 = fmaf(WsT[(d + 1) * H + h], ell[d + 1], p1);
                }
                if (d < D) p0 = fmaf(WsT[d * H + h], ell[d], p0);
                key[j] = score_key((p0 + p1) * Rc[h]);
            }
        }
        __syncwarp();
        const int myh = warp_topk(key, Hp, lane, msk);   // msk doubles as scratch here
        __syncwarp();
        const int rank = topk_rank(myh, Hp, lane);
        int I[HPM];
#pragma unroll
        for (int j = 0; j < HPM; ++j) {
            // the latent with rank j (ascending h)
            const unsigned ball = __ballot_sync(0xffffffffu, lane < Hp && rank == j);
            I[j] = ball ? __shfl_sync(0xffffffffu, myh, __ffs(ball) - 1) : 0;
        }
        // ---- pass 1: depth-first over states, l in log2 units relative to s = 0.
        //      Each lane's share of |y - f|^2 - |y|^2 goes to a 32 x 33 tile;
        //      every 32 states, lane s adds up row s (conflict-free: the pitch of
        //      33 words puts (s, l) in bank (s + l) mod 32), so no state waits on
        //      its own cross-lane reduction.
        int nv = 0;
        float mloc = -INFINITY;
        auto flush = [&](int v0, int cnt) {
            __syncwarp();
            if (lane < cnt) {
                float r = 0.f;
#pragma unroll 8
                for (int l2 = 0; l2 < 32; ++l2) r += part[lane * 33 + l2];
                const float l = lpi * (float)__popc(msk[v0 + lane]) - ih * r;
                ell[v0 + lane] = l;
                mloc = fmaxf(mloc, l);
            }
            __syncwarp();
        };
        auto visit = [&](unsigned mask, const float (&f)[DK]) {
            float r = 0.f;
#pragma unroll
            for (int k = 0; k < DK; ++k) r = fmaf(f[k], f[k] - 2.f * y[k], r);   // |y-f|^2 - |y|^2
            const int slot = nv & 31;
            part[slot * 33 + lane] = r;
            if (lane == 0) msk[nv] = mask;
            ++nv;
            if (slot == 31) flush(nv - 32, 32);
        };
        if (gamma > 5) {
            // generic order (any gamma <= H'): every pattern with <= gamma units,
            // superposition rebuilt from its active units
            for (unsigned mask = 0; mask < (1u << Hp); ++mask) {
                if (__popc(mask) > gamma) continue;
                float f[DK];
#pragma unroll
                for (int k = 0; k < DK; ++k) f[k] = 0.f;
#pragma unroll
                for (int j = 0; j < HPM; ++j) {
                    if (!((mask >> j) & 1u)) continue;
#pragma unroll
                    for (int k = 0; k < DK; ++k) {
                        const int d = lane + 32 * k;
                        f[k] = smax(f[k], d < D ? Ws[I[j] * D + d] : 0.f, A.mm);
                    }
                }
                visit(mask, f);
            }
        } else {
            float f0[DK];
#pragma unroll
            for (int k = 0; k < DK; ++k) f0[k] = 0.f;
            visit(0u, f0);
            for (int i1 = 0; gamma >= 1 && i1 < Hp; ++i1) {
                int g1 = 0;
#pragma unroll
                for (int j = 0; j < HPM; ++j) g1 = (j == i1) ? I[j] : g1;
                float f1[DK];
#pragma unroll
                for (int k = 0; k < DK; ++k) {
                    const int d = lane + 32 * k;
                    f1[k] = smax(f0[k], d < D ? Ws[g1 * D + d] : 0.f, A.mm);
                }
                visit(1u << i1, f1);
                for (int i2 = i1 + 1; gamma >= 2 && i2 < Hp; ++i2) {
                    int g2 = 0;
#pragma unroll
                    for (int j = 0; j < HPM; ++j) g2 = (j == i2) ? I[j] : g2;
                    float f2[DK];
#pragma unroll
                    for (int k = 0; k < DK; ++k) {
                        const int d = lane + 32 * k;
                        f2[k] = smax(f1[k], d < D ? Ws[g2 * D + d] : 0.f, A.mm);
                    }
                    visit((1u << i1) | (1u << i2), f2);
                    for (int i3 = i2 + 1; gamma >= 3 && i3 < Hp; ++i3) {
                        int g3 = 0;
#pragma unroll
                        for (int j = 0; j < HPM; ++j) g3 = (j == i3) ? I[j] : g3;
                        float f3[DK];
#pragma unroll
                        for (int k = 0; k < DK; ++k) {
                            const int d = lane + 32 * k;
                            f3[k] = smax(f2[k], d < D ? Ws[g3 * D + d] : 0.f, A.mm);
                        }
                        visit((1u << i1) | (1u << i2) | (1u << i3), f3);
                        for (int i4 = i3 + 1; gamma >= 4 && i4 < Hp; ++i4) {
                            int g4 = 0;
#pragma unroll
                            for (int j = 0; j < HPM; ++j) g4 = (j == i4) ? I[j] : g4;
                            float f4[DK];
#pragma unroll
                            for (int k = 0; k < DK; ++k) {
                                const int d = lane + 32 * k;
                                f4[k] = smax(f3[k], d < D ? Ws[g4 * D + d] : 0.f, A.mm);
                            }
                            visit((1u << i1) | (1u << i2) | (1u << i3) | (1u << i4), f4);
                            for (int i5 = i4 + 1; gamma >= 5 && i5 < Hp; ++i5) {
                                int g5 = 0;
#pragma unroll
                                for (int j = 0; j < HPM; ++j) g5 = (j == i5) ? I[j] : g5;
                                float f5[DK];
#pragma unroll
                                for (int k = 0; k < DK; ++k) {
                                    const int d = lane + 32 * k;
                                    f5[k] = smax(f4[k], d < D ? Ws[g5 * D + d] : 0.f, A.mm);
                                }
                                visit((1u << i1) | (1u << i2) | (1u << i3) | (1u << i4) | (1u << i5), f5);
                            }
                        }
                    }
                }
            }
        }
        if (nv & 31) flush(nv & ~31, nv & 31);
        const float m = warp_max(mloc);
        // ---- normalisation, posterior means, MAP (lanes over states)
        float Z = 0.f, es[HPM];
#pragma unroll
        for (int j = 0; j < HPM; ++j) es[j] = 0.f;
        float S1 = 0.f;
        int best = 0x7fffffff;
        for (int v = lane; v < nv; v += 32) {
            const float l = ell[v];
            const unsigned mk = msk[v];
            const float e = fast_ex2(l - m);
            Z += e;
            S1 += e * (float)__popc(mk);
#pragma unroll
            for (int j = 0; j < HPM; ++j) es[j] += ((mk >> j) & 1u) ? e : 0.f;
            const int key = (__popc(mk) << 16) + 0xFFFF - (int)(__brev(mk) >> (32 - Hp));
            best = (l == m) ? min(best, key) : best;
        }
        Z = warp_sum(Z);
        S1 = warp_sum(S1);
#pragma unroll
        for (int j = 0; j < HPM; ++j) es[j] = warp_sum(es[j]);
        best = __reduce_min_sync(0xffffffffu, (unsigned)best);
        const float invZ = 1.f / Z;
        const double logZ = ((double)m + (double)log2f(Z)) * (kLn2 * T) + logp00 - (double)yy * i2s2;

        if (ENCODE) {
            if (lane == 0) {
                if (A.sel_out)
                    for (int j = 0; j < Hp; ++j) A.sel_out[n * Hp + j] = (int16_t)I[j];
                if (A.smean_out)
                    for (int j = 0; j < Hp; ++j) A.smean_out[n * Hp + j] = es[j] * invZ;
                if (A.map_out) {
                    const unsigned rm = 0xFFFFu - (unsigned)(best & 0xFFFF);
                    int k = 0;
                    for (int j = 0; j < Hp; ++j)
                        if (((rm >> (Hp - 1 - j)) & 1u) && k < gamma) A.map_out[n * gamma + k++] = (int16_t)I[j];
                    for (; k < gamma; ++k) A.map_out[n * gamma + k] = (int16_t)-1;
                }
                if (A.mapp_out) A.mapp_out[n] = invZ;
                if (A.logz_out) A.logz_out[n] = (float)logZ;
            }
            continue;
        }

        // ---- statistics: E||y-f||^2 and the smoothed-max factors for every
        //      state with nonzero weight (pixel-parallel, in lanes)
        float R2 = 0.f;
        float Abar[HPM][DK];
#pragma unroll
        for (int j = 0; j < HPM; ++j)
#pragma unroll
            for (int k = 0; k < DK; ++k) Abar[j][k] = 0.f;
        for (int v = 0; v < nv; ++v) {
            // a state whose posterior weight is below 2^-32 of the most
            // probable one's is skipped (warp-uniform): the at most 1024 such
            // states hold less than 2^-22 of the largest weight together
            if (ell[v] - m < -32.f) continue;
            const float e = fast_ex2(ell[v] - m);
            const float q = e * invZ;
            const unsigned mk = msk[v];
            R2 += q * (((ell[v] - lpi * (float)__popc(mk)) / -ih) + yy);   // ||y - f||^2
            if (mk == 0u) continue;
#pragma unroll
            for (int k = 0; k < DK; ++k) {
                const int d = lane + 32 * k;
                if (d >= D) continue;
                // log2 W_dh of the state's active units, read once
                float lw[HPM];
                float lmax = -INFINITY;
#pragma unroll
                for (int j = 0; j < HPM; ++j) {
                    lw[j] = ((mk >> j) & 1u) ? Ls[I[j] * D + d] : -INFINITY;
                    lmax = fmaxf(lmax, lw[j]);
                }
                // every active |W_dh| is 0 at this pixel: no smoothed-max factor
                // (2^(rho (lw - lmax)) would be 2^NaN)
                if (lmax == -INFINITY) continue;
                float t = 0.f;
#pragma unroll
                for (int j = 0; j < HPM; ++j)
                    if ((mk >> j) & 1u) t += fast_ex2(rho * (lw[j] - lmax));
                const float lbar = lmax + fast_lg2(t) / rho;     // log2 Wbar_d(s)
#pragma unroll
                for (int j = 0; j < HPM; ++j)
                    if ((mk >> j) & 1u)
                        Abar[j][k] = fmaf(q, fast_ex2((rho - 1.f) * (lw[j] - lbar)), Abar[j][k]);
            }
        }
#pragma unroll
        for (int j = 0; j < HPM; ++j) {
            if (j >= Hp) break;
            const int h = I[j];
#pragma unroll
            for (int k = 0; k < DK; ++k) {
                const int d = lane + 32 * k;
                if (d >= D) continue;
                if (SMEM_STATS) {
                    Ay[h * D + d] = fmaf(Abar[j][k], y[k], Ay[h * D + d]);
                    Aa[h * D + d] += Abar[j][k];
                } else {
                    atomicAdd(A.mca + (size_t)h * D + d, (double)(Abar[j][k] * y[k]));
                    atomicAdd(A.mca + (size_t)H * D + (size_t)h * D + d, (double)Abar[j][k]);
                }
            }
        }
        if (lane == 0) {
            const float fh = (float)logZ;
            two_sum_acc(accF, fh);
            two_sum_acc(accF, (float)(logZ - (double)fh));
            two_sum_acc(accS1, S1 * invZ);
            two_sum_acc(accYY, yy);
            two_sum_acc(accR2, R2);
            ++accN;
        }
    }
    if (ENCODE) return;
    if (lane == 0) {
        atomicAdd(A.scal + PROSPER_SC_F, (double)accF.x + (double)accF.y);
        atomicAdd(A.scal + PROSPER_SC_S1, (double)accS1.x + (double)accS1.y);
        atomicAdd(A.scal + PROSPER_SC_YY, (double)accYY.x + (double)accYY.y);
        atomicAdd(A.scal + PROSPER_SC_MCA_R2, (double)accR2.x + (double)accR2.y);
        atomicAdd(A.scal + PROSPER_SC_N, (double)accN);
    }
    if (SMEM_STATS) {
        __syncthreads();
        float *base = wl + MW * WSTR;
        for (int i = tid; i < 2 * H * D; i += MW * 32) {
            float s = 0.f;
            for (int w = 0; w < MW; ++w) s += base[(size_t)w * 2 * H * D + i];
            if (s != 0.f) atomicAdd(A.mca + i, (double)s);
        }
    }
}

size_t mca_smem(int D, int H, int nK, bool smem_stats) {
    const size_t kw = (size_t)((std::max(std::max(nK, D), 64) + 3) & ~3);
    size_t f = 3 * (size_t)H * D + ((H + 3) & ~3) + (size_t)MW * (2 * kw + 32 * 33);
    if (smem_stats) f += (size_t)MW * 2 * H * D;
    return f * sizeof(float);
}

template <int DK, bool ENC, bool SS>
int mca_launch(McaArgs &A, int grid, size_t smem, cudaStream_t s) {
    if (A.Hp <= 10) {
        if (int rc = ensure_smem_attr((const void *)k_mca_estep<DK, ENC, SS, 10>, smem)) return rc;
        k_mca_estep<DK, ENC, SS, 10><<<grid, MW * 32, smem, s>>>(A);
    } else {
        if (int rc = ensure_smem_attr((const void *)k_mca_estep<DK, ENC, SS, 16>, smem)) return rc;
        k_mca_estep<DK, ENC, SS, 16><<<grid, MW * 32, smem, s>>>(A);
    }
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

template <int DK>
int mca_dispatch(McaArgs &A, bool enc, int grid, cudaStream_t s) {
    const bool ss = mca_smem(A.D, A.H, A.nK, true) <= 227 * 1024;
    const size_t smem = mca_smem(A.D, A.H, A.nK, ss && !enc);
    if (enc) return mca_launch<DK, true, false>(A, grid, smem, s);
    if (ss) return mca_launch<DK, false, true>(A, grid, smem, s);
    return mca_launch<DK, false, false>(A, grid, smem, s);
}

}  // namespace

int launch_mca_prep(prosper_ctx *, const float *, cudaStream_t) { return PROSPER_OK; }

int launch_mca_estep(prosper_ctx *c, const float *W, const double *theta, const float *Y,
                     int64_t N, prosper_stats *st, int16_t *sel_out, float *smean_out,
                     int16_t *map_out, float *mapp_out, float *logz_out, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    McaArgs A;
    A.W = W; A.Y = Y; A.theta = theta; A.N = N;
    A.D = c->D; A.H = c->H; A.Hp = c->Hp; A.gamma = c->gamma; A.nK = c->nK;
    A.mm = c->model == PROSPER_MMCA ? 1 : 0;
    if (c->nK > KMAX) {
        set_error("MCA: %d states per point > %d", c->nK, KMAX);
        return PROSPER_EINVAL;
    }
    A.mca = st ? st->mca : nullptr;
    A.scal = st ? st->scal : nullptr;
    A.sel_out = sel_out; A.map_out = map_out; A.smean_out = smean_out; A.mapp_out = mapp_out;
    A.logz_out = logz_out;
    const bool enc = (st == nullptr);
    const int64_t warps = (N + 3) / 4;     // at least 4 points per warp
    const int grid = (int)std::min<int64_t>((warps + MW - 1) / MW, (int64_t)c->num_sms);
    TraceScope tr(c, enc ? (A.mm ? "mmca_encode" : "mca_encode") : (A.mm ? "mmca_estep" : "mca_estep"), s);
    const int dk = (c->D + 31) / 32;
    if (dk <= 1) return mca_dispatch<1>(A, enc, grid, s);
    if (dk <= 2) return mca_dispatch<2>(A, enc, grid, s);
    if (dk <= 4) return mca_dispatch<4>(A, enc, grid, s);
    if (dk <= 8) return mca_dispatch<8>(A, enc, grid, s);
    set_error("MCA: D=%d > 256", c->D);
    return PROSPER_EINVAL;
}

}  // namespace prosper
