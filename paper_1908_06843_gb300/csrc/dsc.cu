// dsc.cu -- truncated E-step by a table of states, one warp per data point,
// for linear superposition with discrete latents (Table 1 rows TSC and DSC:
// latents in {0, phi_1, .., phi_m}, categorical prior, Gaussian noise) and for
// BSC (the single value 1) when Hprime is above the register-resident state
// kernel's range (11 .. 16).
//
// For a state s over the candidates I (k nonzero units u_a with values
// phi_{v_a}), exact algebra from ||y - W s||^2 = y^T y - 2 s^T W^T y + s^T G s
// (Eq. 2, G = W^T W) gives, relative to s = 0,
//   l(s) = sum_a [log(pi_{v_a}/pi_0) + (phi_{v_a} p_{u_a} - phi_{v_a}^2 G_{u_a u_a}/2)/sigma^2]
//          - sum_{a<b} phi_{v_a} phi_{v_b} G_{u_a u_b} / sigma^2,      p = W_I^T y,
// divided by the annealing temperature T (base 2 inside the kernel).
//
// The state set K (every pattern of at most gamma nonzero units among the
// Hprime candidates, each taking one of m values) is a table built on the host
// in canonical order: by number of nonzero units, then the units' combination
// order, then their value indices.  Lane l of a point's warp evaluates states
// l, l + 32, ...: pass 1 takes the maximum, pass 2 the weights 2^(l - max),
// the MAP state (the first maximum in table order) and the moments
// <s_i>, <s_i s_j> and the per-value counts, summed in lane-private
// shared-memory slots (slot-major, so a lane's updates never conflict) that
// the warp adds up with a skewed read order at the end.
#include "internal.cuh"

#include <cmath>
#include <vector>

namespace prosper {
namespace {

constexpr int XW = 8;   // warps (points in flight) per CTA
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2Pi = 1.8378770664093454836;
constexpr double kLog2e = 1.4426950408889634;

struct DscArgs {
    const int32_t *sel;
    const float *selp;
    const float2 *yy;
    const float *G;
    const uint2 *tab;      // nK states: x = unit of nonzero a in bits 4a..4a+3,
                           //            y = value index of a in bits 2a, 2a+1 | k << 16
    const double *theta;
    int64_t N, n_offset;
    int H, D, Hp, gamma, nK, m, model, nslot, wstride;
    float phi0, phi1, phi2;
    float *es;
    double *B, *scal;
    int16_t *sel_out, *map_out;
    float *mapv_out, *smean_out, *mapp_out, *logz_out;
    // E-step with the data cut: the first pass's log Z of this piece's points
    // and the threshold; a point below it is left out
    const float *cut_logz, *cut_thr;
};

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

template <bool ENCODE>
__global__ void __launch_bounds__(XW * 32, 1) k_dsc_states(DscArgs A) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float s_lp[3], s_is2;
    __shared__ double s_c0, s_inv2s2, s_T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Hp = A.Hp, m = A.m, nK = A.nK, H = A.H, gamma = A.gamma;
    if (threadIdx.x == 0) {
        // prior of the nonzero values: BSC pi; TSC pi/2 each (zero-mean
        // ternary); DSC theta[PROSPER_TH_DSC_P + v]
        const double sigma = A.theta[PROSPER_TH_SIGMA];
        const double th = A.theta[PROSPER_TH_T];
        const double T = th > 0.0 ? th : 1.0;
        double pv[3] = {0.0, 0.0, 0.0};
        if (A.model == PROSPER_TSC) {
            pv[0] = pv[1] = 0.5 * A.theta[PROSPER_TH_PI];
        } else if (A.model == PROSPER_DSC) {
            for (int v = 0; v < m; ++v) pv[v] = A.theta[PROSPER_TH_DSC_P + v];
        } else {
            pv[0] = A.theta[PROSPER_TH_PI];
        }
        double p0 = 1.0;
        for (int v = 0; v < m; ++v) p0 -= pv[v];
        for (int v = 0; v < 3; ++v) s_lp[v] = v < m ? (float)(log(pv[v] / p0) * kLog2e / T) : 0.f;
        s_is2 = (float)(kLog2e / (sigma * sigma * T));
        s_c0 = H * log(p0) - 0.5 * A.D * (kLog2Pi + log(sigma * sigma));
        s_inv2s2 = 0.5 / (sigma * sigma);
        s_T = T;
    }
    __syncthreads();
    const float is2 = s_is2;
    const float phi[3] = {A.phi0, A.phi1, A.phi2};
    float *cA = sm + (size_t)warp * A.wstride;   // m x 16: a_{v,j}
    float *cB = cA + 48;                         // 16 x 16: -G_{I_i I_j} / (sigma^2 T) (log2)
    float *acc = cB + 256;                       // nslot x 32 lane-private sums
    const int NS2 = Hp;                          // first pair slot
    const int NCNT = Hp + Hp * (Hp + 1) / 2;     // first value-count slot
    auto pair_slot = [&](int i, int j) { return NS2 + i * Hp - i * (i - 1) / 2 + (j - i); };
    auto val = [&](int v) { return v == 0 ? phi[0] : (v == 1 ? phi[1] : phi[2]); };

    // log-joint (base 2, relative to s = 0, divided by T) of one table entry
    auto ell = [&](uint2 t) {
        const int k = (int)(t.y >> 16);
        float l = 0.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            if (a >= k) break;
            const int ua = (int)((t.x >> (4 * a)) & 15u), va = (int)((t.y >> (2 * a)) & 3u);
            const float pa = val(va);
            l += cA[va * 16 + ua];
#pragma unroll
            for (int b = 0; b < a; ++b) {
                const int ub = (int)((t.x >> (4 * b)) & 15u), vb = (int)((t.y >> (2 * b)) & 3u);
                l = fmaf(pa * val(vb), cB[ub * 16 + ua], l);
            }
        }
        return l;
    };

    float2 accF = make_float2(0.f, 0.f), accS1 = accF, accYY = accF;
    float2 accC[3] = {accF, accF, accF};
    int accN = 0;
    const int64_t gw = (int64_t)blockIdx.x * XW + warp, nw = (int64_t)gridDim.x * XW;
    for (int64_t n = gw; n < A.N; n += nw) {
        int myI = 0;
        float myP = 0.f;
        if (lane < Hp) {
            myI = min(max(A.sel[n * SEL_STRIDE + lane], 0), H - 1);
            myP = A.selp[n * SEL_STRIDE + lane];
        }
        __syncwarp();   // the previous point's reads of cA / cB / acc are done
        if (lane < Hp) {
            const float gjj = __ldg(A.G + (size_t)myI * H + myI);
            for (int v = 0; v < m; ++v) {
                const float pv = val(v);
                cA[v * 16 + lane] = s_lp[v] + (pv * myP - 0.5f * pv * pv * gjj) * is2;
            }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = lane + 32 * r, i = e >> 4, j = e & 15;
            const int Ii = __shfl_sync(0xffffffffu, myI, i);
            const int Ij = __shfl_sync(0xffffffffu, myI, j);
            if (i < Hp && j < Hp) cB[e] = (i == j) ? 0.f : -__ldg(A.G + (size_t)Ii * H + Ij) * is2;
        }
        if (!ENCODE || A.smean_out)
            for (int o = 0; o < A.nslot; ++o) acc[o * 32 + lane] = 0.f;
        __syncwarp();

        // ---- pass 1: maximum
        float M = -INFINITY;
        for (int kk = lane; kk < nK; kk += 32) M = fmaxf(M, ell(__ldg(A.tab + kk)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));

        // ---- pass 2: weights, MAP, moments
        float Z = 0.f;
        int best = 0x7fffffff;
        for (int kk = lane; kk < nK; kk += 32) {
            const uint2 t = __ldg(A.tab + kk);
            const float l = ell(t);
            const float e = fast_ex2(l - M);
            Z += e;
            best = (l == M) ? min(best, kk) : best;
            if (e == 0.f || (ENCODE && !A.smean_out)) continue;
            const int k = (int)(t.y >> 16);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                if (a >= k) break;
                const int ua = (int)((t.x >> (4 * a)) & 15u), va = (int)((t.y >> (2 * a)) & 3u);
                const float ea = e * val(va);
                acc[ua * 32 + lane] += ea;
                acc[(NCNT + va) * 32 + lane] += e;
#pragma unroll
                for (int b = 0; b <= a; ++b) {
                    const int ub = (int)((t.x >> (4 * b)) & 15u), vb = (int)((t.y >> (2 * b)) & 3u);
                    acc[pair_slot(ub, ua) * 32 + lane] += ea * val(vb);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Z += __shfl_xor_sync(0xffffffffu, Z, o);
            best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        }
        __syncwarp();
        const float invZ = 1.f / Z;
        // slot sums: lane o owns slots o, o + 32, ...; the skewed order l + o
        // puts the 32 lanes' reads of one step in 32 different banks
        if (!ENCODE || A.smean_out) {
            for (int o = lane; o < A.nslot; o += 32) {
                float s = 0.f;
#pragma unroll 8
                for (int l2 = 0; l2 < 32; ++l2) s += acc[o * 32 + ((l2 + o) & 31)];
                acc[o * 32] = s * invZ;
            }
        }
        __syncwarp();
        const float2 yyv = A.yy[n];
        const double yy = (double)yyv.x + (double)yyv.y;
        const double logZ = ((double)M + (double)log2f(Z)) * (kLn2 * s_T) + s_c0 - yy * s_inv2s2;
        // MAP state (first maximum in table order): its units as global indices
        const uint2 tb = __ldg(A.tab + min(best, nK - 1));
        const int kb = (int)(tb.y >> 16);

        if (ENCODE) {
            const int64_t o = A.n_offset + n;
            if (lane < Hp) {
                if (A.sel_out) A.sel_out[o * Hp + lane] = (int16_t)myI;
                if (A.smean_out) A.smean_out[o * Hp + lane] = acc[lane * 32];
            }
            for (int a = 0; a < gamma; a += 32) {
                const int aa = a + lane;
                const int ua = aa < kb ? (int)((tb.x >> (4 * (aa & 7))) & 15u) : 0;
                const int gI = __shfl_sync(0xffffffffu, myI, ua);
                if (aa < gamma) {
                    if (A.map_out) A.map_out[o * gamma + aa] = aa < kb ? (int16_t)gI : (int16_t)-1;
                    if (A.mapv_out)
                        A.mapv_out[o * gamma + aa] = aa < kb ? val((int)((tb.y >> (2 * (aa & 7))) & 3u)) : 0.f;
                }
            }
            if (lane == 0) {
                if (A.mapp_out) A.mapp_out[o] = invZ;   // q(MAP) = 2^0 / Z
                if (A.logz_out) A.logz_out[o] = (float)logZ;
            }
            continue;
        }
        // E-step statistics: <s> for sum y<s>^T, sum <ss^T> (upper triangle,
        // I ascending), scalars; the data cut leaves a point out of all of them
        const bool kept = A.cut_thr == nullptr || A.cut_logz[n] >= *A.cut_thr;
        if (lane < Hp) A.es[n * SEL_STRIDE + lane] = kept ? acc[lane * 32] : 0.f;
        if (!kept) continue;
        const int npair = Hp * (Hp + 1) / 2;
        for (int base = 0; base < npair; base += 32) {
            const int o = base + lane;
            int i = 0, rem = o;
            while (i < Hp - 1 && rem >= Hp - i) { rem -= Hp - i; ++i; }
            const int j = i + rem;
            const int Ii = __shfl_sync(0xffffffffu, myI, i & 15);
            const int Ij = __shfl_sync(0xffffffffu, myI, j & 15);
            if (o < npair) {
                const float v = acc[(NS2 + o) * 32];
                if (v != 0.f) atomicAdd(A.B + (size_t)Ii * H + Ij, (double)v);
            }
        }
        if (lane == 0) {
            float s1 = 0.f;
            for (int v = 0; v < m; ++v) {
                const float c = acc[(NCNT + v) * 32];
                s1 += c;
                two_sum_acc(accC[v], c);
            }
            const float fh = (float)logZ;
            two_sum_acc(accF, fh);
            two_sum_acc(accF, (float)(logZ - (double)fh));
            two_sum_acc(accS1, s1);
            two_sum_acc(accYY, yyv.x);
            two_sum_acc(accYY, yyv.y);
            ++accN;
        }
    }
    if (ENCODE) return;
    if (lane == 0 && accN > 0) {
        atomicAdd(A.scal + PROSPER_SC_F, (double)accF.x + (double)accF.y);
        atomicAdd(A.scal + PROSPER_SC_S1, (double)accS1.x + (double)accS1.y);
        atomicAdd(A.scal + PROSPER_SC_YY, (double)accYY.x + (double)accYY.y);
        atomicAdd(A.scal + PROSPER_SC_N, (double)accN);
        if (A.model == PROSPER_TSC || A.model == PROSPER_DSC)
            for (int v = 0; v < m; ++v)
                atomicAdd(A.scal + PROSPER_SC_DSC0 + v, (double)accC[v].x + (double)accC[v].y);
    }
}

int dsc_wstride(int Hp, int m) {
    const int nslot = Hp + Hp * (Hp + 1) / 2 + m;
    return (48 + 256 + nslot * 32 + 3) & ~3;
}

}  // namespace

size_t dsc_smem_bytes(int Hp, int m) { return (size_t)XW * dsc_wstride(Hp, m) * sizeof(float); }

// The canonical state table (see the file header), packed as described in DscArgs.
int dsc_build_table(prosper_ctx *c) {
    const int Hp = c->Hp, gamma = c->gamma, m = c->dsc_m;
    std::vector<uint2> tab;
    int idx[16];
    for (int k = 0; k <= gamma && k <= Hp; ++k) {
        for (int i = 0; i < k; ++i) idx[i] = i;
        for (;;) {
            unsigned units = 0;
            for (int i = 0; i < k; ++i) units |= (unsigned)idx[i] << (4 * i);
            unsigned nv = 1;
            for (int i = 0; i < k; ++i) nv *= (unsigned)m;
            for (unsigned code = 0; code < nv; ++code) {
                unsigned vc = 0, r = code;
                for (int a = k - 1; a >= 0; --a) {   // first unit most significant
                    vc |= (r % (unsigned)m) << (2 * a);
                    r /= (unsigned)m;
                }
                tab.push_back(make_uint2(units, vc | ((unsigned)k << 16)));
            }
            int i = k - 1;
            while (i >= 0 && idx[i] == Hp - k + i) --i;
            if (i < 0) break;
            ++idx[i];
            for (int j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
        }
    }
    if ((int)tab.size() != c->nK) {
        set_error("state table: %zu states, expected %d", tab.size(), c->nK);
        return PROSPER_EINVAL;
    }
    cudaError_t e = cudaMalloc(&c->dsc_tab, sizeof(uint2) * tab.size());
    if (e != cudaSuccess) {
        set_error("cudaMalloc of the state table failed: %s", cudaGetErrorString(e));
        return PROSPER_ENOMEM;
    }
    PROSPER_CUDA_TRY(cudaMemcpy(c->dsc_tab, tab.data(), sizeof(uint2) * tab.size(), cudaMemcpyHostToDevice));
    return PROSPER_OK;
}

int launch_linear_proj(prosper_ctx *c, const float *Y, const float *W, int64_t n, cudaStream_t s) {
    return (c->precision == PROSPER_BF16_RESCORE) ? launch_bsc_proj_bf16(c, Y, W, n, s)
                                                  : launch_bsc_proj_f32(c, Y, n, s);
}

int launch_linear_states(prosper_ctx *c, const double *theta, int64_t N, int64_t n_offset,
                         prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                         float *mapv_out, float *mapp_out, float *logz_out, cudaStream_t s) {
    if (c->model == PROSPER_BSC && c->Hp <= BSC_REG_MAX_HPRIME)
        return launch_bsc_states(c, theta, N, n_offset, st, sel_out, smean_out, map_out, mapp_out,
                                 logz_out, s);
    return launch_dsc_states(c, theta, N, n_offset, st, sel_out, smean_out, map_out, mapv_out,
                             mapp_out, logz_out, s);
}

int launch_dsc_states(prosper_ctx *c, const double *theta, int64_t N, int64_t n_offset,
                      prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                      float *mapv_out, float *mapp_out, float *logz_out, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    if (!c->dsc_tab) {
        set_error("state table missing");
        return PROSPER_EINVAL;
    }
    DscArgs A;
    A.sel = c->sel; A.selp = c->selp; A.yy = reinterpret_cast<const float2 *>(c->yy); A.G = c->G;
    A.tab = reinterpret_cast<const uint2 *>(c->dsc_tab);
    A.theta = theta; A.N = N; A.n_offset = n_offset;
    A.H = c->H; A.D = c->D; A.Hp = c->Hp; A.gamma = c->gamma; A.nK = c->nK; A.m = c->dsc_m;
    A.model = c->model;
    A.nslot = c->Hp + c->Hp * (c->Hp + 1) / 2 + c->dsc_m;
    A.wstride = dsc_wstride(c->Hp, c->dsc_m);
    A.phi0 = c->dsc_vals[0]; A.phi1 = c->dsc_vals[1]; A.phi2 = c->dsc_vals[2];
    A.es = c->es;
    A.B = st ? st->B : nullptr;
    A.scal = st ? st->scal : nullptr;
    A.sel_out = sel_out; A.map_out = map_out; A.mapv_out = mapv_out; A.smean_out = smean_out;
    A.mapp_out = mapp_out; A.logz_out = logz_out;
    A.cut_thr = (st && c->cut) ? c->cut_thr : nullptr;
    A.cut_logz = A.cut_thr ? c->cut_logz + c->cut_n0 : nullptr;
    const bool enc = (st == nullptr);
    const size_t smem = dsc_smem_bytes(c->Hp, c->dsc_m);
    const void *fn = enc ? (const void *)k_dsc_states<true> : (const void *)k_dsc_states<false>;
    if (int rc = ensure_smem_attr(fn, smem)) return rc;
    const int64_t ctas = (N + XW - 1) / XW;
    const int grid = (int)std::min<int64_t>(ctas, (int64_t)c->num_sms);
    TraceScope tr(c, enc ? "dsc_states_encode" : "dsc_states", s);
    if (enc) k_dsc_states<true><<<grid, XW * 32, smem, s>>>(A);
    else k_dsc_states<false><<<grid, XW * 32, smem, s>>>(A);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

}  // namespace prosper
