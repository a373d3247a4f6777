// bsc.cu -- binary sparse coding (BSC, Table 1 row 1: linear superposition
// f = W s, Gaussian noise, binary latents, Bernoulli prior) truncated E-step.
//
// Path per call (paper Sec. 2, EM with truncated posteriors):
//   k_prep                    per-iteration constants in one launch: G = W^T W,
//                             1/||W_h||, W (D x H), the BF16 unit-norm image
//   k_bsc_proj_f32            FP32 SIMT projection W^T y_n for all H latents of a
//                             64-point tile by 8 product warps, top-H' preselection
//                             by the score W_h^T y / ||W_h|| (ties to the lower h)
//                             by 4 ranking warps, one warp per point
//   k_bsc_states<H'>          one thread per point: every state with <= gamma active
//                             units among the H' candidates, log-sum-exp, posterior
//                             moments, MAP; FP64 accumulation of sum <ss^T>, F, ...
//   k_astat                   sum_n <s>_n y_n^T by a per-tile sort on the latent index
//   k_symmetrize              B lower triangle from the upper one
//
// Log-joint of a state s over the candidates I (exact algebra from
// ||y - W s||^2 = y^T y - 2 s^T W^T y + s^T W^T W s, Eq. 2):
//   log p(s,y) - log p(0,y) = |s| log(pi/(1-pi)) + (s^T p - s^T G_II s / 2) / sigma^2
// with p = W_I^T y.  Kernels work in base 2 (all terms times log2 e).
#include "internal.cuh"
#include "topk.cuh"
#include "f32x2.cuh"
#include "tc.cuh"

#include <cmath>
#include <cuda_bf16.h>

namespace prosper {

namespace {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2Pi = 1.8378770664093454836;

// ------------------------------------------------------------------ prep
// The per-iteration constants in one launch.  Block (x, y) computes the 16 x 16
// tile G[i][j] = sum_d Wt[i][d] Wt[j][d] (i = 16 y + ty, j = 16 x + tx) with the
// tile's 32 rows of Wt staged in shared memory at once (padded rows, so the 16
// rows read in one step fall in different banks).  The diagonal blocks also
// write 1/||W_h|| (0 for a zero row) and, where asked, W in the D x H layout of
// the FP32 projection (Wd[d][h] = Wt[h][d]) and the BF16 image of the unit-norm
// rows W_h / ||W_h|| in the tensor-core operand layout of the BF16 projection:
// K-block kb holds rows h of 128 B (d = 64 kb .. 64 kb + 63), 16-byte chunk c at
// chunk position c ^ (h & 7).
__global__ void __launch_bounds__(256) k_prep(const float *__restrict__ Wt, int H, int D,
                                              float *__restrict__ G, float *__restrict__ rnorm,
                                              float *__restrict__ Wd, uint16_t *__restrict__ Wb) {
    extern __shared__ float prep_sm[];
    __shared__ float s_rn[16];
    const int P = D + 1;
    float *As = prep_sm, *Bs = prep_sm + 16 * P;
    const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
    const bool diag = i0 == j0;                 // block-uniform
    // 256 columns at a time, all 32 rows' loads in flight before the stores
    for (int d0 = 0; d0 < D; d0 += 256) {
        const int d = d0 + threadIdx.x;
        float va[16], vb[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            va[r] = (d < D && i0 + r < H) ? __ldg(Wt + (size_t)(i0 + r) * D + d) : 0.f;
            vb[r] = (d < D && j0 + r < H && !diag) ? __ldg(Wt + (size_t)(j0 + r) * D + d) : 0.f;
        }
        if (d < D) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                As[r * P + d] = va[r];
                if (!diag) Bs[r * P + d] = vb[r];
            }
        }
    }
    __syncthreads();
    const float *Bv = diag ? As : Bs;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc = 0.f;
#pragma unroll 16
    for (int d = 0; d < D; ++d) acc = fmaf(As[ty * P + d], Bv[tx * P + d], acc);
    if (i0 + ty < H && j0 + tx < H) G[(size_t)(i0 + ty) * H + j0 + tx] = acc;
    if (!diag) return;
    if (tx == ty) {
        const float rn = acc > 0.f ? rsqrtf(acc) : 0.f;
        s_rn[ty] = rn;
        if (i0 + ty < H) rnorm[i0 + ty] = rn;
    }
    __syncthreads();
    if (Wd) {
        for (int idx = threadIdx.x; idx < 16 * D; idx += 256) {
            const int d = idx >> 4, r = idx & 15;
            if (i0 + r < H) Wd[(size_t)d * H + i0 + r] = As[r * P + d];
        }
    }
    if (Wb) {
        for (int idx = threadIdx.x; idx < 16 * D; idx += 256) {
            const int r = idx / D, d = idx - r * D, h = i0 + r;
            if (h >= H) continue;
            const int kb = d >> 6, ch = (d & 63) >> 3, w = d & 7;
            const size_t off = (size_t)kb * H * 64 + (size_t)h * 64 + (size_t)((ch ^ (h & 7)) * 8 + w);
            const __nv_bfloat16 bv = __float2bfloat16_rn(As[r * P + d] * s_rn[r]);
            Wb[off] = *reinterpret_cast<const uint16_t *>(&bv);
        }
    }
}

// ------------------------------------------------ FP32 projection + selection
constexpr int PT = 64;        // points per tile
constexpr int PK = 32;        // d per k-chunk
constexpr int PH = 256;       // max H of this kernel
constexpr int PS = PH + 4;    // padded row of the projection tile in smem

constexpr int PNP = 8;        // product warps (256 threads: 8 x 8 blocks of the tile)
constexpr int PNR = 4;        // ranking warps
constexpr unsigned long long kProjWaitNs = 2000000000ull;   // bounded mbarrier wait: 2 s

struct ProjSmem {
    float Ys[2][PK][PT];      // 16 KB  (d-major so a thread reads 8 points with 2 LDS.128)
    float Ws[2][PK][PH];      // 64 KB
    float Ps[2][PT][PS];      // 133 KB (tile t in Ps[t % 2] while tile t + 1 is multiplied)
    unsigned topk[PNR][64];   // per-ranking-warp selection scratch
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = pred ? 16 : 0;   // src-size 0 zero-fills the 16 bytes
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Grid: persistent, one 384-thread CTA per SM, warp-specialised.  Product
// thread (tp = tid & 7, th = tid >> 3, tid < 256) accumulates the 8 x 8 block
// P[tp*8 + i][th*8 + j] of the 64 x 256 tile.  The k-chunks of all tiles form one
// software pipeline: while chunk q is multiplied, the Y values of chunk q+1 are
// in flight into registers and its W rows into the other shared-memory stage
// (cp.async); the product warps meet on named barrier 1 per chunk.  At a tile's
// end they write its projections to Ps[t % 2] and arrive on full[t % 2]; the
// four ranking warps take the top-H' of the tile's 64 points (16 each) while the
// products of the next tile run, then arrive on empty[t % 2], which the product
// warps wait for before they write that buffer again.  Every wait is bounded;
// a wait that gives up stops both roles and the CTA writes in-bounds candidate
// lists for all its points.
// RMAX: the largest Hprime of the instantiation (10 or 16); the selection
// rounds are unrolled up to it
template <int RMAX>
__global__ void __launch_bounds__(32 * (PNP + PNR), 1)
k_bsc_proj_f32(const float *__restrict__ Y, const float *__restrict__ Wd,
               const float *__restrict__ rnorm, int64_t N, int D, int H, int Hp, int score_mode,
               int32_t *__restrict__ sel_out, float *__restrict__ selp_out,
               float2 *__restrict__ yy_out, unsigned *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ProjSmem &sm = *reinterpret_cast<ProjSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tp = tid & 7, th = tid >> 3;
    const int64_t ntiles = (N + PT - 1) / PT;
    const bool vecY = (D % 4) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
    const bool vecW = (H % 4) == 0;
    const int nk = (D + PK - 1) / PK;
    const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int64_t nq = my_tiles * nk;   // chunks this CTA processes

    // score = sign * P_h / ||W_h||; score_mode 1 (discrete latents with values
    // of both signs) ranks by magnitude instead
    const float sgn = score_mode == 2 ? -1.f : 1.f;
    const bool mag = score_mode == 1;
    float rn[8];
    unsigned kmask[8], klow[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int h = lane + 32 * j;
        rn[j] = h < H ? sgn * rnorm[h] : 0.f;
        kmask[j] = h < H ? 0xFFFFFF00u : 0u;
        klow[j] = h < H ? (unsigned)(255 - h) : 0u;
    }
    __shared__ uint64_t bar_full[2], bar_empty[2];
    __shared__ volatile int s_abort;
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tc::smem_u32(&bar_full[b]), 32 * PNP);
            tc::mbar_init(tc::smem_u32(&bar_empty[b]), PNR);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // Y chunk mapping: thread loads float4 (q4 = idx & 7) of point p = idx >> 3, idx = tid + 256 r
    float4 yreg[2];
    auto load_y = [&](int64_t q) {
        const int64_t tile = blockIdx.x + (q / nk) * gridDim.x;
        const int k0 = (int)(q % nk) * PK;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + 256 * r;
            const int p = idx >> 3, q4 = idx & 7;
            const int64_t n = tile * PT + p;
            const int d = k0 + q4 * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n < N) {
                const float *row = Y + n * D;
                if (vecY && d + 3 < D) {
                    v = __ldg(reinterpret_cast<const float4 *>(row + d));
                } else {
                    if (d < D) v.x = row[d];
                    if (d + 1 < D) v.y = row[d + 1];
                    if (d + 2 < D) v.z = row[d + 2];
                    if (d + 3 < D) v.w = row[d + 3];
                }
            }
            yreg[r] = v;
        }
    };
    // partial y^T y of points tid/8 and tid/8 + 32 over this thread's d slices
    float ysq[2] = {0.f, 0.f};
    auto store_y = [&](int st) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + 256 * r;
            const int p = idx >> 3, q4 = idx & 7;
            sm.Ys[st][q4 * 4 + 0][p] = yreg[r].x;
            sm.Ys[st][q4 * 4 + 1][p] = yreg[r].y;
            sm.Ys[st][q4 * 4 + 2][p] = yreg[r].z;
            sm.Ys[st][q4 * 4 + 3][p] = yreg[r].w;
            float q = ysq[r];
            q = fmaf(yreg[r].x, yreg[r].x, q); q = fmaf(yreg[r].y, yreg[r].y, q);
            q = fmaf(yreg[r].z, yreg[r].z, q); q = fmaf(yreg[r].w, yreg[r].w, q);
            ysq[r] = q;
        }
    };
    auto load_w = [&](int64_t q, int st) {
        const int k0 = (int)(q % nk) * PK;
        for (int idx = tid; idx < PK * (PH / 4); idx += 256) {
            const int kk = idx >> 6, c4 = (idx & 63) * 4;
            const int d = k0 + kk;
            const float *src = Wd + (size_t)(d < D ? d : 0) * H + c4;
            if (vecW) {
                cp_async16(&sm.Ws[st][kk][c4], src, d < D && c4 < H);
            } else {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (d < D) {
                    if (c4 < H) v.x = src[0];
                    if (c4 + 1 < H) v.y = src[1];
                    if (c4 + 2 < H) v.z = src[2];
                    if (c4 + 3 < H) v.w = src[3];
                }
                *reinterpret_cast<float4 *>(&sm.Ws[st][kk][c4]) = v;
            }
        }
        cp_async_commit();
    };

    // Top-H' of point p of the tile whose projections are in Ps[pb] (a ranking
    // warp): H'+1 rounds of the warp maximum over packed keys (24-bit score
    // prefix, then 255 - h).  When the H'-th and (H'+1)-th winners differ in the
    // prefix, every latent left out has a smaller exact score than every one
    // taken, so the set is the exact top-H'; otherwise (scores within 2^-15 of
    // each other across the boundary, exact ties included) the exact selection
    // decides.
    auto select_point = [&](int pb, int p, int64_t n) {
        unsigned pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float sc = kmask[j] ? sm.Ps[pb][p][lane + 32 * j] * rn[j] : 0.f;
            pk[j] = packed_key(mag ? fabsf(sc) : sc, kmask[j], klow[j]);
        }
        sort8_desc(pk);
        int myh = 0x7fffffff;
        unsigned wlast = 0u, wnext = 0u;
#pragma unroll
        for (int r = 0; r <= RMAX; ++r) {
            if (r <= Hp) {   // warp-uniform
                const unsigned w = __reduce_max_sync(0xffffffffu, pk[0]);
                if (lane == r && r < Hp) myh = 255 - (int)(w & 0xFFu);
                if (r == Hp - 1) wlast = w;
                if (r == Hp) wnext = w;
                if (pk[0] == w) {
#pragma unroll
                    for (int j = 0; j < 7; ++j) pk[j] = pk[j + 1];
                    pk[7] = 0u;
                }
            }
        }
        if (Hp < H && (wlast >> 8) == (wnext >> 8)) {
            unsigned key[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int h = lane + 32 * j;
                const float sc = sm.Ps[pb][p][lane + 32 * j] * rn[j];
                key[j] = h < H ? score_key(mag ? fabsf(sc) : sc) : 0u;
            }
            myh = warp_topk(key, Hp, lane, sm.topk[warp - PNP]);
        }
        int rank = 0;
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            const int o = __shfl_sync(0xffffffffu, myh, r);
            rank += (r < Hp && o < myh) ? 1 : 0;
        }
        if (lane < Hp) {
            sel_out[n * SEL_STRIDE + rank] = myh;
            selp_out[n * SEL_STRIDE + rank] = sm.Ps[pb][p][myh];
        }
    };

    if (warp < PNP) {
        // ------------------------------------------------------ product warps
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

        if (nq > 0) {
            load_y(0);
            load_w(0, 0);
        }
        for (int64_t q = 0; q < nq; ++q) {
            const int st = (int)(q & 1);
            store_y(st);
            cp_async_wait_all();
            tc::named_sync(1, 32 * PNP);
            if (q + 1 < nq) {
                load_y(q + 1);
                load_w(q + 1, st ^ 1);
            }
#pragma unroll 4
            for (int kk = 0; kk < PK; ++kk) {
                float4 y0 = *reinterpret_cast<const float4 *>(&sm.Ys[st][kk][tp * 8]);
                float4 y1 = *reinterpret_cast<const float4 *>(&sm.Ys[st][kk][tp * 8 + 4]);
                float4 w0 = *reinterpret_cast<const float4 *>(&sm.Ws[st][kk][th * 8]);
                float4 w1 = *reinterpret_cast<const float4 *>(&sm.Ws[st][kk][th * 8 + 4]);
                float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
                float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; j += 2) ffma2(acc[i][j], acc[i][j + 1], yv[i], wv[j], wv[j + 1]);
            }
            if ((q % nk) != nk - 1) continue;

            // ---- tile end: projections to Ps[t % 2] once the ranking warps are
            //      done with its previous tile (the same decision in every
            //      product thread: they share named barrier 1)
            const int t = (int)(q / nk);
            const int b = t & 1;
            bool ok = true;
            if (t >= 2) ok = tc::mbar_wait(tc::smem_u32(&bar_empty[b]), (uint32_t)(((t - 2) >> 1) & 1), kProjWaitNs);
            if (tc::named_sync_or(1, 32 * PNP, !ok)) {
                if (tid == 0) s_abort = 1;
                break;
            }
            const int64_t n0 = (blockIdx.x + (int64_t)t * gridDim.x) * PT;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float *row = &sm.Ps[b][tp * 8 + i][th * 8];
                *reinterpret_cast<float4 *>(row) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                *reinterpret_cast<float4 *>(row + 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            }
            // y^T y of the tile's points: the 8 threads of a point add their slices
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float yq = ysq[r];
                yq += __shfl_xor_sync(0xffffffffu, yq, 1);
                yq += __shfl_xor_sync(0xffffffffu, yq, 2);
                yq += __shfl_xor_sync(0xffffffffu, yq, 4);
                const int64_t n = n0 + (tid >> 3) + 32 * r;
                if ((tid & 7) == 0 && n < N) {
                    yy_out[n] = make_float2(yq, 0.f);
                    if (!isfinite(yq)) atomicOr(status, ST_NONFINITE);
                }
                ysq[r] = 0.f;
            }
            tc::mbar_arrive(tc::smem_u32(&bar_full[b]));
        }
        cp_async_wait_all();   // no copy outlives the loop (it may have been left early)
    } else {
        // ------------------------------------------------------ ranking warps
        const int rw = warp - PNP;
        for (int64_t t = 0; t < my_tiles; ++t) {
            const int b = (int)(t & 1);
            // a sleeping wait: the ranking warps leave the issue slots to the
            // product warps until the tile is there
            if (!__all_sync(0xffffffffu, tc::mbar_wait_sleep(tc::smem_u32(&bar_full[b]), (uint32_t)((t >> 1) & 1),
                                                                kProjWaitNs))) {
                s_abort = 1;
                break;
            }
            const int64_t n0 = (blockIdx.x + t * gridDim.x) * PT;
            for (int sp = 0; sp < PT / PNR; ++sp) {
                const int p = rw * (PT / PNR) + sp;
                if (n0 + p >= N) break;   // warp-uniform
                select_point(b, p, n0 + p);
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_u32(&bar_empty[b]));
        }
    }
    __syncthreads();
    if (s_abort) {
        // a wait gave up: flag it and give every point of this CTA a valid (if
        // meaningless) candidate list so that the later kernels stay in bounds
        if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
        for (int64_t t = 0; t < my_tiles; ++t) {
            const int64_t n0 = (blockIdx.x + t * gridDim.x) * PT;
            for (int k = tid; k < PT * SEL_STRIDE; k += 32 * (PNP + PNR)) {
                const int64_t n = n0 + k / SEL_STRIDE;
                if (n >= N) continue;
                const int j = k % SEL_STRIDE;
                sel_out[n * SEL_STRIDE + j] = j < H ? j : 0;
                selp_out[n * SEL_STRIDE + j] = 0.f;
                if (j == 0) yy_out[n] = make_float2(0.f, 0.f);
            }
        }
    }
}

// ----------------------------------------------------------- state kernel
// Bit helpers on compile-time-constant patterns: written with intrinsics so that
// they fold to constants inside unrolled loops (recursive constexpr helpers are
// not inlined by the device compiler and would run at run time).
#define cpopc(t) __popc((unsigned)(t))
#define cctz(t) (__ffs((int)(t)) - 1)
// sum over the hi units u in t of 2^(HP-1-(LB+u)): the weight of t in the
// bit-reversed state mask (lower local unit = higher weight).
#define crev_hi(t, LB, HP) ((int)(__brev((unsigned)(t) << (LB)) >> (32 - (HP))))

// FP32 -> FP64 by the IEEE-754 field layout on the integer pipe (exact for
// every normal float; subnormals become 0, infinities and NaNs keep their
// class).  On this part the FP64 pipe issues one warp instruction per ~20
// clocks per SM, so the 55 conversions per point of the B accumulation are
// kept off it.
__device__ __forceinline__ double f32_to_f64_bits(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned m = (e == 0u) ? 0u : (u & 0x7FFFFFu);
    const unsigned e64 = (e == 0u) ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u);
    return __hiloint2double((int)((u & 0x80000000u) | (e64 << 20) | (m >> 3)), (int)(m << 29));
}

__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct StateArgs {
    const int32_t *sel;
    const float *selp;
    const float2 *yy;
    const float *G;
    int64_t N;
    int H, D, gamma;
    const double *theta;
    // outputs (estep)
    float *es;
    double *B, *scal;
    // outputs (encode)
    int16_t *sel_out, *map_out;
    float *smean_out, *mapp_out, *logz_out;
    int64_t n_offset;   // row offset of this piece in the encode outputs
    // E-step with the data cut: the first pass's log Z of this piece's points
    // and the threshold; a point below it is left out
    const float *cut_logz, *cut_thr;
    prosper_ctx *trace_ctx;
};

// L(lo) = sum_{j in lo} a_j + sum_{i<j in lo} b_ij and c_u(lo) = a_u + sum_{i in lo} b_iu,
// branch-free with 0/1 multipliers (fmaf(0, x, s) = s and fmaf(1, x, s) = s + x
// exactly, so these equal the plain sums), then C[t] = L + sum_{u in t} c_u,
// held as pairs CP[k] = (C[2k], C[2k+1]): CP[k] = CP[k minus its lowest bit] +
// c_{ctz(k)+1} on both halves (packed adds), CP[0] = (L, L + c_0).
#define PROSPER_LO_TERMS()                                                        \
    float mk[LBX];                                                                 \
    float2 CP[NT2];                                                                \
    {                                                                              \
        _Pragma("unroll") for (int i = 0; i < LB; ++i) mk[i] = (float)((lo >> i) & 1); \
        float L = 0.f;                                                             \
        _Pragma("unroll") for (int i = 0; i < LB; ++i) {                           \
            L = fmaf(mk[i], a[i], L);                                              \
            _Pragma("unroll") for (int j = i + 1; j < LB; ++j)                     \
                L = fmaf(mk[i] * mk[j], b[i][j], L);                               \
        }                                                                          \
        float c[HB];                                                               \
        _Pragma("unroll") for (int u = 0; u < HB; ++u) {                           \
            float v = a[LB + u];                                                   \
            _Pragma("unroll") for (int i = 0; i < LB; ++i) v = fmaf(mk[i], b[i][LB + u], v); \
            c[u] = v;                                                              \
        }                                                                          \
        CP[0] = make_float2(L, L + c[0]);                                          \
        _Pragma("unroll") for (int k = 1; k < NT2; ++k) {                          \
            const float cc = c[cctz(k) + 1];                                       \
            CP[k] = add2(CP[k & (k - 1)], make_float2(cc, cc));                    \
        }                                                                          \
    }

// l(t) of the current lo pattern from the packed pairs
#define PROSPER_L(t) (((t) & 1) ? LP[(t) >> 1].y : LP[(t) >> 1].x)

// Pass 1 body for group K: running maximum.
#define PROSPER_P1_GROUP(K)                                                        \
    if ((K) <= HB && (K) <= cap) {                                                 \
        _Pragma("unroll") for (int t = 0; t < NT; ++t) {                           \
            if (cpopc(t) == (K)) m = fmaxf(m, PROSPER_L(t));                       \
        }                                                                          \
    }

// Pass 2 body for group K: e = 2^(l - m) and the MAP key of states with l == m.
#define PROSPER_P2_GROUP(K)                                                        \
    if ((K) <= HB) {                                                               \
        if ((K) <= cap) {                                                          \
            _Pragma("unroll") for (int t = 0; t < NT; ++t) {                       \
                if (cpopc(t) == (K)) {                                             \
                    const float d = ((t) & 1) ? DP[(t) >> 1].y : DP[(t) >> 1].x;   \
                    const float ev = fast_ex2(d);                                  \
                    if ((t) & 1) EP[(t) >> 1].y = ev; else EP[(t) >> 1].x = ev;   \
                    const int key = klo + ((cpopc(t) << 16) - crev_hi(t, LB, HP)); \
                    best = min(best, (d == 0.f) ? key : 0x7fffffff);               \
                }                                                                  \
            }                                                                      \
        } else {                                                                   \
            _Pragma("unroll") for (int t = 0; t < NT; ++t)                         \
                if (cpopc(t) == (K)) {                                             \
                    if ((t) & 1) EP[(t) >> 1].y = 0.f; else EP[(t) >> 1].x = 0.f;  \
                }                                                                  \
        }                                                                          \
    }

// One thread per data point.  Local units 0..LB-1 ("lo") are enumerated by a
// warp-uniform loop; units LB..HP-1 ("hi", HB = min(HP,5) of them) are
// unrolled, so each lo pattern evaluates its 2^HB hi patterns from registers:
//   l(lo, t) = L(lo) + sum_{u in t} c_u(lo) + M(t),   M(t) = sum_{u<v in t} b_uv,
// with a_j = log2e (log(pi/(1-pi)) + (p_j - G_jj/2)/sigma^2) / T, b_ij = -log2e G_ij/(sigma^2 T).
// Hi patterns are grouped by their number of active units; a group is skipped
// by one warp-uniform branch when lo plus the group exceeds gamma units.
// Pass 1 finds the maximum m; pass 2 forms e = 2^(l - m), the moments and the
// MAP state (the canonically first state with l == m, found by a min over the
// key (|s| << 16) + 0xFFFF - bitreverse(s)).
// The E-step form at H' >= 9 keeps its second-moment table in registers at two
// CTAs per SM (about 230 registers); at three it spills (A/B at H' = 10,
// 200,000 points: 0.175 -> 0.160 ms).
template <int HP, bool ENCODE>
__global__ void __launch_bounds__(128, (HP >= 9 && !ENCODE) ? 2 : 3) k_bsc_states(StateArgs A) {
    constexpr int HB = HP < 5 ? HP : 5;
    constexpr int LB = HP - HB;
    constexpr int NT = 1 << HB;
    constexpr int NT2 = NT / 2;       // packed pairs of hi patterns (HB >= 1)
    constexpr int NLO = 1 << LB;
    constexpr int LBX = LB > 0 ? LB : 1;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = n < A.N;
    const int64_t nn = valid ? n : 0;

    // per-call constants, formed once per CTA (FP64 logs and divisions are
    // slow on this part):  lpi = log2e log(pi/(1-pi)),  is2 = log2e / sigma^2,
    // log p(y, s=0) = c0 - y^T y / (2 sigma^2)
    // (the FP64 chains run in lane 0 of four different warps, i.e. on four
    // SM sub-partitions, while every thread loads its candidate list and G block)
    // Deterministic annealing: every log-joint is divided by the temperature T
    // (theta[3]; <= 0 reads as 1) before the log-sum-exp, so q ~ p(s,y)^(1/T) and
    // log Z = T log sum_{K_n} p(s,y)^(1/T).
    __shared__ float s_lpi, s_is2;
    __shared__ double s_c0, s_inv2s2, s_T;
    if ((threadIdx.x & 31) == 0) {
        const double pi = A.theta[PROSPER_TH_PI], sigma = A.theta[PROSPER_TH_SIGMA];
        const double th = A.theta[PROSPER_TH_T];
        const double T = th > 0.0 ? th : 1.0;
        const double s2 = sigma * sigma;
        switch (threadIdx.x >> 5) {
            case 0: s_lpi = (float)(log(pi / (1.0 - pi)) * 1.4426950408889634 / T); break;
            case 1: s_is2 = (float)(1.4426950408889634 / (s2 * T)); break;
            case 2: s_c0 = A.H * log(1.0 - pi) - 0.5 * A.D * (kLog2Pi + log(s2)); s_T = T; break;
            default: s_inv2s2 = 0.5 / s2; break;
        }
    }
    const int gamma = A.gamma;
    const int H = A.H;

    // candidate lists and their projections: rows of SEL_STRIDE (16) entries,
    // 64-byte aligned, read as 16-byte vectors
    constexpr int NV = (HP + 3) / 4;
    int I[HP];
    float P[HP];
    {
        const int4 *sr = reinterpret_cast<const int4 *>(A.sel + nn * SEL_STRIDE);
        const float4 *pr = reinterpret_cast<const float4 *>(A.selp + nn * SEL_STRIDE);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int4 iv = sr[q];
            const float4 pv = pr[q];
            const int ia[4] = {iv.x, iv.y, iv.z, iv.w};
            const float pa[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (4 * q + k < HP) {
                    I[4 * q + k] = min(max(ia[k], 0), H - 1);   // defensive
                    P[4 * q + k] = pa[k];
                }
        }
    }
    float g[HP][HP];
#pragma unroll
    for (int i = 0; i < HP; ++i)
#pragma unroll
        for (int j = i; j < HP; ++j) g[i][j] = __ldg(A.G + (size_t)I[i] * H + I[j]);
    __syncthreads();
    const float lpi = s_lpi, is2 = s_is2;
    float a[HP], b[HP][HP];
#pragma unroll
    for (int j = 0; j < HP; ++j) {
        float pj = P[j];
        float gjj = g[j][j];
        a[j] = lpi + (pj - 0.5f * gjj) * is2;
        b[j][j] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < HP; ++i)
#pragma unroll
        for (int j = i + 1; j < HP; ++j) {
            b[i][j] = -g[i][j] * is2;
            b[j][i] = b[i][j];
        }

    float2 MP[NT2];                   // (M[2k], M[2k+1])
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < HB; ++u)
#pragma unroll
            for (int v = u + 1; v < HB; ++v)
                if (((t >> u) & 1) && ((t >> v) & 1)) s += b[LB + u][LB + v];
        if (t & 1) MP[t >> 1].y = s; else MP[t >> 1].x = s;
    }

    // -------- pass 1: maximum log-joint over the valid states
    float m = -INFINITY;
#pragma unroll 1
    for (int lo = 0; lo < NLO; ++lo) {
        const int cap = gamma - __popc(lo);
        if (cap < 0) continue;
        PROSPER_LO_TERMS();
        float2 LP[NT2];
#pragma unroll
        for (int k = 0; k < NT2; ++k) LP[k] = add2(CP[k], MP[k]);
        PROSPER_P1_GROUP(0);
        PROSPER_P1_GROUP(1);
        PROSPER_P1_GROUP(2);
        PROSPER_P1_GROUP(3);
        PROSPER_P1_GROUP(4);
        PROSPER_P1_GROUP(5);
    }

    // -------- pass 2: exponentials, moments, MAP
    float Z = 0.f;
    float LL[LBX][LBX];
    float LH[LBX][HB];
    float2 GP[NT2];                   // (Gacc[2k], Gacc[2k+1])
#pragma unroll
    for (int i = 0; i < LBX; ++i) {
#pragma unroll
        for (int j = 0; j < LBX; ++j) LL[i][j] = 0.f;
#pragma unroll
        for (int u = 0; u < HB; ++u) LH[i][u] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < NT2; ++k) GP[k] = make_float2(0.f, 0.f);
    int best = 0x7fffffff;

#pragma unroll 1
    for (int lo = 0; lo < NLO; ++lo) {
        const int cap = gamma - __popc(lo);
        if (cap < 0) continue;
        PROSPER_LO_TERMS();
        const int klo = (__popc(lo) << 16) + 0xFFFF - (int)(__brev((unsigned)lo) >> (32 - HP));
        float2 DP[NT2], EP[NT2];          // l - m and 2^(l - m), pairs
#pragma unroll
        for (int k = 0; k < NT2; ++k) DP[k] = sub2(add2(CP[k], MP[k]), make_float2(m, m));
        PROSPER_P2_GROUP(0);
        PROSPER_P2_GROUP(1);
        PROSPER_P2_GROUP(2);
        PROSPER_P2_GROUP(3);
        PROSPER_P2_GROUP(4);
        PROSPER_P2_GROUP(5);
#pragma unroll
        for (int k = 0; k < NT2; ++k) GP[k] = add2(GP[k], EP[k]);
        // R[u] = sum_{t contains u} e[t] and the total Zlo, folding the pairs
        // on the highest hi unit first (packed adds), then the pair itself
        float R[HB];
        float Zlo;
        {
            int np = NT2;
#pragma unroll
            for (int u = HB - 1; u >= 1; --u) {
                np >>= 1;
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < NT2 / 2; ++k) {
                    if (k < np) {
                        acc = add2(acc, EP[k + np]);
                        EP[k] = add2(EP[k], EP[k + np]);
                    }
                }
                R[u] = acc.x + acc.y;
            }
            R[0] = EP[0].y;
            Zlo = EP[0].x + EP[0].y;
        }
#pragma unroll
        for (int i = 0; i < LB; ++i) {
#pragma unroll
            for (int u = 0; u < HB; ++u) LH[i][u] = fmaf(mk[i], R[u], LH[i][u]);
            LL[i][i] = fmaf(mk[i], Zlo, LL[i][i]);
#pragma unroll
            for (int j = i + 1; j < LB; ++j) LL[i][j] = fmaf(mk[i] * mk[j], Zlo, LL[i][j]);
        }
        Z += Zlo;
    }

    // second moments <s_i s_j> (unnormalised) in one symmetric table
    float S2[HP][HP];
#pragma unroll
    for (int i = 0; i < HP; ++i)
#pragma unroll
        for (int j = i; j < HP; ++j) {
            float v;
            if (j < LB) {
                v = LL[i < LB ? i : 0][j < LB ? j : 0];
            } else if (i < LB) {
                v = LH[i < LB ? i : 0][j - LB];
            } else {
                const int u = i - LB, w = j - LB;
                float s = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t)
                    if (((t >> u) & 1) && ((t >> w) & 1)) s += ((t & 1) ? GP[t >> 1].y : GP[t >> 1].x);
                v = s;
            }
            S2[i][j] = v;
        }
    const float invZ = 1.f / Z;
    float es[HP];
#pragma unroll
    for (int j = 0; j < HP; ++j) es[j] = S2[j][j] * invZ;

    const float2 yyv = A.yy[nn];
    const double yy = (double)yyv.x + (double)yyv.y;
    const double logp0 = fma(-yy, s_inv2s2, s_c0);
    const double logZ = ((double)m + (double)log2f(Z)) * (kLn2 * s_T) + logp0;
    // MAP state mask from the winning key
    const unsigned rmask = 0xFFFFu - (unsigned)(best & 0xFFFF);
    unsigned mapmask = 0u;
#pragma unroll
    for (int j = 0; j < HP; ++j) mapmask |= ((rmask >> (HP - 1 - j)) & 1u) << j;

    if (ENCODE) {
        if (valid) {
            const int64_t o = A.n_offset + n;
            if (A.sel_out)
#pragma unroll
                for (int j = 0; j < HP; ++j) A.sel_out[o * HP + j] = (int16_t)I[j];
            if (A.smean_out)
#pragma unroll
                for (int j = 0; j < HP; ++j) A.smean_out[o * HP + j] = es[j];
            if (A.map_out) {
                int k = 0;
#pragma unroll
                for (int j = 0; j < HP; ++j)
                    if (((mapmask >> j) & 1u) && k < gamma) A.map_out[o * gamma + k++] = (int16_t)I[j];
                for (; k < gamma; ++k) A.map_out[o * gamma + k] = (int16_t)-1;
            }
            if (A.mapp_out) A.mapp_out[o] = invZ;
            if (A.logz_out) A.logz_out[o] = (float)logZ;
        }
        return;
    }

    // the data cut leaves a point out of every statistic (its <s> row is
    // zeroed for sum y<s>^T); the decision reads the FP32 log Z the first
    // pass stored, so it is the one the threshold was taken on
    const bool kept = valid && (A.cut_thr == nullptr || A.cut_logz[n] >= *A.cut_thr);
    if (valid && !kept) {
        float4 *er = reinterpret_cast<float4 *>(A.es + n * SEL_STRIDE);
#pragma unroll
        for (int q = 0; q < NV; ++q) er[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (kept) {
        float4 *er = reinterpret_cast<float4 *>(A.es + n * SEL_STRIDE);
#pragma unroll
        for (int q = 0; q < NV; ++q)
            er[q] = make_float4(es[4 * q], 4 * q + 1 < HP ? es[(4 * q + 1) % HP] : 0.f,
                                4 * q + 2 < HP ? es[(4 * q + 2) % HP] : 0.f,
                                4 * q + 3 < HP ? es[(4 * q + 3) % HP] : 0.f);
        // sum <s s^T> into the upper triangle of B (I ascending -> I_i < I_j);
        // the candidate list is read again here rather than kept in registers
        int J[HP];
        {
            const int4 *sr = reinterpret_cast<const int4 *>(A.sel + nn * SEL_STRIDE);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const int4 iv = sr[q];
                const int ia[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (4 * q + k < HP) J[4 * q + k] = min(max(ia[k], 0), H - 1);
            }
        }
#pragma unroll
        for (int i = 0; i < HP; ++i) {
            double *row = A.B + (size_t)J[i] * H;
#pragma unroll
            for (int j = i; j < HP; ++j) atomicAdd(row + J[j], f32_to_f64_bits(S2[i][j] * invZ));
        }
    }
    // scalar statistics: warp sums (F and y^T y in FP64, sum <|s|> in FP32 over
    // the 32 points, the count by ballot), one atomic per warp
    float s1 = 0.f;
    double f = 0.0, y2 = 0.0;
    if (kept) {
#pragma unroll
        for (int j = 0; j < HP; ++j) s1 += es[j];
        f = logZ;
        y2 = yy;
    }
    const unsigned cnt = __popc(__ballot_sync(0xffffffffu, kept));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        f += __shfl_xor_sync(0xffffffffu, f, o);
        y2 += __shfl_xor_sync(0xffffffffu, y2, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0u) {
        atomicAdd(A.scal + PROSPER_SC_F, f);
        atomicAdd(A.scal + PROSPER_SC_S1, (double)s1);
        atomicAdd(A.scal + PROSPER_SC_YY, y2);
        atomicAdd(A.scal + PROSPER_SC_N, (double)cnt);
    }
}

// ----------------------------------------------------- sum_n <s>_n y_n^T
// Grid (ceil(D/64), ranges).  A CTA owns a 64-wide slice of d for its range of
// points and keeps At[:, slice] in shared memory.  Per 256-point chunk the
// (point, <s>) pairs are bucketed by latent h; warp w then owns latents
// h = w, w+8, ... so every shared-memory row has a single writer.
constexpr int AT = 128;   // points per chunk
constexpr int AD = 64;    // d per slice

__global__ void __launch_bounds__(256, 2)
k_astat(const float *__restrict__ Y, const int32_t *__restrict__ sel, const float *__restrict__ es,
        int64_t N, int D, int H, int Hp, int64_t pts_per_cta, double *__restrict__ At) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Apart = reinterpret_cast<float *>(smem_raw);              // H x AD
    float *Ys = Apart + (size_t)H * AD;                              // AT x AD
    float *lv = Ys + AT * AD;                                        // AT*Hp values
    int *ln = reinterpret_cast<int *>(lv + AT * PROSPER_MAX_HPRIME);  // AT*Hp point ids
    int *cnt = ln + AT * PROSPER_MAX_HPRIME;                         // H+1
    int *off = cnt + (H + 1);                                        // H+1
    int *fill = off + (H + 1);                                       // H

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int d0 = blockIdx.x * AD;
    const int64_t p_begin = (int64_t)blockIdx.y * pts_per_cta;
    const int64_t p_end = min(N, p_begin + pts_per_cta);
    for (int i = tid; i < H * AD; i += 256) Apart[i] = 0.f;

    for (int64_t c0 = p_begin; c0 < p_end; c0 += AT) {
        const int np = (int)min((int64_t)AT, p_end - c0);
        for (int h = tid; h < H; h += 256) { cnt[h] = 0; fill[h] = 0; }
        __syncthreads();
        for (int i = tid; i < np * Hp; i += 256) {
            int p = i / Hp, j = i - p * Hp;
            atomicAdd(&cnt[min(max(sel[(c0 + p) * SEL_STRIDE + j], 0), H - 1)], 1);
        }
        // Y slice of the chunk
        if ((D % 4) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
            for (int i = tid; i < AT * AD / 4; i += 256) {
                const int p = i / (AD / 4), c = (i - p * (AD / 4)) * 4;
                const int d = d0 + c;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (p < np && d < D) v = __ldg(reinterpret_cast<const float4 *>(Y + (c0 + p) * D + d));
                *reinterpret_cast<float4 *>(&Ys[p * AD + c]) = v;
            }
        } else {
            for (int i = tid; i < AT * AD; i += 256) {
                int p = i / AD, c = i - p * AD;
                int d = d0 + c;
                Ys[i] = (p < np && d < D) ? Y[(c0 + p) * D + d] : 0.f;
            }
        }
        __syncthreads();
        if (warp == 0) {   // exclusive scan of cnt -> off
            int carry = 0;
            for (int base = 0; base < H; base += 32) {
                int h = base + lane;
                int v = h < H ? cnt[h] : 0;
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += t;
                }
                if (h < H) off[h] = carry + x - v;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) off[H] = carry;
        }
        __syncthreads();
        for (int i = tid; i < np * Hp; i += 256) {
            int p = i / Hp, j = i - p * Hp;
            int h = min(max(sel[(c0 + p) * SEL_STRIDE + j], 0), H - 1);
            int pos = off[h] + atomicAdd(&fill[h], 1);
            ln[pos] = p;
            lv[pos] = es[(c0 + p) * SEL_STRIDE + j];
        }
        __syncthreads();
        for (int h = warp; h < H; h += 8) {
            // four independent accumulator pairs keep the shared-memory loads in flight
            float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, c0 = 0.f, c1 = 0.f, d0 = 0.f, d1 = 0.f;
            const int e1 = off[h + 1];
            int e = off[h];
            for (; e + 4 <= e1; e += 4) {
                const float v0 = lv[e], v1 = lv[e + 1], v2 = lv[e + 2], v3 = lv[e + 3];
                const float2 y0 = *reinterpret_cast<const float2 *>(&Ys[ln[e] * AD + 2 * lane]);
                const float2 y1 = *reinterpret_cast<const float2 *>(&Ys[ln[e + 1] * AD + 2 * lane]);
                const float2 y2 = *reinterpret_cast<const float2 *>(&Ys[ln[e + 2] * AD + 2 * lane]);
                const float2 y3 = *reinterpret_cast<const float2 *>(&Ys[ln[e + 3] * AD + 2 * lane]);
                a0 = fmaf(v0, y0.x, a0); a1 = fmaf(v0, y0.y, a1);
                b0 = fmaf(v1, y1.x, b0); b1 = fmaf(v1, y1.y, b1);
                c0 = fmaf(v2, y2.x, c0); c1 = fmaf(v2, y2.y, c1);
                d0 = fmaf(v3, y3.x, d0); d1 = fmaf(v3, y3.y, d1);
            }
            for (; e < e1; ++e) {
                const float v = lv[e];
                const float2 y = *reinterpret_cast<const float2 *>(&Ys[ln[e] * AD + 2 * lane]);
                a0 = fmaf(v, y.x, a0);
                a1 = fmaf(v, y.y, a1);
            }
            float2 *dst = reinterpret_cast<float2 *>(&Apart[h * AD + 2 * lane]);
            float2 cur = *dst;
            cur.x += (a0 + b0) + (c0 + d0);
            cur.y += (a1 + b1) + (c1 + d1);
            *dst = cur;
        }
        __syncthreads();
    }
    for (int i = tid; i < H * AD; i += 256) {
        int h = i / AD, c = i - h * AD;
        int d = d0 + c;
        if (d < D && Apart[i] != 0.f) atomicAdd(At + (size_t)h * D + d, (double)Apart[i]);
    }
}

__global__ void k_symmetrize(double *B, int H) {
    int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i < H && j < H && j < i) B[(size_t)i * H + j] = B[(size_t)j * H + i];
}

}  // namespace

// ================================================================ launchers
int launch_bsc_prep(prosper_ctx *c, const float *W, cudaStream_t s) {
    const int H = c->H, D = c->D;
    const size_t smem = sizeof(float) * 32 * (size_t)(D + 1);
    if (int rc = ensure_smem_attr((const void *)k_prep, smem)) return rc;
    TraceScope tr(c, "bsc_prep", s);
    dim3 gg((H + 15) / 16, (H + 15) / 16);
    k_prep<<<gg, 256, smem, s>>>(W, H, D, c->G, c->rnorm, c->Wd, c->Wb);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

int launch_bsc_proj_f32(prosper_ctx *c, const float *Y, int64_t N, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    const size_t smem = sizeof(ProjSmem);
    const bool wide = c->Hp > BSC_REG_MAX_HPRIME;
    const void *fn = wide ? (const void *)k_bsc_proj_f32<PROSPER_MAX_HPRIME>
                          : (const void *)k_bsc_proj_f32<BSC_REG_MAX_HPRIME>;
    if (int rc = ensure_smem_attr(fn, smem)) return rc;
    int64_t ntiles = (N + PT - 1) / PT;
    int grid = (int)std::min<int64_t>(ntiles, (int64_t)c->num_sms);
    TraceScope tr(c, "bsc_proj_f32", s);
    if (wide)
        k_bsc_proj_f32<PROSPER_MAX_HPRIME><<<grid, 32 * (PNP + PNR), smem, s>>>(
            Y, c->Wd, c->rnorm, N, c->D, c->H, c->Hp, c->score_mode, c->sel, c->selp,
            reinterpret_cast<float2 *>(c->yy), c->d_status);
    else
        k_bsc_proj_f32<BSC_REG_MAX_HPRIME><<<grid, 32 * (PNP + PNR), smem, s>>>(
            Y, c->Wd, c->rnorm, N, c->D, c->H, c->Hp, c->score_mode, c->sel, c->selp,
            reinterpret_cast<float2 *>(c->yy), c->d_status);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

template <int HP>
static int states_dispatch(StateArgs &A, bool encode, int64_t N, cudaStream_t s) {
    int grid = (int)((N + 127) / 128);
    TraceScope tr(A.trace_ctx, encode ? "bsc_states_encode" : "bsc_states", s);
    if (encode) k_bsc_states<HP, true><<<grid, 128, 0, s>>>(A);
    else k_bsc_states<HP, false><<<grid, 128, 0, s>>>(A);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

int launch_bsc_states(prosper_ctx *c, const double *theta, int64_t N, int64_t n_offset,
                      prosper_stats *st, int16_t *sel_out, float *smean_out, int16_t *map_out,
                      float *mapp_out, float *logz_out, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    StateArgs A;
    A.sel = c->sel; A.selp = c->selp; A.yy = reinterpret_cast<const float2 *>(c->yy); A.G = c->G;
    A.N = N; A.H = c->H; A.D = c->D; A.gamma = c->gamma; A.theta = theta;
    A.es = c->es;
    A.B = st ? st->B : nullptr;
    A.scal = st ? st->scal : nullptr;
    A.sel_out = sel_out; A.map_out = map_out; A.smean_out = smean_out; A.mapp_out = mapp_out;
    A.logz_out = logz_out; A.n_offset = n_offset; A.trace_ctx = c;
    A.cut_thr = (st && c->cut) ? c->cut_thr : nullptr;
    A.cut_logz = A.cut_thr ? c->cut_logz + c->cut_n0 : nullptr;
    const bool enc = (st == nullptr);
    switch (c->Hp) {
        case 1: return states_dispatch<1>(A, enc, N, s);
        case 2: return states_dispatch<2>(A, enc, N, s);
        case 3: return states_dispatch<3>(A, enc, N, s);
        case 4: return states_dispatch<4>(A, enc, N, s);
        case 5: return states_dispatch<5>(A, enc, N, s);
        case 6: return states_dispatch<6>(A, enc, N, s);
        case 7: return states_dispatch<7>(A, enc, N, s);
        case 8: return states_dispatch<8>(A, enc, N, s);
        case 9: return states_dispatch<9>(A, enc, N, s);
        case 10: return states_dispatch<10>(A, enc, N, s);
        default: set_error("BSC: unsupported Hprime %d", c->Hp); return PROSPER_EINVAL;
    }
}

int launch_astat(prosper_ctx *c, const float *Y, int64_t N, double *At, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    if (astat_tc_ok(c->D, c->H) && c->apart && !c->astat_simt &&
        (reinterpret_cast<uintptr_t>(Y) & 15) == 0)   // bulk copies need 16-byte aligned rows
        return launch_astat_tc(c, Y, N, s);
    const int H = c->H, D = c->D;
    const size_t smem = sizeof(float) * ((size_t)H * AD + AT * AD + AT * PROSPER_MAX_HPRIME) +
                        sizeof(int) * (AT * PROSPER_MAX_HPRIME + 3 * (H + 1));
    if (int rc = ensure_smem_attr((const void *)k_astat, smem)) return rc;
    const int slices = (D + AD - 1) / AD;
    int ranges = std::max(1, 2 * c->num_sms / slices);
    int64_t per = (N + ranges - 1) / ranges;
    per = ((per + AT - 1) / AT) * AT;
    ranges = (int)((N + per - 1) / per);
    dim3 grid(slices, ranges);
    TraceScope tr(c, "astat", s);
    k_astat<<<grid, 256, smem, s>>>(Y, c->sel, c->es, N, D, H, c->Hp, per, At);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

int launch_symmetrize(prosper_ctx *c, double *B, cudaStream_t s) {
    const int H = c->H;
    dim3 b(16, 16), g((H + 15) / 16, (H + 15) / 16);
    TraceScope tr(c, "symmetrize", s);
    k_symmetrize<<<g, b, 0, s>>>(B, H);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

}  // namespace prosper
