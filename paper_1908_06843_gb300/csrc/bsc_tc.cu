// bsc_tc.cu -- BSC preselection with the projection W^T y on the tcgen05 tensor
// cores in BF16 (FP32 accumulation in tensor memory), then the H' selected
// projections recomputed in FP32 ("rescore").
//
// Method (paper Sec. 2-3: truncated posteriors with H' candidates per point):
// the preselection score of latent h is W_h^T y / ||W_h||.  Here the N x H
// score matrix is produced 128 points at a time by one tcgen05.mma chain
// (M = 128 points, N = H latents, K = D pixels) whose A operand is the Y tile
// converted to BF16 in shared memory and whose B operand is the BF16 copy of W
// resident in shared memory for the whole persistent CTA.  The accumulator
// tile (128 lanes x H columns, FP32) is read back with tcgen05.ld, staged in
// shared memory 64 points at a time, and every warp takes the top-H' of its
// points.  The ranking key is the score rounded down to 15 mantissa bits with
// 255 - h in the low byte (ties, including the ones the rounding makes, go to
// the lower h); the rounding is far below the BF16 error of the score itself.
// Each lane sorts its 8 keys, then H' rounds of a warp maximum pop the winners.
// The H' selected projections are then recomputed in FP32 from the FP32 Y and
// W, so BF16 only decides which latents are candidates.
//
// Shared memory (1024-byte aligned, K-major, 128-byte swizzle, 8-row core groups):
//   W  : D/64 K-blocks, each H rows x 128 B    (H*D*2 bytes, resident)
//   Y  : D/64 K-blocks, each 128 rows x 128 B  (128*D*2 bytes), reused after the
//        MMA as the FP32 projection stage P (64 rows x H floats, 16-byte chunks
//        XOR-swizzled by row so row-wise stores and column reads are conflict-free)
#include "internal.cuh"
#include "topk.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace prosper {
namespace {
using namespace tc;

constexpr int TM = 128;                       // points per tile (MMA M)
constexpr int NW = 16;                        // warps per CTA
constexpr unsigned long long kWaitNs = 2000000000ull;   // bounded mbarrier wait: 2 s

// index of float (row, col) in the swizzled projection stage (rows of H floats)
__device__ __forceinline__ int pidx(int row, int col, int H) {
    return row * H + ((((col >> 2) ^ (row & 7))) << 2) + (col & 3);
}

// byte offset of the 16-byte chunk c (8 BF16 values, d = 8c .. 8c+7) of row r in a
// K-major 128-byte-swizzled operand with `rows` rows per 64-wide K-block
__device__ __forceinline__ uint32_t opnd_off(int r, int c, int rows) {
    const int kb = c >> 3, ch = c & 7;
    return (uint32_t)(kb * rows * 128 + r * 128 + ((ch ^ (r & 7)) << 4));
}

__global__ void __launch_bounds__(NW * 32, 1)
k_bsc_proj_bf16(const float *__restrict__ Y, const float *__restrict__ Wt,
                const uint16_t *__restrict__ Wimg, const float *__restrict__ rnorm, int64_t N,
                int D, int H, int Hp, uint32_t tmem_cols, int32_t *__restrict__ sel_out,
                float *__restrict__ selp_out, float2 *__restrict__ yy_out,
                unsigned *__restrict__ status, unsigned long long wait_ns, int test_no_commit) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *sbase = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const size_t wbytes = (size_t)H * D * 2;
    unsigned char *Wsm = sbase;
    unsigned char *Ysm = sbase + ((wbytes + 1023) & ~(size_t)1023);
    float *Psm = reinterpret_cast<float *>(Ysm);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nchunk = D / 8;                 // 16-byte chunks per row
    const int nkb = D / 64;
    const int64_t ntiles = (N + TM - 1) / TM;
    const uint32_t idesc = idesc_bf16(TM, H);
    const uint32_t bar = smem_u32(&mbar);

    // resident BF16 dictionary (already in the operand image layout)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(Wimg);
        uint4 *dst = reinterpret_cast<uint4 *>(Wsm);
        for (size_t i = tid; i < wbytes / 16; i += NW * 32) dst[i] = __ldg(src + i);
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // per-lane key constants for h = lane + 32 j: the mask keeps the top 24 bits
    // of the score key, the low byte holds 255 - h; both 0 for an absent latent
    unsigned kmask[8], klow[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int h = lane + 32 * j;
        kmask[j] = h < H ? 0xFFFFFF00u : 0u;
        klow[j] = h < H ? (unsigned)(255 - h) : 0u;
    }

    uint32_t phase = 0;
    bool aborted = false;
    for (int64_t tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x) {
        const int64_t n0 = tile * TM;
        // ---- Y tile -> BF16 operand; exact y^T y on the way.  Warp w owns the
        //      rows w + NW i (i < 8); all eight rows' loads are issued first.
        float sq[TM / NW];
#pragma unroll
        for (int i = 0; i < TM / NW; ++i) sq[i] = 0.f;
        for (int cb = 0; cb < nchunk; cb += 32) {
            const int c = cb + lane;
            float4 v0[TM / NW], v1[TM / NW];
#pragma unroll
            for (int i = 0; i < TM / NW; ++i) {
                const int64_t n = n0 + warp + NW * i;
                v0[i] = v1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (c < nchunk && n < N) {
                    const float4 *row = reinterpret_cast<const float4 *>(Y + n * D + 8 * c);
                    v0[i] = __ldg(row);
                    v1[i] = __ldg(row + 1);
                }
            }
#pragma unroll
            for (int i = 0; i < TM / NW; ++i) {
                float q = sq[i];
                q = fmaf(v0[i].x, v0[i].x, q); q = fmaf(v0[i].y, v0[i].y, q);
                q = fmaf(v0[i].z, v0[i].z, q); q = fmaf(v0[i].w, v0[i].w, q);
                q = fmaf(v1[i].x, v1[i].x, q); q = fmaf(v1[i].y, v1[i].y, q);
                q = fmaf(v1[i].z, v1[i].z, q); q = fmaf(v1[i].w, v1[i].w, q);
                sq[i] = q;
                if (c < nchunk) {
                    __nv_bfloat162 b0 = __floats2bfloat162_rn(v0[i].x, v0[i].y);
                    __nv_bfloat162 b1 = __floats2bfloat162_rn(v0[i].z, v0[i].w);
                    __nv_bfloat162 b2 = __floats2bfloat162_rn(v1[i].x, v1[i].y);
                    __nv_bfloat162 b3 = __floats2bfloat162_rn(v1[i].z, v1[i].w);
                    uint4 pk;
                    pk.x = *reinterpret_cast<uint32_t *>(&b0);
                    pk.y = *reinterpret_cast<uint32_t *>(&b1);
                    pk.z = *reinterpret_cast<uint32_t *>(&b2);
                    pk.w = *reinterpret_cast<uint32_t *>(&b3);
                    *reinterpret_cast<uint4 *>(Ysm + opnd_off(warp + NW * i, c, TM)) = pk;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < TM / NW; ++i) {
            float q = sq[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
            const int64_t n = n0 + warp + NW * i;
            if (lane == 0 && n < N) {
                yy_out[n] = make_float2(q, 0.f);
                if (!isfinite(q)) atomicOr(status, ST_NONFINITE);
            }
        }
        fence_proxy_async();
        __syncthreads();
        // ---- projection tile on the tensor cores
        if (tid == 0 && !test_no_commit) {
            tc_fence_after();
            const uint32_t ya = smem_u32(Ysm), wa = smem_u32(Wsm);
            for (int kb = 0; kb < nkb; ++kb)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t a = desc_sw128(ya + kb * TM * 128 + ks * 32);
                    const uint64_t b = desc_sw128(wa + kb * H * 128 + ks * 32);
                    umma_bf16(tmem, a, b, idesc, (kb | ks) != 0);
                }
            umma_commit(bar);
        }
        const bool ok = mbar_wait(bar, phase, wait_ns);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
            aborted = true;
            // give every point this CTA still owned a valid (if meaningless)
            // candidate list so that later kernels stay in bounds
            for (int64_t t2 = tile; t2 < ntiles; t2 += gridDim.x)
                for (int i = tid; i < TM * SEL_STRIDE; i += NW * 32) {
                    const int64_t nn = t2 * TM + i / SEL_STRIDE;
                    if (nn >= N) continue;
                    const int j = i % SEL_STRIDE;
                    sel_out[nn * SEL_STRIDE + j] = j < H ? j : 0;
                    selp_out[nn * SEL_STRIDE + j] = 0.f;
                    if (j == 0) yy_out[nn] = make_float2(0.f, 0.f);
                }
            break;
        }
        tc_fence_after();

        // ---- two halves of 64 points: TMEM -> shared P -> selection + FP32 rescore
        for (int half = 0; half < 2; ++half) {
            const int q = warp & 3;                 // TMEM lane quadrant of this warp
            if ((q >> 1) == half) {
                const int prow = (q & 1) * 32 + lane;   // row within the half
                const int part = warp >> 2;             // 4 warps share a quadrant: H/4 columns each
                const int cbeg = part * (H / 4);
                const int cend = cbeg + H / 4;
                for (int c0 = cbeg; c0 < cend; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                    for (int k = 0; k < 16; k += 4)
                        *reinterpret_cast<float4 *>(&Psm[pidx(prow, c0 + k, H)]) =
                            make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                }
            }
            tc_fence_before();
            __syncthreads();
            // packed keys: score key rounded down to 24 bits, then 255 - h, so that
            // one 32-bit maximum ranks by score and breaks ties to the lower h
            // (H <= 256); 0 marks an absent latent
            auto make_keys = [&](int p, unsigned (&pk)[8]) {
                const float *prow_p = Psm + pidx(p, lane, H);   // + 32 j for h = lane + 32 j
#pragma unroll
                for (int j = 0; j < 8; ++j) pk[j] = packed_key(kmask[j] ? prow_p[32 * j] : 0.f, kmask[j], klow[j]);
                sort8_desc(pk);
            };
            auto rescore = [&](int64_t n, int myh) {
                    // FP32 rescore: partial dot products over this lane's d, then a
                    // transposed warp reduction (16 slots -> one total per lane pair)
                    float v[16];
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = 0.f;
                    const float *yrow = Y + n * D;
                    int hsel[PROSPER_MAX_HPRIME];
#pragma unroll
                    for (int r = 0; r < PROSPER_MAX_HPRIME; ++r)
                        hsel[r] = __shfl_sync(0xffffffffu, myh, r < Hp ? r : 0);
                    for (int c = lane; c < nchunk; c += 32) {
                        const float4 y0 = __ldg(reinterpret_cast<const float4 *>(yrow + 8 * c));
                        const float4 y1 = __ldg(reinterpret_cast<const float4 *>(yrow + 8 * c + 4));
                        // rows in batches of 8: all of a batch's row loads first
                        // (always in bounds), then its dot products
#pragma unroll
                        for (int rb = 0; rb < PROSPER_MAX_HPRIME; rb += 8) {
                            if (rb >= Hp) break;   // warp-uniform
                            float4 w[16];
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                const float *wrow = Wt + (size_t)hsel[rb + r] * D + 8 * c;
                                w[2 * r] = __ldg(reinterpret_cast<const float4 *>(wrow));
                                w[2 * r + 1] = __ldg(reinterpret_cast<const float4 *>(wrow + 4));
                            }
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                const float4 w0 = w[2 * r], w1 = w[2 * r + 1];
                                float s = v[rb + r];
                                s = fmaf(y0.x, w0.x, s); s = fmaf(y0.y, w0.y, s);
                                s = fmaf(y0.z, w0.z, s); s = fmaf(y0.w, w0.w, s);
                                s = fmaf(y1.x, w1.x, s); s = fmaf(y1.y, w1.y, s);
                                s = fmaf(y1.z, w1.z, s); s = fmaf(y1.w, w1.w, s);
                                v[rb + r] = (rb + r < Hp) ? s : 0.f;
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const bool up = (lane & 16) != 0;
                        const float send = up ? v[k] : v[k + 8];
                        const float keep = up ? v[k + 8] : v[k];
                        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool up = (lane & 8) != 0;
                        const float send = up ? v[k] : v[k + 4];
                        const float keep = up ? v[k + 4] : v[k];
                        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const bool up = (lane & 4) != 0;
                        const float send = up ? v[k] : v[k + 2];
                        const float keep = up ? v[k + 2] : v[k];
                        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                    }
                    {
                        const bool up = (lane & 2) != 0;
                        const float send = up ? v[0] : v[1];
                        const float keep = up ? v[1] : v[0];
                        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                    }
                    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
                    // this lane now holds the total of round index jr
                    const int jr = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                                   ((lane >> 1) & 1);
                    int rank = 0;
#pragma unroll
                    for (int r = 0; r < PROSPER_MAX_HPRIME; ++r) {
                        const int o = __shfl_sync(0xffffffffu, myh, r);
                        rank += (r < Hp && o < myh) ? 1 : 0;
                    }
                    const int h_jr = __shfl_sync(0xffffffffu, myh, jr & 31);
                    const int rank_jr = __shfl_sync(0xffffffffu, rank, jr & 31);
                    if ((lane & 1) == 0 && jr < Hp) {
                        sel_out[n * SEL_STRIDE + rank_jr] = h_jr;
                        selp_out[n * SEL_STRIDE + rank_jr] = v[0];
                    }
                };
            // two points at a time, so that the two selections' latency chains
            // (warp maxima) interleave; then one rescore each
            for (int i = 0; i < 64 / NW; i += 2) {
                const int pa = warp * (64 / NW) + i, pb = pa + 1;
                const int64_t na = n0 + 64 * half + pa, nb = na + 1;
                if (na >= N) break;
                unsigned ka[8], kb[8];
                make_keys(pa, ka);
                make_keys(pb, kb);
                // Hp rounds of the warp maximum; the winning lane pops its head
                int ha = 0, hb = 0;
#pragma unroll
                for (int r = 0; r < PROSPER_MAX_HPRIME; ++r) {
                    if (r < Hp) {
                        const unsigned wa = __reduce_max_sync(0xffffffffu, ka[0]);
                        const unsigned wb = __reduce_max_sync(0xffffffffu, kb[0]);
                        if (lane == r) {
                            ha = 255 - (int)(wa & 0xFFu);
                            hb = 255 - (int)(wb & 0xFFu);
                        }
                        if (ka[0] == wa) {
#pragma unroll
                            for (int j = 0; j < 7; ++j) ka[j] = ka[j + 1];
                            ka[7] = 0u;
                        }
                        if (kb[0] == wb) {
#pragma unroll
                            for (int j = 0; j < 7; ++j) kb[j] = kb[j + 1];
                            kb[7] = 0u;
                        }
                    }
                }
                rescore(na, ha);
                if (nb < N) rescore(nb, hb);
            }
            __syncthreads();
        }
    }
    if (aborted && tid == 0) {
        // give the MMA chain that timed out one more bounded chance to finish
        // before its tensor memory is released
        mbar_wait(bar, phase ^ 1u, wait_ns / 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
    }
}

// BF16 image of the unit-norm rows W_h / ||W_h|| (zero rows stay zero), so that
// the tensor cores produce the preselection scores directly, in the operand
// layout above: K-block kb holds rows h of 128 B
// (d = 64 kb .. 64 kb + 63), 16-byte chunk c stored at chunk position c ^ (h & 7).
__global__ void k_w_image(const float *__restrict__ Wt, const float *__restrict__ rnorm, int H, int D,
                          uint16_t *__restrict__ img) {
    const int64_t total = (int64_t)H * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int h = (int)(i / D), d = (int)(i % D);
        const int kb = d >> 6, ch = (d & 63) >> 3, w = d & 7;
        const size_t off = (size_t)kb * H * 64 + (size_t)h * 64 + (size_t)((ch ^ (h & 7)) * 8 + w);
        const __nv_bfloat16 b = __float2bfloat16_rn(Wt[i] * rnorm[h]);
        img[off] = *reinterpret_cast<const uint16_t *>(&b);
    }
}

}  // namespace

size_t bf16_smem_bytes(int D, int H) {
    const size_t w = ((size_t)H * D * 2 + 1023) & ~(size_t)1023;
    const size_t y = std::max((size_t)TM * D * 2, (size_t)64 * H * 4);
    return 1024 + w + y;
}

int launch_bsc_bf16_prep(prosper_ctx *c, const float *W, cudaStream_t s) {
    TraceScope tr(c, "bsc_w_image", s);
    k_w_image<<<c->num_sms * 2, 256, 0, s>>>(W, c->rnorm, c->H, c->D, c->Wb);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

int launch_bsc_proj_bf16(prosper_ctx *c, const float *Y, const float *W, int64_t N, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    if ((reinterpret_cast<uintptr_t>(Y) & 15) || (reinterpret_cast<uintptr_t>(W) & 15)) {
        set_error("BF16 path needs 16-byte aligned Y and W");
        return PROSPER_EINVAL;
    }
    const size_t smem = bf16_smem_bytes(c->D, c->H);
    if (int rc = ensure_smem_attr((const void *)k_bsc_proj_bf16, smem)) return rc;
    uint32_t cols = 32;
    while ((int)cols < c->H) cols <<= 1;
    const int64_t ntiles = (N + TM - 1) / TM;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)c->num_sms);
    TraceScope tr(c, "bsc_proj_bf16", s);
    // fault-injection hook for the failure-detection test: the MMA chain is not
    // issued, so the bounded wait runs out and the kernel reports a timeout
    const unsigned long long wait_ns = c->tc_test_no_commit_ms > 0
                                           ? (unsigned long long)c->tc_test_no_commit_ms * 1000000ull
                                           : kWaitNs;
    k_bsc_proj_bf16<<<grid, NW * 32, smem, s>>>(Y, W, c->Wb, c->rnorm, N, c->D, c->H, c->Hp, cols,
                                            c->sel, c->selp, reinterpret_cast<float2 *>(c->yy),
                                            c->d_status, wait_ns, c->tc_test_no_commit_ms > 0);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

}  // namespace prosper
