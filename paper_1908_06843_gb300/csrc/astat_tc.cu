// astat_tc.cu -- the BSC/GSC sufficient statistic A = sum_n y_n <s>_n^T
// (Sec. 2, the E-step's contribution to the M-step W = A B^{-1}) on the
// tcgen05 tensor cores.
//
// For a tile of 64 points, A^T gains E^T Y, where E (64 x H) holds each point's
// posterior means <s_h> at its H' candidates (zero elsewhere) and Y (64 x D)
// the tile's data.  One MMA chain per tile accumulates into tensor memory:
// M = 128 latents per half (one or two halves), N = D pixels, K = 64 points,
// so the whole H x D accumulator (FP32, up to 512 TMEM columns) stays on chip
// for every tile the persistent CTA processes and is added to the FP64 result
// once per CTA.  The operands are BF16 with a hi/lo split of both factors,
// x = x_hi + x_lo with x_hi = bf16(x), x_lo = bf16(x - x_hi), and three products
// (hi*hi + hi*lo + lo*hi) per tile; the dropped lo*lo term and the residuals
// are below 2^-16 of each product, far below the FP32 accumulation's own
// rounding over the data set.  Both operands are built K-major (points
// contiguous) in shared memory with the 128-byte swizzle, so the same
// descriptor form as the projection kernel applies.
#include "internal.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace prosper {
namespace {
using namespace tc;

constexpr int AT_T = 64;      // points per tile (one 128-byte K atom of BF16)
constexpr int AT_CW = 8;      // converter warps (+ one control warp)
constexpr int AT_NT = 32 * (AT_CW + 1);
constexpr unsigned long long kAtWaitNs = 2000000000ull;

// byte offset of element (row r, point k) in a K-major 64-wide swizzled operand
__device__ __forceinline__ uint32_t kmaj_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + ((k & 7) << 1));
}

// the same split for two values at once: packed BF16 pairs (x0 in the low half)
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t &hi2, uint32_t &lo2) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    hi2 = *reinterpret_cast<const uint32_t *>(&h);
    const float r0 = x0 - __uint_as_float(hi2 << 16);
    const float r1 = x1 - __uint_as_float(hi2 & 0xFFFF0000u);
    const __nv_bfloat162 l = __floats2bfloat162_rn(r0, r1);
    lo2 = *reinterpret_cast<const uint32_t *>(&l);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__global__ void __launch_bounds__(AT_NT, 1)
k_astat_tc(const float *__restrict__ Y, const int32_t *__restrict__ sel, const float *__restrict__ es,
           int64_t N, int D, int H, int Hp, int halves, uint32_t tmem_cols, float *__restrict__ part,
           int accumulate, unsigned *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t lbar[2], cbar[2];   // data of half q arrived / MMAs of half q done
    __shared__ uint32_t tmem_slot;
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *sb = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const int Hpad = halves * 128;
    const int SP = D * 4;                               // staging row pitch (bytes)
    unsigned char *Ehi = sb;                            // Hpad rows x 128 B
    unsigned char *Elo = Ehi + Hpad * 128;
    unsigned char *Yhi = Elo + Hpad * 128;              // D rows x 128 B
    unsigned char *Ylo = Yhi + D * 128;
    unsigned char *Stg = Ylo + D * 128;                 // AT_T rows x SP bytes (FP32 Y)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool conv = warp < AT_CW;                     // converter warps; warp AT_CW controls
    const int64_t ntiles = (N + AT_T - 1) / AT_T;
    const uint32_t idesc = idesc_bf16(128, D);

    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&lbar[q]), 1);
            mbar_init(smem_u32(&cbar[q]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // E starts zeroed once; afterwards every entry is cleared by the thread
    // that wrote it
    {
        uint4 *z = reinterpret_cast<uint4 *>(Ehi);
        const int nz = 2 * Hpad * 128 / 16;
        for (int i = tid; i < nz; i += AT_NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // control warp: rows [32 q, 32 q + 32) of tile t into the staging rows
    // (contiguous in Y and in shared memory: one bulk copy)
    auto load_half = [&](int64_t t, int q) {
        if (lane == 0) {
            const int64_t r0 = t * AT_T + 32 * q;
            const int64_t left = N - r0;
            const int rows = (int)(left < 0 ? 0 : (left > 32 ? 32 : left));
            const uint32_t lb = smem_u32(&lbar[q]);
            mbar_arrive_expect_tx(lb, (uint32_t)(rows * D * 4));
            if (rows > 0) bulk_g2s(smem_u32(Stg + (size_t)(32 * q) * SP), Y + r0 * D, (uint32_t)(rows * D * 4), lb);
        }
        __syncwarp();
    };

    // converter item (one per thread and half): 4 consecutive d x 8 points.
    // Within each 8-lane store wavefront the 8 lanes take 8 consecutive d4 and
    // chunks c rotated so that both the staging reads (dense rows of D floats,
    // D a multiple of 32) and the swizzled operand writes touch 8 different
    // 16-byte bank groups.
    const int G = D / 32;
    int it_d4 = 0, it_c = 0;
    {
        const int wf = tid >> 3, l8 = tid & 7;
        const int g = wf % G, rot = wf / G;             // rot in 0..3 for tid < D
        it_d4 = 4 * (8 * g + l8);
        it_c = ((l8 >> 1) + rot) & 3;                   // + 4 q
    }
    const bool has_item = conv && tid < D;

    // E entries: point 32 q + (tid & 31), candidate slots j = tid/32 and tid/32 + 8
    constexpr int EPT = (PROSPER_MAX_HPRIME + 7) / 8;
    int prev_h[2][EPT];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int i = 0; i < EPT; ++i) prev_h[q][i] = -1;
    int sh[EPT];
    float sv[EPT];
    auto fetch_e = [&](int64_t t, int q) {
        const int64_t n = t * AT_T + 32 * q + lane;
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            const int j = warp + 8 * i;
            const bool ok = conv && t < ntiles && n < N && j < Hp;
            sh[i] = ok ? min(max(__ldg(sel + n * SEL_STRIDE + j), 0), H - 1) : -1;
            sv[i] = ok ? __ldg(es + n * SEL_STRIDE + j) : 0.f;
        }
    };

    bool aborted = false;
    int done_tiles = 0;
    int64_t tile = blockIdx.x;
    if (warp == AT_CW && tile < ntiles) {
        load_half(tile, 0);
        load_half(tile, 1);
    }
    fetch_e(tile, 0);
    for (int it = 0; tile < ntiles && !aborted; ++it, tile += gridDim.x) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            bool ok = true;
            if (conv) {
                ok = mbar_wait(smem_u32(&lbar[q]), (uint32_t)(it & 1), kAtWaitNs);
                if (ok && it > 0) ok = mbar_wait(smem_u32(&cbar[q]), (uint32_t)((it - 1) & 1), kAtWaitNs);
                tc_fence_after();
                // E columns of this half: clear the previous tile's entries, then
                // write the new ones.  The converter warps meet in between (a
                // latent may move between candidate slots of a point), and the
                // meeting also makes the wait outcome uniform among them.
                const int p = 32 * q + lane;
                if (ok) {
#pragma unroll
                    for (int i = 0; i < EPT; ++i)
                        if (prev_h[q][i] >= 0) {
                            const uint32_t off = kmaj_off(prev_h[q][i], p);
                            *reinterpret_cast<uint16_t *>(Ehi + off) = 0;
                            *reinterpret_cast<uint16_t *>(Elo + off) = 0;
                            prev_h[q][i] = -1;
                        }
                }
                {
                    unsigned anyfail;
                    asm volatile("{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
                                 " bar.red.or.pred po, 1, %2, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
                                 : "=r"(anyfail) : "r"((unsigned)!ok), "r"(AT_CW * 32) : "memory");
                    ok = !anyfail;
                }
                if (ok) {
#pragma unroll
                    for (int i = 0; i < EPT; ++i) {
                        const int h = sh[i];
                        if (h < 0) continue;
                        __nv_bfloat16 hi, lo;
                        split_bf16(sv[i], hi, lo);
                        const uint32_t off = kmaj_off(h, p);
                        *reinterpret_cast<__nv_bfloat16 *>(Ehi + off) = hi;
                        *reinterpret_cast<__nv_bfloat16 *>(Elo + off) = lo;
                        prev_h[q][i] = h;
                    }
                    // Y of this half: FP32 staging -> BF16 hi / lo, transposed
                    if (has_item) {
                        const int c = 4 * q + it_c;
                        const int64_t n0 = tile * AT_T + 8 * c;
                        float4 v[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            v[i] = (n0 + i < N) ? *reinterpret_cast<const float4 *>(Stg + (size_t)(8 * c + i) * SP + it_d4 * 4)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            uint32_t ph[4], pl[4];
#pragma unroll
                            for (int i = 0; i < 8; i += 2) {
                                const float x0 = e == 0 ? v[i].x : e == 1 ? v[i].y : e == 2 ? v[i].z : v[i].w;
                                const float x1 = e == 0 ? v[i + 1].x : e == 1 ? v[i + 1].y : e == 2 ? v[i + 1].z : v[i + 1].w;
                                split_bf16x2(x0, x1, ph[i >> 1], pl[i >> 1]);
                            }
                            const int d = it_d4 + e;
                            const uint32_t off = (uint32_t)(d * 128 + ((c ^ (d & 7)) << 4));
                            *reinterpret_cast<uint4 *>(Yhi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                            *reinterpret_cast<uint4 *>(Ylo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
                        }
                    }
                }
                // candidate lists of the next half travel while the rest proceeds
                if (q == 0) fetch_e(tile, 1);
                else fetch_e(tile + gridDim.x, 0);
            }
            fence_proxy_async();
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
                aborted = true;
                break;
            }
            if (warp == AT_CW) {
                // the staging rows of this half are free again: next tile's rows
                if (tile + gridDim.x < ntiles) load_half(tile + gridDim.x, q);
                if (lane == 0) {
                    tc_fence_after();
                    const uint32_t eh = smem_u32(Ehi), el = smem_u32(Elo), yh = smem_u32(Yhi), yl = smem_u32(Ylo);
                    for (int hf = 0; hf < halves; ++hf) {
                        const uint32_t d_tm = tmem + (uint32_t)(hf * D);
#pragma unroll
                        for (int k2 = 0; k2 < 2; ++k2) {
                            const int ks = 2 * q + k2;
                            const uint32_t ao = (uint32_t)(hf * 128 * 128 + ks * 32), bo = (uint32_t)(ks * 32);
                            umma_bf16(d_tm, desc_sw128(eh + ao), desc_sw128(yh + bo), idesc,
                                      (it > 0 || ks > 0) ? 1u : 0u);
                            umma_bf16(d_tm, desc_sw128(eh + ao), desc_sw128(yl + bo), idesc, 1u);
                            umma_bf16(d_tm, desc_sw128(el + ao), desc_sw128(yh + bo), idesc, 1u);
                        }
                    }
                    umma_commit(smem_u32(&cbar[q]));
                }
                __syncwarp();
            }
        }
        if (!aborted) ++done_tiles;
    }
    // the last chain (half 1 of the last tile) covers every MMA of this CTA
    bool ok_end = true;
    if (done_tiles > 0)
        ok_end = mbar_wait(smem_u32(&cbar[1]), (uint32_t)((done_tiles - 1) & 1), kAtWaitNs);
    tc_fence_after();
    if (__syncthreads_or(!ok_end)) {
        if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
        aborted = true;
    }
    // ---- epilogue: this CTA's FP32 partial of A^T to global memory (stored by
    //      the first launch of an E-step, added to by the later ones; the
    //      partials are summed once per E-step by k_reduce_parts)
    if (!aborted && conv && (!accumulate || done_tiles > 0)) {
        const int qd = warp & 3;
        const int h_in = qd * 32 + lane;
        const int cb = (warp < 4) ? 0 : D / 2, ce = (warp < 4) ? D / 2 : D;
        float *mine = part + (size_t)blockIdx.x * H * D;
        for (int hf = 0; hf < halves; ++hf) {
            const int h = hf * 128 + h_in;
            for (int c0 = cb; c0 < ce; c0 += 16) {
                float v[16];
                if (done_tiles > 0) {
                    tmem_ld16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(hf * D + c0), v);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = 0.f;
                }
                if (h < H) {
                    float4 *dst = reinterpret_cast<float4 *>(mine + (size_t)h * D + c0);
#pragma unroll
                    for (int k = 0; k < 16; k += 4) {
                        float4 o = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                        if (accumulate) {
                            const float4 a = dst[k / 4];
                            o.x += a.x; o.y += a.y; o.z += a.z; o.w += a.w;
                        }
                        dst[k / 4] = o;
                    }
                }
            }
        }
    }
    if (aborted && tid == 0) {
        // let copies and MMA chains still in flight finish (bounded) before
        // the shared and tensor memory are released
        for (int q = 0; q < 2; ++q) {
            mbar_wait(smem_u32(&lbar[q]), 0u, kAtWaitNs / 8);
            mbar_wait(smem_u32(&lbar[q]), 1u, kAtWaitNs / 8);
            mbar_wait(smem_u32(&cbar[q]), 0u, kAtWaitNs / 8);
            mbar_wait(smem_u32(&cbar[q]), 1u, kAtWaitNs / 8);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
    }
}

// FP32 -> FP64 from the IEEE-754 fields on the integer pipe (exact for normal
// floats, subnormals to 0): the FP64 pipe of this part is too slow for one
// conversion per element.
__device__ __forceinline__ double widen(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned m = (e == 0u) ? 0u : (u & 0x7FFFFFu);
    const unsigned e64 = (e == 0u) ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u);
    return __hiloint2double((int)((u & 0x80000000u) | (e64 << 20) | (m >> 3)), (int)(m << 29));
}

// At += sum over the per-CTA partials in CTA order.  The sum is carried as an
// unevaluated FP32 pair hi + lo (Knuth's TwoSum per addition, error about
// 2^-44 relative) on the FP32 pipe and widened to FP64 once at the end.
// Fixed-order sum of the per-CTA partials.  A 256-thread block owns 32 float4
// groups of elements; its thread (g, q) adds partials q, q + 8, q + 16, ... of
// group g with TwoSum (every load of a thread is independent, so ~19 are in
// flight), and thread q = 0 then adds the eight (hi, lo) slices in order q =
// 0..7: the result does not depend on timing.
constexpr int RP_SL = 8;     // partial slices per element group
__global__ void __launch_bounds__(256) k_reduce_parts(const float *__restrict__ part, int nparts,
                                                      int64_t HD, double *__restrict__ At) {
    __shared__ float4 shi[RP_SL][32], slo[RP_SL][32];
    const int g = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int64_t i4 = ((int64_t)blockIdx.x * 32 + g) * 4;     // first element of the group
    float4 hi = make_float4(0.f, 0.f, 0.f, 0.f), lo = hi;
    auto add = [](float &h, float &l, float b) {
        const float s = h + b;
        const float bb = s - h;
        l += (h - (s - bb)) + (b - bb);
        h = s;
    };
    if (i4 < HD) {
#pragma unroll 4
        for (int p = q; p < nparts; p += RP_SL) {
            const float4 b = __ldg(reinterpret_cast<const float4 *>(part + (size_t)p * HD + i4));
            add(hi.x, lo.x, b.x); add(hi.y, lo.y, b.y); add(hi.z, lo.z, b.z); add(hi.w, lo.w, b.w);
        }
    }
    shi[q][g] = hi;
    slo[q][g] = lo;
    __syncthreads();
    if (q == 0 && i4 < HD) {
        float4 H4 = shi[0][g], L4 = slo[0][g];
        for (int k = 1; k < RP_SL; ++k) {
            const float4 h2 = shi[k][g], l2 = slo[k][g];
            add(H4.x, L4.x, h2.x); add(H4.y, L4.y, h2.y); add(H4.z, L4.z, h2.z); add(H4.w, L4.w, h2.w);
            L4.x += l2.x; L4.y += l2.y; L4.z += l2.z; L4.w += l2.w;
        }
        At[i4] += widen(H4.x) + widen(L4.x);
        At[i4 + 1] += widen(H4.y) + widen(L4.y);
        At[i4 + 2] += widen(H4.z) + widen(L4.z);
        At[i4 + 3] += widen(H4.w) + widen(L4.w);
    }
}

}  // namespace

bool astat_tc_ok(int D, int H) { return D % 64 == 0 && D <= 256 && H <= 256 && (D / 2) % 16 == 0; }

int launch_astat_tc(prosper_ctx *c, const float *Y, int64_t N, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    const int D = c->D, H = c->H;
    const int halves = (H + 127) / 128;
    const size_t smem = 1024 + (size_t)2 * halves * 128 * 128 + (size_t)2 * D * 128 +
                        (size_t)AT_T * D * 4;
    if (int rc = ensure_smem_attr((const void *)k_astat_tc, smem)) return rc;
    uint32_t cols = 32;
    while ((int)cols < halves * D) cols <<= 1;
    // one CTA per SM whatever N is, so that every partial is written by the
    // first launch of the E-step (CTAs without tiles store zeros)
    const int grid = c->num_sms;
    TraceScope tr(c, "astat_tc", s);
    k_astat_tc<<<grid, AT_NT, smem, s>>>(Y, c->sel, c->es, N, D, H, c->Hp, halves, cols, c->apart,
                                         c->apart_pieces > 0 ? 1 : 0, c->d_status);
    PROSPER_LAUNCH_CHECK();
    ++c->apart_pieces;
    return PROSPER_OK;
}

int finish_astat_tc(prosper_ctx *c, double *At, cudaStream_t s) {
    if (c->apart_pieces == 0) return PROSPER_OK;
    const int64_t HD = (int64_t)c->H * c->D;
    TraceScope tr(c, "astat_tc_reduce", s);
    // H D is a multiple of 4 (D % 64 == 0 on this path): one block per 128 elements
    k_reduce_parts<<<(int)((HD + 127) / 128), 256, 0, s>>>(c->apart, c->num_sms, HD, At);
    PROSPER_LAUNCH_CHECK();
    c->apart_pieces = 0;
    return PROSPER_OK;
}

}  // namespace prosper
