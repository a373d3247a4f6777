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
constexpr int AT_NT = 256;    // threads per CTA
constexpr unsigned long long kAtWaitNs = 2000000000ull;

// byte offset of element (row r, point k) in a K-major 64-wide swizzled operand
__device__ __forceinline__ uint32_t kmaj_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__global__ void __launch_bounds__(AT_NT, 1)
k_astat_tc(const float *__restrict__ Y, const int32_t *__restrict__ sel, const float *__restrict__ es,
           int64_t N, int D, int H, int Hp, int halves, uint32_t tmem_cols, float *__restrict__ part,
           unsigned *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *sb = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const int Hpad = halves * 128;
    unsigned char *Ehi = sb;                           // Hpad rows x 128 B
    unsigned char *Elo = Ehi + Hpad * 128;
    // two Y buffers (hi, lo each D rows x 128 B): the next tile's Y is built
    // while the tensor cores read the current one
    unsigned char *Ybuf = Elo + Hpad * 128;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (N + AT_T - 1) / AT_T;
    const uint32_t idesc = idesc_bf16(128, D);
    const uint32_t bar = smem_u32(&mbar);

    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // E starts zeroed once; afterwards every entry is cleared by the thread
    // that wrote it
    {
        uint4 *z = reinterpret_cast<uint4 *>(Ehi);
        const int nz = 2 * Hpad * 128 / 16;
        for (int i = tid; i < nz; i += AT_NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    int prev_h[(PROSPER_MAX_HPRIME + 3) / 4];
#pragma unroll
    for (int j = 0; j < (PROSPER_MAX_HPRIME + 3) / 4; ++j) prev_h[j] = -1;

    // Y of a tile in registers: work item w = (4 consecutive d, 8-point chunk c)
    // with c = 4 ((w >> 2) / (D/4)) + (w & 3), d = 4 ((w >> 2) % (D/4)) + 0..3: a
    // warp's loads cover 4 point rows x 128 contiguous bytes, and the 8 lanes of
    // one shared-memory store wavefront write 8 different swizzle chunk positions
    const int items = (D / 4) * (AT_T / 8);            // <= 512 for D <= 256
    float4 yv[2][8];
    auto item_cd = [&](int w, int &c, int &d4) {
        const int rest = w >> 2;
        d4 = (rest % (D / 4)) * 4;
        c = 4 * (rest / (D / 4)) + (w & 3);
    };
    auto prefetch = [&](int64_t t) {
        const int64_t base = t * AT_T;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int w = tid + AT_NT * r;
            int c, d4;
            item_cd(w, c, d4);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t n = base + 8 * c + i;
                yv[r][i] = (w < items && n < N) ? __ldg(reinterpret_cast<const float4 *>(Y + n * D + d4))
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };

    // the tile's candidate lists and posterior means: thread t handles point
    // t % 64 and its entries j = t / 64 + 4 i
    constexpr int EPT = (PROSPER_MAX_HPRIME + 3) / 4;   // entries per thread
    const int ept_j0 = tid / AT_T, ept_p = tid % AT_T;
    int sh[EPT];
    float sv[EPT];
    auto prefetch_e = [&](int64_t t) {
        const int64_t n = t * AT_T + ept_p;
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            const int j = ept_j0 + 4 * i;
            const bool ok = n < N && j < Hp;
            sh[i] = ok ? min(max(__ldg(sel + n * SEL_STRIDE + j), 0), H - 1) : -1;
            sv[i] = ok ? __ldg(es + n * SEL_STRIDE + j) : 0.f;
        }
    };

    // Y of the prefetched tile (registers) -> hi and lo operands, transposed
    // (points contiguous)
    auto build_y = [&](unsigned char *Yhi, unsigned char *Ylo) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int w = tid + AT_NT * r;
            if (w >= items) continue;
            int c, d4;
            item_cd(w, c, d4);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint32_t ph[4], pl[4];
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const float a = e == 0 ? yv[r][i].x : e == 1 ? yv[r][i].y : e == 2 ? yv[r][i].z : yv[r][i].w;
                    const float b = e == 0 ? yv[r][i + 1].x : e == 1 ? yv[r][i + 1].y : e == 2 ? yv[r][i + 1].z : yv[r][i + 1].w;
                    __nv_bfloat16 ah, al, bh, bl;
                    split_bf16(a, ah, al);
                    split_bf16(b, bh, bl);
                    ph[i >> 1] = (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
                    pl[i >> 1] = (uint32_t)__bfloat16_as_ushort(al) | ((uint32_t)__bfloat16_as_ushort(bl) << 16);
                }
                const int d = d4 + e;
                const uint32_t off = (uint32_t)(d * 128 + ((c ^ (d & 7)) << 4));
                *reinterpret_cast<uint4 *>(Yhi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                *reinterpret_cast<uint4 *>(Ylo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
            }
        }
    };

    uint32_t phase = 0;
    bool aborted = false;
    int done_tiles = 0;
    int64_t tile = blockIdx.x;
    if (tile < ntiles) {
        prefetch(tile);
        prefetch_e(tile);
        build_y(Ybuf, Ybuf + D * 128);
        if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
    }
    for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
        unsigned char *Yhi = Ybuf + (size_t)(it & 1) * 2 * D * 128, *Ylo = Yhi + D * 128;
        // ---- E operand: clear this column's previous entries, write the new ones
        //      (the previous tile's MMA chain has completed)
        // (the entries of one point are distinct latents, so the four threads of
        // a point never write the same element)
#pragma unroll
        for (int i = 0; i < EPT; ++i)
            if (prev_h[i] >= 0) {
                const uint32_t off = kmaj_off(prev_h[i], ept_p);
                *reinterpret_cast<uint16_t *>(Ehi + off) = 0;
                *reinterpret_cast<uint16_t *>(Elo + off) = 0;
                prev_h[i] = -1;
            }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            const int h = sh[i];
            if (h < 0) continue;
            __nv_bfloat16 hi, lo;
            split_bf16(sv[i], hi, lo);
            const uint32_t off = kmaj_off(h, ept_p);
            *reinterpret_cast<__nv_bfloat16 *>(Ehi + off) = hi;
            *reinterpret_cast<__nv_bfloat16 *>(Elo + off) = lo;
            prev_h[i] = h;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t eh = smem_u32(Ehi), el = smem_u32(Elo), yh = smem_u32(Yhi), yl = smem_u32(Ylo);
            for (int hf = 0; hf < halves; ++hf) {
                const uint32_t d_tm = tmem + (uint32_t)(hf * D);
#pragma unroll
                for (int ks = 0; ks < AT_T / 16; ++ks) {
                    const uint32_t ao = (uint32_t)(hf * 128 * 128 + ks * 32), bo = (uint32_t)(ks * 32);
                    umma_bf16(d_tm, desc_sw128(eh + ao), desc_sw128(yh + bo), idesc,
                              (done_tiles > 0 || ks > 0) ? 1u : 0u);
                    umma_bf16(d_tm, desc_sw128(eh + ao), desc_sw128(yl + bo), idesc, 1u);
                    umma_bf16(d_tm, desc_sw128(el + ao), desc_sw128(yh + bo), idesc, 1u);
                }
            }
            umma_commit(bar);
        }
        // while the tensor cores work: the next tile's Y operand goes into the
        // other buffer (last read by the previous, completed chain), and the
        // data of the tile after it start to travel
        if (tile + gridDim.x < ntiles) {
            unsigned char *Yn = Ybuf + (size_t)((it + 1) & 1) * 2 * D * 128;
            build_y(Yn, Yn + D * 128);
            prefetch_e(tile + gridDim.x);
            if (tile + 2 * (int64_t)gridDim.x < ntiles) prefetch(tile + 2 * (int64_t)gridDim.x);
        }
        const bool ok = mbar_wait(bar, phase, kAtWaitNs);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
            aborted = true;
            break;
        }
        tc_fence_after();
        ++done_tiles;
    }
    // ---- epilogue: this CTA's FP32 partial of A^T to global memory (plain
    //      stores; k_reduce_parts sums the partials in FP64 in a fixed order)
    if (!aborted) {
        const int q = warp & 3;
        const int h_in = q * 32 + lane;
        const int cb = (warp < 4) ? 0 : D / 2, ce = (warp < 4) ? D / 2 : D;
        float *mine = part + (size_t)blockIdx.x * H * D;
        for (int hf = 0; hf < halves; ++hf) {
            const int h = hf * 128 + h_in;
            for (int c0 = cb; c0 < ce; c0 += 16) {
                float v[16];
                if (done_tiles > 0) {
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hf * D + c0), v);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = 0.f;
                }
                if (h < H) {
                    float4 *dst = reinterpret_cast<float4 *>(mine + (size_t)h * D + c0);
#pragma unroll
                    for (int k = 0; k < 16; k += 4) dst[k / 4] = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                }
            }
        }
    }
    if (aborted && tid == 0) mbar_wait(bar, phase ^ 1u, kAtWaitNs / 2);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
    }
}

// At += sum over the per-CTA partials, in FP64 and in CTA order
__global__ void k_reduce_parts(const float *__restrict__ part, int nparts, int64_t HD,
                               double *__restrict__ At) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < HD;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll 8
        for (int p = 0; p < nparts; ++p) s += (double)__ldg(part + (size_t)p * HD + i);
        At[i] += s;
    }
}

}  // namespace

bool astat_tc_ok(int D, int H) { return D % 64 == 0 && D <= 256 && H <= 256 && (D / 2) % 16 == 0; }

int launch_astat_tc(prosper_ctx *c, const float *Y, int64_t N, double *At, cudaStream_t s) {
    if (N <= 0) return PROSPER_OK;
    const int D = c->D, H = c->H;
    const int halves = (H + 127) / 128;
    const size_t smem = 1024 + (size_t)2 * halves * 128 * 128 + (size_t)4 * D * 128;
    static size_t attr = 0;
    if (smem > attr) {
        PROSPER_CUDA_TRY(cudaFuncSetAttribute(k_astat_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        attr = smem;
    }
    uint32_t cols = 32;
    while ((int)cols < halves * D) cols <<= 1;
    const int64_t ntiles = (N + AT_T - 1) / AT_T;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)c->num_sms);
    TraceScope tr(c, "astat_tc", s, 2);
    k_astat_tc<<<grid, AT_NT, smem, s>>>(Y, c->sel, c->es, N, D, H, c->Hp, halves, cols, c->apart,
                                         c->d_status);
    PROSPER_LAUNCH_CHECK();
    const int64_t HD = (int64_t)H * D;
    k_reduce_parts<<<(int)std::min<int64_t>((HD + 255) / 256, 4 * c->num_sms), 256, 0, s>>>(
        c->apart, grid, HD, At);
    PROSPER_LAUNCH_CHECK();
    return PROSPER_OK;
}

}  // namespace prosper
