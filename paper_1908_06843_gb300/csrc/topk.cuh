// topk.cuh -- exact warp-wide top-H' preselection (paper Sec. 3: the H'
// candidate latents of a data point), shared by the FP32 and BF16 projection
// kernels.  Scores are compared as order-preserving 32-bit keys; exact ties go
// to the lower latent index h.
#pragma once

#include <cstdint>

namespace prosper {

__device__ __forceinline__ unsigned score_key(float s) {
    const unsigned b = __float_as_uint(s);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Reference selection by rounds: Hp rounds of (warp max key, lowest h among the
// lanes holding it).  Returns in lane r < Hp the h chosen in round r.
__device__ __forceinline__ int topk_rounds(unsigned (&key)[8], int Hp, int lane) {
    unsigned lk = key[0];
    int lj = 0;
#pragma unroll
    for (int j = 1; j < 8; ++j)
        if (key[j] > lk) { lk = key[j]; lj = j; }
    int mine = 0x7fffffff;
    for (int r = 0; r < Hp; ++r) {
        const unsigned wmax = __reduce_max_sync(0xffffffffu, lk);
        const unsigned code = (lk == wmax) ? (unsigned)(lj * 32 + lane) : 0xffffffffu;
        const unsigned hw = __reduce_min_sync(0xffffffffu, code);
        if (lane == r) mine = (int)hw;
        if ((int)(hw & 31u) == lane) {
            const int jw = (int)(hw >> 5);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j == jw) key[j] = 0u;
            lk = key[0];
            lj = 0;
#pragma unroll
            for (int j = 1; j < 8; ++j)
                if (key[j] > lk) { lk = key[j]; lj = j; }
        }
    }
    return mine;
}

// Exact top-Hp of the 256 keys held 8 per lane (h = lane + 32 j; key 0 = absent).
// 1. tau = the Hp-th largest of the 32 lane maxima (a bitonic sort across the
//    warp).  The Hp-th largest key overall is >= tau, so every winner is >= tau.
// 2. The C keys >= tau are compacted into the warp (one per lane) through a
//    64-word shared scratch and bitonic-sorted by (key descending, h ascending).
// If C > 32 (many equal keys) the rounds method runs instead.  Returns in lane
// r < Hp the r-th best h (descending score); other lanes get 0x7fffffff.
__device__ __forceinline__ int warp_topk(unsigned (&key)[8], int Hp, int lane,
                                         volatile unsigned *scratch) {
    unsigned lk = key[0];
#pragma unroll
    for (int j = 1; j < 8; ++j) lk = max(lk, key[j]);
    unsigned v = lk;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool keep_max = ((lane & k) == 0) == ((lane & j) == 0);
            v = keep_max ? max(v, o) : min(v, o);
        }
    const unsigned tau = __shfl_sync(0xffffffffu, v, Hp - 1);
    unsigned msk = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) msk |= (key[j] >= tau && key[j] != 0u) ? (1u << j) : 0u;
    const int c = __popc(msk);
    const int C = (int)__reduce_add_sync(0xffffffffu, (unsigned)c);
    if (C > 32 || tau == 0u) return topk_rounds(key, Hp, lane);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    int pos = x - c;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if ((msk >> j) & 1u) {
            scratch[pos] = key[j];
            scratch[32 + pos] = (unsigned)(lane + 32 * j);
            ++pos;
        }
    __syncwarp();
    unsigned ck = lane < C ? scratch[lane] : 0u;
    int chh = lane < C ? (int)scratch[32 + lane] : 0x7fffffff;
    __syncwarp();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned ok = __shfl_xor_sync(0xffffffffu, ck, j);
            const int oh = __shfl_xor_sync(0xffffffffu, chh, j);
            const bool other_better = ok > ck || (ok == ck && oh < chh);
            const bool keep_better = ((lane & k) == 0) == ((lane & j) == 0);
            if (keep_better == other_better) { ck = ok; chh = oh; }
        }
    return lane < Hp ? chh : 0x7fffffff;
}

// Rank of this lane's selected h among the Hp selected ones (ascending h).
__device__ __forceinline__ int topk_rank(int myh, int Hp, int lane) {
    int rank = 0;
    for (int r = 0; r < Hp; ++r) {
        const int o = __shfl_sync(0xffffffffu, myh, r);
        rank += (o < myh) ? 1 : 0;
    }
    return rank;
}

}  // namespace prosper
