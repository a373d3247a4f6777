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

// descending sort of 8 keys: Batcher's odd-even merge network (19 comparators)
__device__ __forceinline__ void sort8_desc(unsigned (&k)[8]) {
#define PROSPER_CE(i, j) { const unsigned a = max(k[i], k[j]), b = min(k[i], k[j]); k[i] = a; k[j] = b; }
    PROSPER_CE(0, 1) PROSPER_CE(2, 3) PROSPER_CE(4, 5) PROSPER_CE(6, 7)
    PROSPER_CE(0, 2) PROSPER_CE(1, 3) PROSPER_CE(4, 6) PROSPER_CE(5, 7)
    PROSPER_CE(1, 2) PROSPER_CE(5, 6)
    PROSPER_CE(0, 4) PROSPER_CE(1, 5) PROSPER_CE(2, 6) PROSPER_CE(3, 7)
    PROSPER_CE(2, 4) PROSPER_CE(3, 5)
    PROSPER_CE(1, 2) PROSPER_CE(3, 4) PROSPER_CE(5, 6)
#undef PROSPER_CE
}

// Packed preselection key of score s for latent h (H <= 256): the
// order-preserving key of s rounded down to its top 24 bits, with 255 - h in
// the low byte, so that one 32-bit comparison ranks by score and breaks ties
// (exact ones and those the rounding makes) to the lower h.  kmask / klow are
// 0xFFFFFF00 / 255 - h for a present latent and 0 / 0 for an absent one.
__device__ __forceinline__ unsigned packed_key(float s, unsigned kmask, unsigned klow) {
    const unsigned b = __float_as_uint(s);
    // flip all bits of a negative score, only the sign bit of a positive one
    const unsigned key = b ^ ((unsigned)((int)b >> 31) | 0x80000000u);
    return (key & kmask) | klow;
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
