// Device-side building blocks shared by the libhc kernels: the Hilbert
// extended-key C^-1 (Sec. 2.2.1), the float32 key quantisation and the
// projection of a vector onto one curve's subspace (the per-curve step of
// Algorithms 1 and 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hc.h"
#include "hc_check.cuh"

namespace hc {

// Where the m coordinates of curve c come from.
struct Projection {
    uint32_t d;                 // coordinates per row
    uint32_t curves;            // curves per partition
    uint32_t m;                 // coordinates per curve (<= 16)
    const uint32_t* dim_map;    // device, curves*m entries; nullptr = consecutive
    hc_dtype dtype;
};

// 8x8 bit-matrix transpose of a 64-bit word whose byte i is row i: afterwards
// byte j holds bit j of every input byte (bit i = input byte i).  Three
// delta swaps (the classic transpose of Hacker's Delight, Sec. 7-3).
__device__ __forceinline__ uint64_t transpose8x8(uint64_t x) {
    uint64_t t;
    t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x = x ^ t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x = x ^ t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x = x ^ t ^ (t << 28);
    return x;
}

// Hilbert extended-key of M coordinates of 8 bits (Skilling's transpose
// formulation of the iterative Gray-code method), written branch-free.
//  - levels q = 7..1: an axis with bit q set inverts the low q bits of axis
//    0; otherwise axis 0 and the axis exchange their low q bits;
//  - Gray code across axes (prefix xor), then the correction whose bit r is
//    the parity of the last axis's bits above r;
//  - key = bit plane 7 (axis 0 as its most significant bit), then plane 6,
//    ... plane 0.  For M = 16 the planes come from two 8x8 bit transposes.
template <int M>
__device__ __forceinline__ void hilbert_key(uint32_t (&X)[16], uint64_t& hi, uint64_t& lo) {
#pragma unroll
    for (int q = 7; q >= 1; --q) {
        const uint32_t low = (1u << q) - 1u;
        X[0] ^= low & (0u - ((X[0] >> q) & 1u));
#pragma unroll
        for (int i = 1; i < M; ++i) {
            const uint32_t set = 0u - ((X[i] >> q) & 1u);
            const uint32_t t = (X[0] ^ X[i]) & low & ~set;
            X[0] ^= t ^ (low & set);
            X[i] ^= t;
        }
    }
#pragma unroll
    for (int i = 1; i < M; ++i) X[i] ^= X[i - 1];
    uint32_t corr = X[M - 1] >> 1;
    corr ^= corr >> 1;
    corr ^= corr >> 2;
    corr ^= corr >> 4;
#pragma unroll
    for (int i = 0; i < M; ++i) X[i] ^= corr;

    if constexpr (M == 16) {
        uint32_t a0 = X[0] | (X[1] << 8) | (X[2] << 16) | (X[3] << 24);
        uint32_t a1 = X[4] | (X[5] << 8) | (X[6] << 16) | (X[7] << 24);
        uint32_t b0 = X[8] | (X[9] << 8) | (X[10] << 16) | (X[11] << 24);
        uint32_t b1 = X[12] | (X[13] << 8) | (X[14] << 16) | (X[15] << 24);
        uint64_t A = transpose8x8((uint64_t)a0 | ((uint64_t)a1 << 32));
        uint64_t B = transpose8x8((uint64_t)b0 | ((uint64_t)b1 << 32));
        // byte j of A (B) = plane j of axes 0..7 (8..15), axis i at bit i.
        const uint32_t Al = (uint32_t)A, Ah = (uint32_t)(A >> 32);
        const uint32_t Bl = (uint32_t)B, Bh = (uint32_t)(B >> 32);
        // word = [A_q1, B_q1, A_q0, B_q0]; bit reversal puts plane q1 (axis 0
        // first) in the high half and plane q0 in the low half.
        const uint32_t w76 = __byte_perm(Ah, Bh, 0x6273);
        const uint32_t w54 = __byte_perm(Ah, Bh, 0x4051);
        const uint32_t w32 = __byte_perm(Al, Bl, 0x6273);
        const uint32_t w10 = __byte_perm(Al, Bl, 0x4051);
        hi = ((uint64_t)__brev(w76) << 32) | __brev(w54);
        lo = ((uint64_t)__brev(w32) << 32) | __brev(w10);
    } else {
        unsigned __int128 key = 0;
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            uint32_t plane = 0;
#pragma unroll
            for (int i = 0; i < M; ++i) plane |= ((X[i] >> q) & 1u) << (M - 1 - i);
            key = (key << M) | plane;
        }
        hi = (uint64_t)(key >> 64);
        lo = (uint64_t)key;
    }
}

// 4x4 byte transpose: out[b] byte k = in[k] byte b.
__device__ __forceinline__ void transpose4x4_bytes(uint32_t a0, uint32_t a1, uint32_t a2,
                                                   uint32_t a3, uint32_t (&out)[4]) {
    const uint32_t t0 = __byte_perm(a0, a1, 0x5140), t1 = __byte_perm(a0, a1, 0x7362);
    const uint32_t t2 = __byte_perm(a2, a3, 0x5140), t3 = __byte_perm(a2, a3, 0x7362);
    out[0] = __byte_perm(t0, t2, 0x5410);
    out[1] = __byte_perm(t0, t2, 0x7632);
    out[2] = __byte_perm(t1, t3, 0x5410);
    out[3] = __byte_perm(t1, t3, 0x7632);
}

// Four 16-coordinate Hilbert keys at once, SIMD within a register: byte k of
// X[i] is coordinate i of key k, and every step of hilbert_key<16> becomes
// byte-parallel logic (per-byte masks from a multiply by 0xFF, which runs on
// the FMA pipe and spares the integer ALU pipe).  c[k] holds key k's 16
// coordinate bytes (coordinate i = byte i % 4 of word i / 4).
// HI_ONLY: only the high words (bit planes 7..4) are wanted.  Level q changes
// only bits below q and decides on bit q, so planes 7..4 are final after the
// levels 7, 6 and 5; the Gray code and the correction of a plane depend on
// that plane and the planes above it.  Levels 4..1 are skipped and lo is
// left unset.
template <bool HI_ONLY = false>
__device__ __forceinline__ void hilbert_keys4(const uint4 (&c)[4], uint64_t (&hi)[4],
                                              uint64_t (&lo)[4]) {
    constexpr uint32_t ONES = 0x01010101u;
    uint32_t X[16];
    {
        const uint32_t w[4][4] = {{c[0].x, c[0].y, c[0].z, c[0].w},
                                  {c[1].x, c[1].y, c[1].z, c[1].w},
                                  {c[2].x, c[2].y, c[2].z, c[2].w},
                                  {c[3].x, c[3].y, c[3].z, c[3].w}};
#pragma unroll
        for (int wi = 0; wi < 4; ++wi) {
            uint32_t t[4];
            transpose4x4_bytes(w[0][wi], w[1][wi], w[2][wi], w[3][wi], t);
#pragma unroll
            for (int b = 0; b < 4; ++b) X[4 * wi + b] = t[b];
        }
    }
#pragma unroll
    for (int q = 7; q >= (HI_ONLY ? 5 : 1); --q) {
        const uint32_t low = ((1u << q) - 1u) * ONES;
        X[0] ^= low & (((X[0] >> q) & ONES) * 0xFFu);
#pragma unroll
        for (int i = 1; i < 16; ++i) {
            const uint32_t set = ((X[i] >> q) & ONES) * 0xFFu;
            const uint32_t d = (X[0] ^ X[i]) & low;
            X[0] ^= (set & low) | (~set & d);
            X[i] ^= d & ~set;
        }
    }
#pragma unroll
    for (int i = 1; i < 16; ++i) X[i] ^= X[i - 1];
    uint32_t corr = (X[15] >> 1) & 0x7F7F7F7Fu;
    corr ^= (corr >> 1) & 0x7F7F7F7Fu;
    corr ^= (corr >> 2) & 0x3F3F3F3Fu;
    corr ^= (corr >> 4) & 0x0F0F0F0Fu;
#pragma unroll
    for (int i = 0; i < 16; ++i) X[i] ^= corr;
    // back to one 16-byte group per key, then the bit-plane transposes
    uint32_t y[4][4];   // y[g][k]: axes 4g..4g+3 of key k
#pragma unroll
    for (int g = 0; g < 4; ++g)
        transpose4x4_bytes(X[4 * g], X[4 * g + 1], X[4 * g + 2], X[4 * g + 3], y[g]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t A = transpose8x8((uint64_t)y[0][k] | ((uint64_t)y[1][k] << 32));
        const uint64_t B = transpose8x8((uint64_t)y[2][k] | ((uint64_t)y[3][k] << 32));
        const uint32_t Al = (uint32_t)A, Ah = (uint32_t)(A >> 32);
        const uint32_t Bl = (uint32_t)B, Bh = (uint32_t)(B >> 32);
        hi[k] = ((uint64_t)__brev(__byte_perm(Ah, Bh, 0x6273)) << 32) |
                __brev(__byte_perm(Ah, Bh, 0x4051));
        if (!HI_ONLY)
            lo[k] = ((uint64_t)__brev(__byte_perm(Al, Bl, 0x6273)) << 32) |
                    __brev(__byte_perm(Al, Bl, 0x4051));
    }
}

__device__ __forceinline__ void hilbert_key_m(uint32_t m, uint32_t (&X)[16], uint64_t& hi,
                                              uint64_t& lo) {
    switch (m) {
        case 16: hilbert_key<16>(X, hi, lo); break;
        case 15: hilbert_key<15>(X, hi, lo); break;
        case 14: hilbert_key<14>(X, hi, lo); break;
        case 13: hilbert_key<13>(X, hi, lo); break;
        case 12: hilbert_key<12>(X, hi, lo); break;
        case 11: hilbert_key<11>(X, hi, lo); break;
        case 10: hilbert_key<10>(X, hi, lo); break;
        case 9: hilbert_key<9>(X, hi, lo); break;
        case 8: hilbert_key<8>(X, hi, lo); break;
        case 7: hilbert_key<7>(X, hi, lo); break;
        case 6: hilbert_key<6>(X, hi, lo); break;
        case 5: hilbert_key<5>(X, hi, lo); break;
        case 4: hilbert_key<4>(X, hi, lo); break;
        case 3: hilbert_key<3>(X, hi, lo); break;
        case 2: hilbert_key<2>(X, hi, lo); break;
        default: hilbert_key<1>(X, hi, lo); break;
    }
}

// Float32 coordinate -> 8-bit key coordinate: rint(x * 255) in float32
// (ties to even), NaN and negatives to 0, clamped at 255.
__device__ __forceinline__ uint32_t quantize_coord(float x) {
    const float s = __fmul_rn(x, 255.0f);
    if (!(s > 0.0f)) return 0u;
    if (s >= 255.0f) return 255u;
    return __float2uint_rn(s);
}

// The 16 coordinate bytes of curve c (consecutive dims, m = 16) of a row.
__device__ __forceinline__ uint4 curve_bytes16(const void* row, hc_dtype dtype, uint32_t c) {
    if (dtype == HC_U8)
        return __ldg(reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(row) + (size_t)c * 16));
    const float4* f = reinterpret_cast<const float4*>(static_cast<const float*>(row) + (size_t)c * 16);
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float4 v = __ldg(f + t);
        w[t] = quantize_coord(v.x) | (quantize_coord(v.y) << 8) | (quantize_coord(v.z) << 16) |
               (quantize_coord(v.w) << 24);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// proj[j] <- v[a[c][j]] for the m coordinates of curve c, as 8-bit values.
__device__ __forceinline__ void load_projection(const void* row, const Projection& P, uint32_t c,
                                                uint32_t (&X)[16]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) X[j] = 0;
    if (P.dim_map == nullptr && P.m == 16) {
        if (P.dtype == HC_U8) {
            // 16 consecutive bytes starting at a multiple of 16
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(
                static_cast<const uint8_t*>(row) + (size_t)c * 16));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 16; ++j) X[j] = (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
        } else {
            const float4* f = reinterpret_cast<const float4*>(
                static_cast<const float*>(row) + (size_t)c * 16);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float4 v = __ldg(f + t);
                X[4 * t + 0] = quantize_coord(v.x);
                X[4 * t + 1] = quantize_coord(v.y);
                X[4 * t + 2] = quantize_coord(v.z);
                X[4 * t + 3] = quantize_coord(v.w);
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if ((uint32_t)j < P.m) {
            const uint32_t dim = P.dim_map ? __ldg(P.dim_map + c * P.m + j) : c * P.m + j;
            X[j] = P.dtype == HC_U8 ? (uint32_t)__ldg(static_cast<const uint8_t*>(row) + dim)
                                    : quantize_coord(__ldg(static_cast<const float*>(row) + dim));
        }
    }
}

__device__ __forceinline__ void curve_key(const void* row, const Projection& P, uint32_t c,
                                          uint64_t& hi, uint64_t& lo) {
    uint32_t X[16];
    load_projection(row, P, c, X);
    hilbert_key_m(P.m, X, hi, lo);
}

// curve_key out of line, for code that computes a few keys per query (one
// copy per translation unit instead of one per kernel instantiation)
static __device__ __noinline__ void curve_key_call(const void* row, const Projection& P, uint32_t c,
                                            uint64_t& hi, uint64_t& lo) {
    curve_key(row, P, c, hi, lo);
}

// Low key word of one row on curve c (the index keeps high words only when
// they carry 64 key bits; ties of the high words are rare and decided here).
// (out of line: it is on rare paths, and one copy per translation unit keeps
// the many query-kernel instantiations small)
static __device__ __noinline__ uint64_t row_key_lo(const void* db, uint32_t row_bytes,
                                            const Projection& P, uint32_t row, uint32_t c) {
    uint64_t h, l;
    curve_key_call(static_cast<const uint8_t*>(db) + (size_t)row * row_bytes, P, c, h, l);
    return l;
}

// Partition of row r when n rows are split into l contiguous ranges
// [floor(j*n/l), floor((j+1)*n/l)): the largest j whose range starts at or
// before r, i.e. floor(((r+1)*l - 1) / n).
__host__ __device__ __forceinline__ uint32_t partition_of(uint64_t r, uint64_t n, uint32_t l) {
    return (uint32_t)(((r + 1) * (uint64_t)l - 1) / n);
}

__host__ __device__ __forceinline__ uint64_t partition_start(uint32_t j, uint64_t n, uint32_t l) {
    return ((uint64_t)j * n) / l;
}

}  // namespace hc
