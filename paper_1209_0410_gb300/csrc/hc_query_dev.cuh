// Device helpers of the query path shared by the query kernel, the exact
// brute force and the depth predictor: 16-byte row gathers, exact distances,
// the reduce-scatter of per-lane partial sums, and lower_bound on 128-bit
// keys.
#pragma once

#include <type_traits>

#include "hc_internal.h"
#include "hc_topk.cuh"

namespace hc {

__device__ __forceinline__ uint4 ldg16(const void* p) {
    return __ldg(reinterpret_cast<const uint4*>(p));
}

__device__ __forceinline__ uint32_t acc_vec(uint4 a, uint4 b, uint32_t acc) {
    uint32_t t;
    t = __vabsdiffu4(a.x, b.x);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.y, b.y);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.z, b.z);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.w, b.w);
    acc = __dp4a(t, t, acc);
    return acc;
}

__device__ __forceinline__ float acc_vec(uint4 a, uint4 b, float acc) {
    float t;
    t = __uint_as_float(a.x) - __uint_as_float(b.x);
    acc = fmaf(t, t, acc);
    t = __uint_as_float(a.y) - __uint_as_float(b.y);
    acc = fmaf(t, t, acc);
    t = __uint_as_float(a.z) - __uint_as_float(b.z);
    acc = fmaf(t, t, acc);
    t = __uint_as_float(a.w) - __uint_as_float(b.w);
    acc = fmaf(t, t, acc);
    return acc;
}

__device__ __forceinline__ uint32_t dist_bits(uint32_t d) { return d; }
__device__ __forceinline__ uint32_t dist_bits(float d) { return __float_as_uint(d); }

// v[j] = this lane's partial of sub-batch j (j < LPR).  Returns the full sum of
// sub-batch (lane % LPR) over the LPR lanes of the lane's group.
template <int LPR, typename Acc>
__device__ __forceinline__ Acc reduce_scatter(Acc (&v)[LPR], uint32_t s) {
#pragma unroll
    for (int w = LPR / 2; w >= 1; w >>= 1) {
        const bool upper = (s & (uint32_t)w) != 0;
#pragma unroll
        for (int t = 0; t < w; ++t) {
            const Acc send = upper ? v[t] : v[t + w];
            const Acc keep = upper ? v[t + w] : v[t];
            v[t] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

// Distances of up to 32 rows (row r of the chunk has id shfl(id, r), valid
// for r < cnt) to the query; returns this lane's packed candidate: the row
// (lane % LPR) * (32 / LPR) + lane / LPR of the chunk, or kEmpty.
template <bool F32, int LPR>
__device__ __forceinline__ uint64_t chunk_candidates(const uint8_t* __restrict__ db,
                                                     uint32_t row_bytes, const uint8_t* qrow,
                                                     uint4 qv0, uint32_t id, uint32_t cnt,
                                                     int lane) {
    using Acc = typename std::conditional<F32, float, uint32_t>::type;
    constexpr int RPI = 32 / LPR;
    constexpr int G = LPR < 8 ? LPR : 8;
    const uint32_t s = (uint32_t)lane % LPR, g = (uint32_t)lane / LPR;
    const uint32_t vecs = row_bytes >> 4;
    const uint32_t vpl = (vecs + LPR - 1) / LPR;
    Acc part[LPR];
#pragma unroll
    for (int j = 0; j < LPR; ++j) part[j] = Acc(0);
    for (uint32_t v = 0; v < vpl; ++v) {
        const uint32_t col = s + v * LPR;
        const bool colok = col < vecs;
        const uint4 qv = v == 0 ? qv0 : (colok ? ldg16(qrow + col * 16) : make_uint4(0, 0, 0, 0));
#pragma unroll
        for (int j0 = 0; j0 < LPR; j0 += G) {
            uint4 rv[G];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const uint32_t r = (uint32_t)(j0 + j) * RPI + g;
                const uint32_t rid = __shfl_sync(0xffffffffu, id, (int)r);
                rv[j] = (r < cnt && colok) ? ldg16(db + (size_t)rid * row_bytes + col * 16)
                                           : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < G; ++j) part[j0 + j] = acc_vec(rv[j], qv, part[j0 + j]);
        }
    }
    const Acc dsum = reduce_scatter<LPR>(part, s);
    const uint32_t r = s * RPI + g;
    const uint32_t cid = __shfl_sync(0xffffffffu, id, (int)r);
    return r < cnt ? ((uint64_t)dist_bits(dsum) << 32) | cid : kEmpty;
}

// first i in [0, n) with key[i] >= (kh, kl), else n
__device__ __forceinline__ uint32_t lower_bound_key(const uint64_t* __restrict__ hi,
                                                    const uint64_t* __restrict__ lo, uint32_t n,
                                                    uint64_t kh, uint64_t kl) {
    uint32_t first = 0, count = n;
    while (count > 0) {
        const uint32_t step = count >> 1, mid = first + step;
        const uint64_t h = __ldg(hi + mid);
        bool less = h < kh;
        if (h == kh) less = __ldg(lo + mid) < kl;
        if (less) {
            first = mid + 1;
            count -= step + 1;
        } else {
            count = step;
        }
    }
    return first;
}

// K1 + K3 for one query: positions of the query key in every list, written
// to pos_w[0..lists).
__device__ __forceinline__ void query_positions(const IndexView& ix, const uint8_t* qrow,
                                                uint32_t* pos_w, int lane) {
    const uint32_t curves = ix.P.curves;
    uint64_t khi = 0, klo = 0;
    if ((uint32_t)lane < curves) curve_key(qrow, ix.P, (uint32_t)lane, khi, klo);
    for (uint32_t b = 0; b < ix.lists; b += 32) {
        const uint32_t L = b + (uint32_t)lane;
        const int c = (int)(L % curves);
        const uint64_t kh = __shfl_sync(0xffffffffu, khi, c);
        const uint64_t kl = __shfl_sync(0xffffffffu, klo, c);
        if (L < ix.lists) {
            const uint64_t off = ix.list_off[L];
            const uint32_t n = (uint32_t)(ix.list_off[L + 1] - off);
            pos_w[L] = lower_bound_key(ix.keys_hi + off, ix.keys_lo + off, n, kh, kl);
        }
    }
    __syncwarp();
}


}  // namespace hc
