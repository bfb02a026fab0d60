// Warp-wide running top-k over packed candidates (FindTopK of Sec. 5.1 and
// the Aggregator's reduction of Sec. 4.1 in one structure).
//
// A candidate is the 64-bit value (distance bits << 32) | id, so ascending
// packed order is ascending (distance, id): ties go to the lower id.  uint8
// distances are non-negative int32; float32 distances are non-negative
// floats, whose bit patterns order like the values.  ~0 marks an empty slot
// and sorts after every real candidate.
//
// The list is kept sorted across the warp: element e = r*32 + lane lives in
// register r of that lane, KR registers per lane (k <= 32*KR).  A batch of 32
// candidates (one per lane) is filtered against the k-th element; survivors
// are inserted one at a time with a ballot rank and a one-slot shuffle.  An
// id already in the list has an identical packed value (same row, same
// query), so an equal value is dropped: that is the de-duplication of
// candidates returned by several curves or windows.
#pragma once

#include <stdint.h>

namespace hc {

constexpr uint64_t kEmpty = ~0ull;

template <int KR>
struct WarpTopK {
    uint64_t v[KR];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int r = 0; r < KR; ++r) v[r] = kEmpty;
    }

    // element k-1 (warp-uniform result)
    __device__ __forceinline__ uint64_t kth(uint32_t k) const {
        const uint32_t e = k - 1, rr = e >> 5;
        uint64_t x = v[0];
#pragma unroll
        for (int r = 1; r < KR; ++r)
            if ((uint32_t)r == rr) x = v[r];
        return __shfl_sync(0xffffffffu, x, (int)(e & 31));
    }

    __device__ __forceinline__ void insert(uint64_t y, int lane) {
        uint32_t pos = 0;
        bool dup = false;
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            pos += __popc(__ballot_sync(0xffffffffu, v[r] < y));
            dup |= __any_sync(0xffffffffu, v[r] == y) != 0;
        }
        if (dup) return;
#pragma unroll
        for (int r = KR - 1; r >= 0; --r) {
            const uint64_t up = __shfl_up_sync(0xffffffffu, v[r], 1);
            uint64_t carry = kEmpty;
            if (r > 0) carry = __shfl_sync(0xffffffffu, v[r > 0 ? r - 1 : 0], 31);
            const uint64_t prev = lane == 0 ? carry : up;
            const uint32_t e = (uint32_t)r * 32 + lane;
            v[r] = e > pos ? prev : (e == pos ? y : v[r]);
        }
    }

    // offer one candidate per lane
    __device__ __forceinline__ void offer(uint64_t cand, uint32_t k, int lane) {
        uint64_t thr = kth(k);
        uint32_t m = __ballot_sync(0xffffffffu, cand < thr);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint64_t y = __shfl_sync(0xffffffffu, cand, src);
            if (y < thr) {
                insert(y, lane);
                thr = kth(k);
            }
        }
    }

    // results e < k: ids (-1 for empty) and distances (empty -> int32 max or +inf)
    template <bool F32>
    __device__ __forceinline__ void store(uint32_t k, int lane, int32_t* ids, void* dist) const {
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            const uint32_t e = (uint32_t)r * 32 + lane;
            if (e < k) {
                const uint64_t x = v[r];
                const bool empty = x == kEmpty;
                ids[e] = empty ? -1 : (int32_t)(uint32_t)x;
                const uint32_t dbits = (uint32_t)(x >> 32);
                if (F32)
                    static_cast<uint32_t*>(dist)[e] = empty ? 0x7F800000u : dbits;
                else
                    static_cast<int32_t*>(dist)[e] = empty ? 0x7FFFFFFF : (int32_t)dbits;
            }
        }
    }
};

}  // namespace hc
