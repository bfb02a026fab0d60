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

// Candidates produced per lane by one 32-row chunk: rows wider than 8 lanes
// are reduced 8 sub-batches at a time, leaving one candidate per group.
#ifndef HC_GROUP_MAX
#define HC_GROUP_MAX 8   // sub-batches (rows per lane group) loaded before reducing
#endif

template <int LPR>
struct ChunkWidth {
    static constexpr int G = LPR < HC_GROUP_MAX ? LPR : HC_GROUP_MAX;
    static constexpr int NG = LPR / G;            // groups, candidates per lane
};

// Distances of up to 32 rows (row r of the chunk has id shfl(id, r), valid for
// r < cnt) to the query.  LPR lanes read one row, 32 / LPR rows per warp
// instruction, so the chunk takes LPR sub-batches; they are processed in
// groups of G = min(LPR, 8): the G partial sums of a group are reduce-scattered
// over the LPR lanes (G - 1 shuffles, then log2(LPR / G) plain ones), after
// which lane s holds sub-batch s / (LPR / G) of the group.  out[g] is the
// packed (distance, id) candidate of that row, or kEmpty (rows past cnt, and
// the LPR / G - 1 lanes that hold a copy).
template <bool F32, int LPR>
__device__ __forceinline__ void chunk_candidates_n(const uint8_t* __restrict__ db,
                                                   uint32_t row_bytes, const uint8_t* qrow,
                                                   uint4 qv0, uint32_t id, uint32_t cnt, int lane,
                                                   uint64_t (&out)[ChunkWidth<LPR>::NG]) {
    using Acc = typename std::conditional<F32, float, uint32_t>::type;
    constexpr int RPI = 32 / LPR;
    constexpr int G = ChunkWidth<LPR>::G;
    constexpr int NG = ChunkWidth<LPR>::NG;
    constexpr int COPIES = LPR / G;
    const uint32_t s = (uint32_t)lane % LPR, g = (uint32_t)lane / LPR;
    const uint32_t vecs = row_bytes >> 4;
    const uint32_t vpl = (vecs + LPR - 1) / LPR;
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
        Acc part[G];
#pragma unroll
        for (int j = 0; j < G; ++j) part[j] = Acc(0);
        for (uint32_t v = 0; v < vpl; ++v) {
            const uint32_t col = s + v * LPR;
            const bool colok = col < vecs;
            const uint4 qv =
                v == 0 ? qv0 : (colok ? ldg16(qrow + col * 16) : make_uint4(0, 0, 0, 0));
            uint4 rv[G];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const uint32_t r = (uint32_t)(gi * G + j) * RPI + g;
                const uint32_t rid = __shfl_sync(0xffffffffu, id, (int)r);
                rv[j] = (r < cnt && colok) ? ldg16(db + (size_t)rid * row_bytes + col * 16)
                                           : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < G; ++j) part[j] = acc_vec(rv[j], qv, part[j]);
        }
        // halving steps over the top log2(G) bits of s
#pragma unroll
        for (int w = LPR / 2, half = G / 2; half >= 1; w >>= 1, half >>= 1) {
            const bool upper = (s & (uint32_t)w) != 0;
#pragma unroll
            for (int t = 0; t < half; ++t) {
                const Acc send = upper ? part[t] : part[t + half];
                const Acc keep = upper ? part[t + half] : part[t];
                part[t] = keep + __shfl_xor_sync(0xffffffffu, send, w);
            }
        }
        // plain sums over the low log2(LPR / G) bits
        Acc dsum = part[0];
#pragma unroll
        for (int w = COPIES / 2; w >= 1; w >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, w);
        const uint32_t j = s / COPIES;
        const uint32_t r = (uint32_t)(gi * G + j) * RPI + g;
        const uint32_t cid = __shfl_sync(0xffffffffu, id, (int)(r < 32 ? r : 0));
        out[gi] = (r < cnt && (s % COPIES) == 0) ? ((uint64_t)dist_bits(dsum) << 32) | cid : kEmpty;
    }
}

// Low key word of entry g (global entry index) of list L.
__device__ __forceinline__ uint64_t entry_key_lo(const IndexView& ix, uint32_t L, uint64_t g) {
    if (ix.keys_lo) return __ldg(ix.keys_lo + g);
    const uint32_t id = __ldg(ix.ids + g);
    return row_key_lo(ix.db, ix.row_bytes, ix.P, HC_IN_BOUNDS(kSiteRow, id, ix.rows) ? id : 0u,
                      L % ix.P.curves);
}

// first i in [first, first + count) (global entries of list L) with key[i] >=
// (kh, kl), else first + count; the low word is consulted only when the high
// words tie
__device__ __forceinline__ uint64_t lower_bound_range(const IndexView& ix, uint32_t L,
                                                      uint64_t first, uint32_t count,
                                                      uint64_t end, uint64_t kh, uint64_t kl) {
    while (count > 0) {
        const uint32_t step = count >> 1;
        const uint64_t mid = first + step;
        if (!HC_IN_BOUNDS(kSiteSearch, mid, end)) break;
        const uint64_t h = __ldg(ix.keys_hi + mid);
        bool less = h < kh;
        if (h == kh) less = entry_key_lo(ix, L, mid) < kl;
        if (less) {
            first = mid + 1;
            count -= step + 1;
        } else {
            count = step;
        }
    }
    return first;
}

// first i in [0, n) of list L (entries off ..) with key[i] >= (kh, kl), else n.
// With a fence (the top 48 bits of every 16th high word of the index), the
// fence words inside the list are searched first against pk = kh &
// kFenceMask: the last one below pk and the first one above it bracket the
// answer, which is then found among the at most 15 entries between them (one
// 128-byte line of high words) instead of by probes spread over the whole
// list.  Fence words equal to pk widen the bracket to the fence words that
// tie.
__device__ __forceinline__ uint32_t lower_bound_key(const IndexView& ix, uint32_t L, uint64_t off,
                                                    uint32_t n, uint64_t kh, uint64_t kl) {
    if (!ix.fence) return (uint32_t)(lower_bound_range(ix, L, off, n, off + n, kh, kl) - off);
    const uint64_t ja = (off + 15) >> kFenceShift, jb = (off + n + 15) >> kFenceShift;
    const uint64_t pk = kh & kFenceMask;
    // jl = first fence point of the list whose fence word is >= pk
    uint64_t jl = ja;
    for (uint32_t count = (uint32_t)(jb - ja); count > 0;) {
        const uint32_t step = count >> 1;
        const uint64_t mid = jl + step;
        if (!HC_IN_BOUNDS(kSiteSearch, mid, ix.fence_len)) break;
        if (__ldg(ix.fence + mid) < pk) {
            jl = mid + 1;
            count -= step + 1;
        } else {
            count = step;
        }
    }
    // entries before lo are below the key (fence point jl - 1 is); the entry
    // at hi, a fence point whose word is above pk, is not
    const uint64_t lo = jl > ja ? ((jl - 1) << kFenceShift) + 1 : off;
    uint64_t hi = off + n;
    if (jl < jb && HC_IN_BOUNDS(kSiteSearch, jl, ix.fence_len)) {
        if (__ldg(ix.fence + jl) > pk) {
            hi = jl << kFenceShift;
        } else {
            // fence points tying pk: the first one above it ends the bracket
            uint64_t ju = jl + 1;
            for (uint32_t count = (uint32_t)(jb - ju); count > 0;) {
                const uint32_t step = count >> 1;
                const uint64_t mid = ju + step;
                if (!HC_IN_BOUNDS(kSiteSearch, mid, ix.fence_len)) break;
                if (__ldg(ix.fence + mid) <= pk) {
                    ju = mid + 1;
                    count -= step + 1;
                } else {
                    count = step;
                }
            }
            if (ju < jb) hi = ju << kFenceShift;
        }
    }
    return (uint32_t)(lower_bound_range(ix, L, lo, (uint32_t)(hi - lo), off + n, kh, kl) - off);
}

// lower_bound_key of G keys (kh[g], kl[g]) in G lists (lists[g], skipped
// where on[g] is false), the G searches in lockstep so that G loads are in
// flight per lane.  Each search halves without branches (the probe picks the
// half, the length shrinks by the same amount whatever the outcome), so lanes
// searching lists of one length run the same steps: the fence points of the
// list (first word >= kh[g] & kFenceMask), the bracket, then the first entry of the
// bracket whose key is >= (kh[g], kl[g]).  pos[g] is list-relative.  Entry indexes fit 32
// bits (an index holds fewer than 2^32 entries).
template <int G>
__device__ __forceinline__ void lower_bound_lists(const IndexView& ix, const uint32_t (&lists)[G],
                                                  const bool (&on)[G], const uint64_t (&kh)[G],
                                                  const uint64_t (&kl)[G], uint32_t (&pos)[G]) {
    if (!ix.fence) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (!on[g]) continue;
            const uint64_t off = ix.list_off[lists[g]];
            pos[g] = lower_bound_key(ix, lists[g], off,
                                     (uint32_t)(ix.list_off[lists[g] + 1] - off), kh[g], kl[g]);
        }
        return;
    }
    uint64_t pk[G];
#pragma unroll
    for (int g = 0; g < G; ++g) pk[g] = kh[g] & kFenceMask;
    uint32_t off[G], end[G], base[G], len[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        off[g] = on[g] ? (uint32_t)ix.list_off[lists[g]] : 0u;
        end[g] = on[g] ? (uint32_t)ix.list_off[lists[g] + 1] : 0u;
        base[g] = (uint32_t)(((uint64_t)off[g] + 15) >> kFenceShift);   // ja
        len[g] = (uint32_t)(((uint64_t)end[g] + 15) >> kFenceShift) - base[g];
    }
    // fence points [ja, jb): the answer jl lies in [base, base + len]
    for (;;) {
        bool busy = false;
        uint64_t f[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t mid = base[g] + (len[g] >> 1) - 1;
            const bool go = len[g] > 1 && HC_IN_BOUNDS(kSiteSearch, mid, ix.fence_len);
            f[g] = go ? __ldg(ix.fence + mid) : 0ull;
            if (!go) len[g] = min(len[g], 1u);
            busy |= go;
        }
        if (!busy) break;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (len[g] <= 1) continue;
            const uint32_t half = len[g] >> 1;
            base[g] += f[g] < pk[g] ? half : 0u;
            len[g] -= half;
        }
    }
    // jl = base (+1 when the last candidate is below pk); fence word of jl
    uint32_t jl[G];
    uint64_t fj[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const bool one = len[g] == 1 && HC_IN_BOUNDS(kSiteSearch, base[g], ix.fence_len);
        const uint64_t fb = one ? __ldg(ix.fence + base[g]) : 0ull;
        jl[g] = base[g] + (one && fb < pk[g] ? 1u : 0u);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const uint32_t jbg = (uint32_t)(((uint64_t)end[g] + 15) >> kFenceShift);
        fj[g] = jl[g] < jbg && HC_IN_BOUNDS(kSiteSearch, jl[g], ix.fence_len)
                    ? __ldg(ix.fence + jl[g]) : ~0ull;
    }
    // brackets [base, base + len) as in lower_bound_key
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const uint32_t ja = (uint32_t)(((uint64_t)off[g] + 15) >> kFenceShift);
        const uint32_t jbg = (uint32_t)(((uint64_t)end[g] + 15) >> kFenceShift);
        const uint32_t lo = jl[g] > ja ? ((jl[g] - 1) << kFenceShift) + 1 : off[g];
        uint32_t hi = end[g];
        if (jl[g] < jbg) {
            if (fj[g] > pk[g]) {
                hi = jl[g] << kFenceShift;
            } else {
                // fence points tying pk: the first one above it ends the bracket
                uint32_t ju = jl[g] + 1;
                for (uint32_t cnt = jbg - ju; cnt > 0;) {
                    const uint32_t step = cnt >> 1;
                    const uint32_t mid = ju + step;
                    if (!HC_IN_BOUNDS(kSiteSearch, mid, ix.fence_len)) break;
                    if (__ldg(ix.fence + mid) <= pk[g]) {
                        ju = mid + 1;
                        cnt -= step + 1;
                    } else {
                        cnt = step;
                    }
                }
                if (ju < jbg) hi = ju << kFenceShift;
            }
        }
        base[g] = lo;
        len[g] = hi - lo;
    }
    // first entry of each bracket with key >= (kh, kl): the answer lies in
    // [base, base + len]
    for (;;) {
        bool busy = false;
        uint64_t h[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t mid = base[g] + (len[g] >> 1) - 1;
            const bool go = len[g] > 1 && HC_IN_BOUNDS(kSiteSearch, mid, end[g]);
            h[g] = go ? __ldg(ix.keys_hi + mid) : 0ull;
            if (!go) len[g] = min(len[g], 1u);
            busy |= go;
        }
        if (!busy) break;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (len[g] <= 1) continue;
            const uint32_t half = len[g] >> 1;
            bool less = h[g] < kh[g];
            if (h[g] == kh[g]) less = entry_key_lo(ix, lists[g], base[g] + half - 1) < kl[g];
            base[g] += less ? half : 0u;
            len[g] -= half;
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        uint32_t at = base[g];
        if (len[g] == 1 && HC_IN_BOUNDS(kSiteSearch, at, end[g])) {
            const uint64_t h = __ldg(ix.keys_hi + at);
            bool less = h < kh[g];
            if (h == kh[g]) less = entry_key_lo(ix, lists[g], at) < kl[g];
            at += less ? 1u : 0u;
        }
        if (on[g]) pos[g] = at - off[g];
    }
}

// K1 + K3 for one query: positions of the query key in lists L0, L0 + Lstep,
// ... written to pos_w[L].
__device__ __forceinline__ void query_positions(const IndexView& ix, const uint8_t* qrow,
                                                uint32_t* pos_w, int lane, uint32_t L0 = 0,
                                                uint32_t Lstep = 1) {
    const uint32_t curves = ix.P.curves;
    uint64_t khi = 0, klo = 0;
    if ((uint32_t)lane < curves) curve_key_call(qrow, ix.P, (uint32_t)lane, khi, klo);
    const uint32_t mine = (ix.lists > L0) ? (ix.lists - L0 + Lstep - 1) / Lstep : 0;
    for (uint32_t b = 0; b < mine; b += 32) {
        const uint32_t t = b + (uint32_t)lane;
        const uint32_t L = L0 + t * Lstep;
        const int c = (int)(L % curves);
        const uint64_t kh = __shfl_sync(0xffffffffu, khi, c);
        const uint64_t kl = __shfl_sync(0xffffffffu, klo, c);
        if (t < mine) {
            const uint64_t off = ix.list_off[L];
            const uint32_t n = (uint32_t)(ix.list_off[L + 1] - off);
            pos_w[L] = lower_bound_key(ix, L, off, n, kh, kl);
        }
    }
    __syncwarp();
}

// The query's positions in lists L0, L0 + Lstep, ... into pos_w[L]: read
// from a batch pass when one ran (pos_in: list order, int64; pos_cm: curve-
// major uint32, entry c * partitions + j for list j * curves + c), else
// searched here.
__device__ __forceinline__ void load_positions(const IndexView& ix, const uint8_t* qrow,
                                               uint32_t* pos_w, int lane, uint32_t L0,
                                               uint32_t Lstep, const int64_t* pos_in,
                                               const uint32_t* pos_cm) {
    if (pos_cm) {
        const uint32_t curves = ix.P.curves, parts = ix.lists / curves;
        for (uint32_t L = L0 + (uint32_t)lane * Lstep; L < ix.lists; L += 32 * Lstep)
            pos_w[L] = __ldg(pos_cm + (L % curves) * parts + L / curves);
        __syncwarp();
    } else if (pos_in) {
        for (uint32_t L = L0 + (uint32_t)lane * Lstep; L < ix.lists; L += 32 * Lstep)
            pos_w[L] = (uint32_t)__ldg(pos_in + L);
        __syncwarp();
    } else {
        query_positions(ix, qrow, pos_w, lane, L0, Lstep);
    }
}

// Algorithm 2 for one query over the lists L0, L0 + Lstep, ... into the
// warp's running top-k: keys, positions, then every window in 32-entry steps
// (the next step's ids are loaded while the current rows are in flight).
template <bool F32, int LPR, int KR>
__device__ __forceinline__ void search_lists(const IndexView& ix, const uint8_t* qrow,
                                             uint32_t depth, uint32_t k, uint32_t L0,
                                             uint32_t Lstep, uint32_t* pos_w, WarpTopK<KR>& top,
                                             int lane, const int64_t* pos_in = nullptr,
                                             const uint32_t* pos_cm = nullptr) {
    load_positions(ix, qrow, pos_w, lane, L0, Lstep, pos_in, pos_cm);
    const uint32_t s = (uint32_t)lane % LPR;
    const uint4 qv0 = s < (ix.row_bytes >> 4) ? ldg16(qrow + s * 16) : make_uint4(0, 0, 0, 0);
    const uint8_t* db = static_cast<const uint8_t*>(ix.db);
    for (uint32_t L = L0; L < ix.lists; L += Lstep) {
        const uint64_t off = ix.list_off[L];
        const uint32_t n = (uint32_t)(ix.list_off[L + 1] - off);
        const uint32_t pos = pos_w[L];
        const uint32_t lo = pos > depth ? pos - depth : 0u;
        const uint32_t hi = (uint64_t)pos + depth < (uint64_t)n ? pos + depth : n;
        if (!HC_IN_BOUNDS(kSiteWindow, hi, (uint64_t)n + 1)) continue;
        const uint32_t* idl = ix.ids + off;
        uint32_t next = lo + (uint32_t)lane < hi ? __ldg(idl + lo + lane) : 0u;
        for (uint32_t base = lo; base < hi; base += 32) {
            const uint32_t id = HC_IN_BOUNDS(kSiteRow, next, ix.rows) ? next : 0u;
            const uint32_t cnt = min(32u, hi - base);
            if (base + 32 < hi)
                next = base + 32 + (uint32_t)lane < hi ? __ldg(idl + base + 32 + lane) : 0u;
            uint64_t cand[ChunkWidth<LPR>::NG];
            chunk_candidates_n<F32, LPR>(db, ix.row_bytes, qrow, qv0, id, cnt, lane, cand);
#pragma unroll
            for (int c = 0; c < ChunkWidth<LPR>::NG; ++c) top.offer(cand[c], k, lane);
        }
    }
}


// ---------------------------------------------------------------------------
// Staged form of the window walk for rows of at most 128 bytes (one 16-byte
// vector per lane of a row group, LPR <= 8): the windows of all lists are
// packed back to back and walked in steps of 32 entries (a step may span
// several short windows, so short or uneven windows fill whole steps); the
// rows of the next step are copied into a per-warp shared-memory ring with
// cp.async (no registers held while they are in flight) while the current
// step's rows are reduced, and the step after that has its ids loaded.
// Waits are the hardware's cp.async group waits.
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The windows of the lists this warp walks (L = L0 + m Lstep), packed back
// to back: win_at[m] = first ids entry of window m (global entry index),
// win_pre[m] = number of window entries before window m.  Returns the total.
// win_at may alias pos_w (each slot is read before it is written).
__device__ __forceinline__ uint32_t pack_windows(const IndexView& ix, uint32_t depth, uint32_t L0,
                                                 uint32_t Lstep, const uint32_t* pos_w,
                                                 uint32_t* win_at, uint32_t* win_pre, int lane) {
    const uint32_t nm = ix.lists > L0 ? (ix.lists - L0 + Lstep - 1) / Lstep : 0;
    uint32_t carry = 0;
    for (uint32_t b = 0; b < nm; b += 32) {
        const uint32_t m = b + (uint32_t)lane;
        uint32_t len = 0, at = 0;
        if (m < nm) {
            const uint32_t L = L0 + m * Lstep;
            const uint64_t off = ix.list_off[L];
            const uint32_t n = (uint32_t)(ix.list_off[L + 1] - off);
            const uint32_t pos = pos_w[L];
            const uint32_t lo = pos > depth ? pos - depth : 0u;
            const uint32_t hi = (uint64_t)pos + depth < (uint64_t)n ? pos + depth : n;
            len = hi > lo && HC_IN_BOUNDS(kSiteWindow, hi, (uint64_t)n + 1) ? hi - lo : 0u;
            at = (uint32_t)(off + lo);   // index entries < 2^32
        }
        uint32_t x = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncwarp();
        if (m < nm) {
            win_at[m] = at;
            win_pre[m] = carry + x - len;
        }
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    __syncwarp();
    return carry;
}

// ids of packed step s (entries 32 s .. 32 s + 31 of the concatenated
// windows): lane l finds its window by binary search over win_pre
__device__ __forceinline__ uint32_t packed_ids(const IndexView& ix, const uint32_t* win_at,
                                               const uint32_t* win_pre, uint32_t nm,
                                               uint32_t total, uint32_t s, int lane) {
    const uint32_t e = 32 * s + (uint32_t)lane;
    if (e >= total) return 0u;
    uint32_t lo = 0, count = nm;   // largest m with win_pre[m] <= e
    while (count > 1) {
        const uint32_t half = count >> 1;
        if (win_pre[lo + half] <= e) {
            lo += half;
            count -= half;
        } else {
            count = half;
        }
    }
    const uint64_t ent = (uint64_t)win_at[lo] + (e - win_pre[lo]);
    if (!HC_IN_BOUNDS(kSiteEntry, ent, ix.list_off[ix.lists])) return 0u;
    const uint32_t id = __ldg(ix.ids + ent);
    return HC_IN_BOUNDS(kSiteRow, id, ix.rows) ? id : 0u;
}

// copies of one step: lane (c = lane % 8, g = lane / 8) moves vector c of
// rows g, g + 4, ..., g + 28 (rows past cnt and vectors past the row are
// skipped)
__device__ __forceinline__ void issue_step(const uint8_t* __restrict__ db, uint32_t row_bytes,
                                           uint32_t sbuf, uint32_t id, uint32_t cnt, int lane) {
    const uint32_t c = (uint32_t)lane & 7u, g = (uint32_t)lane >> 3;
    const bool colok = c < (row_bytes >> 4);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const uint32_t r = g + 4u * (uint32_t)t;
        const uint32_t rid = __shfl_sync(0xffffffffu, id, (int)r);
        if (colok && r < cnt)
            cp_async16(sbuf + r * row_bytes + c * 16, db + (size_t)rid * row_bytes + c * 16);
    }
}

// chunk_candidates_n over rows staged in shared memory (LPR <= 8, so one
// candidate per lane)
template <bool F32, int LPR>
__device__ __forceinline__ uint64_t staged_candidates(const uint8_t* sbuf, uint32_t row_bytes,
                                                      uint4 qv0, uint32_t id, uint32_t cnt,
                                                      int lane) {
    static_assert(LPR <= 8, "staged rows are read one vector per lane");
    using Acc = typename std::conditional<F32, float, uint32_t>::type;
    constexpr int RPI = 32 / LPR;
    const uint32_t s = (uint32_t)lane % LPR, g = (uint32_t)lane / LPR;
    const bool colok = s < (row_bytes >> 4);
    Acc part[LPR];
#pragma unroll
    for (int j = 0; j < LPR; ++j) {
        const uint32_t r = (uint32_t)j * RPI + g;
        const uint4 rv = colok ? *reinterpret_cast<const uint4*>(sbuf + r * row_bytes + s * 16)
                               : make_uint4(0, 0, 0, 0);
        part[j] = acc_vec(rv, qv0, Acc(0));
    }
    const Acc dsum = reduce_scatter<LPR>(part, s);
    const uint32_t r = s * RPI + g;
    const uint32_t cid = __shfl_sync(0xffffffffu, id, (int)r);
    return r < cnt ? ((uint64_t)dist_bits(dsum) << 32) | cid : kEmpty;
}

// S ring stages: the copies of S - 1 steps are in flight while one is
// reduced, and the ids of the step after those are loaded.
template <bool F32, int LPR, int KR, int S = 2>
__device__ __forceinline__ void search_lists_staged(const IndexView& ix, const uint8_t* qrow,
                                                    uint32_t depth, uint32_t k, uint32_t L0,
                                                    uint32_t Lstep, uint32_t* pos_w,
                                                    uint32_t* win_pre, uint8_t* ring,
                                                    WarpTopK<KR>& top, int lane,
                                                    const int64_t* pos_in = nullptr,
                                                    const uint32_t* pos_cm = nullptr) {
    static_assert(S >= 2, "one step reduced while another is in flight");
    load_positions(ix, qrow, pos_w, lane, L0, Lstep, pos_in, pos_cm);
    const uint32_t s = (uint32_t)lane % LPR;
    const uint4 qv0 = s < (ix.row_bytes >> 4) ? ldg16(qrow + s * 16) : make_uint4(0, 0, 0, 0);
    const uint8_t* db = static_cast<const uint8_t*>(ix.db);
    const uint32_t row_bytes = ix.row_bytes;
    const uint32_t stage_bytes = 32 * row_bytes;
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
    const uint32_t nm = ix.lists > L0 ? (ix.lists - L0 + Lstep - 1) / Lstep : 0;
    uint32_t* win_at = pos_w;   // positions are consumed by pack_windows
    const uint32_t total = pack_windows(ix, depth, L0, Lstep, pos_w, win_at, win_pre, lane);
    const uint32_t steps = (total + 31) / 32;
    if (steps == 0) return;
    // ids[j]: this lane's id of step a + j; steps a .. a + S - 2 are in flight
    uint32_t ids[S];
#pragma unroll
    for (int j = 0; j < S; ++j)
        ids[j] = (uint32_t)j < steps ? packed_ids(ix, win_at, win_pre, nm, total, j, lane) : 0u;
#pragma unroll
    for (int j = 0; j < S - 1; ++j) {
        if ((uint32_t)j < steps)
            issue_step(db, row_bytes, ring_s + (uint32_t)j * stage_bytes, ids[j],
                       min(32u, total - 32 * (uint32_t)j), lane);
        cp_async_commit();
    }
    uint32_t st = 0;   // stage of step a
    for (uint32_t a = 0; a < steps; ++a) {
        const uint32_t sn = st == 0 ? S - 1 : st - 1;   // stage of step a + S - 1
        if (a + S - 1 < steps)
            issue_step(db, row_bytes, ring_s + sn * stage_bytes, ids[S - 1],
                       min(32u, total - 32 * (a + S - 1)), lane);
        cp_async_commit();
        const uint32_t nid = a + S < steps ? packed_ids(ix, win_at, win_pre, nm, total, a + S, lane)
                                           : 0u;
        cp_async_wait<S - 1>();   // step a has landed
        __syncwarp();
        top.offer(staged_candidates<F32, LPR>(ring + st * stage_bytes, row_bytes, qv0, ids[0],
                                              min(32u, total - 32 * a), lane),
                  k, lane);
        __syncwarp();             // every lane is done with stage st before it is refilled
#pragma unroll
        for (int j = 0; j < S - 1; ++j) ids[j] = ids[j + 1];
        ids[S - 1] = nid;
        st = st + 1 == S ? 0u : st + 1;
    }
    cp_async_wait<0>();
}

}  // namespace hc
