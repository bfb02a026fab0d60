// K2 for indexes of 16-coordinate curves: the sorted lists of Algorithm 1
// ("insert <key, b> into the sorted list"), built in bulk by a sample sort.
//
// Every list is a segment of records (high key word, position); position p
// of list L stands for id = id_base[L] + p, and the lists leave ordered by
// (high word, low word, id), the low word recomputed from the row when two
// high words tie.  Instead of radix passes over every record, each segment
// is cut into buckets of about kTarget records by splitters (order
// statistics of a sample of its keys), every record is moved once to its
// bucket, and each bucket is then sorted inside one block's shared memory:
//
//   level 0  sub-sample (<= kCap keys per segment) sorted by one block
//            -> splitters of level A
//   level A  sample (kSpb keys per final bucket) counted, moved to buckets
//            and sorted -> splitters of level B
//   level B  every record: count (bucket of each record by binary search
//            over the splitters in shared memory, per-block histograms),
//            scan (per bucket over the blocks, then over the buckets),
//            scatter (one 16-byte record per key to its bucket), local sort
//
// A local sort loads a bucket (<= kCap records), packs each key relative to
// the bucket's minimum above the record's index in the bucket, radix-sorts
// the packed words in shared memory (stable 8-bit passes ranked by warp
// ballots) over the bits in which the bucket's keys differ (the lowest ones
// left out when that saves a pass), then one warp per run of equal sorted
// bits orders the run by (key, low word, id) and the bucket leaves in order.
// A bucket above kCap records, or with a run above 32 records, is listed for
// fallback_kernel, which sorts it by (key, low word, id) through global
// memory.  Every step is a kernel on the caller's stream: nothing waits on
// the host.
#include <algorithm>
#include <cstring>
#include <vector>

#include "hc_block.cuh"
#include "hc_internal.h"

namespace hc {

namespace {

constexpr uint32_t kTarget = 2048;      // mean records per bucket
constexpr uint32_t kSpb = 16;           // sample records per bucket of the next level
constexpr uint32_t kMaxBuckets = 8192;  // per segment (splitters in shared memory)
constexpr int kLiBits = 13;             // a record's index in its bucket
constexpr uint64_t kLiMask = (1ull << kLiBits) - 1;
constexpr int kKeyBits = 64 - kLiBits;  // key bits packed above the index
constexpr uint32_t kCap = 5632;         // records one local-sort block holds (< 2^kLiBits)
constexpr int kLThreads = 512;
constexpr int kLWarps = kLThreads / 32;
constexpr int kHistStride = 257;
constexpr int kMaxRounds = (kCap + kLThreads - 1) / kLThreads;   // 32-record rounds per warp
constexpr uint32_t kMaxRuns = 1024;
constexpr int kCThreads = 512;          // count / scatter blocks
constexpr uint32_t kMaxBlkPerSeg = 160;
constexpr uint32_t kMinTileA = 4096;    // items per count / scatter block, level A
constexpr uint32_t kMinTileB = 65536;   // level B
constexpr int kFThreads = 1024;         // fallback blocks
constexpr int kFWarps = kFThreads / 32;

static_assert(kCap < (1u << kLiBits), "bucket index fits its bits");
static_assert(kLWarps * 32 * kMaxRounds >= (int)kCap, "rounds cover a full bucket");

// One segment at one level.
struct LevelSeg {
    uint64_t src;    // first item of the segment in the level's key / record arrays
    uint64_t len;    // items
    uint32_t nb;     // buckets (0: no items at this level)
    uint32_t spl;    // first of the segment's nb - 1 splitters in the level's splitter array
    uint32_t b0;     // first bucket (over all segments of the level)
    uint32_t nblk;   // count / scatter blocks
    uint32_t blk0;   // first count / scatter block
    uint32_t tile;   // items per count / scatter block
    uint64_t cnt0;   // first word of the segment's counts (nb x nblk, bucket-major)
};

__device__ __forceinline__ uint64_t rec_key(uint4 r) {
    return ((uint64_t)r.y << 32) | r.x;
}

// the segment holding unit x (a block, bucket or item) when segment s holds
// [first(s), first(s) + count(s)); segments without units are skipped
template <typename First, typename Count>
__device__ __forceinline__ uint32_t seg_lookup(uint32_t nseg, uint64_t x, First first,
                                               Count count) {
    uint32_t lo = 0, hi = nseg;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (first(mid) <= x) lo = mid; else hi = mid;
    }
    while (lo + 1 < nseg && (count(lo) == 0 || first(lo) + count(lo) <= x)) ++lo;
    return lo;
}

__device__ __forceinline__ uint32_t seg_of_block(const LevelSeg* L, uint32_t nseg, uint32_t blk) {
    return seg_lookup(nseg, blk, [&](uint32_t s) { return (uint64_t)L[s].blk0; },
                      [&](uint32_t s) { return (uint64_t)L[s].nblk; });
}
__device__ __forceinline__ uint32_t seg_of_bucket(const LevelSeg* L, uint32_t nseg, uint32_t b) {
    return seg_lookup(nseg, b, [&](uint32_t s) { return (uint64_t)L[s].b0; },
                      [&](uint32_t s) { return (uint64_t)L[s].nb; });
}
__device__ __forceinline__ uint32_t seg_of_item(const LevelSeg* L, uint32_t nseg, uint64_t t) {
    return seg_lookup(nseg, t, [&](uint32_t s) { return L[s].src; },
                      [&](uint32_t s) { return L[s].len; });
}

// bucket of key k: the number of splitters <= k (spl sorted, nspl of them;
// top = the largest power of two <= nspl, or 0)
__device__ __forceinline__ uint32_t bucket_of(const uint64_t* spl, uint32_t nspl, uint32_t top,
                                              uint64_t k) {
    uint32_t pos = 0;
    for (uint32_t step = top; step > 0; step >>= 1)
        if (pos + step <= nspl && spl[pos + step - 1] <= k) pos += step;
    return pos;
}

__device__ __forceinline__ uint32_t pow2_floor(uint32_t x) {
    return x ? 1u << (31 - __clz(x)) : 0u;
}

// ------------------------------------------------------------ sampling
struct SampleArgs {
    const LevelSeg* lv0;
    const LevelSeg* lvA;
    const LevelSeg* lvB;
    uint32_t nseg;
    const uint64_t* keys;    // level-B keys
    uint64_t* keysA;         // level-A keys (the sample)
    uint4* recs0;            // level-0 records (the sub-sample)
    uint64_t itemsA, items0;
};

// Sample item j of a segment with S sample items is record floor(j L / S);
// sub-sample item j of U is sample item floor(j S / U).
__global__ void __launch_bounds__(256) sample_kernel(SampleArgs a) {
    const uint64_t total = a.itemsA + a.items0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        if (t < a.itemsA) {
            const uint32_t s = seg_of_item(a.lvA, a.nseg, t);
            const LevelSeg A = a.lvA[s], B = a.lvB[s];
            const uint64_t j = t - A.src;
            a.keysA[t] = __ldg(a.keys + B.src + j * B.len / A.len);
        } else {
            const uint64_t u = t - a.itemsA;
            const uint32_t s = seg_of_item(a.lv0, a.nseg, u);
            const LevelSeg Z = a.lv0[s], A = a.lvA[s], B = a.lvB[s];
            const uint64_t j = u - Z.src;
            const uint64_t i = j * A.len / Z.len;
            const uint64_t k = __ldg(a.keys + B.src + i * B.len / A.len);
            a.recs0[u] = make_uint4((uint32_t)k, (uint32_t)(k >> 32), (uint32_t)j, 0u);
        }
    }
}

// ------------------------------------------------- count, scan, scatter
struct LevelArgs {
    const LevelSeg* segs;
    uint32_t nseg;
    const uint64_t* keys;    // items
    const uint64_t* spl;     // the level's splitters
    uint16_t* bkt;           // bucket of every item
    uint32_t* cnt;           // counts, then their per-bucket prefixes over the blocks
    uint32_t* bucket_off;    // per bucket: first item within the segment
    uint32_t* bucket_cnt;    // per bucket: items
    uint4* recs;             // items in bucket order (key, position in the segment)
};

// one block per tile: the bucket of every item, and the tile's histogram
__global__ void __launch_bounds__(kCThreads) count_kernel(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s = seg_of_block(a.segs, a.nseg, blockIdx.x);
    const LevelSeg L = a.segs[s];
    const uint32_t blk = blockIdx.x - L.blk0;
    const uint32_t nspl = L.nb - 1;
    uint64_t* spl = reinterpret_cast<uint64_t*>(smem);
    uint32_t* hist = reinterpret_cast<uint32_t*>(spl + nspl);
    for (uint32_t i = threadIdx.x; i < nspl; i += kCThreads) spl[i] = __ldg(a.spl + L.spl + i);
    for (uint32_t i = threadIdx.x; i < L.nb; i += kCThreads) hist[i] = 0;
    __syncthreads();
    const uint32_t top = pow2_floor(nspl);
    const uint64_t i0 = (uint64_t)blk * L.tile;
    const uint64_t i1 = min(L.len, i0 + L.tile);
    for (uint64_t i = i0 + threadIdx.x; i < i1; i += kCThreads) {
        const uint32_t b = bucket_of(spl, nspl, top, __ldg(a.keys + L.src + i));
        atomicAdd(&hist[b], 1u);
        a.bkt[L.src + i] = (uint16_t)b;
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < L.nb; b += kCThreads)
        a.cnt[L.cnt0 + (uint64_t)b * L.nblk + blk] = hist[b];
}

// one warp per bucket: exclusive scan of its counts over the blocks (in
// place); the total is the bucket's size
__global__ void __launch_bounds__(256) rowscan_kernel(LevelArgs a, uint32_t nbuckets) {
    const int lane = threadIdx.x & 31;
    const uint32_t row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= nbuckets) return;
    const uint32_t s = seg_of_bucket(a.segs, a.nseg, row);
    const LevelSeg L = a.segs[s];
    uint32_t* r = a.cnt + L.cnt0 + (uint64_t)(row - L.b0) * L.nblk;
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < L.nblk; c0 += 32) {
        const uint32_t c = c0 + (uint32_t)lane;
        const uint32_t v = c < L.nblk ? r[c] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (c < L.nblk) r[c] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) a.bucket_cnt[row] = carry;
}

// one block per segment: exclusive scan of the bucket sizes
__global__ void __launch_bounds__(kCThreads) bucketscan_kernel(LevelArgs a) {
    constexpr int kNW = kCThreads / 32;
    constexpr uint32_t kPer = 8;
    __shared__ uint32_t warp_sums[kNW];
    const LevelSeg L = a.segs[blockIdx.x];
    if (L.nb == 0) return;
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < L.nb; c0 += kCThreads * kPer) {
        const uint32_t b = c0 + threadIdx.x * kPer;
        uint32_t v[kPer], sum = 0;
#pragma unroll
        for (uint32_t j = 0; j < kPer; ++j) {
            v[j] = b + j < L.nb ? a.bucket_cnt[L.b0 + b + j] : 0u;
            sum += v[j];
        }
        uint32_t run = carry + block_exclusive_scan<kNW>(sum, warp_sums);
        const uint32_t chunk = warp_sums[kNW - 1];
#pragma unroll
        for (uint32_t j = 0; j < kPer; ++j) {
            if (b + j < L.nb) a.bucket_off[L.b0 + b + j] = run;
            run += v[j];
        }
        carry += chunk;
        __syncthreads();
    }
}

// the tiles of count_kernel again: every item to the next free slot of its
// bucket (a shared-memory cursor per bucket; order within a bucket is free,
// the local sort fixes it)
__global__ void __launch_bounds__(kCThreads) scatter_kernel(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* cur = reinterpret_cast<uint32_t*>(smem);
    const uint32_t s = seg_of_block(a.segs, a.nseg, blockIdx.x);
    const LevelSeg L = a.segs[s];
    const uint32_t blk = blockIdx.x - L.blk0;
    for (uint32_t b = threadIdx.x; b < L.nb; b += kCThreads)
        cur[b] = __ldg(a.bucket_off + L.b0 + b) + __ldg(a.cnt + L.cnt0 + (uint64_t)b * L.nblk + blk);
    __syncthreads();
    const uint64_t i0 = (uint64_t)blk * L.tile;
    const uint64_t i1 = min(L.len, i0 + L.tile);
    for (uint64_t i = i0 + threadIdx.x; i < i1; i += kCThreads) {
        const uint32_t b = a.bkt[L.src + i];
        const uint64_t k = __ldg(a.keys + L.src + i);
        const uint32_t slot = atomicAdd(&cur[b], 1u);
        a.recs[L.src + slot] = make_uint4((uint32_t)k, (uint32_t)(k >> 32), (uint32_t)(i), 0u);
    }
}

// ----------------------------------------------------------- local sort
struct LocalArgs {
    const LevelSeg* segs;
    uint32_t nseg;
    const uint32_t* bucket_off;   // null: one bucket per segment holding all its items
    const uint32_t* bucket_cnt;
    const uint4* recs;
    const uint64_t* spl;          // the level's splitters (lower bound of an oversize bucket)
    // SPLIT: the next level's splitters are order statistics of this level
    const LevelSeg* next;
    uint64_t* next_spl;
    // MAIN: the sorted lists
    uint64_t* out_hi;
    uint32_t* out_ids;
    const uint64_t* id_base;
    RowKeys rows;
    uint4* fb_list;
    uint32_t* fb_count;
};

struct LocalSmem {
    uint64_t red_lo[kLWarps], red_hi[kLWarps];
    uint32_t warp_sums[kLWarps];
    uint32_t runs[kMaxRuns];
    uint32_t nruns;
    int bad;
};

// Stable pass over n packed words by their 8-bit digit at bit `bit`: warp w
// takes the contiguous records [w per, (w + 1) per), 32 per round; a record's
// rank among the warp's earlier records of its digit comes from ballots and
// the warp's digit counters, and a digit-major scan of the counters places
// every warp's records of a digit after those of the lower digits and of the
// earlier warps.
__device__ __forceinline__ void radix_pass(const uint64_t* src, uint64_t* dst, uint32_t n, int bit,
                                           uint32_t* hist, uint32_t* warp_sums) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t per = (n + kLThreads - 1) / kLThreads * 32;
    const uint32_t base = (uint32_t)warp * per;
    uint32_t* wh = hist + warp * kHistStride;
    for (int i = t; i < kLWarps * kHistStride; i += kLThreads) hist[i] = 0;
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t rank[kMaxRounds];
#pragma unroll
    for (int r = 0; r < kMaxRounds; ++r) {
        if ((uint32_t)r * 32 >= per) break;
        const uint32_t i = base + (uint32_t)r * 32 + (uint32_t)lane;
        const bool valid = i < n;
        const uint32_t d = valid ? (uint32_t)(src[i] >> bit) & 0xFFu : 0u;
        const uint32_t peers = digit_peers(d) & __ballot_sync(0xffffffffu, valid);
        const uint32_t before = wh[d];
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wh[d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // thread t owns digit t / 2 over warps 8 (t % 2) .. 8 (t % 2) + 7
        static_assert(kLWarps == 16 && kLThreads == 512, "two threads per digit");
        const uint32_t d = (uint32_t)t >> 1, w0 = ((uint32_t)t & 1u) * 8;
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] = hist[(w0 + j) * kHistStride + d];
            sum += v[j];
        }
        uint32_t run = block_exclusive_scan<kLWarps>(sum, warp_sums);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hist[(w0 + j) * kHistStride + d] = run;
            run += v[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kMaxRounds; ++r) {
        if ((uint32_t)r * 32 >= per) break;
        const uint32_t i = base + (uint32_t)r * 32 + (uint32_t)lane;
        if (i < n) {
            const uint64_t v = src[i];
            dst[wh[(uint32_t)(v >> bit) & 0xFFu] + rank[r]] = v;
        }
    }
    __syncthreads();
}

// next-level splitter j (1 <= j < nb) is the item of rank floor(j len / nb)
__device__ __forceinline__ void emit_splitter(const LevelSeg& N, uint64_t len, uint64_t r,
                                              uint64_t key, uint64_t* next_spl) {
    if (N.nb < 2) return;
    const uint64_t j = (r * N.nb + len - 1) / len;
    if (j >= 1 && j < N.nb && j * len / N.nb == r) next_spl[N.spl + j - 1] = key;
}

template <bool MAIN>
__global__ void __launch_bounds__(kLThreads, 2) local_sort_kernel(LocalArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* va = reinterpret_cast<uint64_t*>(smem);
    uint64_t* vb = va + kCap;
    uint32_t* hist = reinterpret_cast<uint32_t*>(vb + kCap);
    __shared__ LocalSmem sm;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    const uint32_t gb = blockIdx.x;
    const uint32_t s = seg_of_bucket(a.segs, a.nseg, gb);
    const LevelSeg L = a.segs[s];
    const uint32_t b = gb - L.b0;
    const uint32_t off = a.bucket_off ? __ldg(a.bucket_off + gb) : 0u;
    const uint32_t n = a.bucket_off ? __ldg(a.bucket_cnt + gb) : (uint32_t)L.len;
    if (n == 0) return;
    const uint4* recs = a.recs + L.src + off;

    if (n > kCap) {
        if (MAIN) {
            if (t == 0) a.fb_list[atomicAdd(a.fb_count, 1u)] = make_uint4(s, off, n, 0u);
        } else {
            // too many equal sample keys to sort here: every splitter of the
            // next level in this bucket's ranks takes the bucket's lower
            // bound, so the next level gets one bucket for the whole range
            const uint64_t lower = b ? __ldg(a.spl + L.spl + b - 1) : 0ull;
            const LevelSeg N = a.next[s];
            for (uint32_t i = t; i < n; i += kLThreads)
                emit_splitter(N, L.len, (uint64_t)off + i, lower, a.next_spl);
        }
        return;
    }

    // key range of the bucket
    uint64_t kmin = ~0ull, kmax = 0;
    for (uint32_t i = t; i < n; i += kLThreads) {
        const uint64_t k = rec_key(recs[i]);
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (lane == 0) {
        sm.red_lo[warp] = kmin;
        sm.red_hi[warp] = kmax;
    }
    if (t == 0) {
        sm.nruns = 0;
        sm.bad = 0;
    }
    __syncthreads();
    kmin = sm.red_lo[0];
    kmax = sm.red_hi[0];
    for (int w = 1; w < kLWarps; ++w) {
        kmin = min(kmin, sm.red_lo[w]);
        kmax = max(kmax, sm.red_hi[w]);
    }
    const uint64_t range = kmax - kmin;
    const int rb = range ? 64 - __clzll((long long)range) : 0;   // bits of key - kmin
    const int shift = rb > kKeyBits ? rb - kKeyBits : 0;
    const int D = rb - shift;                                     // bits packed
    int P = (D + 7) / 8;
    if (P >= 3) --P;                  // the lowest 1..8 bits go to the run fix-up
    const int low = D > 8 * P ? D - 8 * P : 0;
    for (uint32_t i = t; i < n; i += kLThreads)
        va[i] = (((rec_key(recs[i]) - kmin) >> shift) << kLiBits) | i;
    __syncthreads();
    uint64_t* src = va;
    uint64_t* dst = vb;
    for (int p = 0; p < P; ++p) {
        radix_pass(src, dst, n, kLiBits + low + 8 * p, hist, sm.warp_sums);
        uint64_t* x = src;
        src = dst;
        dst = x;
    }

    if (MAIN) {
        // runs of equal sorted bits: order by (key, low word, id)
        const int run_bit = kLiBits + low;
        for (uint32_t i = t; i + 1 < n; i += kLThreads) {
            const uint64_t pi = src[i] >> run_bit;
            if ((src[i + 1] >> run_bit) == pi && (i == 0 || (src[i - 1] >> run_bit) != pi)) {
                const uint32_t e = atomicAdd(&sm.nruns, 1u);
                if (e < kMaxRuns) sm.runs[e] = i; else sm.bad = 1;
            }
        }
        __syncthreads();
        const uint32_t nr = min(sm.nruns, kMaxRuns);
        if (!sm.bad) {
            const uint64_t idb = __ldg(a.id_base + s);
            const uint32_t curve = s % a.rows.P.curves;
            for (uint32_t r = warp; r < nr; r += kLWarps) {
                const uint32_t rs = sm.runs[r];
                const uint64_t pre = src[rs] >> run_bit;
                const uint32_t e = rs + (uint32_t)lane;
                const bool in = e < n && (src[e] >> run_bit) == pre;
                const uint32_t inmask = __ballot_sync(0xffffffffu, in);
                const uint32_t len = ~inmask ? (uint32_t)(__ffs(~inmask) - 1) : 32u;
                if (len == 32 && rs + 32 < n && (src[rs + 32] >> run_bit) == pre) {
                    if (lane == 0) sm.bad = 1;
                    continue;
                }
                const bool mine = (uint32_t)lane < len;
                const uint64_t ve = mine ? src[e] : 0ull;
                const uint4 rec = mine ? recs[ve & kLiMask] : make_uint4(0u, 0u, 0u, 0u);
                const uint64_t key = mine ? rec_key(rec) : ~0ull;
                const uint32_t pos = mine ? rec.z : 0xFFFFFFFFu;
                const uint32_t lenmask = len == 32 ? 0xffffffffu : (1u << len) - 1u;
                const uint32_t peers = __match_any_sync(0xffffffffu, key) & lenmask;
                const uint64_t lo = (mine && __popc(peers) > 1)
                                        ? row_key_lo(a.rows.db, a.rows.row_bytes, a.rows.P,
                                                     (uint32_t)(idb + pos), curve)
                                        : 0ull;
                uint32_t rank = 0;
                for (uint32_t u = 0; u < len; ++u) {
                    const uint64_t ku = __shfl_sync(0xffffffffu, key, (int)u);
                    const uint64_t lu = __shfl_sync(0xffffffffu, lo, (int)u);
                    const uint32_t pu = __shfl_sync(0xffffffffu, pos, (int)u);
                    rank += (ku < key || (ku == key && (lu < lo || (lu == lo && pu < pos)))) ? 1u
                                                                                             : 0u;
                }
                __syncwarp();
                if (mine) src[rs + rank] = ve;
                __syncwarp();
            }
        }
        __syncthreads();
        if (sm.bad) {
            if (t == 0) a.fb_list[atomicAdd(a.fb_count, 1u)] = make_uint4(s, off, n, 0u);
            return;
        }
        const uint64_t ob = L.src + off;
        const uint64_t idb = __ldg(a.id_base + s);
        for (uint32_t i = t; i < n; i += kLThreads) {
            const uint4 rec = recs[src[i] & kLiMask];
            a.out_hi[ob + i] = rec_key(rec);
            a.out_ids[ob + i] = (uint32_t)(idb + rec.z);
        }
    } else {
        // splitters of the next level from the sorted keys; a running maximum
        // keeps them non-decreasing where low bits were left unsorted
        const uint32_t per = (n + kLThreads - 1) / kLThreads;
        const uint32_t i0 = min(n, (uint32_t)t * per), i1 = min(n, i0 + per);
        uint64_t m = 0;
        for (uint32_t i = i0; i < i1; ++i) m = max(m, rec_key(recs[src[i] & kLiMask]));
        uint64_t inc = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = max(inc, y);
        }
        if (lane == 31) sm.red_hi[warp] = inc;
        __syncthreads();
        uint64_t run = 0;
        for (int w = 0; w < warp; ++w) run = max(run, sm.red_hi[w]);
        const uint64_t up = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane > 0) run = max(run, up);
        const LevelSeg N = a.next[s];
        for (uint32_t i = i0; i < i1; ++i) {
            run = max(run, rec_key(recs[src[i] & kLiMask]));
            emit_splitter(N, L.len, (uint64_t)off + i, run, a.next_spl);
        }
    }
}

// ------------------------------------------------------------- fallback
struct FallbackArgs {
    const LevelSeg* segs;     // level B
    const uint4* recs;        // level-B records in bucket order
    uint64_t* keys;           // level-B keys (read by nothing after the scatter): two
                              // permutation arrays per listed bucket
    uint64_t* out_hi;         // also holds a listed bucket's low words until its output
    uint32_t* out_ids;
    const uint64_t* id_base;
    RowKeys rows;
    const uint4* fb_list;
    const uint32_t* fb_count;
};

struct FallbackSmem {
    uint32_t hist[256];
    uint32_t wcnt[kFWarps][256];
    uint32_t warp_sums[kFWarps];
    uint64_t red[3][2][kFWarps];
    uint32_t redp[2][kFWarps];
};

// byte `byte` of field f (0: position, 1: low word, 2: high word) of record r
__device__ __forceinline__ uint32_t fb_digit(int f, int byte, uint32_t r, const uint4* recs,
                                             const uint64_t* lo) {
    const uint64_t x = f == 0 ? (uint64_t)recs[r].z : (f == 1 ? lo[r] : rec_key(recs[r]));
    return (uint32_t)(x >> (8 * byte)) & 0xFFu;
}

// Stable pass of one block over the n records of a listed bucket: in (null:
// identity) is the order so far, out the order by the digit.
__device__ void fb_pass(const uint32_t* in, uint32_t* out, uint32_t n, int f, int byte,
                        const uint4* recs, const uint64_t* lo, FallbackSmem& sm) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int i = t; i < 256; i += kFThreads) sm.hist[i] = 0;
    for (int i = t; i < kFWarps * 256; i += kFThreads) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    for (uint32_t i = t; i < n; i += kFThreads)
        atomicAdd(&sm.hist[fb_digit(f, byte, in ? in[i] : i, recs, lo)], 1u);
    __syncthreads();
    {
        const uint32_t v = t < 256 ? sm.hist[t] : 0u;
        const uint32_t ex = block_exclusive_scan<kFWarps>(v, sm.warp_sums);
        if (t < 256) sm.hist[t] = ex;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t c0 = 0; c0 < n; c0 += kFThreads) {
        const uint32_t i = c0 + (uint32_t)t;
        const bool valid = i < n;
        const uint32_t r = valid ? (in ? in[i] : i) : 0u;
        const uint32_t d = valid ? fb_digit(f, byte, r, recs, lo) : 0u;
        const uint32_t peers = digit_peers(d) & __ballot_sync(0xffffffffu, valid);
        if (valid && (peers & lt) == 0) sm.wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (t < 256) {
            uint32_t run = sm.hist[t];
            for (int w = 0; w < kFWarps; ++w) {
                const uint32_t c = sm.wcnt[w][t];
                sm.wcnt[w][t] = run;
                run += c;
            }
            sm.hist[t] = run;
        }
        __syncthreads();
        if (valid) out[sm.wcnt[warp][d] + __popc(peers & lt)] = r;
        __syncthreads();
        for (int j = t; j < kFWarps * 256; j += kFThreads) (&sm.wcnt[0][0])[j] = 0;
        __syncthreads();
    }
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, T* red, Op op) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = op(r, red[w]);
    __syncthreads();
    return r;
}

// One block per listed bucket (grid-stride over the list; with an empty list
// every block returns at once): low words from the rows, then stable 8-bit
// passes over the bytes in which the bucket's records differ -- position,
// then low word, then high word -- so the bucket leaves ordered by
// (high word, low word, id).
__global__ void __launch_bounds__(kFThreads) fallback_kernel(FallbackArgs a) {
    __shared__ FallbackSmem sm;
    const int t = threadIdx.x;
    const uint32_t total = *a.fb_count;
    for (uint32_t e = blockIdx.x; e < total; e += gridDim.x) {
        const uint4 fe = a.fb_list[e];
        const uint32_t s = fe.x, off = fe.y, n = fe.z;
        const LevelSeg L = a.segs[s];
        const uint4* recs = a.recs + L.src + off;
        uint64_t* lo = a.out_hi + L.src + off;
        uint32_t* pa = reinterpret_cast<uint32_t*>(a.keys + L.src + off);
        uint32_t* pb = pa + n;
        const uint64_t idb = __ldg(a.id_base + s);
        const uint32_t curve = s % a.rows.P.curves;
        uint64_t oh = 0, ah = ~0ull, ol = 0, al = ~0ull;
        uint32_t op = 0, ap = ~0u;
        for (uint32_t i = t; i < n; i += kFThreads) {
            const uint4 rec = recs[i];
            const uint64_t k = rec_key(rec);
            const uint64_t l = row_key_lo(a.rows.db, a.rows.row_bytes, a.rows.P,
                                          (uint32_t)(idb + rec.z), curve);
            lo[i] = l;
            oh |= k; ah &= k; ol |= l; al &= l; op |= rec.z; ap &= rec.z;
        }
        auto bor = [](uint64_t x, uint64_t y) { return x | y; };
        auto band = [](uint64_t x, uint64_t y) { return x & y; };
        auto bor32 = [](uint32_t x, uint32_t y) { return x | y; };
        auto band32 = [](uint32_t x, uint32_t y) { return x & y; };
        const uint64_t vary_h = block_reduce(oh, sm.red[0][0], bor) &
                                ~block_reduce(ah, sm.red[0][1], band);
        const uint64_t vary_l = block_reduce(ol, sm.red[1][0], bor) &
                                ~block_reduce(al, sm.red[1][1], band);
        const uint32_t vary_p = block_reduce(op, sm.redp[0], bor32) &
                                ~block_reduce(ap, sm.redp[1], band32);
        const uint32_t* in = nullptr;
        uint32_t* out = pa;
        for (int f = 0; f < 3; ++f) {
            const uint64_t vary = f == 0 ? vary_p : (f == 1 ? vary_l : vary_h);
            for (int byte = 0; byte < (f == 0 ? 4 : 8); ++byte) {
                if (((vary >> (8 * byte)) & 0xFFu) == 0) continue;
                fb_pass(in, out, n, f, byte, recs, lo, sm);
                in = out;
                out = out == pa ? pb : pa;
            }
        }
        for (uint32_t i = t; i < n; i += kFThreads) {
            const uint4 rec = recs[in ? in[i] : i];
            a.out_hi[L.src + off + i] = rec_key(rec);
            a.out_ids[L.src + off + i] = (uint32_t)(idb + rec.z);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------- host plan
uint32_t ceil_div(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

uint32_t buckets_for(uint64_t len) {
    if (len == 0) return 0;
    return std::min<uint32_t>(kMaxBuckets, std::max<uint32_t>(1, ceil_div(len, kTarget)));
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
    uint32_t nseg = 0;
    std::vector<LevelSeg> lv[3];           // level 0, A, B
    uint64_t items[3] = {0, 0, 0};
    uint32_t buckets[3] = {0, 0, 0};
    uint32_t splitters[3] = {0, 0, 0};
    uint32_t blocks[3] = {0, 0, 0};
    uint64_t counts[3] = {0, 0, 0};
    uint32_t max_nb[3] = {0, 0, 0};
    // scratch layout
    size_t off_head = 0, off_splA = 0, off_splB = 0, off_keysA = 0, off_recs0 = 0,
           off_recsA = 0, off_recsB = 0, off_bkt = 0, off_cnt = 0, off_boff = 0, off_bcnt = 0,
           off_fb = 0, bytes = 0;
    size_t head_bytes = 0;                 // fallback counter + the three level tables
};

void fill_level(std::vector<LevelSeg>& lv, const std::vector<uint64_t>& len,
                const std::vector<uint32_t>& nb, uint32_t min_tile, uint64_t* items,
                uint32_t* buckets, uint32_t* splitters, uint32_t* blocks, uint64_t* counts,
                uint32_t* max_nb) {
    uint64_t src = 0, cnt = 0;
    uint32_t b0 = 0, spl = 0, blk0 = 0;
    for (size_t s = 0; s < len.size(); ++s) {
        LevelSeg& L = lv[s];
        L.src = src;
        L.len = len[s];
        L.nb = len[s] ? nb[s] : 0;
        L.spl = spl;
        L.b0 = b0;
        L.nblk = min_tile ? (L.len ? std::min(kMaxBlkPerSeg, ceil_div(L.len, min_tile)) : 0) : 0;
        L.blk0 = blk0;
        L.tile = L.nblk ? ceil_div(L.len, L.nblk) : 0;
        L.cnt0 = cnt;
        src += L.len;
        b0 += L.nb;
        spl += L.nb ? L.nb - 1 : 0;
        blk0 += L.nblk;
        cnt += (uint64_t)L.nb * L.nblk;
        *max_nb = std::max(*max_nb, L.nb);
    }
    *items = src;
    *buckets = b0;
    *splitters = spl;
    *blocks = blk0;
    *counts = cnt;
}

Plan make_plan(const std::vector<uint64_t>& seg_off) {
    Plan p;
    p.nseg = (uint32_t)(seg_off.size() - 1);
    std::vector<uint64_t> lenB(p.nseg), lenA(p.nseg), len0(p.nseg);
    std::vector<uint32_t> nbB(p.nseg), nbA(p.nseg), nb0(p.nseg);
    for (uint32_t s = 0; s < p.nseg; ++s) {
        lenB[s] = seg_off[s + 1] - seg_off[s];
        nbB[s] = buckets_for(lenB[s]);
        lenA[s] = nbB[s] >= 2 ? (uint64_t)kSpb * nbB[s] : 0;   // <= lenB[s]
        nbA[s] = buckets_for(lenA[s]);
        len0[s] = nbA[s] >= 2 ? std::min<uint64_t>((uint64_t)kSpb * nbA[s], kCap) : 0;
        nb0[s] = len0[s] ? 1 : 0;
    }
    for (int l = 0; l < 3; ++l) p.lv[l].resize(p.nseg);
    fill_level(p.lv[0], len0, nb0, 0, &p.items[0], &p.buckets[0], &p.splitters[0], &p.blocks[0],
               &p.counts[0], &p.max_nb[0]);
    fill_level(p.lv[1], lenA, nbA, kMinTileA, &p.items[1], &p.buckets[1], &p.splitters[1],
               &p.blocks[1], &p.counts[1], &p.max_nb[1]);
    fill_level(p.lv[2], lenB, nbB, kMinTileB, &p.items[2], &p.buckets[2], &p.splitters[2],
               &p.blocks[2], &p.counts[2], &p.max_nb[2]);
    // level B's segments start where the caller's segments do
    for (uint32_t s = 0; s < p.nseg; ++s) p.lv[2][s].src = seg_off[s];

    size_t o = 0;
    p.head_bytes = 16 + 3 * sizeof(LevelSeg) * p.nseg;
    p.off_head = o;   o = align_up(o + p.head_bytes);
    p.off_splA = o;   o = align_up(o + 8 * (size_t)std::max<uint32_t>(1, p.splitters[1]));
    p.off_splB = o;   o = align_up(o + 8 * (size_t)std::max<uint32_t>(1, p.splitters[2]));
    p.off_keysA = o;  o = align_up(o + 8 * (size_t)std::max<uint64_t>(1, p.items[1]));
    p.off_recs0 = o;  o = align_up(o + 16 * (size_t)std::max<uint64_t>(1, p.items[0]));
    p.off_recsA = o;  o = align_up(o + 16 * (size_t)std::max<uint64_t>(1, p.items[1]));
    p.off_recsB = o;  o = align_up(o + 16 * (size_t)std::max<uint64_t>(1, p.items[2]));
    p.off_bkt = o;    o = align_up(o + 2 * (size_t)std::max<uint64_t>(1, std::max(p.items[1],
                                                                                   p.items[2])));
    p.off_cnt = o;    o = align_up(o + 4 * (size_t)std::max<uint64_t>(1, std::max(p.counts[1],
                                                                                   p.counts[2])));
    const size_t nbk = (size_t)p.buckets[1] + p.buckets[2] + 1;
    p.off_boff = o;   o = align_up(o + 4 * nbk);
    p.off_bcnt = o;   o = align_up(o + 4 * nbk);
    p.off_fb = o;     o = align_up(o + 16 * (size_t)std::max<uint32_t>(1, p.buckets[2]));
    p.bytes = o;
    return p;
}

constexpr size_t kLocalSmem = 2 * sizeof(uint64_t) * kCap + sizeof(uint32_t) * kLWarps * kHistStride;

cudaError_t set_smem(const void* f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t bucket_sort_scratch_bytes(const std::vector<uint64_t>& seg_off) {
    if (seg_off.size() < 2) return 256;
    return make_plan(seg_off).bytes;
}

int bucket_sort(const BucketSortProblem& bp, void* scratch, cudaStream_t s) {
    if (bp.seg_off.size() < 2) return HC_ERR_ARG;
    const Plan p = make_plan(bp.seg_off);
    if (p.items[2] == 0) return HC_OK;
    if (p.items[2] > 0xFFFFFFFFull) return HC_ERR_ARG;
    char* base = static_cast<char*>(scratch);
    // head: fallback counter (zeroed), then the level tables
    std::vector<uint8_t> head(p.head_bytes, 0);
    for (int l = 0; l < 3; ++l)
        std::memcpy(head.data() + 16 + (size_t)l * sizeof(LevelSeg) * p.nseg, p.lv[l].data(),
                    sizeof(LevelSeg) * p.nseg);
    if (upload_small(base + p.off_head, head.data(), head.size(), s) != cudaSuccess)
        return HC_ERR_CUDA;
    uint32_t* fb_count = reinterpret_cast<uint32_t*>(base + p.off_head);
    const LevelSeg* lv[3];
    for (int l = 0; l < 3; ++l)
        lv[l] = reinterpret_cast<const LevelSeg*>(base + p.off_head + 16 +
                                                   (size_t)l * sizeof(LevelSeg) * p.nseg);
    uint64_t* splA = reinterpret_cast<uint64_t*>(base + p.off_splA);
    uint64_t* splB = reinterpret_cast<uint64_t*>(base + p.off_splB);
    uint64_t* keysA = reinterpret_cast<uint64_t*>(base + p.off_keysA);
    uint4* recs0 = reinterpret_cast<uint4*>(base + p.off_recs0);
    uint4* recsA = reinterpret_cast<uint4*>(base + p.off_recsA);
    uint4* recsB = reinterpret_cast<uint4*>(base + p.off_recsB);
    uint16_t* bkt = reinterpret_cast<uint16_t*>(base + p.off_bkt);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(base + p.off_cnt);
    uint32_t* boff = reinterpret_cast<uint32_t*>(base + p.off_boff);
    uint32_t* bcnt = reinterpret_cast<uint32_t*>(base + p.off_bcnt);
    uint4* fb_list = reinterpret_cast<uint4*>(base + p.off_fb);

    if (set_smem(reinterpret_cast<const void*>(local_sort_kernel<true>), kLocalSmem) ||
        set_smem(reinterpret_cast<const void*>(local_sort_kernel<false>), kLocalSmem))
        return HC_ERR_CUDA;
    const size_t count_smem = 12 * (size_t)std::max(p.max_nb[1], p.max_nb[2]);
    if (count_smem > 48 * 1024 &&
        set_smem(reinterpret_cast<const void*>(count_kernel), count_smem))
        return HC_ERR_CUDA;
    const size_t scatter_smem = 4 * (size_t)std::max(p.max_nb[1], p.max_nb[2]);
    if (scatter_smem > 48 * 1024 &&
        set_smem(reinterpret_cast<const void*>(scatter_kernel), scatter_smem))
        return HC_ERR_CUDA;

    auto launched = [](int n) {
        count_launches((uint64_t)n);
        return cudaGetLastError() == cudaSuccess;
    };

    // splitters of level A (sub-sample) and level B (sample)
    if (p.items[1] > 0) {
        SampleArgs sa{lv[0], lv[1], lv[2], p.nseg, bp.keys, keysA, recs0, p.items[1], p.items[0]};
        const uint64_t work = p.items[1] + p.items[0];
        sample_kernel<<<(unsigned)std::min<uint64_t>((work + 255) / 256, 152 * 8), 256, 0, s>>>(sa);
        if (!launched(1)) return HC_ERR_CUDA;
        if (p.buckets[0] > 0) {
            LocalArgs la{};
            la.segs = lv[0];
            la.nseg = p.nseg;
            la.recs = recs0;
            la.next = lv[1];
            la.next_spl = splA;
            local_sort_kernel<false><<<p.buckets[0], kLThreads, kLocalSmem, s>>>(la);
            if (!launched(1)) return HC_ERR_CUDA;
        }
    }
    // levels A and B: count, scan, scatter, local sort
    for (int l = 1; l <= 2; ++l) {
        if (p.items[l] == 0) continue;
        LevelArgs a{lv[l], p.nseg, l == 1 ? keysA : bp.keys, l == 1 ? splA : splB, bkt, cnt,
                    boff + (l == 2 ? p.buckets[1] : 0), bcnt + (l == 2 ? p.buckets[1] : 0),
                    l == 1 ? recsA : recsB};
        const size_t csm = 12 * (size_t)p.max_nb[l];
        count_kernel<<<p.blocks[l], kCThreads, csm, s>>>(a);
        rowscan_kernel<<<(p.buckets[l] + 7) / 8, 256, 0, s>>>(a, p.buckets[l]);
        bucketscan_kernel<<<p.nseg, kCThreads, 0, s>>>(a);
        scatter_kernel<<<p.blocks[l], kCThreads, 4 * (size_t)p.max_nb[l], s>>>(a);
        if (!launched(4)) return HC_ERR_CUDA;
        LocalArgs la{};
        la.segs = lv[l];
        la.nseg = p.nseg;
        la.bucket_off = a.bucket_off;
        la.bucket_cnt = a.bucket_cnt;
        la.recs = a.recs;
        la.spl = a.spl;
        if (l == 1) {
            la.next = lv[2];
            la.next_spl = splB;
            local_sort_kernel<false><<<p.buckets[1], kLThreads, kLocalSmem, s>>>(la);
        } else {
            la.out_hi = bp.out_hi;
            la.out_ids = bp.out_ids;
            la.id_base = bp.id_base_dev;
            la.rows = bp.rows;
            la.fb_list = fb_list;
            la.fb_count = fb_count;
            local_sort_kernel<true><<<p.buckets[2], kLThreads, kLocalSmem, s>>>(la);
        }
        if (!launched(1)) return HC_ERR_CUDA;
    }
    FallbackArgs fa{lv[2], recsB, bp.keys, bp.out_hi, bp.out_ids, bp.id_base_dev, bp.rows,
                    fb_list, fb_count};
    fallback_kernel<<<std::min<uint32_t>(p.buckets[2], 256), kFThreads, 0, s>>>(fa);
    if (!launched(1)) return HC_ERR_CUDA;
    return HC_OK;
}

}  // namespace hc
