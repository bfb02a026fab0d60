// K2: stable LSD radix sort of (128-bit key, id) records within segments --
// the "insert <key, b> into the sorted list" of Algorithm 1, done in bulk.
//
// Digits are 8 bits, least significant first (digit t covers key bits
// 8t..8t+7).  Each pass moves only the 64-bit key word that holds the digit
// plus a 32-bit record position (12 bytes), not the whole 20-byte record:
//   - passes over the low word carry (lo, position);
//   - the high words are then gathered by position and the passes over the
//     high word carry (hi, position);
//   - at the end the low words and ids are gathered by the final positions.
// Digits above key_bits are zero by contract and are skipped.
//
// The high-word-first path sorts only the top bytes of the high word (hi_skip
// low bytes left out) and a fix-up orders the short runs of equal prefixes by
// (high word, low word, id).  For an index with affine ids and no stored low
// words (hc_build) the last pass writes the final high words and ids and the
// fix-up works in place and on the device alone: find_runs orders the short
// runs inside 32-record chunks and lists the others, sort_runs orders each
// listed run of at most 8 records with one lane and of at most 32 with one
// warp, sort_mid_runs each run of up to 256 with one warp in shared memory,
// and long_run_kernel the longer ones with one block each through global
// memory.  Otherwise (low words stored, ids gathered) the
// path is taken only when the caller may wait once on the stream: a run
// longer than 32 then sends it back to sort by every byte.
//
// Per pass, three kernels, none of which waits on another block:
//   hist    one 4096-record tile per block: digit counts -> counts[seg][digit][tile]
//   scan    one block per (segment, digit): exclusive scan over the tiles
//   scatter one tile per block: stable in-tile ranking (warp-level multisplit
//           by ballots plus per-warp digit counts), a shared-memory reorder
//           by digit, then coalesced runs to global memory.
#include <algorithm>
#include <cstring>

#include "hc_block.cuh"
#include "hc_internal.h"

namespace hc {

namespace {

constexpr int kThreads = 256;                 // histogram / scan / gather blocks
constexpr int kTile = 4096;                    // records per tile
// scatter blocks: 16 warps of 256 consecutive records each (8 rounds of 32)
constexpr int kSThreads = 512;
constexpr int kSWarps = kSThreads / 32;
constexpr int kIpt = kTile / kSThreads;        // 8 records per thread
constexpr int kWarpItems = kTile / kSWarps;    // 256 consecutive records per warp

struct SegInfo {
    uint64_t start;     // first record
    uint64_t len;       // records
    uint64_t cnt_base;  // offset of the segment's counts block (256 x ntiles)
    uint32_t ntiles;
    uint32_t tile0;     // first global tile of the segment
};

// Final step: the low key words by the final positions, and the ids either by
// the same gather or, when the ids are an affine function of the record
// position (id = id_base[seg] + position - seg start, as hc_build lays them
// out), computed without touching memory.
struct FinalIds {
    const uint32_t* ids;        // gathered when id_base is null
    const uint64_t* id_base;    // device, one per segment, or null
};

// segment of global tile t: the last segment whose first tile is <= t
// (segments without tiles share tile0 with the next one and are skipped)
__device__ __forceinline__ uint32_t seg_of_tile(const SegInfo* segs, uint32_t nseg, uint32_t t) {
    uint32_t lo = 0, hi = nseg;  // invariant: answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (segs[mid].tile0 <= t) lo = mid; else hi = mid;
    }
    while (segs[lo].ntiles == 0 || segs[lo].tile0 + segs[lo].ntiles <= t) ++lo;
    return lo;
}

__device__ __forceinline__ void tile_of(uint32_t nseg, const SegInfo* segs, SegInfo& si,
                                        uint32_t& seg, uint32_t& lt, uint64_t& start,
                                        uint32_t& count) {
    const uint32_t t = blockIdx.x;
    seg = seg_of_tile(segs, nseg, t);
    si = segs[seg];
    lt = t - si.tile0;
    start = si.start + (uint64_t)lt * kTile;
    const uint64_t left = si.len - (uint64_t)lt * kTile;
    count = (uint32_t)(left < (uint64_t)kTile ? left : (uint64_t)kTile);
}

// digits (null: read the words): this pass's digit of every record, one byte
// each, written by the previous pass's scatter
__global__ void __launch_bounds__(kThreads) hist_kernel(const uint64_t* __restrict__ words,
                                                        const uint8_t* __restrict__ digits,
                                                        int shift, uint32_t nseg,
                                                        const SegInfo* __restrict__ segs,
                                                        uint32_t* __restrict__ counts) {
    __shared__ uint32_t h[256];
    SegInfo si;
    uint32_t seg, lt, count;
    uint64_t start;
    tile_of(nseg, segs, si, seg, lt, start, count);
    h[threadIdx.x] = 0;
    __syncthreads();
    if (digits) {
        const uint8_t* dg = digits + start;
        // sixteen digits per 16-byte load where the tile starts aligned (one
        // load per thread for a whole tile), the rest one byte at a time
        uint32_t i0 = 0;
        if ((reinterpret_cast<uintptr_t>(dg) & 15u) == 0) {
            const uint32_t nv = count / 16;
            const uint4* dv = reinterpret_cast<const uint4*>(dg);
            for (uint32_t v = threadIdx.x; v < nv; v += kThreads) {
                const uint4 x = __ldg(dv + v);
                const uint32_t q[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int b = 0; b < 4; ++b) atomicAdd(&h[(q[j] >> (8 * b)) & 0xFFu], 1u);
            }
            i0 = nv * 16;
        }
        for (uint32_t i = i0 + threadIdx.x; i < count; i += kThreads)
            atomicAdd(&h[__ldg(dg + i)], 1u);
    } else {
        const uint64_t* w = words + start;
        if (count == (uint32_t)kTile) {
            // a whole tile: all sixteen loads of a thread in flight at once
            constexpr int kPer = kTile / kThreads;
            uint64_t x[kPer];
#pragma unroll
            for (int r = 0; r < kPer; ++r) x[r] = __ldg(w + threadIdx.x + r * kThreads);
#pragma unroll
            for (int r = 0; r < kPer; ++r) atomicAdd(&h[(uint32_t)(x[r] >> shift) & 0xFFu], 1u);
        } else {
            for (uint32_t i = threadIdx.x; i < count; i += kThreads)
                atomicAdd(&h[(uint32_t)(__ldg(w + i) >> shift) & 0xFFu], 1u);
        }
    }
    __syncthreads();
    counts[si.cnt_base + (uint64_t)threadIdx.x * si.ntiles + lt] = h[threadIdx.x];
}

// grid (256 digits, segments): exclusive scan of one digit row over the tiles.
// Small blocks (sixteen resident per SM) walk the row in
// chunks of kScanPer consecutive tiles per thread, every load of a chunk in
// flight, with the running total carried from chunk to chunk.
constexpr int kScanThreads = 128;
constexpr int kScanPer = 8;

__global__ void __launch_bounds__(kScanThreads, 16) scan_kernel(const SegInfo* __restrict__ segs,
                                                                uint32_t* __restrict__ counts,
                                                                uint32_t* __restrict__ totals) {
    constexpr int kNW = kScanThreads / 32;
    __shared__ uint32_t warp_sums[kNW];
    const SegInfo si = segs[blockIdx.y];
    const uint32_t digit = blockIdx.x;
    uint32_t* row = counts + si.cnt_base + (uint64_t)digit * si.ntiles;
    const uint32_t T = si.ntiles;
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < T; c0 += (uint32_t)(kScanThreads * kScanPer)) {
        const uint32_t b = c0 + threadIdx.x * kScanPer;
        uint32_t v[kScanPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            v[j] = b + j < T ? row[b + j] : 0u;
            sum += v[j];
        }
        uint32_t run = carry + block_exclusive_scan<kNW>(sum, warp_sums);
        const uint32_t chunk_total = warp_sums[kNW - 1];   // inclusive total of the last warp
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            if (b + j < T) row[b + j] = run;
            run += v[j];
        }
        carry += chunk_total;
        __syncthreads();   // the next chunk's scan rewrites warp_sums
    }
    if (threadIdx.x == 0) totals[(uint64_t)blockIdx.y * 256 + digit] = carry;
}

// One scatter tile in shared memory: the words and positions of the tile in
// digit order (padded against bank conflicts on the striped read-out), the
// per-warp digit counts (then their digit-major exclusive prefixes), and the
// global destination base per digit.
constexpr int kPadW = kTile + kTile / 16;   // one spare word slot per 16
constexpr int kPadP = kTile + kTile / 32;   // one spare position slot per 32
constexpr int kHistStride = 257;            // warps' count rows, odd stride
__device__ __forceinline__ int padw(int i) { return i + (i >> 4); }
__device__ __forceinline__ int padp(int i) { return i + (i >> 5); }

struct ScatterSmem {
    uint64_t w[kPadW];
    uint32_t p[kPadP];
    uint32_t hist[kSWarps * kHistStride];   // [warp][digit]
    uint64_t gbase[256];
    uint32_t warp_sums[kSWarps];
};

// Tile ranking: warp w owns records [256 w, 256 w + 256), lane l of round r
// holds record 256 w + 32 r + l (coalesced loads).  Each round ranks its 32
// records among the warp's earlier records of the same digit (ballot peers +
// the warp's running digit counts); the digit-major scan of the 16 x 256
// counts then gives every record its place in the digit-sorted tile, stable
// in record order.  Records past the tile's end carry digit 255 and sort last.
// id_base (final pass of an affine-id sort, else null): the carried
// positions leave as ids, id = id_base[seg] + position - segment start.
// next_digit (null: none): the next pass's digit of every record, one byte
// each at its destination, so the next histogram reads bytes, not words.
__global__ void __launch_bounds__(kSThreads, 2) scatter_kernel(
    const uint64_t* __restrict__ wsrc, const uint32_t* __restrict__ psrc,
    uint64_t* __restrict__ wdst, uint32_t* __restrict__ pdst, int shift, uint32_t nseg,
    const SegInfo* __restrict__ segs, const uint32_t* __restrict__ counts,
    const uint32_t* __restrict__ totals, const uint64_t* __restrict__ id_base,
    uint8_t* __restrict__ next_digit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem& sm = *reinterpret_cast<ScatterSmem*>(smem_raw);

    SegInfo si;
    uint32_t seg, lt, count;
    uint64_t start;
    tile_of(nseg, segs, si, seg, lt, start, count);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    uint64_t w[kIpt];
    uint32_t p[kIpt];
#pragma unroll
    for (int r = 0; r < kIpt; ++r) {
        const uint32_t i = (uint32_t)warp * kWarpItems + (uint32_t)r * 32 + (uint32_t)lane;
        const bool valid = i < count;
        w[r] = valid ? __ldg(wsrc + start + i) : (0xFFull << shift);
        p[r] = valid ? (psrc ? __ldg(psrc + start + i) : (uint32_t)(start + i)) : 0u;
    }
    for (int i = t; i < kSWarps * kHistStride; i += kSThreads) sm.hist[i] = 0;
    __syncthreads();

    uint32_t* wh = sm.hist + warp * kHistStride;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t rank[kIpt];
#pragma unroll
    for (int r = 0; r < kIpt; ++r) {
        const uint32_t d = (uint32_t)(w[r] >> shift) & 0xFFu;
        const uint32_t peers = digit_peers(d);
        const uint32_t before = wh[d];
        rank[r] = before + __popc(peers & lt_mask);
        __syncwarp();
        if ((peers & lt_mask) == 0) wh[d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();

    // digit-major exclusive scan of hist[warp][digit]: thread t owns digit
    // t / tpd, warps 8 (t % tpd) .. 8 (t % tpd) + 7 (tpd = threads per digit)
    {
        constexpr uint32_t tpd = kSThreads / 256;
        static_assert(kSWarps == 8 * tpd, "eight warps per thread slot");
        const uint32_t d = (uint32_t)t / tpd, w0 = ((uint32_t)t % tpd) * 8;
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] = sm.hist[(w0 + j) * kHistStride + d];
            sum += v[j];
        }
        uint32_t run = block_exclusive_scan<kSWarps>(sum, sm.warp_sums);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sm.hist[(w0 + j) * kHistStride + d] = run;
            run += v[j];
        }
    }
    {
        // global destination of sorted-tile slot i with digit d: gbase[d] + i
        const uint32_t dg = t;
        const bool own = dg < 256;
        const uint32_t seg_prefix = block_exclusive_scan<kSWarps>(
            own ? __ldg(totals + (uint64_t)seg * 256 + dg) : 0u, sm.warp_sums);
        if (own) {
            const uint32_t before = __ldg(counts + si.cnt_base + (uint64_t)dg * si.ntiles + lt);
            sm.gbase[dg] = si.start + seg_prefix + before - sm.hist[dg];
        }
    }
#pragma unroll
    for (int r = 0; r < kIpt; ++r) {
        const uint32_t d = (uint32_t)(w[r] >> shift) & 0xFFu;
        const uint32_t slot = wh[d] + rank[r];
        sm.w[padw(slot)] = w[r];
        sm.p[padp(slot)] = p[r];
    }
    __syncthreads();
    const uint32_t idoff = id_base ? (uint32_t)(__ldg(id_base + seg) - si.start) : 0u;
    for (uint32_t i = t; i < count; i += kSThreads) {
        const uint64_t v = sm.w[padw(i)];
        const uint64_t g = sm.gbase[(uint32_t)(v >> shift) & 0xFFu] + i;
        if (!HC_IN_BOUNDS(kSiteScatter, g - si.start, si.len)) continue;
        wdst[g] = v;
        pdst[g] = sm.p[padp(i)] + idoff;
        if (next_digit) next_digit[g] = (uint8_t)(v >> (shift + 8));
    }
}

// the segment table from the device offsets (one thread: nseg is small)
__global__ void seg_setup_kernel(const uint64_t* __restrict__ seg_off, uint32_t nseg,
                                 SegInfo* __restrict__ segs) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t tiles = 0;
    uint64_t cnt = 0;
    for (uint32_t s = 0; s < nseg; ++s) {
        SegInfo si;
        si.start = seg_off[s];
        si.len = seg_off[s + 1] - seg_off[s];
        si.ntiles = (uint32_t)((si.len + kTile - 1) / kTile);
        si.tile0 = tiles;
        si.cnt_base = cnt;
        cnt += 256ull * si.ntiles;
        tiles += si.ntiles;
        segs[s] = si;
    }
}

// dst[i] = src[pos[i]] (pos == nullptr: identity)
__global__ void __launch_bounds__(256) gather_words_kernel(const uint64_t* __restrict__ src,
                                                           const uint32_t* __restrict__ pos,
                                                           uint64_t* __restrict__ dst,
                                                           uint64_t total) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
        dst[i] = __ldg(src + (pos ? __ldg(pos + i) : i));
}

// one tile per block, so the block knows its segment
__global__ void __launch_bounds__(256) gather_final_kernel(
    const uint64_t* __restrict__ lo, FinalIds fid, const uint32_t* __restrict__ pos,
    uint64_t* __restrict__ out_lo, uint32_t* __restrict__ out_ids, uint32_t nseg,
    const SegInfo* __restrict__ segs) {
    SegInfo si;
    uint32_t seg, lt, count;
    uint64_t start;
    tile_of(nseg, segs, si, seg, lt, start, count);
    const uint64_t base = fid.id_base ? __ldg(fid.id_base + seg) - si.start : 0;
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) {
        const uint32_t p = pos ? __ldg(pos + start + i) : (uint32_t)(start + i);
        out_lo[start + i] = __ldg(lo + p);
        out_ids[start + i] = fid.id_base ? (uint32_t)(base + p) : __ldg(fid.ids + p);
    }
}

// After sorting by the high word's top bytes alone (records with equal
// prefixes w >> run_shift stay in position order), runs of equal prefixes
// must end ordered by (high word, low word, position).  One tile per block: a
// record outside any run is written in place; a record in a run of at most
// kMaxRun finds the run's bounds, ranks itself among the run's records and is
// written at run start + rank.  A longer run sets *long_run, and the caller
// redoes the sort with every digit.  The low words and ids are gathered here.
constexpr uint32_t kMaxRun = 32;

// lo == nullptr: low words are recomputed from the rows (affine ids) when
// two records of a run have equal high words, and out_lo is not written.
__global__ void __launch_bounds__(256) fixup_final_kernel(
    const uint64_t* __restrict__ w, int run_shift, const uint32_t* __restrict__ pos,
    const uint64_t* __restrict__ lo, RowKeys rows, FinalIds fid, uint64_t* __restrict__ out_hi,
    uint64_t* __restrict__ out_lo, uint32_t* __restrict__ out_ids, uint32_t nseg,
    const SegInfo* __restrict__ segs, uint32_t* __restrict__ long_run) {
    SegInfo si;
    uint32_t seg, lt, count;
    uint64_t start;
    tile_of(nseg, segs, si, seg, lt, start, count);
    const uint64_t id_base = fid.id_base ? __ldg(fid.id_base + seg) - si.start : 0;
    const uint64_t seg_end = si.start + si.len;
    const uint32_t curve = lo ? 0u : seg % rows.P.curves;
    for (uint32_t t = threadIdx.x; t < count; t += blockDim.x) {
        const uint64_t i = start + t;
        const uint64_t wi = __ldg(w + i);
        const uint64_t key = wi >> run_shift;
        const uint32_t pi = __ldg(pos + i);
        uint64_t li = lo ? __ldg(lo + pi) : 0;
        bool li_ok = lo != nullptr;
        const uint32_t idi = fid.id_base ? (uint32_t)(id_base + pi) : __ldg(fid.ids + pi);
        const bool prev_eq = i > si.start && (__ldg(w + i - 1) >> run_shift) == key;
        const bool next_eq = i + 1 < seg_end && (__ldg(w + i + 1) >> run_shift) == key;
        uint64_t dst = i;
        if (prev_eq || next_eq) {
            uint64_t rs = i, re = i + 1;
            while (rs > si.start && i - rs <= kMaxRun && (__ldg(w + rs - 1) >> run_shift) == key)
                --rs;
            while (re < seg_end && re - i <= kMaxRun && (__ldg(w + re) >> run_shift) == key) ++re;
            if (re - rs > kMaxRun) {
                atomicOr(long_run, 1u);
            } else {
                uint32_t rank = 0;
                for (uint64_t j = rs; j < re; ++j) {
                    if (j == i) continue;
                    const uint64_t wj = __ldg(w + j);
                    const uint32_t pj = __ldg(pos + j);
                    bool before = wj < wi;
                    if (wj == wi) {
                        if (!li_ok) {
                            li = row_key_lo(rows.db, rows.row_bytes, rows.P, idi, curve);
                            li_ok = true;
                        }
                        const uint64_t lj =
                            lo ? __ldg(lo + pj)
                               : row_key_lo(rows.db, rows.row_bytes, rows.P,
                                            (uint32_t)(id_base + pj), curve);
                        before = lj < li || (lj == li && pj < pi);
                    }
                    rank += before ? 1u : 0u;
                }
                dst = rs + rank;
            }
        }
        out_hi[dst] = wi;
        if (out_lo) out_lo[dst] = li;
        out_ids[dst] = idi;
    }
}

// In-place fix-up after a sort whose last pass wrote the final high words
// and ids (affine ids, low words recomputed from rows).  Runs of equal
// prefixes hi >> run_shift (ordered by id, i.e. by position) must end
// ordered by (hi, low word, id).  Four kernels, each reading what the one
// before it listed:
//   find_runs      streams the high words and ids and orders the short runs
//                  inside each 32-record chunk (below), listing the others;
//   sort_runs      listed runs: a lane per run of at most kLaneRun records
//                  without equal high words, otherwise a warp per run of at
//                  most kMaxRun = 32 (one record per lane: lanes whose high
//                  words tie compute their low words, every lane counts the
//                  run's records below its own, all write after all read),
//                  listing longer ones;
//   sort_mid_runs  a warp per run of at most kMidRun, ranked in shared memory;
//   long_run       a block per longer run.
// A reader past its run's end sees only prefixes, which a permutation inside
// another run leaves unchanged, so the in-place writes race with nothing.
constexpr int kFindWarps = 8;
constexpr int kFindChunks = kTile / 32 / kFindWarps;   // 16 chunks of 32 records per warp
constexpr int kFindBatch = 4;                          // chunks loaded at once
constexpr int kLaneRun = 8;   // runs ordered inside find_runs: at most this long

// find_runs: one tile per block, each warp four 32-record chunks at a time.
// A run (records with equal prefixes hi >> run_shift) of at most kLaneRun
// records that lies inside one chunk and has no two equal high words is
// ordered right there: its records share the prefix, so each lane counts the
// run's records whose low run_shift bits are below its own (32-bit shuffles)
// and writes itself at run start + rank.  Every other run (longer, crossing a
// chunk's edge, or with equal high words, which need the low words) has its
// start listed for sort_runs.  A run's records are permuted among the run's
// own positions, so the prefix at every position -- all that neighbouring
// chunks read here -- never changes.  run_shift <= 32.  For the same reason
// the fence (nullable; only when kFenceMask clears the run_shift low bits) is
// final here: fence[i / 16] = hi[i] & kFenceMask for every position i that is
// a multiple of 16.
template <int SHIFT>
__global__ void __launch_bounds__(kFindWarps * 32) find_runs_kernel(
    uint64_t* __restrict__ hi, uint32_t* __restrict__ ids, uint32_t nseg,
    const SegInfo* __restrict__ segs, uint64_t* __restrict__ run_pos,
    uint32_t* __restrict__ run_seg, unsigned long long* __restrict__ nruns,
    uint64_t* __restrict__ fence) {
    static_assert(kFindChunks % kFindBatch == 0, "whole batches");
    static_assert(SHIFT > 0 && SHIFT <= 32, "low bits in a 32-bit word");
    __shared__ uint32_t masks[kFindWarps][kFindChunks];
    __shared__ uint32_t wbase[kFindWarps];
    __shared__ unsigned long long bbase;
    SegInfo si;
    uint32_t seg, lt, count;
    uint64_t start;
    tile_of(nseg, segs, si, seg, lt, start, count);
    const int lane = threadIdx.x & 31;
    const uint32_t warp = threadIdx.x >> 5;
    constexpr uint32_t low_mask = SHIFT >= 32 ? 0xFFFFFFFFu : (1u << SHIFT) - 1u;
    // the segment goes on before this tile / after its last record
    const bool tile_after = lt + 1 < si.ntiles;
    uint32_t found = 0;
    // fence words of the warp's 32 x 16 records: word l (lane l) is the high
    // word at wbeg + a0 + 16 l, the l-th position of the warp that is a
    // multiple of 16; chunk c holds words 2c and 2c + 1 at its offsets a0 and
    // a0 + 16
    const uint64_t wbeg = start + (uint64_t)warp * kFindChunks * 32;
    const uint32_t a0 = (uint32_t)((16 - (wbeg & 15)) & 15);
    uint64_t fw = 0;
    for (int c0 = 0; c0 < kFindChunks; c0 += kFindBatch) {
        // a chunk's words and ids, plus the word before it (lane 0) or after
        // it (lane 31)
        uint64_t hv[kFindBatch], halo[kFindBatch];
        uint32_t dv[kFindBatch];
#pragma unroll
        for (int j = 0; j < kFindBatch; ++j) {
            const uint32_t off = (warp * kFindChunks + (uint32_t)(c0 + j)) * 32 + (uint32_t)lane;
            const uint64_t i = start + off;
            const bool ok = off < count;
            hv[j] = ok ? __ldg(hi + i) : 0;
            dv[j] = ok ? __ldg(ids + i) : 0u;
            uint64_t h = 0;
            if (ok && lane == 0 && (lt > 0 || off > 0)) h = hi[i - 1];
            if (ok && lane == 31 && (off + 1 < count || tile_after)) h = hi[i + 1];
            halo[j] = h;
        }
        if (fence) {
#pragma unroll
            for (int j = 0; j < kFindBatch; ++j) {
                const uint32_t c = (uint32_t)(c0 + j);
                const uint64_t f0 = __shfl_sync(0xffffffffu, hv[j], (int)a0);
                const uint64_t f1 = __shfl_sync(0xffffffffu, hv[j], (int)a0 + 16);
                if ((uint32_t)lane == 2 * c) fw = f0;
                if ((uint32_t)lane == 2 * c + 1) fw = f1;
            }
        }
#pragma unroll
        for (int j = 0; j < kFindBatch; ++j) {
            const uint32_t base = (warp * kFindChunks + (uint32_t)(c0 + j)) * 32;
            const uint32_t off = base + (uint32_t)lane;
            const bool ok = off < count;
            const uint64_t w = hv[j];
            // every lane takes part in both shuffles; the end lanes then use their halo
            const uint64_t up = __shfl_up_sync(0xffffffffu, w, 1);
            const uint64_t dn = __shfl_down_sync(0xffffffffu, w, 1);
            const uint64_t prev = lane == 0 ? halo[j] : up;
            const uint64_t next = lane == 31 ? halo[j] : dn;
            // run goes on before / after this record (equal prefixes w >> SHIFT)
            const bool ps = ok && (lt > 0 || off > 0) && ((prev ^ w) >> SHIFT) == 0;
            const bool ns = ok && (off + 1 < count || tile_after) && ((next ^ w) >> SHIFT) == 0;
            const uint32_t brk = __ballot_sync(0xffffffffu, !ps);
            const uint32_t ends = __ballot_sync(0xffffffffu, !ns);
            uint32_t listed = 0;
            if ((brk & ends) != 0xffffffffu) {
                // this lane's run inside the chunk: lanes s..e (cut at the chunk's edges)
                const uint32_t below = brk & (0xFFFFFFFFu >> (31 - lane));
                const uint32_t above = ends >> lane;
                const bool cut = below == 0 || above == 0;   // the run crosses an edge
                const int s = below ? 31 - __clz(below) : 0;
                const int e = above ? lane + __ffs(above) - 1 : 31;
                const bool in_run = ps || ns;
                const uint32_t lw = (uint32_t)w & low_mask;
                uint32_t rank = 0;
                bool tie = false;
                // offsets up to the chunk's longest run that can be ordered here
                const int len0 = e - s + 1;
                const int reach = __reduce_max_sync(
                    0xffffffffu, (in_run && !cut && len0 <= kLaneRun) ? (uint32_t)len0 : 1u);
                for (int o = 1; o < reach; ++o) {
                    const uint32_t lu = __shfl_up_sync(0xffffffffu, lw, o);
                    const uint32_t ld = __shfl_down_sync(0xffffffffu, lw, o);
                    if (lane - o >= s) {
                        rank += lu < lw ? 1u : 0u;
                        tie |= lu == lw;
                    }
                    if (lane + o <= e) {
                        rank += ld < lw ? 1u : 0u;
                        tie |= ld == lw;
                    }
                }
                const int len = e - s + 1;
                const bool short_run = in_run && !cut && len <= kLaneRun;
                const uint32_t ties = __ballot_sync(0xffffffffu, short_run && tie);
                const bool run_tie = short_run && ((ties >> s) & ((1u << len) - 1u)) != 0;
                const bool here = short_run && !run_tie;
                // the run's true start lane lists a run not ordered here
                listed = __ballot_sync(0xffffffffu, in_run && !ps && !here);
                if (here && rank != (uint32_t)(lane - s)) {
                    const uint64_t dst = start + base + (uint32_t)s + rank;
                    hi[dst] = w;
                    ids[dst] = dv[j];
                }
            }
            if (lane == 0) masks[warp][c0 + j] = listed;
            found += (uint32_t)__popc(listed);
        }
    }
    if (fence) {
        // one coalesced store of the warp's fence words
        const uint64_t fpos = wbeg + a0 + 16 * (uint64_t)lane;
        if (fpos < start + count) fence[fpos >> kFenceShift] = fw & kFenceMask;
    }
    if (lane == 0) wbase[warp] = found;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t total = 0;
        for (int w = 0; w < kFindWarps; ++w) {
            const uint32_t c = wbase[w];
            wbase[w] = total;
            total += c;
        }
        bbase = total ? atomicAdd(nruns, (unsigned long long)total) : 0ull;
    }
    __syncthreads();
    uint64_t slot = bbase + wbase[warp];
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int c = 0; c < kFindChunks; ++c) {
        const uint32_t m = masks[warp][c];
        if ((m >> lane) & 1u) {
            const uint64_t r = slot + (uint32_t)__popc(m & lt_mask);
            if (HC_IN_BOUNDS(kSiteRunList, r,
                             (segs[nseg - 1].start + segs[nseg - 1].len) / 2)) {
                run_pos[r] = start + (warp * kFindChunks + (uint32_t)c) * 32 + (uint32_t)lane;
                run_seg[r] = seg;
            }
        }
        slot += (uint32_t)__popc(m);
    }
}

// One listed run by the whole warp, one record per lane: a run longer than
// kMaxRun goes to the long list; otherwise lanes whose high words tie compute
// their low words, every lane counts the run's records below its own, and
// all lanes write after all have read.
__device__ __forceinline__ void warp_sort_run(uint64_t* hi, uint32_t* ids, int run_shift,
                                              const RowKeys& rows, const SegInfo* segs,
                                              uint64_t rs, uint32_t seg, uint4* long_list,
                                              uint32_t* long_count, uint32_t long_cap,
                                              int lane) {
    const uint64_t seg_end = segs[seg].start + segs[seg].len;
    const uint32_t curve = seg % rows.P.curves;
    const uint64_t e = rs + lane;
    const bool inseg = e < seg_end;
    const uint64_t he = inseg ? hi[e] : ~0ull;
    const uint32_t de = inseg ? ids[e] : 0xFFFFFFFFu;
    const uint64_t rkey = __shfl_sync(0xffffffffu, he, 0) >> run_shift;
    const bool in = inseg && (he >> run_shift) == rkey;
    const uint32_t inmask = __ballot_sync(0xffffffffu, in);
    const uint32_t len = __ffs(~inmask) ? (uint32_t)(__ffs(~inmask) - 1) : 32u;
    if (len == 32 && rs + 32 < seg_end && (hi[rs + 32] >> run_shift) == rkey) {
        if (lane == 0) {
            const uint32_t li = atomicAdd(long_count, 1u);
            if (HC_IN_BOUNDS(kSiteRunList, li, long_cap))
                long_list[li] = make_uint4((uint32_t)rs, (uint32_t)(rs >> 32), seg, 0u);
        }
        return;
    }
    const bool mine = (uint32_t)lane < len;
    const uint64_t h = mine ? he : ~0ull;
    const uint32_t d = mine ? de : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, h);
    const uint64_t l = (mine && __popc(peers) > 1)
                           ? row_key_lo(rows.db, rows.row_bytes, rows.P, d, curve)
                           : 0;
    uint32_t rank = 0;
    for (uint32_t u = 0; u < len; ++u) {
        const uint64_t hu = __shfl_sync(0xffffffffu, h, (int)u);
        const uint64_t lu = __shfl_sync(0xffffffffu, l, (int)u);
        const uint32_t du = __shfl_sync(0xffffffffu, d, (int)u);
        rank += (hu < h || (hu == h && (lu < l || (lu == l && du < d)))) ? 1u : 0u;
    }
    __syncwarp();
    if (mine && HC_IN_BOUNDS(kSiteRunWrite, rs + rank - segs[seg].start, segs[seg].len)) {
        hi[rs + rank] = h;
        ids[rs + rank] = d;
    }
    __syncwarp();
}

// The runs find_runs listed, one per lane: a run of at most kLaneRun records
// without two equal high words is ordered by that lane alone (its records
// share the prefix, so the low run_shift bits order them); every other run is
// appended to `deferred` for sort_runs_warp (one atomic per warp).
__global__ void __launch_bounds__(256) sort_runs_kernel(
    uint64_t* hi, uint32_t* ids, int run_shift, const SegInfo* __restrict__ segs,
    const uint64_t* __restrict__ run_pos, const uint32_t* __restrict__ run_seg,
    const unsigned long long* __restrict__ nruns, uint4* __restrict__ deferred,
    uint32_t* __restrict__ deferred_count, uint32_t deferred_cap) {
    const int lane = threadIdx.x & 31;
    const uint64_t n = *nruns;
    const uint32_t low_mask = run_shift >= 32 ? 0xFFFFFFFFu : (1u << run_shift) - 1u;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t r0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         r0 < n; r0 += nw * 32) {
        const uint64_t r = r0 + (uint64_t)lane;
        uint64_t rs = 0;
        uint32_t seg = 0;
        bool left = false;
        if (r < n) {
            rs = __ldg(run_pos + r);
            seg = __ldg(run_seg + r);
            const uint64_t seg_end = segs[seg].start + segs[seg].len;
            // the next kLaneRun + 1 words, all loads in flight at once
            uint64_t hw[kLaneRun + 1];
#pragma unroll
            for (int t = 0; t <= kLaneRun; ++t) hw[t] = rs + t < seg_end ? hi[rs + t] : 0;
            const uint64_t pre = hw[0] >> run_shift;
            uint32_t lw[kLaneRun];
            int len = 0;
            bool more = true;
#pragma unroll
            for (int t = 0; t < kLaneRun; ++t) {
                const bool in = more && rs + t < seg_end && (hw[t] >> run_shift) == pre;
                lw[t] = in ? (uint32_t)hw[t] & low_mask : 0u;
                if (in) len = t + 1;
                more = in;
            }
            // longer than kLaneRun, or two equal high words: the warp's turn
            left = more && rs + kLaneRun < seg_end && (hw[kLaneRun] >> run_shift) == pre;
#pragma unroll
            for (int a = 0; a < kLaneRun; ++a)
#pragma unroll
                for (int b = a + 1; b < kLaneRun; ++b)
                    if (b < len && lw[a] == lw[b]) left = true;
            if (!left) {
                uint32_t dv[kLaneRun];
#pragma unroll
                for (int t = 0; t < kLaneRun; ++t) dv[t] = t < len ? ids[rs + t] : 0u;
#pragma unroll
                for (int t = 0; t < kLaneRun; ++t) {
                    if (t < len) {
                        uint32_t rank = 0;
#pragma unroll
                        for (int u = 0; u < kLaneRun; ++u)
                            rank += (u < len && lw[u] < lw[t]) ? 1u : 0u;
                        if (rank != (uint32_t)t &&
                            HC_IN_BOUNDS(kSiteRunWrite, rs + rank - segs[seg].start,
                                         segs[seg].len)) {
                            hi[rs + rank] = hw[t];
                            ids[rs + rank] = dv[t];
                        }
                    }
                }
            }
        }
        const uint32_t todo = __ballot_sync(0xffffffffu, left);
        if (todo) {
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(deferred_count, (uint32_t)__popc(todo));
            at = __shfl_sync(0xffffffffu, at, 0) + (uint32_t)__popc(todo & ((1u << lane) - 1u));
            if (left && HC_IN_BOUNDS(kSiteRunList, at, deferred_cap))
                deferred[at] = make_uint4((uint32_t)rs, (uint32_t)(rs >> 32), seg, 0u);
        }
    }
}

// The runs sort_runs deferred: one warp each (warp_sort_run).
__global__ void __launch_bounds__(256) sort_runs_warp_kernel(
    uint64_t* hi, uint32_t* ids, int run_shift, RowKeys rows, const SegInfo* __restrict__ segs,
    const uint4* __restrict__ deferred, const uint32_t* __restrict__ deferred_count,
    uint4* __restrict__ long_list, uint32_t* __restrict__ long_count, uint32_t long_cap) {
    const int lane = threadIdx.x & 31;
    const uint32_t n = *deferred_count;
    const uint32_t nw = gridDim.x * (blockDim.x >> 5);
    for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += nw) {
        const uint4 fe = deferred[r];
        warp_sort_run(hi, ids, run_shift, rows, segs, ((uint64_t)fe.y << 32) | fe.x, fe.z,
                      long_list, long_count, long_cap, lane);
    }
}

// Runs of kMaxRun + 1 .. kMidRun records, as listed by sort_runs_warp: one
// block per run (grid-stride over the list), one record per thread.  The
// block finds the run's end, stages its records in shared memory, and each
// thread counts the records below its own by the low run_shift bits (the
// records share the prefix); equal low bits are equal high words, and then
// every record's low word is computed from its row and the counts are taken
// by (high word, low word, id).  A longer run is listed for long_run_kernel.
constexpr uint32_t kMidRun = 256;

__global__ void __launch_bounds__(kMidRun) sort_mid_runs_kernel(
    uint64_t* hi, uint32_t* ids, int run_shift, RowKeys rows, const SegInfo* __restrict__ segs,
    const uint4* __restrict__ long_list, const uint32_t* __restrict__ long_count,
    uint4* __restrict__ vlong_list, uint32_t* __restrict__ vlong_count, uint32_t vlong_cap) {
    __shared__ uint64_t sh[kMidRun];
    __shared__ uint64_t sl[kMidRun];
    __shared__ uint32_t sd[kMidRun];
    __shared__ uint32_t s_n;
    __shared__ int s_tie;
    const uint32_t t = threadIdx.x;
    const uint32_t low_mask = run_shift >= 32 ? 0xFFFFFFFFu : (1u << run_shift) - 1u;
    const uint32_t total = *long_count;
    for (uint32_t e = blockIdx.x; e < total; e += gridDim.x) {
        const uint4 fe = long_list[e];
        const uint64_t rs = ((uint64_t)fe.y << 32) | fe.x;
        const uint32_t seg = fe.z;
        const uint64_t seg_end = segs[seg].start + segs[seg].len;
        const uint64_t pre = hi[rs] >> run_shift;
        if (t == 0) {
            s_n = kMidRun + 1;
            s_tie = 0;
        }
        __syncthreads();
        // the first of the next kMidRun + 1 records outside the run bounds it
        for (uint32_t k = t; k <= kMidRun; k += blockDim.x) {
            const uint64_t i = rs + k;
            if (i >= seg_end || (hi[i] >> run_shift) != pre) atomicMin(&s_n, k);
        }
        __syncthreads();
        const uint32_t n = s_n;
        if (n > kMidRun) {
            if (t == 0) {
                const uint32_t vi = atomicAdd(vlong_count, 1u);
                if (HC_IN_BOUNDS(kSiteRunList, vi, vlong_cap)) vlong_list[vi] = fe;
            }
            __syncthreads();
            continue;
        }
        uint64_t h = 0;
        uint32_t d = 0;
        if (t < n) {
            h = hi[rs + t];
            d = ids[rs + t];
            sh[t] = h;
            sd[t] = d;
        }
        __syncthreads();
        uint32_t r = 0;
        if (t < n) {
            const uint32_t x = (uint32_t)h & low_mask;
            bool tie = false;
            for (uint32_t j = 0; j < n; ++j) {
                const uint32_t y = (uint32_t)sh[j] & low_mask;
                r += (y < x || (y == x && j < t)) ? 1u : 0u;
                tie |= y == x && j != t;
            }
            if (tie) s_tie = 1;
        }
        __syncthreads();
        if (s_tie) {
            if (t < n) sl[t] = row_key_lo(rows.db, rows.row_bytes, rows.P, d, seg % rows.P.curves);
            __syncthreads();
            if (t < n) {
                const uint64_t lx = sl[t];
                r = 0;
                for (uint32_t j = 0; j < n; ++j) {
                    const uint64_t hj = sh[j], lj = sl[j];
                    r += (hj < h || (hj == h && (lj < lx || (lj == lx && sd[j] < d)))) ? 1u : 0u;
                }
            }
        }
        if (t < n && HC_IN_BOUNDS(kSiteRunWrite, r, n)) {
            hi[rs + r] = h;
            ids[rs + r] = d;
        }
        __syncthreads();
    }
}

// Runs of more than kMidRun records with equal prefixes hi >> run_shift, as
// listed by sort_mid_runs: one block per run (grid-stride over the list; with an
// empty list every block returns at once).  A run's records arrive in id
// order; stable 8-bit passes over the bytes in which their low words (from
// the rows), then the bits of their high words below run_shift, differ leave
// them ordered by (high word, low word, id).  Scratch, the run's own stretch
// of each: the low words in lo_buf, two permutations in pa_buf and pb_buf.
constexpr int kRThreads = 1024;
constexpr int kRWarps = kRThreads / 32;

struct LongRunSmem {
    uint32_t hist[256];
    uint32_t wcnt[kRWarps][256];
    uint32_t warp_sums[kRWarps];
    uint64_t red[2][kRWarps];
    unsigned long long end;
};

// byte `byte` of element i's low word (f = 0) or high word (f = 1)
__device__ __forceinline__ uint32_t run_digit(int f, int byte, uint32_t i, const uint64_t* h,
                                              const uint64_t* lo) {
    const uint64_t x = f ? h[i] : lo[i];
    return (uint32_t)(x >> (8 * byte)) & 0xFFu;
}

// Stable pass of one block over n elements: `in` (null: identity) is the
// order so far, `out` receives the order by the digit.  Elements go in
// chunks of one per thread; within a chunk a warp ranks its lanes by ballots
// and the per-warp digit counts are scanned digit by digit over the warps.
__device__ void long_run_pass(const uint32_t* in, uint32_t* out, uint32_t n, int f, int byte,
                              const uint64_t* h, const uint64_t* lo, LongRunSmem& sm) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int i = t; i < 256; i += kRThreads) sm.hist[i] = 0;
    for (int i = t; i < kRWarps * 256; i += kRThreads) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    for (uint32_t i = t; i < n; i += kRThreads)
        atomicAdd(&sm.hist[run_digit(f, byte, in ? in[i] : i, h, lo)], 1u);
    __syncthreads();
    {
        const uint32_t v = t < 256 ? sm.hist[t] : 0u;
        const uint32_t ex = block_exclusive_scan<kRWarps>(v, sm.warp_sums);
        if (t < 256) sm.hist[t] = ex;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t c0 = 0; c0 < n; c0 += kRThreads) {
        const uint32_t i = c0 + (uint32_t)t;
        const bool valid = i < n;
        const uint32_t r = valid ? (in ? in[i] : i) : 0u;
        const uint32_t d = valid ? run_digit(f, byte, r, h, lo) : 0u;
        const uint32_t peers = digit_peers(d) & __ballot_sync(0xffffffffu, valid);
        if (valid && (peers & lt) == 0) sm.wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (t < 256) {
            uint32_t run = sm.hist[t];
            for (int w = 0; w < kRWarps; ++w) {
                const uint32_t c = sm.wcnt[w][t];
                sm.wcnt[w][t] = run;
                run += c;
            }
            sm.hist[t] = run;
        }
        __syncthreads();
        if (valid && HC_IN_BOUNDS(kSiteLongRun, sm.wcnt[warp][d] + __popc(peers & lt), n))
            out[sm.wcnt[warp][d] + __popc(peers & lt)] = r;
        __syncthreads();
        for (int j = t; j < kRWarps * 256; j += kRThreads) (&sm.wcnt[0][0])[j] = 0;
        __syncthreads();
    }
}

template <typename Op>
__device__ __forceinline__ uint64_t block_reduce64(uint64_t v, uint64_t* red, Op op) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    uint64_t r = red[0];
    for (int w = 1; w < kRWarps; ++w) r = op(r, red[w]);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kRThreads) long_run_kernel(
    uint64_t* hi, uint32_t* ids, uint64_t* lo_buf, uint32_t* pa_buf, uint32_t* pb_buf,
    int run_shift, RowKeys rows, const SegInfo* __restrict__ segs,
    const uint4* __restrict__ long_list, const uint32_t* __restrict__ long_count) {
    __shared__ LongRunSmem sm;
    const int t = threadIdx.x;
    const uint32_t total = *long_count;
    for (uint32_t e = blockIdx.x; e < total; e += gridDim.x) {
        const uint4 fe = long_list[e];
        const uint64_t rs = ((uint64_t)fe.y << 32) | fe.x;
        const uint32_t seg = fe.z;
        const uint64_t seg_end = segs[seg].start + segs[seg].len;
        const uint64_t pre = hi[rs] >> run_shift;
        // the run ends at the first position after rs with another prefix
        if (t == 0) sm.end = seg_end;
        __syncthreads();
        for (uint64_t c0 = rs + 1;; c0 += kRThreads) {
            const uint64_t i = c0 + (uint64_t)t;
            if (i < seg_end && (hi[i] >> run_shift) != pre) atomicMin(&sm.end, i);
            __syncthreads();
            const bool done = sm.end != seg_end || c0 + kRThreads >= seg_end;
            __syncthreads();
            if (done) break;
        }
        const uint32_t n = (uint32_t)(sm.end - rs);
        uint64_t* h = hi + rs;
        uint32_t* d = ids + rs;
        uint64_t* lo = lo_buf + rs;
        uint32_t* pa = pa_buf + rs;
        uint32_t* pb = pb_buf + rs;
        const uint32_t curve = seg % rows.P.curves;
        uint64_t ol = 0, al = ~0ull, oh = 0, ah = ~0ull;
        for (uint32_t i = t; i < n; i += kRThreads) {
            const uint64_t l = row_key_lo(rows.db, rows.row_bytes, rows.P, d[i], curve);
            lo[i] = l;
            ol |= l;
            al &= l;
            oh |= h[i];
            ah &= h[i];
        }
        auto bor = [](uint64_t x, uint64_t y) { return x | y; };
        auto band = [](uint64_t x, uint64_t y) { return x & y; };
        const uint64_t vary_l = block_reduce64(ol, sm.red[0], bor) &
                                ~block_reduce64(al, sm.red[1], band);
        const uint64_t vary_h = block_reduce64(oh, sm.red[0], bor) &
                                ~block_reduce64(ah, sm.red[1], band);
        const uint32_t* in = nullptr;
        uint32_t* out = pa;
        for (int f = 0; f < 2; ++f) {
            const uint64_t vary = f ? vary_h : vary_l;
            const int bytes = f ? run_shift / 8 : 8;
            for (int byte = 0; byte < bytes; ++byte) {
                if (((vary >> (8 * byte)) & 0xFFu) == 0) continue;
                long_run_pass(in, out, n, f, byte, h, lo, sm);
                in = out;
                out = out == pa ? pb : pa;
            }
        }
        if (in) {
            // permute in place through the buffers no longer needed
            uint32_t* dcopy = in == pa ? pb : pa;
            for (uint32_t i = t; i < n; i += kRThreads) {
                lo[i] = h[i];
                dcopy[i] = d[i];
            }
            __syncthreads();
            for (uint32_t i = t; i < n; i += kRThreads) {
                const uint32_t r = in[i];
                h[i] = lo[r];
                d[i] = dcopy[r];
            }
        }
        __syncthreads();
    }
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

uint32_t* pbuf_of(uint32_t* a, uint32_t* b, int which) { return which ? b : a; }

struct Layout {
    uint64_t total = 0;
    uint32_t nseg = 0, ntiles = 0;
    uint64_t ncounts = 0;
    size_t off_w = 0, off_pa = 0, off_pb = 0, off_counts = 0, off_totals = 0, off_segs = 0,
           off_flag = 0, off_digits = 0, off_long = 0, off_vlong = 0, bytes = 0;
};

Layout make_layout(const SortProblem& p) {
    Layout L;
    L.nseg = (uint32_t)(p.seg_off.size() - 1);
    L.total = p.seg_off.back();
    for (uint32_t s = 0; s < L.nseg; ++s) {
        const uint64_t len = p.seg_off[s + 1] - p.seg_off[s];
        const uint32_t nt = (uint32_t)((len + kTile - 1) / kTile);
        L.ncounts += 256ull * nt;
        L.ntiles += nt;
    }
    size_t o = 0;
    L.off_w = o;       o = align_up(o + sizeof(uint64_t) * L.total);
    L.off_pa = o;      o = align_up(o + sizeof(uint32_t) * L.total);
    L.off_pb = o;      o = align_up(o + sizeof(uint32_t) * L.total);
    L.off_counts = o;  o = align_up(o + sizeof(uint32_t) * (L.ncounts ? L.ncounts : 1));
    L.off_totals = o;  o = align_up(o + sizeof(uint32_t) * 256 * (L.nseg ? L.nseg : 1));
    L.off_segs = o;    o = align_up(o + sizeof(SegInfo) * (L.nseg ? L.nseg : 1));
    L.off_flag = o;    o = align_up(o + 32);   // flag; counts of long runs (+4), runs (+8), very long runs (+16), deferred runs (+20)
    L.off_digits = o;  o = align_up(o + L.total);
    // runs longer than kMaxRun: at most total / (kMaxRun + 1) of them
    L.off_long = o;    o = align_up(o + sizeof(uint4) * (L.total / (kMaxRun + 1) + 1));
    // runs longer than kMidRun in the in-place fix-up (a sort without low
    // words), at most total / (kMidRun + 1).  Callers size the scratch before
    // they set the ids, so the region depends on the low words alone: a
    // problem sized without them never needs more than was reserved.
    L.off_vlong = o;
    if (p.lo == nullptr) o = align_up(o + sizeof(uint4) * (L.total / (kMidRun + 1) + 1));
    L.bytes = o;
    return L;
}

// min(cap, per_sm x SMs) blocks, at least one
unsigned grid_blocks(uint64_t cap, unsigned per_sm) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (uint64_t)sms * per_sm;
    return (unsigned)std::max<uint64_t>(1, std::min(cap, want));
}

unsigned grid_stride_blocks(uint64_t work) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (work + 255) / 256;
    const uint64_t cap = (uint64_t)sms * 8;
    return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

}  // namespace

size_t sort_scratch_bytes(const SortProblem& p) { return make_layout(p).bytes; }

FirstDigits sort_first_digits(const SortProblem& p, void* scratch) {
    FirstDigits f;
    const int digits = (int)((p.key_bits + 7) / 8);
    const int hi_passes = std::max(digits - 8, 0);
    const bool in_place = p.lo == nullptr && p.id_base_dev != nullptr;
    if (!in_place || hi_passes == 0 || p.seg_off.size() < 2) return f;
    const int skip = (p.hi_skip > 0 && hi_passes > p.hi_skip) ? p.hi_skip : 0;
    f.buf = static_cast<uint8_t*>(scratch) + make_layout(p).off_digits;
    f.shift = ((8 + skip) & 7) * 8;
    return f;
}

namespace {
struct SmallBlock {
    uint64_t w[kMaxParamWords];
};
__global__ void upload_small_kernel(uint64_t* dst, SmallBlock b, uint32_t words) {
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = b.w[i];
}
}  // namespace

cudaError_t upload_small(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    // dst is 8-byte aligned device memory of at least round_up(bytes, 8)
    const uint8_t* p = static_cast<const uint8_t*>(src);
    uint64_t* d = static_cast<uint64_t*>(dst);
    while (bytes > 0) {
        const size_t chunk = bytes < kMaxParamWords * 8 ? bytes : kMaxParamWords * 8;
        SmallBlock b;
        memset(&b, 0, sizeof(b));
        memcpy(b.w, p, chunk);
        const uint32_t words = (uint32_t)((chunk + 7) / 8);
        upload_small_kernel<<<1, 128, 0, s>>>(d, b, words);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        p += chunk;
        d += words;
        bytes -= chunk;
    }
    return cudaSuccess;
}

namespace {

// The sort; fenced: the fence was written on the way (find_runs).
int sort_body(const SortProblem& p, void* scratch, cudaStream_t s, bool& fenced) {
    if (p.seg_off.size() < 2 || p.key_bits < 1 || p.key_bits > 128) return HC_ERR_ARG;
    Layout L = make_layout(p);
    if (L.total == 0) return HC_OK;
    if (L.total > 0xFFFFFFFFull) return HC_ERR_ARG;
    char* base = static_cast<char*>(scratch);
    uint64_t* wtmp = reinterpret_cast<uint64_t*>(base + L.off_w);
    uint32_t* pa = reinterpret_cast<uint32_t*>(base + L.off_pa);
    uint32_t* pb = reinterpret_cast<uint32_t*>(base + L.off_pb);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + L.off_counts);
    uint32_t* totals = reinterpret_cast<uint32_t*>(base + L.off_totals);
    SegInfo* segs = reinterpret_cast<SegInfo*>(base + L.off_segs);

    cudaError_t e;
    seg_setup_kernel<<<1, 32, 0, s>>>(p.seg_off_dev, L.nseg, segs);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return HC_ERR_CUDA;
    const size_t dyn_smem = sizeof(ScatterSmem);
    e = cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn_smem);
    if (e != cudaSuccess) return HC_ERR_CUDA;

    const int digits = (int)((p.key_bits + 7) / 8);
    const int lo_passes = std::min(digits, 8);
    const int hi_passes = std::max(digits - 8, 0);
    const dim3 scan_grid(256, L.nseg);
    uint32_t* flag = reinterpret_cast<uint32_t*>(base + L.off_flag);
    // next-pass digits, one byte per record, written by a scatter for the
    // following histogram (within one key word)
    uint8_t* dgt = reinterpret_cast<uint8_t*>(base + L.off_digits);

    // affine ids without low words: the last pass writes the final high
    // words and ids, and only runs are fixed up in place, on the device
    const bool in_place = p.lo == nullptr && p.id_base_dev != nullptr;
    if ((p.allow_sync || in_place) && hi_passes > 0 && L.ntiles) {
        // sort by the high word's top bytes alone (skipping its lowest
        // hi_skip digits when more remain), then order runs of equal prefixes
        const int skip = (p.hi_skip > 0 && hi_passes > p.hi_skip) ? p.hi_skip : 0;
        const int npass = hi_passes - skip;
        uint64_t* wb[2] = {wtmp, p.out_hi};
        // the last pass writes wtmp (or out_hi when in place)
        int wn = ((npass % 2 == 1) != in_place) ? 0 : 1;
        int pn = 0;
        const uint64_t* cw = p.hi;
        const uint32_t* cp = nullptr;
        for (int t = 8 + skip; t < 8 + hi_passes; ++t) {
            const int shift = (t & 7) * 8;
            const bool last = t + 1 == 8 + hi_passes;
            uint32_t* pd = (last && in_place) ? p.out_ids : pbuf_of(pa, pb, pn);
            const bool first = t == 8 + skip;
            // the first pass reads words unless the key producer left its digits
            const uint8_t* hd = first && !p.first_digits_ready ? nullptr : dgt;
            hist_kernel<<<L.ntiles, kThreads, 0, s>>>(cw, hd, shift, L.nseg, segs, counts);
            scan_kernel<<<scan_grid, kScanThreads, 0, s>>>(segs, counts, totals);
            scatter_kernel<<<L.ntiles, kSThreads, dyn_smem, s>>>(
                cw, cp, wb[wn], pd, shift, L.nseg, segs, counts, totals,
                (last && in_place) ? p.id_base_dev : nullptr, last ? nullptr : dgt);
            count_launches(3);
            if (cudaGetLastError() != cudaSuccess) return HC_ERR_CUDA;
            cw = wb[wn];
            cp = pd;
            wn ^= 1;
            pn ^= 1;
        }
        // the flag word, the count of long runs (4 bytes on), then (8 bytes
        // on) the run count of the in-place fix-up
        uint32_t* long_count = reinterpret_cast<uint32_t*>(base + L.off_flag + 4);
        unsigned long long* nruns = reinterpret_cast<unsigned long long*>(base + L.off_flag + 8);
        uint32_t* vlong_count = reinterpret_cast<uint32_t*>(base + L.off_flag + 16);
        if (cudaMemsetAsync(flag, 0, 32, s) != cudaSuccess) return HC_ERR_CUDA;
        if (in_place) {
            if (cw != p.out_hi) return HC_ERR_STATE;
            // both position buffers are free once the last pass has run: at
            // most total / 2 runs (two records or more each) fit in either
            uint64_t* run_pos = reinterpret_cast<uint64_t*>(pa);
            uint32_t* run_seg = pb;
            uint4* long_list = reinterpret_cast<uint4*>(base + L.off_long);
            // the fence from find_runs when its mask clears every bit the
            // fix-up may still change (the low 8 skip bits)
            uint64_t* fence =
                (kFenceMask & ((1ull << (8 * skip)) - 1)) == 0 ? p.out_fence : nullptr;
            fenced = fence != nullptr;
            switch (skip) {
#define HC_FIND(K)                                                                          \
    case K:                                                                                 \
        find_runs_kernel<8 * K><<<L.ntiles, kFindWarps * 32, 0, s>>>(                       \
            p.out_hi, p.out_ids, L.nseg, segs, run_pos, run_seg, nruns, fence);             \
        break;
                HC_FIND(1) HC_FIND(2) HC_FIND(3) HC_FIND(4)
#undef HC_FIND
                default: return HC_ERR_STATE;   // prefixes of at least 32 bits are sorted
            }
            // the word buffer is free after the last pass: the list of runs the
            // lanes leave to warps (at most total / 2 entries of 16 bytes)
            uint4* deferred = reinterpret_cast<uint4*>(wtmp);
            uint32_t* deferred_count = reinterpret_cast<uint32_t*>(base + L.off_flag + 20);
            sort_runs_kernel<<<grid_stride_blocks(L.total / 64), 256, 0, s>>>(
                p.out_hi, p.out_ids, 8 * skip, segs, run_pos, run_seg, nruns, deferred,
                deferred_count, (uint32_t)(L.total / 2));
            sort_runs_warp_kernel<<<grid_blocks(L.ntiles, 8), 256, 0, s>>>(
                p.out_hi, p.out_ids, 8 * skip, p.rows, segs, deferred, deferred_count, long_list,
                long_count, (uint32_t)(L.total / (kMaxRun + 1) + 1));
            uint4* vlong_list = reinterpret_cast<uint4*>(base + L.off_vlong);
            sort_mid_runs_kernel<<<grid_blocks(L.ntiles, 8), kMidRun, 0, s>>>(
                p.out_hi, p.out_ids, 8 * skip, p.rows, segs, long_list, long_count, vlong_list,
                vlong_count, (uint32_t)(L.total / (kMidRun + 1) + 1));
            // the word and position buffers are free now: scratch of the long runs
            long_run_kernel<<<std::min<uint32_t>(L.ntiles, 152), kRThreads, 0, s>>>(
                p.out_hi, p.out_ids, wtmp, pa, pb, 8 * skip, p.rows, segs, vlong_list,
                vlong_count);
            count_launches(5);
            if (cudaGetLastError() != cudaSuccess) return HC_ERR_CUDA;
            return HC_OK;
        } else {
            if (cw != wtmp) return HC_ERR_STATE;
            fixup_final_kernel<<<L.ntiles, 256, 0, s>>>(
                wtmp, 8 * skip, cp, p.lo, p.rows, FinalIds{p.ids, p.id_base_dev}, p.out_hi,
                p.lo ? p.out_lo : nullptr, p.out_ids, L.nseg, segs, flag);
        }
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return HC_ERR_CUDA;
        uint32_t long_run = 1;
        if (cudaMemcpyAsync(&long_run, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HC_ERR_CUDA;
        if (!long_run) return HC_OK;
        // a run of equal high words longer than the fix-up handles: sort
        // again with every digit (the sources are untouched)
    }
    if (!p.lo) return HC_ERR_STATE;   // every digit needs the low words
    // word buffers written in sequence: each lo pass, the hi gather, each hi
    // pass; alternate so that the last write lands in out_hi.
    const int writes = lo_passes + 1 + hi_passes;
    uint64_t* wbuf[2] = {p.out_hi, wtmp};
    int wnext = (writes % 2 == 1) ? 0 : 1;
    uint32_t* pbuf[2] = {pa, pb};
    int pnext = 0;

    const uint64_t* cur_w = p.lo;
    const uint32_t* cur_p = nullptr;
    // digits of the next pass were written by the previous scatter when both
    // passes read the same key word
    bool have_digits = false;
    // final_ids: the pass writes the final ids (id_base) instead of positions
    auto run_pass = [&](int digit, bool next_same_word, bool final_ids = false) -> int {
        const int shift = (digit & 7) * 8;
        if (L.ntiles) {
            hist_kernel<<<L.ntiles, kThreads, 0, s>>>(cur_w, have_digits ? dgt : nullptr, shift,
                                                      L.nseg, segs, counts);
            scan_kernel<<<scan_grid, kScanThreads, 0, s>>>(segs, counts, totals);
            uint64_t* wd = wbuf[wnext];
            uint32_t* pd = final_ids ? p.out_ids : pbuf[pnext];
            scatter_kernel<<<L.ntiles, kSThreads, dyn_smem, s>>>(
                cur_w, cur_p, wd, pd, shift, L.nseg, segs, counts, totals,
                final_ids ? p.id_base_dev : nullptr, next_same_word ? dgt : nullptr);
            count_launches(3);
            if (cudaGetLastError() != cudaSuccess) return HC_ERR_CUDA;
            cur_w = wd;
            cur_p = pd;
            wnext ^= 1;
            pnext ^= 1;
        }
        have_digits = next_same_word;
        return HC_OK;
    };
    if (p.ids_only && hi_passes == 0 && p.id_base_dev) {
        // the last pass writes the ids; no word is gathered
        for (int t = 0; t < lo_passes; ++t)
            if (int rc = run_pass(t, t + 1 < lo_passes && (t & 7) != 7, t + 1 == lo_passes))
                return rc;
        return HC_OK;
    }
    for (int t = 0; t < lo_passes; ++t)
        if (int rc = run_pass(t, t + 1 < lo_passes && (t & 7) != 7)) return rc;
    {
        uint64_t* wd = wbuf[wnext];
        gather_words_kernel<<<grid_stride_blocks(L.total), 256, 0, s>>>(p.hi, cur_p, wd, L.total);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return HC_ERR_CUDA;
        cur_w = wd;
        wnext ^= 1;
    }
    have_digits = false;   // the high words were just gathered
    for (int t = 8; t < 8 + hi_passes; ++t)
        if (int rc = run_pass(t, t + 1 < 8 + hi_passes && (t & 7) != 7)) return rc;
    if (cur_w != p.out_hi) return HC_ERR_STATE;  // buffer bookkeeping broken
    gather_final_kernel<<<L.ntiles, 256, 0, s>>>(p.lo, FinalIds{p.ids, p.id_base_dev}, cur_p,
                                                  p.out_lo, p.out_ids, L.nseg, segs);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return HC_ERR_CUDA;
    return HC_OK;
}

}  // namespace

int sort_segments(const SortProblem& p, void* scratch, cudaStream_t s) {
    bool fenced = false;
    int rc = sort_body(p, scratch, s, fenced);
    if (rc == HC_OK && p.out_fence && !fenced &&
        launch_fence(p.out_hi, p.seg_off.back(), p.out_fence, s) != cudaSuccess)
        rc = HC_ERR_CUDA;
    return rc;
}

}  // namespace hc
