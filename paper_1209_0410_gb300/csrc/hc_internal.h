// Host-side declarations shared by the libhc translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "hc.h"
#include "hc_device.cuh"

namespace hc {

// Every kernel launch the library issues is counted here (hc_launch_count).
void count_launches(uint64_t n);

// Host-side fault injection (hc_debug_fail_alloc): true when the library's
// next allocation must report out-of-memory.
bool alloc_should_fail();

// ------------------------------------------------------------ K1: keys
// Keys of every row for every curve, written at the row's slot of each list
// of its partition: list L = part*curves + c, slot list_off[L] + (r - start).
struct BuildKeysArgs {
    const void* db;
    uint64_t n;
    uint32_t row_bytes;
    Projection P;
    uint32_t partitions;
    const uint64_t* list_off;  // device, lists+1
    uint64_t* hi;
    uint64_t* lo;
    uint32_t* ids;             // may be null: ids are then implied by the slot
    // may be null: digits[g] = (hi[g] >> digit_shift) & 0xFF, the first radix
    // pass's digit of every key (sort_first_digits), so that its histogram
    // reads bytes instead of words
    uint8_t* digits;
    int digit_shift;
};
cudaError_t launch_build_keys(const BuildKeysArgs& a, cudaStream_t s);

// count x curves keys of standalone vectors
cudaError_t launch_vector_keys(const void* x, uint64_t count, uint32_t row_bytes,
                               const Projection& P, uint64_t* hi, uint64_t* lo, cudaStream_t s);

// ------------------------------------------------------------ K2: sort
// Stable LSD radix sort of 128-bit keys by segment.  The sources stay
// untouched; the sorted keys and the carried ids land in out_*.
// Where the key of a database row comes from: the rows and their projection.
struct RowKeys {
    const void* db = nullptr;
    uint32_t row_bytes = 0;
    Projection P{};
};

struct SortProblem {
    const uint64_t* hi = nullptr;   // device, total records
    const uint64_t* lo = nullptr;
    const uint32_t* ids = nullptr;
    std::vector<uint64_t> seg_off;  // host, nseg+1 (grid sizes)
    const uint64_t* seg_off_dev = nullptr;    // the same offsets on the device
    uint32_t key_bits = 0;         // 1..128
    // With lo words (or gathered ids): may the sort synchronise the stream
    // once (to learn whether a run of equal high words is too long for the
    // high-word-first path)?  With false, every digit is sorted and nothing
    // waits on the device.  Affine ids without lo words never wait: long
    // runs are sorted on the device.
    bool allow_sync = false;
    // On that path, low digits of the high word left to the run fix-up (runs
    // of records whose other high-word bits are equal); 0 sorts every digit.
    int hi_skip = 0;
    const uint64_t* id_base_dev = nullptr;  // device, nseg: ids[i] = id_base[s] + i - seg start
                                            // (then `ids` is not read); null = gather ids
    // lo == nullptr (high-word-first path with affine ids only): the low word
    // of record i of segment s is recomputed from row id_base[s] + i - seg
    // start on curve s % rows.P.curves, when a tie of the high words needs
    // it; out_lo is not written.
    RowKeys rows{};
    uint64_t* out_hi = nullptr;   // device, total records (distinct from sources)
    uint64_t* out_lo = nullptr;
    uint32_t* out_ids = nullptr;
    // nullable: out_fence[j] = out_hi[16 j] & kFenceMask for j < ceil(seg_off
    // back / 16), written by the run fix-up's first kernel on the high-word-
    // first path (the bits of the high word the radix passes leave final),
    // else by a pass over out_hi after the sort
    uint64_t* out_fence = nullptr;
    // only out_ids is wanted (affine ids: id_base_dev set, keys of at most 64
    // bits): the last radix pass writes the ids and nothing is gathered;
    // out_hi and out_lo serve as scratch and are left undefined
    bool ids_only = false;
    // high-word-first path with affine ids only: the caller wrote the first
    // pass's digit bytes into sort_first_digits(...).buf before the sort
    bool first_digits_ready = false;
};
// Scratch bytes the sort needs for this problem (queried before allocating).
size_t sort_scratch_bytes(const SortProblem& p);
// Enqueues the whole sort on s using the given scratch (>= sort_scratch_bytes).
int sort_segments(const SortProblem& p, void* scratch, cudaStream_t s);
// Where a producer of the keys may leave the first radix pass's digit of
// every record (one byte at the record's position) for the high-word-first
// path with affine ids: buf (inside scratch) and the digit's shift in the high
// word; buf is null for problems that take another path.
struct FirstDigits {
    uint8_t* buf = nullptr;
    int shift = 0;
};
FirstDigits sort_first_digits(const SortProblem& p, void* scratch);

// Small host tables written to device memory by a kernel that takes them
// as a by-value parameter, so that no pageable copy (and its implicit
// stream synchronisation) sits on the build path.
constexpr uint32_t kMaxParamWords = 480;  // 8-byte words per launch (< 4 KB)
cudaError_t upload_small(void* dst, const void* src, size_t bytes, cudaStream_t s);

// ---------------------------------------------------- K3..K6: queries
struct IndexView {
    const void* db;
    uint32_t row_bytes;
    uint32_t d;
    Projection P;
    uint32_t lists;            // partitions * curves
    const uint64_t* list_off;  // device, lists+1
    const uint64_t* keys_hi;
    const uint64_t* keys_lo;   // null: low words recomputed from the rows (16-coordinate keys)
    const uint32_t* ids;
    uint64_t rows;             // database rows (bound of the row ids)
    // fence[j] = keys_hi[j << kFenceShift] & kFenceMask over every list's
    // entries (global entry index), fence_len = ceil(entries / 16); null:
    // plain binary search
    const uint64_t* fence;
    uint64_t fence_len;
};

// One fence word per 16 entries: 128 bytes of high words, one L2 line.
constexpr uint32_t kFenceShift = 4;
// A fence word keeps the top 48 bits of its high word: the build's radix
// passes leave those final (the run fix-up only reorders entries whose top 48
// bits are equal), so the fix-up's first pass over the sorted words writes
// the fence.  Comparing (kh &
// kFenceMask) with a fence word still orders the key against the entry
// whenever the two differ.
constexpr uint64_t kFenceMask = ~0xFFFFull;
// fence[j] = keys_hi[j << kFenceShift] & kFenceMask for j < ceil(total / 16).
cudaError_t launch_fence(const uint64_t* keys_hi, uint64_t total, uint64_t* fence,
                         cudaStream_t s);

// p_query (device, nq entries, nullable) gives each query its own depth.
// pos_in (device, nq x lists, nullable): lower_bound positions computed
// earlier (hc_query_positions), so the kernel skips its own search.
// Low key words of every entry (list_off order) of an index without keys_lo.
cudaError_t launch_entry_lo(const IndexView& ix, uint64_t* out, cudaStream_t s);
// order (device, nq entries, nullable): warp w answers query order[w] (a
// permutation of 0..nq-1); results still land at each query's own row.
// pos_cm (device, nq x lists uint32, nullable): positions of
// launch_batch_positions (curve-major rows), so the kernel skips its search.
cudaError_t launch_query(const IndexView& ix, const void* q, uint32_t nq, uint32_t k, uint32_t p,
                         int32_t* out_ids, void* out_dist, cudaStream_t s,
                         const uint32_t* p_query = nullptr, const int64_t* pos_in = nullptr,
                         const uint32_t* order = nullptr, const uint32_t* pos_cm = nullptr);
// Bits of each curve's key that order a batch in hc_query_ordered: 65,536
// buckets keep a batch's neighbouring queries together at two radix passes
// (24 and 32 bits measured no faster on 1 to 32 partitions).
constexpr uint32_t kOrderBits = 16;
// keys[c nq + i]: the top kOrderBits bits of query i's curve-c extended-key
// for c < ncurves, as the low word of a sort key (curve 0: the order in which
// hc_query_ordered answers the queries); qhi / qlo (nullable, same layout):
// the keys' two words.
cudaError_t launch_order_keys(const IndexView& ix, const void* q, uint32_t nq, uint32_t ncurves,
                              uint64_t* keys, uint64_t* qhi, uint64_t* qlo, cudaStream_t s);
// lower_bound of every query in every list, one warp per 32 queries of one
// curve's key order (order: curves x nq ranks -> query; qhi / qlo: curves x nq
// query keys).  pos[i * lists + c * partitions + j] = position of query i in
// list j * curves + c.
cudaError_t launch_batch_positions(const IndexView& ix, uint32_t nq, const uint32_t* order,
                                   const uint64_t* qhi, const uint64_t* qlo, uint32_t* pos,
                                   cudaStream_t s);
cudaError_t launch_positions(const IndexView& ix, const void* q, uint32_t nq, int64_t* pos,
                             cudaStream_t s);
cudaError_t launch_bruteforce(const void* db, hc_dtype dtype, uint64_t n, uint32_t d,
                              const void* q, uint32_t nq, uint32_t k, int32_t* out_ids,
                              void* out_dist, cudaStream_t s);

}  // namespace hc
