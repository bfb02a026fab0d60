// K3..K6: the fused query kernel (Algorithm 2 for a batch of queries); the
// exact brute-force kNN (Eq. 3), which shares its distance and top-k code,
// is in brute.cu.
//
// One warp per query:
//   K1  lanes c < curves compute the query's extended-key on curve c;
//   K3  lanes L < lists run lower_bound in list L (128-bit compares; the low
//       word is consulted only when the high words tie, recomputed from the
//       entry's row when the index keeps high words only);
//   K4  the windows [max(0,pos-p), min(n,pos+p)) are walked 32 entries at a
//       time: the 32 ids are one load, then each row is read as 16-byte
//       vectors by LPR lanes (LPR = 8 for 128-byte uint8 rows: four rows per
//       warp instruction).  Rows of at most 128 bytes are staged: all windows
//       of the query are packed back to back (a step may span several), and
//       the next step's rows are copied into a two-step per-warp shared-
//       memory ring with cp.async while the current step is reduced, so the
//       bytes in flight are bounded by shared memory instead of registers;
//       wider rows are gathered into registers, eight 16-byte loads in flight
//       per lane.  uint8 partial distances use
//       vabsdiffu4 + dp4a (exact in 32-bit integers), float32 use fma;
//       a reduce-scatter over the LPR lanes leaves lane l with the distance
//       of one row of the 32 (LPR-1 shuffles for LPR partial sums);
//   K5/K6 the 32 packed (distance, id) candidates are offered to one running
//       warp top-k for the whole query, which drops duplicate ids: the union
//       over curves and partitions and the Aggregator's reduction in one.
// The path is a gather bounded by HBM bandwidth; no tensor cores are used.
#include <algorithm>

#include "hc_dispatch.cuh"
#include "hc_internal.h"
#include "hc_query_dev.cuh"
#include "hc_topk.cuh"

namespace hc {

namespace {

constexpr int kQWarps = 8;
constexpr int kStages = 2;   // ring stages per warp (deeper rings measured slower)

struct QueryArgs {
    IndexView ix;
    const void* q;
    uint32_t nq, k, p;
    int32_t* out_ids;
    void* out_dist;
    int64_t* out_pos;            // positions-only kernel
    const uint32_t* p_query;     // per-query depth (overrides p), or null
    const int64_t* pos_in;       // precomputed lower_bound positions (nq x lists), or null
    const uint32_t* order;       // warp w answers query order[w], or null (w itself)
};

#ifndef HC_QUERY_MIN_BLOCKS
#define HC_QUERY_MIN_BLOCKS 3    // resident blocks per SM the query kernel is compiled for
                                 // (3 x 8 warps: best at p = 128 and 512 on GB300)
#endif

// STAGED: rows of at most 128 bytes go through a two-step cp.async ring in
// shared memory (kQWarps x 2 x 32 rows after the positions and the window
// prefixes)
template <bool F32, int LPR, int KR, bool STAGED>
__global__ void __launch_bounds__(kQWarps * 32, HC_QUERY_MIN_BLOCKS) query_kernel(QueryArgs a) {
    extern __shared__ __align__(16) uint32_t s_pos[];  // kQWarps x lists, then the rings
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t w = blockIdx.x * kQWarps + warp;
    if (w >= a.nq) return;
    const uint32_t qi = a.order ? __ldg(a.order + w) : w;
    if (!HC_IN_BOUNDS(kSiteQuery, qi, a.nq)) return;
    const IndexView& ix = a.ix;
    const uint8_t* qrow = static_cast<const uint8_t*>(a.q) + (size_t)qi * ix.row_bytes;
    const uint32_t depth = a.p_query ? __ldg(a.p_query + qi) : a.p;
    WarpTopK<KR> top;
    top.init();
    if constexpr (STAGED) {
        // after the positions: kQWarps x lists window prefixes, then the rings
        uint32_t* s_pre = s_pos + kQWarps * ix.lists;
        uint8_t* ring = reinterpret_cast<uint8_t*>(s_pre + kQWarps * ix.lists) +
                        (size_t)warp * kStages * 32 * ix.row_bytes;
        search_lists_staged<F32, LPR, KR, kStages>(
            ix, qrow, depth, a.k, 0, 1, s_pos + warp * ix.lists, s_pre + warp * ix.lists, ring,
            top, lane, a.pos_in ? a.pos_in + (size_t)qi * ix.lists : nullptr);
    } else {
        search_lists<F32, LPR, KR>(ix, qrow, depth, a.k, 0, 1, s_pos + warp * ix.lists, top,
                                   lane, a.pos_in ? a.pos_in + (size_t)qi * ix.lists : nullptr);
    }
    top.template store<F32>(a.k, lane, a.out_ids + (size_t)qi * a.k,
                            static_cast<uint32_t*>(a.out_dist) + (size_t)qi * a.k);
}

// keys[i] = top kOrderBits bits of query i's curve-0 extended-key (one thread each)
__global__ void __launch_bounds__(256) order_keys_kernel(IndexView ix, const uint8_t* q,
                                                         uint32_t nq, uint64_t* keys) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    uint64_t h, l;
    curve_key_call(q + (size_t)i * ix.row_bytes, ix.P, 0, h, l);
    const uint32_t bits = 8 * ix.P.m;   // key bits, right-aligned in (h, l)
    const uint64_t top = bits > 64 ? (h << (128 - bits)) | (bits < 128 ? l >> (bits - 64) : 0)
                                   : l << (64 - bits);
    keys[i] = top >> (64 - kOrderBits);
}

__global__ void __launch_bounds__(kQWarps * 32) positions_kernel(QueryArgs a) {
    extern __shared__ uint32_t s_pos[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t qi = blockIdx.x * kQWarps + warp;
    if (qi >= a.nq) return;
    const uint8_t* qrow = static_cast<const uint8_t*>(a.q) + (size_t)qi * a.ix.row_bytes;
    uint32_t* pos_w = s_pos + warp * a.ix.lists;
    query_positions(a.ix, qrow, pos_w, lane);
    for (uint32_t L = lane; L < a.ix.lists; L += 32)
        a.out_pos[(size_t)qi * a.ix.lists + L] = (int64_t)pos_w[L];
}

template <bool F32, int LPR, int KR>
struct QueryLaunch {
    template <bool STAGED>
    static cudaError_t go(const QueryArgs& a, size_t smem, cudaStream_t s) {
        const unsigned blocks = (a.nq + kQWarps - 1) / kQWarps;
        if (STAGED) {
            cudaError_t e = cudaFuncSetAttribute(query_kernel<F32, LPR, KR, STAGED>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        query_kernel<F32, LPR, KR, STAGED><<<blocks, kQWarps * 32, smem, s>>>(a);
        count_launches(1);
        return cudaGetLastError();
    }
    static cudaError_t run(const QueryArgs& a, cudaStream_t s) {
        const size_t pos_bytes = sizeof(uint32_t) * kQWarps * a.ix.lists;
        // rows of at most 128 bytes (all rows of 4 or 8 lanes) are staged
        if constexpr (LPR <= 8) {
            const size_t smem = 2 * pos_bytes + (size_t)kQWarps * kStages * 32 * a.ix.row_bytes;
            return go<true>(a, smem, s);
        } else {
            return go<false>(a, pos_bytes, s);
        }
    }
};

}  // namespace

cudaError_t launch_query(const IndexView& ix, const void* q, uint32_t nq, uint32_t k, uint32_t p,
                         int32_t* out_ids, void* out_dist, cudaStream_t s,
                         const uint32_t* p_query, const int64_t* pos_in,
                         const uint32_t* order) {
    if (nq == 0) return cudaSuccess;
    QueryArgs a{ix, q, nq, k, p, out_ids, out_dist, nullptr, p_query, pos_in, order};
    return dispatch<QueryLaunch>(ix.P.dtype == HC_F32, lanes_per_row(ix.row_bytes), regs_for_k(k),
                                 a, s);
}

cudaError_t launch_order_keys(const IndexView& ix, const void* q, uint32_t nq, uint64_t* keys,
                              cudaStream_t s) {
    if (nq == 0) return cudaSuccess;
    order_keys_kernel<<<(nq + 255) / 256, 256, 0, s>>>(ix, static_cast<const uint8_t*>(q), nq,
                                                       keys);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_positions(const IndexView& ix, const void* q, uint32_t nq, int64_t* pos,
                             cudaStream_t s) {
    if (nq == 0) return cudaSuccess;
    QueryArgs a{ix, q, nq, 1, 0, nullptr, nullptr, pos, nullptr, nullptr, nullptr};
    const unsigned blocks = (nq + kQWarps - 1) / kQWarps;
    positions_kernel<<<blocks, kQWarps * 32, sizeof(uint32_t) * kQWarps * ix.lists, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hc
