// K3..K6: the fused query kernel (Algorithm 2 for a batch of queries); the
// exact brute-force kNN (Eq. 3), which shares its distance and top-k code,
// is in brute.cu.
//
// One warp per query:
//   K1  lanes c < curves compute the query's extended-key on curve c;
//   K3  lanes L < lists run lower_bound in list L (128-bit compares; the low
//       word is consulted only when the high words tie, recomputed from the
//       entry's row when the index keeps high words only), starting on the
//       index's fence of every 16th high word.  For hc_query_ordered, K1 and
//       K3 run before the walk as passes over the whole batch instead
//       (order_keys_kernel: every curve's key of every query; a sort by each
//       curve's key; batch_positions_kernel: a warp per 32 neighbouring keys
//       of one curve), and the walk reads the positions;
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
    const uint32_t* pos_cm;      // positions of the batch pass (curve-major rows), or null
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
            top, lane, a.pos_in ? a.pos_in + (size_t)qi * ix.lists : nullptr,
            a.pos_cm ? a.pos_cm + (size_t)qi * ix.lists : nullptr);
    } else {
        search_lists<F32, LPR, KR>(ix, qrow, depth, a.k, 0, 1, s_pos + warp * ix.lists, top,
                                   lane, a.pos_in ? a.pos_in + (size_t)qi * ix.lists : nullptr,
                                   a.pos_cm ? a.pos_cm + (size_t)qi * ix.lists : nullptr);
    }
    top.template store<F32>(a.k, lane, a.out_ids + (size_t)qi * a.k,
                            static_cast<uint32_t*>(a.out_dist) + (size_t)qi * a.k);
}

// keys[c nq + i] = top kOrderBits bits of query i's curve-c extended-key
// for c < ncurves; with qhi / qlo, also the key's two words.  One thread per
// query: 16-coordinate curves of consecutive dimensions four at a time as
// byte lanes of 32-bit words (as the build's key pass), others one by one.
__device__ __forceinline__ void put_order_key(const IndexView& ix, uint32_t nq, uint32_t i,
                                              uint32_t c, uint64_t h, uint64_t l, uint64_t* keys,
                                              uint64_t* qhi, uint64_t* qlo) {
    const size_t t = (size_t)c * nq + i;
    const uint32_t bits = 8 * ix.P.m;   // key bits, right-aligned in (h, l)
    const uint64_t top = bits > 64 ? (h << (128 - bits)) | (bits < 128 ? l >> (bits - 64) : 0)
                                   : l << (64 - bits);
    keys[t] = top >> (64 - kOrderBits);
    if (qhi) {
        qhi[t] = h;
        qlo[t] = l;
    }
}

__global__ void __launch_bounds__(256) order_keys_kernel(IndexView ix, const uint8_t* q,
                                                         uint32_t nq, uint32_t ncurves,
                                                         uint64_t* keys, uint64_t* qhi,
                                                         uint64_t* qlo) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const uint8_t* row = q + (size_t)i * ix.row_bytes;
    uint32_t c = 0;
    if (ix.P.m == 16 && ix.P.dim_map == nullptr) {
        for (; c + 4 <= ncurves; c += 4) {
            uint4 cb[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) cb[t] = curve_bytes16(row, ix.P.dtype, c + t);
            uint64_t hi[4], lo[4];
            hilbert_keys4<false>(cb, hi, lo);
#pragma unroll
            for (int t = 0; t < 4; ++t) put_order_key(ix, nq, i, c + t, hi[t], lo[t], keys, qhi, qlo);
        }
    }
    for (; c < ncurves; ++c) {
        uint64_t h, l;
        curve_key_call(row, ix.P, c, h, l);
        put_order_key(ix, nq, i, c, h, l, keys, qhi, qlo);
    }
}

// searches a lane of batch_positions_kernel runs side by side (1, 2 and 8
// measured slower on 32 partitions)
constexpr int kBatchILP = 4;

// at[0 .. G) to p[0 .. G), p aligned to 4 G bytes
template <int G>
__device__ __forceinline__ void store_group(uint32_t* p, const uint32_t (&at)[G]) {
    if constexpr (G == 4) {
        *reinterpret_cast<uint4*>(p) = make_uint4(at[0], at[1], at[2], at[3]);
    } else if constexpr (G == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(at[0], at[1]);
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) p[g] = at[g];
    }
}

// Queries a lane of batch_positions_kernel takes: kBatchILP searches side by
// side are kBatchILP partitions of one query (three partitions or more: the
// last group may be partial), or the partitions of four queries (one
// partition) or of two (two partitions).
__host__ __device__ __forceinline__ uint32_t batch_queries_per_lane(uint32_t parts) {
    return parts == 1 ? 4u : (parts == 2 ? 2u : 1u);
}
static_assert(kBatchILP == 4, "queries per lane assume four searches side by side");

// K3 for a whole batch.  Warp w takes curve c = w / tiles and tile t = w %
// tiles: the 32 qpl queries at ranks 32 qpl t .. of curve c's key order, lane
// l the ranks 32 qpl t + 32 u + l (u < qpl, qpl queries per lane).  Each lane
// searches its queries' curve-c keys in list j * curves + c of every
// partition j and writes the position to pos[query][c * partitions + j].  The
// 32 keys of a warp's round are neighbours on curve c, so the lanes' probes
// fall on the same few lines (one request serves many lanes) where lanes of a
// per-query warp would each probe a different list.
template <int QPL>   // batch_queries_per_lane(partitions)
__global__ void __launch_bounds__(256) batch_positions_kernel(IndexView ix, uint32_t nq,
                                                              const uint32_t* __restrict__ order,
                                                              const uint64_t* __restrict__ qhi,
                                                              const uint64_t* __restrict__ qlo,
                                                              uint32_t* __restrict__ pos) {
    constexpr int G = kBatchILP;
    constexpr uint32_t qpl = QPL;
    const int lane = threadIdx.x & 31;
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t curves = ix.P.curves, parts = ix.lists / curves;
    const uint32_t span = 32 * qpl;
    const uint32_t tiles = (uint32_t)(((uint64_t)nq + span - 1) / span);
    if (w >= (uint64_t)tiles * curves) return;
    const uint32_t c = (uint32_t)(w / tiles), t = (uint32_t)(w % tiles);
    // the lane's queries; lanes past the batch search with query 0's key and
    // write nothing
    uint32_t qi[QPL];
    bool live[QPL];
    uint64_t kh[QPL], kl[QPL];
#pragma unroll
    for (int u = 0; u < QPL; ++u) {
        const uint32_t r = t * span + (uint32_t)u * 32 + (uint32_t)lane;
        live[u] = r < nq;
        qi[u] = live[u] ? __ldg(order + (size_t)c * nq + r) : 0u;
        if (live[u] && !HC_IN_BOUNDS(kSiteQuery, qi[u], nq)) {
            live[u] = false;
            qi[u] = 0;
        }
        kh[u] = __ldg(qhi + (size_t)c * nq + qi[u]);
        kl[u] = __ldg(qlo + (size_t)c * nq + qi[u]);
    }
    uint32_t lists[G], at[G];
    bool on[G];
    uint64_t gh[G], gl[G];
    if constexpr (QPL > 1) {
        // one round: search g is partition g % (G / QPL) of query g / (G / QPL)
        constexpr int PP = G / QPL;   // partitions (1 or 2)
#pragma unroll
        for (int g = 0; g < G; ++g) {
            on[g] = live[g / PP];
            gh[g] = kh[g / PP];
            gl[g] = kl[g / PP];
            lists[g] = (uint32_t)(g % PP) * curves + c;
        }
        lower_bound_lists<G>(ix, lists, on, gh, gl, at);
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (on[g])
                pos[(size_t)qi[g / PP] * ix.lists + (size_t)c * PP + (uint32_t)(g % PP)] = at[g];
        return;
    }
    uint32_t* out = pos + (size_t)qi[0] * ix.lists + (size_t)c * parts;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        gh[g] = kh[0];
        gl[g] = kl[0];
    }
    // G partitions at a time: their searches share the key
    for (uint32_t j0 = 0; j0 < parts; j0 += G) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            on[g] = j0 + g < parts;
            lists[g] = on[g] ? (j0 + g) * curves + c : 0u;
        }
        lower_bound_lists<G>(ix, lists, on, gh, gl, at);
        if (!live[0]) continue;
        if (parts % G == 0) {
            // whole groups: one vector store (the row offset is a multiple
            // of the group since partitions are)
            store_group(out + j0, at);
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (on[g]) out[j0 + g] = at[g];
        }
    }
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

// fence[j] = keys_hi[16 j] & kFenceMask: one thread per fence word
__global__ void __launch_bounds__(256) fence_kernel(const uint64_t* __restrict__ keys_hi,
                                                    uint64_t len, uint64_t* __restrict__ fence) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += stride)
        fence[j] = __ldg(keys_hi + (j << kFenceShift)) & kFenceMask;
}

template <bool F32, int LPR, int KR>
struct QueryLaunch {
    template <bool STAGED>
    static cudaError_t go(const QueryArgs& a, size_t smem, cudaStream_t s) {
        const unsigned blocks = (unsigned)(((uint64_t)a.nq + kQWarps - 1) / kQWarps);
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
                         const uint32_t* order, const uint32_t* pos_cm) {
    if (nq == 0) return cudaSuccess;
    QueryArgs a{ix, q, nq, k, p, out_ids, out_dist, nullptr, p_query, pos_in, order, pos_cm};
    return dispatch<QueryLaunch>(ix.P.dtype == HC_F32, lanes_per_row(ix.row_bytes), regs_for_k(k),
                                 a, s);
}

cudaError_t launch_order_keys(const IndexView& ix, const void* q, uint32_t nq, uint32_t ncurves,
                              uint64_t* keys, uint64_t* qhi, uint64_t* qlo, cudaStream_t s) {
    if (nq == 0 || ncurves == 0) return cudaSuccess;
    order_keys_kernel<<<(unsigned)(((uint64_t)nq + 255) / 256), 256, 0, s>>>(ix, static_cast<const uint8_t*>(q), nq,
                                                       ncurves, keys, qhi, qlo);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batch_positions(const IndexView& ix, uint32_t nq, const uint32_t* order,
                                   const uint64_t* qhi, const uint64_t* qlo, uint32_t* pos,
                                   cudaStream_t s) {
    const uint32_t qpl = batch_queries_per_lane(ix.lists / ix.P.curves), span = 32 * qpl;
    const uint64_t warps = (((uint64_t)nq + span - 1) / span) * ix.P.curves;
    if (warps == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    if (qpl == 4)
        batch_positions_kernel<4><<<blocks, 256, 0, s>>>(ix, nq, order, qhi, qlo, pos);
    else if (qpl == 2)
        batch_positions_kernel<2><<<blocks, 256, 0, s>>>(ix, nq, order, qhi, qlo, pos);
    else
        batch_positions_kernel<1><<<blocks, 256, 0, s>>>(ix, nq, order, qhi, qlo, pos);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fence(const uint64_t* keys_hi, uint64_t total, uint64_t* fence,
                         cudaStream_t s) {
    const uint64_t len = (total + 15) >> kFenceShift;
    if (len == 0) return cudaSuccess;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (len + 255) / 256, cap = (uint64_t)std::max(sms, 1) * 8;
    fence_kernel<<<(unsigned)std::min(want, cap), 256, 0, s>>>(keys_hi, len, fence);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_positions(const IndexView& ix, const void* q, uint32_t nq, int64_t* pos,
                             cudaStream_t s) {
    if (nq == 0) return cudaSuccess;
    QueryArgs a{ix, q, nq, 1, 0, nullptr, nullptr, pos, nullptr, nullptr, nullptr};
    const unsigned blocks = (unsigned)(((uint64_t)nq + kQWarps - 1) / kQWarps);
    positions_kernel<<<blocks, kQWarps * 32, sizeof(uint32_t) * kQWarps * ix.lists, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hc
