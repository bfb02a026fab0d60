// Exact kNN (Eq. 3) over every row of the database: the ground truth for
// recall, with the same distance and top-k code as the query kernel.
#include "hc_dispatch.cuh"
#include "hc_internal.h"
#include "hc_query_dev.cuh"
#include "hc_topk.cuh"

namespace hc {

namespace {

constexpr int kQWarps = 8;

// Exact kNN: every row of the database, 32 rows per step, same distance and
// top-k code as the query kernel.
template <bool F32, int LPR, int KR>
__global__ void __launch_bounds__(kQWarps * 32) brute_kernel(const uint8_t* __restrict__ db,
                                                            uint64_t n, uint32_t row_bytes,
                                                            const uint8_t* __restrict__ q,
                                                            uint32_t nq, uint32_t k,
                                                            int32_t* out_ids, void* out_dist) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t qi = blockIdx.x * kQWarps + warp;
    if (qi >= nq) return;
    const uint8_t* qrow = q + (size_t)qi * row_bytes;
    const uint32_t s = (uint32_t)lane % LPR;
    const uint4 qv0 = s < (row_bytes >> 4) ? ldg16(qrow + s * 16) : make_uint4(0, 0, 0, 0);
    WarpTopK<KR> top;
    top.init();
    for (uint64_t base = 0; base < n; base += 32) {
        const uint32_t cnt = n - base < 32 ? (uint32_t)(n - base) : 32u;
        const uint32_t id = (uint32_t)(base + lane);
        uint64_t cand[ChunkWidth<LPR>::NG];
        chunk_candidates_n<F32, LPR>(db, row_bytes, qrow, qv0, id, cnt, lane, cand);
#pragma unroll
        for (int c = 0; c < ChunkWidth<LPR>::NG; ++c) top.offer(cand[c], k, lane);
    }
    top.template store<F32>(k, lane, out_ids + (size_t)qi * k,
                            static_cast<uint32_t*>(out_dist) + (size_t)qi * k);
}

template <bool F32, int LPR, int KR>
struct BruteLaunch {
    static cudaError_t run(const uint8_t* db, uint64_t n, uint32_t row_bytes, const uint8_t* q,
                           uint32_t nq, uint32_t k, int32_t* ids, void* dist, cudaStream_t s) {
        const unsigned blocks = (nq + kQWarps - 1) / kQWarps;
        brute_kernel<F32, LPR, KR><<<blocks, kQWarps * 32, 0, s>>>(db, n, row_bytes, q, nq, k,
                                                                   ids, dist);
        count_launches(1);
        return cudaGetLastError();
    }
};

}  // namespace

cudaError_t launch_bruteforce(const void* db, hc_dtype dtype, uint64_t n, uint32_t d,
                              const void* q, uint32_t nq, uint32_t k, int32_t* out_ids,
                              void* out_dist, cudaStream_t s) {
    if (nq == 0) return cudaSuccess;
    const uint32_t row_bytes = dtype == HC_F32 ? d * 4 : d;
    return dispatch<BruteLaunch>(dtype == HC_F32, lanes_per_row(row_bytes), regs_for_k(k),
                                 static_cast<const uint8_t*>(db), n, row_bytes,
                                 static_cast<const uint8_t*>(q), nq, k, out_ids, out_dist, s);
}

}  // namespace hc
