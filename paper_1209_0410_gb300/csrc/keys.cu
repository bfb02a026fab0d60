// K1: Hilbert extended-keys of database rows (Algorithm 1, per-curve step)
// and of standalone vectors.  One thread per row computes the keys of every
// curve, four 16-coordinate keys at a time as byte lanes of 32-bit words;
// the Hilbert map itself is ALU work, and for an index that keeps high words
// only, just the levels that decide bit planes 7..4 are run.  The row read
// and the key words written are coalesced across the warp.
#include "hc_internal.h"

namespace hc {

__global__ void __launch_bounds__(256) build_keys_kernel(BuildKeysArgs a) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += stride) {
        const uint32_t part = partition_of(r, a.n, a.partitions);
        const uint64_t local = r - partition_start(part, a.n, a.partitions);
        const void* row = static_cast<const uint8_t*>(a.db) + r * a.row_bytes;
        uint32_t c = 0;
        if (a.P.m == 16 && a.P.dim_map == nullptr) {
            // four curves at a time, SIMD within a register
            for (; c + 4 <= a.P.curves; c += 4) {
                uint4 cb[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) cb[t] = curve_bytes16(row, a.P.dtype, c + t);
                uint64_t hi[4], lo[4];
                if (a.lo)
                    hilbert_keys4<false>(cb, hi, lo);
                else
                    hilbert_keys4<true>(cb, hi, lo);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint64_t g = a.list_off[part * a.P.curves + c + t] + local;
                    if (!HC_IN_BOUNDS(kSiteKeySlot, g, a.list_off[a.partitions * a.P.curves]))
                        continue;
                    a.hi[g] = hi[t];
                    if (a.lo) a.lo[g] = lo[t];
                    if (a.ids) a.ids[g] = (uint32_t)r;
                    if (a.digits) a.digits[g] = (uint8_t)(hi[t] >> a.digit_shift);
                }
            }
        }
        for (; c < a.P.curves; ++c) {
            uint64_t hi, lo;
            curve_key(row, a.P, c, hi, lo);
            const uint64_t g = a.list_off[part * a.P.curves + c] + local;
            if (!HC_IN_BOUNDS(kSiteKeySlot, g, a.list_off[a.partitions * a.P.curves])) continue;
            a.hi[g] = hi;
            if (a.lo) a.lo[g] = lo;
            if (a.ids) a.ids[g] = (uint32_t)r;
            if (a.digits) a.digits[g] = (uint8_t)(hi >> a.digit_shift);
        }
    }
}

__global__ void __launch_bounds__(256) vector_keys_kernel(const void* x, uint64_t count,
                                                          uint32_t row_bytes, Projection P,
                                                          uint64_t* hi, uint64_t* lo) {
    const uint64_t total = count * P.curves;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t v = t / P.curves;
        const uint32_t c = (uint32_t)(t % P.curves);
        uint64_t h, l;
        curve_key(static_cast<const uint8_t*>(x) + v * row_bytes, P, c, h, l);
        hi[t] = h;
        lo[t] = l;
    }
}

// low key words of every entry of an index that keeps high words only
// (grid y = list)
__global__ void __launch_bounds__(256) entry_lo_kernel(IndexView ix, uint64_t* __restrict__ out) {
    const uint32_t L = blockIdx.y;
    const uint64_t off = ix.list_off[L], n = ix.list_off[L + 1] - off;
    const uint32_t c = L % ix.P.curves;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[off + i] = row_key_lo(ix.db, ix.row_bytes, ix.P, __ldg(ix.ids + off + i), c);
}

static unsigned grid_for(uint64_t work, unsigned threads) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (work + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sms * 16;   // grid-stride beyond 16 waves of 256
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

cudaError_t launch_build_keys(const BuildKeysArgs& a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    build_keys_kernel<<<grid_for(a.n, 256), 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_vector_keys(const void* x, uint64_t count, uint32_t row_bytes,
                               const Projection& P, uint64_t* hi, uint64_t* lo, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    vector_keys_kernel<<<grid_for(count * P.curves, 256), 256, 0, s>>>(x, count, row_bytes, P, hi,
                                                                       lo);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_entry_lo(const IndexView& ix, uint64_t* out, cudaStream_t s) {
    if (ix.lists == 0) return cudaSuccess;
    entry_lo_kernel<<<dim3(64, ix.lists), 256, 0, s>>>(ix, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hc
