// hc_sort_keys_noalloc: the segmented 128-bit key sort of sort.cu run on a
// fixed scratch area that lives inside this library's device image, for
// callers that must not have the library allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a process whose memory
// manager has already reserved the whole device (a further cudaMalloc would
// fail or break its budget), or a latency-sensitive caller that cannot take
// the implicit device synchronisation of cudaMalloc/cudaFree.  For them the
// scratch below is a file-scope device array: every GPU on which the library
// is loaded holds it (kNoAllocScratchBytes) until the process exits.
#include <mutex>

#include "hc_internal.h"

namespace {

constexpr uint64_t kNoAllocMaxRecords = 1ull << 18;   // 262,144 records per call
constexpr uint32_t kNoAllocMaxSegments = 256;
constexpr size_t kNoAllocScratchBytes = 10ull << 20;  // 10 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device (the first
// call on a device, with that device current).  In host code the array's
// name only stands in for the symbol; handing it to a kernel would not give
// the device address.  The module holding the array is loaded on a device
// by that first lookup (lazy module loading), so that is when the array's
// memory is taken; the cached address does not survive cudaDeviceReset.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return HC_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return HC_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return HC_OK;
}

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" HC_API int hc_sort_keys_noalloc(uint64_t* hi_dev, uint64_t* lo_dev, uint32_t* ids_dev,
                                          const uint64_t* seg_off_host, uint32_t nseg,
                                          uint32_t key_bits, void* cuda_stream) {
    using namespace hc;
    if (!seg_off_host || nseg < 1 || key_bits < 1 || key_bits > 128) return HC_ERR_ARG;
    if (nseg > kNoAllocMaxSegments) return HC_ERR_ARG;
    if (seg_off_host[0] != 0) return HC_ERR_ARG;
    for (uint32_t i = 0; i < nseg; ++i)
        if (seg_off_host[i + 1] < seg_off_host[i]) return HC_ERR_ARG;
    const uint64_t total = seg_off_host[nseg];
    if (total > kNoAllocMaxRecords) return HC_ERR_ARG;
    // the per-device set-up comes first, so that a call with no records does it
    void* base = nullptr;
    if (int rc = scratch_address(&base)) return rc;
    if (total == 0) return HC_OK;
    if (!on_device(hi_dev) || !on_device(lo_dev) || !on_device(ids_dev)) return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // scratch layout: sorted outputs | segment offsets | sort working area
    SortProblem sp;
    sp.hi = hi_dev;
    sp.lo = lo_dev;
    sp.ids = ids_dev;
    sp.seg_off.assign(seg_off_host, seg_off_host + nseg + 1);
    sp.key_bits = key_bits;
    const size_t out_bytes = round256((sizeof(uint64_t) * 2 + sizeof(uint32_t)) * total);
    const size_t off_bytes = round256(sizeof(uint64_t) * (nseg + 1));
    const size_t need = out_bytes + off_bytes + sort_scratch_bytes(sp);
    if (need > kNoAllocScratchBytes) return HC_ERR_ARG;
    char* b = static_cast<char*>(base);
    sp.out_hi = reinterpret_cast<uint64_t*>(b);
    sp.out_lo = sp.out_hi + total;
    sp.out_ids = reinterpret_cast<uint32_t*>(sp.out_lo + total);
    uint64_t* off_dev = reinterpret_cast<uint64_t*>(b + out_bytes);
    sp.seg_off_dev = off_dev;

    // Nothing in the scratch has to start at zero: every count, offset and
    // buffer the sort reads is written earlier in the same call.
    if (cudaError_t e = upload_small(off_dev, seg_off_host, sizeof(uint64_t) * (nseg + 1), s))
        return e == cudaErrorMemoryAllocation ? HC_ERR_OOM : HC_ERR_CUDA;
    if (int rc = sort_segments(sp, b + out_bytes + off_bytes, s)) return rc;
    if (cudaMemcpyAsync(hi_dev, sp.out_hi, 8 * total, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(lo_dev, sp.out_lo, 8 * total, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ids_dev, sp.out_ids, 4 * total, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HC_ERR_CUDA;
    return HC_OK;
}
