// The C ABI of include/hc.h: argument checks, ownership and allocation
// around the kernels of keys.cu (K1), sort.cu (K2) and query.cu (K3..K6).
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "hc_index.h"
#include "hc_trace.h"

using namespace hc;


static std::atomic<uint64_t> g_launches{0};

namespace hc {
void count_launches(uint64_t n) { g_launches.fetch_add(n); }
// true when p is page-locked host memory (cudaHostAlloc / cudaHostRegister)
bool is_pinned_host(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

}  // namespace hc

namespace {

// Host-side fault injection for tests: the allocation numbered fail_after
// (0-based, counted from the hc_debug_fail_alloc call) reports OOM.
std::atomic<long> g_fail_after{-1};
std::atomic<long> g_alloc_count{0};

bool injected_failure() {
    const long after = g_fail_after.load();
    if (after < 0) return false;
    return g_alloc_count.fetch_add(1) == after;
}

}  // namespace

bool hc::alloc_should_fail() { return injected_failure(); }

namespace hc {

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return HC_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return HC_ERR_OOM;
    }
    return HC_ERR_CUDA;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// true when p is device memory of the current device (or managed)
bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace hc

namespace {

#ifdef HC_CHECK
// Checked build: every stream-ordered buffer is followed by a guard of
// kGuardBytes bytes of kGuardByte, checked on the device before the buffer is
// freed and on the host by hc_check_status.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
std::mutex g_guard_mu;
std::unordered_map<void*, size_t> g_guards;   // buffer -> bytes before its guard

__global__ void guard_check_kernel(const unsigned char* g, uint32_t n) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
        if (g[i] != kGuardByte) hc::check_index(kSitePad, i, 0);
}
#endif

int dev_alloc_async(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (injected_failure()) return HC_ERR_OOM;
    if (bytes == 0) bytes = 16;
#ifdef HC_CHECK
    if (int rc = status_of(cudaMallocAsync(p, bytes + kGuardBytes, s))) return rc;
    {
        std::lock_guard<std::mutex> g(g_guard_mu);
        g_guards[*p] = bytes;
    }
    return status_of(cudaMemsetAsync(static_cast<char*>(*p) + bytes, kGuardByte, kGuardBytes, s));
#else
    return status_of(cudaMallocAsync(p, bytes, s));
#endif
}

void keep_pool_memory() {
    // stream-ordered scratch stays in the memory pool (not released to CUDA)
    // between builds of this process
    static std::atomic<bool> done{false};
    if (done.exchange(true)) return;
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}

uint32_t row_bytes_of(hc_dtype t, uint32_t d) { return t == HC_F32 ? d * 4u : d; }

int check_params(const hc_build_params* p) {
    if (!p) return HC_ERR_ARG;
    if (p->dtype != HC_U8 && p->dtype != HC_F32) return HC_ERR_ARG;
    if (p->n < 1 || p->n >= (1ull << 31)) return HC_ERR_ARG;
    if (p->d < 1 || p->d > 4096) return HC_ERR_ARG;
    if (row_bytes_of(p->dtype, p->d) % 16 != 0) return HC_ERR_ARG;
    if (p->curves < 1 || p->curves > 32) return HC_ERR_ARG;
    if (p->dims_per_curve < 1 || p->dims_per_curve > 16) return HC_ERR_ARG;
    if (p->bits != 8) return HC_ERR_ARG;
    const uint32_t parts = p->partitions ? p->partitions : 1;
    if ((uint64_t)parts * p->curves > 256) return HC_ERR_ARG;
    if ((uint64_t)p->curves * p->n >= (1ull << 32)) return HC_ERR_ARG;
    if (p->dim_map) {
        for (uint32_t i = 0; i < p->curves * p->dims_per_curve; ++i)
            if (p->dim_map[i] >= p->d) return HC_ERR_ARG;
    } else if ((uint64_t)p->curves * p->dims_per_curve > p->d) {
        return HC_ERR_ARG;
    }
    return HC_OK;
}


// The index arrays come from the stream-ordered pool and are released in
// stream order, so build/free cycles reuse pool memory without device syncs.
// By default on the legacy stream, which waits for the work of every blocking
// stream (safe whatever stream used the index); hc_free_async names the stream.
cudaError_t pool_free(void* p, cudaStream_t s = cudaStreamLegacy) {
    if (!p) return cudaSuccess;
#ifdef HC_CHECK
    size_t body = 0;
    {
        std::lock_guard<std::mutex> g(g_guard_mu);
        auto it = g_guards.find(p);
        if (it != g_guards.end()) {
            body = it->second;
            g_guards.erase(it);
        }
    }
    if (body) {
        guard_check_kernel<<<1, 256, 0, s>>>(static_cast<const unsigned char*>(p) + body,
                                             (uint32_t)kGuardBytes);
        count_launches(1);
    }
#endif
    return cudaFreeAsync(p, s);
}

}  // namespace

namespace hc {

static std::mutex g_readers_mu;
static std::vector<CheckReader>& check_readers() {
    static std::vector<CheckReader> v;
    return v;
}

void register_check_reader(CheckReader r) {
    std::lock_guard<std::mutex> g(g_readers_mu);
    check_readers().push_back(r);
}

void index_destroy(hc_index* x, cudaStream_t s) {
    if (!x) return;
    pool_free(x->dim_map_dev, s);
    pool_free(x->db_owned, s);
    pool_free(x->keys_hi, s);
    pool_free(x->keys_lo, s);
    pool_free(x->ids, s);
    pool_free(x->fence, s);
    pool_free(x->list_off_dev, s);
    pool_free(x->st_q, s);
    pool_free(x->st_out, s);
    if (x->st_done) cudaEventDestroy(x->st_done);
    cudaGetLastError();
    delete x;
}

void index_layout(hc_index* x) {
    const hc_build_params& P = x->params;
    const uint32_t parts = P.partitions;
    x->lists = parts * P.curves;
    x->row_bytes = row_bytes_of(P.dtype, P.d);
    x->list_off.assign(x->lists + 1, 0);
    for (uint32_t L = 0; L < x->lists; ++L) {
        const uint32_t j = L / P.curves;
        const uint64_t len = partition_start(j + 1, P.n, parts) - partition_start(j, P.n, parts);
        x->list_off[L + 1] = x->list_off[L] + len;
    }
}

bool index_keeps_lo(const hc_build_params& P) { return P.dims_per_curve < 16; }

int index_alloc(hc_index* x, cudaStream_t s) {
    const uint64_t total = x->list_off[x->lists];
    int rc;
    keep_pool_memory();
    if ((rc = dev_alloc_async((void**)&x->list_off_dev, sizeof(uint64_t) * (x->lists + 1), s)))
        return rc;
    if (!x->dim_map.empty()) {
        if ((rc = dev_alloc_async((void**)&x->dim_map_dev,
                                  sizeof(uint32_t) * (x->dim_map.size() + 1), s)))
            return rc;
        if ((rc = status_of(upload_small(x->dim_map_dev, x->dim_map.data(),
                                         sizeof(uint32_t) * x->dim_map.size(), s))))
            return rc;
    }
    if ((rc = status_of(upload_small(x->list_off_dev, x->list_off.data(),
                                     sizeof(uint64_t) * (x->lists + 1), s))))
        return rc;
    if ((rc = dev_alloc_async((void**)&x->keys_hi, sizeof(uint64_t) * total, s))) return rc;
    if (index_keeps_lo(x->params) &&
        (rc = dev_alloc_async((void**)&x->keys_lo, sizeof(uint64_t) * total, s)))
        return rc;
    if (total > 0 && (rc = dev_alloc_async((void**)&x->fence,
                                           sizeof(uint64_t) * ((total + 15) >> kFenceShift), s)))
        return rc;
    return dev_alloc_async((void**)&x->ids, sizeof(uint32_t) * total, s);
}

int index_new(const void* db, const hc_build_params* params, hc_index** out, hc_index** made) {
    *made = nullptr;
    if (!out) return HC_ERR_ARG;
    *out = nullptr;
    if (int rc = check_params(params)) return rc;
    hc_index* x = new (std::nothrow) hc_index();
    if (!x) return HC_ERR_OOM;
    x->params = *params;
    if (!x->params.partitions) x->params.partitions = 1;
    if (params->dim_map)
        x->dim_map.assign(params->dim_map, params->dim_map + params->curves * params->dims_per_curve);
    x->params.dim_map = nullptr;
    x->db = db;
    *made = x;
    return HC_OK;
}

}  // namespace hc

namespace {

// Algorithm 1 for an index whose params, db and dim_map are set.
int build_index(hc_index* x, cudaStream_t s) {
    const hc_build_params& P = x->params;
    const uint32_t parts = P.partitions;
    index_layout(x);
    const uint64_t total = x->list_off[x->lists];
    // 16-coordinate keys: the high word holds 64 key bits and ties of it are
    // rare, so the index keeps high words only and recomputes a low word from
    // its row when a tie needs it (12 instead of 20 bytes per entry)
    const bool keep_lo = index_keeps_lo(P);
    int rc;
    if ((rc = index_alloc(x, s))) return rc;
    // ids are implied by the slot: list L holds its partition's rows in id
    // order before the sort, so id = partition start + (slot - list start)
    std::vector<uint64_t> id_base(x->lists);
    for (uint32_t L = 0; L < x->lists; ++L)
        id_base[L] = partition_start(L / P.curves, P.n, parts);
    // 16-coordinate keys: the top 6 bytes of the high words are radix-sorted,
    // the last pass writing the final high words and ids, and runs of equal
    // 48-bit prefixes are ordered by (high word, low word, id) on the device,
    // the low words recomputed from the rows where two high words tie.
    // Shorter keys: every key byte is sorted (the low words are stored).
    // Neither waits on the host.
    SortProblem sp;
    sp.seg_off = x->list_off;
    sp.seg_off_dev = x->list_off_dev;
    sp.key_bits = 8 * P.dims_per_curve;
    sp.allow_sync = false;
    sp.hi_skip = keep_lo ? 0 : 2;
    sp.out_hi = x->keys_hi;
    sp.out_lo = x->keys_lo;
    sp.out_ids = x->ids;
    sp.out_fence = x->fence;
    const size_t sort_bytes = sort_scratch_bytes(sp);
    const size_t key_bytes = ((sizeof(uint64_t) * (keep_lo ? 2 : 1) * total) + 255) & ~(size_t)255;
    const size_t base_bytes = (sizeof(uint64_t) * x->lists + 255) & ~(size_t)255;
    void* scratch = nullptr;
    if ((rc = dev_alloc_async(&scratch, key_bytes + base_bytes + sort_bytes, s))) return rc;
    uint64_t* hi0 = static_cast<uint64_t*>(scratch);
    uint64_t* lo0 = keep_lo ? hi0 + total : nullptr;
    uint64_t* id_base_dev = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + key_bytes);
    void* sort_scratch = static_cast<char*>(scratch) + key_bytes + base_bytes;

    sp.hi = hi0;
    sp.lo = lo0;
    sp.ids = nullptr;
    sp.id_base_dev = id_base_dev;
    sp.rows = RowKeys{x->db, x->row_bytes, view_of(x).P};
    // the key pass also leaves the first radix pass's digit bytes, so that
    // pass's histogram reads bytes instead of words
    const FirstDigits fd = sort_first_digits(sp, sort_scratch);
    sp.first_digits_ready = fd.buf != nullptr;
    BuildKeysArgs ka{x->db, P.n, x->row_bytes, view_of(x).P, parts, x->list_off_dev, hi0, lo0,
                     nullptr, fd.buf, fd.shift};
    {
        TraceRange tk("keys");
        rc = status_of(launch_build_keys(ka, s));
    }
    if (rc == HC_OK)
        rc = status_of(upload_small(id_base_dev, id_base.data(), sizeof(uint64_t) * x->lists, s));
    if (rc == HC_OK) {
        TraceRange ts("sort");
        rc = sort_segments(sp, sort_scratch, s);
    }
    const int frc = status_of(pool_free(scratch, s));
    return rc ? rc : frc;
}

}  // namespace

extern "C" {

HC_API const char* hc_strerror(int status) {
    switch (status) {
        case HC_OK: return "ok";
        case HC_PENDING: return "pending";
        case HC_ERR_ARG: return "invalid argument";
        case HC_ERR_OOM: return "out of memory";
        case HC_ERR_CUDA: return "CUDA runtime error";
        case HC_ERR_BUDGET: return "admission refused: over the memory budget";
        case HC_ERR_TIMEOUT: return "timed out";
        case HC_ERR_DEVICE_STATUS: return "a kernel reported an error status";
        case HC_ERR_STATE: return "object in the wrong state";
        case HC_ERR_IO: return "file input/output failed";
        case HC_ERR_FORMAT: return "not a valid index file for this database";
        default: return "unknown status";
    }
}

HC_API int hc_build(const void* db_dev, const hc_build_params* params, void* cuda_stream,
                    hc_index** out) {
    TraceRange tr("hc_build");
    hc_index* x;
    if (int rc = index_new(db_dev, params, out, &x)) return rc;
    if (!is_device_ptr(db_dev) || !aligned16(db_dev)) {
        index_destroy(x);
        return HC_ERR_ARG;
    }
    const int rc = build_index(x, static_cast<cudaStream_t>(cuda_stream));
    if (rc) {
        cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
        index_destroy(x);
        return rc;
    }
    *out = x;
    return HC_OK;
}

HC_API int hc_build_host(const void* db_host, const hc_build_params* params, void* cuda_stream,
                         hc_index** out) {
    TraceRange tr("hc_build_host");
    if (!db_host) return HC_ERR_ARG;
    hc_index* x;
    if (int rc = index_new(nullptr, params, out, &x)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t bytes = (size_t)params->n * row_bytes_of(params->dtype, params->d);
    keep_pool_memory();
    int rc = dev_alloc_async(&x->db_owned, bytes, s);
    if (!rc) rc = status_of(cudaMemcpyAsync(x->db_owned, db_host, bytes, cudaMemcpyHostToDevice, s));
    x->db = x->db_owned;
    if (!rc) rc = build_index(x, s);
    const int src = status_of(cudaStreamSynchronize(s));
    if (!rc) rc = src;
    if (rc) {
        index_destroy(x);
        return rc;
    }
    *out = x;
    return HC_OK;
}

HC_API int hc_build_host_async(const void* db_host, const hc_build_params* params,
                               void* copy_stream, void* cuda_stream, hc_index** out) {
    TraceRange tr("hc_build_host_async");
    hc_index* x;
    if (int rc = index_new(nullptr, params, out, &x)) return rc;
    if (!is_pinned_host(db_host)) {
        index_destroy(x);
        return HC_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaStream_t cs = copy_stream ? static_cast<cudaStream_t>(copy_stream) : s;
    const size_t bytes = (size_t)params->n * row_bytes_of(params->dtype, params->d);
    keep_pool_memory();
    // the rows' buffer is allocated in the copy stream's order, so the upload
    // waits for nothing queued on cuda_stream; the build waits for the upload
    int rc = dev_alloc_async(&x->db_owned, bytes, cs);
    x->db = x->db_owned;
    cudaEvent_t landed = nullptr;
    if (!rc) {
        TraceRange tc("upload");
        rc = status_of(cudaMemcpyAsync(x->db_owned, db_host, bytes, cudaMemcpyHostToDevice, cs));
    }
    if (!rc && cs != s) {
        rc = status_of(cudaEventCreateWithFlags(&landed, cudaEventDisableTiming));
        if (!rc) rc = status_of(cudaEventRecord(landed, cs));
        if (!rc) rc = status_of(cudaStreamWaitEvent(s, landed, 0));
    }
    // destroying a recorded event is allowed: it is released once it completes
    if (landed) cudaEventDestroy(landed);
    if (!rc) rc = build_index(x, s);
    if (rc) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(s);
        index_destroy(x);
        return rc;
    }
    *out = x;
    return HC_OK;
}

HC_API void hc_free(hc_index* idx) { index_destroy(idx); }

HC_API void hc_free_async(hc_index* idx, void* cuda_stream) {
    index_destroy(idx, static_cast<cudaStream_t>(cuda_stream));
}

HC_API int hc_query(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k, uint32_t p,
                    int32_t* out_ids_dev, void* out_dist_dev, void* cuda_stream) {
    TraceRange tr("hc_query");
    if (!idx || k < 1 || k > 128 || p > (1u << 30)) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!q_dev || !out_ids_dev || !out_dist_dev || !aligned16(q_dev)) return HC_ERR_ARG;
    if (!is_device_ptr(q_dev) || !is_device_ptr(out_ids_dev) || !is_device_ptr(out_dist_dev))
        return HC_ERR_ARG;
    return status_of(launch_query(view_of(idx), q_dev, nq, k, p, out_ids_dev, out_dist_dev,
                                  static_cast<cudaStream_t>(cuda_stream)));
}

HC_API int hc_query_depths(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k,
                           const uint32_t* p_dev, int32_t* out_ids_dev, void* out_dist_dev,
                           void* cuda_stream) {
    TraceRange tr("hc_query_depths");
    if (!idx || k < 1 || k > 128) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!q_dev || !p_dev || !out_ids_dev || !out_dist_dev || !aligned16(q_dev)) return HC_ERR_ARG;
    if (!is_device_ptr(q_dev) || !is_device_ptr(p_dev) || !is_device_ptr(out_ids_dev) ||
        !is_device_ptr(out_dist_dev))
        return HC_ERR_ARG;
    return status_of(launch_query(view_of(idx), q_dev, nq, k, 0, out_ids_dev, out_dist_dev,
                                  static_cast<cudaStream_t>(cuda_stream), p_dev));
}

HC_API int hc_query_at(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k, uint32_t p,
                       const int64_t* pos_dev, int32_t* out_ids_dev, void* out_dist_dev,
                       void* cuda_stream) {
    TraceRange tr("hc_query_at");
    if (!idx || k < 1 || k > 128 || p > (1u << 30)) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!q_dev || !pos_dev || !out_ids_dev || !out_dist_dev || !aligned16(q_dev))
        return HC_ERR_ARG;
    if (!is_device_ptr(q_dev) || !is_device_ptr(pos_dev) || !is_device_ptr(out_ids_dev) ||
        !is_device_ptr(out_dist_dev))
        return HC_ERR_ARG;
    return status_of(launch_query(view_of(idx), q_dev, nq, k, p, out_ids_dev, out_dist_dev,
                                  static_cast<cudaStream_t>(cuda_stream), nullptr, pos_dev));
}

}  // extern "C"

namespace {

// Workspace of hc_query_ordered for nq queries: the order keys of every
// curve, the segment table (a segment per curve, at most 32: one small
// upload), the sorted keys and the permutations (curve 0's first: the walk
// order), the query keys and the positions of the batch search, then the
// sort's own scratch.
struct OrderLayout {
    size_t keys = 0, seg = 0, out_hi = 0, out_lo = 0, order = 0, qhi = 0, qlo = 0, pos = 0,
           sort = 0, bytes = 0;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// hc_query_host answers batches of at least this many queries in key order
constexpr uint32_t kHostOrderedMin = 4096;

// one segment of nq order keys per sorted curve
SortProblem order_problem(uint32_t nq, uint32_t ncurves) {
    SortProblem sp;
    sp.seg_off.resize(ncurves + 1);
    for (uint32_t c = 0; c <= ncurves; ++c) sp.seg_off[c] = (uint64_t)c * nq;
    sp.key_bits = kOrderBits;
    sp.allow_sync = false;   // no stream wait: every key byte is sorted
    return sp;
}

OrderLayout order_layout(const hc_index* idx, uint32_t nq) {
    OrderLayout L;
    const uint32_t curves = idx->params.curves;
    const uint64_t r = (uint64_t)nq * curves;
    size_t o = 0;
    L.keys = o;    o = align256(o + 8 * r);
    L.seg = o;     o = align256(o + 8 * (2 * curves + 1));   // seg_off, then id_base
    L.out_hi = o;  o = align256(o + 8 * r);
    L.out_lo = o;  o = align256(o + 8 * r);
    L.order = o;   o = align256(o + 4 * r);
    L.qhi = o;     o = align256(o + 8 * r);
    L.qlo = o;     o = align256(o + 8 * r);
    L.pos = o;     o = align256(o + 4ull * nq * idx->lists);
    L.sort = o;    o = align256(o + sort_scratch_bytes(order_problem(nq, curves)));
    L.bytes = o;
    return L;
}

// hc_query_ordered's work on a checked workspace of order_layout(idx, nq).bytes:
// the order keys, their sort, the batch search, then the walk in curve-0 order.
int enqueue_ordered(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k, uint32_t p,
                    int32_t* out_ids_dev, void* out_dist_dev, char* ws, cudaStream_t s) {
    const OrderLayout L = order_layout(idx, nq);
    const uint32_t curves = idx->params.curves;
    uint64_t* keys = reinterpret_cast<uint64_t*>(ws + L.keys);
    uint64_t* seg = reinterpret_cast<uint64_t*>(ws + L.seg);
    uint64_t* qhi = reinterpret_cast<uint64_t*>(ws + L.qhi);
    uint64_t* qlo = reinterpret_cast<uint64_t*>(ws + L.qlo);
    uint32_t* pos = reinterpret_cast<uint32_t*>(ws + L.pos);
    const IndexView v = view_of(idx);
    int rc = status_of(launch_order_keys(v, q_dev, nq, curves, keys, qhi, qlo, s));
    std::vector<uint64_t> small(2 * curves + 1, 0);   // seg_off, then id_base = 0
    for (uint32_t c = 0; c <= curves; ++c) small[c] = (uint64_t)c * nq;
    if (!rc) rc = status_of(upload_small(seg, small.data(), 8 * small.size(), s));
    if (rc) return rc;
    SortProblem sp = order_problem(nq, curves);
    sp.seg_off_dev = seg;
    sp.hi = keys;   // gathered along, not compared (key_bits <= 64)
    sp.lo = keys;
    sp.ids = nullptr;
    sp.id_base_dev = seg + curves + 1;   // ids = ranks 0..nq-1 in every segment
    sp.out_hi = reinterpret_cast<uint64_t*>(ws + L.out_hi);
    sp.out_lo = reinterpret_cast<uint64_t*>(ws + L.out_lo);
    sp.out_ids = reinterpret_cast<uint32_t*>(ws + L.order);
    sp.ids_only = true;   // the permutations alone
    {
        TraceRange to("order");
        if ((rc = sort_segments(sp, ws + L.sort, s))) return rc;
    }
    {
        TraceRange tb("search");
        if ((rc = status_of(launch_batch_positions(v, nq, sp.out_ids, qhi, qlo, pos, s))))
            return rc;
    }
    TraceRange tq("walk");
    return status_of(launch_query(v, q_dev, nq, k, p, out_ids_dev, out_dist_dev, s, nullptr,
                                  nullptr, sp.out_ids, pos));
}

// hc_query_host's work: the queries up on cs (into the index's staging), the
// walk on s behind them (in key order for large batches), the results down
// on s.  The staging is reused by the next call on the index only after this
// call's results have left (an event).
int enqueue_host_query(hc_index* idx, const void* q_host, uint32_t nq, uint32_t k, uint32_t p,
                       int32_t* out_ids_host, void* out_dist_host, cudaStream_t cs,
                       cudaStream_t s) {
    const size_t qbytes = (size_t)nq * idx->row_bytes;
    const size_t obytes = (size_t)nq * k * 4;
    // large batches are answered in curve-0 key order (hc_query_ordered: the
    // same results, fewer DRAM reads); its workspace follows the results, on
    // the walk's stream, so that only the query buffer comes and goes in the
    // copy stream's order
    const bool ordered = nq >= kHostOrderedMin;
    const size_t ws_off = align256(2 * obytes);
    const size_t out_bytes = ordered ? ws_off + order_layout(idx, nq).bytes : 2 * obytes;
    int rc;
    if (!idx->st_done &&
        (rc = status_of(cudaEventCreateWithFlags(&idx->st_done, cudaEventDisableTiming))))
        return rc;
    // staging from the stream-ordered pool, replaced in stream order: no
    // device-wide synchronisation, so work queued on other streams runs on;
    // the query buffer is allocated in the copy stream's order
    keep_pool_memory();
    if ((rc = status_of(cudaStreamWaitEvent(cs, idx->st_done, 0)))) return rc;
    if (qbytes > idx->st_q_cap) {
        pool_free(idx->st_q, cs);
        idx->st_q = nullptr;
        idx->st_q_cap = 0;
        if ((rc = dev_alloc_async(&idx->st_q, qbytes, cs))) return rc;
        idx->st_q_cap = qbytes;
    }
    if (out_bytes > idx->st_out_cap) {
        pool_free(idx->st_out, s);
        idx->st_out = nullptr;
        idx->st_out_cap = 0;
        if ((rc = dev_alloc_async(&idx->st_out, out_bytes, s))) return rc;
        idx->st_out_cap = out_bytes;
    }
    int32_t* d_ids = static_cast<int32_t*>(idx->st_out);
    void* d_dist = static_cast<char*>(idx->st_out) + obytes;
    if ((rc = status_of(cudaMemcpyAsync(idx->st_q, q_host, qbytes, cudaMemcpyHostToDevice, cs))))
        return rc;
    if (cs != s) {
        cudaEvent_t landed = nullptr;
        rc = status_of(cudaEventCreateWithFlags(&landed, cudaEventDisableTiming));
        if (!rc) rc = status_of(cudaEventRecord(landed, cs));
        if (!rc) rc = status_of(cudaStreamWaitEvent(s, landed, 0));
        if (landed) cudaEventDestroy(landed);
        if (rc) return rc;
    }
    rc = ordered ? enqueue_ordered(idx, idx->st_q, nq, k, p, d_ids, d_dist,
                                   static_cast<char*>(idx->st_out) + ws_off, s)
                 : status_of(launch_query(view_of(idx), idx->st_q, nq, k, p, d_ids, d_dist, s));
    if (rc) return rc;
    if ((rc = status_of(cudaMemcpyAsync(out_ids_host, d_ids, obytes, cudaMemcpyDeviceToHost, s))))
        return rc;
    if ((rc = status_of(cudaMemcpyAsync(out_dist_host, d_dist, obytes, cudaMemcpyDeviceToHost, s))))
        return rc;
    return status_of(cudaEventRecord(idx->st_done, s));
}

}  // namespace

extern "C" {

HC_API size_t hc_query_ordered_workspace(const hc_index* idx, uint32_t nq) {
    return idx && nq ? order_layout(idx, nq).bytes : 0;
}

HC_API int hc_query_ordered(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k, uint32_t p,
                            int32_t* out_ids_dev, void* out_dist_dev, void* workspace_dev,
                            size_t workspace_bytes, void* cuda_stream) {
    TraceRange tr("hc_query_ordered");
    if (!idx || k < 1 || k > 128 || p > (1u << 30)) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!q_dev || !out_ids_dev || !out_dist_dev || !aligned16(q_dev) || !workspace_dev ||
        ((uintptr_t)workspace_dev & 255))
        return HC_ERR_ARG;
    const OrderLayout L = order_layout(idx, nq);
    if (workspace_bytes < L.bytes) return HC_ERR_ARG;
    if (!is_device_ptr(q_dev) || !is_device_ptr(out_ids_dev) || !is_device_ptr(out_dist_dev) ||
        !is_device_ptr(workspace_dev))
        return HC_ERR_ARG;
    return enqueue_ordered(idx, q_dev, nq, k, p, out_ids_dev, out_dist_dev,
                           static_cast<char*>(workspace_dev), static_cast<cudaStream_t>(cuda_stream));
}

HC_API int hc_query_host(hc_index* idx, const void* q_host, uint32_t nq, uint32_t k, uint32_t p,
                         int32_t* out_ids_host, void* out_dist_host, void* cuda_stream) {
    TraceRange tr("hc_query_host");
    if (!idx || k < 1 || k > 128 || p > (1u << 30)) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!q_host || !out_ids_host || !out_dist_host) return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (int rc = enqueue_host_query(idx, q_host, nq, k, p, out_ids_host, out_dist_host, s, s))
        return rc;
    return status_of(cudaStreamSynchronize(s));
}

HC_API int hc_query_host_async(hc_index* idx, const void* q_host, uint32_t nq, uint32_t k,
                               uint32_t p, int32_t* out_ids_host, void* out_dist_host,
                               void* copy_stream, void* cuda_stream) {
    TraceRange tr("hc_query_host_async");
    if (!idx || k < 1 || k > 128 || p > (1u << 30)) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!is_pinned_host(q_host) || !is_pinned_host(out_ids_host) ||
        !is_pinned_host(out_dist_host))
        return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaStream_t cs = copy_stream ? static_cast<cudaStream_t>(copy_stream) : s;
    return enqueue_host_query(idx, q_host, nq, k, p, out_ids_host, out_dist_host, cs, s);
}

HC_API int hc_index_describe(const hc_index* idx, hc_index_info* info, uint64_t* list_off_host) {
    if (!idx || !info) return HC_ERR_ARG;
    info->n = idx->params.n;
    info->d = idx->params.d;
    info->curves = idx->params.curves;
    info->dims_per_curve = idx->params.dims_per_curve;
    info->partitions = idx->params.partitions;
    info->lists = idx->lists;
    info->dtype = idx->params.dtype;
    info->keys_hi_dev = idx->keys_hi;
    info->keys_lo_dev = idx->keys_lo;
    info->ids_dev = idx->ids;
    info->db_dev = idx->db;
    if (list_off_host)
        std::memcpy(list_off_host, idx->list_off.data(), sizeof(uint64_t) * (idx->lists + 1));
    return HC_OK;
}

HC_API int hc_index_copy_lists(const hc_index* idx, uint64_t* keys_hi_dev, uint64_t* keys_lo_dev,
                               uint32_t* ids_dev, void* cuda_stream) {
    if (!idx) return HC_ERR_ARG;
    const uint64_t total = idx->list_off[idx->lists];
    if (total == 0) return HC_OK;
    if (!is_device_ptr(keys_hi_dev) || !is_device_ptr(keys_lo_dev) || !is_device_ptr(ids_dev))
        return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc = status_of(cudaMemcpyAsync(keys_hi_dev, idx->keys_hi, 8 * total,
                                       cudaMemcpyDeviceToDevice, s));
    if (!rc)
        rc = status_of(idx->keys_lo ? cudaMemcpyAsync(keys_lo_dev, idx->keys_lo, 8 * total,
                                                      cudaMemcpyDeviceToDevice, s)
                                    : launch_entry_lo(view_of(idx), keys_lo_dev, s));
    if (!rc)
        rc = status_of(cudaMemcpyAsync(ids_dev, idx->ids, 4 * total, cudaMemcpyDeviceToDevice, s));
    return rc;
}

HC_API int hc_hilbert_keys(const void* x_dev, hc_dtype dtype, uint64_t count, uint32_t d,
                           uint32_t curves, uint32_t m, const uint32_t* dim_map_host,
                           uint64_t* hi_dev, uint64_t* lo_dev, void* cuda_stream) {
    TraceRange tr("hc_hilbert_keys");
    if (dtype != HC_U8 && dtype != HC_F32) return HC_ERR_ARG;
    if (d < 1 || d > 4096 || curves < 1 || curves > 32 || m < 1 || m > 16) return HC_ERR_ARG;
    const uint32_t rb = row_bytes_of(dtype, d);
    if (rb % 16) return HC_ERR_ARG;
    if (dim_map_host) {
        for (uint32_t i = 0; i < curves * m; ++i)
            if (dim_map_host[i] >= d) return HC_ERR_ARG;
    } else if ((uint64_t)curves * m > d) {
        return HC_ERR_ARG;
    }
    if (count == 0) return HC_OK;
    if (!is_device_ptr(x_dev) || !aligned16(x_dev) || !is_device_ptr(hi_dev) ||
        !is_device_ptr(lo_dev))
        return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint32_t* dm = nullptr;
    int rc;
    if (dim_map_host) {
        if ((rc = dev_alloc_async((void**)&dm, sizeof(uint32_t) * curves * m, s))) return rc;
        if ((rc = status_of(cudaMemcpyAsync(dm, dim_map_host, sizeof(uint32_t) * curves * m,
                                            cudaMemcpyHostToDevice, s)))) {
            pool_free(dm, s);
            return rc;
        }
    }
    Projection P{d, curves, m, dm, dtype};
    rc = status_of(launch_vector_keys(x_dev, count, rb, P, hi_dev, lo_dev, s));
    if (dm) {
        // the copy above reads a host buffer the caller may free after return
        cudaStreamSynchronize(s);
        pool_free(dm, s);
    }
    return rc;
}

HC_API int hc_sort_keys(uint64_t* hi_dev, uint64_t* lo_dev, uint32_t* ids_dev,
                        const uint64_t* seg_off_host, uint32_t nseg, uint32_t key_bits,
                        void* cuda_stream) {
    TraceRange tr("hc_sort_keys");
    if (!seg_off_host || nseg < 1 || key_bits < 1 || key_bits > 128) return HC_ERR_ARG;
    for (uint32_t i = 0; i < nseg; ++i)
        if (seg_off_host[i + 1] < seg_off_host[i]) return HC_ERR_ARG;
    if (seg_off_host[0] != 0) return HC_ERR_ARG;
    const uint64_t total = seg_off_host[nseg];
    if (total >= (1ull << 32)) return HC_ERR_ARG;
    if (total == 0) return HC_OK;
    if (!is_device_ptr(hi_dev) || !is_device_ptr(lo_dev) || !is_device_ptr(ids_dev))
        return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    SortProblem sp;
    sp.hi = hi_dev;
    sp.lo = lo_dev;
    sp.ids = ids_dev;
    sp.seg_off.assign(seg_off_host, seg_off_host + nseg + 1);
    sp.key_bits = key_bits;
    sp.allow_sync = true;   // this entry point synchronises anyway
    sp.hi_skip = 1;
    const size_t out_bytes = (sizeof(uint64_t) * 2 + sizeof(uint32_t)) * total;
    const size_t off_bytes = sizeof(uint64_t) * (nseg + 1);
    const size_t head = ((out_bytes + 255) & ~(size_t)255) + ((off_bytes + 255) & ~(size_t)255);
    const size_t sb = sort_scratch_bytes(sp);
    keep_pool_memory();
    void* buf = nullptr;
    int rc;
    if ((rc = dev_alloc_async(&buf, head + sb, s))) return rc;
    sp.out_hi = static_cast<uint64_t*>(buf);
    sp.out_lo = sp.out_hi + total;
    sp.out_ids = reinterpret_cast<uint32_t*>(sp.out_lo + total);
    uint64_t* off_dev = reinterpret_cast<uint64_t*>(static_cast<char*>(buf) +
                                                    ((out_bytes + 255) & ~(size_t)255));
    sp.seg_off_dev = off_dev;
    rc = status_of(cudaMemcpyAsync(off_dev, seg_off_host, off_bytes, cudaMemcpyHostToDevice, s));
    if (!rc) rc = sort_segments(sp, static_cast<char*>(buf) + head, s);
    if (!rc) rc = status_of(cudaMemcpyAsync(hi_dev, sp.out_hi, 8 * total, cudaMemcpyDeviceToDevice, s));
    if (!rc) rc = status_of(cudaMemcpyAsync(lo_dev, sp.out_lo, 8 * total, cudaMemcpyDeviceToDevice, s));
    if (!rc)
        rc = status_of(cudaMemcpyAsync(ids_dev, sp.out_ids, 4 * total, cudaMemcpyDeviceToDevice, s));
    const int frc = status_of(pool_free(buf, s));
    const int src = status_of(cudaStreamSynchronize(s));
    return rc ? rc : (frc ? frc : src);
}

HC_API int hc_query_positions(hc_index* idx, const void* q_dev, uint32_t nq, int64_t* pos_dev,
                              void* cuda_stream) {
    TraceRange tr("hc_query_positions");
    if (!idx) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!is_device_ptr(q_dev) || !aligned16(q_dev) || !is_device_ptr(pos_dev)) return HC_ERR_ARG;
    return status_of(
        launch_positions(view_of(idx), q_dev, nq, pos_dev, static_cast<cudaStream_t>(cuda_stream)));
}

HC_API int hc_bruteforce(const void* db_dev, hc_dtype dtype, uint64_t n, uint32_t d,
                         const void* q_dev, uint32_t nq, uint32_t k, int32_t* out_ids_dev,
                         void* out_dist_dev, void* cuda_stream) {
    TraceRange tr("hc_bruteforce");
    if (dtype != HC_U8 && dtype != HC_F32) return HC_ERR_ARG;
    if (k < 1 || k > 128 || d < 1 || d > 4096 || n >= (1ull << 31)) return HC_ERR_ARG;
    if (row_bytes_of(dtype, d) % 16) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!is_device_ptr(db_dev) || !is_device_ptr(q_dev) || !is_device_ptr(out_ids_dev) ||
        !is_device_ptr(out_dist_dev) || !aligned16(db_dev) || !aligned16(q_dev))
        return HC_ERR_ARG;
    return status_of(launch_bruteforce(db_dev, dtype, n, d, q_dev, nq, k, out_ids_dev, out_dist_dev,
                                       static_cast<cudaStream_t>(cuda_stream)));
}

HC_API int hc_check_status(hc_check_report* out, int reset) {
    if (!out) return HC_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
#ifdef HC_CHECK
    out->enabled = 1;
    if (cudaDeviceSynchronize() != cudaSuccess) return HC_ERR_CUDA;
    {
        // guards of the buffers still alive
        std::lock_guard<std::mutex> g(g_guard_mu);
        for (const auto& kv : g_guards) {
            unsigned char h[kGuardBytes];
            if (cudaMemcpy(h, static_cast<const char*>(kv.first) + kv.second, kGuardBytes,
                           cudaMemcpyDeviceToHost) != cudaSuccess)
                return HC_ERR_CUDA;
            for (size_t i = 0; i < kGuardBytes; ++i) {
                if (h[i] == kGuardByte) continue;
                if (!out->violations) {
                    out->site = kSitePad;
                    out->index = i;
                    out->bound = 0;
                }
                ++out->violations;
            }
        }
    }
    for (CheckReader r : check_readers()) {
        CheckRecord rec{};
        if (r(&rec, reset != 0) != 0) return HC_ERR_CUDA;
        if (rec.count && !out->violations) {
            out->site = rec.site;
            out->index = rec.index;
            out->bound = rec.bound;
        }
        out->violations += rec.count;
    }
#else
    (void)reset;
#endif
    return HC_OK;
}

HC_API uint64_t hc_launch_count(void) { return g_launches.load(); }

HC_API void hc_debug_fail_alloc(long after) {
    g_alloc_count.store(0);
    g_fail_after.store(after);
}

}  // extern "C"
