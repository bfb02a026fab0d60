// Many indexes, uneven batches, one persistent launch.
//
// Each job is one hc_query call (an index, its queries, k, p).  The host cuts
// every job into tasks of (warps per block / warps per query) x tile queries,
// orders the tasks by their estimated bytes, largest first (a longest-job-
// first list, so that small tasks fill the tail), and one persistent kernel
// whose blocks take tasks from an atomic counter answers all of them.  Inside
// a task a query is shared by warps_per_query warps: each searches the lists
// L = sub, sub + wpq, ... into its own top-k, and the group's first warp folds
// the others' lists into its own through shared memory (Algorithm 2's union
// over curves is order-free, so the result equals hc_query's bit for bit).
// The element type, lanes per row and top-k width of each job select one
// instantiation of the query code inside the kernel.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "hc_index.h"
#include "hc_trace.h"
#include "hc_query_dev.cuh"

using namespace hc;

namespace {

struct MultiJob {
    IndexView ix;
    const uint8_t* q;
    int32_t* ids;
    void* dist;
    uint32_t nq, k, p;
    uint32_t variant;   // row class * 2 + (k > 32), see variant_of
    uint32_t wpq;       // warps per query: 1, 2, 4, 8
};

struct MultiTask {
    uint32_t job, q0, cnt;
};

constexpr int kMaxWarps = 16;
constexpr uint32_t kMaxLists = 256;
constexpr size_t kRingBytes = 64 * 128;   // two 32-row steps of rows up to 128 bytes

// Instantiations inside the persistent kernel: row classes uint8 with 4, 8 or
// 16 lanes per row (wider uint8 rows take 16 lanes and loop), float32 with 16
// or 32 lanes (narrower float32 rows take 16); top-k of 1 register (k <= 32)
// or 4 (k <= 128).
uint32_t variant_of(hc_dtype t, uint32_t row_bytes, uint32_t k) {
    const uint32_t v = row_bytes / 16;
    uint32_t cls;
    if (t == HC_U8)
        cls = v <= 4 ? 0 : (v <= 8 ? 1 : 2);
    else
        cls = v <= 16 ? 3 : 4;
    return cls * 2 + (k > 32 ? 1 : 0);
}

// One query's share (lists sub, sub + wpq, ...) into `top`, then the group's
// merge; templated on the job's variant.
// group_buf: 4 x 32 slots per warp of the query's group (warp `sub` owns
// group_buf + sub * 128).
// ring: the warp's two-step row ring (64 x 128 bytes) when the plan has
// rows of at most 128 bytes, else null.
template <bool F32, int LPR, int KR>
__device__ void multi_query(const MultiJob& J, uint32_t qi, bool active, uint32_t sub,
                            uint32_t* pos_w, uint32_t lists_cap, uint64_t* group_buf,
                            uint8_t* ring, int lane) {
    WarpTopK<KR> top;
    top.init();
    if (active && !HC_IN_BOUNDS(kSiteMultiQuery, qi, J.nq)) active = false;
    if (active) {
        const uint8_t* qrow = J.q + (size_t)qi * J.ix.row_bytes;
        if constexpr (LPR <= 8) {
            if (ring && J.ix.row_bytes <= 128) {
                search_lists_staged<F32, LPR, KR>(J.ix, qrow, J.p, J.k, sub, J.wpq, pos_w,
                                                  pos_w + lists_cap, ring, top, lane);
            } else {
                search_lists<F32, LPR, KR>(J.ix, qrow, J.p, J.k, sub, J.wpq, pos_w, top, lane);
            }
        } else {
            search_lists<F32, LPR, KR>(J.ix, qrow, J.p, J.k, sub, J.wpq, pos_w, top, lane);
        }
    }
    // one warp per query (the same for every warp of the block: one job per
    // task): the warp's list is the query's, written without a block barrier
    if (J.wpq == 1) {
        if (active)
            top.template store<F32>(J.k, lane, J.ids + (size_t)qi * J.k,
                                    static_cast<uint32_t*>(J.dist) + (size_t)qi * J.k);
        return;
    }
    // every warp publishes its list; the group leader folds the others in
    uint64_t* mine = group_buf + (size_t)sub * 4 * 32;
#pragma unroll
    for (int r = 0; r < KR; ++r) mine[r * 32 + lane] = top.v[r];
    __syncthreads();
    if (active && sub == 0) {
        for (uint32_t s = 1; s < J.wpq; ++s) {
            const uint64_t* other = group_buf + (size_t)s * 4 * 32;
#pragma unroll
            for (int r = 0; r < KR; ++r) top.offer(other[r * 32 + lane], J.k, lane);
        }
        top.template store<F32>(J.k, lane, J.ids + (size_t)qi * J.k,
                                static_cast<uint32_t*>(J.dist) + (size_t)qi * J.k);
    }
    __syncthreads();
}

template <int V>
__device__ __forceinline__ void run_variant(const MultiJob& J, uint32_t qi, bool active,
                                            uint32_t sub, uint32_t* pos_w, uint32_t lists_cap,
                                            uint64_t* mb, uint8_t* ring, int lane) {
    constexpr int CLS = V / 2;
    constexpr bool F32 = CLS >= 3;
    constexpr int LPR = CLS == 0 ? 4 : (CLS == 1 ? 8 : (CLS == 2 ? 16 : (CLS == 3 ? 16 : 32)));
    constexpr int KR = (V & 1) ? 4 : 1;
    multi_query<F32, LPR, KR>(J, qi, active, sub, pos_w, lists_cap, mb, ring, lane);
}

__global__ void __launch_bounds__(kMaxWarps * 32)
    multi_kernel(const MultiJob* __restrict__ jobs, const MultiTask* __restrict__ tasks,
                 uint32_t ntasks, uint32_t tile, uint32_t* __restrict__ counter, bool staged,
                 uint32_t lists_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t nwarps = blockDim.x >> 5;
    uint64_t* merge = reinterpret_cast<uint64_t*>(smem_raw);             // nwarps x 4 x 32
    // per warp: lists_cap positions, then lists_cap window prefixes (lists_cap:
    // the plan's largest index, a multiple of 4, so the rings stay 16-byte aligned)
    uint32_t* pos = reinterpret_cast<uint32_t*>(merge + nwarps * 4 * 32);
    uint8_t* rings = reinterpret_cast<uint8_t*>(pos + nwarps * 2 * lists_cap); // nwarps x kRingBytes
    __shared__ uint32_t s_task;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t t = s_task;
        __syncthreads();
        if (t >= ntasks) return;
        const MultiTask T = tasks[t];
        const MultiJob& J = jobs[T.job];
        if (!HC_IN_BOUNDS(kSiteMultiLists, J.ix.lists, lists_cap + 1)) continue;
        const uint32_t group = warp / J.wpq, sub = warp % J.wpq;
        const uint32_t per_pass = nwarps / J.wpq;
        uint64_t* mb = merge + (size_t)(group * J.wpq) * 4 * 32;
        for (uint32_t rep = 0; rep < tile; ++rep) {
            const uint32_t qo = rep * per_pass + group;
            const bool active = group < per_pass && qo < T.cnt;
            const uint32_t qi = T.q0 + qo;
            uint32_t* pw = pos + (size_t)warp * 2 * lists_cap;
            uint8_t* ring = staged ? rings + (size_t)warp * kRingBytes : nullptr;
            switch (J.variant) {
#define HC_V(n) \
    case n: run_variant<n>(J, qi, active, sub, pw, lists_cap, mb, ring, lane); break;
                HC_V(0) HC_V(1) HC_V(2) HC_V(3) HC_V(4) HC_V(5) HC_V(6) HC_V(7) HC_V(8)
                HC_V(9)
#undef HC_V
                default: break;
            }
            if ((rep + 1) * per_pass >= T.cnt) break;   // task done (uniform)
        }
    }
}

__global__ void reset_counter_kernel(uint32_t* c) { *c = 0; }

size_t multi_smem(uint32_t nwarps, bool staged, uint32_t lists_cap) {
    return (size_t)nwarps * 4 * 32 * sizeof(uint64_t) +
           (size_t)nwarps * 2 * lists_cap * sizeof(uint32_t) + (staged ? nwarps * kRingBytes : 0);
}

}  // namespace

struct hc_multi_plan {
    hc_multi_config cfg{};
    uint32_t njobs = 0, ntasks = 0;
    MultiJob* jobs_dev = nullptr;
    MultiTask* tasks_dev = nullptr;
    uint32_t* counter = nullptr;
    unsigned grid = 0;
    size_t smem = 0;
    bool staged = false;   // some job has rows of at most 128 bytes and <= 8 lanes per row
    uint32_t lists_cap = 4;   // largest number of lists of a job's index, rounded up to 4
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int enqueue(hc_multi_plan* P, cudaStream_t s) {
    reset_counter_kernel<<<1, 1, 0, s>>>(P->counter);
    multi_kernel<<<P->grid, P->cfg.warps_per_block * 32, P->smem, s>>>(
        P->jobs_dev, P->tasks_dev, P->ntasks, P->cfg.tile, P->counter, P->staged, P->lists_cap);
    count_launches(2);
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}

void free_plan(hc_multi_plan* P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    cudaFree(P->jobs_dev);
    cudaFree(P->tasks_dev);
    cudaFree(P->counter);
    cudaGetLastError();
    delete P;
}

}  // namespace

extern "C" {

HC_API int hc_multi_plan_create(const hc_multi_job* jobs, uint32_t njobs,
                                const hc_multi_config* cfg_in, void* cuda_stream,
                                hc_multi_plan** out) {
    if (!out) return HC_ERR_ARG;
    *out = nullptr;
    if (!jobs || njobs < 1) return HC_ERR_ARG;
    hc_multi_config cfg{8, 4, 2, 1};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.warps_per_block < 1 || cfg.warps_per_block > kMaxWarps ||
        (cfg.warps_per_block & (cfg.warps_per_block - 1)) || cfg.blocks_per_sm < 1 ||
        cfg.blocks_per_sm > 32 || cfg.tile < 1 || cfg.tile > 64)
        return HC_ERR_ARG;
    std::vector<MultiJob> hj(njobs);
    std::vector<MultiTask> ht;
    std::vector<double> tcost;
    for (uint32_t j = 0; j < njobs; ++j) {
        const hc_multi_job& in = jobs[j];
        if (!in.index || in.k < 1 || in.k > 128 || in.p > (1u << 30)) return HC_ERR_ARG;
        const uint32_t wpq = in.warps_per_query ? in.warps_per_query : 1;
        if ((wpq & (wpq - 1)) || wpq > cfg.warps_per_block || wpq > 8) return HC_ERR_ARG;
        if (in.index->lists > kMaxLists) return HC_ERR_ARG;
        if (in.nq && (!on_device(in.q_dev) || !on_device(in.out_ids_dev) ||
                      !on_device(in.out_dist_dev) || ((uintptr_t)in.q_dev & 15)))
            return HC_ERR_ARG;
        MultiJob& J = hj[j];
        J.ix = view_of(in.index);
        J.q = static_cast<const uint8_t*>(in.q_dev);
        J.ids = in.out_ids_dev;
        J.dist = in.out_dist_dev;
        J.nq = in.nq;
        J.k = in.k;
        J.p = in.p;
        J.wpq = wpq;
        J.variant = variant_of(in.index->params.dtype, in.index->row_bytes, in.k);
        // task = the queries one block answers for this job
        const uint32_t per_task = (cfg.warps_per_block / wpq) * cfg.tile;
        const uint64_t n_list = in.index->list_off[in.index->lists] / (in.index->lists ? in.index->lists : 1);
        const double per_query = (double)in.index->lists *
                                 (double)std::min<uint64_t>(2ull * in.p, n_list) *
                                 (double)(in.index->row_bytes + 4);
        for (uint32_t q0 = 0; q0 < in.nq; q0 += per_task) {
            const uint32_t cnt = std::min(per_task, in.nq - q0);
            ht.push_back(MultiTask{j, q0, cnt});
            tcost.push_back(per_query * cnt);
        }
    }
    // largest estimated bytes first
    std::vector<uint32_t> order(ht.size());
    for (uint32_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return tcost[a] > tcost[b]; });
    std::vector<MultiTask> sorted(ht.size());
    for (uint32_t i = 0; i < order.size(); ++i) sorted[i] = ht[order[i]];

    hc_multi_plan* P = new (std::nothrow) hc_multi_plan();
    if (!P) return HC_ERR_OOM;
    P->cfg = cfg;
    P->njobs = njobs;
    P->ntasks = (uint32_t)sorted.size();
    (void)cuda_stream;   // the tables are copied synchronously
    bool ok = !alloc_should_fail() &&
              cudaMalloc(&P->jobs_dev, sizeof(MultiJob) * njobs) == cudaSuccess &&
              cudaMalloc(&P->tasks_dev, sizeof(MultiTask) * std::max<size_t>(1, sorted.size())) ==
                  cudaSuccess &&
              cudaMalloc(&P->counter, sizeof(uint32_t)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_plan(P);
        return HC_ERR_OOM;
    }
    if (cudaMemcpy(P->jobs_dev, hj.data(), sizeof(MultiJob) * njobs, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        (P->ntasks && cudaMemcpy(P->tasks_dev, sorted.data(), sizeof(MultiTask) * P->ntasks,
                                 cudaMemcpyHostToDevice) != cudaSuccess)) {
        free_plan(P);
        return HC_ERR_CUDA;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (const MultiJob& j : hj) {
        P->staged |= j.variant / 2 <= 1;   // uint8 rows <= 128 bytes
        P->lists_cap = std::max(P->lists_cap, (j.ix.lists + 3u) & ~3u);
    }
    P->smem = multi_smem(cfg.warps_per_block, P->staged, P->lists_cap);
    if (cudaFuncSetAttribute(multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)P->smem) != cudaSuccess) {
        free_plan(P);
        return HC_ERR_CUDA;
    }
    P->grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((uint64_t)sms * cfg.blocks_per_sm, std::max<uint32_t>(1, P->ntasks)));
    if (cfg.use_graph) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            free_plan(P);
            return HC_ERR_CUDA;
        }
        int rc = HC_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            rc = HC_ERR_CUDA;
        if (!rc) rc = enqueue(P, cs);
        if (cudaStreamEndCapture(cs, &P->graph) != cudaSuccess) rc = HC_ERR_CUDA;
        if (!rc && cudaGraphInstantiate(&P->exec, P->graph, 0) != cudaSuccess) rc = HC_ERR_CUDA;
        cudaStreamDestroy(cs);
        if (rc) {
            cudaGetLastError();
            free_plan(P);
            return rc;
        }
    }
    *out = P;
    return HC_OK;
}

HC_API int hc_multi_run(hc_multi_plan* P, void* cuda_stream) {
    TraceRange tr("hc_multi_run");
    if (!P) return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (P->exec) {
        if (cudaGraphLaunch(P->exec, s) != cudaSuccess) return HC_ERR_CUDA;
        count_launches(2);
        return HC_OK;
    }
    return enqueue(P, s);
}

HC_API void hc_multi_plan_free(hc_multi_plan* P) { free_plan(P); }

HC_API int hc_query_multi(const hc_multi_job* jobs, uint32_t njobs, const hc_multi_config* cfg,
                          void* cuda_stream) {
    TraceRange tr("hc_query_multi");
    hc_multi_config c{8, 4, 2, 0};
    if (cfg) {
        c = *cfg;
        c.use_graph = 0;
    }
    hc_multi_plan* P = nullptr;
    if (int rc = hc_multi_plan_create(jobs, njobs, &c, cuda_stream, &P)) return rc;
    int rc = hc_multi_run(P, cuda_stream);
    cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    free_plan(P);
    return rc;
}

}  // extern "C"
