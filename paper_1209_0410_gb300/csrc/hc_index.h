// The library's index object (opaque hc_index of include/hc.h), shared by the
// C-ABI translation units.
#pragma once

#include <vector>

#include "hc_internal.h"

struct hc_index {
    hc_build_params params{};
    std::vector<uint32_t> dim_map;   // host copy, empty = consecutive
    uint32_t* dim_map_dev = nullptr;
    const void* db = nullptr;
    void* db_owned = nullptr;
    uint64_t* keys_hi = nullptr;
    uint64_t* keys_lo = nullptr;
    uint32_t* ids = nullptr;
    uint64_t* fence = nullptr;       // every 16th high word (IndexView::fence)
    uint64_t* list_off_dev = nullptr;
    std::vector<uint64_t> list_off;
    uint32_t lists = 0, row_bytes = 0;
    // device staging of hc_query_host
    void* st_q = nullptr;
    void* st_out = nullptr;
    size_t st_q_cap = 0, st_out_cap = 0;
    cudaEvent_t st_done = nullptr;   // the last host query's results have left
};

namespace hc {

inline IndexView view_of(const hc_index* x) {
    IndexView v;
    v.db = x->db;
    v.row_bytes = x->row_bytes;
    v.d = x->params.d;
    v.P = Projection{x->params.d, x->params.curves, x->params.dims_per_curve, x->dim_map_dev,
                     x->params.dtype};
    v.lists = x->lists;
    v.list_off = x->list_off_dev;
    v.keys_hi = x->keys_hi;
    v.keys_lo = x->keys_lo;
    v.ids = x->ids;
    v.rows = x->params.n;
    v.fence = x->fence;
    v.fence_len = x->fence && !x->list_off.empty() ? (x->list_off.back() + 15) >> kFenceShift : 0;
    return v;
}

// Index set-up shared by the entry points that make an index (api.cu:
// hc_build, hc_build_host; persist.cu: hc_load).
int status_of(cudaError_t e);
bool aligned16(const void* p);
// true when p is device memory of the current device (or managed)
bool is_device_ptr(const void* p);
// true when p is page-locked host memory
bool is_pinned_host(const void* p);
// a new index object for these parameters (checked; HC_ERR_ARG when they are
// invalid), nothing allocated on the device yet
int index_new(const void* db, const hc_build_params* params, hc_index** out, hc_index** made);
// lists, row_bytes and list_off from the parameters (Sec. 4.1: partition j
// holds ids [floor(j n / l), floor((j + 1) n / l)))
void index_layout(hc_index* x);
// whether the lists store low key words (keys of fewer than 16 coordinates)
bool index_keeps_lo(const hc_build_params& P);
// the device arrays of a laid-out index: list offsets and dim map (both
// uploaded), keys and ids (uninitialised), from the stream-ordered pool on s
int index_alloc(hc_index* x, cudaStream_t s);
// frees in stream order on s (default: the legacy stream)
void index_destroy(hc_index* x, cudaStream_t s = cudaStreamLegacy);

}  // namespace hc

struct hc_mlp;

namespace hc {
// The learned depth predictor (learned.cu): per-query depths into p_out.
cudaError_t launch_predict_depths(hc_mlp* M, const hc_index* idx, const void* q, uint32_t nq,
                                  float margin, uint32_t p_lo, uint32_t p_hi, uint32_t* p_out,
                                  cudaStream_t s);
// Makes the bf16 inference weights current and waits for them (call before
// the model is used from several streams).
// HC_ERR_ARG when the model's input size is not 4 * curves of the index.
int mlp_prepare_inference(hc_mlp* M, const hc_index* idx, cudaStream_t s);
}  // namespace hc
