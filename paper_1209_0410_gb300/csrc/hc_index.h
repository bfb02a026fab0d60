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
    uint64_t* list_off_dev = nullptr;
    std::vector<uint64_t> list_off;
    uint32_t lists = 0, row_bytes = 0;
    // device staging of hc_query_host
    void* st_q = nullptr;
    void* st_out = nullptr;
    size_t st_q_cap = 0, st_out_cap = 0;
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
    return v;
}

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
