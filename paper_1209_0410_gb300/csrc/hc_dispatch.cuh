// Launch dispatch on (element type, lanes per row, top-k registers), shared
// by the query and brute-force translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hc {
namespace {

inline int lanes_per_row(uint32_t row_bytes) {
    const uint32_t vecs = row_bytes / 16;
    if (vecs <= 4) return 4;
    if (vecs <= 8) return 8;
    if (vecs <= 16) return 16;
    return 32;
}

inline int regs_for_k(uint32_t k) { return k <= 32 ? 1 : (k <= 64 ? 2 : 4); }

// dispatch on (dtype, lanes per row, top-k registers)
template <template <bool, int, int> class Launch, typename... Args>
cudaError_t dispatch(bool f32, int lpr, int kr, Args... args) {
#define HC_CASE(F, L, K)                                   \
    if (f32 == F && lpr == L && kr == K) return Launch<F, L, K>::run(args...);
#define HC_CASES_L(F, L) HC_CASE(F, L, 1) HC_CASE(F, L, 2) HC_CASE(F, L, 4)
#define HC_CASES_F(F) HC_CASES_L(F, 4) HC_CASES_L(F, 8) HC_CASES_L(F, 16) HC_CASES_L(F, 32)
    HC_CASES_F(false)
    HC_CASES_F(true)
#undef HC_CASES_F
#undef HC_CASES_L
#undef HC_CASE
    return cudaErrorInvalidValue;
}


}  // namespace
}  // namespace hc
