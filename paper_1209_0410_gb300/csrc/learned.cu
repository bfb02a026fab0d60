// Learned probe depth: a small MLP predicts, per query, the depth p that
// reproduces the top-k of a large fixed depth.  Not in the paper, where the
// probe depth is one fixed number per subindex (Algorithm 2); the fixed-depth
// method stays as the fallback and as the source of the training labels.
//
//   features   4 per curve: octave encodings of the key gaps to the list
//              neighbours of the query key, and of the min / mean distance of
//              the 8 list entries around it (exact, integer-derived values)
//   labels     minimal p in [0, p_max] whose top-k equals the top-k at p_max,
//              by a per-query binary search driven by the query kernel
//              (valid because windows, hence results, are nested in p)
//   model      x^ = (x - mu) * isd;  h1 = relu(x^ W1 + b1);
//              h2 = relu(h1 W2 + b2);  y = h2 . W3 + b3   (y ~ log2 p)
//   training   FP32 forward / backward by small-GEMM kernels, MSE loss, Adam
//   inference  BF16 inputs and weights, FP32 accumulation, fused with the
//              feature computation: one warp per query
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "hc_index.h"
#include "hc_trace.h"
#include "hc_query_dev.cuh"

using namespace hc;

// ---------------------------------------------------------------- model
struct hc_mlp {
    uint32_t in = 0, h1 = 0, h2 = 0, max_batch = 0;
    uint32_t nparam = 0;          // trained parameters
    float* params = nullptr;      // device: W1 b1 W2 b2 W3 b3 | mu isd
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* wbf = nullptr; // device: W1 W2 W3 in bf16 (inference)
    float* work = nullptr;        // device: per-batch activations
    float* loss = nullptr;        // device scalar
    uint64_t steps = 0;
    bool bf_stale = true;
};

namespace {

struct Layout {
    uint32_t W1, b1, W2, b2, W3, b3, mu, isd, total_trained, total;
};

Layout layout_of(uint32_t in, uint32_t h1, uint32_t h2) {
    Layout L;
    L.W1 = 0;
    L.b1 = L.W1 + in * h1;
    L.W2 = L.b1 + h1;
    L.b2 = L.W2 + h1 * h2;
    L.W3 = L.b2 + h2;
    L.b3 = L.W3 + h2;
    L.total_trained = L.b3 + 1;
    L.mu = L.total_trained;
    L.isd = L.mu + in;
    L.total = L.isd + in;
    return L;
}

// activations of one batch inside hc_mlp::work
struct Work {
    float *xn, *a1, *a2, *y, *dy, *d2, *d1;
};

Work work_of(const hc_mlp* M) {
    Work w;
    const size_t B = M->max_batch;
    w.xn = M->work;
    w.a1 = w.xn + B * M->in;
    w.a2 = w.a1 + B * M->h1;
    w.y = w.a2 + B * M->h2;
    w.dy = w.y + B;
    w.d2 = w.dy + B;
    w.d1 = w.d2 + B * M->h2;
    return w;
}

size_t work_floats(uint32_t in, uint32_t h1, uint32_t h2, uint32_t B) {
    return (size_t)B * (in + h1 + h2 + 1 + 1 + h2 + h1);
}

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[N]) (relu) (* [mask > 0]);
// A(m,k) = TA ? A[k*lda+m] : A[m*lda+k];  B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n]
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                    int lda, const float* __restrict__ Bm, int ldb,
                                                    float* __restrict__ C, int ldc,
                                                    const float* __restrict__ bias, int relu,
                                                    const float* __restrict__ mask) {
    __shared__ float As[32][33];
    __shared__ float Bs[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int m = m0 + r, k = k0 + tx;
            As[r][tx] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k])
                                         : 0.f;
            const int kk = k0 + r, n = n0 + tx;
            Bs[r][tx] = (kk < K && n < N) ? (TB ? Bm[(size_t)n * ldb + kk] : Bm[(size_t)kk * ldb + n])
                                          : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float b = Bs[kk][tx];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = fmaf(As[ty + 8 * i][kk], b, acc[i]);
        }
        __syncthreads();
    }
    const int n = n0 + tx;
    if (n >= N) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 8 * i;
        if (m >= M) continue;
        float v = acc[i];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
        if (mask && !(mask[(size_t)m * ldc + n] > 0.f)) v = 0.f;
        C[(size_t)m * ldc + n] = v;
    }
}

template <bool TA, bool TB>
void sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
           int ldc, const float* bias, bool relu, const float* mask, cudaStream_t s) {
    dim3 grid((N + 31) / 32, (M + 31) / 32);
    sgemm_kernel<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu ? 1 : 0,
                                              mask);
    count_launches(1);
}

__global__ void normalize_kernel(const float* __restrict__ x, uint32_t n, uint32_t in,
                                 const float* __restrict__ mu, const float* __restrict__ isd,
                                 float* __restrict__ xn) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * in) return;
    const uint32_t j = (uint32_t)(t % in);
    xn[t] = (x[t] - mu[j]) * isd[j];
}

// dY = 2 (Y - T) / n and the mean squared error
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, uint32_t n,
                            float* __restrict__ dy, float* __restrict__ loss) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < n) {
        const float e = y[i] - t[i];
        dy[i] = 2.f * e / (float)n;
        l = e * e / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// out[j] = sum_m A[m*N + j]
__global__ void colsum_kernel(const float* __restrict__ A, uint32_t M, uint32_t N,
                              float* __restrict__ out) {
    const uint32_t j = blockIdx.x;
    float s = 0.f;
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) s += A[(size_t)m * N + j];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, uint32_t n, float lr,
                            float beta1, float beta2, float eps, float corr1, float corr2) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / corr1, vh = vi / corr2;
    p[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                               uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// forward pass and gradients of one batch into M->grads (trained layout)
int forward_backward(hc_mlp* M, const float* x, const float* t, uint32_t n, cudaStream_t s,
                     bool backward) {
    const Layout L = layout_of(M->in, M->h1, M->h2);
    const Work w = work_of(M);
    float* P = M->params;
    float* G = M->grads;
    const uint32_t in = M->in, h1 = M->h1, h2 = M->h2;
    normalize_kernel<<<(unsigned)(((size_t)n * in + 255) / 256), 256, 0, s>>>(x, n, in, P + L.mu,
                                                                              P + L.isd, w.xn);
    count_launches(1);
    sgemm<false, false>(n, h1, in, w.xn, in, P + L.W1, h1, w.a1, h1, P + L.b1, true, nullptr, s);
    sgemm<false, false>(n, h2, h1, w.a1, h1, P + L.W2, h2, w.a2, h2, P + L.b2, true, nullptr, s);
    sgemm<false, false>(n, 1, h2, w.a2, h2, P + L.W3, 1, w.y, 1, P + L.b3, false, nullptr, s);
    if (!backward) return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
    cudaMemsetAsync(M->loss, 0, sizeof(float), s);
    loss_kernel<<<(n + 255) / 256, 256, 0, s>>>(w.y, t, n, w.dy, M->loss);
    count_launches(1);
    // output layer
    sgemm<true, false>(h2, 1, n, w.a2, h2, w.dy, 1, G + L.W3, 1, nullptr, false, nullptr, s);
    colsum_kernel<<<1, 256, 0, s>>>(w.dy, n, 1, G + L.b3);
    // second hidden layer: d2 = (dY W3^T) * [a2 > 0]
    sgemm<false, false>(n, h2, 1, w.dy, 1, P + L.W3, h2, w.d2, h2, nullptr, false, w.a2, s);
    sgemm<true, false>(h1, h2, n, w.a1, h1, w.d2, h2, G + L.W2, h2, nullptr, false, nullptr, s);
    colsum_kernel<<<h2, 256, 0, s>>>(w.d2, n, h2, G + L.b2);
    // first hidden layer: d1 = (d2 W2^T) * [a1 > 0]
    sgemm<false, true>(n, h1, h2, w.d2, h2, P + L.W2, h2, w.d1, h1, nullptr, false, w.a1, s);
    sgemm<true, false>(in, h1, n, w.xn, in, w.d1, h1, G + L.W1, h1, nullptr, false, nullptr, s);
    colsum_kernel<<<h1, 256, 0, s>>>(w.d1, n, h1, G + L.b1);
    count_launches(3);
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}

int refresh_bf16(hc_mlp* M, cudaStream_t s) {
    if (!M->bf_stale) return HC_OK;
    const Layout L = layout_of(M->in, M->h1, M->h2);
    const uint32_t n1 = M->in * M->h1, n2 = M->h1 * M->h2, n3 = M->h2;
    to_bf16_kernel<<<(n1 + 255) / 256, 256, 0, s>>>(M->params + L.W1, M->wbf, n1);
    to_bf16_kernel<<<(n2 + 255) / 256, 256, 0, s>>>(M->params + L.W2, M->wbf + n1, n2);
    to_bf16_kernel<<<(n3 + 255) / 256, 256, 0, s>>>(M->params + L.W3, M->wbf + n1 + n2, n3);
    count_launches(3);
    M->bf_stale = false;
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}

// ---------------------------------------------------------- inference
constexpr int kPredWarps = 8;
constexpr uint32_t kMaxDim = 64;

struct MlpView {
    uint32_t in, h1, h2;
    const __nv_bfloat16* wbf;   // W1 | W2 | W3
    const float* params;        // for b1 b2 b3 mu isd
    Layout L;
};

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// y of one sample whose raw features sit in xs[0..in) (warp-shared memory).
// Weights in shared memory (bf16), inputs of each layer rounded to bf16,
// accumulation in float32.  Lane j computes hidden units j and j + 32.
__device__ float mlp_warp_forward(const MlpView& V, const __nv_bfloat16* sW1,
                                  const __nv_bfloat16* sW2, const __nv_bfloat16* sW3,
                                  const float* sb, float* xs, float* hs, int lane) {
    const float* b1 = sb;
    const float* b2 = sb + kMaxDim;
    const float b3 = sb[2 * kMaxDim];
    const float* mu = sb + 2 * kMaxDim + 1;
    const float* isd = mu + kMaxDim;
    for (uint32_t i = lane; i < V.in; i += 32) xs[i] = bf((xs[i] - mu[i]) * isd[i]);
    __syncwarp();
    for (uint32_t j = lane; j < V.h1; j += 32) {
        float a = 0.f;
        for (uint32_t i = 0; i < V.in; ++i) a = fmaf(xs[i], __bfloat162float(sW1[i * V.h1 + j]), a);
        hs[j] = bf(fmaxf(a + b1[j], 0.f));
    }
    __syncwarp();
    float part = 0.f;
    for (uint32_t j = lane; j < V.h2; j += 32) {
        float a = 0.f;
        for (uint32_t i = 0; i < V.h1; ++i) a = fmaf(hs[i], __bfloat162float(sW2[i * V.h2 + j]), a);
        const float h2v = bf(fmaxf(a + b2[j], 0.f));
        part = fmaf(h2v, __bfloat162float(sW3[j]), part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __syncwarp();
    return part + b3;
}

// Stages bf16 weights and float biases / normalisation in shared memory.
__device__ void stage_weights(const MlpView& V, __nv_bfloat16* sW, float* sb) {
    const uint32_t nw = V.in * V.h1 + V.h1 * V.h2 + V.h2;
    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) sW[i] = V.wbf[i];
    for (uint32_t i = threadIdx.x; i < 4 * kMaxDim + 1; i += blockDim.x) {
        float v = 0.f;
        if (i < kMaxDim) v = i < V.h1 ? V.params[V.L.b1 + i] : 0.f;
        else if (i < 2 * kMaxDim) v = i - kMaxDim < V.h2 ? V.params[V.L.b2 + i - kMaxDim] : 0.f;
        else if (i == 2 * kMaxDim) v = V.params[V.L.b3];
        else if (i < 3 * kMaxDim + 1) {
            const uint32_t j = i - 2 * kMaxDim - 1;
            v = j < V.in ? V.params[V.L.mu + j] : 0.f;
        } else {
            const uint32_t j = i - 3 * kMaxDim - 1;
            v = j < V.in ? V.params[V.L.isd + j] : 1.f;
        }
        sb[i] = v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPredWarps * 32) mlp_infer_kernel(MlpView V,
                                                                    const float* __restrict__ x,
                                                                    uint32_t n, float* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    const uint32_t nw = V.in * V.h1 + V.h1 * V.h2 + V.h2;
    float* sb = reinterpret_cast<float*>(smem_raw + ((nw * 2 + 15) & ~15u));
    float* sx = sb + 4 * kMaxDim + 1 + 3;
    stage_weights(V, sW, sb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* xs = sx + warp * 2 * kMaxDim;
    float* hs = xs + kMaxDim;
    for (uint32_t i = blockIdx.x * kPredWarps + warp; i < n; i += gridDim.x * kPredWarps) {
        for (uint32_t j = lane; j < V.in; j += 32) xs[j] = x[(size_t)i * V.in + j];
        __syncwarp();
        const float yi = mlp_warp_forward(V, sW, sW + V.in * V.h1, sW + V.in * V.h1 + V.h1 * V.h2,
                                          sb, xs, hs, lane);
        if (lane == 0) y[i] = yi;
        __syncwarp();
    }
}

size_t pred_smem(const MlpView& V) {
    const uint32_t nw = V.in * V.h1 + V.h1 * V.h2 + V.h2;
    return ((nw * 2 + 15) & ~15u) + sizeof(float) * (4 * kMaxDim + 1 + 3) +
           sizeof(float) * kPredWarps * 2 * kMaxDim + sizeof(uint32_t) * kPredWarps * (64 + 128);
}

// ------------------------------------------------------------ features
// Octave encoding: 0 for g = 0, else 1 + e + f / 65536 with e the top set bit
// of the 128-bit g and f the 16 bits below it.  Exact in float32.
__device__ __forceinline__ float octave128(uint64_t hi, uint64_t lo) {
    if (!hi && !lo) return 0.f;
    const int e = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    const unsigned __int128 g = ((unsigned __int128)hi << 64) | lo;
    const uint32_t f = e >= 16 ? (uint32_t)(g >> (e - 16)) & 0xFFFFu
                               : (uint32_t)(g << (16 - e)) & 0xFFFFu;
    return 1.0f + (float)e + (float)f * (1.0f / 65536.0f);
}

constexpr float kFeatNone = 130.0f;

// 128-bit gap (a - b) of two keys, octave-encoded
__device__ __forceinline__ float key_gap_octave(uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl) {
    const uint64_t gl = al - bl, gh = ah - bh - (al < bl ? 1u : 0u);
    return octave128(gh, gl);
}

// The 4 * curves features of one query into xs (warp-shared), from the
// positions pos_w of lists 0..curves-1 (khi/klo: lane c holds curve c's key).
// All curves at once: the 8-entry centre windows fill 32-row steps (slot
// 8 c + j = entry j of curve c's window, distances parked in sd), and lanes
// 2 c, 2 c + 1 take curve c's predecessor and successor gaps (a low key word
// recomputed from its row where the index keeps high words only).
__device__ void query_features(const IndexView& ix, const uint8_t* qrow, uint4 qv0,
                               const uint32_t* pos_w, uint64_t khi, uint64_t klo, float* xs,
                               uint32_t* sd, int lane) {
    const uint8_t* db = static_cast<const uint8_t*>(ix.db);
    const uint32_t C = ix.P.curves;
    // centre window of curve c = lane / 8 (per slot)
    for (uint32_t t = 0; t < C; t += 4) {
        const uint32_t c = t + (uint32_t)lane / 8, j = (uint32_t)lane % 8;
        uint32_t id = 0;
        bool valid = false;
        if (c < C) {
            const uint64_t off = ix.list_off[c];
            const uint32_t n = (uint32_t)(ix.list_off[c + 1] - off);
            const uint32_t pos = pos_w[c];
            const uint32_t lo = pos > 4 ? pos - 4 : 0u, hi = pos + 4 < n ? pos + 4 : n;
            valid = lo + j < hi;
            if (valid) id = __ldg(ix.ids + off + lo + j);
            if (!HC_IN_BOUNDS(kSiteRow, id, ix.rows)) id = 0u;
        }
        uint64_t cands[ChunkWidth<8>::NG];
        chunk_candidates_n<false, 8>(db, ix.row_bytes, qrow, qv0, id, 32u, lane, cands);
        // lane l holds the row (l % 8) * 4 + l / 8 of the step
        const uint32_t r = ((uint32_t)lane % 8) * 4 + (uint32_t)lane / 8;
        const bool rvalid = __shfl_sync(0xffffffffu, valid, (int)r);
        sd[8 * t + r] = rvalid ? (uint32_t)(cands[0] >> 32) : 0xFFFFFFFFu;
    }
    __syncwarp();
    float f0 = kFeatNone, f1 = kFeatNone, f2 = kFeatNone, f3 = kFeatNone;
    {
        // lanes 2c, 2c+1: predecessor / successor gap of curve c
        const uint32_t c = (uint32_t)lane / 2;
        const uint64_t kh = __shfl_sync(0xffffffffu, khi, (int)(c < C ? c : 0));
        const uint64_t kl = __shfl_sync(0xffffffffu, klo, (int)(c < C ? c : 0));
        float gap = kFeatNone;
        if (c < C) {
            const uint64_t off = ix.list_off[c];
            const uint32_t n = (uint32_t)(ix.list_off[c + 1] - off);
            const uint32_t pos = pos_w[c];
            if ((lane & 1) == 0 && pos > 0) {
                const uint64_t g = off + pos - 1;
                gap = key_gap_octave(kh, kl, ix.keys_hi[g], entry_key_lo(ix, c, g));
            } else if ((lane & 1) == 1 && pos < n) {
                const uint64_t g = off + pos;
                gap = key_gap_octave(ix.keys_hi[g], entry_key_lo(ix, c, g), kh, kl);
            }
        }
        const float other = __shfl_xor_sync(0xffffffffu, gap, 1);
        f0 = (lane & 1) ? other : gap;
        f1 = (lane & 1) ? gap : other;
    }
    if ((uint32_t)lane < C) {
        // centre-window distances of curve lane
        uint32_t dmin = 0xFFFFFFFFu, cnt = 0;
        uint64_t dsum = 0;
        for (uint32_t j = 0; j < 8; ++j) {
            const uint32_t v = sd[8 * lane + j];
            if (v != 0xFFFFFFFFu) {
                dmin = min(dmin, v);
                dsum += v;
                ++cnt;
            }
        }
        if (cnt) {
            f2 = octave128(0, dmin);
            f3 = octave128(0, dsum / cnt);
        }
    }
    // lane c < C gathers its curve's gap pair from lane 2c
    const float g0 = __shfl_sync(0xffffffffu, f0, (2 * lane) & 31);
    const float g1 = __shfl_sync(0xffffffffu, f1, (2 * lane) & 31);
    if ((uint32_t)lane < C) {
        xs[4 * lane + 0] = g0;
        xs[4 * lane + 1] = g1;
        xs[4 * lane + 2] = f2;
        xs[4 * lane + 3] = f3;
    }
    __syncwarp();
}

__device__ __forceinline__ void warp_keys_positions(const IndexView& ix, const uint8_t* qrow,
                                                    uint32_t* pos_w, uint64_t& khi, uint64_t& klo,
                                                    int lane) {
    khi = 0;
    klo = 0;
    const uint32_t curves = ix.P.curves;
    if ((uint32_t)lane < curves) curve_key_call(qrow, ix.P, (uint32_t)lane, khi, klo);
    if ((uint32_t)lane < curves) {
        const uint64_t off = ix.list_off[lane];
        const uint32_t n = (uint32_t)(ix.list_off[lane + 1] - off);
        pos_w[lane] = lower_bound_key(ix, (uint32_t)lane, off, n, khi, klo);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kPredWarps * 32) features_kernel(IndexView ix, const uint8_t* q,
                                                                   uint32_t nq, float* feat) {
    __shared__ uint32_t s_pos[kPredWarps][64 + 128];   // positions, then window distances
    __shared__ float s_x[kPredWarps][4 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t qi = blockIdx.x * kPredWarps + warp;
    if (qi >= nq) return;
    const uint8_t* qrow = q + (size_t)qi * ix.row_bytes;
    uint64_t khi, klo;
    warp_keys_positions(ix, qrow, s_pos[warp], khi, klo, lane);
    const uint32_t s = (uint32_t)lane % 8;
    const uint4 qv0 = s < (ix.row_bytes >> 4) ? ldg16(qrow + s * 16) : make_uint4(0, 0, 0, 0);
    query_features(ix, qrow, qv0, s_pos[warp], khi, klo, s_x[warp], s_pos[warp] + 64, lane);
    for (uint32_t j = lane; j < 4 * ix.P.curves; j += 32)
        feat[(size_t)qi * 4 * ix.P.curves + j] = s_x[warp][j];
}

// features -> MLP -> p = clamp(ceil(2^(y + margin)), p_lo, p_hi), per query
__global__ void __launch_bounds__(kPredWarps * 32, 4) predict_depths_kernel(
    IndexView ix, MlpView V, const uint8_t* q, uint32_t nq, float margin, uint32_t p_lo,
    uint32_t p_hi, uint32_t* p_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    const uint32_t nw = V.in * V.h1 + V.h1 * V.h2 + V.h2;
    float* sb = reinterpret_cast<float*>(smem_raw + ((nw * 2 + 15) & ~15u));
    float* sx = sb + 4 * kMaxDim + 1 + 3;
    uint32_t* spos = reinterpret_cast<uint32_t*>(sx + kPredWarps * 2 * kMaxDim);
    stage_weights(V, sW, sb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* xs = sx + warp * 2 * kMaxDim;
    float* hs = xs + kMaxDim;
    uint32_t* pos_w = spos + warp * (64 + 128);
    for (uint32_t qi = blockIdx.x * kPredWarps + warp; qi < nq; qi += gridDim.x * kPredWarps) {
        const uint8_t* qrow = q + (size_t)qi * ix.row_bytes;
        uint64_t khi, klo;
        warp_keys_positions(ix, qrow, pos_w, khi, klo, lane);
        const uint32_t s = (uint32_t)lane % 8;
        const uint4 qv0 = s < (ix.row_bytes >> 4) ? ldg16(qrow + s * 16) : make_uint4(0, 0, 0, 0);
        query_features(ix, qrow, qv0, pos_w, khi, klo, xs, pos_w + 64, lane);
        const float y = mlp_warp_forward(V, sW, sW + V.in * V.h1, sW + V.in * V.h1 + V.h1 * V.h2,
                                         sb, xs, hs, lane);
        if (lane == 0) {
            const float e = fminf(fmaxf(y + margin, -1.0f), 30.0f);
            float pf = ceilf(exp2f(e));
            uint32_t p = (uint32_t)pf;
            p = p < p_lo ? p_lo : (p > p_hi ? p_hi : p);
            p_out[qi] = p;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- labels
__global__ void fill_kernel(uint32_t* __restrict__ a, uint32_t v, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void label_mid_kernel(const uint32_t* __restrict__ lo, const uint32_t* __restrict__ hi,
                                 uint32_t* __restrict__ mid, uint32_t nq) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nq) mid[i] = lo[i] < hi[i] ? (lo[i] + hi[i]) / 2 : hi[i];
}

__global__ void label_update_kernel(const int32_t* __restrict__ ids, const int32_t* __restrict__ ref,
                                    uint32_t nq, uint32_t k, uint32_t* __restrict__ lo,
                                    uint32_t* __restrict__ hi, const uint32_t* __restrict__ mid) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq || lo[i] >= hi[i]) return;
    bool same = true;
    for (uint32_t j = 0; j < k; ++j) same &= ids[(size_t)i * k + j] == ref[(size_t)i * k + j];
    if (same) hi[i] = mid[i];
    else lo[i] = mid[i] + 1;
}

MlpView view_of_mlp(const hc_mlp* M) {
    MlpView V;
    V.in = M->in;
    V.h1 = M->h1;
    V.h2 = M->h2;
    V.wbf = M->wbf;
    V.params = M->params;
    V.L = layout_of(M->in, M->h1, M->h2);
    return V;
}

bool dev_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int features_ok(const hc_index* idx) {
    if (!idx) return HC_ERR_ARG;
    if (idx->params.dtype != HC_U8 || idx->params.partitions != 1) return HC_ERR_ARG;
    if (idx->params.curves > 16 || idx->row_bytes > 8 * 16 * 32) return HC_ERR_ARG;
    return HC_OK;
}

// -------------------------------------------------------------- training
// regression target of a depth label: log2(max(label, 1))
__global__ void fit_targets_kernel(const uint32_t* __restrict__ labels, uint32_t n,
                                   float* __restrict__ t) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) t[i] = log2f((float)(labels[i] > 1u ? labels[i] : 1u));
}

// One block per feature column: mean, then the unbiased standard deviation
// about it (two passes, float64 sums); mu = mean, isd = 1 / max(sd, 1e-3).
__global__ void __launch_bounds__(256) fit_stats_kernel(const float* __restrict__ x, uint32_t n,
                                                        uint32_t in, float* __restrict__ mu,
                                                        float* __restrict__ isd) {
    __shared__ double red[8];
    __shared__ double mean_s;
    const uint32_t c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc = 0.0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) acc += (double)x[(size_t)i * in + c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        mean_s = t / (double)n;
    }
    __syncthreads();
    const double mean = mean_s;
    acc = 0.0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = (double)x[(size_t)i * in + c] - mean;
        acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __syncthreads();
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        const double sd = n > 1 ? sqrt(t / (double)(n - 1)) : 0.0;
        mu[c] = (float)mean;
        isd[c] = (float)(1.0 / (sd > 1e-3 ? sd : 1e-3));
    }
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of a counter
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// random 32-bit sort keys of epoch e: the order of the samples in that epoch
__global__ void fit_keys_kernel(uint64_t seed, uint32_t epoch, uint32_t n,
                                uint64_t* __restrict__ keys) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        keys[i] = splitmix64(seed ^ ((uint64_t)epoch << 40) ^ (uint64_t)i) >> 32;
}

// minibatch j of an epoch: rows perm[b0 .. b0 + b) of x and t, made contiguous
__global__ void fit_gather_kernel(const float* __restrict__ x, const float* __restrict__ t,
                                  const uint32_t* __restrict__ perm, uint32_t b0, uint32_t b,
                                  uint32_t in, float* __restrict__ xb, float* __restrict__ tb) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= b * in) return;
    const uint32_t j = k / in, c = k % in;
    const uint32_t r = perm[b0 + j];
    xb[k] = x[(size_t)r * in + c];
    if (c == 0) tb[j] = t[r];
}

}  // namespace

// predictor launch used by the serving loop (serve.cu)
namespace hc {
int mlp_prepare_inference(hc_mlp* M, const hc_index* idx, cudaStream_t s) {
    if (!M || !idx || M->in != 4 * idx->params.curves) return HC_ERR_ARG;
    if (int rc = refresh_bf16(M, s)) return rc;
    return cudaStreamSynchronize(s) == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}

cudaError_t launch_predict_depths(hc_mlp* M, const hc_index* idx, const void* q, uint32_t nq,
                                  float margin, uint32_t p_lo, uint32_t p_hi, uint32_t* p_out,
                                  cudaStream_t s) {
    if (nq == 0) return cudaSuccess;
    if (refresh_bf16(M, s) != HC_OK) return cudaErrorUnknown;
    const MlpView V = view_of_mlp(M);
    const size_t smem = pred_smem(V);
    cudaError_t e = cudaFuncSetAttribute(predict_depths_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned blocks = (nq + kPredWarps - 1) / kPredWarps;
    if (blocks > (unsigned)sms * 8) blocks = sms * 8;
    predict_depths_kernel<<<blocks, kPredWarps * 32, smem, s>>>(
        view_of(idx), V, static_cast<const uint8_t*>(q), nq, margin, p_lo, p_hi, p_out);
    count_launches(1);
    return cudaGetLastError();
}
}  // namespace hc

extern "C" {

HC_API int hc_features(hc_index* idx, const void* q_dev, uint32_t nq, float* feat_dev,
                       void* cuda_stream) {
    TraceRange tr("hc_features");
    if (int rc = features_ok(idx)) return rc;
    if (nq == 0) return HC_OK;
    if (!dev_ptr(q_dev) || !dev_ptr(feat_dev) || ((uintptr_t)q_dev & 15)) return HC_ERR_ARG;
    features_kernel<<<(nq + kPredWarps - 1) / kPredWarps, kPredWarps * 32, 0,
                      static_cast<cudaStream_t>(cuda_stream)>>>(
        view_of(idx), static_cast<const uint8_t*>(q_dev), nq, feat_dev);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}

HC_API int hc_probe_labels(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k,
                           uint32_t p_max, uint32_t* p_min_dev, void* cuda_stream) {
    TraceRange tr("hc_probe_labels");
    if (!idx || k < 1 || k > 128 || p_max > (1u << 30)) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!dev_ptr(q_dev) || !dev_ptr(p_min_dev) || ((uintptr_t)q_dev & 15)) return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t res = (size_t)nq * k * 4;
    const size_t bytes = 3 * res + 2 * (size_t)nq * 4 + 1024;
    if (alloc_should_fail()) return HC_ERR_OOM;
    char* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return HC_ERR_OOM;
    }
    int32_t* ref = reinterpret_cast<int32_t*>(buf);
    int32_t* ids = reinterpret_cast<int32_t*>(buf + res);
    void* dist = buf + 2 * res;
    uint32_t* lo = reinterpret_cast<uint32_t*>(buf + 3 * res);
    uint32_t* mid = lo + nq;
    uint32_t* hi = p_min_dev;
    const IndexView ix = view_of(idx);
    int rc = HC_OK;
    if (launch_query(ix, q_dev, nq, k, p_max, ref, dist, s) != cudaSuccess) rc = HC_ERR_CUDA;
    if (!rc && (cudaMemsetAsync(lo, 0, (size_t)nq * 4, s) != cudaSuccess)) rc = HC_ERR_CUDA;
    if (!rc) {
        fill_kernel<<<(nq + 255) / 256, 256, 0, s>>>(hi, p_max, nq);   // hi = p_max
        count_launches(1);
    }
    uint32_t iters = 1;
    while ((1u << iters) <= p_max + 1) ++iters;
    for (uint32_t it = 0; !rc && it <= iters; ++it) {
        const unsigned g = (nq + 255) / 256;
        label_mid_kernel<<<g, 256, 0, s>>>(lo, hi, mid, nq);
        if (launch_query(ix, q_dev, nq, k, 0, ids, dist, s, mid) != cudaSuccess) rc = HC_ERR_CUDA;
        label_update_kernel<<<g, 256, 0, s>>>(ids, ref, nq, k, lo, hi, mid);
        count_launches(2);
        if (cudaGetLastError() != cudaSuccess) rc = HC_ERR_CUDA;
    }
    cudaFreeAsync(buf, s);
    return rc;
}

HC_API int hc_mlp_create(uint32_t in_dim, uint32_t hidden1, uint32_t hidden2, uint32_t max_batch,
                         hc_mlp** out) {
    if (!out) return HC_ERR_ARG;
    *out = nullptr;
    if (in_dim < 1 || in_dim > kMaxDim || hidden1 < 1 || hidden1 > kMaxDim || hidden2 < 1 ||
        hidden2 > kMaxDim || max_batch < 1 || max_batch > (1u << 20))
        return HC_ERR_ARG;
    hc_mlp* M = new (std::nothrow) hc_mlp();
    if (!M) return HC_ERR_OOM;
    M->in = in_dim;
    M->h1 = hidden1;
    M->h2 = hidden2;
    M->max_batch = max_batch;
    const Layout L = layout_of(in_dim, hidden1, hidden2);
    M->nparam = L.total_trained;
    const size_t nw = (size_t)in_dim * hidden1 + (size_t)hidden1 * hidden2 + hidden2;
    bool ok = !alloc_should_fail();
    ok = ok && cudaMalloc(&M->params, sizeof(float) * L.total) == cudaSuccess;
    ok = ok && cudaMalloc(&M->grads, sizeof(float) * L.total_trained) == cudaSuccess;
    ok = ok && cudaMalloc(&M->adam_m, sizeof(float) * L.total_trained) == cudaSuccess;
    ok = ok && cudaMalloc(&M->adam_v, sizeof(float) * L.total_trained) == cudaSuccess;
    ok = ok && cudaMalloc(&M->wbf, sizeof(__nv_bfloat16) * nw) == cudaSuccess;
    ok = ok && cudaMalloc(&M->work, sizeof(float) * work_floats(in_dim, hidden1, hidden2,
                                                                  max_batch)) == cudaSuccess;
    ok = ok && cudaMalloc(&M->loss, sizeof(float)) == cudaSuccess;
    if (ok) {
        ok = cudaMemset(M->params, 0, sizeof(float) * L.total) == cudaSuccess &&
             cudaMemset(M->adam_m, 0, sizeof(float) * L.total_trained) == cudaSuccess &&
             cudaMemset(M->adam_v, 0, sizeof(float) * L.total_trained) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        hc_mlp_free(M);
        return HC_ERR_OOM;
    }
    *out = M;
    return HC_OK;
}

HC_API uint32_t hc_mlp_param_count(const hc_mlp* M) { return M ? M->nparam : 0; }

HC_API int hc_mlp_set_params(hc_mlp* M, const float* params_host, const float* mu_host,
                             const float* isd_host) {
    if (!M || !params_host || !mu_host || !isd_host) return HC_ERR_ARG;
    const Layout L = layout_of(M->in, M->h1, M->h2);
    if (cudaMemcpy(M->params, params_host, sizeof(float) * L.total_trained,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(M->params + L.mu, mu_host, sizeof(float) * M->in, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(M->params + L.isd, isd_host, sizeof(float) * M->in, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(M->adam_m, 0, sizeof(float) * L.total_trained) != cudaSuccess ||
        cudaMemset(M->adam_v, 0, sizeof(float) * L.total_trained) != cudaSuccess)
        return HC_ERR_CUDA;
    M->steps = 0;
    M->bf_stale = true;
    return HC_OK;
}

HC_API int hc_mlp_get_params(const hc_mlp* M, float* params_host, float* mu_host, float* isd_host) {
    if (!M || !params_host) return HC_ERR_ARG;
    const Layout L = layout_of(M->in, M->h1, M->h2);
    if (cudaMemcpy(params_host, M->params, sizeof(float) * L.total_trained,
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return HC_ERR_CUDA;
    if (mu_host && cudaMemcpy(mu_host, M->params + L.mu, sizeof(float) * M->in,
                              cudaMemcpyDeviceToHost) != cudaSuccess)
        return HC_ERR_CUDA;
    if (isd_host && cudaMemcpy(isd_host, M->params + L.isd, sizeof(float) * M->in,
                               cudaMemcpyDeviceToHost) != cudaSuccess)
        return HC_ERR_CUDA;
    return HC_OK;
}

HC_API int hc_mlp_gradients(hc_mlp* M, const float* x_dev, const float* t_dev, uint32_t n,
                            float* grads_dev, float* loss_host, void* cuda_stream) {
    if (!M || n < 1 || n > M->max_batch || !dev_ptr(x_dev) || !dev_ptr(t_dev)) return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (int rc = forward_backward(M, x_dev, t_dev, n, s, true)) return rc;
    if (grads_dev && cudaMemcpyAsync(grads_dev, M->grads, sizeof(float) * M->nparam,
                                     cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HC_ERR_CUDA;
    if (loss_host) {
        if (cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HC_ERR_CUDA;
    }
    return HC_OK;
}

}  // extern "C"

namespace {
// forward, backward and one Adam step (beta 0.9 / 0.999, eps 1e-8) on a batch
int train_step(hc_mlp* M, const float* x_dev, const float* t_dev, uint32_t n, float lr,
               cudaStream_t s) {
    if (int rc = forward_backward(M, x_dev, t_dev, n, s, true)) return rc;
    M->steps += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)M->steps));
    const float c2 = (float)(1.0 - std::pow(b2, (double)M->steps));
    adam_kernel<<<(M->nparam + 255) / 256, 256, 0, s>>>(M->params, M->grads, M->adam_m, M->adam_v,
                                                        M->nparam, lr, (float)b1, (float)b2, 1e-8f,
                                                        c1, c2);
    count_launches(1);
    M->bf_stale = true;
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}
}  // namespace

extern "C" {

HC_API int hc_mlp_train_step(hc_mlp* M, const float* x_dev, const float* t_dev, uint32_t n,
                             float lr, float* loss_host, void* cuda_stream) {
    if (!M || n < 1 || n > M->max_batch || !(lr > 0.f)) return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (int rc = train_step(M, x_dev, t_dev, n, lr, s)) return rc;
    if (loss_host) {
        if (cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HC_ERR_CUDA;
    }
    return HC_OK;
}

HC_API int hc_mlp_fit(hc_mlp* M, const float* feat_dev, const uint32_t* labels_dev, uint32_t n,
                      uint32_t epochs, uint32_t batch, float lr, uint64_t seed, float* losses_host,
                      void* cuda_stream) {
    TraceRange tr("hc_mlp_fit");
    if (!M || batch < 1 || batch > M->max_batch || n < batch || epochs < 1 || !(lr > 0.f) ||
        !losses_host || !dev_ptr(feat_dev) || !dev_ptr(labels_dev))
        return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const Layout L = layout_of(M->in, M->h1, M->h2);
    const uint32_t nbatch = n / batch;              // whole minibatches per epoch
    const uint32_t every = 50;                      // minibatches between recorded losses
    const uint32_t logs = (nbatch + every - 1) / every;
    // scratch: targets | sort keys | sorted keys (two) | permutation | batch | losses | sort
    SortProblem sp;
    sp.seg_off = {0, (uint64_t)n};
    sp.key_bits = 32;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_t = 0, o_keys = al(4ull * n), o_sh = o_keys + al(8ull * n),
                 o_sl = o_sh + al(8ull * n), o_perm = o_sl + al(8ull * n),
                 o_seg = o_perm + al(4ull * n), o_xb = o_seg + 256,
                 o_tb = o_xb + al(4ull * batch * M->in), o_log = o_tb + al(4ull * batch),
                 o_sort = o_log + al(4ull * logs * epochs), bytes = o_sort + sort_scratch_bytes(sp);
    if (alloc_should_fail()) return HC_ERR_OOM;
    char* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return HC_ERR_OOM;
    }
    float* t = reinterpret_cast<float*>(buf + o_t);
    uint64_t* keys = reinterpret_cast<uint64_t*>(buf + o_keys);
    uint32_t* perm = reinterpret_cast<uint32_t*>(buf + o_perm);
    uint64_t* seg = reinterpret_cast<uint64_t*>(buf + o_seg);   // seg_off[2], id_base[1]
    float* xb = reinterpret_cast<float*>(buf + o_xb);
    float* tb = reinterpret_cast<float*>(buf + o_tb);
    float* lg = reinterpret_cast<float*>(buf + o_log);
    int rc = HC_OK;
    fit_targets_kernel<<<(n + 255) / 256, 256, 0, s>>>(labels_dev, n, t);
    fit_stats_kernel<<<M->in, 256, 0, s>>>(feat_dev, n, M->in, M->params + L.mu,
                                           M->params + L.isd);
    count_launches(2);
    const uint64_t small[3] = {0, (uint64_t)n, 0};
    if (upload_small(seg, small, sizeof(small), s) != cudaSuccess) rc = HC_ERR_CUDA;
    sp.seg_off_dev = seg;
    sp.hi = keys;   // carried along; only the 32 key bits in the low word are compared
    sp.lo = keys;
    sp.ids = nullptr;
    sp.id_base_dev = seg + 2;   // ids = positions: the sorted ids are the permutation
    sp.out_hi = reinterpret_cast<uint64_t*>(buf + o_sh);
    sp.out_lo = reinterpret_cast<uint64_t*>(buf + o_sl);
    sp.out_ids = perm;
    std::vector<float> host_log((size_t)logs * epochs, 0.f);
    for (uint32_t e = 0; !rc && e < epochs; ++e) {
        fit_keys_kernel<<<(n + 255) / 256, 256, 0, s>>>(seed, e, n, keys);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess || (rc = sort_segments(sp, buf + o_sort, s))) {
            if (!rc) rc = HC_ERR_CUDA;
            break;
        }
        for (uint32_t j = 0; !rc && j < nbatch; ++j) {
            const uint32_t cnt = batch * M->in;
            fit_gather_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(feat_dev, t, perm, j * batch, batch,
                                                                M->in, xb, tb);
            count_launches(1);
            rc = train_step(M, xb, tb, batch, lr, s);
            if (!rc && j % every == 0 &&
                cudaMemcpyAsync(lg + (size_t)e * logs + j / every, M->loss, sizeof(float),
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                rc = HC_ERR_CUDA;
        }
    }
    if (!rc && (cudaMemcpyAsync(host_log.data(), lg, sizeof(float) * host_log.size(),
                                cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess))
        rc = HC_ERR_CUDA;
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    for (uint32_t e = 0; e < epochs; ++e) {
        double sum = 0.0;
        for (uint32_t j = 0; j < logs; ++j) sum += host_log[(size_t)e * logs + j];
        losses_host[e] = (float)(sum / logs);
    }
    return HC_OK;
}

HC_API int hc_mlp_forward(hc_mlp* M, const float* x_dev, uint32_t n, int bf16, float* y_dev,
                          void* cuda_stream) {
    if (!M || !dev_ptr(x_dev) || !dev_ptr(y_dev)) return HC_ERR_ARG;
    if (n == 0) return HC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!bf16) {
        const Work w = work_of(M);
        for (uint32_t b0 = 0; b0 < n; b0 += M->max_batch) {
            const uint32_t b = n - b0 < M->max_batch ? n - b0 : M->max_batch;
            if (int rc = forward_backward(M, x_dev + (size_t)b0 * M->in, nullptr, b, s, false))
                return rc;
            if (cudaMemcpyAsync(y_dev + b0, w.y, sizeof(float) * b, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                return HC_ERR_CUDA;
        }
        return HC_OK;
    }
    if (int rc = refresh_bf16(M, s)) return rc;
    const MlpView V = view_of_mlp(M);
    const size_t smem = pred_smem(V);
    if (cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return HC_ERR_CUDA;
    unsigned blocks = (n + kPredWarps - 1) / kPredWarps;
    if (blocks > 2048) blocks = 2048;
    mlp_infer_kernel<<<blocks, kPredWarps * 32, smem, s>>>(V, x_dev, n, y_dev);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}

HC_API int hc_mlp_predict_depths(hc_mlp* M, hc_index* idx, const void* q_dev, uint32_t nq,
                                 float margin, uint32_t p_lo, uint32_t p_hi, uint32_t* p_dev,
                                 void* cuda_stream) {
    TraceRange tr("hc_mlp_predict_depths");
    if (!M || features_ok(idx) != HC_OK || M->in != 4 * idx->params.curves) return HC_ERR_ARG;
    if (p_lo > p_hi || p_hi > (1u << 30)) return HC_ERR_ARG;
    if (nq == 0) return HC_OK;
    if (!dev_ptr(q_dev) || !dev_ptr(p_dev) || ((uintptr_t)q_dev & 15)) return HC_ERR_ARG;
    return launch_predict_depths(M, idx, q_dev, nq, margin, p_lo, p_hi, p_dev,
                                 static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
               ? HC_OK
               : HC_ERR_CUDA;
}

HC_API void hc_mlp_free(hc_mlp* M) {
    if (!M) return;
    cudaFree(M->params);
    cudaFree(M->grads);
    cudaFree(M->adam_m);
    cudaFree(M->adam_v);
    cudaFree(M->wbf);
    cudaFree(M->work);
    cudaFree(M->loss);
    cudaGetLastError();
    delete M;
}

}  // extern "C"
