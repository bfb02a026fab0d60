/*
 * hc.h -- C ABI of libhc.so: batched approximate kNN over Hilbert-curve
 * subindexes (Multicurves / Hypercurves, Teodoro et al., arXiv:1209.0410),
 * GPU-resident on one NVIDIA GB300 (sm_103a).
 *
 * Vocabulary (the paper's notation):
 *   B, n     database of n vectors of d coordinates (Algorithm 1 input)
 *   curves   number of subindexes per partition; each curve c indexes the
 *            dims_per_curve coordinates a[c][0..m) of every vector
 *   C^-1     the Hilbert extended-key of a projection (Sec. 2.2.1): m
 *            coordinates of 8 bits -> one key of 8m bits (at most 128)
 *   p        probe depth per side: the search takes the p list entries below
 *            the query key and the p at or above it (the paper's depth is 2p)
 *   k        neighbours returned per query
 *   l        partitions (Hypercurves, Sec. 4.1): the database is split into
 *            l disjoint id ranges, each with its own curves sorted lists
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_dev are device pointers on the current CUDA device;
 *     *_host are host pointers (pinned or pageable).  The caller owns every
 *     buffer it passes in.  Row-major layouts throughout.
 *   - cuda_stream is a cudaStream_t cast to void* (NULL = legacy default
 *     stream).  Entry points taking device buffers are asynchronous on that
 *     stream unless stated otherwise; results are valid once the stream
 *     reaches the point of the call.
 *   - Every entry point returns an hc_status; no C++ exception crosses the
 *     ABI.  hc_strerror() names a status.  On an error return nothing has
 *     been written to the caller's output buffers unless stated otherwise.
 *   - Distances are squared Euclidean (Eq. 2 squared: same ranking).  uint8
 *     data gives exact int32 distances; float32 data accumulates in float32.
 *   - Results are ordered by ascending (distance, id): equal distances rank
 *     the lower id first.  When fewer than k distinct candidates exist the
 *     tail is padded with id -1 and distance INT32_MAX (uint8) or +inf
 *     (float32).
 *   - The Hilbert orientation is that of Skilling's transpose formulation
 *     ("Programming the Hilbert curve", 2004): key bits are read level by
 *     level from the top coordinate bit, axis 0 first.  Float32 coordinates
 *     enter keys as (uint8)clamp(rint(x * 255f), 0, 255), decided in float32.
 */
#ifndef HC_H
#define HC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HC_API __attribute__((visibility("default")))
#else
#define HC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- statuses */
typedef enum {
    HC_OK = 0,
    HC_PENDING = 1,             /* hc_serve_poll: the request has not finished */
    HC_ERR_ARG = -1,            /* an argument is out of range or inconsistent */
    HC_ERR_OOM = -2,            /* a device or host allocation failed */
    HC_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    HC_ERR_BUDGET = -4,         /* admission refused: over the HBM budget */
    HC_ERR_TIMEOUT = -5,        /* a host-side wait ran out of time */
    HC_ERR_DEVICE_STATUS = -6,  /* a kernel reported an error status */
    HC_ERR_STATE = -7,          /* object used in the wrong state (e.g. an unknown ticket) */
    HC_ERR_IO = -8,             /* a file could not be opened, read or written */
    HC_ERR_FORMAT = -9          /* a file is not an index file of this library, is damaged,
                                   or does not index the database it is loaded over */
} hc_status;

typedef enum { HC_U8 = 0, HC_F32 = 1 } hc_dtype;

typedef struct hc_index hc_index;

/* Index construction parameters (Algorithm 1 inputs B, curves, dims[], a). */
typedef struct {
    uint64_t n;                /* rows, 1 <= n < 2^31 and curves * n < 2^32 */
    uint32_t d;                /* coordinates per row; rows must be a multiple
                                  of 16 bytes (d % 16 == 0 for HC_U8,
                                  d % 4 == 0 for HC_F32), d <= 4096 */
    uint32_t curves;           /* subindexes per partition, 1..32 */
    uint32_t dims_per_curve;   /* m, 1..16 (keys of 8m bits) */
    uint32_t bits;             /* coordinate bits; must be 8 */
    hc_dtype dtype;            /* HC_U8 or HC_F32 */
    const uint32_t* dim_map;   /* HOST array a[c][j], curves*m entries, each < d;
                                  NULL = consecutive dims (a[c][j] = c*m + j,
                                  needs curves*m <= d).  Copied at build. */
    uint32_t partitions;       /* l >= 1 (0 is read as 1); partition j holds
                                  ids [floor(j*n/l), floor((j+1)*n/l));
                                  l * curves <= 256 */
} hc_build_params;

/*
 * hc_build -- Algorithm 1 on the GPU: for every partition and curve, the
 * extended-key of each row's projection, then a stable device radix sort of
 * (key, id), giving one list sorted by (key, id) per (partition, curve).  For
 * 16-coordinate curves the top 48 bits of the key are radix-sorted and runs
 * of equal 48-bit prefixes are then ordered by the whole key (the low word
 * recomputed from the rows) and id; shorter keys are sorted by every byte.
 *   db_dev   n x d rows (uint8 or float32 per params->dtype), 16-byte aligned.
 *            NOT copied: the index keeps the pointer, so the caller keeps the
 *            buffer alive and unchanged until hc_free.
 *   out      receives the new index (owned by the library; free with hc_free).
 * The library allocates the index arrays (12 bytes per row and curve for
 * 16-coordinate curves, whose lists keep the high key word and the id; 20
 * bytes otherwise) and, during the call, stream-ordered scratch of about 26
 * bytes per row and curve (33 when low words are kept); HC_ERR_OOM if that
 * fails.  All work is queued on cuda_stream and the call returns without
 * waiting on it; the index may be used by later work on the same stream (or
 * on another stream after an event).  On an error return nothing of the
 * index remains (the call then waits for its queued work before freeing).
 */
HC_API int hc_build(const void* db_dev, const hc_build_params* params, void* cuda_stream,
                    hc_index** out);

/*
 * hc_build_host -- as hc_build, but db_host is a HOST buffer: the library
 * copies it into device memory it owns (freed by hc_free).  Returns once the
 * index is complete on the device (synchronises cuda_stream).
 */
HC_API int hc_build_host(const void* db_host, const hc_build_params* params, void* cuda_stream,
                         hc_index** out);

/*
 * hc_build_host_async -- as hc_build_host, without waiting: the rows are
 * copied from db_host into device memory the index owns on copy_stream, and
 * the build is queued on cuda_stream behind that copy (an event), so that the
 * upload of one database can run on the copy engine while the GPU still
 * builds or queries another.
 *   db_host      n x d rows in PAGE-LOCKED host memory (cudaHostAlloc or
 *                cudaHostRegister; HC_ERR_ARG otherwise).  Read by the copy:
 *                keep it alive and unchanged until cuda_stream has reached
 *                the point of the call.
 *   copy_stream  stream of the upload; NULL = cuda_stream (no overlap).
 *   cuda_stream  the build, as for hc_build; the index is ready for later
 *                work on cuda_stream (or on a stream that waits for it).
 * The call returns once the work is queued.  Errors as hc_build; on an error
 * the call waits for both streams and nothing of the index remains.
 */
HC_API int hc_build_host_async(const void* db_host, const hc_build_params* params,
                               void* copy_stream, void* cuda_stream, hc_index** out);

/*
 * hc_query -- Algorithm 2 for nq queries at once (queries grouped into one
 * GPU batch, Sec. 5.1), fused into one kernel: per query, the extended-key
 * of every curve's projection, lower_bound in each sorted list, the window
 * [max(0, pos-p), min(n_list, pos+p)), exact distances of the window rows,
 * and one running top-k over the union of all windows of all curves and
 * partitions with duplicate ids dropped (the Aggregator's reduction of
 * Sec. 4.1 folded into the selection).
 *   q_dev         nq x d queries of the index's dtype, 16-byte aligned rows
 *   k             1..128;  p: 0..2^30 (p = 0 gives all-padding results)
 *   out_ids_dev   nq x k int32
 *   out_dist_dev  nq x k int32 (HC_U8) or float (HC_F32)
 * nq = 0 is a no-op.  No allocation; asynchronous on cuda_stream.
 */
HC_API int hc_query(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k, uint32_t p,
                    int32_t* out_ids_dev, void* out_dist_dev, void* cuda_stream);

/*
 * hc_query_ordered -- hc_query with the queries answered in the order of
 * their curve-0 extended-keys (the top 16 key bits, radix-sorted on the
 * device), so that queries answered at the same time read overlapping
 * windows and share their rows in L2.  The batch is also sorted by every
 * other curve's key, and the lower_bound of every query in every list
 * (Algorithm 2's search) runs first as one pass over the batch, 32
 * neighbouring keys of one curve per warp, into the workspace; the walk then
 * reads those positions.  The paper batches
 * queries in arrival order (Sec. 5.1); the order changes no result: every
 * query's ids and distances land in its own row and equal those of hc_query.
 *   workspace_dev    device memory of at least
 *                    hc_query_ordered_workspace(idx, nq) bytes (it depends on
 *                    the index's curves and lists, not on its rows), 256-byte
 *                    aligned, owned by the caller (contents scratch; one call
 *                    at a time per workspace)
 * Other arguments as hc_query.  No allocation; asynchronous on cuda_stream.
 * HC_ERR_ARG if the workspace is missing, misaligned or too small.
 * hc_query_ordered_workspace returns 0 for idx = NULL or nq = 0.
 */
HC_API size_t hc_query_ordered_workspace(const hc_index* idx, uint32_t nq);
HC_API int hc_query_ordered(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k, uint32_t p,
                            int32_t* out_ids_dev, void* out_dist_dev, void* workspace_dev,
                            size_t workspace_bytes, void* cuda_stream);

/*
 * hc_query_host -- hc_query from HOST buffers: copies the queries in, runs
 * the query kernel and copies the results back, on cuda_stream, and returns
 * once the results are in the host buffers.  Batches of 4096 queries or more
 * are answered in curve-0 key order as by hc_query_ordered (the same
 * results).  Device staging buffers (queries, the ordering workspace,
 * results) are owned by the index and grow on demand (HC_ERR_OOM if they
 * cannot).  Calls on the same index must not overlap (they share the
 * staging).
 */
HC_API int hc_query_host(hc_index* idx, const void* q_host, uint32_t nq, uint32_t k, uint32_t p,
                         int32_t* out_ids_host, void* out_dist_host, void* cuda_stream);

/*
 * hc_query_host_async -- as hc_query_host, without waiting: the queries go up
 * on copy_stream (NULL = cuda_stream), the walk and the copy of the results
 * back run on cuda_stream behind them (an event), and the call returns once
 * the work is queued.
 *   q_host, out_ids_host, out_dist_host   PAGE-LOCKED host buffers
 *                (HC_ERR_ARG otherwise), laid out as for hc_query_host; keep
 *                them alive and q_host unchanged until cuda_stream reaches the
 *                point of the call, which is also when the results are valid.
 * A later host query on the same index waits, on its copy stream, until this
 * call's results have left the staging.  Errors as hc_query_host.
 */
HC_API int hc_query_host_async(hc_index* idx, const void* q_host, uint32_t nq, uint32_t k,
                               uint32_t p, int32_t* out_ids_host, void* out_dist_host,
                               void* copy_stream, void* cuda_stream);

/*
 * hc_query_depths -- hc_query with one probe depth per query: p_dev holds nq
 * uint32 depths (each 0..2^30) in device memory.  Used by the serving loop to
 * mix requests of different depths in one launch and by the learned depth
 * predictor.  No allocation; asynchronous on cuda_stream.
 */
HC_API int hc_query_depths(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k,
                           const uint32_t* p_dev, int32_t* out_ids_dev, void* out_dist_dev,
                           void* cuda_stream);

/*
 * hc_query_at -- hc_query with the lower_bound step done beforehand:
 * pos_dev holds the nq x lists int64 positions of hc_query_positions for the
 * same queries (any other values give windows around those positions).  The
 * kernel then only gathers, ranks and selects.  No allocation; asynchronous.
 */
HC_API int hc_query_at(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k, uint32_t p,
                       const int64_t* pos_dev, int32_t* out_ids_dev, void* out_dist_dev,
                       void* cuda_stream);

/* hc_free -- releases an index and everything it owns (not db_dev).  The
 * caller makes sure no work using the index is still queued.  NULL is ok. */
HC_API void hc_free(hc_index* idx);

/* hc_free_async -- hc_free with the device memory released in stream order on
 * cuda_stream: work on the index queued earlier on that stream completes
 * first, and the call does not wait for other streams (the caller orders any
 * other stream's work on the index before it).  Host memory of the index is
 * released at once.  NULL is ok. */
HC_API void hc_free_async(hc_index* idx, void* cuda_stream);

/* hc_strerror -- static text for an hc_status value. */
HC_API const char* hc_strerror(int status);

/* ------------------------------------------------------- introspection */
typedef struct {
    uint64_t n;
    uint32_t d, curves, dims_per_curve, partitions, lists;
    hc_dtype dtype;
    const uint64_t* keys_hi_dev;  /* lists concatenated, list L = part*curves + c */
    const uint64_t* keys_lo_dev;  /* low 64 bits of each key; NULL when the index keeps
                                     high words only (dims_per_curve = 16: a low word is
                                     recomputed from its row when high words tie) */
    const uint32_t* ids_dev;      /* row id of each entry */
    const void* db_dev;
} hc_index_info;

/* hc_index_describe -- fills *info; the device arrays stay owned by idx.
 * list_off_host (nullable) receives lists+1 offsets of the lists. */
HC_API int hc_index_describe(const hc_index* idx, hc_index_info* info, uint64_t* list_off_host);

/* hc_index_copy_lists -- copies the sorted lists (all lists concatenated,
 * list_off order) into caller-owned device buffers of total = n * curves
 * entries each; low key words the index does not keep are recomputed from
 * the rows.  Asynchronous on cuda_stream; no allocation. */
HC_API int hc_index_copy_lists(const hc_index* idx, uint64_t* keys_hi_dev, uint64_t* keys_lo_dev,
                               uint32_t* ids_dev, void* cuda_stream);

/* ----------------------------------------------------- separate steps */

/*
 * hc_hilbert_keys -- the extended-key C^-1 of each vector's projection onto
 * every curve (Sec. 2.2.1; the per-curve step of Algorithms 1 and 2).
 *   x_dev        count x d vectors (dtype), 16-byte aligned rows
 *   dim_map_host curves*m attribution, NULL = consecutive
 *   hi_dev/lo_dev count x curves uint64 each: key = hi * 2^64 + lo
 * Asynchronous on cuda_stream; allocates only a small copy of dim_map.
 */
HC_API int hc_hilbert_keys(const void* x_dev, hc_dtype dtype, uint64_t count, uint32_t d,
                           uint32_t curves, uint32_t m, const uint32_t* dim_map_host,
                           uint64_t* hi_dev, uint64_t* lo_dev, void* cuda_stream);

/*
 * hc_sort_keys -- stable LSD radix sort of (key, id) records by their 128-bit
 * key, independently within each segment [seg_off[s], seg_off[s+1]) (the
 * sorted lists of Algorithm 1).  Equal keys keep their input order, so ids
 * that enter ascending leave ordered by (key, id).
 *   hi_dev, lo_dev, ids_dev  total = seg_off_host[nseg] records, in place
 *   seg_off_host             nseg+1 offsets (host), non-decreasing,
 *                            total < 2^32
 *   key_bits                 significant low bits of every key (1..128);
 *                            digits above them are taken as zero and skipped
 * Allocates scratch of about 36 bytes per record for the call; synchronises
 * cuda_stream before returning (the scratch is freed).
 */
HC_API int hc_sort_keys(uint64_t* hi_dev, uint64_t* lo_dev, uint32_t* ids_dev,
                        const uint64_t* seg_off_host, uint32_t nseg, uint32_t key_bits,
                        void* cuda_stream);

/*
 * hc_sort_keys_noalloc -- hc_sort_keys for callers that cannot let the
 * library allocate device memory.  The paper has no counterpart: this entry
 * point exists for deployment.  A process whose memory manager reserves the
 * whole GPU up front (where a further cudaMalloc would fail or break its
 * budget), or a latency-sensitive caller that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree, can sort with this call instead: it
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   Arguments and results are those of hc_sort_keys, with two limits:
 *   seg_off_host[nseg] <= 262,144 records and nseg <= 256 segments; larger
 *   problems return HC_ERR_ARG and touch nothing.
 *   Scratch: a fixed 10 MiB device array inside libhc.so.  Every GPU on which
 *   the library is loaded holds it until the process exits.  Every call uses
 *   the same array and it keeps the last call's contents (the sort writes
 *   everything it reads, so nothing has to be cleared first).  Calls that
 *   overlap on the GPU (different streams, or different host threads on the
 *   same device) race on that array and give wrong results: order them.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, and that lookup is when
 *   the device loads the array (CUDA loads modules lazily).  Make that first
 *   call -- a call with seg_off_host[nseg] == 0 does the set-up and nothing
 *   else -- before any stream capture begins and before the caller's memory
 *   manager reserves the device's memory.  cuda_stream must belong to the
 *   current device.  cudaDeviceReset is not supported: the address looked up
 *   before it is not valid after it.
 *   Unlike hc_sort_keys, the call is asynchronous on cuda_stream: the sorted
 *   arrays, and the scratch, are in use until the stream reaches it.
 */
HC_API int hc_sort_keys_noalloc(uint64_t* hi_dev, uint64_t* lo_dev, uint32_t* ids_dev,
                                const uint64_t* seg_off_host, uint32_t nseg, uint32_t key_bits,
                                void* cuda_stream);

/*
 * hc_query_positions -- the lower_bound step of Algorithm 2 alone: for each
 * query and list, the first entry whose key is >= the query's key.
 *   pos_dev   nq x lists int64
 */
HC_API int hc_query_positions(hc_index* idx, const void* q_dev, uint32_t nq, int64_t* pos_dev,
                              void* cuda_stream);

/*
 * hc_bruteforce -- exact kNN (Eq. 3) of nq queries over all n rows, same
 * ordering, padding and distance arithmetic as hc_query.  Used as recall
 * ground truth.  k: 1..128.  No allocation; asynchronous on cuda_stream.
 */
HC_API int hc_bruteforce(const void* db_dev, hc_dtype dtype, uint64_t n, uint32_t d,
                         const void* q_dev, uint32_t nq, uint32_t k, int32_t* out_ids_dev,
                         void* out_dist_dev, void* cuda_stream);

/* -------------------------------------------- many indexes, one launch */

/*
 * Batched uneven indexes: many hc_query calls (each an index with its own
 * dtype, d, k, p and batch size) answered by one persistent kernel.  The
 * queries are cut into tasks of (warps_per_block / warps_per_query) * tile
 * queries, the tasks are ordered by their estimated bytes (largest first) and
 * the kernel's blocks take them from an atomic counter.  warps_per_query
 * warps share a query: each searches every warps_per_query-th list into its
 * own top-k and the first folds the others' in (same results as hc_query).
 */
typedef struct {
    hc_index* index;
    const void* q_dev;           /* nq x d queries of the index's dtype */
    uint32_t nq, k, p;           /* k 1..128, p 0..2^30 */
    int32_t* out_ids_dev;        /* nq x k */
    void* out_dist_dev;          /* nq x k int32 (HC_U8) or float (HC_F32) */
    uint32_t warps_per_query;    /* 1, 2, 4 or 8 (0 = 1) */
} hc_multi_job;

typedef struct {
    uint32_t warps_per_block;    /* 1..16, a power of two (default 8) */
    uint32_t blocks_per_sm;      /* persistent blocks per SM (default 4) */
    uint32_t tile;               /* query groups per task (default 2) */
    uint32_t use_graph;          /* capture the launch in a CUDA graph */
} hc_multi_config;

typedef struct hc_multi_plan hc_multi_plan;

/*
 * hc_multi_plan_create -- validates the jobs, uploads the job and task
 * tables and, with use_graph, captures the launch in a CUDA graph.  The
 * plan refers to the jobs' buffers: new queries written into the same
 * q_dev buffers are answered by the next hc_multi_run.  cfg may be NULL.
 * The tables are copied synchronously (blocking copies); cuda_stream is not
 * used by this call.
 */
HC_API int hc_multi_plan_create(const hc_multi_job* jobs, uint32_t njobs,
                                const hc_multi_config* cfg, void* cuda_stream,
                                hc_multi_plan** out);
/* hc_multi_run -- one persistent launch (graph replay when captured). */
HC_API int hc_multi_run(hc_multi_plan* plan, void* cuda_stream);
HC_API void hc_multi_plan_free(hc_multi_plan* plan);
/* hc_query_multi -- plan, run and free in one call (no graph); returns after
 * the results are complete. */
HC_API int hc_query_multi(const hc_multi_job* jobs, uint32_t njobs, const hc_multi_config* cfg,
                          void* cuda_stream);

/* ------------------------------------------------- learned probe depth */

/*
 * Learned probe depth (not in the paper, which fixes one probe depth per
 * subindex, Algorithm 2): a small MLP predicts from cheap per-query features
 * the depth that reproduces the top-k of a large fixed depth.  The fixed-
 * depth method stays the fallback and produces the training labels.
 */
typedef struct hc_mlp hc_mlp;

/*
 * hc_features -- 4 * curves float features per query (uint8 indexes with one
 * partition, curves <= 16): for each curve c, with pos the lower_bound of the
 * query key in list c,
 *   [4c+0] oct(query key - key[pos-1]),  [4c+1] oct(key[pos] - query key),
 *   [4c+2] oct(min distance), [4c+3] oct(floor(mean distance)) over the list
 *   entries [pos-4, pos+4) clipped to the list;
 * oct(0) = 0, oct(g) = 1 + e + f/65536 with e the top set bit of g and f the
 * 16 bits below it; a missing neighbour or empty range gives 130.
 *   feat_dev  nq x (4*curves) float.  Asynchronous; no allocation.
 */
HC_API int hc_features(hc_index* idx, const void* q_dev, uint32_t nq, float* feat_dev,
                       void* cuda_stream);

/*
 * hc_probe_labels -- for each query, the minimal p in [0, p_max] whose top-k
 * (ids) equals the top-k at p_max: a per-query binary search, valid because
 * the windows and so the results are nested in p.  p_min_dev: nq uint32.
 * Allocates scratch of about 12*k + 8 bytes per query on cuda_stream.
 */
HC_API int hc_probe_labels(hc_index* idx, const void* q_dev, uint32_t nq, uint32_t k,
                           uint32_t p_max, uint32_t* p_min_dev, void* cuda_stream);

/*
 * hc_mlp_create -- an MLP in -> hidden1 -> hidden2 -> 1 (ReLU; each size
 * 1..64), y = h2 . W3 + b3 after input normalisation (x - mu) * isd.  FP32
 * parameters start at zero (set them with hc_mlp_set_params); Adam state is
 * kept on the device.  max_batch bounds the training batch.
 * Parameter layout (float): W1[in][h1], b1[h1], W2[h1][h2], b2[h2], W3[h2], b3.
 */
HC_API int hc_mlp_create(uint32_t in_dim, uint32_t hidden1, uint32_t hidden2, uint32_t max_batch,
                         hc_mlp** out);
HC_API uint32_t hc_mlp_param_count(const hc_mlp* mlp);
/* host arrays: params (param_count floats), mu and isd (in_dim floats each);
 * setting parameters resets the Adam state.  Both calls synchronise. */
HC_API int hc_mlp_set_params(hc_mlp* mlp, const float* params_host, const float* mu_host,
                             const float* isd_host);
HC_API int hc_mlp_get_params(const hc_mlp* mlp, float* params_host, float* mu_host,
                             float* isd_host);
/*
 * hc_mlp_gradients -- FP32 forward and backward of the mean squared error
 * over n <= max_batch samples (x_dev: n x in, t_dev: n targets), gradients
 * into grads_dev (param_count floats, nullable); loss_host (nullable) gets
 * the loss and makes the call synchronous.
 */
HC_API int hc_mlp_gradients(hc_mlp* mlp, const float* x_dev, const float* t_dev, uint32_t n,
                            float* grads_dev, float* loss_host, void* cuda_stream);
/* hc_mlp_train_step -- one Adam step (beta 0.9 / 0.999, eps 1e-8) at
 * learning rate lr on one batch; loss_host as above. */
HC_API int hc_mlp_train_step(hc_mlp* mlp, const float* x_dev, const float* t_dev, uint32_t n,
                             float lr, float* loss_host, void* cuda_stream);
/*
 * hc_mlp_fit -- trains the MLP on n samples, every step on the device:
 * regression targets t = log2(max(label, 1)) of the depth labels; input
 * normalisation mu = mean and isd = 1 / max(sd, 1e-3) of every feature
 * column (unbiased sd), replacing the MLP's; then `epochs` passes, each over
 * a fresh order of the samples (random 32-bit keys from SplitMix64 of
 * (seed, epoch, sample), radix-sorted), in whole minibatches of `batch`
 * samples (the remainder of an epoch is left out) gathered into contiguous
 * buffers, one Adam step (hc_mlp_train_step) per minibatch at rate lr.
 * losses_host[epochs] receives, per epoch, the mean training loss over every
 * 50th minibatch.  feat_dev: n x in float; labels_dev: n uint32.  Set the
 * initial parameters first (hc_mlp_set_params).  Allocates about
 * 50 n + 4 batch (in + 1) bytes of scratch on cuda_stream and returns when
 * the training has finished.  HC_ERR_ARG if batch > max_batch or n < batch.
 */
HC_API int hc_mlp_fit(hc_mlp* mlp, const float* feat_dev, const uint32_t* labels_dev, uint32_t n,
                      uint32_t epochs, uint32_t batch, float lr, uint64_t seed, float* losses_host,
                      void* cuda_stream);
/* hc_mlp_forward -- y for n samples; bf16 = 0: FP32 throughout; bf16 = 1:
 * inputs of every layer and weights rounded to bfloat16, FP32 accumulation
 * (the inference arithmetic of hc_mlp_predict_depths). */
HC_API int hc_mlp_forward(hc_mlp* mlp, const float* x_dev, uint32_t n, int bf16, float* y_dev,
                          void* cuda_stream);
/*
 * hc_mlp_predict_depths -- fused features + BF16 inference: for every query
 * p = clamp(ceil(2^(y + margin)), p_lo, p_hi) into p_dev (nq uint32), ready
 * for hc_query_depths.  Requires in_dim = 4 * curves.
 */
HC_API int hc_mlp_predict_depths(hc_mlp* mlp, hc_index* idx, const void* q_dev, uint32_t nq,
                                 float margin, uint32_t p_lo, uint32_t p_hi, uint32_t* p_dev,
                                 void* cuda_stream);
HC_API void hc_mlp_free(hc_mlp* mlp);

/* ------------------------------------------------------------ serving */

/*
 * Online serving over resident indexes: continuous batching under an HBM
 * budget.  The paper sends a GPU buffer of queued queries to the GPU when it
 * is full or when the GPU is idle (Sec. 6, Algorithm 3, without its CPU
 * branch here) and double-buffers the transfers (Sec. 5.2).  The server's
 * dispatcher thread dispatches a batch when no batch is running, when the
 * queued queries fill a batch, or when the oldest queued request has waited
 * max_wait_us; up to `streams` batches run at once, so requests that arrive
 * while others are on the GPU overlap with them.  The
 * device state of every in-flight request (queries, depths, results) lives in
 * an arena of exactly hbm_budget bytes allocated at creation: a request is
 * admitted into a batch only when its state fits, and one that cannot fit even
 * alone is refused at submission.  Each query is answered independently, so a
 * request's result is the same alone and in any mix.  All calls are
 * thread-safe.
 */
typedef struct hc_server hc_server;

typedef struct {
    uint32_t streams;            /* batches in flight at once, 1..16 (default 4) */
    uint32_t max_batch_queries;  /* queries that fill a batch (default 16384) */
    uint32_t default_p;          /* depth used for requests submitted with p = 0
                                    (default 128) */
    uint32_t max_wait_us;        /* latency bound: a batch also goes out, to a free
                                    stream, once the oldest queued request has waited
                                    this long (default 200; 0 = no bound) */
} hc_serve_params;

typedef struct {
    uint64_t requests;           /* submitted */
    uint64_t batches;            /* dispatched */
    uint64_t batches_done;
    uint64_t queries_done;
    uint32_t max_inflight;       /* most batches seen on the GPU at once */
    uint64_t arena_used;         /* bytes of the budget in use now */
    uint64_t queued_queries;     /* waiting for admission now */
} hc_serve_stats;

/*
 * hc_serve_create(_ex) -- starts a server over n_idx built indexes (borrowed:
 * they must outlive the server).  hbm_budget >= 4096 bytes of device memory
 * (plus the same of pinned host memory) are allocated now.  params may be
 * NULL (defaults).  HC_ERR_OOM if the budget cannot be allocated.  The call
 * first waits for all work queued on the device (the server's own streams do
 * not wait on the streams that built the indexes).
 */
HC_API int hc_serve_create(hc_index* const* idx, uint32_t n_idx, uint64_t hbm_budget,
                           hc_server** out);
HC_API int hc_serve_create_ex(hc_index* const* idx, uint32_t n_idx, uint64_t hbm_budget,
                              const hc_serve_params* params, hc_server** out);

/*
 * hc_serve_submit -- queues nq queries (HOST buffer, copied before return)
 * against index index_id, k neighbours (1..128), depth p per side (0 = the
 * server's depth predictor if one is attached, else params.default_p).
 * *ticket identifies the request.  HC_ERR_BUDGET if the request's device
 * state exceeds hbm_budget on its own.
 */
HC_API int hc_serve_submit(hc_server* srv, uint32_t index_id, const void* q_host, uint32_t nq,
                           uint32_t k, uint32_t p, uint64_t* ticket);

/*
 * hc_serve_poll -- waits up to timeout_us (0 = just check) for a request.
 * HC_OK: the nq x k ids (int32) and distances (int32 for uint8 indexes, float
 * for float32) are copied to the HOST buffers and the ticket is released.
 * HC_PENDING: not finished yet (the ticket stays valid).  HC_ERR_STATE:
 * unknown or already collected ticket.  Other errors: the request failed (the
 * ticket is released).
 */
HC_API int hc_serve_poll(hc_server* srv, uint64_t ticket, int32_t* ids_host, void* dist_host,
                         uint32_t timeout_us);

/* hc_serve_poll_ex -- hc_serve_poll that also reports, on completion, the
 * request's latency in nanoseconds: from its submission to its results
 * being ready in host memory (latency_ns nullable). */
HC_API int hc_serve_poll_ex(hc_server* srv, uint64_t ticket, int32_t* ids_host, void* dist_host,
                            uint32_t timeout_us, uint64_t* latency_ns);

/*
 * hc_serve_attach_predictor -- requests on index_id submitted with p = 0 get
 * a per-query depth from the learned predictor (hc_mlp_predict_depths with
 * these margin / p_lo / p_hi) instead of params.default_p.  mlp is borrowed
 * (outlives the server); NULL detaches.  The index must qualify for
 * hc_features.
 */
HC_API int hc_serve_attach_predictor(hc_server* srv, uint32_t index_id, hc_mlp* mlp, float margin,
                                     uint32_t p_lo, uint32_t p_hi);

/* hc_serve_stats_get -- counters of the server (see hc_serve_stats). */
HC_API int hc_serve_stats_get(hc_server* srv, hc_serve_stats* out);

/* hc_serve_destroy -- finishes the queued and running requests, then frees
 * the server (uncollected results are dropped).  NULL is ok. */
HC_API void hc_serve_destroy(hc_server* srv);

/* --------------------------------------------------------- index files */

/*
 * hc_save -- writes an index to the file `path`: its build parameters, list
 * offsets, and every list's sorted high key words, stored low key words
 * (curves of fewer than 16 coordinates) and ids, i.e. the output of
 * Algorithm 1.  The database rows are NOT written: hc_load takes them again.
 * No counterpart in the paper, which rebuilds its index from the database.
 *   idx          an index (hc_build, hc_build_host or hc_load); unchanged.
 *   path         file name; written as path + ".tmp", then renamed over path,
 *                so a reader never sees a half-written file.
 *   cuda_stream  waited for first (the index may still be building on it);
 *                the lists are then copied to the host through a 32 MB buffer.
 * Layout (little-endian, each section a multiple of 8 bytes): an 80-byte
 * header ("HCURVIDX", u32 version 1, u32 byte-order mark 0x01020304, u64 n,
 * u32 d, curves, dims_per_curve, bits, dtype, partitions, lists, row_bytes,
 * flags (bit 0: low words stored, bit 1: dim map stored), u32 0, u64 total
 * entries), u64 list_off[lists + 1], u32 dim_map[curves * dims_per_curve]
 * (flag bit 1, zero-padded), u64 keys_hi[total], u64 keys_lo[total] (flag
 * bit 0), u32 ids[total] (zero-padded), then a u64 checksum of every 64-bit
 * word before it.  About 12 bytes per row and curve (20 with low words).
 * Returns HC_ERR_ARG for a null index or path, HC_ERR_IO when the file cannot
 * be written (the temporary file is removed), HC_ERR_CUDA if a copy fails.
 * Synchronous; safe while other threads query the same index.
 */
HC_API int hc_save(const hc_index* idx, const char* path, void* cuda_stream);

/*
 * hc_load -- an index from a file hc_save wrote, over the database it was
 * built from.
 *   path         the file.
 *   db_dev       the n x d rows the index was built from (device memory,
 *                16-byte aligned).  NOT copied: as with hc_build, the index
 *                keeps the pointer and the caller keeps the rows alive and
 *                unchanged until hc_free.
 *   cuda_stream  the lists are uploaded on it; the call returns once they are
 *                on the device and checked.
 *   out          receives the index (free with hc_free).  It answers every
 *                query exactly as the index that was saved.
 * Nothing in the file is trusted.  Checked on the host before any device
 * work: the header (magic, version, byte order, parameters valid as for
 * hc_build), the list offsets against the layout hc_build makes for those
 * parameters, and the file size.  Checked while the lists stream in: each
 * list holds every row of its partition exactly once, high key words do not
 * decrease along a list, and the checksum agrees.  Checked last on the
 * device: the keys of up to 4096 entries per list, spread over the list and
 * recomputed from db_dev's rows, equal the stored keys.  Returns HC_ERR_ARG
 * for a null path or out, or a db_dev that is not 16-byte aligned device
 * memory (checked after the header); HC_ERR_IO when the file cannot be
 * opened or read; HC_ERR_FORMAT when any check fails; HC_ERR_OOM /
 * HC_ERR_CUDA.  On an error nothing is allocated and *out is NULL.
 */
HC_API int hc_load(const char* path, const void* db_dev, void* cuda_stream, hc_index** out);

/* ------------------------------------------------------------ testing */

/*
 * hc_check_status -- the bounds checks of the checked build.  The library
 * also builds as libhc_check.so (every translation unit compiled with
 * -DHC_CHECK): there, each checked device access first tests its index; an
 * index out of range is counted, the first one is recorded and the access
 * is skipped (a row id is replaced by row 0, a write is dropped), and every
 * stream-ordered library buffer is followed by a 256-byte guard whose bytes
 * are checked on the device before the buffer is freed and here for the
 * buffers still alive.  Checked sites (hc_check_report.site):
 *   1 key pass: a row's slot in its list      2 radix scatter: a destination
 *   3 run fix-up: the run lists               4 run fix-up: a place in a run
 *   5 long-run pass: an output place           6 lower_bound: a probed entry
 *   7 a window's end against its list          8 a window entry index
 *   9 a row id against the database rows     10 a query against the batch
 *  11 persistent launch: a query of a job     12 persistent launch: lists
 *  13 a guard byte overwritten (index = offset in the guard, bound 0)
 * No counterpart in the paper: it stands in for a memory checker.
 *   out    receives the report; violations counts every refused access (and
 *          overwritten guard byte) since the last reset, site / index / bound
 *          describe the first (index >= bound).  In the normal build
 *          enabled = 0 and the rest is zero.
 *   reset  nonzero: clear the device records after reading them.
 * Waits for the whole device first (checked build only).  HC_ERR_ARG if out
 * is NULL, HC_ERR_CUDA if a read fails.
 */
typedef struct {
    uint32_t enabled;      /* 1 in libhc_check.so, 0 in libhc.so */
    uint32_t site;         /* check site of the first violation, 0 = none */
    uint64_t violations;   /* refused accesses and overwritten guard bytes */
    uint64_t index;        /* the first violation's index ... */
    uint64_t bound;        /* ... and the bound it broke */
} hc_check_report;
HC_API int hc_check_status(hc_check_report* out, int reset);

/* hc_launch_count -- number of CUDA kernel launches the library has issued
 * since it was loaded (all entry points, all devices).  No counterpart in the
 * paper: it lets a caller count the kernels inside a timed region. */
HC_API uint64_t hc_launch_count(void);

/*
 * hc_debug_fail_alloc -- host-side fault injection (no counterpart in the
 * paper; it exists so that allocation-failure handling can be tested without
 * exhausting a GPU).  After this call, the library allocation numbered
 * `after` (0-based, counting device allocations made by any entry point)
 * fails as if the device were out of memory, and the entry point returns
 * HC_ERR_OOM after releasing what it had allocated.  after < 0 disables the
 * injection.  Not thread-safe with concurrent library calls.
 */
HC_API void hc_debug_fail_alloc(long after);

#ifdef __cplusplus
}
#endif

#endif /* HC_H */
