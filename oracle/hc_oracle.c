/*
 * CPU oracle for the Hypercurves / Multicurves kNN method
 * (Teodoro, Valle, Mariano, Torres, Meira, Saltz, "Approximate Similarity
 * Search for Online Multimedia Services on Distributed CPU-GPU Platforms",
 * arXiv:1209.0410).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference the CUDA
 * path is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library's product path never does.
 * It shares no source with the CUDA path.
 *
 * Everything is scalar C: plain loops, qsort for the sorted lists, exact
 * integer distances for uint8 data and double-precision sums for float32.
 *
 * Readings of the paper taken here (the paper is silent or loose on them):
 *  - Hilbert orientation: the curve is the one produced by Skilling's
 *    transpose formulation (J. Skilling, "Programming the Hilbert curve",
 *    AIP Conf. Proc. 707, 2004), an iterative Gray-code method of the family
 *    the paper cites for computing the extended-key (Sec. 2.2.1).  Key bits
 *    are emitted level by level from the top bit, axis 0 first.
 *  - Float32 key coordinates: (uint8) clamp(rint(x * 255f), 0, 255), computed
 *    in float32.  NaN and negatives map to 0.
 *  - Ties between equal keys in a sorted list: ascending id.
 *  - Which entries Algorithm 2 takes around the query key: with pos = first list entry
 *    whose key is >= the query key, the window is [max(0,pos-p), min(n,pos+p))
 *    -- p entries below and p at-or-above, clipped at the list ends without
 *    shifting (the half-list picture of Sec. 4.2).  The paper's "depth" = 2p.
 *  - Result order: ascending (distance, id); fewer than k candidates are
 *    padded with id -1 and distance +inf.
 *  - Partitioned (Hypercurves) search: each of the l partitions answers its
 *    local kNN over its own subindexes with its own depth, and the local
 *    answers are reduced to the global k (Sec. 4.1).
 *  - Equivalence bound (Sec. 4.2, Eq. 6): the union-bound multiplier is
 *    printed as Phi; orc_equiv_bound takes the multiplier as an argument.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_U8 = 0, ORC_F32 = 1 };

/* ------------------------------------------------------------------------ */
/* Hilbert extended-key C^-1 (Sec. 2.2.1): n coordinates of b bits -> one    */
/* key of n*b bits (bijective at finite order).                              */
/* ------------------------------------------------------------------------ */

/* Append one bit to a 128-bit big integer held as (hi, lo). */
static void push_bit(uint64_t* hi, uint64_t* lo, unsigned bit) {
    *hi = (*hi << 1) | (*lo >> 63);
    *lo = (*lo << 1) | (uint64_t)(bit & 1u);
}

/* Bit number pos (0 = least significant) of the 128-bit integer (hi, lo). */
static unsigned get_bit(uint64_t hi, uint64_t lo, unsigned pos) {
    return pos >= 64 ? (unsigned)((hi >> (pos - 64)) & 1u) : (unsigned)((lo >> pos) & 1u);
}

/*
 * Forward map: axes x[0..n-1] (each < 2^b) -> key.  Steps:
 *  1. for every bit level from the top one down to bit 1, visit the axes in
 *     order; when the axis has that bit set, the lower bits of axis 0 are
 *     inverted, otherwise the lower bits of axis 0 and of the axis swap;
 *  2. Gray-encode across the axes (each axis xor-ed with the one before);
 *  3. a correction mask taken from the last axis is xor-ed into every axis;
 *  4. the key reads bit level b-1 of axes 0..n-1, then level b-2, ... 0.
 * Returns 0, or -1 when the shape is not supported (n*b > 128).
 */
int orc_hilbert_key(int n, int b, const uint32_t* x, uint64_t* key_hi, uint64_t* key_lo) {
    if (n < 1 || n > 32 || b < 1 || b > 32 || n * b > 128) return -1;
    uint32_t X[32];
    for (int i = 0; i < n; ++i) X[i] = x[i];

    for (int q = b - 1; q >= 1; --q) {
        uint32_t bitq = 1u << q, low = bitq - 1u;
        for (int i = 0; i < n; ++i) {
            if (X[i] & bitq) {
                X[0] ^= low;
            } else {
                uint32_t t = (X[0] ^ X[i]) & low;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < n; ++i) X[i] ^= X[i - 1];
    uint32_t corr = 0;
    for (int q = b - 1; q >= 1; --q)
        if (X[n - 1] & (1u << q)) corr ^= (1u << q) - 1u;
    for (int i = 0; i < n; ++i) X[i] ^= corr;

    uint64_t hi = 0, lo = 0;
    for (int q = b - 1; q >= 0; --q)
        for (int i = 0; i < n; ++i) push_bit(&hi, &lo, (X[i] >> q) & 1u);
    *key_hi = hi;
    *key_lo = lo;
    return 0;
}

/*
 * Inverse map: key -> axes.  Undoes the forward steps in reverse order:
 * de-interleave the key bits, undo the Gray code and its correction, then
 * replay the exchange/invert steps from the lowest level upward with the
 * axes in reverse order.
 */
int orc_hilbert_axes(int n, int b, uint64_t key_hi, uint64_t key_lo, uint32_t* x) {
    if (n < 1 || n > 32 || b < 1 || b > 32 || n * b > 128) return -1;
    uint32_t X[32];
    for (int i = 0; i < n; ++i) X[i] = 0;
    unsigned pos = (unsigned)(n * b);
    for (int q = b - 1; q >= 0; --q)
        for (int i = 0; i < n; ++i) {
            --pos;
            X[i] |= get_bit(key_hi, key_lo, pos) << q;
        }

    uint32_t t = X[n - 1] >> 1;
    for (int i = n - 1; i >= 1; --i) X[i] ^= X[i - 1];
    X[0] ^= t;

    for (int q = 1; q <= b - 1; ++q) {
        uint32_t bitq = 1u << q, low = bitq - 1u;
        for (int i = n - 1; i >= 0; --i) {
            if (X[i] & bitq) {
                X[0] ^= low;
            } else {
                uint32_t s = (X[0] ^ X[i]) & low;
                X[0] ^= s;
                X[i] ^= s;
            }
        }
    }
    for (int i = 0; i < n; ++i) x[i] = X[i];
    return 0;
}

int orc_hilbert_keys_batch(int n, int b, uint64_t count, const uint32_t* axes, uint64_t* hi,
                           uint64_t* lo) {
    for (uint64_t r = 0; r < count; ++r)
        if (orc_hilbert_key(n, b, axes + r * (uint64_t)n, hi + r, lo + r) != 0) return -1;
    return 0;
}

int orc_hilbert_axes_batch(int n, int b, uint64_t count, const uint64_t* hi, const uint64_t* lo,
                           uint32_t* axes) {
    for (uint64_t r = 0; r < count; ++r)
        if (orc_hilbert_axes(n, b, hi[r], lo[r], axes + r * (uint64_t)n) != 0) return -1;
    return 0;
}

/* Float32 coordinate -> 8-bit key coordinate, decided in float32. */
uint32_t orc_quantize(float x) {
    float s = x * 255.0f;
    if (!(s > 0.0f)) return 0;
    if (s >= 255.0f) return 255;
    return (uint32_t)nearbyintf(s);
}

/* ------------------------------------------------------------------------ */
/* Shared shape description                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int dtype;                 /* ORC_U8 or ORC_F32 */
    uint64_t n;                /* database rows */
    uint32_t d;                /* dimensions */
    uint32_t curves;           /* subindexes per partition */
    uint32_t m;                /* dims per curve (dims[c] in Alg. 1, all equal) */
    const uint32_t* dim_map;   /* a[c][j] as curves*m entries; NULL = c*m + j */
    uint32_t ell;              /* partitions (1 = sequential Multicurves) */
} orc_shape;

static uint32_t attr(const orc_shape* s, uint32_t c, uint32_t j) {
    return s->dim_map ? s->dim_map[c * s->m + j] : c * s->m + j;
}

/* projection proj[j] <- v[a[c,j]] onto the curve's subspace, then key <- C^-1(proj)
 * (Algorithm 1, per-curve step) */
static void vector_key(const orc_shape* s, const void* v, uint32_t c, uint64_t* hi, uint64_t* lo) {
    uint32_t proj[32];
    for (uint32_t j = 0; j < s->m; ++j) {
        uint32_t dim = attr(s, c, j);
        if (s->dtype == ORC_U8)
            proj[j] = ((const uint8_t*)v)[dim];
        else
            proj[j] = orc_quantize(((const float*)v)[dim]);
    }
    orc_hilbert_key((int)s->m, 8, proj, hi, lo);
}

static const void* row_ptr(const orc_shape* s, const void* base, uint64_t r) {
    size_t es = s->dtype == ORC_U8 ? 1 : 4;
    return (const char*)base + r * (uint64_t)s->d * es;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: index construction                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t hi, lo;
    uint32_t id;
} entry;

static int entry_cmp(const void* a, const void* b) {
    const entry* x = (const entry*)a;
    const entry* y = (const entry*)b;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* Partition of row r: given by part_of, else contiguous id ranges
 * [floor(j*n/ell), floor((j+1)*n/ell)). */
static uint32_t part_of_row(const orc_shape* s, const uint32_t* part_of, uint64_t r) {
    if (part_of) return part_of[r];
    /* largest j with floor(j*n/ell) <= r */
    uint32_t j = (uint32_t)(((unsigned __int128)r * s->ell) / s->n);
    while (j + 1 < s->ell && (uint64_t)(((unsigned __int128)(j + 1) * s->n) / s->ell) <= r) ++j;
    while (j > 0 && (uint64_t)(((unsigned __int128)j * s->n) / s->ell) > r) --j;
    return j;
}

typedef struct {
    const orc_shape* s;
    const void* db;
    const uint32_t* part_of;
    const uint64_t* list_off;
    uint64_t* keys_hi;
    uint64_t* keys_lo;
    uint32_t* ids;
    uint32_t list0, list1;
    int status;
} build_job;

static void* build_worker(void* arg) {
    build_job* j = (build_job*)arg;
    const orc_shape* s = j->s;
    for (uint32_t L = j->list0; L < j->list1; ++L) {
        uint32_t part = L / s->curves, c = L % s->curves;
        uint64_t len = j->list_off[L + 1] - j->list_off[L];
        entry* e = (entry*)malloc(sizeof(entry) * (len ? len : 1));
        if (!e) { j->status = -2; return NULL; }
        uint64_t t = 0;
        /* every b of this partition: insert <key, b> into the list (Algorithm 1) */
        for (uint64_t r = 0; r < s->n; ++r) {
            if (part_of_row(s, j->part_of, r) != part) continue;
            vector_key(s, row_ptr(s, j->db, r), c, &e[t].hi, &e[t].lo);
            e[t].id = (uint32_t)r;
            ++t;
        }
        qsort(e, t, sizeof(entry), entry_cmp);
        uint64_t o = j->list_off[L];
        for (uint64_t i = 0; i < t; ++i) {
            j->keys_hi[o + i] = e[i].hi;
            j->keys_lo[o + i] = e[i].lo;
            j->ids[o + i] = e[i].id;
        }
        free(e);
    }
    return NULL;
}

/*
 * Build ell*curves sorted lists.  List L = part*curves + c occupies
 * [list_off[L], list_off[L+1]) of keys_hi/keys_lo/ids.  list_off has
 * ell*curves+1 entries and is written here.
 */
int orc_build(int dtype, const void* db, uint64_t n, uint32_t d, uint32_t curves, uint32_t m,
              const uint32_t* dim_map, uint32_t ell, const uint32_t* part_of, uint64_t* list_off,
              uint64_t* keys_hi, uint64_t* keys_lo, uint32_t* ids, int nthreads) {
    if (m < 1 || m > 16 || curves < 1 || ell < 1 || d < 1 || n < 1 || n > 0xFFFFFFFFull) return -1;
    orc_shape s = {dtype, n, d, curves, m, dim_map, ell};
    for (uint32_t c = 0; c < curves; ++c)
        for (uint32_t j = 0; j < m; ++j)
            if (attr(&s, c, j) >= d) return -1;
    uint64_t* count = (uint64_t*)calloc(ell, sizeof(uint64_t));
    if (!count) return -2;
    for (uint64_t r = 0; r < n; ++r) {
        uint32_t pj = part_of_row(&s, part_of, r);
        if (pj >= ell) { free(count); return -1; }
        count[pj]++;
    }
    uint32_t lists = ell * curves;
    list_off[0] = 0;
    for (uint32_t L = 0; L < lists; ++L) list_off[L + 1] = list_off[L] + count[L / curves];
    free(count);

    if (nthreads < 1) nthreads = 1;
    if ((uint32_t)nthreads > lists) nthreads = (int)lists;
    if (nthreads > 256) nthreads = 256;
    build_job jobs[256];
    pthread_t th[256];
    uint32_t per = (lists + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        uint32_t a = per * t, b = a + per;
        if (a > lists) a = lists;
        if (b > lists) b = lists;
        build_job j = {&s, db, part_of, list_off, keys_hi, keys_lo, ids, a, b, 0};
        jobs[t] = j;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, build_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status) return jobs[t].status;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Distances (Eq. 2, squared) and ranking                                    */
/* ------------------------------------------------------------------------ */

static double sq_dist(const orc_shape* s, const void* q, const void* b) {
    if (s->dtype == ORC_U8) {
        const uint8_t* x = (const uint8_t*)q;
        const uint8_t* y = (const uint8_t*)b;
        int64_t acc = 0;
        for (uint32_t t = 0; t < s->d; ++t) {
            int64_t diff = (int64_t)x[t] - (int64_t)y[t];
            acc += diff * diff;
        }
        return (double)acc;
    } else {
        const float* x = (const float*)q;
        const float* y = (const float*)b;
        double acc = 0.0;
        for (uint32_t t = 0; t < s->d; ++t) {
            double diff = (double)x[t] - (double)y[t];
            acc += diff * diff;
        }
        return acc;
    }
}

typedef struct {
    double dist;
    int64_t id;
} scored;

static int scored_cmp(const void* a, const void* b) {
    const scored* x = (const scored*)a;
    const scored* y = (const scored*)b;
    if (x->dist != y->dist) return x->dist < y->dist ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static int u32_cmp(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* first i in [0, len) with (hi[i], lo[i]) >= (qh, ql), else len */
static uint64_t lower_bound128(const uint64_t* hi, const uint64_t* lo, uint64_t len, uint64_t qh,
                               uint64_t ql) {
    uint64_t first = 0, count = len;
    while (count > 0) {
        uint64_t step = count / 2, mid = first + step;
        int less = hi[mid] < qh || (hi[mid] == qh && lo[mid] < ql);
        if (less) {
            first = mid + 1;
            count -= step + 1;
        } else {
            count = step;
        }
    }
    return first;
}

/* write the k smallest of cand[0..nc) by (dist, id), padded */
static void take_k(scored* cand, uint64_t nc, uint32_t k, int32_t* out_ids, double* out_dist) {
    qsort(cand, nc, sizeof(scored), scored_cmp);
    for (uint32_t i = 0; i < k; ++i) {
        if (i < nc) {
            out_ids[i] = (int32_t)cand[i].id;
            out_dist[i] = cand[i].dist;
        } else {
            out_ids[i] = -1;
            out_dist[i] = INFINITY;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: search (and its partitioned form, Sec. 4.1)                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_shape* s;
    const void* db;
    const uint64_t* list_off;
    const uint64_t* keys_hi;
    const uint64_t* keys_lo;
    const uint32_t* ids;
    const void* queries;
    uint32_t k, p;
    int32_t* out_ids;
    double* out_dist;
    int64_t* out_pos;          /* nullable: nq x lists lower_bound positions */
    uint64_t q0, q1;
    int status;
} search_job;

static void* search_worker(void* arg) {
    search_job* J = (search_job*)arg;
    const orc_shape* s = J->s;
    uint32_t lists = s->ell * s->curves;
    uint64_t max_cand = (uint64_t)s->curves * 2u * J->p;
    uint32_t* cand_ids = (uint32_t*)malloc(sizeof(uint32_t) * (max_cand ? max_cand : 1));
    scored* cand = (scored*)malloc(sizeof(scored) * (max_cand ? max_cand : 1));
    scored* local = (scored*)malloc(sizeof(scored) * ((uint64_t)s->ell * J->k + 1));
    int32_t* lid = (int32_t*)malloc(sizeof(int32_t) * (J->k + 1));
    double* ldist = (double*)malloc(sizeof(double) * (J->k + 1));
    if (!cand_ids || !cand || !local || !lid || !ldist) {
        J->status = -2;
        goto done;
    }
    for (uint64_t qi = J->q0; qi < J->q1; ++qi) {
        const void* q = row_ptr(s, J->queries, qi);
        uint64_t nlocal = 0;
        for (uint32_t part = 0; part < s->ell; ++part) {
            /* candidates <- union over curves of the window around key */
            uint64_t nc = 0;
            for (uint32_t c = 0; c < s->curves; ++c) {
                uint32_t L = part * s->curves + c;
                uint64_t off = J->list_off[L], len = J->list_off[L + 1] - off;
                uint64_t kh, kl;
                vector_key(s, q, c, &kh, &kl);
                uint64_t pos = lower_bound128(J->keys_hi + off, J->keys_lo + off, len, kh, kl);
                if (J->out_pos) J->out_pos[qi * lists + L] = (int64_t)pos;
                uint64_t lo = pos > J->p ? pos - J->p : 0;
                uint64_t hi = pos + J->p < len ? pos + J->p : len;
                for (uint64_t i = lo; i < hi; ++i) cand_ids[nc++] = J->ids[off + i];
            }
            qsort(cand_ids, nc, sizeof(uint32_t), u32_cmp);
            uint64_t nu = 0;
            for (uint64_t i = 0; i < nc; ++i)
                if (i == 0 || cand_ids[i] != cand_ids[i - 1]) cand_ids[nu++] = cand_ids[i];
            /* knn <- the k candidates closest to q (Algorithm 2, final step) */
            for (uint64_t i = 0; i < nu; ++i) {
                cand[i].id = cand_ids[i];
                cand[i].dist = sq_dist(s, q, row_ptr(s, J->db, cand_ids[i]));
            }
            take_k(cand, nu, J->k, lid, ldist);
            for (uint32_t i = 0; i < J->k; ++i)
                if (lid[i] >= 0) {
                    local[nlocal].id = lid[i];
                    local[nlocal].dist = ldist[i];
                    ++nlocal;
                }
        }
        /* Aggregator: reduce the local answers to the global k (Sec. 4.1);
         * an id can only occur in one partition, the dedupe is defensive */
        qsort(local, nlocal, sizeof(scored), scored_cmp);
        uint64_t nu = 0;
        for (uint64_t i = 0; i < nlocal; ++i)
            if (nu == 0 || local[i].id != local[nu - 1].id) local[nu++] = local[i];
        take_k(local, nu, J->k, J->out_ids + qi * J->k, J->out_dist + qi * J->k);
    }
done:
    free(cand_ids);
    free(cand);
    free(local);
    free(lid);
    free(ldist);
    return NULL;
}

static int run_search_jobs(search_job* proto, uint64_t nq, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > nq) nthreads = nq ? (int)nq : 1;
    search_job jobs[256];
    pthread_t th[256];
    uint64_t per = (nq + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].q0 = per * t < nq ? per * t : nq;
        jobs[t].q1 = per * (t + 1) < nq ? per * (t + 1) : nq;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, search_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status) return jobs[t].status;
    return 0;
}

/*
 * Search nq queries at depth p on each side (per list).  With ell > 1 each
 * partition answers locally and the answers are reduced (Hypercurves);
 * with ell == 1 this is Alg. 2 as printed.  out_pos (nullable) receives the
 * lower_bound position of every query in every list.
 */
int orc_search(int dtype, const void* db, uint64_t n, uint32_t d, uint32_t curves, uint32_t m,
               const uint32_t* dim_map, uint32_t ell, const uint64_t* list_off,
               const uint64_t* keys_hi, const uint64_t* keys_lo, const uint32_t* ids,
               const void* queries, uint64_t nq, uint32_t k, uint32_t p, int32_t* out_ids,
               double* out_dist, int64_t* out_pos, int nthreads) {
    if (k < 1 || m < 1 || m > 16) return -1;
    orc_shape s = {dtype, n, d, curves, m, dim_map, ell};
    search_job proto = {&s, db, list_off, keys_hi, keys_lo, ids, queries, k, p,
                        out_ids, out_dist, out_pos, 0, 0, 0};
    return run_search_jobs(&proto, nq, nthreads);
}

/* Query extended-keys for every (query, curve): hi/lo are nq x curves. */
int orc_query_keys(int dtype, const void* queries, uint64_t nq, uint32_t d, uint32_t curves,
                   uint32_t m, const uint32_t* dim_map, uint64_t* hi, uint64_t* lo) {
    if (m < 1 || m > 16) return -1;
    orc_shape s = {dtype, 0, d, curves, m, dim_map, 1};
    for (uint64_t qi = 0; qi < nq; ++qi)
        for (uint32_t c = 0; c < curves; ++c)
            vector_key(&s, row_ptr(&s, queries, qi), c, hi + qi * curves + c, lo + qi * curves + c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact kNN (Eq. 3) by brute force                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_shape* s;
    const void* db;
    const void* queries;
    uint32_t k;
    int32_t* out_ids;
    double* out_dist;
    uint64_t q0, q1;
    int status;
} brute_job;

static void* brute_worker(void* arg) {
    brute_job* J = (brute_job*)arg;
    const orc_shape* s = J->s;
    scored* all = (scored*)malloc(sizeof(scored) * s->n);
    if (!all) { J->status = -2; return NULL; }
    for (uint64_t qi = J->q0; qi < J->q1; ++qi) {
        const void* q = row_ptr(s, J->queries, qi);
        for (uint64_t r = 0; r < s->n; ++r) {
            all[r].id = (int64_t)r;
            all[r].dist = sq_dist(s, q, row_ptr(s, J->db, r));
        }
        take_k(all, s->n, J->k, J->out_ids + qi * J->k, J->out_dist + qi * J->k);
    }
    free(all);
    return NULL;
}

int orc_bruteforce(int dtype, const void* db, uint64_t n, uint32_t d, const void* queries,
                   uint64_t nq, uint32_t k, int32_t* out_ids, double* out_dist, int nthreads) {
    if (k < 1 || n < 1) return -1;
    orc_shape s = {dtype, n, d, 1, 1, NULL, 1};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > nq) nthreads = nq ? (int)nq : 1;
    brute_job jobs[256];
    pthread_t th[256];
    uint64_t per = (nq + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        brute_job j = {&s, db, queries, k, out_ids, out_dist,
                       per * t < nq ? per * t : nq, per * (t + 1) < nq ? per * (t + 1) : nq, 0};
        jobs[t] = j;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, brute_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status) return jobs[t].status;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Probabilistic equivalence Multicurves <-> Hypercurves (Sec. 4.2)          */
/* ------------------------------------------------------------------------ */

/* P(Bin(Phi, 1/ell) > phi), the tail summed term by term in long double. */
double orc_binom_tail(uint32_t Phi, uint32_t ell, uint32_t phi) {
    long double pr = 1.0L / (long double)ell, qr = 1.0L - pr, sum = 0.0L;
    for (uint32_t j = phi + 1; j <= Phi; ++j) {
        long double lc = lgammal((long double)Phi + 1) - lgammal((long double)j + 1) -
                         lgammal((long double)(Phi - j) + 1);
        long double lt = lc + (long double)j * logl(pr);
        if (Phi - j > 0) lt += (long double)(Phi - j) * logl(qr);
        sum += expl(lt);
    }
    return (double)sum;
}

/*
 * Upper bound on the probability that some half-list of some partition holds
 * more than phi of the 2*Phi window entries (Sec. 4.2, Eq. 6):
 *   1 - max(0, 1 - mult * P(Bin(Phi, 1/ell) > phi))^2,
 * mult being the union-bound multiplier (printed as Phi).
 */
double orc_equiv_bound(uint32_t Phi, uint32_t ell, uint32_t phi, double mult) {
    long double tail = (long double)orc_binom_tail(Phi, ell, phi);
    long double inner = 1.0L - (long double)mult * tail;
    if (inner < 0.0L) inner = 0.0L;
    return (double)(1.0L - inner * inner);
}

/* phi = ceil((1 + slack) * ceil(Phi / ell)) (Sec. 4.2) */
uint32_t orc_slack_depth(uint32_t Phi, uint32_t ell, double slack) {
    uint32_t base = (Phi + ell - 1) / ell;
    long double v = (1.0L + (long double)slack) * (long double)base;
    uint32_t r = (uint32_t)ceill(v - 1e-12L);
    return r;
}

int orc_quantize_batch(const float* x, uint64_t count, uint32_t* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = orc_quantize(x[i]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-query features for the learned probe depth (not in the paper: the    */
/* depth the paper fixes per subindex is predicted per query instead).      */
/* ------------------------------------------------------------------------ */

/* Octave encoding of a non-negative integer g (up to 128 bits): 0 for g = 0,
 * else 1 + e + f/65536 with e the index of the top set bit and f the 16 bits
 * below it (zero-filled).  Exact in float32 for every g < 2^128. */
static double octave128(uint64_t hi, uint64_t lo) {
    if (hi == 0 && lo == 0) return 0.0;
    int e;
    if (hi) {
        e = 127;
        while (!((hi >> (e - 64)) & 1ull)) --e;
    } else {
        e = 63;
        while (!((lo >> e) & 1ull)) --e;
    }
    /* the 16 bits below bit e */
    uint64_t f = 0;
    for (int b = 1; b <= 16; ++b) {
        int pos = e - b;
        unsigned bit = 0;
        if (pos >= 0) bit = pos >= 64 ? (unsigned)((hi >> (pos - 64)) & 1ull)
                                      : (unsigned)((lo >> pos) & 1ull);
        f = (f << 1) | bit;
    }
    return 1.0 + (double)e + (double)f / 65536.0;
}

/* (a - b) as 128-bit, a >= b */
static void sub128(uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, uint64_t* rh,
                   uint64_t* rl) {
    *rl = al - bl;
    *rh = ah - bh - (al < bl ? 1u : 0u);
}

#define ORC_FEAT_NONE 130.0

/*
 * Features of nq uint8 queries on the first `curves` lists (partition 0):
 * per curve c, with pos = lower_bound of the query key in list c:
 *   [c*4+0] octave(query key - key[pos-1])          (NONE when pos = 0)
 *   [c*4+1] octave(key[pos] - query key)            (NONE when pos = n)
 *   [c*4+2] octave(min distance over entries [pos-4, pos+4) clipped)
 *   [c*4+3] octave(floor(sum / count) of the same distances)  (NONE if empty)
 * feat is nq x (4 * curves) float.
 */
int orc_features(const void* db, uint64_t n, uint32_t d, uint32_t curves, uint32_t m,
                 const uint32_t* dim_map, const uint64_t* list_off, const uint64_t* keys_hi,
                 const uint64_t* keys_lo, const uint32_t* ids, const void* queries, uint64_t nq,
                 float* feat) {
    orc_shape s = {ORC_U8, n, d, curves, m, dim_map, 1};
    for (uint64_t qi = 0; qi < nq; ++qi) {
        const void* q = row_ptr(&s, queries, qi);
        for (uint32_t c = 0; c < curves; ++c) {
            uint64_t off = list_off[c], len = list_off[c + 1] - off;
            uint64_t kh, kl;
            vector_key(&s, q, c, &kh, &kl);
            uint64_t pos = lower_bound128(keys_hi + off, keys_lo + off, len, kh, kl);
            double f0 = ORC_FEAT_NONE, f1 = ORC_FEAT_NONE, f2 = ORC_FEAT_NONE,
                   f3 = ORC_FEAT_NONE;
            uint64_t gh, gl;
            if (pos > 0) {
                sub128(kh, kl, keys_hi[off + pos - 1], keys_lo[off + pos - 1], &gh, &gl);
                f0 = octave128(gh, gl);
            }
            if (pos < len) {
                sub128(keys_hi[off + pos], keys_lo[off + pos], kh, kl, &gh, &gl);
                f1 = octave128(gh, gl);
            }
            uint64_t lo = pos > 4 ? pos - 4 : 0, hi = pos + 4 < len ? pos + 4 : len;
            if (hi > lo) {
                int64_t mn = -1;
                uint64_t sum = 0;
                for (uint64_t i = lo; i < hi; ++i) {
                    int64_t dd = (int64_t)sq_dist(&s, q, row_ptr(&s, db, ids[off + i]));
                    if (mn < 0 || dd < mn) mn = dd;
                    sum += (uint64_t)dd;
                }
                f2 = octave128(0, (uint64_t)mn);
                f3 = octave128(0, sum / (hi - lo));
            }
            float* fo = feat + qi * 4 * curves + 4 * c;
            fo[0] = (float)f0;
            fo[1] = (float)f1;
            fo[2] = (float)f2;
            fo[3] = (float)f3;
        }
    }
    return 0;
}

double orc_octave(uint64_t hi, uint64_t lo) { return octave128(hi, lo); }
