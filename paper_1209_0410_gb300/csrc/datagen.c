/*
 * Seeded synthetic inputs for the Hypercurves kNN path.
 *
 * This file holds no arithmetic of the indexing method itself: it only draws
 * the database and query vectors that both the CPU oracle and the CUDA path
 * consume.  The recipe stands in for the 128-d SIFT collection the paper
 * measures on (Sec. 7, experimental setup), which is not available here:
 *
 *   centres   : n_clusters x d values, uniform in [0, 255]          (stream 1)
 *   cluster   : per row, uniform in [0, n_clusters)                 (stream 2)
 *   row value : centre + N(0, sigma), rounded half-to-even, clipped (stream 3)
 *   query     : database row r (r uniform in [0, N), stream 1 of the query
 *               seed) + N(0, sigma_q) per dim, rounded, clipped     (stream 2)
 *
 * Random numbers come from a counter-based generator: the idx-th output of
 * the SplitMix64 sequence (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) whose state starts at a key
 * derived from (seed, stream).  Every value depends only on (seed, stream,
 * index), so the bytes are identical for any thread count.  Gaussians use the
 * Box-Muller transform in double precision on the host.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* key of the stream (seed, stream): a SplitMix64 output of its own */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return sm_mix(sm_mix(seed + GOLDEN) + stream * GOLDEN);
}

/* idx-th SplitMix64 output of the sequence whose state starts at key */
static inline uint64_t draw(uint64_t key, uint64_t idx) {
    return sm_mix(key + (idx + 1) * GOLDEN);
}

static inline double unit_open0(uint64_t u) { /* (0, 1] */
    return (double)((u >> 11) + 1) * 0x1.0p-53;
}
static inline double unit_open1(uint64_t u) { /* [0, 1) */
    return (double)(u >> 11) * 0x1.0p-53;
}

static inline uint8_t round_clip(double v) {
    v = nearbyint(v); /* default rounding mode: half to even */
    if (!(v > 0.0)) return 0;
    if (v > 255.0) return 255;
    return (uint8_t)v;
}

/* Gaussian numbers 2*pair and 2*pair+1 of a stream: Box-Muller on draws
 * 2*pair and 2*pair+1 (cosine branch first, sine branch second). */
static inline void gauss_pair(uint64_t key, uint64_t pair, double* z0, double* z1) {
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = unit_open0(draw(key, 2 * pair));
    double u2 = unit_open1(draw(key, 2 * pair + 1));
    double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(two_pi * u2);
    *z1 = r * sin(two_pi * u2);
}

static inline double gauss(uint64_t key, uint64_t e) {
    double z0, z1;
    gauss_pair(key, e >> 1, &z0, &z1);
    return (e & 1) ? z1 : z0;
}

/* row[t] = round_clip(base[t] + sigma * gauss(key, e0 + t)), t < d, pairing
 * the Box-Muller outputs whenever both members of a pair fall in the row. */
static void noisy_row(uint64_t key, uint64_t e0, uint64_t d, double sigma,
                      const double* base_f, const uint8_t* base_u, uint8_t* row) {
    uint64_t t = 0;
    while (t < d) {
        uint64_t e = e0 + t;
        double b0 = base_f ? base_f[t] : (double)base_u[t];
        if ((e & 1) == 0 && t + 1 < d) {
            double z0, z1;
            gauss_pair(key, e >> 1, &z0, &z1);
            double b1 = base_f ? base_f[t + 1] : (double)base_u[t + 1];
            row[t] = round_clip(b0 + sigma * z0);
            row[t + 1] = round_clip(b1 + sigma * z1);
            t += 2;
        } else {
            row[t] = round_clip(b0 + sigma * gauss(key, e));
            t += 1;
        }
    }
}

/* unbiased-enough bounded draw: high 64 bits of u * n */
static inline uint64_t bounded(uint64_t u, uint64_t n) {
    return (uint64_t)(((unsigned __int128)u * n) >> 64);
}

typedef struct {
    uint64_t seed, n, d, n_clusters;
    double sigma;
    const double* centres;
    uint8_t* out;
    uint64_t r0, r1;
} db_job;

static void* db_worker(void* arg) {
    db_job* j = (db_job*)arg;
    uint64_t k_cl = stream_key(j->seed, 2), k_noise = stream_key(j->seed, 3);
    for (uint64_t r = j->r0; r < j->r1; ++r) {
        uint64_t c = bounded(draw(k_cl, r), j->n_clusters);
        const double* ctr = j->centres + c * j->d;
        uint8_t* row = j->out + r * j->d;
        noisy_row(k_noise, r * j->d, j->d, j->sigma, ctr, NULL, row);
    }
    return NULL;
}

typedef struct {
    uint64_t seed, n_db, d;
    double sigma;
    const uint8_t* db;
    uint8_t* out;
    uint64_t* src_rows;
    uint64_t q0, q1;
} q_job;

static void* q_worker(void* arg) {
    q_job* j = (q_job*)arg;
    uint64_t k_src = stream_key(j->seed, 1), k_noise = stream_key(j->seed, 2);
    for (uint64_t q = j->q0; q < j->q1; ++q) {
        uint64_t r = bounded(draw(k_src, q), j->n_db);
        if (j->src_rows) j->src_rows[q] = r;
        const uint8_t* src = j->db + r * j->d;
        uint8_t* dst = j->out + q * j->d;
        noisy_row(k_noise, q * j->d, j->d, j->sigma, NULL, src, dst);
    }
    return NULL;
}

static int run_jobs(void* jobs, size_t job_size, int nthreads, void* (*fn)(void*)) {
    pthread_t th[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, fn, (char*)jobs + t * job_size) != 0) {
            for (int u = 0; u < t; ++u) pthread_join(th[u], NULL);
            return -1;
        }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* Database: n rows of d bytes, row-major, into out (n*d bytes). */
int hcgen_db_u8(uint64_t seed, uint64_t n, uint32_t d, uint32_t n_clusters, double sigma,
                uint8_t* out, int nthreads) {
    if (!out || d == 0 || n_clusters == 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    double* centres = (double*)malloc(sizeof(double) * n_clusters * d);
    if (!centres) return -2;
    uint64_t k_ctr = stream_key(seed, 1);
    for (uint64_t i = 0; i < (uint64_t)n_clusters * d; ++i)
        centres[i] = 255.0 * unit_open1(draw(k_ctr, i));
    db_job jobs[256];
    uint64_t per = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t r0 = per * t, r1 = r0 + per;
        if (r0 > n) r0 = n;
        if (r1 > n) r1 = n;
        db_job j = {seed, n, d, n_clusters, sigma, centres, out, r0, r1};
        jobs[t] = j;
    }
    int rc = run_jobs(jobs, sizeof(db_job), nthreads, db_worker);
    free(centres);
    return rc;
}

/* Queries: nq rows of d bytes; each is a database row plus Gaussian noise.
 * src_rows (nullable) receives the database row each query was drawn from. */
int hcgen_queries_u8(uint64_t seed, const uint8_t* db, uint64_t n_db, uint32_t d, uint64_t nq,
                     double sigma, uint8_t* out, uint64_t* src_rows, int nthreads) {
    if (!db || !out || n_db == 0 || d == 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    q_job jobs[256];
    uint64_t per = (nq + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t q0 = per * t, q1 = q0 + per;
        if (q0 > nq) q0 = nq;
        if (q1 > nq) q1 = nq;
        q_job j = {seed, n_db, d, sigma, db, out, src_rows, q0, q1};
        jobs[t] = j;
    }
    return run_jobs(jobs, sizeof(q_job), nthreads, q_worker);
}

/* Raw counter-based draws, exposed so tests can check the generator itself. */
void hcgen_draws(uint64_t seed, uint64_t stream, uint64_t idx0, uint64_t count, uint64_t* out) {
    uint64_t key = stream_key(seed, stream);
    for (uint64_t i = 0; i < count; ++i) out[i] = draw(key, idx0 + i);
}

void hcgen_gauss(uint64_t seed, uint64_t stream, uint64_t e0, uint64_t count, double* out) {
    uint64_t key = stream_key(seed, stream);
    for (uint64_t i = 0; i < count; ++i) out[i] = gauss(key, e0 + i);
}

/* The plain SplitMix64 sequence from a given state (its published definition),
 * so that tests can check the generator against known outputs. */
void hcgen_splitmix64_seq(uint64_t state, uint64_t count, uint64_t* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = draw(state, i);
}
