/* gz_cpu_batched.c -- the paper's own CPU ingestion design, as a timed
 * baseline.  MEASUREMENT INFRASTRUCTURE ONLY: it is timed beside the oracle by
 * bench.py and checked against the oracle by tests; the CUDA library never
 * uses it.
 *
 * Section 5.1 buffers the updates of each node (the leaf gutters) and lets
 * Graph Worker threads apply a node's whole buffer to that node's sketch, one
 * worker per node at a time, so the sketches need no locks.  Here the stream
 * is cut into chunks; each chunk is bucketed by endpoint (per-thread
 * histograms, a prefix sum, a scatter of the edge index into the buffer of
 * each endpoint) and the node buffers are then applied in parallel, a node per
 * OpenMP iteration, with the update rule of Fig. cube_code (nested rows, the
 * form the paper's system stores).  The hashes follow the oracle's definition
 * (the same keys and pieces), computed the way a tuned CPU system would:
 * the edge is decoded once per record, and the depth reads only the pieces
 * it needs.
 *
 * Only nodes in [node_lo, node_hi) are sketched (alpha/gamma hold exactly
 * those nodes' sketches, in the oracle's nested layout), so a bounded node
 * range can stand in for the whole graph when host memory is short. */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GZB_COLS 7

int gzo_geometry(uint32_t V, uint32_t *K, uint32_t *R);
void gzo_keys(uint64_t seed, uint32_t K, uint32_t *keys);
void gzo_pieces(uint32_t V, uint32_t *p, uint32_t *m1, uint32_t *m2);
#define GZB_KEYS 256 /* key words per column: h1 pieces at [0, 128), h2 at [128, 256) */

typedef struct {
    uint32_t V, K, R, p, m1, m2;
    const uint32_t *keys;
} gzb_geo;

/* the top p bits of piece i with keys k on (u, v) */
static inline uint32_t piece(const uint32_t *k, uint32_t i, uint32_t p, uint32_t u, uint32_t v)
{
    return (k[3 * i] * u + k[3 * i + 1] * v + k[3 * i + 2]) >> (32 - p);
}

/* Fig. cube_code update_sketch for every CubeSketch of one node sketch */
static void node_apply(const gzb_geo *g, uint64_t *alpha, uint32_t *gamma, uint64_t idx)
{
    const uint32_t u = (uint32_t)(idx / g->V), v = (uint32_t)(idx % g->V), p = g->p, R = g->R;
    for (uint32_t col = 0; col < g->K * GZB_COLS; col++) {
        const uint32_t *k1 = g->keys + (size_t)col * GZB_KEYS, *k2 = k1 + 128;
        /* depth: leading zeros of the h1 pieces, capped at R-1 */
        uint32_t d = 0;
        for (uint32_t i = 0; i < g->m1 && d < R - 1; i++) {
            uint32_t t = piece(k1, i, p, u, v);
            if (t) {
                d += (uint32_t)__builtin_clz(t) - (32 - p);
                break;
            }
            d += p;
        }
        if (d > R - 1) d = R - 1;
        /* checksum: the first 32 bits of the h2 pieces */
        uint64_t acc = 0;
        for (uint32_t i = 0; i < g->m2; i++) acc |= (uint64_t)piece(k2, i, p, u, v) << (64 - p * (i + 1));
        const uint32_t gsum = (uint32_t)(acc >> 32);
        uint64_t *A = alpha + (size_t)col * R;
        uint32_t *G = gamma + (size_t)col * R;
        for (uint32_t row = 0; row <= d; row++) {
            A[row] ^= idx;
            G[row] ^= gsum;
        }
    }
}

/* Returns 0, -1 on an invalid update (nothing changed), -2 on allocation
 * failure.  threads <= 0 uses every core OpenMP offers. */
int gzb_ingest_batched(uint32_t V, uint64_t seed, size_t n, const uint32_t *u, const uint32_t *v,
                       uint32_t node_lo, uint32_t node_hi, uint64_t *alpha, uint32_t *gamma,
                       int threads, size_t chunk)
{
    uint32_t K, R;
    if (gzo_geometry(V, &K, &R) || node_lo >= node_hi || node_hi > V || chunk == 0) return -1;
    for (size_t i = 0; i < n; i++)
        if (u[i] == v[i] || u[i] >= V || v[i] >= V) return -1;
    if (threads <= 0) threads = omp_get_max_threads();
    const size_t ncol = (size_t)K * GZB_COLS, nb = ncol * R, span = node_hi - node_lo;
    uint32_t *keys = malloc(ncol * GZB_KEYS * 4);
    gzb_geo geo = {V, K, R, 0, 0, 0, keys};
    gzo_pieces(V, &geo.p, &geo.m1, &geo.m2);
    uint32_t *hist = calloc((size_t)threads * span, 4);
    uint32_t *off = malloc((span + 1) * 4);
    uint64_t *rec = malloc(2 * chunk * 8);
    int rc = 0;
    if (!keys || !hist || !off || !rec) {
        rc = -2;
        goto out;
    }
    gzo_keys(seed, K, keys);
    for (size_t base = 0; base < n; base += chunk) {
        const size_t m = n - base < chunk ? n - base : chunk;
        const uint32_t *cu = u + base, *cv = v + base;
        memset(hist, 0, (size_t)threads * span * 4);
        /* per-thread histograms of both endpoints over equal slices */
#pragma omp parallel num_threads(threads)
        {
            const int t = omp_get_thread_num(), nt = omp_get_num_threads();
            uint32_t *hh = hist + (size_t)t * span;
            const size_t lo = m * t / nt, hi = m * (t + 1) / nt;
            for (size_t i = lo; i < hi; i++) {
                if (cu[i] >= node_lo && cu[i] < node_hi) hh[cu[i] - node_lo]++;
                if (cv[i] >= node_lo && cv[i] < node_hi) hh[cv[i] - node_lo]++;
            }
        }
        /* node-major prefix: off[x] = start of node x's buffer; hist becomes
         * each thread's write cursor inside it */
        uint32_t run = 0;
        for (size_t x = 0; x < span; x++) {
            off[x] = run;
            for (int t = 0; t < threads; t++) {
                uint32_t cnt = hist[(size_t)t * span + x];
                hist[(size_t)t * span + x] = run;
                run += cnt;
            }
        }
        off[span] = run;
#pragma omp parallel num_threads(threads)
        {
            const int t = omp_get_thread_num(), nt = omp_get_num_threads();
            uint32_t *hh = hist + (size_t)t * span;
            const size_t lo = m * t / nt, hi = m * (t + 1) / nt;
            for (size_t i = lo; i < hi; i++) {
                const uint32_t a = cu[i] < cv[i] ? cu[i] : cv[i];
                const uint32_t b = cu[i] < cv[i] ? cv[i] : cu[i];
                const uint64_t idx = (uint64_t)a * V + b;
                if (a >= node_lo && a < node_hi) rec[hh[a - node_lo]++] = idx;
                if (b >= node_lo && b < node_hi) rec[hh[b - node_lo]++] = idx;
            }
        }
        /* Graph Workers: one node buffer per iteration */
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads)
        for (size_t x = 0; x < span; x++) {
            uint64_t *A = alpha + x * nb;
            uint32_t *G = gamma + x * nb;
            for (uint32_t r = off[x]; r < off[x + 1]; r++) node_apply(&geo, A, G, rec[r]);
        }
    }
out:
    free(keys);
    free(hist);
    free(off);
    free(rec);
    return rc;
}

int gzb_max_threads(void) { return omp_get_max_threads(); }
