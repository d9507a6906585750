/*
 * gz_gen.h -- device generator of the seeded Kronecker insert/delete streams
 * used as benchmark input (inputs only: no sketch arithmetic).
 *
 * The paper turns Graph500 Kronecker graphs into insert/delete streams
 * (Section 6.1, "Synthesizing Dense Graphs and Streams": (i) every insert
 * precedes its delete, (ii) an edge never gets two consecutive updates of one
 * type, (iii) fewer than 150 nodes are cut off, (iv) the final graph is the
 * input graph).  This generator produces, chunk by chunk on the device,
 * exactly the stream that paper_2203_14927_b300/streams.py (KronSpec.chunk)
 * produces on the host from the same parameters:
 *   - position p in [0, V^2) maps to an ordered pair (u, v) by a 4-round
 *     Feistel permutation on the two L-bit halves (round function
 *     mix64(right ^ k_feistel[i]) & (V-1)), V = 2^L; only u < v is used;
 *   - (u,v) is a final edge iff mix64(idx ^ k_kron) >> 11 < table[n00][n11]
 *     (idx = u*V+v, n11 = popcount(u&v), n00 = L - popcount(u|v)) and neither
 *     endpoint is cut off (mix64(x ^ k_iso) >> 11 < t_iso);
 *   - a non-final pair is a churn pair iff mix64(idx ^ k_churn) >> 11 < t_churn;
 *   - chunk c = the inserts (final or churn pairs) of slice c, then the
 *     deletes (churn pairs) of slice c-1, each in position order; slice c is
 *     positions [c*2^slice_log2, (c+1)*2^slice_log2); chunks 0..V^2/2^slice_log2.
 * mix64 is the SplitMix64 output function (Steele, Lea & Flood 2014).
 */
#ifndef GZ_GEN_H
#define GZ_GEN_H

#include <stddef.h>
#include <stdint.h>

#include "gz.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gz_gen gz_gen;

typedef struct {
    uint32_t L;            /* V = 2^L, 1 <= L <= 31 */
    uint32_t slice_log2;   /* positions per slice = 2^slice_log2, <= 2L */
    uint64_t k_feistel[4];
    uint64_t k_kron, k_churn, k_iso;
    uint64_t t_iso, t_churn; /* 53-bit thresholds */
} gz_kron_params;

/* table: host, (L+1)*(L+1) thresholds, row n00, column n11.  stream: a
 * cudaStream_t for all work of the generator.  Allocates scratch. */
gz_status gz_gen_kron_create(const gz_kron_params* p, const uint64_t* table, void* stream,
                             gz_gen** out);

/* Number of chunks (slices + 1). */
gz_status gz_gen_kron_num_chunks(gz_gen* g, uint64_t* n_chunks);

/* Write chunk c to device arrays u, v (capacity entries each, u < v per
 * update) and store its length in *n (host).  Synchronous.  Returns
 * GZ_EINVAL when c is out of range or the chunk does not fit. */
gz_status gz_gen_kron_chunk(gz_gen* g, uint64_t c, uint32_t* u, uint32_t* v, uint64_t capacity,
                            uint64_t* n);

gz_status gz_gen_destroy(gz_gen* g);

#ifdef __cplusplus
}
#endif

#endif /* GZ_GEN_H */
