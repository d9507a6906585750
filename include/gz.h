/*
 * gz.h -- C ABI of the B300 GraphZeppelin hot path.
 *
 * GraphZeppelin (Tench et al., SIGMOD 2022, arXiv 2203.14927) answers
 * connected-components queries on a graph given as a stream of edge
 * insertions and deletions, by keeping one "node sketch" per vertex: K
 * CubeSketch l0-samplers of the vertex's characteristic vector (Section 2.2,
 * Section 3.2) and running Boruvka's algorithm on the sketches when queried.
 * This library keeps every node sketch resident in device memory and runs
 * ingestion and queries in CUDA kernels for sm_103a.
 *
 * Conventions shared by every call:
 *   - Return value: gz_status.  GZ_OK on success.  On any other value a
 *     one-line reason is available from gz_last_error(handle).
 *   - Pointers: "host" pointers are ordinary CPU memory (pinned memory gives
 *     faster copies); "device" pointers are CUDA global memory of the device
 *     current when the handle was created.  Buffers stay owned by the caller.
 *   - Streams: all device work of a handle is issued on the handle's CUDA
 *     stream (gz_create / gz_set_stream; NULL = the legacy default stream).
 *     Calls return once the work is queued unless stated otherwise.
 *   - Threading: a handle must not be used by two threads at once; distinct
 *     handles are independent and may be driven concurrently.
 *   - Geometry (readings of Section 5.1 and Table tab:size): every node sketch
 *     holds K = ceil(log_{3/2} V) CubeSketches of 7 columns x R rows,
 *     R = 2*ceil(log2 V); a bucket is a 64-bit alpha and a 32-bit gamma, so a
 *     node sketch takes K*7*R*12 bytes.
 *   - Edge index of an unordered pair {u,v}: idx = min*V + max (a position
 *     of the characteristic vector of Section 2.2).
 *   - Hashes (readings of Section 3.2, which asks for 2-wise independent h1
 *     and h2), functions of an edge's endpoints u < v: with L = ceil(log2 V)
 *     and p = 33 - L, a piece with 32-bit keys (k0, k1, k2) is the top p bits
 *     of (k0*u + k1*v + k2) mod 2^32 (strongly universal); pieces are
 *     concatenated, the first most significant.  The edge lies in nested
 *     rows 0..d, d = min(leading zeros of ceil((R-1)/p) pieces, R-1); its
 *     checksum h2 is the first 32 bits of ceil(32/p) pieces.  Key word w of
 *     column col = 7k+j is the low half of SplitMix64 output 256*col + w of
 *     the seed; words 0..127 feed the depth pieces, 128..255 the checksum's.
 */
#ifndef GZ_H
#define GZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gz_handle gz_handle;

typedef enum {
    GZ_OK = 0,
    GZ_EINVAL = 1,       /* bad argument, or a rejected update batch */
    GZ_ENOMEM = 2,       /* device or host allocation failed */
    GZ_ECUDA = 3,        /* a CUDA call failed; see gz_last_error */
    GZ_ESKETCH_FAIL = 4, /* query finished but a sketch failed (result may be wrong) */
    GZ_ETIMEOUT = 5,     /* a bounded wait in the update kernel ran out (reported,
                            like a discarded batch, by the next sync, query or export) */
    GZ_EBUSY = 6         /* reserved */
} gz_status;

/* Ingestion kernel choice. */
enum {
    GZ_KERNEL_BATCHED = 0, /* partition by endpoint + per-node batched update (default) */
    GZ_KERNEL_PLAIN = 1    /* one thread per (update, column), global atomics */
};

/* Tuning knobs; a zero field takes the built-in default. */
typedef struct {
    uint32_t chunk_log2;    /* updates processed per partition pass = 2^chunk_log2 (default 24) */
    uint32_t kernel;        /* GZ_KERNEL_BATCHED (V <= 2^21) or GZ_KERNEL_PLAIN (any V) */
    uint32_t smem_rows;     /* exact-depth rows staged in shared memory (default 16; at most 16
                               and R-1) */
    uint32_t tile_records;  /* records per work tile of the batched kernel (default 512) */
    uint32_t ctas_per_sm;   /* resident CTAs per SM of the persistent batched kernel (default: max) */
    uint32_t small_segment; /* node segments shorter than this skip shared-memory staging (default 4) */
    uint32_t smem_mode;     /* delta update in shared memory: 0 default (= 1), 1 32-bit shared
                               atomics, 2 load-xor-store */
    uint32_t no_graph;      /* 1: no CUDA graphs: launch a chunk's kernels one by one instead of
                               replaying the graph captured after the handle's 8th chunk, and drive
                               a CC query's rounds from the host instead of one captured graph
                               with a device-side loop (default 0) */
    uint32_t device_sketch_mb; /* HBM for node sketches, MiB (0: all of them in HBM).  When the
                               sketches need more, nodes beyond the budget live in pinned host
                               memory (sketches beyond HBM, below) */
    uint32_t no_pipeline;   /* 1: partition and update every chunk on the handle's stream.  By
                               default (0) the batched kernel's handles partition chunk i+1 on a
                               second stream while chunk i's sketch update runs, in a second set
                               of partition buffers (2 * 2^chunk_log2 * 4 bytes of records more);
                               handles with sketches beyond HBM never do */
    uint32_t reserved[2];
} gz_config;

/* Sketches beyond HBM (the paper's hybrid streaming model of Section 4, with
 * host memory as the slow tier): with cfg.device_sketch_mb set below the
 * sketches' size, the nodes are cut into shards of a quarter of the budget
 * (at most 512 MiB, at least one node);
 * the first shards that fit the budget stay in HBM and the others live in
 * pinned host memory.  Each chunk of updates is partitioned once; the batched
 * update then runs on the resident shards in place and on each host shard
 * after copying it into one of three device slots, the copy-in of the next
 * shard and the copy-out of the previous one overlapping the update of the
 * current one (so large chunks amortise the transfers, as large buffers amortise disk
 * I/O in the paper).  Queries copy CubeSketch r of every node into one device
 * array per Boruvka round.  Results are identical to an all-HBM handle. */

/* Statistics of the last query. */
typedef struct {
    uint32_t rounds;        /* Boruvka rounds run */
    uint32_t fails_last;    /* components whose CubeSketch failed in the last round run */
    uint32_t exhausted;     /* 1 when round K-1 still produced merges */
    uint32_t n_components;  /* connected components reported */
    uint32_t fails_total;   /* FAIL results summed over all rounds */
    uint32_t reserved;
    float ms;               /* wall time of the query, host clock, milliseconds */
} gz_query_stats;

/* Geometry for V vertices: K CubeSketches per node, R rows per column.
 * Returns GZ_EINVAL for V < 2 or V > 2^31. */
gz_status gz_geometry(uint32_t V, uint32_t *K, uint32_t *R);

/* Bytes of device memory a handle for V vertices holds (sketches + scratch)
 * under cfg (may be NULL). */
gz_status gz_memory_bytes(uint32_t V, const gz_config *cfg, size_t *bytes);

/* Allocate zeroed node sketches for V vertices with hash keys derived from
 * seed (Section 5, initialisation: "allocates log(V) CubeSketches per node").
 * cfg may be NULL.  stream is a cudaStream_t (NULL = default stream).
 * On success *out owns V*K*7*R*12 bytes of device memory plus scratch. */
gz_status gz_create(uint32_t V, uint64_t seed, const gz_config *cfg,
                    void *stream, gz_handle **out);

/* Free everything the handle owns (synchronises its stream first). */
gz_status gz_destroy(gz_handle *h);

/* Change the stream later work is issued on. */
gz_status gz_set_stream(gz_handle *h, void *stream);

/* Apply n updates: update i toggles edge {u[i], v[i]} in the sketches of both
 * endpoints (Section 2.2; Fig. cube_code update_sketch; Delta is implicit
 * because the vectors live in Z_2, Section 3.2).  An insert and a delete of
 * the same edge are the same toggle; the caller keeps the stream valid in the
 * sense of Section 2.1 (insert only absent edges, delete only present ones).
 *   u, v       : n vertex ids each; host memory if on_device == 0, else device
 *                memory.  Any order of endpoints is accepted.
 *   Validation : an update with u == v or an id >= V invalidates its batch.
 *                With device input a batch is the whole call when
 *                n <= 2^chunk_log2, else each consecutive slice of
 *                2^chunk_log2 updates.  With host input the slices of a call
 *                ramp up: 2^chunk_log2 / 16 updates, then 2^chunk_log2 / 4,
 *                then 2^chunk_log2 each (at least 256), so the first copy to
 *                the device, which nothing overlaps, is short.  An invalid
 *                batch is discarded whole before any sketch changes.  Validation
 *                runs on the device, so the call itself returns GZ_OK and the
 *                error is reported as GZ_EINVAL by the next gz_sync, query or
 *                export call on this handle.
 *   Ownership  : host inputs may be reused when the call returns; device
 *                inputs must stay unchanged until the handle's stream has
 *                completed the work queued by this call. */
gz_status gz_edge_update(gz_handle *h, const uint32_t *u, const uint32_t *v,
                         size_t n, int on_device);

/* The same updates given as packed edge indices: idx[i] = min(u,v)*V +
 * max(u,v), the coordinate of edge {u,v} in the node vectors of Section 3.1.
 *   idx        : n u64 indices; host memory if on_device == 0, else device
 *                memory (8-byte aligned).
 *   Validation : an index that is not canonical (min >= max, so also a self
 *                loop, or idx >= V^2) invalidates its batch, with the same
 *                batches (device or host input), discard rule and deferred
 *                GZ_EINVAL report as gz_edge_update.
 *   Ownership  : as gz_edge_update.  The first call allocates a decode
 *                buffer of 8 * 2^chunk_log2 bytes on the device. */
gz_status gz_edge_update_idx(gz_handle *h, const uint64_t *idx, size_t n, int on_device);

/* Wait for all queued work of the handle; returns GZ_EINVAL once if a batch
 * was rejected since the last report, GZ_ETIMEOUT once if a bounded wait of
 * the update kernel ran out (its sketches are then incomplete). */
gz_status gz_sync(gz_handle *h);

/* Zero every node sketch (the empty graph). */
gz_status gz_reset(gz_handle *h);

/* Connected components by Boruvka over the sketches (Section 2.2; the three
 * phases of each round in the proof of Lemma (CC I/O)): round r samples one
 * edge per component from CubeSketch r of the XOR of its members' sketches,
 * then merges.  Synchronous.
 *   labels : host, V entries, or NULL: labels[x] = minimum vertex id of x's
 *            component.
 *   n_cc   : host, or NULL: number of components.
 *   st     : host, or NULL: statistics.
 * Returns GZ_ESKETCH_FAIL (labels still filled) when a component's sketch had
 * no usable bucket in the last round run, or all K rounds still merged. */
gz_status gz_connected_components(gz_handle *h, uint32_t *labels, uint32_t *n_cc,
                                  gz_query_stats *st);

/* Spanning forest by the same Boruvka rounds (list_spanning_forest of
 * Section 5).  uv: host, 2*(V-1) entries; edges are written as (u,v) pairs
 * with u < v, round by round and, within a round, by ascending component id
 * (the order in which a sequential union-find over the sampled edges accepts
 * them).  *n_edges = V - number of components.  labels may be NULL.
 * Synchronous; same return values as gz_connected_components. */
gz_status gz_list_spanning_forest(gz_handle *h, uint32_t *uv, size_t *n_edges,
                                  uint32_t *labels, gz_query_stats *st);

/* Per-round samples of the last query, for checking: out[r*V + c] for round
 * r < K and vertex c = the sampled edge index of component c (c its minimum
 * vertex id), -1 when the component's sketch was empty, -2 on FAIL, -3 when c
 * was not a component id in that round, -4 when round r was not run.
 * out: host, K*V entries.  Only filled when the query ran after
 * gz_enable_trace(h, 1). */
gz_status gz_enable_trace(gz_handle *h, int enable);
gz_status gz_query_trace(gz_handle *h, int64_t *out);

/* Copy node sketches [node_lo, node_hi) in the paper's NESTED form (bucket
 * (i,j) = XOR over indices e with h1(e) = 0 mod 2^i, Eq. 1-2) to
 * alpha[node][k][j][row] (u64) and gamma[node][k][j][row] (u32), rows
 * ascending.  on_device selects device (1) or host (0) output buffers.
 * Synchronous. */
gz_status gz_export_sketch(gz_handle *h, uint32_t node_lo, uint32_t node_hi,
                           uint64_t *alpha, uint32_t *gamma, int on_device);

/* Checkpoint / resume.  By linearity the node sketches are the whole state of
 * a graph (Section 2.2: the stream is summarised by them), so a checkpoint is
 * a 64-byte header -- magic "GZB3CKP1", version (3), V, K, R, seed, bytes per
 * node sketch -- followed by the raw sketch array (the device form of
 * gz_info).  Both calls
 * are synchronous; buf is host memory owned by the caller.
 *   gz_checkpoint_bytes: size a checkpoint of h needs.
 *   gz_checkpoint      : write it (GZ_EINVAL if size is too small, or if a
 *                        rejected batch is still unreported).
 *   gz_restore         : new handle holding exactly the checkpointed state
 *                        (GZ_EINVAL on a bad magic, version or geometry). */
gz_status gz_checkpoint_bytes(gz_handle *h, size_t *bytes);
gz_status gz_checkpoint(gz_handle *h, void *buf, size_t size);
gz_status gz_restore(const void *buf, size_t size, const gz_config *cfg, void *stream,
                     gz_handle **out);

/* Geometry and device pointer of the raw sketch array of a handle.  Device
 * form: exact-depth rows (an index is XORed into the one row of its depth; the
 * paper's nested row i is the XOR of rows i..R-1), layout per node: for each
 * k, alpha[row][j] (u64) then gamma[row][j] (u32, the XOR of the checksums
 * h2 of the row's indices).  For a handle with sketches beyond HBM the device
 * array holds only part of the nodes, so *sketch_device is set to NULL there.
 * Any output pointer may be NULL. */
gz_status gz_info(gz_handle *h, uint32_t *V, uint32_t *K, uint32_t *R,
                  size_t *node_bytes, void **sketch_device);

/* Device-time profile of ingestion, for measurement.  Times come from CUDA
 * events recorded on the handle's stream around each launch, summed over the
 * window since gz_profile_enable(h, 1). */
typedef struct {
    uint64_t batches;          /* partition passes (chunks) timed */
    uint64_t updates;          /* updates in those passes */
    double partition_ms;       /* validation + histogram, scan, scatter */
    double update_ms;          /* batched (or plain) sketch-update kernel */
    uint64_t rows_flushed;     /* (node, column, row) buckets the batched kernel's flush XORed into HBM */
    uint64_t deep_updates;     /* column updates that bypassed shared memory */
    uint64_t kernel_launches;  /* kernels launched by this handle in the window */
} gz_profile;

/* Start (enable != 0) or stop a profiling window; starting clears totals. */
gz_status gz_profile_enable(gz_handle *h, int enable);

/* Synchronise and read the totals of the current window. */
gz_status gz_profile_read(gz_handle *h, gz_profile *out);

/* ------------------------------------------------------------------ serving
 * Many independent graphs on one GPU.  The paper serves one graph and lets a
 * query wait for the buffered updates before it (Section 6.6, "Connectivity
 * Queries are Fast"); a server holds many graphs' node sketches resident and
 * keeps the GPU busy across them:
 *   - admission by memory: a graph takes device memory (its sketches and
 *     scratch, gz_memory_bytes plus query scratch) when its first request is
 *     served, and only while the running total stays within hbm_budget;
 *     otherwise it waits; a closed graph gives its memory back when its last
 *     request is done;
 *   - eviction: when a graph has waited 20 ms for memory, the least recently
 *     used resident graph with no pending request (and all its sketches in
 *     HBM) has its sketches copied into pinned host memory (a pool of 256 MB
 *     chunks kept until gz_server_destroy) and its device memory freed; its
 *     next request restores them into a fresh handle, bit for bit;
 *   - continuous batching: `slots` workers, each a host thread with its own
 *     CUDA stream, repeatedly take a resident graph with pending requests
 *     (oldest request first; finishing resident graphs is what frees memory),
 *     else the admissible graph with the oldest request, and serve up to
 *     max_batch of its pending requests in order; an admissible graph whose
 *     request is 20 ms older than every resident one goes first.  Requests
 *     that arrive while others run join the queue and are picked up as soon
 *     as a slot and memory free up, and the work of different graphs overlaps
 *     on the device;
 *   - server graphs run with no_pipeline set (the server overlaps graphs,
 *     not the partition and update of one graph);
 *   - a graph is served by one worker at a time, so each graph sees its
 *     requests in submission order and gets exactly the result it would get
 *     alone.
 * Times are host-clock milliseconds since the server started. */
typedef struct gz_server gz_server;

typedef struct {
    uint64_t hbm_budget; /* device bytes the server may hold for graphs (0 = 80% of free memory) */
    uint32_t slots;      /* worker threads / CUDA streams (0 = 4) */
    uint32_t max_batch;  /* most requests one worker takes from a graph at a time (0 = 64) */
    uint32_t host_pool_mb; /* pinned host memory for evictions to pin at creation (pinning
                              runs at a few GB/s; 0 = pin on demand) */
    uint32_t reserved[5];
} gz_server_config;

typedef struct {
    uint64_t req_id;
    uint32_t graph;
    uint32_t kind;         /* 0 update batch, 1 connected-components query */
    int32_t status;        /* gz_status of the request */
    uint32_t n_components; /* queries: number of components */
    uint64_t n_updates;    /* update batches: updates applied */
    double submit_ms, start_ms, done_ms;
} gz_completion;

typedef struct {
    uint64_t resident_bytes, peak_resident_bytes, budget_bytes;
    uint32_t graphs, resident_graphs, waiting_graphs, pending_requests;
    uint64_t completed_requests;
    uint64_t evictions;      /* graphs checkpointed to host memory to make room */
    uint32_t evicted_graphs; /* graphs held in host memory now */
    uint32_t pinned_chunks;  /* 256 MB pinned host chunks the server holds for evictions */
    double evict_ms;         /* host time spent checkpointing evicted graphs out */
    double restore_ms;       /* host time spent restoring them */
} gz_server_stats;

/* Start a server on the current device (cfg may be NULL).  The server raises
 * the release threshold of the device's default stream-ordered memory pool to
 * its HBM budget, so memory of released graphs is kept for later admissions
 * (the setting is the device's, shared with the rest of the process). */
gz_status gz_server_create(const gz_server_config *cfg, gz_server **out);

/* Finish every accepted request, then stop the workers and free everything. */
gz_status gz_server_destroy(gz_server *s);

/* Register a graph (no device memory is taken yet).  cfg may be NULL. */
gz_status gz_server_add_graph(gz_server *s, uint32_t V, uint64_t seed, const gz_config *cfg,
                              uint32_t *graph);

/* Queue an update batch (host arrays; same meaning as gz_edge_update).  By
 * default the call copies u and v; with flags & GZ_SUBMIT_NOCOPY it keeps the
 * pointers instead, and the caller must keep both arrays unchanged until the
 * request's completion has been polled (pinned memory gives the fastest
 * host-to-device copies).  *req_id identifies its completion. */
#define GZ_SUBMIT_NOCOPY 1u
gz_status gz_server_submit_update(gz_server *s, uint32_t graph, const uint32_t *u,
                                  const uint32_t *v, size_t n, uint32_t flags, uint64_t *req_id);

/* Queue a connected-components query; labels (host, V entries, or NULL) is
 * written before the completion is reported and must stay valid until then. */
gz_status gz_server_submit_query(gz_server *s, uint32_t graph, uint32_t *labels,
                                 uint64_t *req_id);

/* No more requests for this graph: its memory is released once its queue is
 * empty. */
gz_status gz_server_close_graph(gz_server *s, uint32_t graph);

/* Move up to max completions into out (oldest first); waits up to wait_ms
 * milliseconds for the first one (0 = do not wait). */
gz_status gz_server_poll(gz_server *s, gz_completion *out, size_t max, size_t *n, int wait_ms);

/* Wait until every submitted request has completed. */
gz_status gz_server_drain(gz_server *s);

gz_status gz_server_stats_read(gz_server *s, gz_server_stats *out);

/* Change the HBM budget while the server runs.  A smaller budget than the
 * bytes now resident makes admissions wait (and idle graphs be evicted) until
 * the total fits; graphs registered with more bytes than the new budget wait
 * until it grows again.  GZ_EINVAL for a zero budget. */
gz_status gz_server_set_budget(gz_server *s, uint64_t hbm_budget);

/* Reason of the most recent failed request ("" if none); valid until the next
 * call of this function by the same thread. */
const char *gz_server_last_error(gz_server *s);

/* Allocation-free ingestion (the paper has no counterpart).  Some callers
 * cannot let a library call cudaMalloc: a host framework whose caching
 * allocator owns the device memory and must account for every byte (an
 * allocation behind its back can fail, or fragment its pool); a latency-bound
 * loop in which cudaMalloc, which may synchronise the device and takes a
 * driver lock, is not allowed.  This call applies a batch of updates like
 * gz_edge_update but allocates and frees nothing: its scratch is a fixed
 * array of about 10 MB in the library's static device memory, which every GPU
 * that loads the library holds until the process exits.
 *   sketch : device, all V*K*84*R bytes of node sketches in the device form
 *            of gz_info (per node, for each k, alpha[R][7] u64 then
 *            gamma[R][7] u32), zeroed for the empty graph: memory the caller
 *            owns, or the array of an all-HBM handle from gz_info.  An array
 *            holding fewer nodes (gz_info reports NULL for a handle with
 *            sketches beyond HBM) is not valid: the kernel would write past
 *            its end.
 *   V, seed: vertex count (2 <= V <= GZ_NOALLOC_MAX_V) and the hash seed the
 *            sketches were built with.
 *   u, v   : device, n updates (n <= GZ_NOALLOC_MAX_UPDATES), same meaning and
 *            validation as gz_edge_update: a self loop or an id >= V discards
 *            the whole batch.
 *   status : device u32 or NULL; set on the stream to 1 when the batch was
 *            discarded, 2 when a bounded wait of the update kernel ran out
 *            (the sketches are then incomplete), else 0.
 *   stream : cudaStream_t of all the work (NULL = default stream).
 * Returns GZ_EINVAL (nothing queued) for V or n beyond the limits or null
 * pointers, GZ_ECUDA when a CUDA call fails: the set-up and the occupancy
 * query run before anything is queued, so a failure there leaves everything
 * untouched; a failure after the update kernel was queued leaves the sketches
 * unknown.  The status word is written only when GZ_OK is returned.  An error
 * left pending by earlier, unrelated work of the calling thread is cleared on
 * entry and not reported.  The first call on a device sets up
 * that device (it looks up the scratch array's device address and the update
 * kernel's occupancy); make that first call before any stream capture
 * begins.  All calls share the one scratch array, which keeps the last call's
 * contents (each call clears what must start at zero), so calls that overlap
 * on the GPU race: issue them on one stream, or order them. */
#define GZ_NOALLOC_MAX_V (1u << 17)
#define GZ_NOALLOC_MAX_UPDATES (1ull << 20)
gz_status gz_sketch_update_noalloc(void *sketch, uint32_t V, uint64_t seed,
                                   const uint32_t *u, const uint32_t *v, size_t n,
                                   uint32_t *status, void *stream);

/* Bound of the update kernel's waits, for testing the timeout path.  The
 * batched kernel's warps hand tiles to each other through shared-memory
 * barriers, and every wait on one is bounded: at most `polls` polls, each of
 * which may suspend the thread for up to about suspend_ns nanoseconds
 * (defaults 2^22 and 1000).  A wait that runs out makes the kernel stop and
 * report: the next gz_sync, query or export returns GZ_ETIMEOUT (the
 * allocation-free call sets status 2), and the sketches are incomplete until
 * gz_reset or a restore.  With polls = 1 and suspend_ns = 0 the waits run out
 * almost at once, so a test can drive that path without any GPU fault.
 * polls = 0 restores the defaults.  h = NULL sets the bound of the
 * allocation-free entry point on the current device.  Synchronous. */
gz_status gz_set_wait_limit(gz_handle *h, uint32_t polls, uint32_t suspend_ns);

/* Human-readable reason of the last non-OK status of h (never NULL); with
 * h == NULL, the reason the calling thread's last gz_create failed. */
const char *gz_last_error(gz_handle *h);

/* Library version string. */
/* Single-vector l0 sketches, for the micro-benchmark of Fig. l0speedup: the
 * standard l0 sampler of Fig. agm_code (Section 3.1) beside CubeSketch
 * (Fig. cube_code) on a plain vector of length n.  Both use 7 columns and
 * R = ceil(log2 n) rows, column keys a_j = SM(seed,5j)|1, b_j = SM(seed,5j+1),
 * c0_j, c1_j, c2_j = SM(seed,5j+2..5j+4) (SplitMix64, the node sketches'
 * schedule), and put position x into rows 0..d,
 * d = min(clz64(a_j*x + b_j), R-1) (nested rows, as in both figures).
 *   GZ_L0_CUBE     bucket (alpha u64, gamma u32): alpha ^= x,
 *                  gamma ^= ((c0_j*lo32(x) + c1_j*hi32(x) + c2_j) mod 2^64) >> 32.
 *                  Layout per sketch: alpha[7][R] then gamma[7][R], padded
 *                  to a multiple of 8 bytes (84R rounded up).
 *   GZ_L0_STANDARD bucket (a, b, c), u64 each: a += x*delta, b += delta
 *                  (two's complement), c = (c + delta * r_j^x) mod p with
 *                  p = 2^61 - 1 and r_j = 1 + c0_j mod (p - 1).
 *                  Layout per sketch: a[7][R], b[7][R], c[7][R]. */
#define GZ_L0_CUBE 0
#define GZ_L0_STANDARD 1

/* rows R and the bytes of one sketch of each kind for vector length n >= 2 */
gz_status gz_l0_geometry(uint64_t n, uint32_t *rows, uint32_t *bytes_cube, uint32_t *bytes_standard);

/* Apply m updates to each of `sketches` independent sketches of one kind.
 *   x       : device, sketches*m positions in 1..n, sketch-major (sketch s
 *             takes x[s*m .. s*m+m), in that order).
 *   delta   : device, sketches*m values +1 or -1, or NULL for all +1
 *             (CubeSketch ignores it: a delete is the same toggle).
 *   buckets : device, sketches * bytes-per-sketch, updated in place.
 *   stream  : cudaStream_t of the work (NULL = default stream); asynchronous.
 * Positions outside 1..n and deltas other than +-1 are not checked on the
 * device; they give meaningless buckets, not faults.  Returns GZ_EINVAL for an
 * unknown kind, n < 2 or n >= 2^61, or null buffers. */
gz_status gz_l0_update(int kind, uint64_t n, uint64_t seed, uint32_t sketches, uint32_t m,
                       const uint64_t *x, const int32_t *delta, void *buckets, void *stream);

/* Measured integer throughput of the current device, the ceilings of the
 * batched update kernel (its work per (record, column) pair is integer only):
 * kind 0 = 32-bit multiply-add, 1 = three-input logic op, 2 = the two
 * interleaved, 3 = leading-zero count, 4 = 32-bit shared-memory atomic XOR.
 * *ops_per_s = thread-operations per second over all SMs, the best of nine
 * timed launches of a few milliseconds each (after one untimed).
 * Synchronous; uses its own stream and a 4-byte device allocation. */
gz_status gz_int_peak(int kind, double *ops_per_s);

const char *gz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GZ_H */
