// gz_handle.cuh -- host-side state of one graph (one gz_handle) and the internal
// launch entry points shared by the library's .cu files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gz.h"
#include "gz_internal.cuh"

// The partition buffers of one chunk: counts, offsets, front and back
// cursors (V+1 each), 2 * 2^chunk_log2 records, the tile table and 8 flag
// words ([0] batch invalid, [1] tile counter, [2] sticky invalid, [3] sticky
// timeout, [4..5] node window, [6..7] wait limit).
struct gz_partset {
    uint32_t *counts = nullptr, *offsets = nullptr, *cursor = nullptr, *cursor_hi = nullptr, *records = nullptr,
             *tile_node = nullptr, *flags = nullptr;
};

struct gz_handle {
    // geometry
    uint32_t V = 0, K = 0, R = 0, ncol = 0;  // ncol = 7K columns
    uint64_t seed = 0;
    uint64_t node_bytes = 0;
    uint32_t per_k_bytes = 0;
    gz_config cfg{};
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;

    // sketches (exact-depth form) and hash keys (kKeyWords 32-bit words per
    // column, word-major)
    uint8_t* d_sketch = nullptr;
    uint32_t* d_keys = nullptr;

    // ingestion scratch
    uint64_t chunk = 0;            // updates per partition pass
    uint32_t* d_counts = nullptr;  // V+1
    uint32_t* d_offsets = nullptr; // V+1
    uint32_t* d_cursor = nullptr;  // V: front cursors; after the scatter, the split of every segment
    uint32_t* d_cursor_hi = nullptr;  // V: back cursors of the scatter
    uint32_t* d_records = nullptr; // 2*chunk
    uint32_t* d_tile_node = nullptr; // first node of every record tile (2*chunk/tile + 2)
    uint32_t* d_stage = nullptr;   // 2 buffers x (u, v) x chunk, host-input staging (lazy)
    uint32_t* d_decode = nullptr;  // (u, v) x chunk decoded from packed indices (lazy)
    cudaStream_t copy_stream = nullptr;  // H2D copies of host input (lazy)
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    uint32_t* d_flags = nullptr;   // [0] batch invalid, [1] work counter, [2] sticky invalid, [4..5] node window
    uint32_t* d_scan_tmp = nullptr; // ceil((V+1)/1024) tile sums of the scans
    gz::PieceGeo geo{};            // hash piece width and counts (gz_internal.cuh)
    uint32_t block = 0;            // columns padded to a warp multiple
    uint32_t smem_rows = 0, tile = 0, small_seg = 0, batched_grid = 0;
    uint32_t delta_mode = 1;       // batched kernel's delta update: 0 load-xor-store, 1 shared atomics
    uint64_t batches_done = 0;     // partition passes issued (graph capture after 8)
    size_t batched_smem = 0;

    // pipelined ingest: chunk i+1 is partitioned on part_stream into the other
    // buffer set while chunk i's update runs on the handle's stream.  Set 0 is
    // the d_* buffers above, set 1 is pset1.  ev_part[b]: set b partitioned;
    // ev_upd[b]: set b's update done (the set may be partitioned again);
    // ev_in: the caller's inputs are ready (recorded at each ingest call).
    bool pipelined = false;
    int pipe_next = 0;
    gz_partset pset1;
    cudaStream_t part_stream = nullptr;
    cudaEvent_t ev_part[2] = {nullptr, nullptr}, ev_upd[2] = {nullptr, nullptr}, ev_in = nullptr;

    // sketches beyond HBM: nodes [0, res_nodes) in d_sketch, the others in
    // pinned host memory h_sketch, streamed shard by shard through two slots
    bool tiered = false;
    uint32_t shard_nodes = 0, res_nodes = 0;
    uint8_t* h_sketch = nullptr;
    static constexpr int kTierSlots = 3;  // copy-in, update and copy-out of three shards in flight
    uint8_t* d_slot[kTierSlots] = {};
    cudaStream_t tier_in = nullptr, tier_out = nullptr;
    cudaEvent_t ev_tin[kTierSlots] = {}, ev_tdone[kTierSlots] = {}, ev_tout[kTierSlots] = {};
    uint8_t* d_gather = nullptr;   // query: CubeSketch r of every node, V * per_k_bytes

    // query scratch (allocated on first query)
    bool query_ready = false;
    uint32_t *q_label = nullptr, *q_parent = nullptr, *q_count = nullptr, *q_off = nullptr,
             *q_cursor = nullptr, *q_members = nullptr, *q_roots = nullptr, *q_target = nullptr,
             *q_slot = nullptr, *q_F = nullptr, *q_F2 = nullptr,
             *q_M = nullptr, *q_M2 = nullptr, *q_flag = nullptr, *q_pos = nullptr,
             *q_forest = nullptr, *q_ctr = nullptr, *h_ctr = nullptr,
             *q_final = nullptr;  // per component root: 1 once it sampled EMPTY and nothing touched it
    uint32_t* h_labels = nullptr;  // pinned, V words: labels on their way to the caller
    int64_t* q_res = nullptr;
    uint64_t* q_acc = nullptr;     // per big component: XOR of its members' CubeSketch
    uint32_t q_slots_cap = 0;
    uint32_t q_merge_occ = 1;               // resident merge blocks per SM
    bool q_acc_dirty = true;                // accumulator slots need clearing before the next query
    cudaGraph_t q_graph = nullptr;          // the CC query as one graph (built at the first query)
    cudaGraphExec_t q_graph_exec = nullptr;
    int64_t* q_trace = nullptr;
    bool trace = false;
    bool trace_valid = false;

    // per-chunk ingest pipeline captured once as a CUDA graph
    bool graph_ready = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphNode_t node_validate = nullptr, node_scatter = nullptr;
    cudaGraphNode_t node_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t cap_ev[4] = {nullptr, nullptr, nullptr, nullptr};

    // profiling window (gz_profile_enable / gz_profile_read)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;  // quadruples: before/after partition, before/after update
    size_t ev_used = 0;
    uint64_t prof_batches = 0, prof_updates = 0, launches = 0;
    uint64_t* d_stats = nullptr;  // [0] rows flushed, [1] deep column updates

    std::string err;
};

namespace gz {

gz_status set_error(gz_handle* h, gz_status s, const std::string& msg);
gz_status cuda_check(gz_handle* h, cudaError_t e, const char* what);

// ingestion (gz_ingest.cu)
gz_status ingest_setup(gz_handle* h);
gz_status ingest_batch(gz_handle* h, const uint32_t* d_u, const uint32_t* d_v, uint64_t n);
// the stream on which the work that reads a call's inputs runs (the partition
// stream of a pipelined handle, else the handle's stream), made to wait for
// `ready` (an event of the caller's inputs; null: the handle stream's work so far)
cudaStream_t input_stream(gz_handle* h, cudaEvent_t ready);
// partition buffer set b (0 or 1)
gz_partset part_set(const gz_handle* h, int b);
// packed indices min*V+max -> (u, v) on stream st; non-canonical indices become (0, 0)
gz_status decode_idx(gz_handle* h, const uint64_t* d_idx, uint64_t n, uint32_t* d_u, uint32_t* d_v,
                     cudaStream_t st);
gz_status export_nested(gz_handle* h, uint32_t lo, uint32_t hi, uint64_t* d_alpha,
                        uint32_t* d_gamma);

// sketches beyond HBM: shard size and resident nodes for a device budget of
// budget_mb MiB (0 = everything resident: *res_nodes = V)
void tier_geometry(uint32_t V, uint64_t node_bytes, uint32_t budget_mb, uint32_t* shard_nodes,
                   uint32_t* res_nodes);
// make the handle stream wait for the last copy-outs of host shards
gz_status tier_settle(gz_handle* h);
// copy the full sketches of nodes [lo, hi) into dst (device, (hi-lo)*node_bytes) on the handle stream
gz_status tier_gather_nodes(gz_handle* h, uint32_t lo, uint32_t hi, uint8_t* dst);

// query (gz_query.cu)
// Every component of more than kSlotAbove members gets an accumulator slot
// (one CubeSketch) that the merge kernel fills; at most V / (kSlotAbove + 1)
// components are that large.
constexpr uint32_t kSlotAbove = 1;
inline uint32_t query_slots(uint32_t V) { return V / (kSlotAbove + 1) + 1; }
gz_status query_setup(gz_handle* h);
gz_status boruvka(gz_handle* h, bool want_forest, uint32_t* labels, uint32_t* forest_uv,
                  size_t* n_edges, uint32_t* n_cc, gz_query_stats* st);


// exclusive scan: out[0..n] with out[n] = total; out2 (optional) = copy of out[0..n);
// out3 (optional) = out[1..n] (inclusive sums); tile_scratch holds ceil(n / 1024) u32
void launch_scan(const uint32_t* in, uint32_t* out, uint32_t* out2, uint32_t* out3, uint32_t n, cudaStream_t s,
                 uint32_t* tile_scratch);

}  // namespace gz
