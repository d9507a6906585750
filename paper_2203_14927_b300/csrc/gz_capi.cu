// gz_capi.cu -- the extern "C" entry points declared in include/gz.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/gz.h"
#include "gz_handle.cuh"

namespace gz {

gz_status set_error(gz_handle* h, gz_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

gz_status cuda_check(gz_handle* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GZ_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return set_error(h, GZ_ENOMEM, m);
    return set_error(h, GZ_ECUDA, m);
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the n-th output (n >= 0) of
// the generator whose state starts at `state`.
static uint64_t splitmix_nth(uint64_t state, uint64_t n) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull * (n + 1);
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

static bool geometry(uint32_t V, uint32_t* K, uint32_t* R) {
    if (V < 2 || V > (1u << 31)) return false;
    uint32_t L = 0;
    while ((1ull << L) < V) ++L;
    // least k with (3/2)^k >= V  <=>  3^k >= V * 2^k
    unsigned __int128 lhs = 1, rhs = V;
    uint32_t k = 0;
    while (lhs < rhs) {
        lhs *= 3;
        rhs *= 2;
        ++k;
    }
    *K = k;
    *R = 2 * L;
    return true;
}

void tier_geometry(uint32_t V, uint64_t node_bytes, uint32_t budget_mb, uint32_t* shard_nodes,
                   uint32_t* res_nodes) {
    const uint64_t budget = (uint64_t)budget_mb << 20;
    // shards of a quarter of the budget, at most 512 MiB and at least one node
    const uint64_t target = std::min<uint64_t>(512ull << 20, budget / 4);
    const uint64_t sn = std::max<uint64_t>(1, std::min<uint64_t>(V, target / node_bytes));
    *shard_nodes = (uint32_t)sn;
    if (budget_mb == 0 || (uint64_t)V * node_bytes <= budget) {
        *res_nodes = V;
        return;
    }
    *res_nodes = (uint32_t)std::min<uint64_t>(V, budget / node_bytes / sn * sn);
}

static size_t scratch_bytes(uint32_t V, uint64_t chunk) {
    return (size_t)4 * (V + 1) * 4 + (size_t)2 * chunk * 4 + 64;
}

}  // namespace gz

using namespace gz;

extern "C" {

const char* gz_version(void) { return "gz-b300 0.1 (sm_103a)"; }

// reason of the calling thread's last failed gz_create (no handle exists then)
static thread_local std::string g_create_err = "no failed gz_create on this thread";

const char* gz_last_error(gz_handle* h) {
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

gz_status gz_geometry(uint32_t V, uint32_t* K, uint32_t* R) {
    uint32_t k, r;
    if (!gz::geometry(V, &k, &r)) return GZ_EINVAL;
    if (K) *K = k;
    if (R) *R = r;
    return GZ_OK;
}

gz_status gz_memory_bytes(uint32_t V, const gz_config* cfg, size_t* bytes) {
    uint32_t K, R;
    if (!gz::geometry(V, &K, &R) || !bytes) return GZ_EINVAL;
    const uint32_t cl = cfg && cfg->chunk_log2 ? cfg->chunk_log2 : 24;
    const uint64_t chunk = 1ull << cl;
    const uint64_t node_bytes = (uint64_t)K * 84ull * R;
    uint32_t shard_nodes = 0, res_nodes = 0;
    tier_geometry(V, node_bytes, cfg ? cfg->device_sketch_mb : 0, &shard_nodes, &res_nodes);
    size_t tier = 0;
    if (res_nodes < V)  // the shard slots and the per-round query gather array
        tier = gz_handle::kTierSlots * (size_t)shard_nodes * node_bytes + (size_t)V * 84ull * R;
    size_t pipe = 0;  // the second partition buffer set of a pipelined handle
    if (res_nodes == V && (!cfg || (cfg->kernel == GZ_KERNEL_BATCHED && !cfg->no_pipeline)))
        pipe = scratch_bytes(V, chunk) + (size_t)(2 * chunk / 256 + 2) * 4;
    *bytes = (size_t)res_nodes * node_bytes + tier + pipe + (size_t)K * 7 * 4 * kKeyWords + scratch_bytes(V, chunk);
    return GZ_OK;
}

gz_status gz_create(uint32_t V, uint64_t seed, const gz_config* cfg, void* stream, gz_handle** out) {
    if (!out) return GZ_EINVAL;
    *out = nullptr;
    uint32_t K, R;
    if (!gz::geometry(V, &K, &R)) return GZ_EINVAL;
    gz_handle* h = new (std::nothrow) gz_handle();
    if (!h) return GZ_ENOMEM;
    if (cfg) h->cfg = *cfg;
    if (h->cfg.chunk_log2 == 0) h->cfg.chunk_log2 = 24;
    if (h->cfg.chunk_log2 < 8 || h->cfg.chunk_log2 > 30 || h->cfg.kernel > GZ_KERNEL_PLAIN) {
        delete h;
        return GZ_EINVAL;
    }
    h->V = V;
    h->K = K;
    h->R = R;
    h->ncol = K * GZ_COLS;
    h->seed = seed;
    h->per_k_bytes = 84u * R;
    h->node_bytes = (uint64_t)K * h->per_k_bytes;
    h->stream = static_cast<cudaStream_t>(stream);
    h->chunk = 1ull << h->cfg.chunk_log2;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    gz_status s = cuda_check(h, e, "device query");
    if (s != GZ_OK) {
        delete h;
        return s;
    }
    // keys: word w of column col is lo32 of SplitMix64 output 256*col + w,
    // stored word-major (word w of every column at hk[w * ncol + col])
    const size_t ncol = h->ncol;
    uint32_t* hk = new (std::nothrow) uint32_t[(size_t)kKeyWords * ncol];
    if (!hk) {
        delete h;
        return GZ_ENOMEM;
    }
    for (size_t col = 0; col < ncol; ++col)
        for (uint32_t w = 0; w < kKeyWords; ++w)
            hk[w * ncol + col] = (uint32_t)splitmix_nth(seed, (uint64_t)kKeyWords * col + w);
    // Stream-ordered allocations: creating or destroying a handle never
    // synchronises the whole device (cudaFree would), so a server can admit
    // and release graphs while other graphs' work runs.
    tier_geometry(V, h->node_bytes, h->cfg.device_sketch_mb, &h->shard_nodes, &h->res_nodes);
    h->tiered = h->res_nodes < V;
    if (h->tiered && h->cfg.kernel != GZ_KERNEL_BATCHED) {
        set_error(h, GZ_EINVAL, "sketches beyond HBM need the batched kernel");
        g_create_err = h->err;
        delete[] hk;
        delete h;
        return GZ_EINVAL;
    }
    const size_t sk = (size_t)h->res_nodes * h->node_bytes;
    cudaStream_t as = h->stream;
    e = sk ? cudaMallocAsync(&h->d_sketch, sk, as) : cudaSuccess;
    if (e == cudaSuccess && sk) e = cudaMemsetAsync(h->d_sketch, 0, sk, h->stream);
    if (h->tiered) {
        const size_t hb = (size_t)(V - h->res_nodes) * h->node_bytes;
        const size_t slot = (size_t)h->shard_nodes * h->node_bytes;
        if (e == cudaSuccess) e = cudaMallocHost(&h->h_sketch, hb);
        if (e == cudaSuccess) std::memset(h->h_sketch, 0, hb);
        for (int b = 0; b < gz_handle::kTierSlots && e == cudaSuccess; ++b) {
            e = cudaMallocAsync(&h->d_slot[b], slot, as);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_tin[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_tdone[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_tout[b], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaMallocAsync(&h->d_gather, (size_t)V * h->per_k_bytes, as);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->tier_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->tier_out, cudaStreamNonBlocking);
    }
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_keys, kKeyWords * ncol * sizeof(uint32_t), as);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_keys, hk, kKeyWords * ncol * sizeof(uint32_t), cudaMemcpyHostToDevice, as);
    if (e == cudaSuccess) e = cudaStreamSynchronize(as);  // hk is freed below
    delete[] hk;
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_counts, (size_t)(V + 1) * 4, as);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_offsets, (size_t)(V + 1) * 4, as);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_cursor, (size_t)(V + 1) * 4, as);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_cursor_hi, (size_t)(V + 1) * 4, as);
    if (e == cudaSuccess && h->cfg.kernel == GZ_KERNEL_BATCHED)
        e = cudaMallocAsync(&h->d_records, (size_t)2 * h->chunk * 4, as);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_flags, 32, as);  // [4], [5]: node window
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_scan_tmp, ((size_t)(V + 1) / 1024 + 2) * 4, as);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->d_stats, 2 * sizeof(uint64_t), as);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_stats, 0, 2 * sizeof(uint64_t), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, 32, h->stream);
    s = cuda_check(h, e, "gz_create allocation");
    if (s == GZ_OK) s = ingest_setup(h);
    // allocations are stream-ordered: complete them before the handle is
    // used from any other stream
    if (s == GZ_OK) s = cuda_check(h, cudaStreamSynchronize(h->stream), "gz_create sync");
    if (s != GZ_OK) {
        g_create_err = h->err;
        gz_destroy(h);
        return s;
    }
    *out = h;
    return GZ_OK;
}

gz_status gz_destroy(gz_handle* h) {
    if (!h) return GZ_EINVAL;
    if (h->part_stream) cudaStreamSynchronize(h->part_stream);
    if (h->tier_in) cudaStreamSynchronize(h->tier_in);
    if (h->tier_out) cudaStreamSynchronize(h->tier_out);
    cudaStreamSynchronize(h->stream);
    void* ptrs[] = {h->d_sketch, h->d_keys, h->d_counts, h->d_offsets, h->d_cursor, h->d_cursor_hi, h->d_records,
                    h->d_stage, h->d_flags, h->q_label, h->q_parent, h->q_count, h->q_off,
                    h->q_cursor, h->q_members, h->q_roots, h->q_target, h->q_slot, h->q_final,
                    h->q_F, h->q_F2,
                    h->q_M, h->q_M2, h->q_flag, h->q_pos, h->q_forest, h->q_ctr, h->q_res,
                    h->q_acc, h->q_trace, h->d_stats, h->d_scan_tmp, h->d_tile_node, h->d_decode,
                    h->d_slot[0], h->d_slot[1], h->d_slot[2], h->d_gather,
                    h->pset1.counts, h->pset1.offsets, h->pset1.cursor, h->pset1.cursor_hi, h->pset1.records,
                    h->pset1.tile_node, h->pset1.flags};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, h->stream);
    delete[] h->h_ctr;
    if (h->h_labels) cudaFreeHost(h->h_labels);
    if (h->q_graph_exec) cudaGraphExecDestroy(h->q_graph_exec);
    if (h->q_graph) cudaGraphDestroy(h->q_graph);
    for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_copied[b]) cudaEventDestroy(h->ev_copied[b]);
        if (h->ev_free[b]) cudaEventDestroy(h->ev_free[b]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (int b = 0; b < gz_handle::kTierSlots; ++b) {
        if (h->ev_tin[b]) cudaEventDestroy(h->ev_tin[b]);
        if (h->ev_tdone[b]) cudaEventDestroy(h->ev_tdone[b]);
        if (h->ev_tout[b]) cudaEventDestroy(h->ev_tout[b]);
    }
    for (int b = 0; b < 2; ++b) {
        if (h->ev_part[b]) cudaEventDestroy(h->ev_part[b]);
        if (h->ev_upd[b]) cudaEventDestroy(h->ev_upd[b]);
    }
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->part_stream) cudaStreamDestroy(h->part_stream);
    if (h->tier_in) cudaStreamDestroy(h->tier_in);
    if (h->tier_out) cudaStreamDestroy(h->tier_out);
    cudaStreamSynchronize(h->stream);
    if (h->h_sketch) cudaFreeHost(h->h_sketch);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (int i = 0; i < 4; ++i)
        if (h->cap_ev[i]) cudaEventDestroy(h->cap_ev[i]);
    delete h;
    return GZ_OK;
}

gz_status gz_set_stream(gz_handle* h, void* stream) {
    if (!h) return GZ_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return GZ_OK;
}

// Updates in slice i of a call with host input: 2^chunk_log2 / 16, then
// 2^chunk_log2 / 4, then 2^chunk_log2 (never below 256).
static uint64_t host_slice(const gz_handle* h, size_t i) {
    const uint64_t c = h->chunk;
    const uint64_t s = i == 0 ? c / 16 : i == 1 ? c / 4 : c;
    return std::max<uint64_t>(s, std::min<uint64_t>(c, 256));
}

static gz_status host_path_setup(gz_handle* h) {
    if (h->d_stage) return GZ_OK;
    cudaError_t e = cudaMallocAsync(&h->d_stage, (size_t)4 * h->chunk * 4, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // the copy stream uses it
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[b], cudaEventDisableTiming);
    }
    return cuda_check(h, e, "host staging setup");
}

gz_status gz_edge_update(gz_handle* h, const uint32_t* u, const uint32_t* v, size_t n, int on_device) {
    if (!h) return GZ_EINVAL;
    if (n == 0) return GZ_OK;
    if (!u || !v) return set_error(h, GZ_EINVAL, "null update arrays");
    if (on_device) {
        // the inputs are ready once the handle stream's earlier work is done
        input_stream(h, nullptr);
        for (size_t off = 0; off < n; off += h->chunk) {
            const uint64_t m = std::min<uint64_t>(h->chunk, n - off);
            gz_status s = ingest_batch(h, u + off, v + off, m);
            if (s != GZ_OK) return s;
        }
        return GZ_OK;
    }
    // Host input: two staging buffers; the copy of slice i+1 (copy stream)
    // overlaps the processing of slice i.  The first slices are short (a
    // sixteenth, then a quarter of a chunk), so the first copy, which nothing
    // hides, is short too.
    gz_status s = host_path_setup(h);
    if (s != GZ_OK) return s;
    cudaError_t e = cudaSuccess;
    size_t i = 0;
    for (size_t off = 0, m = 0; off < n; off += m, ++i) {
        m = std::min<uint64_t>(host_slice(h, i), n - off);
        const int b = (int)(i & 1);
        uint32_t* su = h->d_stage + (size_t)b * 2 * h->chunk;
        uint32_t* sv = su + h->chunk;
        // buffer b is free once the partition of its previous chunk (this call
        // or an earlier one) has read it; an event never recorded is complete
        e = cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(su, u + off, m * 4, cudaMemcpyHostToDevice, h->copy_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sv, v + off, m * 4, cudaMemcpyHostToDevice, h->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_copied[b], h->copy_stream);
        if (e != cudaSuccess) return cuda_check(h, e, "update copy");
        cudaStream_t in = input_stream(h, h->ev_copied[b]);
        s = ingest_batch(h, su, sv, m);
        if (s != GZ_OK) return s;
        e = cudaEventRecord(h->ev_free[b], in);
        if (e != cudaSuccess) return cuda_check(h, e, "update event");
    }
    // the caller may reuse its host buffers once every copy has landed
    e = cudaStreamSynchronize(h->copy_stream);
    if (e != cudaSuccess) return cuda_check(h, e, "update sync");
    return GZ_OK;
}

gz_status gz_edge_update_idx(gz_handle* h, const uint64_t* idx, size_t n, int on_device) {
    if (!h) return GZ_EINVAL;
    if (n == 0) return GZ_OK;
    if (!idx) return set_error(h, GZ_EINVAL, "null index array");
    cudaError_t e = cudaSuccess;
    if (!h->d_decode) {
        e = cudaMallocAsync(&h->d_decode, (size_t)2 * h->chunk * 4, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // the partition stream uses it
        if (e != cudaSuccess) return cuda_check(h, e, "decode buffer");
    }
    uint32_t* du = h->d_decode;
    uint32_t* dv = du + h->chunk;
    gz_status s;
    // the decode runs where the partition reads its output (the partition
    // stream of a pipelined handle), so one decode buffer serves every chunk
    if (on_device) {
        cudaStream_t in = input_stream(h, nullptr);
        for (size_t off = 0; off < n; off += h->chunk) {
            const uint64_t m = std::min<uint64_t>(h->chunk, n - off);
            if ((s = decode_idx(h, idx + off, m, du, dv, in)) != GZ_OK) return s;
            if ((s = ingest_batch(h, du, dv, m)) != GZ_OK) return s;
        }
        return GZ_OK;
    }
    // Host input: the packed slice (8 bytes per update) fills one staging
    // buffer; it is free again once decoded.  Slices ramp up as above.
    if ((s = host_path_setup(h)) != GZ_OK) return s;
    size_t i = 0;
    for (size_t off = 0, m = 0; off < n; off += m, ++i) {
        m = std::min<uint64_t>(host_slice(h, i), n - off);
        const int b = (int)(i & 1);
        uint64_t* sb = reinterpret_cast<uint64_t*>(h->d_stage + (size_t)b * 2 * h->chunk);
        e = cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sb, idx + off, m * 8, cudaMemcpyHostToDevice, h->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_copied[b], h->copy_stream);
        if (e != cudaSuccess) return cuda_check(h, e, "update copy");
        cudaStream_t in = input_stream(h, h->ev_copied[b]);
        if ((s = decode_idx(h, sb, m, du, dv, in)) != GZ_OK) return s;
        e = cudaEventRecord(h->ev_free[b], in);
        if (e != cudaSuccess) return cuda_check(h, e, "update event");
        if ((s = ingest_batch(h, du, dv, m)) != GZ_OK) return s;
    }
    e = cudaStreamSynchronize(h->copy_stream);
    if (e != cudaSuccess) return cuda_check(h, e, "update sync");
    return GZ_OK;
}

// flags[2]: sticky "a batch was discarded"; flags[3]: sticky "a bounded wait
// of the update kernel ran out" (its tile may be partly applied)
static gz_status check_rejected(gz_handle* h) {
    // every partition is followed by its update on the handle's stream, so
    // once that stream is done both buffer sets' flags are final
    uint32_t f[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(f, h->d_flags + 2, 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && h->pset1.flags)
        e = cudaMemcpyAsync(f + 2, h->pset1.flags + 2, 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "sync");
    if (f[0] || f[1]) cudaMemsetAsync(h->d_flags + 2, 0, 8, h->stream);
    if (f[2] || f[3]) cudaMemsetAsync(h->pset1.flags + 2, 0, 8, h->stream);
    if (f[1] || f[3])
        return set_error(h, GZ_ETIMEOUT, "a bounded wait in the update kernel ran out; the sketches are incomplete");
    if (f[0] || f[2])
        return set_error(h, GZ_EINVAL, "an update batch held a self loop or a vertex id >= V and was discarded");
    return GZ_OK;
}

gz_status gz_sync(gz_handle* h) {
    if (!h) return GZ_EINVAL;
    return check_rejected(h);
}

gz_status gz_reset(gz_handle* h) {
    if (!h) return GZ_EINVAL;
    cudaError_t e = cudaSuccess;
    if (h->res_nodes) e = cudaMemsetAsync(h->d_sketch, 0, (size_t)h->res_nodes * h->node_bytes, h->stream);
    if (h->tiered) {  // host shards: wait for every queued update and copy-out, then clear
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->tier_out);
        if (e == cudaSuccess) std::memset(h->h_sketch, 0, (size_t)(h->V - h->res_nodes) * h->node_bytes);
    }
    return cuda_check(h, e, "reset");
}

gz_status gz_connected_components(gz_handle* h, uint32_t* labels, uint32_t* n_cc, gz_query_stats* st) {
    if (!h) return GZ_EINVAL;
    gz_status s = check_rejected(h);
    if (s != GZ_OK) return s;
    return boruvka(h, false, labels, nullptr, nullptr, n_cc, st);
}

gz_status gz_list_spanning_forest(gz_handle* h, uint32_t* uv, size_t* n_edges, uint32_t* labels,
                                  gz_query_stats* st) {
    if (!h) return GZ_EINVAL;
    gz_status s = check_rejected(h);
    if (s != GZ_OK) return s;
    uint32_t ncc = 0;
    return boruvka(h, true, labels, uv, n_edges, &ncc, st);
}

gz_status gz_enable_trace(gz_handle* h, int enable) {
    if (!h) return GZ_EINVAL;
    h->trace = enable != 0;
    h->trace_valid = false;
    return GZ_OK;
}

gz_status gz_query_trace(gz_handle* h, int64_t* out) {
    if (!h || !out) return GZ_EINVAL;
    if (!h->trace_valid || !h->q_trace) return set_error(h, GZ_EINVAL, "no traced query to report");
    cudaError_t e = cudaMemcpy(out, h->q_trace, (size_t)h->K * h->V * sizeof(int64_t), cudaMemcpyDeviceToHost);
    return cuda_check(h, e, "trace copy");
}

gz_status gz_export_sketch(gz_handle* h, uint32_t node_lo, uint32_t node_hi, uint64_t* alpha,
                           uint32_t* gamma, int on_device) {
    if (!h || !alpha || !gamma) return GZ_EINVAL;
    if (node_lo > node_hi || node_hi > h->V) return set_error(h, GZ_EINVAL, "node range out of bounds");
    gz_status s = check_rejected(h);
    if (s != GZ_OK) return s;
    const size_t n = (size_t)(node_hi - node_lo) * h->ncol * h->R;
    if (n == 0) return GZ_OK;
    uint64_t* da = alpha;
    uint32_t* dg = gamma;
    if (!on_device) {
        cudaError_t e = cudaMallocAsync(&da, n * 8, h->stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&dg, n * 4, h->stream);
        if (e != cudaSuccess) return cuda_check(h, e, "export scratch");
    }
    s = export_nested(h, node_lo, node_hi, da, dg);
    cudaError_t e = cudaSuccess;
    if (s == GZ_OK && !on_device) {
        e = cudaMemcpyAsync(alpha, da, n * 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gamma, dg, n * 4, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (!on_device) {
        cudaFreeAsync(da, h->stream);
        cudaFreeAsync(dg, h->stream);
    }
    if (s != GZ_OK) return s;
    return cuda_check(h, e, "export");
}

gz_status gz_profile_enable(gz_handle* h, int enable) {
    if (!h) return GZ_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_stats, 0, 2 * sizeof(uint64_t), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "profile enable");
    h->prof = enable != 0;
    h->ev_used = 0;
    h->prof_batches = h->prof_updates = h->launches = 0;
    return GZ_OK;
}

gz_status gz_profile_read(gz_handle* h, gz_profile* out) {
    if (!h || !out) return GZ_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "profile sync");
    double part = 0, upd = 0;
    if (h->part_stream) {
        e = cudaStreamSynchronize(h->part_stream);
        if (e != cudaSuccess) return cuda_check(h, e, "profile sync");
    }
    for (size_t i = 0; i + 3 < h->ev_used; i += 4) {
        float a = 0, b = 0;
        e = cudaEventElapsedTime(&a, h->ev_pool[i], h->ev_pool[i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, h->ev_pool[i + 2], h->ev_pool[i + 3]);
        if (e != cudaSuccess) return cuda_check(h, e, "cudaEventElapsedTime");
        part += a;
        upd += b;
    }
    uint64_t st[2] = {0, 0};
    e = cudaMemcpy(st, h->d_stats, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(h, e, "profile stats");
    out->batches = h->prof_batches;
    out->updates = h->prof_updates;
    out->partition_ms = part;
    out->update_ms = upd;
    out->rows_flushed = st[0];
    out->deep_updates = st[1];
    out->kernel_launches = h->launches;
    return GZ_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version, V, K, R;
    uint64_t seed, node_bytes;
    uint8_t reserved[24];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
const char kMagic[8] = {'G', 'Z', 'B', '3', 'C', 'K', 'P', '1'};
// 3: sketches of the piece hashes (32-bit multiply-add-shift pieces on the
// endpoint pair); version 2 held another hash family
constexpr uint32_t kCkptVersion = 3;
}  // namespace

gz_status gz_checkpoint_bytes(gz_handle* h, size_t* bytes) {
    if (!h || !bytes) return GZ_EINVAL;
    *bytes = sizeof(CkptHeader) + (size_t)h->V * h->node_bytes;
    return GZ_OK;
}

gz_status gz_checkpoint(gz_handle* h, void* buf, size_t size) {
    if (!h || !buf) return GZ_EINVAL;
    const size_t need = sizeof(CkptHeader) + (size_t)h->V * h->node_bytes;
    if (size < need) return set_error(h, GZ_EINVAL, "checkpoint buffer too small");
    gz_status s = check_rejected(h);
    if (s != GZ_OK) return s;
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = kCkptVersion;
    hd.V = h->V;
    hd.K = h->K;
    hd.R = h->R;
    hd.seed = h->seed;
    hd.node_bytes = h->node_bytes;
    std::memcpy(buf, &hd, sizeof(hd));
    uint8_t* dst = static_cast<uint8_t*>(buf) + sizeof(hd);
    const size_t res = (size_t)h->res_nodes * h->node_bytes;
    cudaError_t e = res ? cudaMemcpyAsync(dst, h->d_sketch, res, cudaMemcpyDeviceToHost, h->stream) : cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (h->tiered && e == cudaSuccess) {
        e = cudaStreamSynchronize(h->tier_out);
        if (e == cudaSuccess) std::memcpy(dst + res, h->h_sketch, need - sizeof(hd) - res);
    }
    return cuda_check(h, e, "checkpoint copy");
}

gz_status gz_restore(const void* buf, size_t size, const gz_config* cfg, void* stream, gz_handle** out) {
    if (!buf || !out || size < sizeof(CkptHeader)) return GZ_EINVAL;
    *out = nullptr;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    uint32_t K, R;
    if (std::memcmp(hd.magic, kMagic, 8) != 0 || hd.version != kCkptVersion || !gz::geometry(hd.V, &K, &R) ||
        K != hd.K || R != hd.R || hd.node_bytes != (uint64_t)K * 84u * R ||
        size < sizeof(hd) + (size_t)hd.V * hd.node_bytes)
        return GZ_EINVAL;
    gz_handle* h = nullptr;
    gz_status s = gz_create(hd.V, hd.seed, cfg, stream, &h);
    if (s != GZ_OK) return s;
    const uint8_t* src = static_cast<const uint8_t*>(buf) + sizeof(hd);
    const size_t res = (size_t)h->res_nodes * hd.node_bytes;
    cudaError_t e = res ? cudaMemcpyAsync(h->d_sketch, src, res, cudaMemcpyHostToDevice, h->stream) : cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (h->tiered && e == cudaSuccess) std::memcpy(h->h_sketch, src + res, (size_t)hd.V * hd.node_bytes - res);
    if (e != cudaSuccess) {
        gz_destroy(h);
        return GZ_ECUDA;
    }
    *out = h;
    return GZ_OK;
}

gz_status gz_info(gz_handle* h, uint32_t* V, uint32_t* K, uint32_t* R, size_t* node_bytes,
                  void** sketch_device) {
    if (!h) return GZ_EINVAL;
    if (V) *V = h->V;
    if (K) *K = h->K;
    if (R) *R = h->R;
    if (node_bytes) *node_bytes = h->node_bytes;
    // a tiered handle's device array holds only the resident nodes
    if (sketch_device) *sketch_device = h->tiered ? nullptr : h->d_sketch;
    return GZ_OK;
}

}  // extern "C"
