// gz_ingest.cu -- stream ingestion: CubeSketch updates of every node touched by a
// batch of edge updates (Fig. cube_code update_sketch; Section 5.1 "Sketch
// updates").
//
// The paper buffers updates per node (leaf-only gutters, Section 5.1) and lets
// Graph Workers apply one node's batch at a time.  Here one batch of updates is
// partitioned by endpoint on the device (histogram, exclusive scan, scatter: each
// update lands in the segment of both endpoints with the other endpoint as the
// record), and a persistent kernel walks fixed-size tiles of the partitioned
// records, staged by a producer warp per CTA.  For every node segment in its
// tile a CTA keeps a zeroed delta sketch of the first `Rs` exact-depth rows in
// shared memory (one thread per CubeSketch column, so no two threads share a
// bucket; the default mode still applies each XOR with one shared-memory
// atomic, a single-instruction read-modify-write), applies the segment, then
// XORs the touched rows into the node's sketch in global memory with
// red.global.xor --
// the "apply to an empty sketch, then add" step of Section 5.1 (linearity), which
// also lets two CTAs share one heavy node whose segment spans tiles.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "gz_handle.cuh"
#include "gz_internal.cuh"

namespace gz {

// ------------------------------------------------------------------ partition

// Validation + endpoint histogram.  flags[0] = this batch is invalid,
// flags[2] = sticky "some batch was invalid" (reported by gz_sync).
__global__ void k_validate_count(const uint32_t* __restrict__ u, const uint32_t* __restrict__ v,
                                 uint64_t n, uint32_t V, uint32_t* __restrict__ counts,
                                 uint32_t* __restrict__ flags) {
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t a = u[i], b = v[i];
        if (a == b || a >= V || b >= V) {
            bad = true;
            continue;
        }
        if (counts) {
            atomicAdd(&counts[a], 1u);
            atomicAdd(&counts[b], 1u);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        atomicOr(&flags[0], 1u);
        atomicOr(&flags[2], 1u);
    }
}

// Exclusive scan of n counts: out[i] = sum in[0..i), out[n] = total; out2
// (optional) receives out[0..n) as well (the scatter cursors).  Two launches:
// per-tile sums, then every tile adds the sums of the tiles before it and
// scans its own 1024 entries (coalesced loads, warp-shuffle scan).
constexpr uint32_t kScanTile = 1024;

__device__ __forceinline__ uint32_t block_scan_excl_1024(uint32_t x, uint32_t* sh, uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t s = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= (uint32_t)o) s += y;
    }
    if (lane == 31) sh[w] = s;
    __syncthreads();
    if (w == 0) {
        uint32_t t = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= (uint32_t)o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const uint32_t r = s - x + (w ? sh[w - 1] : 0);
    *total = sh[31];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanTile) k_scan_sums(const uint32_t* __restrict__ in, uint32_t n,
                                                        uint32_t* __restrict__ tile_sum) {
    __shared__ uint32_t sh[32];
    const uint32_t i = blockIdx.x * kScanTile + threadIdx.x;
    uint32_t x = i < n ? in[i] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) tile_sum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanTile) k_scan_tiles(const uint32_t* __restrict__ in, uint32_t n,
                                                         const uint32_t* __restrict__ tile_sum,
                                                         uint32_t* __restrict__ out,
                                                         uint32_t* __restrict__ out2) {
    __shared__ uint32_t sh[32];
    __shared__ uint32_t s_base;
    // prefix of the tile sums before this tile
    uint32_t acc = 0;
    for (uint32_t t = threadIdx.x; t < blockIdx.x; t += kScanTile) acc += tile_sum[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) s_base = t;
    }
    __syncthreads();
    const uint32_t base = s_base;
    __syncthreads();
    const uint32_t i = blockIdx.x * kScanTile + threadIdx.x;
    const uint32_t x = i < n ? in[i] : 0;
    uint32_t total;
    const uint32_t e = base + block_scan_excl_1024(x, sh, &total);
    if (i < n) {
        out[i] = e;
        if (out2) out2[i] = e;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = base + total;
}

// tile sums live after the n+1 outputs' worth of scratch the caller provides
void launch_scan(const uint32_t* in, uint32_t* out, uint32_t* out2, uint32_t n, cudaStream_t s,
                 uint32_t* tile_scratch) {
    const uint32_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return;
    }
    k_scan_sums<<<tiles, kScanTile, 0, s>>>(in, n, tile_scratch);
    k_scan_tiles<<<tiles, kScanTile, 0, s>>>(in, n, tile_scratch, out, out2);
}

// Scatter: record of update (a,b) in a's segment is b and in b's segment is a.
__global__ void k_scatter(const uint32_t* __restrict__ u, const uint32_t* __restrict__ v, uint64_t n,
                          uint32_t* __restrict__ cursor, uint32_t* __restrict__ records,
                          const uint32_t* __restrict__ flags) {
    if (flags[0]) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t a = u[i], b = v[i];
        records[atomicAdd(&cursor[a], 1u)] = b;
        records[atomicAdd(&cursor[b], 1u)] = a;
    }
}

// ------------------------------------------------------------------ batched update

struct BatchedArgs {
    SketchView s;
    Keys keys;
    const uint32_t* offsets;  // V+1
    const uint32_t* records;
    const uint32_t* tile_node;  // first node of every record tile
    const uint32_t* flags;
    uint32_t* work;  // tile counter
    unsigned long long* stats;  // [0] rows flushed, [1] deep column updates
    uint32_t V, K, R, ncol, Rs, tile, small_seg;
};

// The windowed variant (sketches beyond HBM) applies only the records of nodes
// [flags[4], flags[5]); node x's sketch is at s.base + x * s.node_bytes, so for
// a window whose sketches start at address a the host passes
// s.base = a - node_lo * node_bytes (computed as an integer; only window nodes
// are addressed).  The window lives in device memory, not in BatchedArgs, so
// that the all-HBM kernel's arguments stay as small as they are.
__global__ void k_set_window(uint32_t* flags, uint32_t node_lo, uint32_t node_hi) {
    flags[1] = 0;  // tile counter
    flags[4] = node_lo;
    flags[5] = node_hi;
}

// tile_node[t] = the node x with offsets[x] <= t*tile < offsets[x+1]: node x
// owns the tiles whose first record falls inside its segment.
__global__ void k_tile_nodes(const uint32_t* __restrict__ offsets, uint32_t V, uint32_t tile,
                             const uint32_t* __restrict__ flags, uint32_t* __restrict__ tile_node) {
    if (flags[0]) return;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        const uint32_t lo = offsets[x], hi = offsets[x + 1];
        for (uint32_t t = (lo + tile - 1) / tile; t * tile < hi; ++t) tile_node[t] = x;
    }
}

// The two hashes of one column on 32-bit words, with the key parts held in
// registers.  They compute exactly `depth_word` and `checksum` of
// gz_internal.cuh.
struct ColKey {
    uint32_t a_lo, a_hi;
    uint64_t b;
    uint32_t c_pre;  // t ^ (t >> 16) part of the checksum key: lo32(c) ^ (lo32(c) >> 16)
};

__device__ __forceinline__ ColKey make_colkey(uint64_t a, uint64_t b, uint64_t c) {
    ColKey k;
    k.a_lo = (uint32_t)a;
    k.a_hi = (uint32_t)(a >> 32);
    k.b = b;
    k.c_pre = (uint32_t)c ^ ((uint32_t)c >> 16);
    return k;
}

// high word of a*idx + b (mod 2^64); kWide: idx may reach 2^32 (V > 2^16)
template <bool kWide>
__device__ __forceinline__ uint32_t depth_hi(const ColKey& k, uint32_t x_lo, uint32_t x_hi) {
    const uint64_t p = (uint64_t)k.a_lo * x_lo + k.b;
    uint32_t hi = (uint32_t)(p >> 32) + k.a_hi * x_lo;
    if (kWide) hi += k.a_lo * x_hi;
    return hi;
}

// Per-record half of the checksum's first step: with f = fold32(idx) and
// t = f ^ lo32(c), t ^ (t >> 16) = (f ^ (f >> 16)) ^ c_pre, so the record's
// part is staged once and each column adds its key with one XOR.
__device__ __forceinline__ uint32_t fold_pre(uint64_t idx) {
    const uint32_t f = fold32(idx);
    return f ^ (f >> 16);
}

// stored checksum gamma' of a staged record (= checksum_pre(c, idx))
__device__ __forceinline__ uint32_t checksum_w(const ColKey& k, uint32_t fpre) {
    uint32_t h = fpre ^ k.c_pre;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    return h;
}

// mbarrier handover between the producer warp and the column warps.  Every
// wait is bounded: after kTryLimit polls (each may suspend the thread for up
// to about a microsecond) the waiter records a timeout in flags[3] and leaves
// the kernel, which the host reports as GZ_ETIMEOUT.
constexpr uint32_t kTryLimit = 1u << 22;
constexpr uint32_t kRing = 3;             // staged tiles in flight per CTA
constexpr uint32_t kDone = 0xffffffffu;   // ring entry: no tiles left

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar))
                 : "memory");
}
// true once the phase of the given parity has completed; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kTryLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// One CTA = CP + 32 threads, CP = 32*ceil(7K/32).  Thread c < CP owns CubeSketch
// column c = 7k + j (one "Graph Worker" per column; no two threads write one
// bucket, so each thread also flushes its own delta rows).  The last warp is
// the producer: it claims tiles (equal record counts) from an atomic counter,
// turns each record of a tile into its edge index and checksum part, and
// stages the tile in a kRing-slot shared-memory ring; the column warps consume
// the ring in order.  full[b] (one arrival, the producer) says slot b holds a
// staged tile; empty[b] (one arrival per column warp) says every column warp
// has finished with it.  So no CTA-wide barrier sits in the loop: a column
// warp starts on the next tile as soon as it is done with the current one.
// Dynamic shared memory:
//   delta rows: one 96-word block per (warp of columns, row d < Rs), warp w's
//               block of row d at word (w*Rs + d)*96.  kMode 1 (32-bit
//               shared atomics): alpha lo, alpha hi, gamma' as three 32-word
//               planes at +0, +32, +64; kMode 0 (load-xor-store): alpha as 32
//               u64 (+0), gamma' (+64).  A warp's 32 lanes hit 32 distinct
//               banks whatever rows they update, and the words of a column
//               update share one address register.
//   ring        [kRing] slots of one staged tile: uint2 {idx_lo, fold_pre}
//               per record, record r of the tile at entry r; kWide: then u32
//               idx_hi per record (12 bytes a record in all).  A consumer
//               reads four records' words with 16-byte loads.
template <int kMode, bool kWide, bool kWin>
__global__ void __launch_bounds__(1024) k_batched(BatchedArgs p) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ uint64_t full_bar[kRing], empty_bar[kRing];
    __shared__ uint32_t s_tile[kRing], s_node[kRing];
    if (p.flags[0]) return;
    const uint32_t CP = blockDim.x - 32, c = threadIdx.x;
    const uint32_t Rs = p.Rs, R = p.R, RC = Rs * CP, T = p.tile;
    constexpr uint32_t kStageWords = kWide ? 3u : 2u;
    uint32_t* sw = reinterpret_cast<uint32_t*>(smem);  // delta blocks, 3*RC words
    uint32_t* ring = sw + 3 * RC;  // 16-byte aligned: RC is a multiple of 32, T of 4
    uint32_t* timeout = const_cast<uint32_t*>(p.flags) + 3;
    for (uint32_t i = c; i < 3 * RC; i += blockDim.x) sw[i] = 0;
    if (c == 0) {
        for (uint32_t b = 0; b < kRing; ++b) {
            mbar_init(&full_bar[b], 1);
            mbar_init(&empty_bar[b], CP / 32);
        }
    }
    __syncthreads();
    const uint32_t total = p.offsets[p.V];
    // the window's records [rec_lo, rec_hi) lie in tiles t_lo .. t_lo+ntiles-1
    // (kWin false: the whole chunk, with the bounds known at compile time)
    uint32_t rec_lo = 0, rec_hi = total, t_lo = 0, ntiles = (total + T - 1) / T;
    uint32_t node_lo = 0;
    if constexpr (kWin) {
        node_lo = p.flags[4];
        rec_lo = p.offsets[node_lo];
        rec_hi = p.offsets[p.flags[5]];
        t_lo = rec_lo / T;
        ntiles = rec_hi > rec_lo ? (rec_hi + T - 1) / T - t_lo : 0u;
    }

    if (c >= CP) {
        // ---------------------------------------------------------- producer
        const uint32_t lane = c - CP;
        for (uint32_t it = 0;; ++it) {
            const uint32_t b = it % kRing, ph = (it / kRing) & 1u;
            if (!mbar_wait(&empty_bar[b], ph ^ 1u)) {  // a fresh slot passes at once
                if (lane == 0) atomicOr(timeout, 1u);
                return;
            }
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(p.work, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= ntiles) {
                if (lane == 0) {
                    s_tile[b] = kDone;
                    mbar_arrive(&full_bar[b]);
                }
                return;
            }
            const uint32_t tile_lo = (t_lo + t) * T;
            uint32_t lo, hi;
            if constexpr (kWin) {
                lo = max(tile_lo, rec_lo);
                hi = min(tile_lo + T, rec_hi);
            } else {
                lo = tile_lo;
                hi = min(tile_lo + T, total);
            }
            uint32_t x = kWin ? max(p.tile_node[t_lo + t], node_lo) : p.tile_node[t];
            if (lane == 0) {
                s_tile[b] = t;
                s_node[b] = x;
            }
            uint32_t* slot = ring + b * kStageWords * T;
            // lane takes records lo + 32q + lane: coalesced loads, conflict-free
            // stores, and a per-lane walk over the tile's node segments
            uint32_t xend = p.offsets[x + 1];
            for (uint32_t g = lo; g < hi; g += 256) {
                uint32_t r[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t i = g + 32 * q + lane;
                    r[q] = i < hi ? __ldcs(p.records + i) : 0u;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t i = g + 32 * q + lane;
                    if (i < hi) {
                        while (xend <= i) xend = p.offsets[++x + 1];
                        const uint64_t idx = edge_index(x, r[q], p.V);
                        reinterpret_cast<uint2*>(slot)[i - tile_lo] = make_uint2((uint32_t)idx, fold_pre(idx));
                        if (kWide) slot[2 * T + i - tile_lo] = (uint32_t)(idx >> 32);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[b]);
        }
    }

    // ------------------------------------------------------------ column warps
    const bool active = c < p.ncol;
    const uint32_t k = c / GZ_COLS, j = c - k * GZ_COLS;
    // word of (row 0, column c) in plane 0; row d adds d*96
    uint32_t* cw = sw + (c >> 5) * Rs * 96 + (c & 31);
    uint64_t* ca = reinterpret_cast<uint64_t*>(sw + (c >> 5) * Rs * 96) + (c & 31);  // kMode 0 alpha
    ColKey key{};
    if (active) key = make_colkey(p.keys.a[c], p.keys.b[c], p.keys.c[c]);
    // first node whose records can hold an edge index of 2^32 or more
    const uint32_t xn = kWide ? (uint32_t)((0x100000000ull - p.V) / p.V) + 1u : 0u;
    unsigned long long n_rows = 0, n_deep = 0;
    for (uint32_t it = 0;; ++it) {
        const uint32_t b = it % kRing, ph = (it / kRing) & 1u;
        if (!mbar_wait(&full_bar[b], ph)) {
            atomicOr(timeout, 1u);
            break;
        }
        const uint32_t t = s_tile[b];
        if (t == kDone) break;
        uint32_t x = s_node[b];
        const uint32_t tile_lo = (t_lo + t) * T;
        uint32_t hi, pos;
        if constexpr (kWin) {
            hi = min(tile_lo + T, rec_hi);
            pos = max(tile_lo, rec_lo);
        } else {
            hi = min(tile_lo + T, total);
            pos = tile_lo;
        }
        const uint32_t* slot = ring + b * kStageWords * T;
        while (pos < hi) {
            const uint32_t seg_end = min(p.offsets[x + 1], hi);
            const uint32_t nseg = seg_end - pos;
            if (nseg > 0 && active) {
                const uint32_t sb = pos - tile_lo;  // the segment's first ring entry
                const uint2* stage2 = reinterpret_cast<const uint2*>(slot) + sb;
                const uint32_t* stageh = slot + 2 * T + sb;  // kWide: idx_hi
                if (nseg < p.small_seg) {
                    // short segment: straight to global memory
                    const uint64_t ka = p.keys.a[c], kb = p.keys.b[c];
                    for (uint32_t i = 0; i < nseg; ++i) {
                        const uint2 q = stage2[i];
                        const uint64_t idx = kWide ? ((uint64_t)stageh[i] << 32 | q.x) : q.x;
                        const uint32_t fp = q.y;
                        const uint32_t d = exact_depth(depth_word(ka, kb, idx), R);
                        atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, k, d, j)),
                                  (unsigned long long)idx);
                        atomicXor(p.s.gamma(x, k, d, j), checksum_w(key, fp));
                    }
                } else {
                    // node x's edge indices are at most x*V + V-1, below 2^32
                    // when x < xn: its records then take the 32-bit code
                    auto batched = [&](auto wide_tag) {
                        constexpr bool W = decltype(wide_tag)::value;
                        uint32_t md = 0;  // deepest delta row this column touched
                        // one column update staged in shared memory (d < Rs)
                        auto put = [&](uint32_t d, uint32_t xlo, uint32_t xhi, uint32_t g) {
                            if (kMode == 1) {
                                uint32_t* w = cw + d * 96;
                                atomicXor(w, xlo);
                                if (W) atomicXor(w + 32, xhi);
                                atomicXor(w + 64, g);
                            } else {
                                ca[d * 48] ^= ((uint64_t)xhi << 32) | xlo;
                                cw[d * 96 + 64] ^= g;
                            }
                        };
                        // a column update whose exact depth is Rs or more goes to HBM
                        auto deep = [&](uint32_t xlo, uint32_t xhi, uint32_t g) {
                            ++n_deep;
                            const uint64_t idx = ((uint64_t)xhi << 32) | xlo;
                            const uint32_t dd = exact_depth(depth_word(p.keys.a[c], p.keys.b[c], idx), R);
                            atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, k, dd, j)),
                                      (unsigned long long)idx);
                            atomicXor(p.s.gamma(x, k, dd, j), g);
                        };
                        // one staged record
                        auto one = [&](uint32_t i) {
                            const uint2 q = stage2[i];
                            const uint32_t xlo = q.x, xhi = W ? stageh[i] : 0u, fp = q.y;
                            const uint32_t d = __clz(depth_hi<W>(key, xlo, xhi));
                            const uint32_t g = checksum_w(key, fp);
                            if (d < Rs) {
                                put(d, xlo, xhi, g);
                                md = max(md, d);
                            } else {
                                deep(xlo, xhi, g);
                            }
                        };
                        uint32_t i = 0;
                        // the loop reads 16-byte words (two records' uint2, four
                        // records' idx_hi), so it starts on an aligned ring entry
                        constexpr uint32_t kAlign = W ? 4u : 2u;
                        const uint32_t peel = min(nseg, (kAlign - (sb & (kAlign - 1))) & (kAlign - 1));
                        for (; i < peel; ++i) one(i);
                        // four records at a time in straight-line code, so the
                        // four hash chains interleave; one rare branch for deep rows
                        for (; i + 4 <= nseg; i += 4) {
                            uint32_t xlo[4], xhi[4], fp[4];
                            const uint4 q0 = *reinterpret_cast<const uint4*>(stage2 + i);
                            const uint4 q1 = *reinterpret_cast<const uint4*>(stage2 + i + 2);
                            xlo[0] = q0.x;
                            fp[0] = q0.y;
                            xlo[1] = q0.z;
                            fp[1] = q0.w;
                            xlo[2] = q1.x;
                            fp[2] = q1.y;
                            xlo[3] = q1.z;
                            fp[3] = q1.w;
                            if (W) {
                                const uint4 h = *reinterpret_cast<const uint4*>(stageh + i);
                                xhi[0] = h.x;
                                xhi[1] = h.y;
                                xhi[2] = h.z;
                                xhi[3] = h.w;
                            } else {
    #pragma unroll
                                for (int r = 0; r < 4; ++r) xhi[r] = 0;
                            }
                            uint32_t d[4], g[4];
    #pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                d[r] = __clz(depth_hi<W>(key, xlo[r], xhi[r]));
                                g[r] = checksum_w(key, fp[r]);
                            }
                            const uint32_t dmax = max(max(d[0], d[1]), max(d[2], d[3]));
                            if (dmax < Rs) {
    #pragma unroll
                                for (int r = 0; r < 4; ++r) put(d[r], xlo[r], xhi[r], g[r]);
                                md = max(md, dmax);
                            } else {
    #pragma unroll
                                for (int r = 0; r < 4; ++r) {
                                    if (d[r] < Rs) {
                                        put(d[r], xlo[r], xhi[r], g[r]);
                                        md = max(md, d[r]);
                                    } else {
                                        deep(xlo[r], xhi[r], g[r]);
                                    }
                                }
                            }
                        }
                        for (; i < nseg; ++i) one(i);
                        // flush this column's touched rows into the node sketch
                        for (uint32_t row = 0; row <= md; ++row) {
                            uint32_t* w = cw + row * 96;
                            // (32-bit code: the alpha-hi word was never written, so it is 0)
                            const uint64_t a = kMode == 1 ? (W ? (((uint64_t)w[32] << 32) | w[0]) : w[0])
                                                          : ca[row * 48];
                            const uint32_t g = w[64];
                            if (a | g) {
                                atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, k, row, j)),
                                          (unsigned long long)a);
                                atomicXor(p.s.gamma(x, k, row, j), g);
                                if (kMode == 1) {
                                    w[0] = 0;
                                    if (W) w[32] = 0;
                                } else {
                                    ca[row * 48] = 0;
                                }
                                w[64] = 0;
                                ++n_rows;
                            }
                        }
                    };
                    if constexpr (kWide) {
                        if (x >= xn) batched(std::true_type{});
                        else batched(std::false_type{});
                    } else {
                        batched(std::false_type{});
                    }
                }
            }
            pos = seg_end;
            ++x;
        }
        __syncwarp();  // the whole warp is done with slot b
        if ((c & 31) == 0) mbar_arrive(&empty_bar[b]);
    }
    if (n_rows) atomicAdd(&p.stats[0], n_rows);
    if (n_deep) atomicAdd(&p.stats[1], n_deep);
}

using BatchedFn = void (*)(BatchedArgs);

// mode: 0 load-xor-store, 1 32-bit shared atomics; win: a node window (sketches beyond HBM)
static BatchedFn batched_fn(uint32_t mode, bool wide, bool win = false) {
    if (win) {
        if (mode == 1) return wide ? k_batched<1, true, true> : k_batched<1, false, true>;
        return wide ? k_batched<0, true, true> : k_batched<0, false, true>;
    }
    if (mode == 1) return wide ? k_batched<1, true, false> : k_batched<1, false, false>;
    return wide ? k_batched<0, true, false> : k_batched<0, false, false>;
}

// Raise the dynamic shared-memory cap of every batched-kernel variant to the
// device's opt-in maximum, once per device (idempotent; safe to call from any
// thread: a server creates handles from several worker threads).
static cudaError_t set_smem_cap_once(int device);
static cudaError_t set_smem_cap(int device) {
    constexpr int kDevices = 64;
    static std::atomic<bool> done[kDevices];
    static std::mutex mu;
    if (device >= 0 && device < kDevices && done[device].load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu);
    if (device >= 0 && device < kDevices && done[device].load(std::memory_order_relaxed)) return cudaSuccess;
    const cudaError_t e = set_smem_cap_once(device);
    if (e == cudaSuccess && device >= 0 && device < kDevices) done[device].store(true, std::memory_order_release);
    return e;
}

static cudaError_t set_smem_cap_once(int device) {
    int cap = 0;
    cudaError_t e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    for (int mode = 0; mode < 2 && e == cudaSuccess; ++mode)
        for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
            const void* fn = (const void*)batched_fn(mode, (v & 1) != 0, (v & 2) != 0);
            cudaFuncAttributes fa;
            e = cudaFuncGetAttributes(&fa, fn);  // the kernel's static shared memory counts too
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         cap - (int)fa.sharedSizeBytes);
        }
    return e;
}

// ------------------------------------------------------------------ plain update

// The per-update baseline: thread c of a CTA handles column c of every update
// the CTA visits and XORs straight into both endpoints' sketches with global
// atomics (no buffering; the unbuffered configuration of Section 6.5).
__global__ void __launch_bounds__(1024) k_plain(const uint32_t* __restrict__ u,
                                                const uint32_t* __restrict__ v, uint64_t n,
                                                SketchView s, Keys keys, uint32_t V, uint32_t R,
                                                uint32_t ncol, const uint32_t* __restrict__ flags) {
    if (flags[0]) return;
    const uint32_t c = threadIdx.x;
    if (c >= ncol) return;
    const uint32_t k = c / GZ_COLS, j = c - k * GZ_COLS;
    const uint64_t ka = keys.a[c], kb = keys.b[c], kc = keys.c[c];
    for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t a = u[i], b = v[i];
        const uint64_t idx = edge_index(a, b, V);
        const uint32_t d = exact_depth(depth_word(ka, kb, idx), R);
        const uint32_t g = checksum_pre(kc, idx);
        atomicXor(reinterpret_cast<unsigned long long*>(s.alpha(a, k, d, j)), (unsigned long long)idx);
        atomicXor(s.gamma(a, k, d, j), g);
        atomicXor(reinterpret_cast<unsigned long long*>(s.alpha(b, k, d, j)), (unsigned long long)idx);
        atomicXor(s.gamma(b, k, d, j), g);
    }
}

// ------------------------------------------------------------------ export

// Nested rows (Eq. 1-2) of nodes [lo, hi): thread per (node, k, j), suffix XOR
// from row R-1 down to row 0, gamma' -> gamma on the way out.  Output layout
// [node][k][j][row].
__global__ void k_export(SketchView s, uint32_t lo, uint32_t hi, uint32_t K, uint32_t R,
                         uint64_t* __restrict__ oa, uint32_t* __restrict__ og) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t ncols = (uint64_t)K * GZ_COLS;
    if (gid >= (uint64_t)(hi - lo) * ncols) return;
    const uint32_t node = lo + (uint32_t)(gid / ncols);
    const uint32_t col = (uint32_t)(gid % ncols);
    const uint32_t k = col / GZ_COLS, j = col - k * GZ_COLS;
    uint64_t acc = 0;
    uint32_t accg = 0;
    for (int row = (int)R - 1; row >= 0; --row) {
        acc ^= *s.alpha(node, k, row, j);
        accg ^= *s.gamma(node, k, row, j);
        oa[gid * R + row] = acc;
        og[gid * R + row] = gamma_final(accg);
    }
}

// ------------------------------------------------------------------ host side

static SketchView view_of(const gz_handle* h) {
    SketchView s;
    s.base = h->d_sketch;
    s.node_bytes = h->node_bytes;
    s.per_k_bytes = h->per_k_bytes;
    s.gamma_off = 56u * h->R;
    return s;
}

static Keys keys_of(const gz_handle* h) {
    Keys k;
    k.a = h->d_keys;
    k.b = h->d_keys + h->ncol;
    k.c = h->d_keys + 2 * (size_t)h->ncol;
    return k;
}

gz_status ingest_setup(gz_handle* h) {
    h->block = (h->ncol + 31) / 32 * 32;
    if (h->block + 32 > 1024) return set_error(h, GZ_EINVAL, "too many CubeSketch columns for one CTA");
    uint32_t rs = h->cfg.smem_rows ? h->cfg.smem_rows : 12;
    rs = std::min<uint32_t>(rs, 32);
    rs = std::min<uint32_t>(rs, h->R);
    h->smem_rows = rs;
    h->tile = h->cfg.tile_records ? h->cfg.tile_records : 512;
    h->small_seg = h->cfg.small_segment ? h->cfg.small_segment : 4;
    const bool wide = (uint64_t)h->V * h->V > (1ull << 32);
    if (h->tile % 4 != 0) return set_error(h, GZ_EINVAL, "tile_records must be a multiple of 4");
    h->batched_smem = (size_t)rs * h->block * 12 + (size_t)h->tile * kRing * (wide ? 12 : 8);
    if (h->cfg.smem_mode > 2) return set_error(h, GZ_EINVAL, "smem_mode must be 0, 1 or 2");
    h->delta_mode = h->cfg.smem_mode == 2 ? 0u : 1u;  // kernel mode: 1 shared atomics, 0 load-xor-store
    const void* fn = (const void*)batched_fn(h->delta_mode, wide);
    // The dynamic shared-memory cap is one process-wide setting per kernel, so
    // every caller sets the same value (the device's opt-in maximum); a
    // per-handle value would let handles of different sizes break each other.
    cudaError_t e = set_smem_cap(h->device);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaFuncSetAttribute(k_batched)");
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, (int)h->block + 32, h->batched_smem);
    if (e != cudaSuccess) return cuda_check(h, e, "occupancy(k_batched)");
    if (nb < 1) return set_error(h, GZ_EINVAL, "batched kernel does not fit on an SM");
    uint32_t per_sm = h->cfg.ctas_per_sm ? std::min<uint32_t>(h->cfg.ctas_per_sm, nb) : nb;
    h->batched_grid = per_sm * h->sm_count;
    if (h->cfg.kernel == GZ_KERNEL_BATCHED) {
        e = cudaMallocAsync(&h->d_tile_node, (size_t)(2 * h->chunk / h->tile + 2) * sizeof(uint32_t),
                            h->stream);
        if (e != cudaSuccess) return cuda_check(h, e, "tile table allocation");
    }
    return GZ_OK;
}

static BatchedArgs batched_args(gz_handle* h) {
    BatchedArgs a;
    a.s = view_of(h);
    a.keys = keys_of(h);
    a.offsets = h->d_offsets;
    a.records = h->d_records;
    a.tile_node = h->d_tile_node;
    a.flags = h->d_flags;
    a.work = h->d_flags + 1;
    a.V = h->V;
    a.K = h->K;
    a.R = h->R;
    a.ncol = h->ncol;
    a.Rs = h->smem_rows;
    a.tile = h->tile;
    a.small_seg = h->small_seg;
    a.stats = reinterpret_cast<unsigned long long*>(h->d_stats);
    return a;
}

// Sketches beyond HBM: the batched update of one partitioned chunk, window by
// window.  Resident nodes are updated in place; host shard i is copied into
// device slot i mod kTierSlots on tier_in, updated on st, and copied back on
// tier_out.
// A slot's copy-in waits for its previous copy-out, and tier_out runs its
// copies in issue order, so a shard's copy-in also follows its copy-out of the
// previous chunk.  The tile counter is cleared before every launch.
static void enqueue_tiered_updates(gz_handle* h, cudaStream_t st) {
    const bool wide = (uint64_t)h->V * h->V > (1ull << 32);
    const BatchedFn fn = batched_fn(h->delta_mode, wide, true);
    BatchedArgs a = batched_args(h);
    if (h->res_nodes) {
        k_set_window<<<1, 1, 0, st>>>(h->d_flags, 0, h->res_nodes);
        fn<<<h->batched_grid, h->block + 32, h->batched_smem, st>>>(a);
    }
    uint32_t i = 0;
    for (uint32_t lo = h->res_nodes; lo < h->V; lo += h->shard_nodes, ++i) {
        const uint32_t hi = std::min<uint32_t>(h->V, lo + h->shard_nodes), b = i % gz_handle::kTierSlots;
        const size_t bytes = (size_t)(hi - lo) * h->node_bytes;
        uint8_t* host = h->h_sketch + (size_t)(lo - h->res_nodes) * h->node_bytes;
        cudaStreamWaitEvent(h->tier_in, h->ev_tout[b], 0);  // an event never recorded is complete
        cudaMemcpyAsync(h->d_slot[b], host, bytes, cudaMemcpyHostToDevice, h->tier_in);
        cudaEventRecord(h->ev_tin[b], h->tier_in);
        cudaStreamWaitEvent(st, h->ev_tin[b], 0);
        k_set_window<<<1, 1, 0, st>>>(h->d_flags, lo, hi);
        // node lo lives at the slot's start: base = slot - lo * node_bytes, as an integer
        a.s.base = reinterpret_cast<uint8_t*>(reinterpret_cast<uintptr_t>(h->d_slot[b]) -
                                              (uintptr_t)lo * h->node_bytes);
        fn<<<h->batched_grid, h->block + 32, h->batched_smem, st>>>(a);
        cudaEventRecord(h->ev_tdone[b], st);
        cudaStreamWaitEvent(h->tier_out, h->ev_tdone[b], 0);
        cudaMemcpyAsync(host, h->d_slot[b], bytes, cudaMemcpyDeviceToHost, h->tier_out);
        cudaEventRecord(h->ev_tout[b], h->tier_out);
    }
    // beyond the one batched launch counted per chunk: the other windows and the window setters
    h->launches += 2 * (i + (h->res_nodes ? 1 : 0)) - 1;
}

gz_status tier_settle(gz_handle* h) {
    if (!h->tiered) return GZ_OK;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < gz_handle::kTierSlots && e == cudaSuccess; ++b)
        e = cudaStreamWaitEvent(h->stream, h->ev_tout[b], 0);
    return cuda_check(h, e, "tier settle");
}

gz_status tier_gather_nodes(gz_handle* h, uint32_t lo, uint32_t hi, uint8_t* dst) {
    gz_status s = tier_settle(h);
    if (s != GZ_OK) return s;
    cudaError_t e = cudaSuccess;
    const uint32_t r_hi = std::min(hi, h->res_nodes);
    if (lo < r_hi)
        e = cudaMemcpyAsync(dst, h->d_sketch + (size_t)lo * h->node_bytes, (size_t)(r_hi - lo) * h->node_bytes,
                            cudaMemcpyDeviceToDevice, h->stream);
    const uint32_t h_lo = std::max(lo, h->res_nodes);
    if (e == cudaSuccess && h_lo < hi)
        e = cudaMemcpyAsync(dst + (size_t)(h_lo - lo) * h->node_bytes,
                            h->h_sketch + (size_t)(h_lo - h->res_nodes) * h->node_bytes,
                            (size_t)(hi - h_lo) * h->node_bytes, cudaMemcpyHostToDevice, h->stream);
    return cuda_check(h, e, "tier gather");
}

// The batched pipeline of one chunk on stream st: validation + histogram,
// scan, scatter, tile table, persistent update.  ev (may hold nulls) are
// recorded before the partition, before the update and after it.
static void enqueue_batched(gz_handle* h, const uint32_t* d_u, const uint32_t* d_v, uint64_t n,
                            uint32_t grid, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, cudaEvent_t ev2,
                            bool capturing = false) {
    // under stream capture only an "external" record becomes an event-record node
    auto record = [&](cudaEvent_t ev) {
        if (capturing) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
        else cudaEventRecord(ev, st);
    };
    if (ev0) record(ev0);
    cudaMemsetAsync(h->d_flags, 0, 2 * sizeof(uint32_t), st);  // batch flag + tile counter
    cudaMemsetAsync(h->d_counts, 0, (size_t)(h->V + 1) * sizeof(uint32_t), st);
    k_validate_count<<<grid, 256, 0, st>>>(d_u, d_v, n, h->V, h->d_counts, h->d_flags);
    launch_scan(h->d_counts, h->d_offsets, h->d_cursor, h->V, st, h->d_scan_tmp);
    k_scatter<<<grid, 256, 0, st>>>(d_u, d_v, n, h->d_cursor, h->d_records, h->d_flags);
    k_tile_nodes<<<(h->V + 255) / 256, 256, 0, st>>>(h->d_offsets, h->V, h->tile, h->d_flags, h->d_tile_node);
    if (ev1) record(ev1);
    const bool wide = (uint64_t)h->V * h->V > (1ull << 32);
    if (!h->tiered) {
        batched_fn(h->delta_mode, wide)<<<h->batched_grid, h->block + 32, h->batched_smem, st>>>(
            batched_args(h));
    } else {
        enqueue_tiered_updates(h, st);
    }
    if (ev2) record(ev2);
}

// Capture the pipeline once on a private stream (thread-local capture mode,
// so other threads' CUDA calls are unaffected); the input pointers and count
// are rewritten per launch in the validation and scatter nodes, the three
// event-record nodes are re-pointed when profiling.
static gz_status capture_graph(gz_handle* h) {
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->cap_ev[i]);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (cap) cudaStreamDestroy(cap);
        return cuda_check(h, e, "graph capture begin");
    }
    enqueue_batched(h, h->d_records, h->d_records, 0, (uint32_t)h->sm_count * 8, cap, h->cap_ev[0], h->cap_ev[1],
                    h->cap_ev[2], true);
    e = cudaStreamEndCapture(cap, &h->graph);
    cudaStreamDestroy(cap);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph_exec, h->graph, 0);
    if (e != cudaSuccess) return cuda_check(h, e, "graph capture");
    size_t nn = 0;
    e = cudaGraphGetNodes(h->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess) e = cudaGraphGetNodes(h->graph, nodes.data(), &nn);
    if (e != cudaSuccess) return cuda_check(h, e, "graph nodes");
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess) continue;
        if (ty == cudaGraphNodeTypeKernel) {
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
            if (kp.func == (void*)k_validate_count) h->node_validate = nd;
            if (kp.func == (void*)k_scatter) h->node_scatter = nd;
        } else if (ty == cudaGraphNodeTypeEventRecord) {
            cudaEvent_t ev;
            if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
            for (int i = 0; i < 3; ++i)
                if (ev == h->cap_ev[i]) h->node_ev[i] = nd;
        }
    }
    if (!h->node_validate || !h->node_scatter || !h->node_ev[0] || !h->node_ev[1] || !h->node_ev[2])
        return set_error(h, GZ_ECUDA, "captured ingest graph lacks an expected node");
    h->graph_ready = true;
    return GZ_OK;
}

static gz_status launch_graph(gz_handle* h, const uint32_t* d_u, const uint32_t* d_v, uint64_t n) {
    if (!h->graph_ready) {
        gz_status s = capture_graph(h);
        if (s != GZ_OK) return s;
    }
    cudaKernelNodeParams kp;
    cudaError_t e = cudaGraphKernelNodeGetParams(h->node_validate, &kp);
    const uint32_t V = h->V;
    uint32_t* counts = h->d_counts;
    uint32_t* flags = h->d_flags;
    void* va[] = {(void*)&d_u, (void*)&d_v, (void*)&n, (void*)&V, (void*)&counts, (void*)&flags};
    kp.kernelParams = va;
    kp.extra = nullptr;
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(h->graph_exec, h->node_validate, &kp);
    uint32_t* cursor = h->d_cursor;
    uint32_t* records = h->d_records;
    void* sa[] = {(void*)&d_u, (void*)&d_v, (void*)&n, (void*)&cursor, (void*)&records, (void*)&flags};
    cudaKernelNodeParams kq;
    if (e == cudaSuccess) e = cudaGraphKernelNodeGetParams(h->node_scatter, &kq);
    kq.kernelParams = sa;
    kq.extra = nullptr;
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(h->graph_exec, h->node_scatter, &kq);
    if (e != cudaSuccess) return cuda_check(h, e, "graph parameters");
    for (int i = 0; i < 3; ++i) {
        cudaEvent_t ev = h->cap_ev[i];
        if (h->prof) {
            if (h->ev_used == h->ev_pool.size()) {
                cudaEvent_t nev;
                e = cudaEventCreate(&nev);
                if (e != cudaSuccess) return cuda_check(h, e, "cudaEventCreate");
                h->ev_pool.push_back(nev);
            }
            ev = h->ev_pool[h->ev_used++];
        }
        e = cudaGraphExecEventRecordNodeSetEvent(h->graph_exec, h->node_ev[i], ev);
        if (e != cudaSuccess) return cuda_check(h, e, "graph event");
    }
    return cuda_check(h, cudaGraphLaunch(h->graph_exec, h->stream), "cudaGraphLaunch");
}

// Packed edge index -> endpoints: idx = min*V + max, the coordinate of edge
// {min, max} in the characteristic vector of Section 3.1.  A non-canonical
// index (min >= max, or idx >= V^2) decodes to the self loop (0, 0), which
// the validation of its batch then rejects.
__global__ void k_decode_idx(const uint64_t* __restrict__ idx, uint64_t n, uint32_t V,
                             uint32_t* __restrict__ u, uint32_t* __restrict__ v) {
    const uint64_t VV = (uint64_t)V * V;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = idx[i];
        uint32_t a = 0, b = 0;
        if (x < VV) {
            a = (uint32_t)(x / V);
            b = (uint32_t)(x - (uint64_t)a * V);
            if (a >= b) a = b = 0;
        }
        u[i] = a;
        v[i] = b;
    }
}

gz_status decode_idx(gz_handle* h, const uint64_t* d_idx, uint64_t n, uint32_t* d_u, uint32_t* d_v) {
    if (n == 0) return GZ_OK;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)h->sm_count * 8);
    k_decode_idx<<<grid, 256, 0, h->stream>>>(d_idx, n, h->V, d_u, d_v);
    h->launches += 1;
    return cuda_check(h, cudaGetLastError(), "decode launch");
}

gz_status ingest_batch(gz_handle* h, const uint32_t* d_u, const uint32_t* d_v, uint64_t n) {
    if (n == 0) return GZ_OK;
    cudaStream_t st = h->stream;
    gz_status ps;
    if (h->cfg.kernel == GZ_KERNEL_PLAIN) {
        if ((ps = prof_event(h)) != GZ_OK) return ps;
        cudaError_t e = cudaMemsetAsync(h->d_flags, 0, 2 * sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_check(h, e, "memset flags");
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)h->sm_count * 8);
        k_validate_count<<<grid, 256, 0, st>>>(d_u, d_v, n, h->V, nullptr, h->d_flags);
        if ((ps = prof_event(h)) != GZ_OK) return ps;
        const uint32_t pg = (uint32_t)std::min<uint64_t>(n, (uint64_t)h->sm_count * 16);
        k_plain<<<pg, h->block, 0, st>>>(d_u, d_v, n, view_of(h), keys_of(h), h->V, h->R, h->ncol,
                                         h->d_flags);
        h->launches += 2;
        if ((ps = prof_event(h)) != GZ_OK) return ps;
    } else if (!h->cfg.no_graph && !h->tiered && h->batches_done >= 8) {
        // the captured graph pays off once a handle keeps ingesting
        if ((ps = launch_graph(h, d_u, d_v, n)) != GZ_OK) return ps;
        h->launches += 6;  // validate, 2 scan, scatter, tile table, batched
    } else {
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < 3 && h->prof; ++i) {
            if ((ps = prof_event(h)) != GZ_OK) return ps;
            ev[i] = h->ev_pool[h->ev_used - 1];
        }
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)h->sm_count * 8);
        enqueue_batched(h, d_u, d_v, n, grid, st, ev[0], ev[1], ev[2]);
        h->launches += 6;
    }
    ++h->batches_done;
    if (h->prof) {
        h->prof_batches += 1;
        h->prof_updates += n;
    }
    return cuda_check(h, cudaGetLastError(), "ingest launch");
}

gz_status prof_event(gz_handle* h) {
    if (!h->prof) return GZ_OK;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_check(h, e, "cudaEventCreate");
        h->ev_pool.push_back(ev);
    }
    return cuda_check(h, cudaEventRecord(h->ev_pool[h->ev_used++], h->stream), "cudaEventRecord");
}

gz_status export_nested(gz_handle* h, uint32_t lo, uint32_t hi, uint64_t* d_alpha, uint32_t* d_gamma) {
    const uint64_t threads = (uint64_t)(hi - lo) * h->ncol;
    if (threads == 0) return GZ_OK;
    const uint32_t tpb = 256;
    SketchView v = view_of(h);
    uint8_t* tmp = nullptr;
    if (h->tiered) {  // gather the nodes' full sketches into one device array first
        cudaError_t e = cudaMallocAsync(&tmp, (size_t)(hi - lo) * h->node_bytes, h->stream);
        if (e != cudaSuccess) return cuda_check(h, e, "export gather buffer");
        gz_status s = tier_gather_nodes(h, lo, hi, tmp);
        if (s != GZ_OK) {
            cudaFreeAsync(tmp, h->stream);
            return s;
        }
        v.base = tmp;
        hi -= lo;
        lo = 0;
    }
    k_export<<<(uint32_t)((threads + tpb - 1) / tpb), tpb, 0, h->stream>>>(v, lo, hi, h->K,
                                                                          h->R, d_alpha, d_gamma);
    if (tmp) cudaFreeAsync(tmp, h->stream);
    return cuda_check(h, cudaGetLastError(), "export launch");
}

}  // namespace gz

// ======================================================================
// Allocation-free ingestion entry point (gz_sketch_update_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA stream is
// being captured into a graph (an allocation would break the capture), hosts
// whose device memory is owned by another allocator (a framework pool that
// must see every byte), and latency-bound loops that may not take the
// driver's allocation lock.  For them this variant of the partition + batched
// update runs entirely in a fixed scratch array that lives in this file's
// static device memory: every GPU that loads the library holds it (about
// 10 MB) until the process exits.  The caller passes the sketch memory and
// the update arrays; nothing is allocated or freed.
// ======================================================================

#include <mutex>

namespace gz {
namespace noalloc {

constexpr uint32_t kMaxV = GZ_NOALLOC_MAX_V;
constexpr uint64_t kMaxUpdates = GZ_NOALLOC_MAX_UPDATES;
constexpr uint32_t kMaxCols = 7u * 30u;  // K(2^17) = 30 CubeSketches per node
// layout in 32-bit words; every region starts on a 256-byte boundary
constexpr size_t up64(size_t w) { return (w + 63) / 64 * 64; }
constexpr size_t kKeys = 0;                                         // 3 x kMaxCols u64
constexpr size_t kStats = up64(kKeys + 2 * 3 * kMaxCols);           // 2 u64
constexpr size_t kFlags = kStats + 4;                               // 4 u32
constexpr size_t kCounts = up64(kFlags + 4);                        // kMaxV + 1
constexpr size_t kOffsets = up64(kCounts + kMaxV + 1);              // kMaxV + 1
constexpr size_t kCursor = up64(kOffsets + kMaxV + 1);              // kMaxV + 1
constexpr size_t kTiles = up64(kCursor + kMaxV + 1);                // scan tile sums
constexpr size_t kRecords = up64(kTiles + (kMaxV + 1) / 1024 + 2);  // 2 x kMaxUpdates
constexpr uint32_t kTile = 1024;                                    // records per work tile
constexpr size_t kTileNode = up64(kRecords + 2 * kMaxUpdates);       // first node of every tile
constexpr size_t kWords = kTileNode + 2 * kMaxUpdates / kTile + 2;
static_assert(kRecords % 4 == 0 && kFlags == kStats + 4, "scratch layout");

static __device__ __align__(256) uint32_t g_scratch[kWords];

constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static uint32_t* g_ptr[kMaxDevices];
static int g_sms[kMaxDevices];

// Per-column hash keys from the seed (the same SplitMix64 schedule as
// gz_create): a = SM(seed, 3col) | 1, b = SM(seed, 3col+1), c = SM(seed, 3col+2).
__global__ void k_keys(uint64_t seed, uint32_t ncol, uint64_t* a, uint64_t* b, uint64_t* c) {
    const uint32_t col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    uint64_t out[3];
    for (int w = 0; w < 3; ++w) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (3ull * col + w + 1);
        z ^= z >> 30;
        z *= 0xBF58476D1CE4E5B9ull;
        z ^= z >> 27;
        z *= 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[w] = z;
    }
    a[col] = out[0] | 1ull;
    b[col] = out[1];
    c[col] = out[2];
}

// 1: the batch was discarded; 2: a bounded wait of the update kernel ran out
__global__ void k_status(const uint32_t* flags, uint32_t* status) {
    *status = flags[0] ? 1u : (flags[3] ? 2u : 0u);
}

// Once per device, with that device current: the device address of the
// scratch array (its name is only a host-side stand-in in host code).
static gz_status setup(int dev, uint32_t** ptr, int* sms) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return GZ_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GZ_ECUDA;
        if (set_smem_cap(dev) != cudaSuccess) return GZ_ECUDA;
        g_sms[dev] = n;
        g_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *ptr = g_ptr[dev];
    *sms = g_sms[dev];
    return GZ_OK;
}

}  // namespace noalloc
}  // namespace gz

extern "C" gz_status gz_sketch_update_noalloc(void* sketch, uint32_t V, uint64_t seed, const uint32_t* u,
                                              const uint32_t* v, size_t n, uint32_t* status, void* stream) {
    using namespace gz;
    using namespace gz::noalloc;
    if (!sketch || V < 2 || V > kMaxV || n > kMaxUpdates || (n && (!u || !v))) return GZ_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GZ_ECUDA;
    uint32_t* base = nullptr;
    int sms = 0;
    gz_status s = setup(dev, &base, &sms);
    if (s != GZ_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    uint32_t L = 0;
    while ((1ull << L) < V) ++L;
    uint32_t K = 0;
    {
        unsigned __int128 lhs = 1, rhs = V;
        while (lhs < rhs) {
            lhs *= 3;
            rhs *= 2;
            ++K;
        }
    }
    const uint32_t R = 2 * L, ncol = 7 * K;
    const uint32_t block = (ncol + 31) / 32 * 32;
    const uint32_t Rs = std::min<uint32_t>(12, R), tile = kTile;
    const bool wide = (uint64_t)V * V > (1ull << 32);

    uint64_t* keys = reinterpret_cast<uint64_t*>(base + kKeys);
    uint32_t* flags = base + kFlags;
    uint32_t* counts = base + kCounts;
    // flags (batch, work counter, sticky) and stats start at zero on every call
    if (cudaMemsetAsync(base + kStats, 0, 8 * sizeof(uint32_t), st) != cudaSuccess) return GZ_ECUDA;
    if (cudaMemsetAsync(counts, 0, (size_t)(V + 1) * sizeof(uint32_t), st) != cudaSuccess) return GZ_ECUDA;
    k_keys<<<(ncol + 127) / 128, 128, 0, st>>>(seed, ncol, keys, keys + kMaxCols, keys + 2 * kMaxCols);
    if (n) {
        const uint32_t tpb = 256;
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + tpb - 1) / tpb, (uint64_t)sms * 8);
        k_validate_count<<<grid, tpb, 0, st>>>(u, v, n, V, counts, flags);
        launch_scan(counts, base + kOffsets, base + kCursor, V, st, base + kTiles);
        k_scatter<<<grid, tpb, 0, st>>>(u, v, n, base + kCursor, base + kRecords, flags);
        k_tile_nodes<<<(V + 255) / 256, 256, 0, st>>>(base + kOffsets, V, kTile, flags, base + kTileNode);
        BatchedArgs a;
        a.s.base = static_cast<uint8_t*>(sketch);
        a.s.per_k_bytes = 84u * R;
        a.s.node_bytes = (uint64_t)K * a.s.per_k_bytes;
        a.s.gamma_off = 56u * R;
        a.keys.a = keys;
        a.keys.b = keys + kMaxCols;
        a.keys.c = keys + 2 * kMaxCols;
        a.offsets = base + kOffsets;
        a.records = base + kRecords;
        a.tile_node = base + kTileNode;
        a.flags = flags;
        a.work = flags + 1;
        a.stats = reinterpret_cast<unsigned long long*>(base + kStats);
        a.V = V;
        a.K = K;
        a.R = R;
        a.ncol = ncol;
        a.Rs = Rs;
        a.tile = tile;
        a.small_seg = 4;
        const size_t smem = (size_t)Rs * block * 12 + (size_t)tile * kRing * (wide ? 12 : 8);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_fn(1, wide), (int)block + 32, smem) !=
                cudaSuccess ||
            per_sm < 1)
            return GZ_ECUDA;
        batched_fn(1, wide)<<<per_sm * sms, block + 32, smem, st>>>(a);
    }
    if (status) k_status<<<1, 1, 0, st>>>(flags, status);
    return cudaGetLastError() == cudaSuccess ? GZ_OK : GZ_ECUDA;
}
