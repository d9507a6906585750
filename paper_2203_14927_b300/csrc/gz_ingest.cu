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
// (optional) receives out[0..n) as well and out3 (optional) out[1..n] (the
// front and back cursors of the scatter).  Two launches:
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
                                                         uint32_t* __restrict__ out2,
                                                         uint32_t* __restrict__ out3) {
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
        if (out3) out3[i] = e + x;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = base + total;
}

// tile sums live after the n+1 outputs' worth of scratch the caller provides
void launch_scan(const uint32_t* in, uint32_t* out, uint32_t* out2, uint32_t* out3, uint32_t n, cudaStream_t s,
                 uint32_t* tile_scratch) {
    const uint32_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return;
    }
    k_scan_sums<<<tiles, kScanTile, 0, s>>>(in, n, tile_scratch);
    k_scan_tiles<<<tiles, kScanTile, 0, s>>>(in, n, tile_scratch, out, out2, out3);
}

// Scatter: the record of update (a,b) in a's segment is b and in b's segment
// is a.  Every segment x keeps the records y < x at its front and the records
// y > x at its back (front cursor counting up from offsets[x], back cursor
// down from offsets[x+1]); afterwards front[x] is the split between the two.
// With lo = min(a,b) and hi = max(a,b): lo is a front record of hi, hi a back
// record of lo.
__global__ void k_scatter(const uint32_t* __restrict__ u, const uint32_t* __restrict__ v, uint64_t n,
                          uint32_t* __restrict__ front, uint32_t* __restrict__ back,
                          uint32_t* __restrict__ records, const uint32_t* __restrict__ flags) {
    if (flags[0]) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t a = u[i], b = v[i];
        const uint32_t lo = min(a, b), hi = max(a, b);
        records[atomicAdd(&front[hi], 1u)] = lo;
        records[atomicSub(&back[lo], 1u) - 1u] = hi;
    }
}

// ------------------------------------------------------------------ batched update

struct BatchedArgs {
    SketchView s;
    Keys keys;
    PieceGeo geo;
    const uint32_t* offsets;  // V+1
    const uint32_t* split;    // V: segment x holds records y < x in [offsets[x], split[x])
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

// Slope and offset of the register pieces of one column (the first piece of
// the depth hash h1 and the kM2 pieces of the checksum h2) for one side of one
// node segment.  Inside the segment of node x every record y is an edge with
// one endpoint fixed, so a piece (k0*u + k1*v + k2) mod 2^32 is slope*y + off:
// for y < x (u = y, v = x) slope k0, off k1*x + k2; for y > x (u = x, v = y)
// slope k1, off k0*x + k2.  The keys come from global memory (they stay in
// L1), which keeps them out of the registers of the record loop.
template <int kM2>
struct SideKey {
    uint32_t ds, doff;
    uint32_t cs[kM2], coff[kM2];
};

template <int kM2>
__device__ __forceinline__ SideKey<kM2> side_key(const Keys& keys, uint32_t col, uint32_t x, bool ylo) {
    SideKey<kM2> s;
    const uint32_t d0 = keys.at(0, col), d1 = keys.at(1, col), d2 = keys.at(2, col);
    s.ds = ylo ? d0 : d1;
    s.doff = (ylo ? d1 : d0) * x + d2;
#pragma unroll
    for (int i = 0; i < kM2; ++i) {
        const uint32_t k0 = keys.at(kH2Words + 3 * i, col), k1 = keys.at(kH2Words + 3 * i + 1, col);
        s.cs[i] = ylo ? k0 : k1;
        s.coff[i] = (ylo ? k1 : k0) * x + keys.at(kH2Words + 3 * i + 2, col);
    }
    return s;
}

// h2 of record y: the first 32 bits of the top-p-bit pieces, concatenated
// (kM2 = 2: p = 16, the two top halves joined by one byte permute; kM2 = 3
// covers p in [11, 15]).
template <int kM2>
__device__ __forceinline__ uint32_t side_checksum(const SideKey<kM2>& s, uint32_t y, uint32_t p) {
    const uint32_t g0 = s.cs[0] * y + s.coff[0];
    const uint32_t g1 = s.cs[1] * y + s.coff[1];
    if (kM2 == 2) return __byte_perm(g1, g0, 0x7632);  // (g0 & 0xffff0000) | (g1 >> 16)
    const uint32_t g2 = s.cs[kM2 - 1] * y + s.coff[kM2 - 1];
    // bits [32-p, 32): piece 0; [32-2p, 32-p): piece 1, i.e. g1's top p bits
    // moved down by p; [0, 32-2p): the top 32-2p bits of piece 2 (3p >= 33)
    const uint32_t m0 = 0xffffffffu << (32 - p), m1 = (0xffffffffu >> (32 - p)) << (32 - 2 * p);
    return (g0 & m0) | ((g1 >> p) & m1) | (g2 >> (2 * p));
}

// mbarrier handover between the producer warp and the column warps.  Every
// wait is bounded: after `limit` polls (kTryLimit unless flags[6] sets
// another; each poll may suspend the thread for up to about `hint_ns`, 1000
// unless flags[7] sets another) the waiter records a timeout in flags[3] and
// leaves the kernel, which the host reports as GZ_ETIMEOUT.
constexpr uint32_t kTryLimit = 1u << 22;
constexpr uint32_t kSuspendNs = 1000;
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
// true once the phase of the given parity has completed; false on timeout.
// flags[6] (polls) and flags[7] (suspend hint + 1) override the defaults.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const uint32_t* flags) {
    const uint32_t limit = flags[6] ? flags[6] : kTryLimit;
    const uint32_t hint_ns = flags[7] ? flags[7] - 1u : kSuspendNs;
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// One CTA = CP + 32 threads, CP = 32*ceil(7K/32).  Thread c < CP owns CubeSketch
// column c = 7k + j (one "Graph Worker" per column; no two threads write one
// bucket, so each thread also flushes its own delta rows).  The last warp is
// the producer: it claims tiles (equal record counts) from an atomic counter,
// stages each record of a tile (the other endpoint y and the edge index) in a
// kRing-slot shared-memory ring; the column warps consume the ring in order.
// full[b] (one arrival, the producer) says slot b holds a staged tile;
// empty[b] (one arrival per column warp) says every column warp has finished
// with it.  So no CTA-wide barrier sits in the loop: a column warp starts on
// the next tile as soon as it is done with the current one.
// A node segment is walked side by side (records y < x, then y > x, split by
// the scatter), so the hash offsets of the fixed endpoint x are computed once
// per side and every column update costs one 32-bit multiply-add for the
// depth (the first h1 piece; deeper ones only when its top p bits are all
// zero) and kM2 for the checksum.
// Dynamic shared memory:
//   delta rows: region A, one 64-word block per (warp of columns, row d < Rs)
//               at word (w*Rs + d)*64: alpha lo (+0), gamma (+32); kWide:
//               region H after A, one 32-word block per (warp, row) at word
//               (w*Rs + d)*32: alpha hi.  A warp's 32 lanes hit 32 distinct
//               banks whatever rows they update.  kMode 1 updates them with
//               32-bit shared atomics, kMode 0 with load-xor-store.
//   ring        [kRing] slots of one staged tile: planes of u32 per record,
//               record r of the tile at entry r: y, idx lo, and (kWide) idx
//               hi.  A consumer reads four records' words of a plane with one
//               16-byte load.
// At most kBatchedThreads threads a CTA (7K <= 256 columns: V <= 2^21); the
// bound lets a thread hold 72 registers with three CTAs on an SM.
constexpr uint32_t kBatchedThreads = 288;
template <int kMode, bool kWide, bool kWin, int kM2>
__global__ void __launch_bounds__(kBatchedThreads, 3) k_batched(BatchedArgs p) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ uint64_t full_bar[kRing], empty_bar[kRing];
    __shared__ uint32_t s_tile[kRing], s_node[kRing];
    if (p.flags[0]) return;
    const uint32_t CP = blockDim.x - 32, c = threadIdx.x;
    const uint32_t Rs = p.Rs, R = p.R, RC = Rs * CP, T = p.tile, pw = p.geo.p;
    constexpr uint32_t kStageWords = kWide ? 3u : 2u;
    const uint32_t DA = 2 * RC, DW = kWide ? 3 * RC : DA;  // delta words: region A, A + H
    uint32_t* sw = reinterpret_cast<uint32_t*>(smem);  // delta blocks
    uint32_t* ring = sw + DW;  // 16-byte aligned: RC is a multiple of 32, T of 4
    uint32_t* timeout = const_cast<uint32_t*>(p.flags) + 3;
    for (uint32_t i = c; i < DW; i += blockDim.x) sw[i] = 0;
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
            if (!mbar_wait(&empty_bar[b], ph ^ 1u, p.flags)) {  // a fresh slot passes at once
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
                        slot[i - tile_lo] = r[q];
                        slot[T + i - tile_lo] = (uint32_t)idx;
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
    // this column's word of row 0 in region A (alpha lo; gamma at +32) and,
    // kWide, in region H (alpha hi); row d adds d*64 and d*32 words
    uint32_t* cwA = sw + (c >> 5) * Rs * 64 + (c & 31);
    uint32_t* cwH = sw + DA + (c >> 5) * Rs * 32 + (c & 31);
    // first node whose records can hold an edge index of 2^32 or more
    const uint32_t xn = kWide ? (uint32_t)((0x100000000ull - p.V) / p.V) + 1u : 0u;
    uint32_t n_rows = 0, n_deep = 0;
    for (uint32_t it = 0;; ++it) {
        const uint32_t b = it % kRing, ph = (it / kRing) & 1u;
        if (!mbar_wait(&full_bar[b], ph, p.flags)) {
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
                const uint32_t split = p.split[x];
                if (nseg < p.small_seg) {
                    // short segment: straight to global memory
                    for (uint32_t i = pos - tile_lo; i < seg_end - tile_lo; ++i) {
                        const uint32_t y = slot[i];
                        const uint32_t xlo = slot[T + i], xhi = kWide ? slot[2 * T + i] : 0u;
                        const uint32_t u = min(x, y), v = max(x, y);
                        const uint32_t d = edge_depth(p.keys, p.geo, R, c, u, v);
                        const uint32_t g = edge_checksum(p.keys, p.geo, c, u, v);
                        atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, k, d, j)),
                                  ((unsigned long long)xhi << 32) | xlo);
                        atomicXor(p.s.gamma(x, k, d, j), g);
                    }
                } else {
                    // node x's edge indices are at most x*V + V-1, below 2^32
                    // when x < xn: its records then skip the alpha-hi words
                    auto batched = [&](auto wide_tag) {
                        constexpr bool W = decltype(wide_tag)::value;
                        uint32_t md = 0;  // deepest delta row this column touched
                        // one column update staged in delta row d < Rs
                        auto put = [&](uint32_t d, uint32_t xlo, uint32_t xhi, uint32_t g) {
                            uint32_t* w = cwA + d * 64;
                            if (kMode == 1) {
                                atomicXor(w, xlo);
                                atomicXor(w + 32, g);
                                if (W && xhi) atomicXor(cwH + d * 32, xhi);
                            } else {
                                w[0] ^= xlo;
                                w[32] ^= g;
                                if (W && xhi) cwH[d * 32] ^= xhi;
                            }
                        };
                        // the records [e0, e1) of the ring slot, all on one side of x.
                        // Every column update goes to delta row min(d, Rs-1), so the
                        // record loop holds no code for deep updates; a lane whose
                        // run reached depth Rs (rare) then scans the run again and
                        // moves each deep update from row Rs-1 to its exact row in
                        // HBM.
                        auto run = [&](uint32_t e0, uint32_t e1, bool ylo) {
                            const SideKey<kM2> sk = side_key<kM2>(p.keys, c, x, ylo);
                            const uint32_t* sy = slot;
                            const uint32_t* sl = slot + T;
                            const uint32_t* sh = slot + 2 * T;
                            uint32_t rmax = 0;  // deepest exact depth of the run
                            auto one = [&](uint32_t i) {
                                const uint32_t y = sy[i], xlo = sl[i], xhi = W ? sh[i] : 0u;
                                const uint32_t d = __clz(sk.ds * y + sk.doff);
                                const uint32_t g = side_checksum<kM2>(sk, y, pw);
                                put(min(d, Rs - 1), xlo, xhi, g);
                                rmax = max(rmax, d);
                            };
                            uint32_t i = e0;
                            // the loop reads 16-byte words (four records of a plane),
                            // so it starts on an aligned ring entry
                            const uint32_t peel = min(e1, (e0 + 3u) & ~3u);
                            for (; i < peel; ++i) one(i);
                            // four records at a time in straight-line code, so the
                            // hash chains interleave
                            for (; i + 4 <= e1; i += 4) {
                                const uint4 qy = *reinterpret_cast<const uint4*>(sy + i);
                                const uint4 ql = *reinterpret_cast<const uint4*>(sl + i);
                                uint32_t y[4] = {qy.x, qy.y, qy.z, qy.w};
                                uint32_t xlo[4] = {ql.x, ql.y, ql.z, ql.w};
                                uint32_t xhi[4] = {0u, 0u, 0u, 0u};
                                if (W) {
                                    const uint4 qh = *reinterpret_cast<const uint4*>(sh + i);
                                    xhi[0] = qh.x;
                                    xhi[1] = qh.y;
                                    xhi[2] = qh.z;
                                    xhi[3] = qh.w;
                                }
                                uint32_t d[4], g[4];
#pragma unroll
                                for (int r = 0; r < 4; ++r) {
                                    d[r] = __clz(sk.ds * y[r] + sk.doff);
                                    g[r] = side_checksum<kM2>(sk, y[r], pw);
                                }
#pragma unroll
                                for (int r = 0; r < 4; ++r) put(min(d[r], Rs - 1), xlo[r], xhi[r], g[r]);
                                rmax = max(rmax, max(max(d[0], d[1]), max(d[2], d[3])));
                            }
                            for (; i < e1; ++i) one(i);
                            md = max(md, min(rmax, Rs - 1));
                            if (rmax >= Rs) {
                                // deep updates: depth Rs or more, i.e. a first depth
                                // piece below 2^(32-Rs); take each back out of row
                                // Rs-1 and apply it at its exact row in HBM.  The scan
                                // looks at four records per step (the same aligned
                                // ring words as the record loop).
                                const uint32_t lim = 0xffffffffu >> Rs;
                                auto fix = [&](uint32_t q) {
                                    const uint32_t y = sy[q];
                                    const uint32_t xlo = sl[q], xhi = W ? sh[q] : 0u;
                                    const uint32_t g = side_checksum<kM2>(sk, y, pw);
                                    put(Rs - 1, xlo, xhi, g);
                                    ++n_deep;
                                    const uint32_t dd = edge_depth(p.keys, p.geo, R, c, min(x, y), max(x, y));
                                    atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, k, dd, j)),
                                              ((unsigned long long)xhi << 32) | xlo);
                                    atomicXor(p.s.gamma(x, k, dd, j), g);
                                };
                                uint32_t q = e0;
                                for (; q < peel; ++q)
                                    if (sk.ds * sy[q] + sk.doff <= lim) fix(q);
                                for (; q + 4 <= e1; q += 4) {
                                    const uint4 qy = *reinterpret_cast<const uint4*>(sy + q);
                                    const uint32_t t0 = sk.ds * qy.x + sk.doff, t1 = sk.ds * qy.y + sk.doff;
                                    const uint32_t t2 = sk.ds * qy.z + sk.doff, t3 = sk.ds * qy.w + sk.doff;
                                    if (min(min(t0, t1), min(t2, t3)) > lim) continue;
                                    if (t0 <= lim) fix(q);
                                    if (t1 <= lim) fix(q + 1);
                                    if (t2 <= lim) fix(q + 2);
                                    if (t3 <= lim) fix(q + 3);
                                }
                                for (; q < e1; ++q)
                                    if (sk.ds * sy[q] + sk.doff <= lim) fix(q);
                            }
                        };
                        const uint32_t b0 = pos - tile_lo, b1 = seg_end - tile_lo;
                        const uint32_t bs = min(max(split, pos), seg_end) - tile_lo;
                        if (b0 < bs) run(b0, bs, true);
                        if (bs < b1) run(bs, b1, false);
                        // flush this column's touched rows into the node sketch
                        for (uint32_t row = 0; row <= md; ++row) {
                            uint32_t* w = cwA + row * 64;
                            // (32-bit code: the alpha-hi word was never written, so it is 0)
                            const uint64_t a = W ? (((uint64_t)cwH[row * 32] << 32) | w[0]) : w[0];
                            const uint32_t g = w[32];
                            if (a | g) {
                                atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, k, row, j)),
                                          (unsigned long long)a);
                                atomicXor(p.s.gamma(x, k, row, j), g);
                                w[0] = 0;
                                w[32] = 0;
                                if (W) cwH[row * 32] = 0;
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
    if (n_rows) atomicAdd(&p.stats[0], (unsigned long long)n_rows);
    if (n_deep) atomicAdd(&p.stats[1], (unsigned long long)n_deep);
}

using BatchedFn = void (*)(BatchedArgs);

// mode: 0 load-xor-store, 1 32-bit shared atomics; wide: V^2 > 2^32; win: a
// node window (sketches beyond HBM); m2: checksum pieces (2, of 16 bits, for
// V <= 2^17; 3 for V <= 2^22; the only variants there are)
static BatchedFn batched_fn(uint32_t mode, bool wide, bool win, uint32_t m2) {
    if (!wide) {  // V <= 2^16: p = 16, so m2 = 2
        if (win) return mode == 1 ? k_batched<1, false, true, 2> : k_batched<0, false, true, 2>;
        return mode == 1 ? k_batched<1, false, false, 2> : k_batched<0, false, false, 2>;
    }
    if (m2 == 2) {
        if (win) return mode == 1 ? k_batched<1, true, true, 2> : k_batched<0, true, true, 2>;
        return mode == 1 ? k_batched<1, true, false, 2> : k_batched<0, true, false, 2>;
    }
    if (win) return mode == 1 ? k_batched<1, true, true, 3> : k_batched<0, true, true, 3>;
    return mode == 1 ? k_batched<1, true, false, 3> : k_batched<0, true, false, 3>;
}

// shared memory of the batched kernel: delta blocks (alpha lo + gamma, and
// alpha hi when wide) + staging ring (y, idx lo, and idx hi when wide)
static size_t batched_smem_bytes(bool wide, uint32_t rows, uint32_t block, uint32_t tile) {
    return (size_t)rows * block * (wide ? 12 : 8) + (size_t)tile * kRing * (wide ? 12 : 8);
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
        for (int v = 0; v < 8 && e == cudaSuccess; ++v) {
            const void* fn = (const void*)batched_fn(mode, (v & 1) != 0, (v & 2) != 0, (v & 4) ? 3 : 2);
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
                                                SketchView s, Keys keys, PieceGeo geo, uint32_t V, uint32_t R,
                                                uint32_t ncol, const uint32_t* __restrict__ flags) {
    if (flags[0]) return;
    const uint32_t c = threadIdx.x;
    if (c >= ncol) return;
    const uint32_t k = c / GZ_COLS, j = c - k * GZ_COLS;
    for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t a = u[i], b = v[i];
        const uint64_t idx = edge_index(a, b, V);
        const uint32_t d = edge_depth(keys, geo, R, c, min(a, b), max(a, b));
        const uint32_t g = edge_checksum(keys, geo, c, min(a, b), max(a, b));
        atomicXor(reinterpret_cast<unsigned long long*>(s.alpha(a, k, d, j)), (unsigned long long)idx);
        atomicXor(s.gamma(a, k, d, j), g);
        atomicXor(reinterpret_cast<unsigned long long*>(s.alpha(b, k, d, j)), (unsigned long long)idx);
        atomicXor(s.gamma(b, k, d, j), g);
    }
}

// ------------------------------------------------------------------ export

// Nested rows (Eq. 1-2) of nodes [lo, hi): thread per (node, k, j), suffix XOR
// from row R-1 down to row 0.  Output layout [node][k][j][row].
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
        og[gid * R + row] = accg;
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
    k.w = h->d_keys;
    k.ncol = h->ncol;
    return k;
}

gz_status ingest_setup(gz_handle* h) {
    h->block = (h->ncol + 31) / 32 * 32;
    if (h->block + 32 > 1024) return set_error(h, GZ_EINVAL, "too many CubeSketch columns for one CTA");
    h->geo = piece_geo(h->V);
    // staged rows: the record loop takes the depth from the first h1 piece,
    // which fixes depths below p; the top row R-1 also takes the capped depths
    uint32_t rs = h->cfg.smem_rows ? h->cfg.smem_rows : 16;
    rs = std::min<uint32_t>(rs, 32);
    rs = std::min<uint32_t>(rs, h->R - 1);
    rs = std::min<uint32_t>(rs, h->geo.p);
    h->smem_rows = std::max<uint32_t>(rs, 1);
    h->tile = h->cfg.tile_records ? h->cfg.tile_records : 512;
    h->small_seg = h->cfg.small_segment ? h->cfg.small_segment : 4;
    const bool wide = (uint64_t)h->V * h->V > (1ull << 32);
    if (h->tile % 4 != 0) return set_error(h, GZ_EINVAL, "tile_records must be a multiple of 4");
    if (h->cfg.smem_mode > 2) return set_error(h, GZ_EINVAL, "smem_mode must be 0, 1 or 2");
    if (h->cfg.kernel != GZ_KERNEL_BATCHED) return GZ_OK;
    if (h->geo.m2 > 3 || h->block + 32 > kBatchedThreads)
        return set_error(h, GZ_EINVAL, "the batched kernel supports V <= 2^21 (use the plain kernel)");
    // kernel mode: 1 32-bit shared atomics, 0 load-xor-store
    h->delta_mode = h->cfg.smem_mode == 2 ? 0u : 1u;
    h->batched_smem = batched_smem_bytes(wide, h->smem_rows, h->block, h->tile);
    const void* fn = (const void*)batched_fn(h->delta_mode, wide, false, h->geo.m2);
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
    const size_t tiles = (size_t)(2 * h->chunk / h->tile + 2) * sizeof(uint32_t);
    e = cudaMallocAsync(&h->d_tile_node, tiles, h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "tile table allocation");
    h->pipelined = !h->tiered && !h->cfg.no_pipeline;
    if (!h->pipelined) return GZ_OK;
    // the second partition buffer set, its stream and the hand-over events
    gz_partset& S = h->pset1;
    const size_t vb = (size_t)(h->V + 1) * sizeof(uint32_t);
    e = cudaMallocAsync(&S.counts, vb, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&S.offsets, vb, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&S.cursor, vb, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&S.cursor_hi, vb, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&S.records, (size_t)2 * h->chunk * sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&S.tile_node, tiles, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&S.flags, 32, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.flags, 0, 32, h->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->part_stream, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&h->ev_part[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_upd[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    return cuda_check(h, e, "pipeline setup");
}

gz_partset part_set(const gz_handle* h, int b) {
    if (b == 1) return h->pset1;
    gz_partset S;
    S.counts = h->d_counts;
    S.offsets = h->d_offsets;
    S.cursor = h->d_cursor;
    S.cursor_hi = h->d_cursor_hi;
    S.records = h->d_records;
    S.tile_node = h->d_tile_node;
    S.flags = h->d_flags;
    return S;
}

static BatchedArgs batched_args(gz_handle* h, const gz_partset& S) {
    BatchedArgs a;
    a.s = view_of(h);
    a.keys = keys_of(h);
    a.geo = h->geo;
    a.offsets = S.offsets;
    a.split = S.cursor;
    a.records = S.records;
    a.tile_node = S.tile_node;
    a.flags = S.flags;
    a.work = S.flags + 1;
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
    const BatchedFn fn = batched_fn(h->delta_mode, wide, true, h->geo.m2);
    BatchedArgs a = batched_args(h, part_set(h, 0));
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

// The partition of one chunk into buffer set S on stream st: validation +
// histogram, scan, scatter, tile table.
static void enqueue_partition(gz_handle* h, const gz_partset& S, const uint32_t* d_u, const uint32_t* d_v,
                              uint64_t n, uint32_t grid, cudaStream_t st) {
    cudaMemsetAsync(S.flags, 0, 2 * sizeof(uint32_t), st);  // batch flag + tile counter
    cudaMemsetAsync(S.counts, 0, (size_t)(h->V + 1) * sizeof(uint32_t), st);
    k_validate_count<<<grid, 256, 0, st>>>(d_u, d_v, n, h->V, S.counts, S.flags);
    launch_scan(S.counts, S.offsets, S.cursor, S.cursor_hi, h->V, st, h->d_scan_tmp);
    k_scatter<<<grid, 256, 0, st>>>(d_u, d_v, n, S.cursor, S.cursor_hi, S.records, S.flags);
    k_tile_nodes<<<(h->V + 255) / 256, 256, 0, st>>>(S.offsets, h->V, h->tile, S.flags, S.tile_node);
}

// The sketch update of the chunk partitioned into set S, on stream st.
static void enqueue_update(gz_handle* h, const gz_partset& S, cudaStream_t st) {
    const bool wide = (uint64_t)h->V * h->V > (1ull << 32);
    if (!h->tiered) {
        batched_fn(h->delta_mode, wide, false, h->geo.m2)<<<h->batched_grid, h->block + 32, h->batched_smem, st>>>(
            batched_args(h, S));
    } else {
        enqueue_tiered_updates(h, st);
    }
}

// The batched pipeline of one chunk on stream st, buffer set 0.  ev (may
// hold nulls) are recorded before and after the partition and before and
// after the update.
static void enqueue_batched(gz_handle* h, const uint32_t* d_u, const uint32_t* d_v, uint64_t n,
                            uint32_t grid, cudaStream_t st, const cudaEvent_t* ev, bool capturing = false) {
    // under stream capture only an "external" record becomes an event-record node
    auto record = [&](cudaEvent_t e) {
        if (!e) return;
        if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
    };
    const gz_partset S = part_set(h, 0);
    record(ev[0]);
    enqueue_partition(h, S, d_u, d_v, n, grid, st);
    record(ev[1]);
    record(ev[2]);
    enqueue_update(h, S, st);
    record(ev[3]);
}

// Capture the pipeline once on a private stream (thread-local capture mode,
// so other threads' CUDA calls are unaffected); the input pointers and count
// are rewritten per launch in the validation and scatter nodes, the three
// event-record nodes are re-pointed when profiling.
static gz_status capture_graph(gz_handle* h) {
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->cap_ev[i]);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (cap) cudaStreamDestroy(cap);
        return cuda_check(h, e, "graph capture begin");
    }
    enqueue_batched(h, h->d_records, h->d_records, 0, (uint32_t)h->sm_count * 8, cap, h->cap_ev, true);
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
            for (int i = 0; i < 4; ++i)
                if (ev == h->cap_ev[i]) h->node_ev[i] = nd;
        }
    }
    if (!h->node_validate || !h->node_scatter || !h->node_ev[0] || !h->node_ev[1] || !h->node_ev[2] ||
        !h->node_ev[3])
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
    uint32_t* cursor_hi = h->d_cursor_hi;
    uint32_t* records = h->d_records;
    void* sa[] = {(void*)&d_u, (void*)&d_v, (void*)&n, (void*)&cursor, (void*)&cursor_hi, (void*)&records,
                  (void*)&flags};
    cudaKernelNodeParams kq;
    if (e == cudaSuccess) e = cudaGraphKernelNodeGetParams(h->node_scatter, &kq);
    kq.kernelParams = sa;
    kq.extra = nullptr;
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(h->graph_exec, h->node_scatter, &kq);
    if (e != cudaSuccess) return cuda_check(h, e, "graph parameters");
    for (int i = 0; i < 4; ++i) {
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

gz_status decode_idx(gz_handle* h, const uint64_t* d_idx, uint64_t n, uint32_t* d_u, uint32_t* d_v,
                     cudaStream_t st) {
    if (n == 0) return GZ_OK;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)h->sm_count * 8);
    k_decode_idx<<<grid, 256, 0, st>>>(d_idx, n, h->V, d_u, d_v);
    h->launches += 1;
    return cuda_check(h, cudaGetLastError(), "decode launch");
}

// A profiling event from the handle's pool (recorded by the caller), or null
// when profiling is off.
static cudaEvent_t prof_take(gz_handle* h, gz_status* s) {
    *s = GZ_OK;
    if (!h->prof) return nullptr;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            *s = cuda_check(h, e, "cudaEventCreate");
            return nullptr;
        }
        h->ev_pool.push_back(ev);
    }
    return h->ev_pool[h->ev_used++];
}

cudaStream_t input_stream(gz_handle* h, cudaEvent_t ready) {
    if (!h->pipelined) {
        if (ready) cudaStreamWaitEvent(h->stream, ready, 0);
        return h->stream;
    }
    if (!ready) {
        cudaEventRecord(h->ev_in, h->stream);
        ready = h->ev_in;
    }
    cudaStreamWaitEvent(h->part_stream, ready, 0);
    return h->part_stream;
}

gz_status ingest_batch(gz_handle* h, const uint32_t* d_u, const uint32_t* d_v, uint64_t n) {
    if (n == 0) return GZ_OK;
    cudaStream_t st = h->stream;
    gz_status ps;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4; ++i) {
        ev[i] = prof_take(h, &ps);
        if (ps != GZ_OK) return ps;
    }
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)h->sm_count * 8);
    if (h->cfg.kernel == GZ_KERNEL_PLAIN) {
        if (ev[0]) cudaEventRecord(ev[0], st);
        cudaError_t e = cudaMemsetAsync(h->d_flags, 0, 2 * sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_check(h, e, "memset flags");
        k_validate_count<<<grid, 256, 0, st>>>(d_u, d_v, n, h->V, nullptr, h->d_flags);
        if (ev[1]) cudaEventRecord(ev[1], st);
        if (ev[2]) cudaEventRecord(ev[2], st);
        const uint32_t pg = (uint32_t)std::min<uint64_t>(n, (uint64_t)h->sm_count * 16);
        k_plain<<<pg, h->block, 0, st>>>(d_u, d_v, n, view_of(h), keys_of(h), h->geo, h->V, h->R, h->ncol,
                                         h->d_flags);
        if (ev[3]) cudaEventRecord(ev[3], st);
        h->launches += 2;
    } else if (h->pipelined) {
        // partition into buffer set b on the partition stream (which already
        // waits for the inputs, see input_stream) once set b's previous update
        // is done; the update follows on the handle's stream, so the partition
        // of the next chunk overlaps this update
        const int b = h->pipe_next;
        h->pipe_next ^= 1;
        const gz_partset S = part_set(h, b);
        cudaStream_t P = h->part_stream;
        cudaError_t e = cudaStreamWaitEvent(P, h->ev_upd[b], 0);  // an event never recorded is complete
        if (ev[0]) cudaEventRecord(ev[0], P);
        enqueue_partition(h, S, d_u, d_v, n, grid, P);
        if (ev[1]) cudaEventRecord(ev[1], P);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_part[b], P);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_part[b], 0);
        if (ev[2]) cudaEventRecord(ev[2], st);
        enqueue_update(h, S, st);
        if (ev[3]) cudaEventRecord(ev[3], st);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_upd[b], st);
        if (e != cudaSuccess) return cuda_check(h, e, "pipeline events");
        h->launches += 6;
    } else if (!h->cfg.no_graph && !h->tiered && h->batches_done >= 8) {
        // the captured graph pays off once a handle keeps ingesting
        h->ev_used -= h->prof ? 4 : 0;  // the graph records its own four events
        if ((ps = launch_graph(h, d_u, d_v, n)) != GZ_OK) return ps;
        h->launches += 6;  // validate, 2 scan, scatter, tile table, batched
    } else {
        enqueue_batched(h, d_u, d_v, n, grid, st, ev);
        h->launches += 6;
    }
    ++h->batches_done;
    if (h->prof) {
        h->prof_batches += 1;
        h->prof_updates += n;
    }
    return cuda_check(h, cudaGetLastError(), "ingest launch");
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
// Some callers cannot let a library call cudaMalloc: a host framework whose
// caching allocator owns the device memory and accounts for every byte (an
// allocation behind its back can fail or fragment its pool), and
// latency-bound loops in which cudaMalloc, which may synchronise the device
// and takes a driver lock, is not allowed.  For them this variant of the
// partition + batched update runs entirely in a fixed scratch array that
// lives in this file's static device memory: every GPU that loads the library
// holds it (about 10 MB) until the process exits.  The caller passes the
// sketch memory and the update arrays; nothing is allocated or freed.
// ======================================================================

#include <mutex>

namespace gz {
namespace noalloc {

constexpr uint32_t kMaxV = GZ_NOALLOC_MAX_V;
constexpr uint64_t kMaxUpdates = GZ_NOALLOC_MAX_UPDATES;
constexpr uint32_t kMaxCols = 7u * 30u;  // K(2^17) = 30 CubeSketches per node
// layout in 32-bit words; every region starts on a 256-byte boundary
constexpr size_t up64(size_t w) { return (w + 63) / 64 * 64; }
constexpr size_t kKeys = 0;                                         // kKeyWords x kMaxCols u32
constexpr size_t kStats = up64(kKeys + kKeyWords * kMaxCols);       // 2 u64
constexpr size_t kFlags = kStats + 4;                               // 8 u32 ([6..7]: wait limit)
constexpr size_t kCounts = up64(kFlags + 8);                        // kMaxV + 1
constexpr size_t kOffsets = up64(kCounts + kMaxV + 1);              // kMaxV + 1
constexpr size_t kCursor = up64(kOffsets + kMaxV + 1);              // kMaxV + 1 (front cursors, then splits)
constexpr size_t kCursorHi = up64(kCursor + kMaxV + 1);             // kMaxV + 1 (back cursors)
constexpr size_t kTiles = up64(kCursorHi + kMaxV + 1);              // scan tile sums
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
// gz_create): word w < kKeyWords of column col is lo32(SM(seed, 256 col + w)),
// stored word-major with a row stride of `stride` columns.
__global__ void k_keys(uint64_t seed, uint32_t ncol, uint32_t* keys, uint32_t stride) {
    const uint32_t col = blockIdx.x;
    if (col >= ncol) return;
    for (uint32_t w = threadIdx.x; w < kKeyWords; w += blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * ((uint64_t)kKeyWords * col + w + 1);
        z ^= z >> 30;
        z *= 0xBF58476D1CE4E5B9ull;
        z ^= z >> 27;
        z *= 0x94D049BB133111EBull;
        z ^= z >> 31;
        keys[(size_t)w * stride + col] = (uint32_t)z;
    }
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
    (void)cudaGetLastError();  // an error left by earlier, unrelated work is not this call's
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
    const PieceGeo geo = piece_geo(V);
    const uint32_t Rs = std::min<uint32_t>(std::min<uint32_t>(16, R - 1), geo.p), tile = kTile;
    const bool wide = (uint64_t)V * V > (1ull << 32);
    const size_t smem = batched_smem_bytes(wide, Rs, block, tile);
    const BatchedFn fn = batched_fn(1, wide, false, geo.m2);
    // everything that can fail without queuing work comes first
    int per_sm = 0;
    if (n && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)block + 32, smem) != cudaSuccess ||
              per_sm < 1))
        return GZ_ECUDA;

    uint32_t* keys = base + kKeys;
    uint32_t* flags = base + kFlags;
    uint32_t* counts = base + kCounts;
    // stats and flags[0..3] (batch, work counter, sticky, timeout) start at
    // zero on every call; flags[6..7] keep the wait limit of gz_set_wait_limit
    if (cudaMemsetAsync(base + kStats, 0, 8 * sizeof(uint32_t), st) != cudaSuccess) return GZ_ECUDA;
    if (cudaMemsetAsync(counts, 0, (size_t)(V + 1) * sizeof(uint32_t), st) != cudaSuccess) return GZ_ECUDA;
    k_keys<<<ncol, 256, 0, st>>>(seed, ncol, keys, kMaxCols);
    if (cudaGetLastError() != cudaSuccess) return GZ_ECUDA;
    if (n) {
        const uint32_t tpb = 256;
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + tpb - 1) / tpb, (uint64_t)sms * 8);
        k_validate_count<<<grid, tpb, 0, st>>>(u, v, n, V, counts, flags);
        launch_scan(counts, base + kOffsets, base + kCursor, base + kCursorHi, V, st, base + kTiles);
        k_scatter<<<grid, tpb, 0, st>>>(u, v, n, base + kCursor, base + kCursorHi, base + kRecords, flags);
        k_tile_nodes<<<(V + 255) / 256, 256, 0, st>>>(base + kOffsets, V, kTile, flags, base + kTileNode);
        if (cudaGetLastError() != cudaSuccess) return GZ_ECUDA;  // the sketches are still untouched
        BatchedArgs a;
        a.s.base = static_cast<uint8_t*>(sketch);
        a.s.per_k_bytes = 84u * R;
        a.s.node_bytes = (uint64_t)K * a.s.per_k_bytes;
        a.s.gamma_off = 56u * R;
        a.keys.w = keys;
        a.keys.ncol = kMaxCols;
        a.geo = geo;
        a.offsets = base + kOffsets;
        a.split = base + kCursor;
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
        fn<<<per_sm * sms, block + 32, smem, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) return GZ_ECUDA;
    }
    if (status) {
        k_status<<<1, 1, 0, st>>>(flags, status);
        if (cudaGetLastError() != cudaSuccess) return GZ_ECUDA;
    }
    return GZ_OK;
}

extern "C" gz_status gz_set_wait_limit(gz_handle* h, uint32_t polls, uint32_t suspend_ns) {
    using namespace gz;
    const uint32_t w[2] = {polls, polls ? suspend_ns + 1u : 0u};  // flags[7] = hint + 1; 0 = default
    if (h) {
        cudaError_t e = cudaMemcpyAsync(h->d_flags + 6, w, sizeof(w), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && h->pset1.flags)
            e = cudaMemcpyAsync(h->pset1.flags + 6, w, sizeof(w), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        return cuda_check(h, e, "wait limit");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= noalloc::kMaxDevices) return GZ_ECUDA;
    uint32_t* base = nullptr;
    int sms = 0;
    gz_status s = noalloc::setup(dev, &base, &sms);
    if (s != GZ_OK) return s;
    return cudaMemcpy(base + noalloc::kFlags + 6, w, sizeof(w), cudaMemcpyHostToDevice) == cudaSuccess ? GZ_OK
                                                                                                     : GZ_ECUDA;
}
