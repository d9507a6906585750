// gz_query.cu -- connected components / spanning forest by Boruvka rounds over
// the node sketches (Section 2.2; the three phases of a round in the proof of
// Lemma (CC I/O); list_spanning_forest of Section 5).
//
// Round r:
//   group    nodes by current component (counting sort by label);
//   merge    component sketch = XOR of the members' CubeSketch r, in an
//            accumulator slot per component of two or more members (a
//            block stores a component it holds whole and XORs its part of
//            one that spans blocks in with atomics); the largest component,
//            once it holds more than V/8 nodes, as the XOR of every node
//            outside it (the XOR of all node sketches is zero);
//   sample   nested rows by suffix XOR, then the first bucket in the scan
//            order of Fig. cube_code (columns, then rows ascending) that passes
//            the checksum, decodes to an edge u < v < V and leaves the component;
//   union    lock-free union-find that always hooks the larger root under the
//            smaller (so every root is its set's minimum vertex id);
//   forest   (optional) the sampled edges form a functional graph on the
//            components; a sequential union-find taking them by ascending
//            component id rejects exactly, per cycle, the edge of the cycle's
//            largest component; cycles are found by pointer doubling with a
//            running maximum.
// A round that samples no edge ends the query.  A component whose sketch is
// all zero (EMPTY) is final: later rounds report EMPTY for it without a merge
// or a sample, until a sampled edge touches it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gz_handle.cuh"
#include "gz_internal.cuh"

namespace gz {

// device counters of a query: per round (roots, large components, sampled
// edges, FAIL results), per query (forest edges, components), the round index
// and the loop decision, the statistics of the rounds run so far, and (two
// words from C_GIANT, one u64) the round's largest live component of more
// than V/8 members as (members << 32) | ~id, or 0
enum {
    C_ROOTS = 0, C_BIG = 1, C_EDGES = 2, C_FAILS = 3, C_FOREST = 4, C_NCC = 5, C_ROUND = 6, C_GO = 7,
    C_ROUNDS = 8, C_FLAST = 9, C_FTOT = 10, C_EXH = 11, C_GIANT = 12, C_N = 14
};

__device__ __forceinline__ unsigned long long* giant_word(const uint32_t* ctr) {
    return reinterpret_cast<unsigned long long*>(const_cast<uint32_t*>(ctr) + 12);  // C_GIANT, 8-byte aligned
}

struct QArgs {
    SketchView s;
    Keys keys;     // hash keys (the checksum's pieces)
    PieceGeo geo;
    uint32_t V, K, R, M;  // the round index lives in ctr[C_ROUND]
    uint64_t vinv;        // floor((2^64 - 1) / V): a / V by one high multiply and a correction
    uint32_t *label, *parent, *count, *off, *cursor, *members, *roots, *target;
    uint32_t* slot;     // accumulator slot of a component with more than M members
    uint32_t* final;    // 1 for a component root that sampled EMPTY and that no sampled edge touched since
    uint64_t* acc;      // slots x (21R/2) words, zero between rounds
    int64_t* res;
    int64_t* trace;     // K x V or null
    uint32_t* ctr;
};

// a = u*V + v with a < V^2 -> (u, v): the high product with floor((2^64-1)/V)
// underestimates a / V by at most one
__device__ __forceinline__ void decode_edge(const QArgs& q, uint64_t a, uint32_t& u, uint32_t& v) {
    uint64_t qu = __umul64hi(a, q.vinv);
    uint64_t rem = a - qu * q.V;
    if (rem >= q.V) {
        ++qu;
        rem -= q.V;
    }
    u = (uint32_t)qu;
    v = (uint32_t)rem;
}

__device__ __forceinline__ uint32_t dsu_find(uint32_t* parent, uint32_t x) {
    volatile uint32_t* P = parent;
    uint32_t p = P[x];
    while (p != x) {
        const uint32_t gp = P[p];
        if (gp != p) P[x] = gp;  // path halving; any ancestor is a valid parent
        x = p;
        p = gp;
    }
    return x;
}

__device__ void dsu_unite(uint32_t* parent, uint32_t a, uint32_t b) {
    for (;;) {
        a = dsu_find(parent, a);
        b = dsu_find(parent, b);
        if (a == b) return;
        if (a > b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        const uint32_t old = atomicCAS(&parent[b], b, a);
        if (old == b) return;
        b = old;
    }
}

// Query start: every vertex is its own component (round 0 needs no grouping).
__global__ void k_q_init(QArgs q) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x) {
        q.label[v] = v;
        q.final[v] = 0;
        q.parent[v] = v;
        q.count[v] = 1;
        q.off[v] = v;
        q.members[v] = v;
        q.roots[v] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i < C_N; ++i) q.ctr[i] = 0;
        q.ctr[C_ROOTS] = q.V;
    }
}

// End of round r = ctr[C_ROUND]: record the round's statistics, decide
// whether another round runs (a sampled edge and a fresh CubeSketch left), and
// advance the round index.  With use_cond the decision also sets the
// condition of the graph's WHILE node.
// The per-round counters (roots, large components, edges, FAIL results) are
// cleared here for the next round.
__device__ __forceinline__ void round_end(const QArgs& q, cudaGraphConditionalHandle cond, int use_cond) {
    const uint32_t r = q.ctr[C_ROUND], e = q.ctr[C_EDGES], f = q.ctr[C_FAILS];
    q.ctr[C_ROUNDS] = r + 1;
    q.ctr[C_FLAST] = f;
    q.ctr[C_FTOT] += f;
    if (e > 0 && r + 1 == q.K) q.ctr[C_EXH] = 1;
    const uint32_t go = e > 0 && r + 1 < q.K;
    q.ctr[C_GO] = go;
    q.ctr[C_ROUND] = r + 1;
    q.ctr[C_ROOTS] = q.ctr[C_BIG] = q.ctr[C_EDGES] = q.ctr[C_FAILS] = 0;
    *giant_word(q.ctr) = 0;
    if (use_cond) cudaGraphSetConditional(cond, go);
}

__global__ void k_q_next(QArgs q, cudaGraphConditionalHandle cond, int use_cond) { round_end(q, cond, use_cond); }

__global__ void k_fill64(int64_t* p, uint64_t n, int64_t val) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = val;
}

// Grouping by label (a counting sort).  After a few rounds most vertices
// share a few labels, and a counter bumped per warp would meet thousands of
// atomics on one address.  So a block takes kGroupSpan consecutive vertices
// and first counts their labels in a shared-memory hash table (open
// addressing; a warp adds equal labels once, via match_any), then touches
// each global counter once per distinct label it holds.
constexpr uint32_t kGroupThreads = 256, kGroupPer = 4, kGroupSpan = kGroupThreads * kGroupPer;
constexpr uint32_t kGroupTable = 2 * kGroupSpan;  // load factor <= 1/2
constexpr uint32_t kEmpty = 0xffffffffu;            // labels are < V <= 2^32 - 1
constexpr uint32_t kGroupTableLog2 = 11;
static_assert(kGroupTable == 1u << kGroupTableLog2, "table size");

// slot of `label` in the table, inserting it if absent
__device__ __forceinline__ uint32_t table_slot(uint32_t* keys, uint32_t label) {
    uint32_t h = (label * 0x9E3779B1u) >> (32 - kGroupTableLog2);  // multiplicative hashing
    for (;;) {
        const uint32_t k = *static_cast<volatile uint32_t*>(&keys[h]);
        if (k == label) return h;
        if (k == kEmpty) {
            const uint32_t old = atomicCAS(&keys[h], kEmpty, label);
            if (old == kEmpty || old == label) return h;
        }
        h = (h + 1) & (kGroupTable - 1);
    }
}

// the block's labels into the table: keys and counts; returns, per thread,
// the slot of each of its vertices (kEmpty past V)
__device__ __forceinline__ void table_build(const QArgs& q, uint64_t base, uint32_t* keys, uint32_t* cnt,
                                            uint32_t (&slot)[kGroupPer]) {
    for (uint32_t i = threadIdx.x; i < kGroupTable; i += blockDim.x) {
        keys[i] = kEmpty;
        cnt[i] = 0;
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (uint32_t k = 0; k < kGroupPer; ++k) {
        const uint64_t v = base + k * kGroupThreads + threadIdx.x;
        const uint32_t l = v < q.V ? q.label[v] : kEmpty;
        const uint32_t peers = __match_any_sync(0xffffffffu, l);
        const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
        uint32_t sl = kEmpty;
        if (l != kEmpty && lane == leader) {
            sl = table_slot(keys, l);
            atomicAdd(&cnt[sl], __popc(peers));
        }
        slot[k] = __shfl_sync(0xffffffffu, sl, leader);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kGroupThreads) k_q_count(QArgs q) {
    __shared__ uint32_t keys[kGroupTable], cnt[kGroupTable];
    for (uint64_t base = (uint64_t)blockIdx.x * kGroupSpan; base < q.V; base += (uint64_t)gridDim.x * kGroupSpan) {
        uint32_t slot[kGroupPer];
        table_build(q, base, keys, cnt, slot);
        for (uint32_t i = threadIdx.x; i < kGroupTable; i += blockDim.x)
            if (keys[i] != kEmpty) atomicAdd(&q.count[keys[i]], cnt[i]);
        __syncthreads();  // the table is rebuilt for the next span
    }
}

// After the scan: each block reserves one range of member positions per
// distinct label it holds, then places its vertices in them.
__global__ void __launch_bounds__(kGroupThreads) k_q_group(QArgs q) {
    __shared__ uint32_t keys[kGroupTable], cnt[kGroupTable];
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * kGroupSpan; base < q.V; base += (uint64_t)gridDim.x * kGroupSpan) {
        uint32_t slot[kGroupPer];
        table_build(q, base, keys, cnt, slot);
        for (uint32_t i = threadIdx.x; i < kGroupTable; i += blockDim.x)
            if (keys[i] != kEmpty) cnt[i] = atomicAdd(&q.cursor[keys[i]], cnt[i]);  // now the next position
        __syncthreads();
#pragma unroll
        for (uint32_t k = 0; k < kGroupPer; ++k) {
            const uint32_t v = (uint32_t)(base + k * kGroupThreads + threadIdx.x);  // used only where v < V
            const uint32_t sl = slot[k];
            const uint32_t peers = __match_any_sync(0xffffffffu, sl);
            const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
            uint32_t pos = 0;
            if (sl != kEmpty && lane == leader) pos = atomicAdd(&cnt[sl], __popc(peers));
            pos = __shfl_sync(0xffffffffu, pos, leader);
            if (sl != kEmpty) q.members[pos + __popc(peers & ((1u << lane) - 1u))] = v;
        }
        __syncthreads();
    }
}

// Root list (one append per block of kTpb vertices) and an accumulator slot
// for every component with more than M members.
constexpr uint32_t kTpb = 256;

__global__ void __launch_bounds__(kTpb) k_q_roots(QArgs q) {
    __shared__ uint32_t s_warp[kTpb / 32], s_wbig[kTpb / 32];
    __shared__ uint32_t s_base, s_bbase;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, round = q.ctr[C_ROUND];
    const uint32_t below = (1u << lane) - 1u;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x; b < q.V; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c64 = b + threadIdx.x;
        const uint32_t c = (uint32_t)c64;  // used only where c64 < V
        const uint32_t cnt = c64 < q.V ? q.count[c] : 0u;
        const bool big = cnt > q.M && !q.final[c];
        const uint32_t bal = __ballot_sync(0xffffffffu, cnt > 0);
        const uint32_t bbal = __ballot_sync(0xffffffffu, big);
        if (lane == 0) {
            s_warp[wid] = __popc(bal);
            s_wbig[wid] = __popc(bbal);
        }
        __syncthreads();
        if (threadIdx.x == 0) {  // one reservation per block for roots and for slots
            uint32_t tot = 0, btot = 0;
            for (uint32_t w = 0; w < kTpb / 32; ++w) {
                const uint32_t n = s_warp[w], nb = s_wbig[w];
                s_warp[w] = tot;
                s_wbig[w] = btot;
                tot += n;
                btot += nb;
            }
            s_base = tot ? atomicAdd(&q.ctr[C_ROOTS], tot) : 0u;
            s_bbase = btot ? atomicAdd(&q.ctr[C_BIG], btot) : 0u;
        }
        __syncthreads();
        if (cnt > 0) q.roots[s_base + s_warp[wid] + __popc(bal & below)] = c;
        if (big) q.slot[c] = s_bbase + s_wbig[wid] + __popc(bbal & below);
        if (big && cnt > q.V / 8)  // the largest, ties to the smallest id
            atomicMax(giant_word(q.ctr), ((unsigned long long)cnt << 32) | (uint32_t)~c);
        if (c64 < q.V && cnt == 0 && q.trace) q.trace[(uint64_t)round * q.V + c] = -3;
        __syncthreads();  // the shared counters are reused
    }
}

// XOR of CubeSketch `round` over the members of every component with more
// than M members, into that component's accumulator slot.
//
// The XOR of every node's CubeSketch is zero: an edge index is XORed into the
// same bucket of both endpoints' sketches (the bucket depends on the index and
// the column only).  So any one component is the XOR of every node outside
// it.  The largest live component of more than V/8 members (the giant) is
// merged that way, and its members are never read: every other node's block
// goes into its own component's slot (when that component is live and has
// more than M members) and into the giant's.
//
// The kernel walks the grouped members array without the giant's range (a
// virtual position p is member p, or p + the giant's size past its offset);
// block b takes positions [b * per, (b + 1) * per), thread w word w of a
// CubeSketch (one coalesced pass over each node's 84R bytes).  The block
// first resolves node and slot of up to blockDim of its nodes at once, then
// streams their blocks kMergeDepth at a time.  A component is one run of the
// array: its XOR is stored at the run's end when the component lies wholly in
// the block's range, or XORed in with one atomic per word when it spans
// blocks (slots are zero between rounds); the giant's part is XORed in once
// per block.
constexpr uint32_t kMergeMaxThreads = 704;  // 21R/2 words rounded up to a warp, R <= 64
constexpr uint32_t kMergeDepth = 10;
constexpr uint32_t kWhole = 0x80000000u;    // slot flag: the component lies in this block
constexpr uint32_t kNone = 0xffffffffu;     // no slot of its own (node read for the giant only)
constexpr uint32_t kSkip = 0xfffffffeu;     // node not read at all

__global__ void __launch_bounds__(kMergeMaxThreads) k_q_merge(QArgs q) {
    __shared__ uint32_t s_node[kMergeMaxThreads], s_slot[kMergeMaxThreads];
    const uint32_t nw = 21u * q.R / 2u;  // u64 words of one CubeSketch (84R bytes)
    const uint32_t w = threadIdx.x, round = q.ctr[C_ROUND];
    const unsigned long long gw = *giant_word(q.ctr);
    const bool has_giant = gw != 0;
    const uint32_t giant = ~(uint32_t)gw;
    const uint32_t g_off = has_giant ? q.off[giant] : 0u, g_cnt = has_giant ? q.count[giant] : 0u;
    const uint32_t total = q.V - g_cnt;  // virtual positions
    const uint32_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t lo64 = (uint64_t)blockIdx.x * per;
    if (lo64 >= total) return;  // block-uniform
    const uint32_t lo = (uint32_t)lo64, hi = (uint32_t)(lo64 + per < total ? lo64 + per : total);
    uint32_t cur = kNone;  // slot (with kWhole) of the run being XORed
    uint64_t x = 0, xg = 0;
    auto flush = [&]() {
        if (cur == kNone || w >= nw) return;
        uint64_t* dst = q.acc + (uint64_t)(cur & ~kWhole) * nw + w;
        if (cur & kWhole) *dst = x;
        else if (x) atomicXor(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)x);
    };
    for (uint32_t b = lo; b < hi; b += blockDim.x) {
        const uint32_t n = min(blockDim.x, hi - b);
        __syncthreads();  // the previous segment's s_node / s_slot are consumed
        if (w < n) {
            const uint32_t p = b + w;
            const uint32_t node = q.members[p < g_off ? p : p + g_cnt];
            const uint32_t c = q.label[node];
            const uint32_t cnt = q.count[c], off = q.off[c], sl = q.slot[c];
            const uint32_t voff = off < g_off ? off : off - g_cnt;  // the component's virtual offset
            s_node[w] = node;
            if (cnt > q.M && !q.final[c])
                s_slot[w] = sl | (voff >= lo && voff + cnt <= hi ? kWhole : 0u);
            else
                s_slot[w] = has_giant ? kNone : kSkip;
        }
        __syncthreads();
        for (uint32_t i0 = 0; i0 < n; i0 += kMergeDepth) {
            uint64_t t[kMergeDepth];
#pragma unroll
            for (uint32_t k = 0; k < kMergeDepth; ++k) {
                const uint32_t i = i0 + k;
                t[k] = (i < n && s_slot[i] != kSkip && w < nw)
                           ? __ldg(reinterpret_cast<const uint64_t*>(q.s.cube(s_node[i], round)) + w)
                           : 0ull;
            }
#pragma unroll
            for (uint32_t k = 0; k < kMergeDepth; ++k) {
                const uint32_t i = i0 + k;
                xg ^= t[k];
                const uint32_t sl = i < n ? s_slot[i] : kSkip;
                if (sl == kSkip || sl == kNone) continue;
                if (sl != cur) {
                    flush();
                    cur = sl;
                    x = 0;
                }
                x ^= t[k];
            }
        }
    }
    flush();
    if (has_giant && w < nw && xg)
        atomicXor(reinterpret_cast<unsigned long long*>(q.acc + (uint64_t)q.slot[giant] * nw + w),
                  (unsigned long long)xg);
}

// Sample, one warp per component.  A warp takes up to kSampleBatch
// components at a time and resolves their sizes, slots and first members
// with one load per lane.  Each component's CubeSketch `round` has one
// source: the block of its single member, or its accumulator slot (cleared
// again for the next round).  The warp fetches it into one of two
// shared-memory buffers of its own with asynchronous copies while it still
// works on the previous component; lane l moves u64 words l, l + 32, ... of
// the 84R-byte block, so every access covers 256 contiguous bytes.  Then lane l takes row l of a column
// from the buffer, the nested rows (row i = XOR of exact rows >= i) come
// from a warp-shuffle suffix XOR (rows 32 and up, which only V > 2^16 has,
// by a short loop over the buffer), and the first good bucket in Fig.
// cube_code's order (columns, then rows ascending) is found with ballots.
// The checksum keys of the round's 7 columns sit in shared memory.
constexpr uint32_t kSampleThreads = 256;
constexpr uint32_t kSampleBatch = 8;
constexpr uint32_t kMaxKeyWords = 3 * 32;  // 3 words per piece, at most 32 checksum pieces (p >= 1)

// h2 of edge (u, v) in column j of the round, keys from shared memory
// (word t of column j at sk[t * 7 + j]); the same pieces as edge_checksum
__device__ __forceinline__ uint32_t round_checksum(const uint32_t* sk, const PieceGeo& g, uint32_t j, uint32_t u,
                                                   uint32_t v) {
    uint64_t acc = 0;
    for (uint32_t i = 0; i < g.m2; ++i) {
        const uint32_t t = sk[(3 * i) * GZ_COLS + j] * u + sk[(3 * i + 1) * GZ_COLS + j] * v +
                           sk[(3 * i + 2) * GZ_COLS + j];
        acc |= (uint64_t)(t >> (32 - g.p)) << (64 - g.p * (i + 1));
    }
    return (uint32_t)(acc >> 32);
}

// two pieces of 16 bits (every V <= 2^17): the top halves joined by one byte
// permute, as in the update kernel
__device__ __forceinline__ uint32_t round_checksum2(const uint32_t* sk, uint32_t j, uint32_t u, uint32_t v) {
    const uint32_t t0 = sk[0 * GZ_COLS + j] * u + sk[1 * GZ_COLS + j] * v + sk[2 * GZ_COLS + j];
    const uint32_t t1 = sk[3 * GZ_COLS + j] * u + sk[4 * GZ_COLS + j] * v + sk[5 * GZ_COLS + j];
    return __byte_perm(t1, t0, 0x7632);  // (t0 & 0xffff0000) | (t1 >> 16)
}

__device__ __forceinline__ void cp_async8(uint64_t* dst, const uint64_t* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(static_cast<uint64_t>(__cvta_generic_to_global(src)))
                 : "memory");
}
__device__ __forceinline__ void cp_async16(uint64_t* dst, const uint64_t* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(static_cast<uint64_t>(__cvta_generic_to_global(src)))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kN>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(kN) : "memory");
}

// words of one staging buffer: 21R/2 plus one, so that a block that starts
// 8 bytes past a 16-byte boundary can be staged at the same offset, rounded
// up to keep every buffer 16-byte aligned
__host__ __device__ inline uint32_t sample_stride(uint32_t R) { return (21u * R / 2u + 2u) & ~1u; }

// kW: u64 words per lane, at least ceil(21R/2 / 32); kTwo: the checksum has
// two 16-bit pieces (V <= 2^17)
template <int kW, bool kTwo>
__global__ void __launch_bounds__(kSampleThreads, 4) k_q_sample(QArgs q) {
    extern __shared__ __align__(16) uint64_t q_cube[];  // (kSampleThreads / 32) x 2 x sample_stride(R) words
    __shared__ uint32_t s_keys[kMaxKeyWords * GZ_COLS];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t R = q.R, n_roots = q.ctr[C_ROOTS], nw = 21u * R / 2u, round = q.ctr[C_ROUND];
    for (uint32_t i = threadIdx.x; i < 3 * q.geo.m2 * GZ_COLS; i += blockDim.x)
        s_keys[i] = q.keys.at(kH2Words + i / GZ_COLS, round * GZ_COLS + i % GZ_COLS);
    __syncthreads();
    const uint32_t stride = sample_stride(R);
    uint64_t* bufs = q_cube + (threadIdx.x >> 5) * 2 * stride;
    const uint64_t VV = (uint64_t)q.V * q.V;
    const uint32_t r0 = lane, r1 = lane + 32;
    // source block of component k of the batch when it has one source
    auto single_src = [&](uint32_t cnt, uint32_t src) -> const uint64_t* {
        if (cnt > q.M) return q.acc + (uint64_t)src * nw;
        return reinterpret_cast<const uint64_t*>(q.s.cube(src, round));
    };
    // word offset in the buffer at which a source block is staged: 1 when it
    // starts 8 bytes past a 16-byte boundary, so that both sides of the
    // 16-byte copies are aligned
    auto lead = [&](const uint64_t* src) -> uint32_t {
        return (uint32_t)(reinterpret_cast<uintptr_t>(src) >> 3) & 1u;
    };
    // the block into buf + lead(src): 16-byte copies of word pairs, an
    // 8-byte copy of a leading or trailing single word
    auto fetch = [&](uint64_t* buf, const uint64_t* src) {
        const uint32_t a = lead(src);
        uint64_t* dst = buf + a;  // dst[w] is src[w]
        const uint32_t npairs = (nw - a) >> 1;
#pragma unroll
        for (int i = 0; i < (kW + 1) / 2; ++i) {
            const uint32_t c = lane + 32u * i;
            if (c < npairs) cp_async16(dst + a + 2 * c, src + a + 2 * c);
        }
        const uint32_t tail = a + 2 * npairs;
        if (a && lane == 0) cp_async8(dst, src);
        if (tail < nw && lane == 1) cp_async8(dst + tail, src + tail);
    };
    // components per warp batch: up to kSampleBatch, fewer when the warps
    // outnumber the batches (late rounds have few components)
    const uint32_t bsz = max(1u, min(kSampleBatch, n_roots / nwarps));
    uint32_t n_edges = 0, n_fails = 0;  // lane 0: this warp's sampled edges and FAIL results
    for (uint32_t base = warp * bsz; base < n_roots; base += nwarps * bsz) {
        const uint32_t nb = min(bsz, n_roots - base);
        // lane k < nb: component base + k, its size, member offset and source
        // (accumulator slot of a large component, else its first member)
        // (a final component, one that sampled EMPTY and that no sampled edge
        // touched since, reports EMPTY again without a fetch)
        uint32_t m_c = 0, m_cnt = 0, m_src = 0, m_live = 0;
        if (lane < nb && round == 0) {  // round 0: every vertex is its own live component
            m_c = m_src = base + lane;
            m_cnt = m_live = 1;
        } else if (lane < nb) {
            m_c = q.roots[base + lane];
            m_cnt = q.count[m_c];
            const uint32_t off = q.off[m_c], sl = q.slot[m_c];
            m_live = q.final[m_c] == 0;
            m_src = m_cnt > q.M ? sl : q.members[off];
        }
        {
            const uint32_t cnt = __shfl_sync(0xffffffffu, m_cnt, 0), src = __shfl_sync(0xffffffffu, m_src, 0);
            if (__shfl_sync(0xffffffffu, m_live, 0)) fetch(bufs, single_src(cnt, src));
            cp_async_commit();
        }
        for (uint32_t k = 0; k < nb; ++k) {
            const uint32_t c = __shfl_sync(0xffffffffu, m_c, k);
            const uint32_t cnt = __shfl_sync(0xffffffffu, m_cnt, k);
            const uint32_t src = __shfl_sync(0xffffffffu, m_src, k);
            const bool live = __shfl_sync(0xffffffffu, m_live, k) != 0;
            // prefetch the next component of the batch into the other buffer
            // (its previous contents were consumed before the last __syncwarp)
            const uint32_t kn = k + 1 < nb ? k + 1 : k;
            const uint32_t cnt_n = __shfl_sync(0xffffffffu, m_cnt, kn);
            const uint32_t src_n = __shfl_sync(0xffffffffu, m_src, kn);
            const uint32_t live_n = __shfl_sync(0xffffffffu, m_live, kn);
            if (k + 1 < nb && live_n) fetch(bufs + ((k + 1) & 1) * stride, single_src(cnt_n, src_n));
            cp_async_commit();
            bool nz = false;
            int64_t result = -1;  // warp-uniform
            if (live) {
            uint64_t* cube = bufs + (k & 1) * stride + lead(single_src(cnt, src));
            const uint32_t* cube_g = reinterpret_cast<const uint32_t*>(cube + GZ_COLS * R);
            cp_async_wait<1>();  // component k's copies are done (this lane's) ...
            __syncwarp();        // ... and every lane's
            if (cnt > q.M) {
                uint64_t* slot = q.acc + (uint64_t)src * nw;
#pragma unroll
                for (int i = 0; i < kW; ++i) {
                    const uint32_t w = lane + 32u * i;
                    if (w < nw) slot[w] = 0;
                }
            }
            __syncwarp();
            // columns in order; a column's rows come from the buffer only when
            // it is scanned (most components stop at the first column)
            for (int j = 0; j < GZ_COLS; ++j) {
                if (result >= 0) break;
                // rows 32.. by a loop: lane l < R - 32 takes nested row 32 + l
                uint64_t x1 = 0;
                uint32_t y1 = 0;
                for (uint32_t r = r1; r < R; ++r) {
                    x1 ^= cube[r * GZ_COLS + j];
                    y1 ^= cube_g[r * GZ_COLS + j];
                }
                uint64_t x0 = r0 < R ? cube[r0 * GZ_COLS + j] : 0ull;
                uint32_t y0 = r0 < R ? cube_g[r0 * GZ_COLS + j] : 0u;
                // suffix XOR over rows 0..31
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t lo = __shfl_down_sync(0xffffffffu, (uint32_t)x0, off);
                    const uint32_t hi = __shfl_down_sync(0xffffffffu, (uint32_t)(x0 >> 32), off);
                    const uint32_t u0 = __shfl_down_sync(0xffffffffu, y0, off);
                    if (lane + off < 32) {
                        x0 ^= ((uint64_t)hi << 32) | lo;
                        y0 ^= u0;
                    }
                }
                // rows 0..31 also take every row from 32 on (lane 0's x1)
                const uint64_t carry_a = ((uint64_t)__shfl_sync(0xffffffffu, (uint32_t)(x1 >> 32), 0) << 32) |
                                         __shfl_sync(0xffffffffu, (uint32_t)x1, 0);
                const uint32_t carry_g = __shfl_sync(0xffffffffu, y1, 0);
                x0 ^= carry_a;
                y0 ^= carry_g;
                // h2 is defined on edges: alpha must decode to u < v < V first
                auto good = [&](uint64_t a, uint32_t g, uint32_t row) -> bool {
                    if (row >= R || (a | g) == 0 || a >= VV) return false;
                    uint32_t uu, vv;
                    decode_edge(q, a, uu, vv);
                    if (uu >= vv) return false;
                    const uint32_t h2 = kTwo ? round_checksum2(s_keys, (uint32_t)j, uu, vv)
                                             : round_checksum(s_keys, q.geo, (uint32_t)j, uu, vv);
                    if (g != h2) return false;
                    // round 0: every vertex is its own component (label = id)
                    if (round == 0) return (uu == c) != (vv == c);
                    return (q.label[uu] == c) != (q.label[vv] == c);
                };
                // rows 32.. are almost always empty: their check runs only when not
                const bool deep = __any_sync(0xffffffffu, r1 < R && (x1 | y1)) != 0;
                nz |= deep || __any_sync(0xffffffffu, r0 < R && (x0 | y0)) != 0;
                const uint32_t b0 = __ballot_sync(0xffffffffu, good(x0, y0, r0));
                const uint32_t b1 = deep ? __ballot_sync(0xffffffffu, good(x1, y1, r1)) : 0u;
                if (b0 | b1) {
                    const uint32_t srcl = b0 ? (uint32_t)(__ffs(b0) - 1) : (uint32_t)(__ffs(b1) - 1);
                    const uint64_t pick = b0 ? x0 : x1;
                    result = (int64_t)(((uint64_t)__shfl_sync(0xffffffffu, (uint32_t)(pick >> 32), srcl) << 32) |
                                       __shfl_sync(0xffffffffu, (uint32_t)pick, srcl));
                }
            }
            __syncwarp();  // this buffer may be refilled by the next prefetch
            }  // live
            if (lane == 0) {
                int64_t r;
                if (result >= 0) {
                    r = result;
                    ++n_edges;
                } else if (nz) {
                    r = -2;
                    ++n_fails;
                } else {
                    r = -1;
                    if (live) q.final[c] = 1;  // EMPTY: final until a sampled edge touches it
                }
                q.res[c] = r;
                if (q.trace) q.trace[(uint64_t)round * q.V + c] = r;
            }
        }
        cp_async_wait<0>();
    }
    // the round's counters once per warp (one atomic per component on the
    // same two words would serialise in the L2)
    if (lane == 0 && n_edges) atomicAdd(&q.ctr[C_EDGES], n_edges);
    if (lane == 0 && n_fails) atomicAdd(&q.ctr[C_FAILS], n_fails);
}

__global__ void k_q_link(QArgs q) {
    const uint32_t n_roots = q.ctr[C_ROOTS];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += gridDim.x * blockDim.x) {
        const uint32_t c = q.roots[i];
        const int64_t r = q.res[c];
        if (r <= 0) continue;
        uint32_t uu, vv;
        decode_edge(q, (uint64_t)r, uu, vv);
        const uint32_t a = q.label[uu], b = q.label[vv];
        const uint32_t t = a == c ? b : a;
        q.final[a] = 0;  // both components take part in a merge
        q.final[b] = 0;
        q.target[c] = t;
        dsu_unite(q.parent, c, t);
    }
}

// forest: F = successor in the functional graph of sampled edges, Mx = running max
__global__ void k_q_fj_init(QArgs q, uint32_t* F, uint32_t* Mx, uint32_t* rej) {
    const uint32_t n_roots = q.ctr[C_ROOTS];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += gridDim.x * blockDim.x) {
        const uint32_t c = q.roots[i];
        F[c] = q.res[c] > 0 ? q.target[c] : c;
        Mx[c] = c;
        rej[c] = 0;
    }
}

__global__ void k_q_fj_step(QArgs q, const uint32_t* F, const uint32_t* Mx, uint32_t* F2, uint32_t* Mx2) {
    const uint32_t n_roots = q.ctr[C_ROOTS];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += gridDim.x * blockDim.x) {
        const uint32_t c = q.roots[i];
        const uint32_t f = F[c];
        F2[c] = F[f];
        Mx2[c] = max(Mx[c], Mx[f]);
    }
}

__global__ void k_q_fj_mark(QArgs q, const uint32_t* F, const uint32_t* Mx, uint32_t* rej) {
    const uint32_t n_roots = q.ctr[C_ROOTS];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += gridDim.x * blockDim.x) {
        const uint32_t c = q.roots[i];
        const uint32_t m = Mx[F[c]];
        if (q.res[m] > 0) rej[m] = 1;
    }
}

// accepted[v] for every vertex (0 unless v is a root whose edge is kept)
__global__ void k_q_accept(QArgs q, const uint32_t* rej, uint32_t* acc) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x)
        acc[v] = (q.count[v] > 0 && q.res[v] > 0 && !rej[v]) ? 1u : 0u;
}

__global__ void k_q_forest_write(QArgs q, const uint32_t* acc, const uint32_t* pos, uint32_t* forest) {
    const uint32_t base = q.ctr[C_FOREST];
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x) {
        if (!acc[v]) continue;
        const uint64_t e = (uint64_t)q.res[v];
        const uint32_t p = base + pos[v];
        decode_edge(q, e, forest[2 * p], forest[2 * p + 1]);
    }
}

__global__ void k_q_forest_advance(QArgs q, const uint32_t* pos) {
    q.ctr[C_FOREST] += pos[q.V];
}

// New component of every old root (its set's minimum vertex id) ...
__global__ void k_q_newroot(QArgs q, uint32_t* newroot) {
    const uint32_t n_roots = q.ctr[C_ROOTS];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += gridDim.x * blockDim.x) {
        const uint32_t c = q.roots[i];
        newroot[c] = dsu_find(q.parent, c);
    }
}

// ... then every vertex follows its old root and clears its counter for the
// next round's grouping.  (A find per vertex instead would walk the same
// few root chains from every member of a large component at once.)  With
// end_round (the query graph) the first thread also ends the round
// (round_end): it only touches counters that the sampler and k_q_newroot
// have finished with.
__global__ void k_q_relabel(QArgs q, const uint32_t* newroot, cudaGraphConditionalHandle cond, int end_round) {
    if (end_round && blockIdx.x == 0 && threadIdx.x == 0) round_end(q, cond, 1);
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += (uint64_t)gridDim.x * blockDim.x) {
        q.label[v] = newroot[q.label[v]];
        q.count[v] = 0;
    }
}

__global__ void k_q_ncc(QArgs q) {
    uint32_t n = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x)
        n += q.label[v] == v;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&q.ctr[C_NCC], n);
}

// ------------------------------------------------------------------ host side

// dynamic shared memory of the sampler: two CubeSketch buffers per warp
static size_t sample_smem(uint32_t R) { return (size_t)(kSampleThreads / 32) * 2 * sample_stride(R) * sizeof(uint64_t); }
static uint32_t merge_threads(uint32_t R) { return (21u * R / 2u + 31) / 32 * 32; }  // <= kMergeMaxThreads

constexpr uint32_t kPinnedLabels = 1u << 17;  // graphs this large stage their labels in pinned memory

gz_status query_setup(gz_handle* h) {
    if (h->query_ready) return GZ_OK;
    const size_t V = h->V;
    h->q_slots_cap = query_slots(h->V);
    auto alloc32 = [&](uint32_t** p, size_t n) { return cudaMallocAsync(p, n * sizeof(uint32_t), h->stream); };
    cudaError_t e = cudaSuccess;
    uint32_t** arrs[] = {&h->q_label, &h->q_parent, &h->q_members, &h->q_roots, &h->q_target,
                         &h->q_slot, &h->q_F, &h->q_F2, &h->q_M, &h->q_M2,
                         &h->q_flag, &h->q_cursor};
    for (auto p : arrs)
        if (e == cudaSuccess) e = alloc32(p, V);
    if (e == cudaSuccess) e = alloc32(&h->q_count, V + 1);
    if (e == cudaSuccess) e = alloc32(&h->q_final, V);
    if (e == cudaSuccess) e = alloc32(&h->q_off, V + 1);
    if (e == cudaSuccess) e = alloc32(&h->q_pos, V + 1);
    if (e == cudaSuccess) e = alloc32(&h->q_forest, 2 * V);
    if (e == cudaSuccess) e = alloc32(&h->q_ctr, C_N);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->q_res, V * sizeof(int64_t), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->q_acc, (size_t)h->q_slots_cap * h->per_k_bytes, h->stream);
    if (e == cudaSuccess) {
        // pageable: pinned allocations are expensive to make and free for
        // short-lived handles (a server creates and releases many)
        h->h_ctr = new (std::nothrow) uint32_t[C_N];
        if (!h->h_ctr) return set_error(h, GZ_ENOMEM, "query counters");
        // Large graphs' labels come back through a pinned buffer: a copy of
        // 2^17 or more labels into pageable memory goes through the driver's
        // staging buffers and takes as long as the last Boruvka rounds.
        // Small graphs (a server makes and frees many) copy directly.
        if (V >= kPinnedLabels) {
            e = cudaMallocHost(&h->h_labels, V * sizeof(uint32_t));
            if (e != cudaSuccess) h->h_labels = nullptr;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "query scratch allocation");
    // The sampler's two buffers per warp exceed the default 48 KB of dynamic
    // shared memory for R > 36.  The limit is a property of the kernel, shared
    // by every handle of the process (and set while other threads may launch
    // it), so it is raised once, to what the largest R (64) needs.
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        const int smem = (int)sample_smem(64);
        const void* fns[] = {(const void*)k_q_sample<6, true>,  (const void*)k_q_sample<12, true>,
                             (const void*)k_q_sample<16, true>, (const void*)k_q_sample<21, true>,
                             (const void*)k_q_sample<6, false>, (const void*)k_q_sample<12, false>,
                             (const void*)k_q_sample<16, false>, (const void*)k_q_sample<21, false>};
        for (const void* f : fns)
            if (attr_err == cudaSuccess)
                attr_err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    e = attr_err;
    // the merge runs one wave of resident blocks
    int occ = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_q_merge, (int)merge_threads(h->R), 0);
    if (e != cudaSuccess) return cuda_check(h, e, "query kernel attributes");
    h->q_merge_occ = (uint32_t)std::max(occ, 1);
    h->query_ready = true;
    return GZ_OK;
}

static inline uint32_t grid_for(const gz_handle* h, uint64_t n, uint32_t tpb) {
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((n + tpb - 1) / tpb, (uint64_t)h->sm_count * 8));
}

static QArgs query_args(gz_handle* h) {
    QArgs q;
    q.s.base = h->d_sketch;
    q.s.node_bytes = h->node_bytes;
    q.s.per_k_bytes = h->per_k_bytes;
    q.s.gamma_off = 56u * h->R;
    if (h->tiered) {  // each round reads the gathered array: CubeSketch r of node x at x * per_k_bytes
        q.s.base = h->d_gather;
        q.s.node_bytes = h->per_k_bytes;
        q.s.per_k_bytes = 0;
    }
    q.keys.w = h->d_keys;
    q.keys.ncol = h->ncol;
    q.geo = h->geo;
    q.V = h->V;
    q.vinv = ~0ull / h->V;
    q.K = h->K;
    q.R = h->R;
    q.M = kSlotAbove;
    q.label = h->q_label;
    q.parent = h->q_parent;
    q.count = h->q_count;
    q.off = h->q_off;
    q.cursor = h->q_cursor;
    q.members = h->q_members;
    q.final = h->q_final;
    q.roots = h->q_roots;
    q.target = h->q_target;
    q.slot = h->q_slot;
    q.acc = h->q_acc;
    q.res = h->q_res;
    q.trace = h->trace ? h->q_trace : nullptr;
    q.ctr = h->q_ctr;
    return q;
}

// query start: singletons and counters
static void enqueue_start(gz_handle* h, const QArgs& q, cudaStream_t stm) {
    k_q_init<<<grid_for(h, h->V, kTpb), kTpb, 0, stm>>>(q);
}

// group vertices by component and merge the large components (rounds > 0;
// round 0 starts from singletons)
static void enqueue_grouping(gz_handle* h, const QArgs& q, cudaStream_t stm) {
    const uint32_t V = h->V, gV = grid_for(h, V, kTpb);
    // the counters start at zero: the previous round's relabel cleared them
    // (count[0..V)), and so did its round end (roots, big, edges, fails)
    // one block per span of kGroupSpan vertices
    const uint32_t gS = (uint32_t)std::min<uint64_t>(((uint64_t)V + kGroupSpan - 1) / kGroupSpan,
                                                     (uint64_t)h->sm_count * 8);
    k_q_count<<<gS, kGroupThreads, 0, stm>>>(q);
    launch_scan(h->q_count, h->q_off, h->q_cursor, nullptr, V, stm, h->d_scan_tmp);
    k_q_group<<<gS, kGroupThreads, 0, stm>>>(q);
    k_q_roots<<<gV, kTpb, 0, stm>>>(q);
    // one thread per u64 word of a CubeSketch, contiguous member ranges, one
    // wave of blocks
    const uint32_t mt = merge_threads(h->R);
    const uint32_t nblk = std::max<uint32_t>(1, std::min<uint32_t>((V + 31) / 32, h->sm_count * h->q_merge_occ));
    k_q_merge<<<nblk, mt, 0, stm>>>(q);
}

// u64 words per lane of the sampler's staging loads
static int sample_words(uint32_t R) {
    const uint32_t w = (21u * R / 2u + 31) / 32;
    return w <= 6 ? 6 : w <= 12 ? 12 : w <= 16 ? 16 : 21;
}

static void enqueue_sample(gz_handle* h, const QArgs& q, cudaStream_t stm) {
    const size_t smem = sample_smem(h->R);
    const uint32_t grid = h->sm_count * 16;
    // two checksum pieces means 16-bit pieces (p = 16 whenever m2 = 2)
    const bool two = h->geo.m2 == 2;
    switch (sample_words(h->R) * 2 + (two ? 1 : 0)) {
    case 13: k_q_sample<6, true><<<grid, kSampleThreads, smem, stm>>>(q); break;
    case 25: k_q_sample<12, true><<<grid, kSampleThreads, smem, stm>>>(q); break;
    case 33: k_q_sample<16, true><<<grid, kSampleThreads, smem, stm>>>(q); break;
    case 43: k_q_sample<21, true><<<grid, kSampleThreads, smem, stm>>>(q); break;
    case 12: k_q_sample<6, false><<<grid, kSampleThreads, smem, stm>>>(q); break;
    case 24: k_q_sample<12, false><<<grid, kSampleThreads, smem, stm>>>(q); break;
    case 32: k_q_sample<16, false><<<grid, kSampleThreads, smem, stm>>>(q); break;
    default: k_q_sample<21, false><<<grid, kSampleThreads, smem, stm>>>(q); break;
    }
}

static void enqueue_link(gz_handle* h, const QArgs& q, cudaStream_t stm) {
    k_q_link<<<grid_for(h, h->V, kTpb), kTpb, 0, stm>>>(q);
}

// new component of every old root, then every vertex follows its old root (a
// no-op after a round without a sampled edge: no union happened); in the
// query graph the relabel also ends the round
static void enqueue_relabel(gz_handle* h, const QArgs& q, cudaStream_t stm, cudaGraphConditionalHandle cond,
                            int end_round) {
    const uint32_t gV = grid_for(h, h->V, kTpb);
    k_q_newroot<<<gV, kTpb, 0, stm>>>(q, h->q_cursor);
    k_q_relabel<<<gV, kTpb, 0, stm>>>(q, h->q_cursor, cond, end_round);
}

// kernels of a query run as one CUDA graph: start, round 0, WHILE(another
// round) { round }, component count
constexpr uint64_t kLaunchesStartEnd = 2, kLaunchesRound0 = 4, kLaunchesRound = 10;

// The CC query as one CUDA graph, captured once per handle: round 0, then a
// conditional WHILE node whose body is one more round; the relabel kernel at
// the end of every round sets the node's condition on the device, so the host waits once
// per query instead of once per round.
static gz_status build_query_graph(gz_handle* h) {
    const QArgs q = query_args(h);
    cudaStream_t cs = nullptr, bs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaGraph_t cg = nullptr;
    cudaGraphConditionalHandle cond = 0;
    if (e == cudaSuccess) {
        enqueue_start(h, q, cs);
        enqueue_sample(h, q, cs);
        enqueue_link(h, q, cs);
        cudaStreamCaptureStatus cst;
        e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, nullptr, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cg, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) enqueue_relabel(h, q, cs, cond, 1);
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd);
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp);
        if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1,
                                                                      cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                enqueue_grouping(h, q, bs);
                enqueue_sample(h, q, bs);
                enqueue_link(h, q, bs);
                enqueue_relabel(h, q, bs, cond, 1);
                e = cudaStreamEndCapture(bs, &body);
            }
        }
        if (e == cudaSuccess) k_q_ncc<<<grid_for(h, h->V, kTpb), kTpb, 0, cs>>>(q);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->q_graph_exec, g, 0);
        if (g) h->q_graph = g;
    }
    if (bs) cudaStreamDestroy(bs);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->q_graph_exec) cudaGraphExecDestroy(h->q_graph_exec);
        if (h->q_graph) cudaGraphDestroy(h->q_graph);
        h->q_graph_exec = nullptr;
        h->q_graph = nullptr;
        return cuda_check(h, e, "query graph capture");
    }
    return GZ_OK;
}

gz_status boruvka(gz_handle* h, bool want_forest, uint32_t* labels, uint32_t* forest_uv,
                  size_t* n_edges, uint32_t* n_cc, gz_query_stats* st) {
    auto t0 = std::chrono::steady_clock::now();
    gz_status s = query_setup(h);
    if (s != GZ_OK) return s;
    if (h->trace && !h->q_trace) {
        cudaError_t e = cudaMallocAsync(&h->q_trace, (size_t)h->K * h->V * sizeof(int64_t), h->stream);
        if (e != cudaSuccess) return cuda_check(h, e, "trace allocation");
    }
    cudaStream_t stm = h->stream;
    const QArgs q = query_args(h);
    const uint32_t V = h->V;
    cudaError_t e = cudaSuccess;
    // The sampler clears every accumulator slot it reads, so slots are zero
    // after a query that ran to its end; after an allocation or a failed
    // query they are cleared here.
    if (h->q_acc_dirty) {
        e = cudaMemsetAsync(h->q_acc, 0, (size_t)h->q_slots_cap * h->per_k_bytes, stm);
        if (e != cudaSuccess) return cuda_check(h, e, "query slots");
        h->q_acc_dirty = false;
    }

    if (!want_forest && !h->trace && !h->tiered && !h->cfg.no_graph) {
        if (!h->q_graph_exec && (s = build_query_graph(h)) != GZ_OK) return s;
        e = cudaGraphLaunch(h->q_graph_exec, stm);
        // counters after the graph: pageable host memory stays out of the graph
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->h_ctr, h->q_ctr, C_N * sizeof(uint32_t), cudaMemcpyDeviceToHost, stm);
    } else {
        // forest, trace or sketches beyond HBM: the same rounds driven from
        // the host, which reads the round's counters after the sampler (the
        // forest kernels are sized by the number of components) and, for a
        // tiered handle, first gathers CubeSketch r of every node
        if ((s = tier_settle(h)) != GZ_OK) return s;
        enqueue_start(h, q, stm);
        if (q.trace) k_fill64<<<grid_for(h, (uint64_t)h->K * V, kTpb), kTpb, 0, stm>>>(q.trace, (uint64_t)h->K * V, -4);
        h->launches += 1 + (q.trace ? 1 : 0);
        for (uint32_t r = 0; r < h->K && e == cudaSuccess; ++r) {
            if (h->tiered) {
                const size_t pk = h->per_k_bytes;
                if (h->res_nodes)
                    e = cudaMemcpy2DAsync(h->d_gather, pk, h->d_sketch + (size_t)r * pk, h->node_bytes, pk,
                                          h->res_nodes, cudaMemcpyDeviceToDevice, stm);
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync(h->d_gather + (size_t)h->res_nodes * pk, pk, h->h_sketch + (size_t)r * pk,
                                          h->node_bytes, pk, V - h->res_nodes, cudaMemcpyHostToDevice, stm);
                if (e != cudaSuccess) break;
            }
            if (r > 0) {
                enqueue_grouping(h, q, stm);
                h->launches += 6;
            }
            enqueue_sample(h, q, stm);
            e = cudaMemcpyAsync(h->h_ctr, h->q_ctr, C_N * sizeof(uint32_t), cudaMemcpyDeviceToHost, stm);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
            if (e != cudaSuccess) break;
            const uint32_t n_roots = h->h_ctr[C_ROOTS], n_ed = h->h_ctr[C_EDGES];
            if (n_ed > 0) {
                enqueue_link(h, q, stm);
                if (want_forest) {
                    uint32_t *F = h->q_F, *F2 = h->q_F2, *Mx = h->q_M, *Mx2 = h->q_M2;
                    const uint32_t gR = grid_for(h, n_roots, kTpb), gV = grid_for(h, V, kTpb);
                    k_q_fj_init<<<gR, kTpb, 0, stm>>>(q, F, Mx, h->q_flag);
                    uint32_t J = 1;
                    while ((1ull << (J - 1)) < (uint64_t)n_roots) ++J;
                    for (uint32_t it = 0; it < J; ++it) {
                        k_q_fj_step<<<gR, kTpb, 0, stm>>>(q, F, Mx, F2, Mx2);
                        std::swap(F, F2);
                        std::swap(Mx, Mx2);
                    }
                    k_q_fj_mark<<<gR, kTpb, 0, stm>>>(q, F, Mx, h->q_flag);
                    // q_cursor is free again: reuse it for the accept flags
                    k_q_accept<<<gV, kTpb, 0, stm>>>(q, h->q_flag, h->q_cursor);
                    launch_scan(h->q_cursor, h->q_pos, nullptr, nullptr, V, stm, h->d_scan_tmp);
                    k_q_forest_write<<<gV, kTpb, 0, stm>>>(q, h->q_cursor, h->q_pos, h->q_forest);
                    k_q_forest_advance<<<1, 1, 0, stm>>>(q, h->q_pos);
                    h->launches += J + 7;
                }
                enqueue_relabel(h, q, stm, 0, 0);
                h->launches += 3;  // link, newroot, relabel
            }
            k_q_next<<<1, 1, 0, stm>>>(q, 0, 0);
            h->launches += 2;  // sample, next
            if (n_ed == 0) break;
        }
        if (e == cudaSuccess) {
            k_q_ncc<<<grid_for(h, V, kTpb), kTpb, 0, stm>>>(q);
            h->launches += 1;
            e = cudaMemcpyAsync(h->h_ctr, h->q_ctr, C_N * sizeof(uint32_t), cudaMemcpyDeviceToHost, stm);
        }
    }
    if (e == cudaSuccess && labels)
        e = cudaMemcpyAsync(h->h_labels ? h->h_labels : labels, h->q_label, (size_t)V * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, stm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
    if (e != cudaSuccess) {
        h->q_acc_dirty = true;
        return cuda_check(h, e, "query");
    }
    if (labels && h->h_labels) std::memcpy(labels, h->h_labels, (size_t)V * sizeof(uint32_t));
    const uint32_t ncc = h->h_ctr[C_NCC];
    const uint32_t nf = h->h_ctr[C_FOREST];
    const uint32_t rounds = h->h_ctr[C_ROUNDS], fails_last = h->h_ctr[C_FLAST];
    const uint32_t fails_total = h->h_ctr[C_FTOT], exhausted = h->h_ctr[C_EXH];
    if (!want_forest && !h->trace)
        h->launches += kLaunchesStartEnd + kLaunchesRound0 + (uint64_t)(rounds ? rounds - 1 : 0) * kLaunchesRound;
    if (want_forest) {
        if (forest_uv && nf) {
            e = cudaMemcpy(forest_uv, h->q_forest, (size_t)nf * 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_check(h, e, "forest copy");
        }
        if (n_edges) *n_edges = nf;
    }
    if (n_cc) *n_cc = ncc;
    h->trace_valid = h->trace;
    auto t1 = std::chrono::steady_clock::now();
    if (st) {
        st->rounds = rounds;
        st->fails_last = fails_last;
        st->exhausted = exhausted;
        st->n_components = ncc;
        st->fails_total = fails_total;
        st->reserved = 0;
        st->ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
    }
    if (fails_last || exhausted)
        return set_error(h, GZ_ESKETCH_FAIL, "a CubeSketch failed in the last Boruvka round or rounds ran out");
    return GZ_OK;
}

}  // namespace gz
