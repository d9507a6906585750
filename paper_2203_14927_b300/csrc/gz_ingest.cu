// gz_ingest.cu -- stream ingestion: CubeSketch updates of every node touched by a
// batch of edge updates (Fig. cube_code update_sketch; Section 5.1 "Sketch
// updates").
//
// The paper buffers updates per node (leaf-only gutters, Section 5.1) and lets
// Graph Workers apply one node's batch at a time.  Here one batch of updates is
// partitioned by endpoint on the device (histogram, exclusive scan, scatter: each
// update lands in the segment of both endpoints with the other endpoint as the
// record), and a persistent kernel walks fixed-size tiles of the partitioned
// records.  For every node segment in its tile a CTA keeps a zeroed delta sketch
// of the first `Rs` exact-depth rows in shared memory (one thread per CubeSketch
// column, so no shared-memory atomics), applies the segment, then XORs the
// touched rows into the node's sketch in global memory with red.global.xor --
// the "apply to an empty sketch, then add" step of Section 5.1 (linearity), which
// also lets two CTAs share one heavy node whose segment spans tiles.
#include <cuda_runtime.h>

#include <algorithm>

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

// The two hashes of one column written on 32-bit words, with every part that
// depends only on the column's keys folded into per-thread constants.  They
// compute exactly `depth_word` and `checksum` of gz_internal.cuh.
namespace fm {
constexpr uint32_t C1_LO = 0xED558CCDu, C1_HI = 0xFF51AFD7u;  // MurmurHash3 fmix64 multipliers
constexpr uint32_t C2_LO = 0x1A85EC53u, C2_HI = 0xC4CEB9FEu;
}  // namespace fm

struct ColKey {
    uint32_t a_lo, a_hi;
    uint64_t b;
    uint32_t kfold;  // c_lo ^ (c_hi >> 1): the key's share of the first xor-shift
    uint32_t c_hi;
    uint32_t k2;     // c_hi * C1_LO: the key's share of the first product when idx < 2^32
};

__device__ __forceinline__ ColKey make_colkey(uint64_t a, uint64_t b, uint64_t c) {
    ColKey k;
    k.a_lo = (uint32_t)a;
    k.a_hi = (uint32_t)(a >> 32);
    k.b = b;
    const uint32_t c_lo = (uint32_t)c, c_hi = (uint32_t)(c >> 32);
    k.kfold = c_lo ^ (c_hi >> 1);
    k.c_hi = c_hi;
    k.k2 = c_hi * fm::C1_LO;
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

// hi32(fmix64(idx ^ c)); fold = idx_lo ^ (idx_hi >> 1), precomputed per record
template <bool kWide>
__device__ __forceinline__ uint32_t checksum_w(const ColKey& k, uint32_t x_hi, uint32_t fold) {
    const uint32_t lo1 = fold ^ k.kfold;  // low word after x ^= c; x ^= x >> 33
    uint32_t lo2, hi2;
    if (kWide) {
        const uint32_t hi1 = x_hi ^ k.c_hi;
        const uint64_t q = (uint64_t)lo1 * fm::C1_LO;
        lo2 = (uint32_t)q;
        hi2 = (uint32_t)(q >> 32) + lo1 * fm::C1_HI + hi1 * fm::C1_LO;
    } else {
        const uint64_t q = (uint64_t)lo1 * fm::C1_LO + ((uint64_t)k.k2 << 32);
        lo2 = (uint32_t)q;
        hi2 = (uint32_t)(q >> 32) + lo1 * fm::C1_HI;
    }
    const uint32_t lo3 = lo2 ^ (hi2 >> 1);
    return __umulhi(lo3, fm::C2_LO) + lo3 * fm::C2_HI + hi2 * fm::C2_LO;
}

// One CTA = 32*ceil(7K/32) threads; thread c owns CubeSketch column c = 7k + j
// (one "Graph Worker" per column; no two threads write one bucket).
// Dynamic shared memory:
//   delta alpha  [Rs][CP] u64 (kAtomic: two u32 planes lo[Rs][CP], hi[Rs][CP])
//   delta gamma  [Rs][CP] u32
//   staged records [tile] (kWide: uint4 {idx_lo, idx_hi, fold, 0}; else u32 idx)
//   per-k deepest touched row [K] u32
// With the [row][column] layout the 32 lanes of a warp hit 32 distinct banks
// whatever rows their updates land in.  kAtomic uses shared-memory atomics for
// the XORs, so an update never waits on a shared-memory load.
template <bool kAtomic, bool kWide>
__global__ void __launch_bounds__(1024) k_batched(BatchedArgs p) {
    extern __shared__ __align__(16) uint64_t smem[];
    if (p.flags[0]) return;
    const uint32_t CP = blockDim.x, c = threadIdx.x;
    const uint32_t Rs = p.Rs, R = p.R, RC = Rs * CP;
    uint64_t* dA = smem;                                 // kAtomic == false
    uint32_t* dAlo = reinterpret_cast<uint32_t*>(smem);  // kAtomic == true
    uint32_t* dAhi = dAlo + RC;
    uint32_t* dG = reinterpret_cast<uint32_t*>(smem + RC);
    uint32_t* stage = dG + RC;  // 16-byte aligned: RC*12 bytes, RC a multiple of 32
    uint4* stage4 = reinterpret_cast<uint4*>(stage);
    uint32_t* maxd = stage + (kWide ? 4u : 1u) * p.tile;

    const bool active = c < p.ncol;
    const uint32_t k = c / GZ_COLS, j = c - k * GZ_COLS;
    ColKey key{};
    if (active) key = make_colkey(p.keys.a[c], p.keys.b[c], p.keys.c[c]);
    for (uint32_t i = c; i < RC; i += CP) {
        if (kAtomic) {
            dAlo[i] = 0;
            dAhi[i] = 0;
        } else {
            dA[i] = 0;
        }
        dG[i] = 0;
    }
    for (uint32_t i = c; i < p.K; i += CP) maxd[i] = 0;
    const uint32_t total = p.offsets[p.V];
    const uint32_t ntiles = (total + p.tile - 1) / p.tile;
    unsigned long long n_rows = 0, n_deep = 0;
    __shared__ uint32_t s_t[2];
    if (c == 0) s_t[0] = atomicAdd(p.work, 1u);

    for (uint32_t it = 0;; ++it) {
        __syncthreads();
        const uint32_t t = s_t[it & 1];
        if (t >= ntiles) break;
        // claim the next tile now; its index is read after the next barrier
        if (c == 0) s_t[(it + 1) & 1] = atomicAdd(p.work, 1u);
        const uint32_t lo = t * p.tile, hi = min(lo + p.tile, total);
        uint32_t x = p.tile_node[t], pos = lo;
        while (pos < hi) {
            const uint32_t seg_end = min(p.offsets[x + 1], hi);
            const uint32_t nseg = seg_end - pos;
            if (nseg > 0) {
                for (uint32_t i = c; i < nseg; i += CP) {
                    const uint64_t idx = edge_index(x, p.records[pos + i], p.V);
                    if (kWide) {
                        const uint32_t ilo = (uint32_t)idx, ihi = (uint32_t)(idx >> 32);
                        stage4[i] = make_uint4(ilo, ihi, ilo ^ (ihi >> 1), 0u);
                    } else {
                        stage[i] = (uint32_t)idx;
                    }
                }
                __syncthreads();
                if (nseg < p.small_seg) {
                    // short segment: straight to global memory
                    if (active) {
                        const uint64_t ka = p.keys.a[c], kb = p.keys.b[c], kc = p.keys.c[c];
                        for (uint32_t i = 0; i < nseg; ++i) {
                            const uint64_t idx = kWide ? ((uint64_t)stage4[i].y << 32 | stage4[i].x) : stage[i];
                            const uint32_t d = exact_depth(depth_word(ka, kb, idx), R);
                            atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, k, d, j)),
                                      (unsigned long long)idx);
                            atomicXor(p.s.gamma(x, k, d, j), checksum(kc, idx));
                        }
                    }
                } else {
                    uint32_t md = 0;
                    if (active) {
                        // one column update staged in shared memory (d < Rs)
                        auto put = [&](uint32_t d, uint32_t xlo, uint32_t xhi, uint32_t g) {
                            const uint32_t slot = d * CP + c;
                            if (kAtomic) {
                                atomicXor(dAlo + slot, xlo);
                                if (kWide) atomicXor(dAhi + slot, xhi);
                                atomicXor(dG + slot, g);
                            } else {
                                dA[slot] ^= ((uint64_t)xhi << 32) | xlo;
                                dG[slot] ^= g;
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
                        uint32_t i = 0;
                        // four records at a time in straight-line code, so the
                        // four hash chains interleave; one rare branch for deep rows
                        for (; i + 4 <= nseg; i += 4) {
                            uint32_t xlo[4], xhi[4], fold[4];
                            if (kWide) {
#pragma unroll
                                for (int r = 0; r < 4; ++r) {
                                    const uint4 q = stage4[i + r];
                                    xlo[r] = q.x;
                                    xhi[r] = q.y;
                                    fold[r] = q.z;
                                }
                            } else {
                                const uint4 q = reinterpret_cast<const uint4*>(stage)[i >> 2];
                                xlo[0] = q.x;
                                xlo[1] = q.y;
                                xlo[2] = q.z;
                                xlo[3] = q.w;
#pragma unroll
                                for (int r = 0; r < 4; ++r) {
                                    xhi[r] = 0;
                                    fold[r] = xlo[r];
                                }
                            }
                            uint32_t d[4], g[4];
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                d[r] = __clz(depth_hi<kWide>(key, xlo[r], xhi[r]));
                                g[r] = checksum_w<kWide>(key, xhi[r], fold[r]);
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
                        for (; i < nseg; ++i) {
                            uint32_t xlo, xhi, fold;
                            if (kWide) {
                                const uint4 q = stage4[i];
                                xlo = q.x;
                                xhi = q.y;
                                fold = q.z;
                            } else {
                                xlo = stage[i];
                                xhi = 0;
                                fold = xlo;
                            }
                            const uint32_t d = __clz(depth_hi<kWide>(key, xlo, xhi));
                            const uint32_t g = checksum_w<kWide>(key, xhi, fold);
                            if (d < Rs) {
                                put(d, xlo, xhi, g);
                                md = max(md, d);
                            } else {
                                deep(xlo, xhi, g);
                            }
                        }
                    atomicMax(&maxd[k], md);
                    }
                    __syncthreads();
                    const uint32_t per_k = Rs * GZ_COLS;
                    for (uint32_t q = c; q < p.K * per_k; q += CP) {
                        const uint32_t kk = q / per_k, rem = q - kk * per_k;
                        const uint32_t row = rem / GZ_COLS, jj = rem - row * GZ_COLS;
                        if (row <= maxd[kk]) {
                            const uint32_t slot = row * CP + kk * GZ_COLS + jj;
                            uint64_t a;
                            if (kAtomic) {
                                a = ((uint64_t)dAhi[slot] << 32) | dAlo[slot];
                            } else {
                                a = dA[slot];
                            }
                            const uint32_t g = dG[slot];
                            if (a | g) {
                                atomicXor(reinterpret_cast<unsigned long long*>(p.s.alpha(x, kk, row, jj)),
                                          (unsigned long long)a);
                                atomicXor(p.s.gamma(x, kk, row, jj), g);
                                if (kAtomic) {
                                    dAlo[slot] = 0;
                                    dAhi[slot] = 0;
                                } else {
                                    dA[slot] = 0;
                                }
                                dG[slot] = 0;
                            }
                        }
                    }
                    __syncthreads();
                    for (uint32_t i = c; i < p.K; i += CP) {
                        n_rows += maxd[i] + 1;
                        maxd[i] = 0;
                    }
                }
                __syncthreads();
            }
            pos = seg_end;
            ++x;
        }
    }
    if (n_rows) atomicAdd(&p.stats[0], n_rows);
    if (n_deep) atomicAdd(&p.stats[1], n_deep);
}

using BatchedFn = void (*)(BatchedArgs);

static BatchedFn batched_fn(uint32_t mode, bool wide) {
    if (mode) return wide ? k_batched<true, true> : k_batched<true, false>;
    return wide ? k_batched<false, true> : k_batched<false, false>;
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
        const uint32_t g = checksum(kc, idx);
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
    k.a = h->d_keys;
    k.b = h->d_keys + h->ncol;
    k.c = h->d_keys + 2 * (size_t)h->ncol;
    return k;
}

gz_status ingest_setup(gz_handle* h) {
    h->block = (h->ncol + 31) / 32 * 32;
    if (h->block > 1024) return set_error(h, GZ_EINVAL, "too many CubeSketch columns for one CTA");
    uint32_t rs = h->cfg.smem_rows ? h->cfg.smem_rows : 16;
    rs = std::min<uint32_t>(rs, 32);
    rs = std::min<uint32_t>(rs, h->R);
    h->smem_rows = rs;
    h->tile = h->cfg.tile_records ? h->cfg.tile_records : 512;
    h->small_seg = h->cfg.small_segment ? h->cfg.small_segment : 4;
    const bool wide = (uint64_t)h->V * h->V > (1ull << 32);
    h->batched_smem = (size_t)rs * h->block * 12 + (size_t)h->tile * (wide ? 16 : 4) + (size_t)h->K * 4;
    if (h->cfg.smem_mode > 1) return set_error(h, GZ_EINVAL, "smem_mode must be 0 or 1");
    const void* fn = (const void*)batched_fn(h->cfg.smem_mode, wide);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)h->batched_smem);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaFuncSetAttribute(k_batched)");
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, (int)h->block, h->batched_smem);
    if (e != cudaSuccess) return cuda_check(h, e, "occupancy(k_batched)");
    if (nb < 1) return set_error(h, GZ_EINVAL, "batched kernel does not fit on an SM");
    uint32_t per_sm = h->cfg.ctas_per_sm ? std::min<uint32_t>(h->cfg.ctas_per_sm, nb) : nb;
    h->batched_grid = per_sm * h->sm_count;
    if (h->cfg.kernel == GZ_KERNEL_BATCHED) {
        e = cudaMalloc(&h->d_tile_node, (size_t)(2 * h->chunk / h->tile + 2) * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_check(h, e, "tile table allocation");
    }
    return GZ_OK;
}

gz_status ingest_batch(gz_handle* h, const uint32_t* d_u, const uint32_t* d_v, uint64_t n) {
    if (n == 0) return GZ_OK;
    cudaStream_t st = h->stream;
    gz_status ps = prof_event(h);
    if (ps != GZ_OK) return ps;
    cudaError_t e = cudaMemsetAsync(h->d_flags, 0, 2 * sizeof(uint32_t), st);  // batch flag + work
    if (e != cudaSuccess) return cuda_check(h, e, "memset flags");
    const uint32_t tpb = 256;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + tpb - 1) / tpb, (uint64_t)h->sm_count * 8);
    if (h->cfg.kernel == GZ_KERNEL_PLAIN) {
        k_validate_count<<<grid, tpb, 0, st>>>(d_u, d_v, n, h->V, nullptr, h->d_flags);
        if ((ps = prof_event(h)) != GZ_OK) return ps;
        const uint32_t pg = (uint32_t)std::min<uint64_t>(n, (uint64_t)h->sm_count * 16);
        k_plain<<<pg, h->block, 0, st>>>(d_u, d_v, n, view_of(h), keys_of(h), h->V, h->R, h->ncol,
                                         h->d_flags);
        h->launches += 2;
    } else {
        e = cudaMemsetAsync(h->d_counts, 0, (size_t)(h->V + 1) * sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_check(h, e, "memset counts");
        k_validate_count<<<grid, tpb, 0, st>>>(d_u, d_v, n, h->V, h->d_counts, h->d_flags);
        launch_scan(h->d_counts, h->d_offsets, h->d_cursor, h->V, st, h->d_scan_tmp);
        k_scatter<<<grid, tpb, 0, st>>>(d_u, d_v, n, h->d_cursor, h->d_records, h->d_flags);
        k_tile_nodes<<<(h->V + 255) / 256, 256, 0, st>>>(h->d_offsets, h->V, h->tile, h->d_flags,
                                                       h->d_tile_node);
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
        if ((ps = prof_event(h)) != GZ_OK) return ps;
        const bool wide = (uint64_t)h->V * h->V > (1ull << 32);
        batched_fn(h->cfg.smem_mode, wide)<<<h->batched_grid, h->block, h->batched_smem, st>>>(a);
        h->launches += 6;
    }
    if ((ps = prof_event(h)) != GZ_OK) return ps;
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
    k_export<<<(uint32_t)((threads + tpb - 1) / tpb), tpb, 0, h->stream>>>(view_of(h), lo, hi, h->K,
                                                                          h->R, d_alpha, d_gamma);
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
// layout in 32-bit words (the u64 parts first, so they stay 8-byte aligned)
constexpr size_t kKeys = 0;                                   // 3 x kMaxCols u64
constexpr size_t kStats = kKeys + 2 * 3 * kMaxCols;           // 2 u64
constexpr size_t kFlags = kStats + 4;                         // 4 u32
constexpr size_t kCounts = kFlags + 4;                        // kMaxV + 1
constexpr size_t kOffsets = kCounts + kMaxV + 1;              // kMaxV + 1
constexpr size_t kCursor = kOffsets + kMaxV + 1;              // kMaxV + 1
constexpr size_t kTiles = kCursor + kMaxV + 1;                // scan tile sums
constexpr size_t kRecords = kTiles + (kMaxV + 1) / 1024 + 2;  // 2 x kMaxUpdates
constexpr uint32_t kTile = 1024;                              // records per work tile
constexpr size_t kTileNode = kRecords + 2 * kMaxUpdates;       // first node of every tile
constexpr size_t kWords = kTileNode + 2 * kMaxUpdates / kTile + 2;

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

__global__ void k_status(const uint32_t* flags, uint32_t* status) { *status = flags[0] ? 1u : 0u; }

// Once per device, with that device current: the device address of the
// scratch array (its name is only a host-side stand-in in host code).
static gz_status setup(int dev, uint32_t** ptr, int* sms) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return GZ_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GZ_ECUDA;
        for (int wide = 0; wide < 2; ++wide)
            if (cudaFuncSetAttribute((const void*)batched_fn(1, wide != 0),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024) != cudaSuccess)
                return GZ_ECUDA;
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
    const uint32_t Rs = std::min<uint32_t>(16, R), tile = kTile;
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
        const size_t smem = (size_t)Rs * block * 12 + (size_t)tile * (wide ? 16 : 4) + (size_t)K * 4;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_fn(1, wide), (int)block, smem) !=
                cudaSuccess ||
            per_sm < 1)
            return GZ_ECUDA;
        batched_fn(1, wide)<<<per_sm * sms, block, smem, st>>>(a);
    }
    if (status) k_status<<<1, 1, 0, st>>>(flags, status);
    return cudaGetLastError() == cudaSuccess ? GZ_OK : GZ_ECUDA;
}
