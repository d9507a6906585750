// gz_query.cu -- connected components / spanning forest by Boruvka rounds over
// the node sketches (Section 2.2; the three phases of a round in the proof of
// Lemma (CC I/O); list_spanning_forest of Section 5).
//
// Round r:
//   group    nodes by current component (counting sort by label);
//   merge    component sketch = XOR of the members' CubeSketch r (big
//            components are split into items of M members whose partial XORs
//            are combined afterwards);
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
// A round that samples no edge ends the query.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "gz_handle.cuh"
#include "gz_internal.cuh"

namespace gz {

enum { C_ROOTS = 0, C_ITEMS = 1, C_EDGES = 2, C_FAILS = 3, C_FOREST = 4, C_NCC = 5, C_N = 8 };

struct QArgs {
    SketchView s;
    const uint64_t* kc;  // checksum keys, 7K
    uint32_t V, K, R, round, M;
    uint32_t *label, *parent, *count, *off, *cursor, *members, *roots, *target;
    uint32_t *item_base, *item_cnt, *item_comp, *item_lo, *item_hi;
    uint64_t* partial;  // items x (21R/2) words
    int64_t* res;
    int64_t* trace;     // K x V or null
    uint32_t* ctr;
};

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

__global__ void k_q_init(uint32_t* label, uint32_t* parent, uint32_t V) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        label[v] = v;
        parent[v] = v;
    }
}

__global__ void k_fill64(int64_t* p, uint64_t n, int64_t val) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = val;
}

__global__ void k_q_count(QArgs q) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x)
        atomicAdd(&q.count[q.label[v]], 1u);
}

__global__ void k_q_group(QArgs q) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x)
        q.members[atomicAdd(&q.cursor[q.label[v]], 1u)] = v;
}

__global__ void k_q_roots(QArgs q) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < q.V; c += gridDim.x * blockDim.x) {
        const uint32_t cnt = q.count[c];
        if (cnt == 0) {
            if (q.trace) q.trace[(uint64_t)q.round * q.V + c] = -3;
            continue;
        }
        q.roots[atomicAdd(&q.ctr[C_ROOTS], 1u)] = c;
        if (cnt > q.M) {
            const uint32_t ni = (cnt + q.M - 1) / q.M;
            const uint32_t base = atomicAdd(&q.ctr[C_ITEMS], ni);
            q.item_base[c] = base;
            q.item_cnt[c] = ni;
            const uint32_t o = q.off[c];
            for (uint32_t i = 0; i < ni; ++i) {
                q.item_comp[base + i] = c;
                q.item_lo[base + i] = o + i * q.M;
                q.item_hi[base + i] = o + min(cnt, (i + 1) * q.M);
            }
        } else {
            q.item_cnt[c] = 0;
        }
    }
}

// Partial XOR of CubeSketch `round` over the members of one item.
__global__ void k_q_merge_items(QArgs q) {
    const uint32_t nw = 21u * q.R / 2u;  // u64 words of one CubeSketch (84R bytes)
    const uint32_t n_items = q.ctr[C_ITEMS];
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint32_t lo = q.item_lo[it], hi = q.item_hi[it];
        for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
            uint64_t acc = 0;
            for (uint32_t m = lo; m < hi; ++m) {
                const uint64_t* cube = reinterpret_cast<const uint64_t*>(q.s.cube(q.members[m], q.round));
                acc ^= __ldg(cube + w);
            }
            q.partial[(uint64_t)it * nw + w] = acc;
        }
    }
}

// Merge (small components) + sample, one CTA per component.
__global__ void __launch_bounds__(256) k_q_sample(QArgs q) {
    extern __shared__ __align__(16) uint64_t S[];  // nw words: alpha[R][7] then gamma[R][7]
    __shared__ uint32_t s_best;
    const uint32_t nw = 21u * q.R / 2u, R = q.R, nb = GZ_COLS * R;
    uint64_t* A = S;
    uint32_t* G = reinterpret_cast<uint32_t*>(S + nb);
    const uint32_t n_roots = q.ctr[C_ROOTS];
    const uint64_t VV = (uint64_t)q.V * q.V;
    for (uint32_t ri = blockIdx.x; ri < n_roots; ri += gridDim.x) {
        const uint32_t c = q.roots[ri];
        const uint32_t ni = q.item_cnt[c];
        for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
            uint64_t acc = 0;
            if (ni == 0) {
                const uint32_t lo = q.off[c], hi = lo + q.count[c];
                for (uint32_t m = lo; m < hi; ++m) {
                    const uint64_t* cube = reinterpret_cast<const uint64_t*>(q.s.cube(q.members[m], q.round));
                    acc ^= __ldg(cube + w);
                }
            } else {
                const uint32_t b = q.item_base[c];
                for (uint32_t it = b; it < b + ni; ++it) acc ^= q.partial[(uint64_t)it * nw + w];
            }
            S[w] = acc;
        }
        if (threadIdx.x == 0) s_best = 0xffffffffu;
        __syncthreads();
        // nested rows: row i = XOR of exact rows i..R-1 (one thread per column)
        if (threadIdx.x < GZ_COLS) {
            const uint32_t j = threadIdx.x;
            for (int row = (int)R - 2; row >= 0; --row) {
                A[row * GZ_COLS + j] ^= A[(row + 1) * GZ_COLS + j];
                G[row * GZ_COLS + j] ^= G[(row + 1) * GZ_COLS + j];
            }
        }
        __syncthreads();
        bool nz = false;
        uint32_t best = 0xffffffffu;
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
            const uint32_t row = b / GZ_COLS, j = b - row * GZ_COLS;
            const uint64_t a = A[b];
            const uint32_t g = G[b];
            if ((a | g) == 0) continue;
            nz = true;
            if (g != checksum(q.kc[q.round * GZ_COLS + j], a) || a >= VV) continue;
            const uint32_t uu = (uint32_t)(a / q.V), vv = (uint32_t)(a % q.V);
            if (uu >= vv) continue;
            const bool in_u = q.label[uu] == c, in_v = q.label[vv] == c;
            if (in_u == in_v) continue;
            best = min(best, j * R + row);
        }
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0 && best != 0xffffffffu) atomicMin(&s_best, best);
        const int any_nz = __syncthreads_or(nz);
        if (threadIdx.x == 0) {
            const uint32_t bb = s_best;
            int64_t r;
            if (bb != 0xffffffffu) {
                const uint32_t j = bb / R, row = bb - j * R;
                r = (int64_t)A[row * GZ_COLS + j];
                atomicAdd(&q.ctr[C_EDGES], 1u);
            } else if (any_nz) {
                r = -2;
                atomicAdd(&q.ctr[C_FAILS], 1u);
            } else {
                r = -1;
            }
            q.res[c] = r;
            if (q.trace) q.trace[(uint64_t)q.round * q.V + c] = r;
        }
        __syncthreads();
    }
}

__global__ void k_q_link(QArgs q) {
    const uint32_t n_roots = q.ctr[C_ROOTS];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += gridDim.x * blockDim.x) {
        const uint32_t c = q.roots[i];
        const int64_t r = q.res[c];
        if (r <= 0) continue;
        const uint32_t uu = (uint32_t)((uint64_t)r / q.V), vv = (uint32_t)((uint64_t)r % q.V);
        const uint32_t a = q.label[uu], b = q.label[vv];
        const uint32_t t = a == c ? b : a;
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
        forest[2 * p] = (uint32_t)(e / q.V);
        forest[2 * p + 1] = (uint32_t)(e % q.V);
    }
}

__global__ void k_q_forest_advance(QArgs q, const uint32_t* pos) {
    q.ctr[C_FOREST] += pos[q.V];
}

__global__ void k_q_relabel(QArgs q) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x)
        q.label[v] = dsu_find(q.parent, q.label[v]);
}

__global__ void k_q_ncc(QArgs q) {
    uint32_t n = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < q.V; v += gridDim.x * blockDim.x)
        n += q.label[v] == v;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&q.ctr[C_NCC], n);
}

// ------------------------------------------------------------------ host side

gz_status query_setup(gz_handle* h) {
    if (h->query_ready) return GZ_OK;
    const size_t V = h->V;
    h->q_M_members = 64;
    h->q_items_cap = (uint32_t)(2 * V / h->q_M_members + 2);
    auto alloc32 = [&](uint32_t** p, size_t n) { return cudaMallocAsync(p, n * sizeof(uint32_t), h->stream); };
    cudaError_t e = cudaSuccess;
    uint32_t** arrs[] = {&h->q_label, &h->q_parent, &h->q_members, &h->q_roots, &h->q_target,
                         &h->q_item_base, &h->q_item_cnt, &h->q_F, &h->q_F2, &h->q_M, &h->q_M2,
                         &h->q_flag, &h->q_cursor};
    for (auto p : arrs)
        if (e == cudaSuccess) e = alloc32(p, V);
    if (e == cudaSuccess) e = alloc32(&h->q_count, V + 1);
    if (e == cudaSuccess) e = alloc32(&h->q_off, V + 1);
    if (e == cudaSuccess) e = alloc32(&h->q_pos, V + 1);
    if (e == cudaSuccess) e = alloc32(&h->q_item_comp, h->q_items_cap);
    if (e == cudaSuccess) e = alloc32(&h->q_item_lo, h->q_items_cap);
    if (e == cudaSuccess) e = alloc32(&h->q_item_hi, h->q_items_cap);
    if (e == cudaSuccess) e = alloc32(&h->q_forest, 2 * V);
    if (e == cudaSuccess) e = alloc32(&h->q_ctr, C_N);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->q_res, V * sizeof(int64_t), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&h->q_partial, (size_t)h->q_items_cap * h->per_k_bytes, h->stream);
    if (e == cudaSuccess) {
        h->h_ctr = new (std::nothrow) uint32_t[C_N];
        if (!h->h_ctr) return set_error(h, GZ_ENOMEM, "query counters");
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "query scratch allocation");
    h->query_ready = true;
    return GZ_OK;
}

static inline uint32_t grid_for(const gz_handle* h, uint64_t n, uint32_t tpb) {
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((n + tpb - 1) / tpb, (uint64_t)h->sm_count * 8));
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
    QArgs q;
    q.s.base = h->d_sketch;
    q.s.node_bytes = h->node_bytes;
    q.s.per_k_bytes = h->per_k_bytes;
    q.s.gamma_off = 56u * h->R;
    q.kc = h->d_keys + 2 * (size_t)h->ncol;
    q.V = h->V;
    q.K = h->K;
    q.R = h->R;
    q.M = h->q_M_members;
    q.label = h->q_label;
    q.parent = h->q_parent;
    q.count = h->q_count;
    q.off = h->q_off;
    q.cursor = h->q_cursor;
    q.members = h->q_members;
    q.roots = h->q_roots;
    q.target = h->q_target;
    q.item_base = h->q_item_base;
    q.item_cnt = h->q_item_cnt;
    q.item_comp = h->q_item_comp;
    q.item_lo = h->q_item_lo;
    q.item_hi = h->q_item_hi;
    q.partial = reinterpret_cast<uint64_t*>(h->q_partial);
    q.res = h->q_res;
    q.trace = h->trace ? h->q_trace : nullptr;
    q.ctr = h->q_ctr;

    const uint32_t V = h->V, tpb = 256;
    const uint32_t gV = grid_for(h, V, tpb);
    k_q_init<<<gV, tpb, 0, stm>>>(h->q_label, h->q_parent, V);
    h->launches += 2 + (q.trace ? 1 : 0);  // init, final count (+ trace fill)
    if (q.trace) k_fill64<<<grid_for(h, (uint64_t)h->K * V, tpb), tpb, 0, stm>>>(q.trace, (uint64_t)h->K * V, -4);
    cudaError_t e = cudaMemsetAsync(h->q_ctr, 0, C_N * sizeof(uint32_t), stm);
    if (e != cudaSuccess) return cuda_check(h, e, "memset counters");

    const size_t sample_smem = (size_t)h->per_k_bytes;
    uint32_t rounds = 0, fails_last = 0, fails_total = 0, exhausted = 0;
    for (uint32_t r = 0; r < h->K; ++r) {
        q.round = r;
        rounds = r + 1;
        e = cudaMemsetAsync(h->q_count, 0, (size_t)(V + 1) * sizeof(uint32_t), stm);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->q_ctr, 0, 4 * sizeof(uint32_t), stm);  // roots..fails
        if (e != cudaSuccess) return cuda_check(h, e, "memset round");
        k_q_count<<<gV, tpb, 0, stm>>>(q);
        launch_scan(h->q_count, h->q_off, h->q_cursor, V, stm, h->d_scan_tmp);
        k_q_group<<<gV, tpb, 0, stm>>>(q);
        k_q_roots<<<gV, tpb, 0, stm>>>(q);
        k_q_merge_items<<<h->sm_count * 4, 384, 0, stm>>>(q);
        k_q_sample<<<h->sm_count * 16, 256, sample_smem, stm>>>(q);
        h->launches += 7;
        e = cudaMemcpyAsync(h->h_ctr, h->q_ctr, C_N * sizeof(uint32_t), cudaMemcpyDeviceToHost, stm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
        if (e != cudaSuccess) return cuda_check(h, e, "query round");
        const uint32_t n_roots = h->h_ctr[C_ROOTS], n_ed = h->h_ctr[C_EDGES], n_fail = h->h_ctr[C_FAILS];
        fails_last = n_fail;
        fails_total += n_fail;
        if (n_ed == 0) break;
        if (r == h->K - 1) exhausted = 1;
        k_q_link<<<grid_for(h, n_roots, tpb), tpb, 0, stm>>>(q);
        h->launches += 2;  // link, relabel
        if (want_forest) {
            uint32_t *F = h->q_F, *F2 = h->q_F2, *Mx = h->q_M, *Mx2 = h->q_M2;
            const uint32_t gR = grid_for(h, n_roots, tpb);
            k_q_fj_init<<<gR, tpb, 0, stm>>>(q, F, Mx, h->q_flag);
            uint32_t J = 1;
            while ((1ull << (J - 1)) < (uint64_t)n_roots) ++J;
            for (uint32_t it = 0; it < J; ++it) {
                k_q_fj_step<<<gR, tpb, 0, stm>>>(q, F, Mx, F2, Mx2);
                std::swap(F, F2);
                std::swap(Mx, Mx2);
            }
            k_q_fj_mark<<<gR, tpb, 0, stm>>>(q, F, Mx, h->q_flag);
            // q_cursor is free again: reuse it for the accept flags
            k_q_accept<<<gV, tpb, 0, stm>>>(q, h->q_flag, h->q_cursor);
            launch_scan(h->q_cursor, h->q_pos, nullptr, V, stm, h->d_scan_tmp);
            k_q_forest_write<<<gV, tpb, 0, stm>>>(q, h->q_cursor, h->q_pos, h->q_forest);
            k_q_forest_advance<<<1, 1, 0, stm>>>(q, h->q_pos);
            h->launches += J + 7;
        }
        k_q_relabel<<<gV, tpb, 0, stm>>>(q);
    }
    k_q_ncc<<<gV, tpb, 0, stm>>>(q);
    e = cudaMemcpyAsync(h->h_ctr, h->q_ctr, C_N * sizeof(uint32_t), cudaMemcpyDeviceToHost, stm);
    if (e == cudaSuccess && labels)
        e = cudaMemcpyAsync(labels, h->q_label, (size_t)V * sizeof(uint32_t), cudaMemcpyDeviceToHost, stm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
    if (e != cudaSuccess) return cuda_check(h, e, "query results");
    const uint32_t ncc = h->h_ctr[C_NCC];
    const uint32_t nf = h->h_ctr[C_FOREST];
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
