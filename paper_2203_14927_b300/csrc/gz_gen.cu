// gz_gen.cu -- device twin of the host stream generator (streams.py KronSpec):
// benchmark input only, no sketch arithmetic.  See include/gz_gen.h for the
// stream definition.  Chunk c is produced by a stable compaction: a counting
// pass per block of positions, an exclusive scan of the block counts, and a
// writing pass that recomputes the flags and places every update at its rank
// in position order.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>

#include "../../include/gz_gen.h"
#include "gz_handle.cuh"

struct gz_gen {
    gz_kron_params p{};
    uint64_t* d_table = nullptr;
    uint32_t* d_cnt = nullptr;  // [2][nb] block counts (inserts, deletes)
    uint32_t* d_off = nullptr;  // [2][nb+1]
    uint32_t* h_tot = nullptr;  // pinned [2]
    uint32_t* d_scan_tmp = nullptr;
    uint64_t nb = 0;
    cudaStream_t stream = nullptr;
};

namespace {

constexpr uint32_t kThreads = 256, kPerThread = 16, kPerBlock = kThreads * kPerThread;

struct GenArgs {
    uint32_t L;
    uint64_t M;  // V - 1
    uint64_t kf0, kf1, kf2, kf3, k_kron, k_churn, k_iso, t_iso, t_churn;
    const uint64_t* table;
    uint64_t P;                    // positions per slice
    uint64_t ins_base, del_base;   // first position of each range
    int has_ins, has_del;
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void pair_at(const GenArgs& a, uint64_t pos, uint32_t& u, uint32_t& v) {
    uint64_t l = pos >> a.L, r = pos & a.M;
    const uint64_t kf[4] = {a.kf0, a.kf1, a.kf2, a.kf3};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t t = l ^ (mix64(r ^ kf[i]) & a.M);
        l = r;
        r = t;
    }
    u = (uint32_t)l;
    v = (uint32_t)r;
}

// bit 0: insert (final or churn), bit 1: delete (churn)
__device__ __forceinline__ uint32_t flags_at(const GenArgs& a, uint64_t pos, uint32_t& u, uint32_t& v) {
    pair_at(a, pos, u, v);
    if (u >= v) return 0;
    const uint64_t idx = ((uint64_t)u << a.L) + v;
    const uint32_t n11 = __popc(u & v), n00 = a.L - __popc(u | v);
    const bool kron = (mix64(idx ^ a.k_kron) >> 11) < a.table[n00 * (a.L + 1) + n11];
    const bool iso = ((mix64((uint64_t)u ^ a.k_iso) >> 11) < a.t_iso) ||
                     ((mix64((uint64_t)v ^ a.k_iso) >> 11) < a.t_iso);
    const bool fin = kron && !iso;
    const bool churn = !fin && ((mix64(idx ^ a.k_churn) >> 11) < a.t_churn);
    return (fin || churn ? 1u : 0u) | (churn ? 2u : 0u);
}

__device__ __forceinline__ uint32_t block_excl_sum(uint32_t x, uint32_t* sh, uint32_t* total) {
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
        uint32_t t = lane < kThreads / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= (uint32_t)o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const uint32_t excl = s - x + (w ? sh[w - 1] : 0);
    *total = sh[kThreads / 32 - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kThreads) k_gen_count(GenArgs a, uint32_t* cnt_ins, uint32_t* cnt_del) {
    __shared__ uint32_t sh[32];
    uint32_t ci = 0, cd = 0;
    const uint64_t first = (uint64_t)blockIdx.x * kPerBlock + (uint64_t)threadIdx.x * kPerThread;
    for (uint32_t i = 0; i < kPerThread; ++i) {
        const uint64_t off = first + i;
        if (off >= a.P) break;
        uint32_t u, v;
        if (a.has_ins) ci += flags_at(a, a.ins_base + off, u, v) & 1u;
        if (a.has_del) cd += (flags_at(a, a.del_base + off, u, v) >> 1) & 1u;
    }
    uint32_t ti, td;
    block_excl_sum(ci, sh, &ti);
    block_excl_sum(cd, sh, &td);
    if (threadIdx.x == 0) {
        cnt_ins[blockIdx.x] = ti;
        cnt_del[blockIdx.x] = td;
    }
}

__global__ void __launch_bounds__(kThreads) k_gen_write(GenArgs a, const uint32_t* off_ins, const uint32_t* off_del,
                                                        uint64_t total_ins, uint32_t* out_u, uint32_t* out_v) {
    __shared__ uint32_t sh[32];
    uint32_t ci = 0, cd = 0;
    const uint64_t first = (uint64_t)blockIdx.x * kPerBlock + (uint64_t)threadIdx.x * kPerThread;
    for (uint32_t i = 0; i < kPerThread; ++i) {
        const uint64_t off = first + i;
        if (off >= a.P) break;
        uint32_t u, v;
        if (a.has_ins) ci += flags_at(a, a.ins_base + off, u, v) & 1u;
        if (a.has_del) cd += (flags_at(a, a.del_base + off, u, v) >> 1) & 1u;
    }
    uint32_t ti, td;
    uint64_t pi = off_ins[blockIdx.x] + block_excl_sum(ci, sh, &ti);
    uint64_t pd = total_ins + off_del[blockIdx.x] + block_excl_sum(cd, sh, &td);
    for (uint32_t i = 0; i < kPerThread; ++i) {
        const uint64_t off = first + i;
        if (off >= a.P) break;
        uint32_t u, v;
        if (a.has_ins && (flags_at(a, a.ins_base + off, u, v) & 1u)) {
            out_u[pi] = u;
            out_v[pi] = v;
            ++pi;
        }
        if (a.has_del && (flags_at(a, a.del_base + off, u, v) & 2u)) {
            out_u[pd] = u;
            out_v[pd] = v;
            ++pd;
        }
    }
}

}  // namespace

extern "C" {

gz_status gz_gen_kron_create(const gz_kron_params* p, const uint64_t* table, void* stream, gz_gen** out) {
    if (!p || !table || !out) return GZ_EINVAL;
    *out = nullptr;
    if (p->L < 1 || p->L > 31 || p->slice_log2 > 2 * p->L || p->slice_log2 > 40) return GZ_EINVAL;
    gz_gen* g = new (std::nothrow) gz_gen();
    if (!g) return GZ_ENOMEM;
    g->p = *p;
    g->stream = static_cast<cudaStream_t>(stream);
    const uint64_t P = 1ull << p->slice_log2;
    g->nb = (P + kPerBlock - 1) / kPerBlock;
    const size_t tn = (size_t)(p->L + 1) * (p->L + 1);
    cudaError_t e = cudaMalloc(&g->d_table, tn * 8);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_table, table, tn * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_cnt, 2 * g->nb * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_off, 2 * (g->nb + 1) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_tot, 2 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_scan_tmp, (g->nb / 1024 + 2) * 4);
    if (e != cudaSuccess) {
        gz_gen_destroy(g);
        return e == cudaErrorMemoryAllocation ? GZ_ENOMEM : GZ_ECUDA;
    }
    *out = g;
    return GZ_OK;
}

gz_status gz_gen_kron_num_chunks(gz_gen* g, uint64_t* n_chunks) {
    if (!g || !n_chunks) return GZ_EINVAL;
    const uint64_t slices = std::max<uint64_t>(1, (1ull << (2 * g->p.L)) >> g->p.slice_log2);
    *n_chunks = slices + 1;
    return GZ_OK;
}

gz_status gz_gen_kron_chunk(gz_gen* g, uint64_t c, uint32_t* u, uint32_t* v, uint64_t capacity, uint64_t* n) {
    if (!g || !u || !v || !n) return GZ_EINVAL;
    uint64_t nch;
    gz_gen_kron_num_chunks(g, &nch);
    if (c >= nch) return GZ_EINVAL;
    GenArgs a;
    a.L = g->p.L;
    a.M = (1ull << g->p.L) - 1;
    a.kf0 = g->p.k_feistel[0];
    a.kf1 = g->p.k_feistel[1];
    a.kf2 = g->p.k_feistel[2];
    a.kf3 = g->p.k_feistel[3];
    a.k_kron = g->p.k_kron;
    a.k_churn = g->p.k_churn;
    a.k_iso = g->p.k_iso;
    a.t_iso = g->p.t_iso;
    a.t_churn = g->p.t_churn;
    a.table = g->d_table;
    a.P = 1ull << g->p.slice_log2;
    a.has_ins = c + 1 < nch;
    a.has_del = c >= 1;
    a.ins_base = c * a.P;
    a.del_base = c >= 1 ? (c - 1) * a.P : 0;
    cudaStream_t s = g->stream;
    const uint32_t nb = (uint32_t)g->nb;
    k_gen_count<<<nb, kThreads, 0, s>>>(a, g->d_cnt, g->d_cnt + nb);
    gz::launch_scan(g->d_cnt, g->d_off, nullptr, nullptr, nb, s, g->d_scan_tmp);
    gz::launch_scan(g->d_cnt + nb, g->d_off + nb + 1, nullptr, nullptr, nb, s, g->d_scan_tmp);
    cudaError_t e = cudaMemcpyAsync(&g->h_tot[0], g->d_off + nb, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&g->h_tot[1], g->d_off + nb + 1 + nb, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return GZ_ECUDA;
    const uint64_t ti = g->h_tot[0], td = g->h_tot[1];
    if (ti + td > capacity) return GZ_EINVAL;
    k_gen_write<<<nb, kThreads, 0, s>>>(a, g->d_off, g->d_off + nb + 1, ti, u, v);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return GZ_ECUDA;
    *n = ti + td;
    return GZ_OK;
}

gz_status gz_gen_destroy(gz_gen* g) {
    if (!g) return GZ_EINVAL;
    if (g->d_table) cudaFree(g->d_table);
    if (g->d_cnt) cudaFree(g->d_cnt);
    if (g->d_off) cudaFree(g->d_off);
    if (g->h_tot) cudaFreeHost(g->h_tot);
    if (g->d_scan_tmp) cudaFree(g->d_scan_tmp);
    delete g;
    return GZ_OK;
}

}  // extern "C"
