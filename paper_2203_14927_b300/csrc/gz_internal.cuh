// gz_internal.cuh -- device-side definitions shared by the CUDA sources of the
// library (never by the CPU oracle).
//
// Sketch storage ("exact-depth" form).  The paper's CubeSketch keeps NESTED rows:
// row i of column j holds every index e with h1(e) = 0 mod 2^i (Eq. 1-2), so one
// update touches rows 0..depth.  On the device each update XORs only row
// depth = min(#leading zero bits of (a*idx+b), R-1); nested row i is recovered as
// the XOR of stored rows i..R-1 (a fixed linear map, so merges commute with it).
//
// Gamma words hold gamma' (see fmix32_pre below): the paper's checksum sum of a
// bucket is gamma' ^ (gamma' >> 16).
//
// Layout: node-major; per node, K blocks of (alpha[R][7] u64, gamma'[R][7] u32).
// One CubeSketch (node, k) is therefore a contiguous 84*R-byte block, which is
// what a Boruvka round reads per node.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GZ_COLS 7

namespace gz {

struct SketchView {
    uint8_t* base;
    uint64_t node_bytes;   // K * per_k_bytes
    uint32_t per_k_bytes;  // 84 * R
    uint32_t gamma_off;    // 56 * R

    __device__ __forceinline__ uint64_t* alpha(uint32_t node, uint32_t k, uint32_t row,
                                               uint32_t j) const {
        return reinterpret_cast<uint64_t*>(base + node * node_bytes + (uint64_t)k * per_k_bytes) +
               row * GZ_COLS + j;
    }
    __device__ __forceinline__ uint32_t* gamma(uint32_t node, uint32_t k, uint32_t row,
                                               uint32_t j) const {
        return reinterpret_cast<uint32_t*>(base + node * node_bytes + (uint64_t)k * per_k_bytes +
                                           gamma_off) +
               row * GZ_COLS + j;
    }
    // start of CubeSketch (node, k): alpha block, gamma block follows at gamma_off
    __device__ __forceinline__ uint8_t* cube(uint32_t node, uint32_t k) const {
        return base + node * node_bytes + (uint64_t)k * per_k_bytes;
    }
};

// Per-column keys: depth hash a (odd), b; checksum key c.
struct Keys {
    const uint64_t* a;
    const uint64_t* b;
    const uint64_t* c;
};

// MurmurHash3's 32-bit finalizer (Appleby 2011), without its last step
// h ^= h >> 16.  That step is a linear, invertible map L over GF(2)^32, so it
// commutes with XOR sums: the device keeps gamma' = XOR of fmix32_pre values
// in every bucket, a bucket's paper checksum gamma is L(gamma'), and a
// candidate alpha is good iff gamma' == fmix32_pre(fold(alpha) ^ lo32(c)).
__device__ __forceinline__ uint32_t fmix32_pre(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    return h;
}

// L: stored gamma' -> the checksum sum gamma of Fig. cube_code.
__device__ __forceinline__ uint32_t gamma_final(uint32_t g) { return g ^ (g >> 16); }

// 32-bit fold of an edge index: lo32 ^ lo32(hi32 * 0x9E3779B9) (the identity
// below 2^32).
__device__ __forceinline__ uint32_t fold32(uint64_t idx) {
    return static_cast<uint32_t>(idx) ^ (static_cast<uint32_t>(idx >> 32) * 0x9E3779B9u);
}

// Stored form of checksum h2 (Fig. cube_code) of one index:
// h2(idx) = L(checksum_pre(c, idx)) = fmix32(fold(idx) ^ lo32(c)).
__device__ __forceinline__ uint32_t checksum_pre(uint64_t c, uint64_t idx) {
    return fmix32_pre(fold32(idx) ^ static_cast<uint32_t>(c));
}

// Depth hash: t = a*idx + b (mod 2^64), Dietzfelbinger's multiply-add-shift
// family; an index lies in nested row i iff the top i bits of t are zero.
__device__ __forceinline__ uint64_t depth_word(uint64_t a, uint64_t b, uint64_t idx) {
    return a * idx + b;
}

// Exact depth = min(leading zeros of t, R-1).
__device__ __forceinline__ uint32_t exact_depth(uint64_t t, uint32_t R) {
    uint32_t d = static_cast<uint32_t>(__clzll(static_cast<long long>(t)));
    return d < R - 1 ? d : R - 1;
}

__device__ __forceinline__ uint64_t edge_index(uint32_t x, uint32_t y, uint32_t V) {
    uint32_t lo = x < y ? x : y;
    uint32_t hi = x < y ? y : x;
    return static_cast<uint64_t>(lo) * V + hi;
}

}  // namespace gz
