// gz_internal.cuh -- device-side definitions shared by the CUDA sources of the
// library (never by the CPU oracle).
//
// Sketch storage ("exact-depth" form).  The paper's CubeSketch keeps NESTED rows:
// row i of column j holds every index e with h1(e) = 0 mod 2^i (Eq. 1-2), so one
// update touches rows 0..depth.  On the device each update XORs only row
// depth (edge_depth below); nested row i is recovered as the XOR of stored rows
// i..R-1 (a fixed linear map, so merges commute with it).
//
// Layout: node-major; per node, K blocks of (alpha[R][7] u64, gamma[R][7] u32).
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

// Hash keys of the node sketches: kKeyWords 32-bit words per CubeSketch column,
// stored word-major (word w of column col at w[w * ncol + col], so a thread per
// column loads them coalesced).  Words [0, 128) hold the depth hash h1's
// pieces, [128, 256) the checksum h2's, three words (k0, k1, k2) per piece.
constexpr uint32_t kKeyWords = 256;
constexpr uint32_t kH2Words = 128;

struct Keys {
    const uint32_t* w;  // kKeyWords * ncol
    uint32_t ncol;
    __device__ __forceinline__ uint32_t at(uint32_t word, uint32_t col) const { return w[word * ncol + col]; }
};

// Piece geometry for V vertices: L = ceil(log2 V) (every id < 2^L), piece width
// p = min(16, 33 - L), m1 = ceil((R-1)/p) pieces for h1 (R = 2L) and
// m2 = ceil(32/p) for h2 (2 for every V <= 2^17).
struct PieceGeo {
    uint32_t p, m1, m2;
};

__host__ __device__ inline PieceGeo piece_geo(uint32_t V) {
    uint32_t L = 0;
    while ((1ull << L) < V) ++L;
    PieceGeo g;
    g.p = 33 - L < 16 ? 33 - L : 16;
    g.m1 = (2 * L - 1 + g.p - 1) / g.p;
    g.m2 = (32 + g.p - 1) / g.p;
    return g;
}

// One piece on the endpoint pair (u, v): (k0*u + k1*v + k2) mod 2^32, whose top
// p bits are the hash bits (multiply-add-shift over a vector of two L-bit words,
// Dietzfelbinger 1996 / Thorup 2015: strongly universal since 32 >= L + p - 1).
// Concatenated pieces (the first most significant), left-aligned in 64 bits.
__device__ __forceinline__ uint64_t pieces_cat(const Keys& k, uint32_t base, uint32_t col, uint32_t m,
                                               uint32_t p, uint32_t u, uint32_t v) {
    uint64_t acc = 0;
    for (uint32_t i = 0; i < m; ++i) {
        const uint32_t t = k.at(base + 3 * i, col) * u + k.at(base + 3 * i + 1, col) * v + k.at(base + 3 * i + 2, col);
        acc |= (uint64_t)(t >> (32 - p)) << (64 - p * (i + 1));
    }
    return acc;
}

// Exact depth of edge (u, v) in column col: the leading zeros of h1's pieces,
// capped at R-1 (an index lies in nested rows 0..depth, Fig. cube_code).
__device__ __forceinline__ uint32_t edge_depth(const Keys& k, const PieceGeo& g, uint32_t R, uint32_t col,
                                               uint32_t u, uint32_t v) {
    const uint32_t d = (uint32_t)__clzll((long long)pieces_cat(k, 0, col, g.m1, g.p, u, v));
    return d < R - 1 ? d : R - 1;
}

// Checksum h2 of edge (u, v) in column col: the first 32 bits of its pieces.
__device__ __forceinline__ uint32_t edge_checksum(const Keys& k, const PieceGeo& g, uint32_t col, uint32_t u,
                                                  uint32_t v) {
    return (uint32_t)(pieces_cat(k, kH2Words, col, g.m2, g.p, u, v) >> 32);
}

__device__ __forceinline__ uint64_t edge_index(uint32_t x, uint32_t y, uint32_t V) {
    uint32_t lo = x < y ? x : y;
    uint32_t hi = x < y ? y : x;
    return static_cast<uint64_t>(lo) * V + hi;
}

}  // namespace gz
