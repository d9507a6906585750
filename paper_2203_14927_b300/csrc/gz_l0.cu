// gz_l0.cu -- single-vector l0 sketches for the micro-benchmark of Fig.
// l0speedup: the standard l0 sampler of Fig. agm_code beside CubeSketch
// (Fig. cube_code) on a plain vector of length n.
//
// Both samplers put position x into rows 0..d of column j, with
// d = min(clz64(a_j*x + b_j), R-1) and R = ceil(log2 n) (the membership rule
// is the same by Section 3.2's own remark); they differ in the bucket update:
//   CubeSketch  alpha ^= x, gamma ^= h2(x) (multiply-add-shift over the two
//               32-bit words of x, keys c0, c1, c2; see pos_checksum);
//   standard    a += x*delta, b += delta (two's complement 64-bit),
//               c += delta * r_j^x mod p, p = 2^61 - 1, r_j = 1 + c0_j mod (p-1):
//               a modular exponentiation per column update (Section 3.1).
// One thread owns one column of one sketch and applies the sketch's updates in
// order; the buckets stay in the paper's nested form (rows 0..d per update),
// since this is the paper's own per-update comparison, not the node-sketch
// path.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gz.h"

namespace {

constexpr uint64_t kP61 = (1ull << 61) - 1;

__device__ __forceinline__ uint64_t sm64_at(uint64_t s, uint64_t n) {
    // n-th SplitMix64 output from seed s (Steele, Lea & Flood 2014)
    uint64_t z = s + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// x*y mod 2^61-1 for x, y < 2^61: fold the 122-bit product with 2^61 = 1
__device__ __forceinline__ uint64_t mulmod61(uint64_t x, uint64_t y) {
    const uint64_t lo = x * y, hi = __umul64hi(x, y);
    uint64_t s = (lo & kP61) + ((hi << 3) | (lo >> 61));
    s = (s & kP61) + (s >> 61);
    return s >= kP61 ? s - kP61 : s;
}

// Position hashes of the vector sketches (positions are not edges, so the node
// sketches' pair hashes do not apply): depth = min(leading zeros of
// (a*x + b) mod 2^64, R-1) and checksum ((c0*x0 + c1*x1 + c2) mod 2^64) >> 32
// over the 32-bit words x0, x1 of x (multiply-add-shift, Dietzfelbinger 1996).
__device__ __forceinline__ uint32_t pos_depth(uint64_t a, uint64_t b, uint64_t x, uint32_t R) {
    const uint32_t d = (uint32_t)__clzll((long long)(a * x + b));
    return d < R - 1 ? d : R - 1;
}
__device__ __forceinline__ uint32_t pos_checksum(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t x) {
    return (uint32_t)((c0 * (uint32_t)x + c1 * (x >> 32) + c2) >> 32);
}

// r^e mod 2^61-1, square-and-multiply from the highest set bit of e
__device__ __forceinline__ uint64_t powmod61(uint64_t r, uint64_t e) {
    uint64_t acc = 1;
    for (int bit = 63 - __clzll((long long)e); bit >= 0; --bit) {
        acc = mulmod61(acc, acc);
        if ((e >> bit) & 1u) acc = mulmod61(acc, r);
    }
    return acc;
}

template <int kKind>
__global__ void __launch_bounds__(224) k_l0_update(uint64_t n, uint32_t R, uint64_t seed, uint32_t sketches,
                                                   uint32_t m, const uint64_t* __restrict__ x,
                                                   const int32_t* __restrict__ delta, uint8_t* buckets,
                                                   uint32_t bytes_per_sketch) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)sketches * 7) return;
    const uint32_t s = (uint32_t)(t / 7), j = (uint32_t)(t % 7);
    // column j's keys: SplitMix64 outputs 5j .. 5j+4 (the node sketches' schedule)
    const uint64_t ka = sm64_at(seed, 5 * j) | 1u, kb = sm64_at(seed, 5 * j + 1);
    const uint64_t kc0 = sm64_at(seed, 5 * j + 2), kc1 = sm64_at(seed, 5 * j + 3), kc2 = sm64_at(seed, 5 * j + 4);
    uint8_t* base = buckets + (uint64_t)s * bytes_per_sketch;
    const uint64_t* xs = x + (uint64_t)s * m;
    const int32_t* ds = delta ? delta + (uint64_t)s * m : nullptr;
    if (kKind == 0) {
        uint64_t* A = reinterpret_cast<uint64_t*>(base) + (uint64_t)j * R;
        uint32_t* G = reinterpret_cast<uint32_t*>(reinterpret_cast<uint64_t*>(base) + 7ull * R) + (uint64_t)j * R;
        for (uint32_t i = 0; i < m; ++i) {
            const uint64_t xi = xs[i];
            const uint32_t d = pos_depth(ka, kb, xi, R);
            const uint32_t g = pos_checksum(kc0, kc1, kc2, xi);
            for (uint32_t row = 0; row <= d; ++row) {
                A[row] ^= xi;
                G[row] ^= g;
            }
        }
    } else {
        uint64_t* A = reinterpret_cast<uint64_t*>(base) + (uint64_t)j * R;
        uint64_t* B = A + 7ull * R;
        uint64_t* C = B + 7ull * R;
        const uint64_t r = 1 + kc0 % (kP61 - 1);
        for (uint32_t i = 0; i < m; ++i) {
            const uint64_t xi = xs[i];
            const int64_t dl = ds ? ds[i] : 1;
            const uint32_t d = pos_depth(ka, kb, xi, R);
            const uint64_t chk = powmod61(r, xi);
            const uint64_t add = dl > 0 ? chk : (chk ? kP61 - chk : 0);
            for (uint32_t row = 0; row <= d; ++row) {
                A[row] += xi * (uint64_t)dl;
                B[row] += (uint64_t)dl;
                uint64_t c = C[row] + add;
                C[row] = c >= kP61 ? c - kP61 : c;
            }
        }
    }
}

}  // namespace

extern "C" gz_status gz_l0_geometry(uint64_t n, uint32_t* rows, uint32_t* bytes_cube, uint32_t* bytes_standard) {
    if (n < 2) return GZ_EINVAL;
    uint32_t r = 0;
    while (r < 64 && (1ull << r) < n) ++r;
    if (rows) *rows = r;
    // 84R bytes rounded up to 8, so every sketch's alpha words stay 8-byte aligned
    if (bytes_cube) *bytes_cube = (7u * r * 12u + 7u) & ~7u;
    if (bytes_standard) *bytes_standard = 7u * r * 24u;
    return GZ_OK;
}

extern "C" gz_status gz_l0_update(int kind, uint64_t n, uint64_t seed, uint32_t sketches, uint32_t m,
                                  const uint64_t* x, const int32_t* delta, void* buckets, void* stream) {
    if ((kind != GZ_L0_CUBE && kind != GZ_L0_STANDARD) || n < 2 || n >= (1ull << 61) || !buckets ||
        (sketches && m && !x))
        return GZ_EINVAL;
    if (!sketches || !m) return GZ_OK;
    uint32_t R = 0, bc = 0, bs = 0;
    gz_l0_geometry(n, &R, &bc, &bs);
    const uint64_t threads = (uint64_t)sketches * 7;
    const uint32_t grid = (uint32_t)((threads + 223) / 224);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (kind == GZ_L0_CUBE)
        k_l0_update<0><<<grid, 224, 0, st>>>(n, R, seed, sketches, m, x, delta, static_cast<uint8_t*>(buckets), bc);
    else
        k_l0_update<1><<<grid, 224, 0, st>>>(n, R, seed, sketches, m, x, delta, static_cast<uint8_t*>(buckets), bs);
    return cudaGetLastError() == cudaSuccess ? GZ_OK : GZ_ECUDA;
}
