/*
 * gz_oracle_l0.c -- TEST INFRASTRUCTURE ONLY (part of the oracle library).
 *
 * Single-vector l0 sketches for the micro-benchmark of Fig. l0speedup: the
 * standard l0 sampler of Fig. agm_code and, beside it, CubeSketch
 * (Fig. cube_code) applied to a plain vector of length n.  Plain
 * single-threaded C, shared with nothing on the CUDA side.
 *
 * Readings (the paper gives the algorithm, not its constants):
 *   vector     positions 1..n (0 is never used), n >= 2; deltas are +-1.
 *   geometry   7 columns (delta = 1/100, as for the node sketches) and
 *              R = ceil(log2 n) rows, the depth cap of both samplers.
 *   keys       column j: a = SM(seed, 5j) | 1, b = SM(seed, 5j+1),
 *              c0, c1, c2 = SM(seed, 5j+2), SM(seed, 5j+3), SM(seed, 5j+4)
 *              (SplitMix64).
 *   membership both samplers put x into rows 0..d of column j with
 *              d = min(clz64(a*x + b), R-1): Fig. agm_code's
 *              "col_hash[row-1] == 0" loop with the bit order of
 *              Fig. cube_code (identical membership by the paper's own remark
 *              in Section 3.2).
 *   standard   bucket (a, b, c): a += x*delta and b += delta in two's
 *              complement 64-bit arithmetic, c += delta * r_j^x (mod p) with
 *              p = 2^61 - 1 (a Mersenne prime above every n used) and
 *              r_j = 1 + (c0 mod (p - 1)).  Query (Fig. agm_code): the first
 *              bucket, columns then rows ascending, with b != 0, b | a,
 *              1 <= a/b <= n and c == (b mod p) * r_j^(a/b) (mod p) yields
 *              (a/b, b); all buckets zero -> EMPTY, else FAIL.
 *   CubeSketch bucket (alpha u64, gamma u32): alpha ^= x, gamma ^= h2(x) with
 *              h2(x) = ((c0*x0 + c1*x1 + c2) mod 2^64) >> 32 over the two
 *              32-bit words x0, x1 of the position (positions are not edges,
 *              so the node sketches' pair hashes do not apply); a delta of -1
 *              is the same toggle.
 * Layout of one sketch: standard a[7][R], b[7][R], c[7][R] (u64 each);
 * CubeSketch alpha[7][R] (u64) then gamma[7][R] (u32).
 */
#include <stdint.h>
#include <stdlib.h>

#define L0_COLS 7
#define P61 ((((uint64_t)1) << 61) - 1)

uint64_t gzo_splitmix64_at(uint64_t s, uint64_t n);
/* CubeSketch checksum of a vector position x: multiply-add-shift over the two
 * 32-bit words x0, x1 of x with 64-bit arithmetic (Dietzfelbinger 1996; the
 * vector form in Thorup 2015), ((c0*x0 + c1*x1 + c2) mod 2^64) >> 32,
 * strongly universal for 32-bit words and 32 output bits. */
static uint32_t l0_checksum(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t x)
{
    uint64_t x0 = x & 0xFFFFFFFFu, x1 = x >> 32;
    return (uint32_t)((c0 * x0 + c1 * x1 + c2) >> 32);
}

/* rows of a length-n vector sketch: ceil(log2 n), at least 1 */
uint32_t gzo_l0_rows(uint64_t n)
{
    uint32_t r = 0;
    while (r < 64 && (((uint64_t)1) << r) < n) r++;
    return r ? r : 1;
}

/* x * y mod 2^61 - 1 for x, y < 2^61: the 122-bit product, then the folding
 * identity 2^61 = 1 (mod p). */
uint64_t gzo_mulmod61(uint64_t x, uint64_t y)
{
    unsigned __int128 t = (unsigned __int128)x * y;
    uint64_t s = (uint64_t)(t & P61) + (uint64_t)(t >> 61);
    s = (s & P61) + (s >> 61);
    return s >= P61 ? s - P61 : s;
}

/* r^e mod 2^61 - 1 by square-and-multiply, most significant bit first */
uint64_t gzo_powmod61(uint64_t r, uint64_t e)
{
    uint64_t acc = 1;
    for (int bit = 63; bit >= 0; bit--) {
        acc = gzo_mulmod61(acc, acc);
        if ((e >> bit) & 1u) acc = gzo_mulmod61(acc, r);
    }
    return acc;
}

static uint32_t l0_depth(uint64_t a, uint64_t b, uint64_t x, uint32_t R)
{
    uint64_t t = a * x + b;
    uint32_t d = 0;
    while (d < 64 && !((t >> (63 - d)) & 1u)) d++;
    return d < R - 1 ? d : R - 1;
}

static uint64_t std_root(uint64_t c)
{
    return 1 + c % (P61 - 1);
}

/* Apply m updates (x[i], delta[i]) to one sketch.  kind 0 = CubeSketch,
 * 1 = standard.  delta may be NULL (all +1).  Returns 0, or -1 for a
 * position outside 1..n or a delta other than +-1 (nothing changed). */
int gzo_l0_update(int kind, uint64_t n, uint64_t seed, size_t m, const uint64_t *x,
                  const int32_t *delta, void *buckets)
{
    if (n < 2 || (kind != 0 && kind != 1)) return -1;
    for (size_t i = 0; i < m; i++) {
        if (x[i] < 1 || x[i] > n) return -1;
        if (delta && delta[i] != 1 && delta[i] != -1) return -1;
    }
    const uint32_t R = gzo_l0_rows(n);
    const size_t nb = (size_t)L0_COLS * R;
    for (size_t i = 0; i < m; i++) {
        const int64_t dl = delta ? delta[i] : 1;
        for (uint32_t j = 0; j < L0_COLS; j++) {
            uint64_t ka = gzo_splitmix64_at(seed, 5 * j) | 1u;
            uint64_t kb = gzo_splitmix64_at(seed, 5 * j + 1);
            uint64_t kc0 = gzo_splitmix64_at(seed, 5 * j + 2);
            uint64_t kc1 = gzo_splitmix64_at(seed, 5 * j + 3);
            uint64_t kc2 = gzo_splitmix64_at(seed, 5 * j + 4);
            uint32_t d = l0_depth(ka, kb, x[i], R);
            if (kind == 0) {
                uint64_t *A = (uint64_t *)buckets + (size_t)j * R;
                uint32_t *G = (uint32_t *)((uint64_t *)buckets + nb) + (size_t)j * R;
                uint32_t g = l0_checksum(kc0, kc1, kc2, x[i]);
                for (uint32_t row = 0; row <= d; row++) {
                    A[row] ^= x[i];
                    G[row] ^= g;
                }
            } else {
                uint64_t *A = (uint64_t *)buckets + (size_t)j * R;
                uint64_t *B = A + nb;
                uint64_t *C = B + nb;
                uint64_t chk = gzo_powmod61(std_root(kc0), x[i]);
                uint64_t add = dl > 0 ? chk : (chk ? P61 - chk : 0);
                for (uint32_t row = 0; row <= d; row++) {
                    A[row] += x[i] * (uint64_t)dl;
                    B[row] += (uint64_t)dl;
                    C[row] += add;
                    if (C[row] >= P61) C[row] -= P61;
                }
            }
        }
    }
    return 0;
}

/* Query one sketch: returns the sampled position (> 0) and, for the standard
 * sampler, its value in *value (CubeSketch: 1); -1 EMPTY, -2 FAIL. */
int64_t gzo_l0_query(int kind, uint64_t n, uint64_t seed, const void *buckets, int64_t *value)
{
    const uint32_t R = gzo_l0_rows(n);
    const size_t nb = (size_t)L0_COLS * R;
    int nonzero = 0;
    for (uint32_t j = 0; j < L0_COLS; j++) {
        uint64_t kc0 = gzo_splitmix64_at(seed, 5 * j + 2);
        uint64_t kc1 = gzo_splitmix64_at(seed, 5 * j + 3);
        uint64_t kc2 = gzo_splitmix64_at(seed, 5 * j + 4);
        for (uint32_t row = 0; row < R; row++) {
            if (kind == 0) {
                uint64_t alpha = ((const uint64_t *)buckets)[(size_t)j * R + row];
                uint32_t gamma = ((const uint32_t *)((const uint64_t *)buckets + nb))[(size_t)j * R + row];
                if (alpha == 0 && gamma == 0) continue;
                nonzero = 1;
                if (alpha < 1 || alpha > n || gamma != l0_checksum(kc0, kc1, kc2, alpha)) continue;
                if (value) *value = 1;
                return (int64_t)alpha;
            } else {
                const uint64_t *A = (const uint64_t *)buckets + (size_t)j * R;
                int64_t a = (int64_t)A[row], b = (int64_t)A[nb + row];
                uint64_t c = A[2 * nb + row];
                if (a == 0 && b == 0 && c == 0) continue;
                nonzero = 1;
                if (b == 0 || a % b != 0) continue;
                int64_t v = a / b;
                if (v < 1 || (uint64_t)v > n) continue;
                uint64_t bm = b > 0 ? (uint64_t)b % P61 : P61 - ((uint64_t)(-b) % P61);
                if (bm == P61) bm = 0;
                if (c != gzo_mulmod61(bm, gzo_powmod61(std_root(kc0), (uint64_t)v))) continue;
                if (value) *value = b;
                return v;
            }
        }
    }
    return nonzero ? -2 : -1;
}
