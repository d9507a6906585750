/*
 * gz_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the GraphZeppelin hot path
 * (Tench et al., SIGMOD 2022, arXiv 2203.14927): CubeSketch ingestion of an
 * insert/delete edge stream into per-node sketches, and Boruvka connected
 * components over those sketches.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load this library.  It shares no
 * code, header, table or constant generator with the CUDA library; the two are
 * written separately from the same written definitions.
 *
 * Every sketch here is kept in the paper's NESTED form: bucket (row i, col j)
 * holds the XOR over all indices e with h1(e) = 0 mod 2^i (Section 3.2,
 * Eq. 1-2).  The layout of one node sketch is alpha[k][j][row] (u64) and
 * gamma[k][j][row] (u32), k < K CubeSketches, j < 7 columns, row < R rows.
 *
 * Readings where the paper is silent (listed again with reasons in the design
 * notes of the repository):
 *   geometry   R = 2*ceil(log2 V) rows, 7 columns (Section 5.1 "Sketch updates",
 *              delta = 1/100), K = ceil(log_{3/2} V) CubeSketches per node
 *              (Section 5, total size ~280 V log^2 V bytes; Table tab:size).
 *   index      idx(u,v) = min(u,v)*V + max(u,v)  (a position of the
 *              characteristic vector, Section 2.2); never 0.
 *   pieces     the hashes are built from "pieces" on the endpoint pair of an
 *              edge e = (u, v), u < v < V.  With L = ceil(log2 V) (so u, v < 2^L)
 *              and piece width p = min(16, 33 - L), a piece with keys (k0, k1, k2) is
 *              the top p bits of (k0*u + k1*v + k2) mod 2^32: multiply-add-shift
 *              over a vector of two L-bit words (Dietzfelbinger, STACS 1996;
 *              the vector form in Thorup, "High Speed Hashing for Integers and
 *              Strings", 2015), strongly universal (2-wise independent, as
 *              Section 3.2 asks of h1 and h2) because 32 >= L + p - 1.  Pieces
 *              with independent keys are concatenated (the first piece gives
 *              the most significant bits); the concatenation is strongly
 *              universal too.  e <-> (u, v) is a bijection, so these are hashes
 *              of the index e.
 *   keys       32-bit words: for column col = 7k+j, hash h (1 or 2), piece i
 *              and coefficient c, lo32(SM(seed, 256*col + 128*(h-1) + 3i + c)),
 *              SM(s,n) being the n-th output (n >= 0) of SplitMix64 (Steele,
 *              Lea & Flood, OOPSLA 2014) started at s.
 *   h1         col_hash of Fig. cube_code: H1 = m1 = ceil((R-1)/p) pieces,
 *              read from its most significant bit: bit i of col_hash is the
 *              i-th bit of H1, so "h1(e) = 0 mod 2^i" means the first i bits
 *              of H1 are zero.  Bit order of col_hash: bit 0 first.
 *   h2         checksum of Fig. cube_code: the first 32 bits of
 *              m2 = ceil(32/p) pieces.
 *   rows       the update loop of Fig. cube_code also stops at row R.
 *   query      Fig. cube_code's scan (columns ascending, rows ascending); a
 *              bucket is taken when alpha decodes to u < v < V (h2 is defined
 *              on edges) AND gamma == h2(alpha) AND exactly one endpoint lies
 *              in the queried component.  All buckets zero -> EMPTY, else no
 *              taker -> FAIL.
 *   Boruvka    Section 2.2 / Lemma (CC I/O) proof: round r uses CubeSketch r;
 *              components are processed by ascending minimum vertex id; the
 *              union keeps the smaller root, so every label is the minimum
 *              vertex id of its component; a round without a sampled edge
 *              ends the query.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GZO_COLS 7

/* ---------------------------------------------------------------- hashing */

/* n-th output of SplitMix64 (Steele, Lea & Flood 2014) seeded with s: the
 * state advances by the golden-ratio increment before every output. */
uint64_t gzo_splitmix64_at(uint64_t s, uint64_t n)
{
    uint64_t z = s + (n + 1u) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t bitreverse64(uint64_t x)
{
    uint64_t r = 0;
    for (int i = 0; i < 64; i++) {
        r = (r << 1) | (x & 1u);
        x >>= 1;
    }
    return r;
}

/* L = ceil(log2 V): every vertex id is below 2^L */
static uint32_t id_bits(uint32_t V)
{
    uint32_t L = 0;
    while (((uint64_t)1 << L) < (uint64_t)V) L++;
    return L;
}

/* Piece width p = min(16, 33 - L) and the pieces of h1 (ceil((R-1)/p),
 * R = 2L) and of h2 (ceil(32/p)). */
void gzo_pieces(uint32_t V, uint32_t *p, uint32_t *m1, uint32_t *m2)
{
    uint32_t L = id_bits(V), w = 33 - L < 16 ? 33 - L : 16, need1 = 2 * L - 1;
    *p = w;
    *m1 = (need1 + w - 1) / w;
    *m2 = (32 + w - 1) / w;
}

/* The concatenation of m pieces with keys k[3i], k[3i+1], k[3i+2] on (u, v),
 * left-aligned in 64 bits (m*p <= 62 for every V <= 2^31). */
static uint64_t pieces(const uint32_t *k, uint32_t m, uint32_t p, uint32_t u, uint32_t v)
{
    uint64_t acc = 0;
    for (uint32_t i = 0; i < m; i++) {
        uint32_t t = k[3 * i] * u + k[3 * i + 1] * v + k[3 * i + 2];   /* mod 2^32 */
        uint64_t top = t >> (32 - p);
        acc |= top << (64 - p * (i + 1));
    }
    return acc;
}

/* col_hash of Fig. cube_code for edge index e (u = e / V < v = e % V):
 * bit i is the i-th bit of H1 counted from its most significant end.  k1
 * holds the h1 keys of one column (3 words per piece). */
uint64_t gzo_h1(uint32_t V, const uint32_t *k1, uint64_t e)
{
    uint32_t p, m1, m2;
    gzo_pieces(V, &p, &m1, &m2);
    return bitreverse64(pieces(k1, m1, p, (uint32_t)(e / V), (uint32_t)(e % V)));
}

/* checksum of Fig. cube_code for edge index e: the first 32 bits of the h2
 * pieces.  k2 holds the h2 keys of one column. */
uint32_t gzo_h2(uint32_t V, const uint32_t *k2, uint64_t e)
{
    uint32_t p, m1, m2;
    gzo_pieces(V, &p, &m1, &m2);
    return (uint32_t)(pieces(k2, m2, p, (uint32_t)(e / V), (uint32_t)(e % V)) >> 32);
}

/* ---------------------------------------------------------------- geometry */

/* R = 2*ceil(log2 V) rows ("log(V^2) x 7" buckets, Section 5.1) and
 * K = ceil(log_{3/2} V) CubeSketches per node (Section 5 and Table tab:size).
 * K is the least k with (3/2)^k >= V, i.e. 3^k >= V * 2^k, found exactly. */
int gzo_geometry(uint32_t V, uint32_t *K, uint32_t *R)
{
    if (V < 2) return -1;
    uint32_t L = 0;
    while (((uint64_t)1 << L) < (uint64_t)V) L++;
    unsigned __int128 p3 = 1, v2 = V;
    uint32_t k = 0;
    while (p3 < v2) { p3 *= 3; v2 *= 2; k++; }
    *K = k;
    *R = 2 * L;
    return 0;
}

/* Hash keys of all K*7 columns (k,j), col = 7k+j: GZO_KEYS 32-bit words per
 * column, the h1 pieces' keys at [0, 128) and the h2 pieces' at [128, 256);
 * word w of column col is lo32(SM(seed, 256*col + w)). */
#define GZO_KEYS 256
void gzo_keys(uint64_t seed, uint32_t K, uint32_t *keys)
{
    for (uint64_t col = 0; col < (uint64_t)K * GZO_COLS; col++)
        for (uint32_t w = 0; w < GZO_KEYS; w++)
            keys[col * GZO_KEYS + w] = (uint32_t)gzo_splitmix64_at(seed, GZO_KEYS * col + w);
}

typedef struct {
    uint32_t V, K, R;
    uint32_t *keys;   /* GZO_KEYS words per column */
} gzo_ctx;

static int ctx_open(gzo_ctx *x, uint32_t V, uint64_t seed)
{
    if (gzo_geometry(V, &x->K, &x->R)) return -1;
    x->V = V;
    size_t ncol = (size_t)x->K * GZO_COLS;
    x->keys = malloc(ncol * GZO_KEYS * 4);
    if (!x->keys) return -2;
    gzo_keys(seed, x->K, x->keys);
    return 0;
}

static void ctx_close(gzo_ctx *x)
{
    free(x->keys);
}

/* words of one node sketch: K*7*R buckets */
static size_t node_buckets(const gzo_ctx *x)
{
    return (size_t)x->K * GZO_COLS * x->R;
}

/* ---------------------------------------------------------------- update */

/* update_sketch of Fig. cube_code applied to CubeSketch k of one node:
 * for every column, rows 0.. while row == 0 or bit (row-1) of col_hash is 0,
 * alpha ^= idx and gamma ^= checksum. */
static void cubesketch_update(const gzo_ctx *x, uint32_t k,
                              uint64_t *alpha_k, uint32_t *gamma_k, uint64_t idx)
{
    for (uint32_t j = 0; j < GZO_COLS; j++) {
        size_t col = (size_t)k * GZO_COLS + j;
        const uint32_t *kc = x->keys + col * GZO_KEYS;
        uint64_t col_hash = gzo_h1(x->V, kc, idx);
        uint32_t checksum = gzo_h2(x->V, kc + 128, idx);
        uint64_t *A = alpha_k + (size_t)j * x->R;
        uint32_t *G = gamma_k + (size_t)j * x->R;
        uint32_t row = 0;
        while (row < x->R && (row == 0 || ((col_hash >> (row - 1)) & 1u) == 0)) {
            A[row] ^= idx;
            G[row] ^= checksum;
            row++;
        }
    }
}

/* Toggle position idx in every CubeSketch of one node sketch. */
static void node_update(const gzo_ctx *x, uint64_t *alpha_node,
                        uint32_t *gamma_node, uint64_t idx)
{
    size_t per_k = (size_t)GZO_COLS * x->R;
    for (uint32_t k = 0; k < x->K; k++)
        cubesketch_update(x, k, alpha_node + k * per_k, gamma_node + k * per_k, idx);
}

/* Apply a stream of n updates (u[i], v[i]) to the sketches of all V nodes
 * (Section 2.2: each update touches the vectors of both endpoints).  The
 * arrays alpha (V*K*7*R u64) and gamma (V*K*7*R u32) are updated in place.
 * Returns 0, or -1 for an invalid update (u == v or an id >= V) in which case
 * nothing is changed (the whole stream is checked first). */
int gzo_ingest(uint32_t V, uint64_t seed, size_t n, const uint32_t *u,
               const uint32_t *v, uint64_t *alpha, uint32_t *gamma)
{
    for (size_t i = 0; i < n; i++)
        if (u[i] == v[i] || u[i] >= V || v[i] >= V) return -1;
    gzo_ctx x;
    if (ctx_open(&x, V, seed)) return -2;
    size_t nb = node_buckets(&x);
    for (size_t i = 0; i < n; i++) {
        uint32_t lo = u[i] < v[i] ? u[i] : v[i];
        uint32_t hi = u[i] < v[i] ? v[i] : u[i];
        uint64_t idx = (uint64_t)lo * V + hi;
        node_update(&x, alpha + (size_t)lo * nb, gamma + (size_t)lo * nb, idx);
        node_update(&x, alpha + (size_t)hi * nb, gamma + (size_t)hi * nb, idx);
    }
    ctx_close(&x);
    return 0;
}

/* Sketch ONE node from its list of net neighbours (its characteristic vector
 * directly, which linearity makes equal to sketching any stream whose net
 * graph it is).  alpha/gamma hold one node sketch and are overwritten. */
int gzo_sketch_node(uint32_t V, uint64_t seed, uint32_t node, size_t deg,
                    const uint32_t *nbr, uint64_t *alpha, uint32_t *gamma)
{
    gzo_ctx x;
    if (node >= V) return -1;
    for (size_t i = 0; i < deg; i++)
        if (nbr[i] >= V || nbr[i] == node) return -1;
    if (ctx_open(&x, V, seed)) return -2;
    size_t nb = node_buckets(&x);
    memset(alpha, 0, nb * 8);
    memset(gamma, 0, nb * 4);
    for (size_t i = 0; i < deg; i++) {
        uint32_t lo = node < nbr[i] ? node : nbr[i];
        uint32_t hi = node < nbr[i] ? nbr[i] : node;
        node_update(&x, alpha, gamma, (uint64_t)lo * V + hi);
    }
    ctx_close(&x);
    return 0;
}

/* ---------------------------------------------------------------- query */

#define GZO_EMPTY (-1)
#define GZO_FAIL  (-2)

/* query_sketch of Fig. cube_code on CubeSketch k of a component sketch S
 * (nested form, layout [j][row]).  label[] maps vertices to component ids;
 * comp is the queried component.  Returns the sampled index (>0), GZO_EMPTY
 * when every bucket is zero, or GZO_FAIL. */
static int64_t cubesketch_query(const gzo_ctx *x, uint32_t k,
                                const uint64_t *A, const uint32_t *G,
                                const uint32_t *label, uint32_t comp)
{
    int nonzero = 0;
    uint64_t VV = (uint64_t)x->V * x->V;
    for (uint32_t j = 0; j < GZO_COLS; j++) {
        size_t col = (size_t)k * GZO_COLS + j;
        for (uint32_t row = 0; row < x->R; row++) {
            uint64_t alpha = A[(size_t)j * x->R + row];
            uint32_t gamma = G[(size_t)j * x->R + row];
            if (alpha == 0 && gamma == 0) continue;
            nonzero = 1;
            /* h2 is defined on edge indices: alpha must decode to u < v < V */
            if (alpha >= VV) continue;
            uint64_t uu = alpha / x->V, vv = alpha % x->V;
            if (uu >= vv) continue;
            if (gamma != gzo_h2(x->V, x->keys + col * GZO_KEYS + 128, alpha)) continue;
            int in_u = label[uu] == comp, in_v = label[vv] == comp;
            if (in_u == in_v) continue;
            return (int64_t)alpha;
        }
    }
    return nonzero ? GZO_FAIL : GZO_EMPTY;
}

/* Query CubeSketch k of a single sketch with a single-vertex view of the
 * component test disabled (used by the tests on bare vectors): any good
 * bucket whose index decodes to u < v < V is taken. */
int64_t gzo_query_vector(uint32_t V, uint64_t seed, uint32_t k,
                         const uint64_t *A, const uint32_t *G)
{
    gzo_ctx x;
    if (ctx_open(&x, V, seed)) return -3;
    int nonzero = 0;
    int64_t out = GZO_EMPTY;
    uint64_t VV = (uint64_t)V * V;
    for (uint32_t j = 0; j < GZO_COLS && out < 0; j++) {
        size_t col = (size_t)k * GZO_COLS + j;
        for (uint32_t row = 0; row < x.R; row++) {
            uint64_t alpha = A[(size_t)j * x.R + row];
            uint32_t gamma = G[(size_t)j * x.R + row];
            if (alpha == 0 && gamma == 0) continue;
            nonzero = 1;
            if (alpha >= VV || alpha / V >= alpha % V) continue;
            if (gamma != gzo_h2(V, x.keys + col * GZO_KEYS + 128, alpha)) continue;
            out = (int64_t)alpha;
            break;
        }
    }
    if (out < 0) out = nonzero ? GZO_FAIL : GZO_EMPTY;
    ctx_close(&x);
    return out;
}

/* ---------------------------------------------------------------- DSU */

static uint32_t dsu_find(uint32_t *parent, uint32_t x)
{
    uint32_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) { uint32_t n = parent[x]; parent[x] = r; x = n; }
    return r;
}

/* union keeping the smaller root; returns 1 when two sets were joined */
static int dsu_union(uint32_t *parent, uint32_t a, uint32_t b)
{
    a = dsu_find(parent, a);
    b = dsu_find(parent, b);
    if (a == b) return 0;
    if (a < b) parent[b] = a; else parent[a] = b;
    return 1;
}

/* ---------------------------------------------------------------- Boruvka */

/* Boruvka over node sketches (Section 2.2; Lemma (CC I/O), phases 1-3).
 *   alpha/gamma : V node sketches, nested form, layout [node][k][j][row]
 *   labels      : out, V entries, minimum vertex id of each component
 *   forest      : out, 2*(V-1) entries (u,v) in acceptance order, may be NULL
 *   n_forest    : out, number of forest edges
 *   samples     : out, K*V entries, may be NULL: samples[r*V+c] for round r and
 *                 component root c = sampled index, -1 EMPTY, -2 FAIL,
 *                 -3 c is not a root, -4 round not run
 *   stats       : out[4] = rounds run, FAIL count of the last round run,
 *                 1 if round K-1 still sampled an edge, number of components
 * Returns 0, 1 when the result may be wrong (a FAIL in the last round run or
 * rounds exhausted), negative on bad arguments.
 *
 * A component whose sketch is entirely zero in a round (EMPTY) has a zero
 * characteristic vector as far as the sketches can tell (a sketch is linear
 * in the vector, and the members' shared edges cancel), so no merge can reach
 * it (Section 2.2: Boruvka continues "until no new merges are possible"): it
 * is final, and in later rounds it reports EMPTY without a sample.  A
 * component that a sampled edge touches is no longer final. */
int gzo_boruvka(uint32_t V, uint64_t seed, const uint64_t *alpha,
                const uint32_t *gamma, uint32_t *labels, uint32_t *forest,
                uint64_t *n_forest, int64_t *samples, uint64_t *stats)
{
    gzo_ctx x;
    if (ctx_open(&x, V, seed)) return -2;
    size_t nb = node_buckets(&x);
    size_t per_k = (size_t)GZO_COLS * x.R;
    uint32_t *parent = malloc((size_t)V * 4);
    uint64_t *SA = malloc((size_t)V * per_k * 8);
    uint32_t *SG = malloc((size_t)V * per_k * 4);
    int64_t *res = malloc((size_t)V * 8);
    uint8_t *final = calloc(V, 1);  /* final[c]: component c sampled EMPTY, untouched since */
    if (!parent || !SA || !SG || !res || !final) return -2;
    for (uint32_t i = 0; i < V; i++) { parent[i] = i; labels[i] = i; }
    if (samples)
        for (size_t i = 0; i < (size_t)x.K * V; i++) samples[i] = -4;
    uint64_t nf = 0, rounds = 0, fails_last = 0, exhausted = 0;

    for (uint32_t r = 0; r < x.K; r++) {
        rounds = r + 1;
        /* the sketch of a component is the XOR of its members' CubeSketch r
         * (phase 3 of the previous round, linearity of Definition def:l0) */
        memset(SA, 0, (size_t)V * per_k * 8);
        memset(SG, 0, (size_t)V * per_k * 4);
        for (uint32_t v = 0; v < V; v++) {
            uint32_t c = labels[v];
            const uint64_t *a = alpha + (size_t)v * nb + (size_t)r * per_k;
            const uint32_t *g = gamma + (size_t)v * nb + (size_t)r * per_k;
            for (size_t w = 0; w < per_k; w++) {
                SA[(size_t)c * per_k + w] ^= a[w];
                SG[(size_t)c * per_k + w] ^= g[w];
            }
        }
        /* phase 1: one sample per component */
        uint64_t n_edges = 0, n_fail = 0;
        for (uint32_t c = 0; c < V; c++) {
            if (labels[c] != c) { res[c] = -3; continue; }
            if (final[c]) { res[c] = GZO_EMPTY; continue; }
            res[c] = cubesketch_query(&x, r, SA + (size_t)c * per_k,
                                      SG + (size_t)c * per_k, labels, c);
            if (res[c] > 0) n_edges++;
            else if (res[c] == GZO_FAIL) n_fail++;
            else final[c] = 1;
        }
        if (samples)
            for (uint32_t c = 0; c < V; c++) samples[(size_t)r * V + c] = res[c];
        fails_last = n_fail;
        if (n_edges == 0) break;
        if (r == x.K - 1) exhausted = 1;
        /* phase 2: merge in ascending order of the component id; an edge
         * enters the forest when it joins two sets */
        for (uint32_t c = 0; c < V; c++) {
            if (res[c] <= 0) continue;
            uint32_t uu = (uint32_t)((uint64_t)res[c] / V);
            uint32_t vv = (uint32_t)((uint64_t)res[c] % V);
            final[labels[uu]] = final[labels[vv]] = 0;  /* both components take part in a merge */
            if (dsu_union(parent, uu, vv)) {
                if (forest) {
                    forest[2 * nf] = uu;
                    forest[2 * nf + 1] = vv;
                }
                nf++;
            }
        }
        for (uint32_t v = 0; v < V; v++) labels[v] = dsu_find(parent, v);
    }
    uint64_t ncomp = 0;
    for (uint32_t v = 0; v < V; v++) ncomp += labels[v] == v;
    if (n_forest) *n_forest = nf;
    if (stats) {
        stats[0] = rounds;
        stats[1] = fails_last;
        stats[2] = exhausted;
        stats[3] = ncomp;
    }
    free(parent); free(SA); free(SG); free(res); free(final);
    ctx_close(&x);
    return (fails_last || exhausted) ? 1 : 0;
}

/* ---------------------------------------------------------------- brute force */

/* Connected components of the NET graph of a stream (the edges with an odd
 * number of updates, Section 2.1 with Delta read mod 2) by an adjacency bit
 * vector and union-find, the check of the reliability experiment
 * (Section 6.3).  labels = minimum vertex id per component. */
int gzo_brute_cc(uint32_t V, size_t n, const uint32_t *u, const uint32_t *v,
                 uint32_t *labels)
{
    uint64_t npairs = (uint64_t)V * (V - 1) / 2;
    uint8_t *bits = calloc(npairs / 8 + 1, 1);
    uint32_t *parent = malloc((size_t)V * 4);
    if (!bits || !parent) return -2;
    for (size_t i = 0; i < n; i++) {
        if (u[i] == v[i] || u[i] >= V || v[i] >= V) { free(bits); free(parent); return -1; }
        uint64_t lo = u[i] < v[i] ? u[i] : v[i];
        uint64_t hi = u[i] < v[i] ? v[i] : u[i];
        uint64_t p = hi * (hi - 1) / 2 + lo;     /* triangular position */
        bits[p >> 3] ^= (uint8_t)(1u << (p & 7));
    }
    for (uint32_t i = 0; i < V; i++) parent[i] = i;
    for (uint64_t hi = 1; hi < V; hi++)
        for (uint64_t lo = 0; lo < hi; lo++) {
            uint64_t p = hi * (hi - 1) / 2 + lo;
            if (bits[p >> 3] >> (p & 7) & 1u) dsu_union(parent, (uint32_t)lo, (uint32_t)hi);
        }
    for (uint32_t i = 0; i < V; i++) labels[i] = dsu_find(parent, i);
    free(bits); free(parent);
    return 0;
}

/* Connected components from an explicit list of m edges (a net graph given
 * directly), union-find; labels = minimum vertex id per component. */
int gzo_cc_edges(uint32_t V, size_t m, const uint32_t *u, const uint32_t *v,
                 uint32_t *labels)
{
    uint32_t *parent = malloc((size_t)V * 4);
    if (!parent) return -2;
    for (uint32_t i = 0; i < V; i++) parent[i] = i;
    for (size_t i = 0; i < m; i++) {
        if (u[i] >= V || v[i] >= V) { free(parent); return -1; }
        dsu_union(parent, u[i], v[i]);
    }
    for (uint32_t i = 0; i < V; i++) labels[i] = dsu_find(parent, i);
    free(parent);
    return 0;
}
