"""Single-vector l0 sketches: the standard sampler of Fig. agm_code and
CubeSketch on a plain vector (the comparison of Fig. l0speedup).

The CPU tests pin the oracle against definitions computed here independently
(Python integers, Python's pow) and against the sampler properties of
Section 3 (recovery of a single nonzero entry, linearity, deletion, samples in
the support); the GPU tests compare gz_l0_update with the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle

P = (1 << 61) - 1
MASK = (1 << 64) - 1


def _keys(seed):
    # column j: a, b (depth hash) and the h2 key triple c0, c1, c2
    a = [oracle.splitmix64_at(seed, 5 * j) | 1 for j in range(7)]
    b = [oracle.splitmix64_at(seed, 5 * j + 1) for j in range(7)]
    c = [tuple(oracle.splitmix64_at(seed, 5 * j + w) for w in (2, 3, 4)) for j in range(7)]
    return a, b, c


def _depth(a, b, x, R):
    t = (a * x + b) & MASK
    d = 64 - t.bit_length()  # leading zeros of a 64-bit word
    return min(d, R - 1)


def test_mulmod_and_powmod_match_python_integers():
    rng = np.random.default_rng(3)
    for _ in range(300):
        x, y = (int(v) for v in rng.integers(0, P, 2, dtype=np.uint64))
        assert oracle.mulmod61(x, y) == x * y % P
        r = int(rng.integers(1, P - 1, dtype=np.uint64))
        e = int(rng.integers(0, 1 << 40, dtype=np.uint64))
        assert oracle.powmod61(r, e) == pow(r, e, P)
    assert oracle.powmod61(12345, 0) == 1
    assert oracle.powmod61(P - 1, 2) == 1  # (-1)^2
    assert oracle.mulmod61(P - 1, P - 1) == 1


def test_rows_are_ceil_log2():
    for n, R in [(2, 1), (3, 2), (1000, 10), (1024, 10), (1025, 11), (10 ** 12, 40)]:
        assert oracle.l0_rows(n) == R


@pytest.mark.parametrize("n", [1000, 10 ** 7, 10 ** 12])
def test_standard_buckets_equal_their_definition(n):
    # every bucket (a, b, c) of Fig. agm_code is a sum over its members:
    # a = sum x*delta, b = sum delta (mod 2^64), c = sum delta * r^x (mod p)
    seed = 11
    rng = np.random.default_rng(n % 97)
    x = rng.integers(1, n + 1, 400, dtype=np.uint64)
    dl = rng.choice([-1, 1], 400).astype(np.int32)
    got = oracle.l0_update(oracle.L0_STANDARD, n, seed, x, dl).view(np.uint64)
    R = oracle.l0_rows(n)
    A, B, C = got[: 7 * R], got[7 * R: 14 * R], got[14 * R:]
    ka, kb, kc = _keys(seed)
    for j in range(7):
        r = 1 + kc[j][0] % (P - 1)
        want_a, want_b, want_c = [0] * R, [0] * R, [0] * R
        for xi, di in zip(x.tolist(), dl.tolist()):
            d = _depth(ka[j], kb[j], xi, R)
            for row in range(d + 1):
                want_a[row] = (want_a[row] + xi * di) & MASK
                want_b[row] = (want_b[row] + di) & MASK
                want_c[row] = (want_c[row] + di * pow(r, xi, P)) % P
        assert A[j * R:(j + 1) * R].tolist() == want_a
        assert B[j * R:(j + 1) * R].tolist() == want_b
        assert C[j * R:(j + 1) * R].tolist() == want_c


def test_cubesketch_vector_buckets_equal_their_definition():
    # alpha = XOR of members, gamma = XOR of h2 of members (Eq. 1-2)
    n, seed = 10 ** 6, 5
    rng = np.random.default_rng(1)
    x = rng.integers(1, n + 1, 300, dtype=np.uint64)
    got = oracle.l0_update(oracle.L0_CUBE, n, seed, x)
    R = oracle.l0_rows(n)
    alpha = got[: 7 * R * 8].view(np.uint64)
    gamma = got[7 * R * 8:].view(np.uint32)
    ka, kb, kc = _keys(seed)
    for j in range(7):
        wa, wg = [0] * R, [0] * R
        for xi in x.tolist():
            d = _depth(ka[j], kb[j], xi, R)
            for row in range(d + 1):
                wa[row] ^= xi
                c0, c1, c2 = kc[j]
                wg[row] ^= ((c0 * (xi & 0xFFFFFFFF) + c1 * (xi >> 32) + c2) & MASK) >> 32
        assert alpha[j * R:(j + 1) * R].tolist() == wa
        assert gamma[j * R:(j + 1) * R].tolist() == wg


@pytest.mark.parametrize("kind", [oracle.L0_CUBE, oracle.L0_STANDARD])
def test_single_entry_is_always_recovered(kind):
    # row 0 holds every position, so a vector with one nonzero entry always
    # has a good bucket (Definition l0: sampleable)
    rng = np.random.default_rng(kind)
    for n in (10, 1000, 10 ** 9, 10 ** 12):
        for _ in range(20):
            x = int(rng.integers(1, n + 1, dtype=np.uint64))
            sk = oracle.l0_update(kind, n, 9, [x], [-1] if kind else None)
            pos, val = oracle.l0_query(kind, n, 9, sk)
            assert pos == x
            assert val == (-1 if kind == oracle.L0_STANDARD else 1)


@pytest.mark.parametrize("kind", [oracle.L0_CUBE, oracle.L0_STANDARD])
def test_linearity_and_deletion(kind):
    n, seed = 10 ** 8, 4
    rng = np.random.default_rng(7)
    x1 = rng.integers(1, n + 1, 200, dtype=np.uint64)
    x2 = rng.integers(1, n + 1, 150, dtype=np.uint64)
    s1 = oracle.l0_update(kind, n, seed, x1)
    s2 = oracle.l0_update(kind, n, seed, x2)
    s12 = oracle.l0_update(kind, n, seed, np.concatenate([x1, x2]))
    R = oracle.l0_rows(n)
    if kind == oracle.L0_CUBE:
        assert np.array_equal(s1 ^ s2, s12)
    else:
        a1, a2, a12 = (s.view(np.uint64) for s in (s1, s2, s12))
        assert np.array_equal((a1[:14 * R] + a2[:14 * R]), a12[:14 * R])  # wraps mod 2^64
        c = (a1[14 * R:].astype(object) + a2[14 * R:].astype(object)) % P
        assert c.tolist() == a12[14 * R:].tolist()
    # inserting and then deleting every position gives the zero sketch
    both = np.concatenate([x1, x1])
    dl = np.concatenate([np.ones(200, np.int32), -np.ones(200, np.int32)])
    z = oracle.l0_update(kind, n, seed, both, dl)
    assert not z.any()
    assert oracle.l0_query(kind, n, seed, z)[0] == -1


@pytest.mark.parametrize("kind", [oracle.L0_CUBE, oracle.L0_STANDARD])
def test_samples_lie_in_the_support_and_failures_are_rare(kind):
    n, fails = 10 ** 10, 0
    rng = np.random.default_rng(20 + kind)
    trials = 150
    for t in range(trials):
        k = int(rng.integers(2, 2000))
        supp = np.unique(rng.integers(1, n + 1, k, dtype=np.uint64))
        vals = rng.integers(1, 4, len(supp)).astype(np.int64) if kind else np.ones(len(supp), np.int64)
        x = np.repeat(supp, vals)  # entry value = number of +1 updates
        sk = oracle.l0_update(kind, n, 100 + t, x)
        pos, val = oracle.l0_query(kind, n, 100 + t, sk)
        if pos == -2:
            fails += 1
            continue
        assert pos > 0
        i = np.searchsorted(supp, np.uint64(pos))
        assert i < len(supp) and supp[i] == pos
        if kind == oracle.L0_STANDARD:
            assert val == vals[i]
    assert fails <= 3  # 7 columns: a few in 10^4 per sketch in simulation


# ---------------------------------------------------------------- GPU parity

@pytest.mark.gpu
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("n", [1000, 10 ** 5, 10 ** 7, 3 * 10 ** 10, 10 ** 12])  # R = 10, 17, 24, 35, 40
def test_gpu_l0_update_matches_oracle(kind, n):
    import torch

    import paper_2203_14927_b300 as gz

    sketches, m, seed = 37, 300, 123
    rng = np.random.default_rng(n % 1009 + kind)
    x = rng.integers(1, n + 1, (sketches, m), dtype=np.uint64)
    dl = rng.choice([-1, 1], (sketches, m)).astype(np.int32)
    R, bc, bs = gz.l0_geometry(n)
    nb = bc if kind == 0 else bs
    assert nb == oracle.l0_bytes(kind, n)
    dbuf = torch.zeros(sketches * nb, dtype=torch.uint8, device="cuda")
    gz.l0_update(kind, n, seed, torch.from_numpy(x.view(np.int64)).cuda(), dbuf,
                 torch.from_numpy(dl).cuda())
    torch.cuda.synchronize()
    got = dbuf.cpu().numpy().reshape(sketches, nb)
    for s in range(sketches):
        want = oracle.l0_update(kind, n, seed, x[s], dl[s])
        assert np.array_equal(got[s], want), s
