"""Pins of the oracle's encoder and decoder. Encoding is a linear map on bit-sliced blocks, so it is
fixed by (1) its value on every single-bit input, checked against the field definition
(carry-less product mod the AOP) and the Cauchy entries' defining identity, and (2) linearity.
Decoding is fixed by the MDS property of the code: every pattern of at most m erased blocks is
recovered exactly (brute force over all patterns on tiny stripes)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300.synth import synth_bytes

# (w, k, m): the first is the GF(16) workload's code, the others the GF(2^10) and GF(2^12) codes
CODES = [(4, 4, 2), (10, 10, 4), (12, 16, 4)]


@pytest.mark.parametrize("w,k,m", CODES + [(4, 12, 4), (10, 30, 8)])
def test_cauchy_entries(w, k, m):
    # Systematic top, and every C[i][j] satisfies C[i][j] * (x_i + y_j) = 1 with x_i = k+i,
    # y_j = j, by the field definition (not the oracle's tables).
    G = oracle.cauchy(w, k, m)
    assert np.array_equal(G[:k], np.eye(k, dtype=np.uint32))
    for i in range(m):
        for j in range(k):
            assert oracle.gf_mul_slow(w, int(G[k + i, j]), (k + i) ^ j) == 1


def test_cauchy_length_limit():
    with pytest.raises(ValueError):
        oracle.cauchy(4, 12, 5)  # k + m = 17 > 2^4
    oracle.cauchy(4, 12, 4)


def _det_nonzero(w, M):
    try:
        oracle.gf_invert(w, M)
        return True
    except ValueError:
        return False


@pytest.mark.parametrize("w,k,m", [(4, 4, 2), (10, 10, 4)])
def test_generator_is_mds_exhaustive(w, k, m):
    # Sec. 2.2: every square submatrix of the parity part is invertible, equivalently every k x k
    # row subset of G is; exhaustive over all C(k+m, k) subsets.
    G = oracle.cauchy(w, k, m)
    for rows in itertools.combinations(range(k + m), k):
        assert _det_nonzero(w, G[list(rows)])


def test_generator_is_mds_sampled_w12():
    w, k, m = 12, 16, 4
    G = oracle.cauchy(w, k, m)
    rng = np.random.default_rng(3)
    for _ in range(200):
        rows = sorted(rng.choice(k + m, k, replace=False).tolist())
        assert _det_nonzero(w, G[rows])


@pytest.mark.parametrize("w", [4, 10])
def test_invert_is_an_inverse(w):
    # M Inv = I with products taken by the field definition.
    rng = np.random.default_rng(w)
    k = 6
    for _ in range(20):
        M = rng.integers(0, 1 << w, (k, k)).astype(np.uint32)
        try:
            Inv = oracle.gf_invert(w, M)
        except ValueError:
            continue
        for r in range(k):
            for c in range(k):
                acc = 0
                for t in range(k):
                    acc ^= oracle.gf_mul_slow(w, int(M[r, t]), int(Inv[t, c]))
                assert acc == (r == c)


def test_invert_rejects_singular():
    M = np.array([[1, 2], [1, 2]], np.uint32)
    with pytest.raises(ValueError):
        oracle.gf_invert(4, M)


@pytest.mark.parametrize("w,k,m", CODES)
def test_encode_single_bit_basis(w, k, m):
    # A single set bit at (block j, packet q, byte t, bit b) is the field symbol x^q in lane
    # (t, b) of block j; parity block i must then hold C[i][j] * x^q in lane (t, b) and zeros
    # in every other lane (Sec. 3: the coding is a matrix-vector product over the field).
    G = oracle.cauchy(w, k, m)
    P = 3
    rng = np.random.default_rng(w * 100 + k)
    cases = [(j, q, t, b) for j in range(k) for q in range(w) for t in range(P) for b in range(8)]
    if len(cases) > 200:
        idx = rng.choice(len(cases), 200, replace=False)
        cases = [cases[i] for i in idx] + [(0, 0, 0, 0), (k - 1, w - 1, P - 1, 7)]
    for j, q, t, b in cases:
        data = np.zeros((k, w, P), np.uint8)
        data[j, q, t] = 1 << b
        par = oracle.encode(w, k, m, G, data)
        for i in range(m):
            expect = oracle.gf_mul_slow(w, int(G[k + i, j]), 1 << q)
            lane = np.zeros((w, P), np.uint8)
            for qq in range(w):
                if (expect >> qq) & 1:
                    lane[qq, t] = 1 << b
            assert np.array_equal(par[i], lane), (j, q, t, b, i)


@pytest.mark.parametrize("w,k,m", CODES)
def test_encode_is_linear(w, k, m):
    G = oracle.cauchy(w, k, m)
    P = 40
    a = synth_bytes(11, 0, k * w * P).reshape(k, w, P)
    b = synth_bytes(12, 0, k * w * P).reshape(k, w, P)
    pa, pb = oracle.encode(w, k, m, G, a), oracle.encode(w, k, m, G, b)
    assert np.array_equal(oracle.encode(w, k, m, G, a ^ b), pa ^ pb)
    assert not oracle.encode(w, k, m, G, np.zeros_like(a)).any()


def test_encode_threads_agree():
    w, k, m = 10, 10, 4
    G = oracle.cauchy(w, k, m)
    P = 257
    a = synth_bytes(13, 0, k * w * P).reshape(k, w, P)
    assert np.array_equal(oracle.encode(w, k, m, G, a, nthreads=1), oracle.encode(w, k, m, G, a, nthreads=7))


def _all_patterns(n, m):
    for e in range(1, m + 1):
        for c in itertools.combinations(range(n), e):
            yield sum(1 << x for x in c)


@pytest.mark.parametrize("w,k,m,P", [(4, 4, 2, 16), (10, 10, 4, 4)])
def test_decode_recovers_every_pattern(w, k, m, P):
    # MDS: any <= m erasures are recoverable; brute force over every pattern (22 for (4,2),
    # 1470 for (10,4)). Erased blocks are overwritten with garbage before decoding.
    G = oracle.cauchy(w, k, m)
    data = synth_bytes(20 + w, 0, k * w * P).reshape(k, w, P)
    full = np.concatenate([data, oracle.encode(w, k, m, G, data)])
    n = 0
    for mask in _all_patterns(k + m, m):
        blk = full.copy()
        for e in range(k + m):
            if (mask >> e) & 1:
                blk[e] ^= 0xA5
        assert np.array_equal(oracle.decode(w, k, m, G, blk, mask), full), hex(mask)
        n += 1
    assert n == sum(len(list(itertools.combinations(range(k + m), e))) for e in range(1, m + 1))


def test_decode_sampled_patterns_w12():
    w, k, m, P = 12, 16, 4, 8
    G = oracle.cauchy(w, k, m)
    data = synth_bytes(33, 0, k * w * P).reshape(k, w, P)
    full = np.concatenate([data, oracle.encode(w, k, m, G, data)])
    rng = np.random.default_rng(4)
    for _ in range(60):
        e = int(rng.integers(1, m + 1))
        mask = sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))
        blk = full.copy()
        blk[[i for i in range(k + m) if (mask >> i) & 1]] = 0
        assert np.array_equal(oracle.decode(w, k, m, G, blk, mask), full)


def test_decode_rejects_too_many_erasures():
    w, k, m = 4, 4, 2
    G = oracle.cauchy(w, k, m)
    blk = np.zeros((k + m, w, 4), np.uint8)
    with pytest.raises(ValueError):
        oracle.decode(w, k, m, G, blk, 0b111)


@pytest.mark.parametrize("fill", [0x00, 0xFF])
def test_constant_data(fill):
    # All-zero data gives zero parity; all-ones data gives, in every lane, the field symbol
    # 1 + x + ... + x^{w-1} times the row sum of C.
    w, k, m, P = 10, 10, 4, 5
    G = oracle.cauchy(w, k, m)
    data = np.full((k, w, P), fill, np.uint8)
    par = oracle.encode(w, k, m, G, data)
    if fill == 0:
        assert not par.any()
        return
    ones = (1 << w) - 1
    for i in range(m):
        s = 0
        for j in range(k):
            s ^= oracle.gf_mul_slow(w, int(G[k + i, j]), ones)
        expect = np.array([0xFF if (s >> q) & 1 else 0 for q in range(w)], np.uint8)
        assert np.array_equal(par[i], np.repeat(expect[:, None], P, axis=1))
