"""Pins of the oracle's general factors (Sec. 2.1, Props. 1-2): for odd n, x^n + 1 is a product of
distinct irreducible polynomials p_i, R_{2,n} is the direct sum of the ideals they define, and for
any factor p of degree w the remainder mod p maps R_{2,n} onto GF(2^w) = F2[x]/(p) as a ring
homomorphism. So the embedding transform works for any factor: a field coefficient u is replaced
by a ring element r with r mod p = u (2^(n-w) choices, the sparsest taken) and the ring product,
reduced mod p, is the field product. Besides the all-one and equally spaced polynomials, this
gives e.g. GF(8) from x^3 + x + 1 in R_{2,7} and GF(16) from x^4 + x + 1 in R_{2,15}.

What fixes the oracle here: the textbook factorizations of x^7 + 1 and x^15 + 1, squarefree
factorization by trial division, idempotent counts (2 to the number of factors), the homomorphism
property by brute force, closed forms of the fields, MDS and erasure recovery on small codes.
"""
import itertools
from functools import reduce

import numpy as np
import pytest

import oracle

# (w, n, p): GF(8) in R_{2,7}, GF(16) from x^4 + x + 1 in R_{2,15}, GF(4) in R_{2,9} and R_{2,15}
GENERAL = [(3, 7, 0b1011), (4, 15, 0b10011), (2, 9, 0b111), (2, 15, 0b111)]


def _ring_mul(a, b, n):
    r = 0
    for i in range(n):
        if (a >> i) & 1:
            for j in range(n):
                if (b >> j) & 1:
                    r ^= 1 << ((i + j) % n)
    return r


def _factor(n):
    """Irreducible factors of x^n + 1 by repeated trial division (with multiplicity)."""
    f, out = (1 << n) | 1, []
    d = 1
    while f.bit_length() > 1:
        found = False
        for p in range(1 << d, 1 << (d + 1)):
            if oracle.poly_irreducible(p) and oracle.poly_mod(f, p) == 0:
                q, rem = 0, f  # exact quotient
                while rem.bit_length() - 1 >= d:
                    s = rem.bit_length() - 1 - d
                    q |= 1 << s
                    rem ^= p << s
                assert rem == 0
                out.append(p)
                f = q
                found = True
                break
        if not found:
            d += 1
    return sorted(out)


def test_textbook_factorizations():
    # x^7 + 1 = (x + 1)(x^3 + x + 1)(x^3 + x^2 + 1); x^15 + 1 has the five factors below
    assert _factor(7) == [0b11, 0b1011, 0b1101]
    assert _factor(15) == [0b11, 0b111, 0b10011, 0b11001, 0b11111]
    for n in (3, 5, 7, 9, 11, 13, 15):
        fs = _factor(n)
        assert len(set(fs)) == len(fs), "x^n + 1 is squarefree for odd n (Prop. 1)"
        assert reduce(oracle.poly_mul, fs) == (1 << n) | 1
        # the library's choice of factor: the smallest irreducible factor of each degree
        for w in range(2, n):
            deg_w = [p for p in fs if p.bit_length() - 1 == w]
            assert oracle.ring_factor(w, n) == (deg_w[0] if deg_w else 0), (w, n)


@pytest.mark.parametrize("n", [7, 9])
def test_idempotents_count_the_factors(n):
    # R_{2,n} is the direct sum of one ideal per factor: 2^(number of factors) idempotents
    assert len(oracle.ring_idempotents(n)) == 2 ** len(_factor(n))


@pytest.mark.parametrize("w,n,p", GENERAL)
def test_mod_p_is_a_ring_homomorphism(w, n, p):
    rng = np.random.default_rng(n)
    pairs = itertools.product(range(1 << n), range(1 << n)) if n <= 7 else \
        [(int(a), int(b)) for a, b in rng.integers(0, 1 << n, size=(3000, 2))]
    for a, b in pairs:
        left = oracle.poly_mod(_ring_mul(a, b, n), p)
        right = oracle.gf_mul_mod(w, p, oracle.poly_mod(a, p), oracle.poly_mod(b, p))
        assert left == right, (a, b)


@pytest.mark.parametrize("w,n,p", GENERAL)
def test_sparse_transform_and_ring_path(w, n, p):
    by_u = {}
    for r in range(1 << n):
        by_u.setdefault(oracle.poly_mod(r, p), []).append(r)
    for u in range(1 << w):
        assert len(by_u[u]) == 1 << (n - w)
        best = min(by_u[u], key=lambda r: (bin(r).count("1"), r))
        assert oracle.sparse_rep_mod(w, n, p, u) == best
        for d in range(1 << w):
            assert oracle.poly_mod(_ring_mul(best, d, n), p) == oracle.gf_mul_mod(w, p, u, d)


def test_closed_forms():
    # GF(16) from x^4 + x + 1: x^4 = x + 1 and x is primitive (order 15); under the AOP x has order 5
    assert oracle.gf_mul_mod(4, 0b10011, 0b10, 0b1000) == 0b0011
    v, order = 0b10, 1
    while v != 1:
        v = oracle.gf_mul_mod(4, 0b10011, v, 0b10)
        order += 1
    assert order == 15 and oracle.gf_order(4, 2) == 5
    # GF(8) from x^3 + x + 1: x^3 = x + 1, x^7 = 1
    assert oracle.gf_mul_mod(3, 0b1011, 0b10, 0b100) == 0b011
    v = 1
    for _ in range(7):
        v = oracle.gf_mul_mod(3, 0b1011, v, 0b10)
    assert v == 1


@pytest.mark.parametrize("w,p,k,m", [(3, 0b1011, 4, 4), (4, 0b10011, 8, 4), (2, 0b111, 2, 2)])
def test_cauchy_mds_and_every_pattern(w, p, k, m):
    G = oracle.cauchy_mod(w, p, k, m)
    for i in range(m):  # C[i][j] (x_i + y_j) = 1 in this field
        for j in range(k):
            assert oracle.gf_mul_mod(w, p, int(G[k + i][j]), (k + i) ^ j) == 1
    for rows in itertools.combinations(range(k + m), k):
        oracle.gf_invert_mod(w, p, G[list(rows)])
    rng = np.random.default_rng(w * 10 + k)
    P = 40
    data = rng.integers(0, 256, size=(k, w, P), dtype=np.uint8)
    par = oracle.encode_mod(w, p, k, m, G, data)
    # linearity and one symbol lane by the definition: parity = C d over F2[x]/(p)
    t, b = 7, 3
    sym = [sum(((int(data[j][q][t]) >> b) & 1) << q for q in range(w)) for j in range(k)]
    for i in range(m):
        want = 0
        for j in range(k):
            want ^= oracle.gf_mul_mod(w, p, int(G[k + i][j]), sym[j])
        assert sum(((int(par[i][q][t]) >> b) & 1) << q for q in range(w)) == want
    full = np.concatenate([data, par])
    for e in range(1, m + 1):
        for pat in itertools.combinations(range(k + m), e):
            blocks = full.copy()
            for x in pat:
                blocks[x] = 0x77
            np.testing.assert_array_equal(oracle.decode_mod(w, p, k, m, G, blocks, sum(1 << x for x in pat)), full)
