"""Pins of the oracle's ESP field GF(2^6) (paper Sec. 2.4): GF(2^6) = F2[x]/(g), g = x^6 + x^3 + 1
= p(x^3) for the AOP p of degree 2, carried by the ring R_{2,9} (x^9 + 1 = g(x) (x^3 + 1)).

What fixes the oracle here independently of its own code: the irreducibility criterion the paper
quotes (against trial division), the transforms' printed formulas (golden rows), the idempotent
the paper names, the parity property of the ideal A_1, brute force over the ring's 512 elements,
the field axioms, the MDS property and erasure recovery of small codes.
"""
import itertools
import os

import numpy as np
import pytest

import oracle

W, N, G6 = 6, 9, 0b1001001
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "esp_transforms_w6.txt")


def _ring_mul(a, b, n=N):
    # independent cyclic convolution (not the oracle's)
    r = 0
    for i in range(n):
        if (a >> i) & 1:
            for j in range(n):
                if (b >> j) & 1:
                    r ^= 1 << ((i + j) % n)
    return r


def _itoh_irreducible(r, s):
    """Sec. 2.4: p(x^s) (p the AOP of degree r) is irreducible iff p is and s = (r+1)^(t-1) with
    2^(r (r+1)^(t-2)) != 1 mod (r+1)^t for some t; t = 1 (s = 1) is the AOP itself."""
    if not oracle.aop_irreducible(r):
        return False
    if s == 1:
        return True
    t = 2
    while (r + 1) ** (t - 1) <= s:
        if (r + 1) ** (t - 1) == s:
            return pow(2, r * (r + 1) ** (t - 2), (r + 1) ** t) != 1
        t += 1
    return False


def test_esp_irreducibility_criterion():
    # the paper's first irreducible pairs (r, s): (2,3), (2,9), (4,5); none other with r s <= 24
    for r in (2, 4, 10):
        for s in range(1, 25 // r + 1):
            assert oracle.poly_irreducible(oracle.esp(s, r)) == _itoh_irreducible(r, s), (r, s)
    assert _itoh_irreducible(2, 3) and _itoh_irreducible(2, 9) and _itoh_irreducible(4, 5)


def test_field_is_the_3_esp_of_degree_6():
    assert oracle.esp(3, 2) == G6 and oracle.field_poly(W) == G6 and oracle.ring_size(W) == N
    # x^9 + 1 = g(x) (x^3 + 1) over F2
    assert oracle.poly_mul(G6, 0b1001) == (1 << 9) | 1
    # the other fields keep their AOP and ring w + 1
    for w in (2, 4, 10, 12):
        assert oracle.field_poly(w) == oracle.aop(w) and oracle.ring_size(w) == w + 1


def test_field_axioms_and_tables():
    q = 1 << W
    a, b = np.meshgrid(np.arange(q), np.arange(q), indexing="ij")
    a, b = a.ravel(), b.ravel()
    ab = oracle.gf_mul_slow_vec(W, a, b)
    for x, y in zip(a[::37], b[::37]):  # the definition, written out: product mod g
        assert ab[x * q + y] == oracle.poly_mod(oracle.poly_mul(int(x), int(y)), G6)
    assert np.array_equal(ab, oracle.gf_mul_slow_vec(W, b, a))
    c = np.roll(b, 7)
    assert np.array_equal(oracle.gf_mul_slow_vec(W, a, b ^ c), ab ^ oracle.gf_mul_slow_vec(W, a, c))
    inv_count = (ab.reshape(q, q)[1:, 1:] == 1).sum(axis=1)
    assert np.all(inv_count == 1)
    # x has order 9 in this field (x^9 = 1 mod g); the tables use the smallest primitive element
    assert oracle.gf_order(W, 2) == 9
    g = oracle.gf_primitive(W)
    assert oracle.gf_order(W, g) == q - 1 and all(oracle.gf_order(W, h) < q - 1 for h in range(2, g))
    assert np.array_equal(oracle.gf_mul_vec(W, a, b), ab)


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                kind, x, y = line.split()
                rows.append((kind, int(x, 2), int(y, 2)))
    return rows


def test_golden_transforms():
    rows = _golden()
    assert len(rows) == 10
    for kind, x, y in rows:
        if kind == "embed_inverse":
            assert oracle.poly_mod(x, G6) == y  # phi_E^{-1} is the remainder mod g
        else:
            assert oracle.phi_P(W, N, x) == y


def test_embedding_inverse_closed_form_all_ring_elements():
    # the printed rule: XOR the top block of 3 coefficients into both lower blocks
    for v in range(1 << N):
        top = v >> 6
        assert oracle.poly_mod(v, G6) == (v & 63) ^ top ^ (top << 3)


def test_idempotent_and_ideal():
    # Sec. 2.4: theta_1 = g(x) + 1 = x^6 + x^3 is the idempotent of A_1
    th = G6 ^ 1
    assert th == 0b1001000 and _ring_mul(th, th) == th and th in oracle.ring_idempotents(N)
    A1 = {_ring_mul(b, th) for b in range(1 << W)}
    assert len(A1) == 1 << W
    # A_1 = the elements whose three interleaved words (coefficients j, j+3, j+6) have even weight
    even = {v for v in range(1 << N) if all(bin(v & (0b1001001 << j)).count("1") % 2 == 0 for j in range(3))}
    assert A1 == even
    # phi(b) = b theta_1 is multiplicative and inverted by mod g (Sec. 2.4)
    for a in range(1 << W):
        for b in range(0, 1 << W, 5):
            assert _ring_mul(_ring_mul(a, th), _ring_mul(b, th)) == _ring_mul(oracle.gf_mul_slow(W, a, b), th)
        assert oracle.poly_mod(_ring_mul(a, th), G6) == a


def test_representatives_and_sparse_transform():
    by_u = {}
    for r in range(1 << N):
        by_u.setdefault(oracle.poly_mod(r, G6), []).append(r)
    for u in range(1 << W):
        reps = oracle.ring_representatives(W, N, u)
        assert sorted(reps) == by_u[u] and len(reps) == 1 << (N - W)  # 2^{n-w} = 8
        best = min(by_u[u], key=lambda r: (bin(r).count("1"), r))  # fewest ones, then smallest
        assert oracle.sparse_rep(W, N, u) == best


def test_ring_path_equals_field_product():
    # (phi_S(u) * d) mod g = u d for every u, d: the ring path reaches the field result
    for u in range(1 << W):
        r = oracle.sparse_rep(W, N, u)
        for d in range(1 << W):
            assert oracle.poly_mod(_ring_mul(r, d), G6) == oracle.gf_mul_slow(W, u, d), (u, d)


@pytest.mark.parametrize("k,m", [(4, 2), (8, 4)])
def test_cauchy_is_mds_and_decodes(k, m):
    G = oracle.cauchy(W, k, m)
    for rows in itertools.combinations(range(k + m), k):
        oracle.gf_invert(W, G[list(rows)])  # raises if singular
    rng = np.random.default_rng(k)
    P = 32
    data = rng.integers(0, 256, size=(k, W, P), dtype=np.uint8)
    full = np.concatenate([data, oracle.encode(W, k, m, G, data)])
    pats = [c for e in range(1, m + 1) for c in itertools.combinations(range(k + m), e)]
    if len(pats) > 300:
        pats = [pats[i] for i in rng.choice(len(pats), 300, replace=False)]
    for pat in pats:
        blocks = full.copy()
        for b in pat:
            blocks[b] = 0x3C
        np.testing.assert_array_equal(oracle.decode(W, k, m, G, blocks, sum(1 << b for b in pat)), full)


def _swap(d):
    return ((d >> 3) | (d << 3)) & 63


def test_parity_transform_is_the_half_swapped_field_code():
    """phi_P(d) lies in A_1, phi_P^{-1} drops the three top coefficients, and
    phi_P^{-1}(phi_S(u) phi_P(d)) = psi(u psi(d)) with psi(d) = phi_P(d) mod g, which for this ESP
    swaps the two 3-coefficient halves of d (coefficient t gets d_t + d_(t mod 3) + d_(t mod 3 + 3))."""
    th = G6 ^ 1
    for d in range(1 << W):
        e = oracle.phi_P(W, N, d)
        assert _ring_mul(e, th) == e and e & 63 == d  # in A_1; phi_P^{-1} recovers d
        assert oracle.poly_mod(e, G6) == _swap(d)
    for u in range(1 << W):
        r = oracle.sparse_rep(W, N, u)
        for d in range(1 << W):
            ring = _ring_mul(r, oracle.phi_P(W, N, d)) & 63
            assert ring == _swap(oracle.gf_mul_slow(W, u, _swap(d))), (u, d)


def test_parity_transform_codec():
    k, m, P = 8, 4, 48
    G = oracle.cauchy(W, k, m)
    rng = np.random.default_rng(6)
    data = rng.integers(0, 256, size=(k, W, P), dtype=np.uint8)
    swap = lambda x: np.concatenate([x[..., 3:6, :], x[..., 0:3, :]], axis=-2)  # psi on packets
    par = oracle.encode_pt(W, k, m, G, data)
    np.testing.assert_array_equal(par, swap(oracle.encode(W, k, m, G, swap(data))))
    full = np.concatenate([data, par])
    for pat in [(0,), (3, 9), (1, 2, 10, 11), (8, 9, 10, 11), (0, 5, 7, 8)]:
        blocks = full.copy()
        for b in pat:
            blocks[b] = 0xA5
        np.testing.assert_array_equal(oracle.decode_pt(W, k, m, G, blocks, sum(1 << b for b in pat)), full)
