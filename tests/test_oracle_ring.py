"""Pins of the ring reference and of the algebra that the coding path relies on (paper Sec. 2):
the direct-sum decomposition and its idempotents (Prop. 1), the isomorphism phi_1 and its inverse
(Prop. 2, Eqs. 1-2 and their AOP forms), the even-weight characterisation of A_1, the sparse
transform's representative set, and the fact the GPU path is built on: embedding a field element,
multiplying in the ring by any representative of u and reducing mod p gives the field product."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RINGS = [(4, 5), (10, 11), (12, 13)]


def _poly(s):
    if s == "-":
        return 0
    v = 0
    for e in s.split(","):
        v |= 1 << int(e)
    return v


def _load(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _popcount(v):
    return bin(v).count("1")


def test_golden_worked_example_r25():
    rows = _load("aop_r25_worked_example.txt")
    d = {}
    for r in rows:
        d.setdefault(r[0], []).append(r[1:])
    w, n = int(d["w"][0][0]), int(d["n"][0][0])
    p = oracle.aop(w)
    a, b, c = (_poly(x) for x in d["ring_product"][0])
    assert oracle.ring_mul(n, a, b) == c
    f, p1, p2 = (_poly(x) for x in d["factor"][0])
    assert oracle.poly_mul(p1, p2) == f and p1 == p
    idem = set(oracle.ring_idempotents(n))
    th1, th2 = _poly(d["idempotent_A1"][0][0]), _poly(d["idempotent_A2"][0][0])
    assert th1 in idem and th2 in idem
    # theta_1 lies in A_1 = (p_2) = (x+1), theta_2 in A_2 = (p_1)
    assert oracle.poly_mod(th1, p2) == 0 and oracle.poly_mod(th2, p1) == 0
    u, img = (_poly(x) for x in d["phi1"][0])
    assert oracle.ring_mul(n, u, th1) == img
    zero, pp = (_poly(x) for x in d["ideal_A2"][0])
    # ring elements with no A_1 component: r theta_1 = 0
    no_a1 = [r for r in range(1 << n) if oracle.ring_mul(n, r, th1) == 0]
    assert no_a1 == sorted([zero, pp])
    u, rep = (_poly(x) for x in d["sparse"][0])
    assert oracle.sparse_rep(w, n, u) == rep
    assert sorted(oracle.ring_representatives(w, n, u)) == sorted([img, img ^ pp])


def test_golden_embedding_inverse_w4():
    w = 4
    for op, x, y in _load("embedding_transform_w4.txt"):
        assert op == "inverse"
        assert oracle.poly_mod(int(x, 2), oracle.aop(w)) == int(y, 2)


@pytest.mark.parametrize("w,n", RINGS)
def test_ring_multiply_by_x_is_rotation(w, n):
    a = np.arange(1 << n, dtype=np.uint32)
    rot = ((a << 1) | (a >> (n - 1))) & ((1 << n) - 1)
    assert np.array_equal(oracle.ring_mul_vec(n, a, np.full_like(a, 2)), rot)


def test_ring_axioms_n5_exhaustive():
    n = 5
    q = 1 << n
    a, b, c = (x.ravel() for x in np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij"))
    ab = oracle.ring_mul_vec(n, a, b)
    assert np.array_equal(ab, oracle.ring_mul_vec(n, b, a))
    assert np.array_equal(oracle.ring_mul_vec(n, ab, c), oracle.ring_mul_vec(n, a, oracle.ring_mul_vec(n, b, c)))
    assert np.array_equal(oracle.ring_mul_vec(n, a, b ^ c), ab ^ oracle.ring_mul_vec(n, a, c))


@pytest.mark.parametrize("w,n", RINGS)
def test_idempotents_are_the_aop_closed_forms(w, n):
    # Prop. 1 with the AOP: x^n+1 = p (x+1) has two irreducible factors, so the idempotents are
    # 0, 1, theta_1, theta_2 with theta_1 = p+1 (in A_1) and theta_2 = p (in A_2) (Sec. 2.3).
    p = oracle.aop(w)
    idem = oracle.ring_idempotents(n)
    assert sorted(idem) == sorted([0, 1, p ^ 1, p])
    t1, t2 = p ^ 1, p
    assert oracle.ring_mul(n, t1, t1) == t1 and oracle.ring_mul(n, t2, t2) == t2
    assert oracle.ring_mul(n, t1, t2) == 0 and (t1 ^ t2) == 1
    assert _popcount(t1) % 2 == 0 and oracle.poly_mod(t2, p) == 0


@pytest.mark.parametrize("w,n", RINGS)
def test_phi1_is_an_isomorphism_onto_even_weight(w, n):
    p = oracle.aop(w)
    th1 = p ^ 1
    u = np.arange(1 << w, dtype=np.uint32)
    img = oracle.ring_mul_vec(n, u, np.full_like(u, th1))
    # phi^{-1}(phi(u)) = u (Eq. 2 and its AOP form): reduction mod p
    assert np.array_equal(oracle.poly_mod_vec(p, img), u)
    # image = A_1 = the even-weight polynomials (Sec. 2.3), and phi_1 is injective
    even = [r for r in range(1 << n) if _popcount(r) % 2 == 0]
    assert sorted(img.tolist()) == even


@pytest.mark.parametrize("w,n", RINGS)
def test_phi1_is_multiplicative(w, n):
    # phi(ab) = phi(a) phi(b): exhaustive for w <= 10, 2^20 sampled pairs for w = 12.
    p = oracle.aop(w)
    th1 = p ^ 1
    q = 1 << w
    if w <= 10:
        a = np.repeat(np.arange(q), q).astype(np.uint32)
        b = np.tile(np.arange(q), q).astype(np.uint32)
    else:
        rng = np.random.default_rng(12)
        a = rng.integers(0, q, 1 << 20).astype(np.uint32)
        b = rng.integers(0, q, 1 << 20).astype(np.uint32)
    T = np.full_like(a, th1)
    lhs = oracle.ring_mul_vec(n, oracle.gf_mul_vec(w, a, b), T)
    rhs = oracle.ring_mul_vec(n, oracle.ring_mul_vec(n, a, T), oracle.ring_mul_vec(n, b, T))
    assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("w,n", RINGS)
def test_representative_sets_and_sparse_transform(w, n):
    # Sec. 2.2: the ring elements standing for u are phi_1(u) + (elements with no A_1 part);
    # there are 2^{n-w} of them. phi_S picks the lightest (Sec. 2.2); for an AOP and odd n the
    # two candidates have weights t and n - t, so there is never a tie.
    p = oracle.aop(w)
    th1 = p ^ 1
    reds = oracle.poly_mod_vec(p, np.arange(1 << n, dtype=np.uint32))
    groups = {}
    for r, u in enumerate(reds.tolist()):
        groups.setdefault(u, []).append(r)
    assert sorted(groups) == list(range(1 << w))
    for u, reps in groups.items():
        assert len(reps) == 1 << (n - w)
        phi = oracle.ring_mul(n, u, th1)
        assert sorted(reps) == sorted([phi, phi ^ p])
        assert _popcount(reps[0]) != _popcount(reps[1])
    for u in ([0, 1, 2, (1 << w) - 1] + list(range(3, 1 << w, max(1, (1 << w) // 64)))):
        reps = groups[u]
        assert oracle.sparse_rep(w, n, u) == min(reps, key=lambda r: (_popcount(r), r))
        assert _popcount(oracle.sparse_rep(w, n, u)) <= n // 2


@pytest.mark.parametrize("w,n", RINGS)
def test_ring_path_equals_field_product(w, n):
    # The identity the coding path relies on: for every field u, d,
    # (phi_S(u) * phi_E(d) in R_{2,n}) mod p = u d in GF(2^w) (phi_E pads d with a zero x^w
    # coefficient; phi_E^{-1} is the reduction mod p, Sec. 2.3.2). Exhaustive for w <= 10,
    # all d against a stride of u for w = 12.
    p = oracle.aop(w)
    q = 1 << w
    reds = oracle.poly_mod_vec(p, np.arange(1 << n, dtype=np.uint32))
    # the lighter representative of each u, from the brute-force grouping
    wt = np.array([_popcount(r) for r in range(1 << n)])
    rep = np.zeros(q, np.uint32)
    best = np.full(q, 99)
    for r in range(1 << n):
        u = reds[r]
        if wt[r] < best[u]:
            best[u], rep[u] = wt[r], r
    us = np.arange(q) if w <= 10 else np.arange(0, q, 7)
    u = np.repeat(us, q).astype(np.uint32)
    d = np.tile(np.arange(q), us.size).astype(np.uint32)
    ring = oracle.ring_mul_vec(n, rep[u], d)
    assert np.array_equal(oracle.poly_mod_vec(p, ring), oracle.gf_mul_slow_vec(w, u, d))
    # and the AOP shortcut of phi_E^{-1}: XOR the x^w coefficient into every lower one
    top = (ring >> w) & 1
    short = (ring & (q - 1)) ^ (top * (q - 1))
    assert np.array_equal(short, oracle.poly_mod_vec(p, ring))
