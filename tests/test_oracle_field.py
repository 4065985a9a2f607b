"""Pins of the oracle's field arithmetic (paper Sec. 2.1 and Sec. 2.3) against facts that do not
come from the oracle itself: number theory, the field axioms and closed forms of the AOP."""
import numpy as np
import pytest

import oracle

FIELDS = [4, 10, 12]


def _isprime(x):
    return x > 1 and all(x % d for d in range(2, int(x ** 0.5) + 1))


def _order_of_2(p):
    o, v = 1, 2 % p
    while v != 1:
        v = v * 2 % p
        o += 1
    return o


def test_aop_irreducibility_criterion():
    # Sec. 2.3: the AOP of degree w is irreducible iff w+1 is prime and 2 generates the
    # multiplicative group mod w+1 (the printed "w generates" is read as "2 generates";
    # for w = 4, 4 has order 2 mod 5 and yet the example field exists, so the literal reading
    # fails). The oracle's trial division must agree with the criterion for 2 <= w <= 28.
    for w in range(2, 29):
        crit = _isprime(w + 1) and _order_of_2(w + 1) == w
        assert oracle.aop_irreducible(w) == crit, w
    # The literal reading of the garbled sentence is contradicted by the paper's own example.
    assert _order_of_2(5) == 4 and pow(4, 2, 5) == 1


def test_poly_mod_against_division_identity():
    # a = q p + r with deg r < deg p, checked with an independently written quotient.
    rng = np.random.default_rng(1)
    for _ in range(300):
        p = int(rng.integers(2, 1 << 14)) | 1
        a = int(rng.integers(0, 1 << 40))
        r = oracle.poly_mod(a, p)
        dp = p.bit_length() - 1
        assert r.bit_length() - 1 < dp
        # quotient by plain Python long division
        q, rem = 0, a
        while rem.bit_length() - 1 >= dp:
            s = rem.bit_length() - 1 - dp
            q |= 1 << s
            rem ^= p << s
        assert rem == r


@pytest.mark.parametrize("w", FIELDS)
def test_aop_closed_forms(w):
    # Under the AOP, x^{w+1} = 1 (x^{w+1}+1 = p(x)(x+1)), and x^w = 1 + x + ... + x^{w-1}.
    n = w + 1
    v = 1
    for _ in range(n):
        v = oracle.gf_mul_slow(w, v, 2)
    assert v == 1
    v = 1
    for _ in range(w):
        v = oracle.gf_mul_slow(w, v, 2)
    assert v == (1 << w) - 1
    assert oracle.gf_order(w, 2) == n


def test_field_axioms_exhaustive_w4():
    w = 4
    q = 1 << w
    a, b, c = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    a, b, c = a.ravel(), b.ravel(), c.ravel()
    ab = oracle.gf_mul_slow_vec(w, a, b)
    assert np.array_equal(ab, oracle.gf_mul_slow_vec(w, b, a))
    assert np.array_equal(oracle.gf_mul_slow_vec(w, ab, c),
                          oracle.gf_mul_slow_vec(w, a, oracle.gf_mul_slow_vec(w, b, c)))
    assert np.array_equal(oracle.gf_mul_slow_vec(w, a, b ^ c),
                          ab ^ oracle.gf_mul_slow_vec(w, a, c))


@pytest.mark.parametrize("w", FIELDS)
def test_every_nonzero_element_invertible(w):
    # A field: every nonzero a has some b with a b = 1 (brute force over all pairs).
    q = 1 << w
    a = np.repeat(np.arange(1, q), q - 1)
    b = np.tile(np.arange(1, q), q - 1)
    prod = oracle.gf_mul_slow_vec(w, a, b).reshape(q - 1, q - 1)
    assert np.all((prod == 1).sum(axis=1) == 1)


@pytest.mark.parametrize("w", FIELDS)
def test_primitive_element_and_tables(w):
    q1 = (1 << w) - 1
    g = oracle.gf_primitive(w)
    # order of g is 2^w - 1 and every smaller candidate has a smaller order
    assert oracle.gf_order(w, g) == q1
    for h in range(2, g):
        assert oracle.gf_order(w, h) < q1
    log, alog, g2 = oracle.gf_tables(w)
    assert g2 == g
    # antilog enumerates every nonzero element once; log inverts it
    assert sorted(alog[:q1].tolist()) == list(range(1, q1 + 1))
    assert np.array_equal(log[alog[:q1]], np.arange(q1))


@pytest.mark.parametrize("w", FIELDS)
def test_table_multiply_equals_definition(w):
    q = 1 << w
    a = np.repeat(np.arange(q), q)
    b = np.tile(np.arange(q), q)
    assert np.array_equal(oracle.gf_mul_vec(w, a, b), oracle.gf_mul_slow_vec(w, a, b))


def test_unsupported_fields_rejected():
    # w = 6: the AOP x^6+...+1 = (x^3+x+1)(x^3+x^2+1) is reducible; GF(2^6) comes from the ESP
    # x^6+x^3+1 instead (Sec. 2.4). w = 3, 8, 9: neither an irreducible AOP nor an irreducible ESP.
    assert oracle.poly_mod(oracle.aop(6), 0b1011) == 0 and not oracle.aop_irreducible(6)
    assert oracle.field_poly(6) == 0b1001001
    for w in (3, 8, 9):
        assert oracle.field_poly(w) == 0 and oracle.ring_size(w) == 0
        with pytest.raises(ValueError):
            oracle.gf_tables(w)
        with pytest.raises(ValueError):
            oracle.cauchy(w, 3, 2)
