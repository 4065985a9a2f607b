"""Pins of the oracle's parity-transform code (Sec. 2.3.1).

The paper's phi_P pads a field element with its parity bit (an even-weight ring element, i.e. an
element of the ideal A_1) and phi_P^{-1} drops that bit; encoder and decoder both use it, so the
code differs from the plain field code. What fixes it independently of the oracle's ring-literal
implementation: for psi(d) = phi_P(d) mod p = d + par(d) (1 + x + ... + x^{w-1}),
    phi_P^{-1}( phi_S(u) * phi_P(d) ) = psi^{-1}( u psi(d) )
(phi_P(d) lies in A_1, where multiplying by any representative of u is multiplying by u after
phi_1^{-1} = mod p). So the parity-transform code is the field code conjugated symbol by symbol by
psi, an involution for even w. On bit-sliced blocks psi XORs every symbol's parity packet into
each of its packets.
"""
import itertools

import numpy as np
import pytest

import oracle


def _par(d):
    return bin(int(d)).count("1") & 1


def _phi_P(w, d):
    return int(d) | (_par(d) << w)


def _psi(w, d):
    return int(oracle.poly_mod(_phi_P(w, d), oracle.aop(w)))


@pytest.mark.parametrize("w", [2, 4, 10])
def test_psi_is_an_involution(w):
    for d in range(1 << w):
        assert _psi(w, _psi(w, d)) == d
        # the closed form of psi: every coefficient flipped by the parity bit
        assert _psi(w, d) == d ^ ((1 << w) - 1 if _par(d) else 0)


@pytest.mark.parametrize("w,exhaustive", [(4, True), (10, False)])
def test_parity_transform_product_is_the_conjugated_field_product(w, exhaustive):
    n = w + 1
    rng = np.random.default_rng(w)
    pairs = itertools.product(range(1 << w), range(1 << w)) if exhaustive else \
        [(int(a), int(b)) for a, b in rng.integers(0, 1 << w, size=(4000, 2))]
    for u, d in pairs:
        ring = oracle.ring_mul(n, oracle.sparse_rep(w, n, u), _phi_P(w, d)) & ((1 << w) - 1)
        field = _psi(w, oracle.gf_mul_slow(w, u, _psi(w, d)))
        assert ring == field, (u, d)


def _psi_blocks(blocks):
    """psi on bit-sliced blocks (..., w, P): every lane's parity XORed into each of its packets."""
    par = np.bitwise_xor.reduce(blocks, axis=-2, keepdims=True)
    return blocks ^ par


@pytest.mark.parametrize("w,k,m,P", [(4, 4, 2, 96), (10, 10, 4, 64), (12, 5, 3, 48), (2, 1, 2, 32)])
def test_encode_pt_is_the_field_code_conjugated_by_psi(w, k, m, P):
    rng = np.random.default_rng(k * 31 + m)
    G = oracle.cauchy(w, k, m)
    data = rng.integers(0, 256, size=(k, w, P), dtype=np.uint8)
    got = oracle.encode_pt(w, k, m, G, data)
    want = _psi_blocks(oracle.encode(w, k, m, G, _psi_blocks(data)))
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("w,k,m,P,exhaustive", [(4, 4, 2, 64, True), (10, 10, 4, 48, False)])
def test_decode_pt_recovers_erasures(w, k, m, P, exhaustive):
    rng = np.random.default_rng(97 + k)
    G = oracle.cauchy(w, k, m)
    data = rng.integers(0, 256, size=(k, w, P), dtype=np.uint8)
    full = np.concatenate([data, oracle.encode_pt(w, k, m, G, data)])
    pats = [c for e in range(1, m + 1) for c in itertools.combinations(range(k + m), e)]
    if not exhaustive:
        pats = [pats[i] for i in rng.choice(len(pats), 60, replace=False)]
    for pat in pats:
        blocks = full.copy()
        for b in pat:
            blocks[b] = 0xA5
        np.testing.assert_array_equal(oracle.decode_pt(w, k, m, G, blocks, sum(1 << b for b in pat)), full)
