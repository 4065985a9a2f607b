"""The weight-optimised generalized Cauchy generator (the paper's generalized Cauchy matrices,
Sec. 3; the coding cost is the number of ones of the sparse ring representatives, Sec. 2.2).

The oracle's generator is pinned to what the mathematics fixes: it is a row- and column-scaled
Cauchy matrix (so every square submatrix is nonsingular and the code is MDS, checked over all
k-subsets on small codes), its reported weights are the phi_S weights of its entries, no single
row or column rescaling lowers its weight (the coordinate descent stopped at a local optimum), and
it decodes every erasure pattern. The library's generator must equal the oracle's.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300 import pyrit

CODES = [(4, 4, 2), (10, 10, 4), (12, 16, 4), (4, 12, 4), (2, 1, 2), (12, 32, 8), (10, 20, 6)]


def _mul(w, a, b):
    return oracle.gf_mul_slow(w, int(a), int(b))


def _weight(w, u):
    return bin(oracle.sparse_rep(w, oracle.ring_size(w), int(u))).count("1")


@pytest.mark.parametrize("w,k,m", CODES)
def test_oracle_generator_is_a_scaled_cauchy_matrix(w, k, m):
    G, (w_plain, w_opt) = oracle.cauchy_weighted(w, k, m)
    assert np.array_equal(G[:k], np.eye(k, dtype=np.uint32))
    C = G[k:]
    # C'[i][j] (x_i + y_j) = a_i b_j: a rank-one matrix of nonzero elements
    R = [[_mul(w, C[i][j], (k + i) ^ j) for j in range(k)] for i in range(m)]
    for i in range(m):
        for j in range(k):
            assert R[i][j] != 0
            assert _mul(w, R[i][j], R[0][0]) == _mul(w, R[i][0], R[0][j])
    # the reported weights are the phi_S weights of the default and of the returned entries
    P = oracle.cauchy(w, k, m)[k:]
    assert w_plain == sum(_weight(w, u) for u in P.ravel())
    assert w_opt == sum(_weight(w, u) for u in C.ravel())
    assert w_opt <= w_plain


@pytest.mark.parametrize("w,k,m", [(4, 4, 2), (10, 10, 4), (4, 6, 4)])
def test_oracle_generator_is_mds(w, k, m):
    G, _ = oracle.cauchy_weighted(w, k, m)
    for rows in itertools.combinations(range(k + m), k):
        oracle.gf_invert(w, G[list(rows)])  # raises if singular


@pytest.mark.parametrize("w,k,m", [(4, 4, 2), (10, 10, 4), (4, 12, 4)])
def test_oracle_generator_is_a_local_optimum(w, k, m):
    G, (_, w_opt) = oracle.cauchy_weighted(w, k, m)
    C = G[k:]
    # rescaling one column or one row by any nonzero element never lowers the total weight
    for j in range(k):
        col = sum(_weight(w, C[i][j]) for i in range(m))
        for s in range(1, 1 << w):
            assert sum(_weight(w, _mul(w, s, C[i][j])) for i in range(m)) >= col
    for i in range(m):
        row = sum(_weight(w, C[i][j]) for j in range(k))
        for s in range(1, 1 << w):
            assert sum(_weight(w, _mul(w, s, C[i][j])) for j in range(k)) >= row


def test_oracle_generator_decodes_every_pattern():
    w, k, m, P = 4, 4, 2, 64
    G, _ = oracle.cauchy_weighted(w, k, m)
    rng = np.random.default_rng(11)
    data = rng.integers(0, 256, size=(k, w, P), dtype=np.uint8)
    full = np.concatenate([data, oracle.encode(w, k, m, G, data)])
    for e in range(1, m + 1):
        for pat in itertools.combinations(range(k + m), e):
            er = sum(1 << b for b in pat)
            blocks = full.copy()
            for b in pat:
                blocks[b] = 0
            np.testing.assert_array_equal(oracle.decode(w, k, m, G, blocks, er), full)


@pytest.mark.parametrize("w,k,m", CODES)
def test_library_generator_equals_the_oracle(w, k, m):
    G, wts = pyrit.pyrit_generator_weighted(w, oracle.ring_size(w), k, m)
    Go, wo = oracle.cauchy_weighted(w, k, m)
    np.testing.assert_array_equal(G, Go)
    assert wts == wo


def test_library_generator_errors():
    with pytest.raises(pyrit.PyritError) as ei:
        pyrit.pyrit_generator_weighted(4, 5, 14, 4)
    assert ei.value.status == pyrit.PYRIT_E_TOO_LONG
    with pytest.raises(pyrit.PyritError) as ei:
        pyrit.pyrit_generator_weighted(6, 7, 4, 2)
    assert ei.value.status == pyrit.PYRIT_E_UNSUPPORTED_FIELD
