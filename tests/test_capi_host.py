"""Host-side checks of the C ABI (no GPU): the library exports every declared symbol, and the
planner's field arithmetic, sparse transform (Sec. 2.2), default generator and decoding matrices
(Sec. 4.3) agree with the independent CPU oracle; invalid calls return their documented codes
before any device work."""
import ctypes
import glob
import itertools
import os
import re

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300 import pyrit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RINGS = [(2, 3), (4, 5), (6, 9), (10, 11), (12, 13)]


def test_library_exports_every_declared_symbol():
    declared = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        declared |= set(re.findall(r"PYRIT_API\s+[\w\s\*]+?\b(pyrit_\w+)\s*\(", open(h).read()))
    assert declared, "no declarations found"
    lib = ctypes.CDLL(pyrit.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(pyrit.EXPORTS)


def _brute_sparse(w, n):
    """phi_S for every u by brute force over all 2^n ring elements (oracle reduction)."""
    p = oracle.field_poly(w)
    reds = oracle.poly_mod_vec(p, np.arange(1 << n, dtype=np.uint32))
    best = {}
    for r, u in enumerate(reds.tolist()):
        key = (bin(r).count("1"), r)
        if u not in best or key < best[u][0]:
            best[u] = (key, r)
    return np.array([best[u][1] for u in range(1 << w)], np.uint32)


@pytest.mark.parametrize("w,n", RINGS)
def test_sparse_transform_matches_brute_force(w, n):
    ref = _brute_sparse(w, n)
    got = np.array([pyrit.pyrit_sparse_transform(w, n, u) for u in range(1 << w)], np.uint32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("w", [2, 4, 6, 10, 12])
def test_planner_field_product(w):
    q = 1 << w
    rng = np.random.default_rng(w)
    if w <= 10:
        a = np.repeat(np.arange(q), q)
        b = np.tile(np.arange(q), q)
        if w == 10:
            sel = rng.choice(a.size, 200000, replace=False)
            a, b = a[sel], b[sel]
    else:
        a = rng.integers(0, q, 200000)
        b = rng.integers(0, q, 200000)
    ref = oracle.gf_mul_slow_vec(w, a, b)
    got = np.array([pyrit.pyrit_gf_mul(w, int(x), int(y)) for x, y in zip(a, b)], np.uint32)
    assert np.array_equal(got, ref)


def test_field_support_matches_oracle_irreducibility():
    # The planner accepts (w, n) by the paper's number-theoretic criteria for its native fields
    # (Sec. 2.3 for AOPs, Sec. 2.4 for ESPs) and, for any other odd n <= 15, by the factors of
    # x^n + 1 (Props. 1-2); the oracle finds each modulus by trial division. They must agree on
    # every pair: which (w, n) exist, which modulus is used, which are native.
    for w in range(2, 16):
        for n in range(w + 1, 17):
            native = oracle.ring_size(w) == n and n in (3, 5, 9, 11, 13)
            general = n % 2 == 1 and n <= 15 and oracle.ring_factor(w, n) != 0
            try:
                h = pyrit.pyrit_plan_create(w, n, 1, 1)
            except pyrit.PyritError as e:
                assert e.status == pyrit.PYRIT_E_UNSUPPORTED_FIELD
                assert not native and not general, (w, n)
                continue
            try:
                g, nat = pyrit.pyrit_plan_modulus(h)
                assert nat == native, (w, n)
                assert g == (oracle.field_poly(w) if native else oracle.ring_factor(w, n)), (w, n)
            finally:
                pyrit.pyrit_plan_destroy(h)
    assert oracle.ring_size(6) == 9


@pytest.mark.parametrize("w,k,m", [(2, 2, 2), (4, 4, 2), (10, 10, 4), (12, 16, 4), (4, 12, 4), (12, 32, 8),
                                   (6, 8, 4), (6, 32, 8)])
def test_default_generator_and_encode_masks(w, k, m):
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        assert pyrit.pyrit_plan_info(plan) == (w, oracle.ring_size(w), k, m)
        G = pyrit.pyrit_plan_generator(plan)
        assert np.array_equal(G, oracle.cauchy(w, k, m))
        sp = _brute_sparse(w, oracle.ring_size(w))
        assert np.array_equal(pyrit.pyrit_plan_encode_masks(plan), sp[G[k:]].astype(np.uint16))
    finally:
        pyrit.pyrit_plan_destroy(plan)


@pytest.mark.parametrize("w,k,m", [(10, 10, 4), (12, 16, 4)])
def test_plan_with_16_bit_generator(w, k, m):
    # pyrit_plan takes the generator as 16-bit entries: the oracle's Cauchy matrix given that way,
    # and the default (NULL), make the same plan as pyrit_plan_create; a non-systematic G is refused.
    n = oracle.ring_size(w)
    G = oracle.cauchy(w, k, m)
    for g in (G.astype(np.uint16), None):
        plan = pyrit.pyrit_plan(w, n, k, m, g)
        try:
            assert np.array_equal(pyrit.pyrit_plan_generator(plan), G)
        finally:
            pyrit.pyrit_plan_destroy(plan)
    bad = G.astype(np.uint16)
    bad[0, 1] = 1
    with pytest.raises(pyrit.PyritError) as ei:
        pyrit.pyrit_plan(w, n, k, m, bad)
    assert ei.value.status == pyrit.PYRIT_E_NOT_MDS


def _oracle_decode_matrix(w, k, m, G, erasures):
    surv = [e for e in range(k + m) if not (erasures >> e) & 1][:k]
    erased = [e for e in range(k + m) if (erasures >> e) & 1]
    Inv = oracle.gf_invert(w, G[surv])
    rows = []
    for e in erased:
        if e < k:
            rows.append(Inv[e])
        else:
            r = np.zeros(k, np.uint32)
            for s in range(k):
                acc = 0
                for j in range(k):
                    acc ^= oracle.gf_mul_slow(w, int(G[e, j]), int(Inv[j, s]))
                r[s] = acc
            rows.append(r)
    return np.array(surv), np.array(erased), np.array(rows, np.uint32).reshape(len(erased), k)


@pytest.mark.parametrize("w,k,m,exhaustive", [(4, 4, 2, True), (10, 10, 4, False), (12, 16, 4, False),
                                             (6, 8, 4, False)])
def test_decode_masks_match_oracle(w, k, m, exhaustive):
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    sp = _brute_sparse(w, oracle.ring_size(w))
    try:
        G = oracle.cauchy(w, k, m)  # the oracle's own generator (the library's is pinned equal above)
        if exhaustive:
            pats = [sum(1 << x for x in c) for e in range(0, m + 1) for c in itertools.combinations(range(k + m), e)]
        else:
            rng = np.random.default_rng(k)
            pats = [0] + [sum(1 << int(x) for x in rng.choice(k + m, int(rng.integers(1, m + 1)), replace=False))
                          for _ in range(25)]
        for pat in pats:
            surv, er, M = pyrit.pyrit_plan_decode_masks(plan, pat)
            s2, e2, D = _oracle_decode_matrix(w, k, m, G, pat)
            assert list(surv) == list(s2) and list(er) == list(e2)
            assert np.array_equal(M, sp[D].astype(np.uint16)), hex(pat)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_error_codes():
    E = pyrit
    cases = [
        (lambda: E.pyrit_plan_create(6, 7, 3, 2), E.PYRIT_E_UNSUPPORTED_FIELD),   # AOP reducible (ESP ring: n=9)
        (lambda: E.pyrit_plan_create(4, 6, 3, 2), E.PYRIT_E_UNSUPPORTED_FIELD),   # n != w+1
        (lambda: E.pyrit_plan_create(4, 5, 12, 5), E.PYRIT_E_TOO_LONG),           # k+m > 16
        (lambda: E.pyrit_plan_create(4, 5, 0, 2), E.PYRIT_E_INVALID_ARG),
        (lambda: E.pyrit_plan_create(4, 5, 65, 2), E.PYRIT_E_INVALID_ARG),           # k > 64
        (lambda: E.pyrit_plan_create(6, 9, 40, 25), E.PYRIT_E_INVALID_ARG),          # k + m > 64
        (lambda: E.pyrit_plan_create(4, 5, 33, 2), E.PYRIT_E_TOO_LONG),              # k + m > 16
        (lambda: E.pyrit_plan_create(4, 5, 4, 64), E.PYRIT_E_INVALID_ARG),           # m > 63
    ]
    for f, code in cases:
        with pytest.raises(E.PyritError) as ei:
            f()
        assert ei.value.status == code


def test_user_generator_validation():
    w, k, m = 4, 3, 2
    G = oracle.cauchy(w, k, m)
    h = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m, G)
    pyrit.pyrit_plan_destroy(h)
    bad = G.copy()
    bad[0, 1] = 1  # not systematic
    with pytest.raises(pyrit.PyritError) as ei:
        pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m, bad)
    assert ei.value.status == pyrit.PYRIT_E_NOT_MDS
    sing = G.copy()
    sing[k + 1] = sing[k]  # two equal parity rows: a singular 3x3 subset
    with pytest.raises(pyrit.PyritError) as ei:
        pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m, sing)
    assert ei.value.status == pyrit.PYRIT_E_NOT_MDS
    big = G.copy()
    big[k, 0] = 16
    with pytest.raises(pyrit.PyritError) as ei:
        pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m, big)
    assert ei.value.status == pyrit.PYRIT_E_NOT_MDS


def test_invalid_coding_calls_fail_before_device_work():
    plan = pyrit.pyrit_plan_create(4, 5, 4, 2)
    try:
        fake = [16 * (i + 1) for i in range(6)]
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_decode(plan, fake, 0b111, 64)  # 3 erasures > m = 2
        assert ei.value.status == pyrit.PYRIT_E_TOO_MANY_ERASURES
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_decode(plan, fake, 1 << 6, 64)  # bit outside the stripe
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_encode(plan, fake[:4], fake[4:], 0)  # P = 0
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_encode(plan, fake[:3] + [0], fake[4:], 64)  # null block
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
        assert pyrit.pyrit_decode(plan, fake, 0, 64) == 0  # nothing erased: no work
        # the one-shot batched calls take stripes of their own operation only
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_encode_batch([(plan, pyrit.PYRIT_OP_DECODE, 0b1, 64, fake)])
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_decode_batch([(plan, pyrit.PYRIT_OP_DECODE, 0b1, 64, fake),
                                      (plan, pyrit.PYRIT_OP_ENCODE, 0, 64, fake)])
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
        assert pyrit.pyrit_encode_batch([]) == 0 and pyrit.pyrit_decode_batch([]) == 0
        arr, keep = pyrit.pyrit_requests_array([])
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_server_replay(None, arr, 0, 0)  # no server
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_tune_table_save_load_roundtrip(tmp_path):
    # Host-only: an entry written in the documented format loads back and saves identically.
    path = tmp_path / "t.json"
    path.write_text('[\n  {"n": 13, "shared": 0, "nout": 4, "plog2": 15, "words": 4, "mg": 1, "minb": 1, '
                    '"nc": 12, "dispatch": 0, "stages": 4, "ms": 0.250000}\n]\n')
    assert pyrit.pyrit_tune_load(str(path)) == 1
    out = tmp_path / "o.json"
    pyrit.pyrit_tune_save(str(out))
    assert '"n": 13, "shared": 0, "nout": 4, "plog2": 15, "words": 4' in out.read_text()
    # clearing forgets every entry
    assert pyrit.pyrit_tune_clear() >= 1
    pyrit.pyrit_tune_save(str(out))
    assert '"n": 13' not in out.read_text()
    assert pyrit.pyrit_tune_clear() == 0
