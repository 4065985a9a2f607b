"""Plan-specialised networks on the host (no GPU).

The library writes, for a mask table, the multiply-accumulate step of the staged kernel as
straight-line XORs (one expression per ring accumulator and output, per source). These tests read
that generated source back, interpret its XOR lists on single symbol lanes and compare them with the
oracle: the network of mask r must be multiplication by r in R_{2,n} (paper Sec. 2.3.2 / Sec. 3),
and after the phi_E^{-1} fold (out_t = acc_t + acc_w) the field product by the coefficient whose
sparse representative r is (Sec. 2.2). The map is linear in the source, so checking every basis
vector x^q (q < w) is exhaustive. They also run the run-time compiler (NVRTC) for sm_103a, which
needs no device.
"""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300 import pyrit


SECOND = 1000  # column offset of the second source of a pair step (d2, dp2)


def _terms(text, temps):
    """Source columns of an XOR expression: d[q][x] is packet q of the source; dp[j][x] (the parity
    transform's padding packet j, the parity of the source's interleaved word j) is recorded as
    q = -1 - j; d2 / dp2 (the second source of a pair step) as the same plus SECOND (minus SECOND
    for dp2); a temporary e<id> stands for the columns it was formed from."""
    qs = []
    for name, idx, e in re.findall(r"\b(d|dp|d2|dp2)\[(\d+)\]\[x\]|\be(\d+)\b", text):
        if e:
            qs += temps[int(e)]
        elif name == "d":
            qs.append(int(idx))
        elif name == "dp":
            qs.append(-1 - int(idx))
        elif name == "d2":
            qs.append(SECOND + int(idx))
        else:
            qs.append(-1 - int(idx) - SECOND)
    return qs


def _split_pair(qs):
    """Columns of a pair step's expression, split into (first source's, second source's)."""
    a = [q for q in qs if -SECOND < q < SECOND]
    b = [q - SECOND if q >= SECOND else q + SECOND for q in qs if q >= SECOND or q <= -SECOND]
    return a, b


def _parse(src):
    """Cases of a generated network: entries (slot, accumulator, source columns). A syndrome
    network's case has two bodies: the one taken when every parity row is needed (its entries in
    `cases_all`) and the per-row guarded one (in `cases`, with each entry's guard in `guards`)."""
    nin = int(re.search(r"switch \(g \* (\d+) \+ j\)", src).group(1))
    n, words, mg, nc = map(int, re.search(r"ring_staged_body<(\d+), (\d+), (\d+), (\d+),", src).groups())
    cases, cases_all, cur, temps, guard, guards, in_all, full = {}, {}, None, {}, None, [], False, None
    # pair steps (sources 2p and 2p + 1 in one case of apply2): entries kept per case, split below
    npairs, in_pair, pair_cases = None, False, {}
    for line in src.splitlines():
        sw = re.match(r"\s*switch \(g \* (\d+) \+ j / 2\) \{", line)
        if sw:
            npairs, in_pair = int(sw.group(1)), True
            continue
        c = re.match(r"\s*case (\d+): \{", line)
        if c:
            cur = int(c.group(1))
            if in_pair:
                pair_cases[cur] = []
            else:
                cases.setdefault(cur, [])
                cases_all[cur] = []
            temps, guard, in_all = {}, None, False
            continue
        # syndrome networks: the body for a tile that needs every parity row, then the else branch
        fa = re.match(r"\s*if \(need == (\d+)u\) \{", line)
        if fa:
            full, in_all = int(fa.group(1)), True
            continue
        if re.match(r"\s*\} else \{", line):
            in_all, temps = False, {}  # the guarded body numbers its own temporaries
            continue
        # the accumulations of one parity row under a test of the needed rows
        gd = re.match(r"\s*if \(need & (\d+)u\) \{", line)
        if gd:
            guard = int(gd.group(1))
            continue
        # a shared term: const uint32_t e<id> = a ^ b;   or   = xor3(a, b, c);
        t = re.match(r"\s*const uint32_t e(\d+) = (.*);", line)
        if t:
            assert cur is not None and int(t.group(1)) not in temps, "a temporary is defined once per case"
            temps[int(t.group(1))] = _terms(t.group(2), temps)
            continue
        # acc[i][t][x] ^= term;   or   acc[i][t][x] = xor3(acc[i][t][x], term, term);
        a = re.match(r"\s*acc\[(\d+)\]\[(\d+)\]\[x\] \^= (.*);", line)
        b = re.match(r"\s*acc\[(\d+)\]\[(\d+)\]\[x\] = xor3\(acc\[(\d+)\]\[(\d+)\]\[x\], (.*)\);", line)
        if b:
            assert b.group(1, 2) == b.group(3, 4), "a three-input XOR must update its own accumulator"
            a = b
        if a:
            assert cur is not None
            entry = (int(a.group(1)), int(a.group(2)), _terms(a.groups()[-1], temps))
            if in_pair:
                pair_cases[cur].append(entry)
                continue
            if in_all:
                cases_all[cur].append(entry)
            else:
                cases[cur].append(entry)
                guards.append((int(a.group(1)), guard))
        if "} break;" in line:
            cur = None
    for pc, entries in pair_cases.items():
        g, p = divmod(pc, npairs)
        for (ii, t, qs) in entries:
            a, b = _split_pair(qs)
            cases.setdefault(g * nin + 2 * p, []).append((ii, t, a))
            cases.setdefault(g * nin + 2 * p + 1, []).append((ii, t, b))
            guards += [(ii, None), (ii, None)]
    return dict(nin=nin, n=n, words=words, mg=mg, nc=nc, cases=cases, guards=guards, cases_all=cases_all, full=full,
                npairs=npairs)


def _w_of(n):
    """The field degree the oracle carries on R_{2,n} (n - 1 for an AOP, 6 for n = 9)."""
    return next(w for w in range(2, 16) if oracle.ring_size(w) == n)


def _ring_columns(entries, ii, n, w):
    """Ring accumulators of output slot ii for each basis source x^q: list of n-bit ints."""
    cols = []
    for q in range(w):
        acc = 0
        for (i, t, qs) in entries:
            if i == ii:
                for qq in qs:
                    assert 0 <= qq < w, "the zero packet of the embedding must not be read"
                    if qq == q:
                        acc ^= 1 << t
        cols.append(acc)
    return cols


def _check_network(src, masks, n):
    """masks[o][j]: the table the source was generated for. Every (j, o) must be covered once."""
    net = _parse(src)
    w = _w_of(n)
    nout, nin = masks.shape
    assert net["n"] == n and net["nin"] == nin
    mg = net["mg"]
    seen = set()
    for case, entries in net["cases"].items():
        g, j = divmod(case, nin)
        for ii in range(mg):
            o = g * mg + ii
            if o >= nout:
                assert not [e for e in entries if e[0] == ii], "a slot past the outputs is written"
                continue
            seen.add((j, o))
            cols = _ring_columns(entries, ii, n, w)
            for q in range(w):
                assert cols[q] == oracle.ring_mul(n, int(masks[o][j]), 1 << q), (case, ii, q)
    assert seen == {(j, o) for j in range(nin) for o in range(nout)}
    return net


def _oracle_parity_masks(w, k, m):
    G = oracle.cauchy(w, k, m)
    C = G[k:]
    masks = np.array([[oracle.sparse_rep(w, oracle.ring_size(w), int(C[o][j])) for j in range(k)] for o in range(m)], np.uint16)
    return C, masks


@pytest.mark.parametrize("w,k,m", [(10, 10, 4), (12, 16, 4), (4, 8, 8), (2, 1, 2), (10, 32, 8), (6, 8, 4), (6, 32, 8)])
def test_generated_network_is_the_field_product(w, k, m):
    n = oracle.ring_size(w)
    C, masks = _oracle_parity_masks(w, k, m)
    net = _check_network(pyrit.pyrit_jit_source(n, masks), masks, n)
    # phi_E^{-1} of the ring columns gives the field product by the Cauchy coefficient
    for case, entries in net["cases"].items():
        g, j = divmod(case, k)
        for ii in range(net["mg"]):
            o = g * net["mg"] + ii
            if o >= m:
                continue
            for q, col in enumerate(_ring_columns(entries, ii, n, w)):
                field = oracle.poly_mod(col, oracle.field_poly(w))
                assert field == oracle.gf_mul_slow(w, int(C[o][j]), 1 << q)


@pytest.mark.parametrize("n", [3, 5, 9, 11, 13])
def test_generated_network_random_masks_and_shapes(n):
    rng = np.random.default_rng(1000 + n)
    shapes = [None, {"mg": 0, "nc": 16}, {"words": 2, "nc": 8}]
    for trial in range(6):
        nin = int(rng.integers(1, 65))
        nout = int(rng.integers(1, 9))
        masks = rng.integers(0, 1 << n, size=(nout, nin)).astype(np.uint16)
        masks[0][0] = 0                 # a zero coefficient writes nothing
        masks[-1][-1] = (1 << n) - 1    # every shift
        tile = shapes[trial % len(shapes)]
        if trial == 5 and nout >= 2:
            tile = {"mg": (nout + 1) // 2, "nc": 16}  # two output groups
        _check_network(pyrit.pyrit_jit_source(n, masks, tile), masks, n)


def test_output_groups_split_the_outputs():
    C, masks = _oracle_parity_masks(10, 10, 8)
    net = _check_network(pyrit.pyrit_jit_source(11, masks, {"mg": 4, "nc": 16}), masks, 11)
    assert net["mg"] == 4 and max(net["cases"]) == 2 * 10 - 1


def test_jit_source_rejects_bad_tables():
    masks = np.zeros((4, 10), np.uint16)
    for bad in [(7, masks, None), (11, np.zeros((9, 10), np.uint16), None), (11, np.zeros((4, 65), np.uint16), None),
                (11, masks, {"words": 3}), (11, masks, {"nc": 40})]:
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_jit_source(*bad)
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG


def test_jit_mode_roundtrip():
    prev = pyrit.pyrit_jit_mode()
    try:
        assert pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_OFF) == prev
        assert pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_SYNC) == pyrit.PYRIT_JIT_OFF
        assert pyrit.pyrit_jit_mode() == pyrit.PYRIT_JIT_SYNC
        with pytest.raises(pyrit.PyritError):
            pyrit.pyrit_jit_mode(7)
    finally:
        pyrit.pyrit_jit_mode(prev)


@pytest.mark.parametrize("w,k,m", [(2, 1, 2), (4, 8, 4), (10, 10, 4), (12, 16, 4)])
def test_runtime_compiler_builds_networks_without_a_device(w, k, m):
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        before = pyrit.pyrit_jit_stats()
        pyrit.pyrit_plan_specialise(plan)
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE, 0b11)
        mid = pyrit.pyrit_jit_stats()
        assert mid["failed"] == before["failed"], pyrit.pyrit_jit_log()
        # the same tables again are cache hits: nothing new is compiled
        pyrit.pyrit_plan_specialise(plan)
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE, 0b11)
        after = pyrit.pyrit_jit_stats()
        assert after["compiled"] == mid["compiled"] and after["cached"] == mid["cached"]
        # two networks, each in its batch form and its served form (which stamps completions)
        assert mid["cached"] - before["cached"] <= 4
        # nothing erased: nothing to specialise
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE, 0)
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE, (1 << (m + 1)) - 1)
        assert ei.value.status == pyrit.PYRIT_E_TOO_MANY_ERASURES
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_plan_specialise(plan, tile={"words": 3})
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
    finally:
        pyrit.pyrit_plan_destroy(plan)


@pytest.mark.parametrize("w,k,m", [(4, 4, 2), (10, 10, 4), (12, 16, 4), (6, 8, 4)])
def test_syndrome_network_is_the_parity_check_product(w, k, m):
    """The first phase of a plan's syndrome-decode network, read back: for block column j of
    [C | I_m], parity row i accumulates the ring product of column j's packets by phi_S(C[i][j])
    (by 1 for its own parity block, by 0 for another's), every accumulation of row i sits under
    the tile's test of row i, and the field value after phi_E^{-1} is the oracle's product."""
    n = oracle.ring_size(w)
    C, masks = _oracle_parity_masks(w, k, m)
    plan = pyrit.pyrit_plan_create(w, n, k, m)
    try:
        net = _parse(pyrit.pyrit_plan_network_source(plan, pyrit.PYRIT_OP_DECODE_ANY))
    finally:
        pyrit.pyrit_plan_destroy(plan)
    assert net["nin"] == k + m and net["mg"] >= m
    assert net["guards"] and all(g == 1 << i for i, g in net["guards"])
    # the body taken when every row is needed: same products, terms shared across rows
    assert net["full"] == (1 << net["mg"]) - 1
    for body in (net["cases"], net["cases_all"]):
        for j in range(k + m):
            entries = body[j]
            for i in range(net["mg"]):
                r = int(masks[i][j]) if (i < m and j < k) else int(j - k == i)
                cols = _ring_columns(entries, i, n, w)
                for q in range(w):
                    assert cols[q] == oracle.ring_mul(n, r, 1 << q), (j, i, q)
                    if i < m:
                        u = int(C[i][j]) if j < k else r
                        assert oracle.poly_mod(cols[q], oracle.field_poly(w)) == oracle.gf_mul_slow(w, u, 1 << q)


def _field_of_mask(w, mask):
    """The field element a ring representative stands for: its remainder mod the AOP."""
    return int(oracle.poly_mod(mask, oracle.aop(w)))


@pytest.mark.parametrize("w,k,m", [(4, 4, 2), (10, 10, 4), (12, 16, 4), (4, 6, 4), (10, 24, 8)])
def test_syndrome_tables_rebuild_every_erasure_pattern(w, k, m):
    """The planner's syndrome-form decode (second phase of the syndrome network), checked with the
    oracle's field arithmetic only: random symbols are encoded with the oracle's Cauchy generator,
    the first phase's row sums are formed from the survivors, and every erased symbol must come
    back from the per-pattern coefficients."""
    from itertools import combinations
    rng = np.random.default_rng(77 + w * k + m)
    G = oracle.cauchy(w, k, m)
    C = G[k:]
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        patterns = []
        for e in range(1, m + 1):
            combos = list(combinations(range(k + m), e))
            if len(combos) > 300:
                combos = [combos[i] for i in rng.choice(len(combos), 300, replace=False)]
            patterns += combos
        for pat in patterns:
            er = sum(1 << b for b in pat)
            d = [int(x) for x in rng.integers(0, 1 << w, size=k)]
            p = [0] * m
            for r in range(m):
                for j in range(k):
                    p[r] ^= oracle.gf_mul_slow(w, int(C[r][j]), d[j])
            block = d + p
            erased = sorted(pat)
            survivors = [b for b in range(k + m) if b not in pat][:k]
            U = [b - k for b in survivors if b >= k]
            acc = []
            for r in range(m):
                v = 0
                for j in range(k):
                    if j not in pat:
                        v ^= oracle.gf_mul_slow(w, int(C[r][j]), d[j])
                if r in U:
                    v ^= p[r]
                acc.append(v)
            syn, ne = pyrit.pyrit_plan_syndrome_masks(plan, er)
            assert ne == len(erased)
            for o, b in enumerate(erased):
                base = int(syn[8][o])
                v = acc[base - 1] if base else 0
                assert (base == 0) == (b < k)
                for r in range(m):
                    if syn[r][o]:
                        assert r in U, "only syndrome rows carry coefficients"
                        v ^= oracle.gf_mul_slow(w, _field_of_mask(w, int(syn[r][o])), acc[r])
                assert v == block[b], (pat, b)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def _psi(w, d):
    """phi_P(d) mod the field's modulus (Sec. 2.3.1, Sec. 2.4.1), from the oracle."""
    return oracle.poly_mod(oracle.phi_P(w, oracle.ring_size(w), d), oracle.field_poly(w))


def _parity_columns(entries, ii, n, w):
    """Ring rows of output slot ii for each basis source x^q under the parity transform: padding
    packet j (the parity of the source's interleaved word j, coefficients j, j + S, ...) is 1 for
    the basis vector x^q exactly when q = j mod S, S = n - w."""
    S = n - w
    cols = []
    for q in range(w):
        acc = 0
        for (i, t, qs) in entries:
            if i != ii:
                continue
            assert t < w, "the parity transform drops the top ring rows: they must not be accumulated"
            for qq in qs:
                assert -S <= qq < w
                if qq == q or qq == -1 - q % S:
                    acc ^= 1 << t
        cols.append(acc)
    return cols


@pytest.mark.parametrize("w,k,m", [(10, 10, 4), (12, 16, 4), (4, 8, 8), (2, 1, 2), (10, 32, 8), (6, 8, 4), (6, 20, 8)])
def test_generated_parity_network_is_the_conjugated_field_product(w, k, m):
    """Under the parity transform the network of mask r maps a source d to the low w coefficients
    of r * phi_P(d) in R_{2,n} (phi_P pads d with its parity bit, phi_P^{-1} drops the top one);
    that is psi(u * psi(d)) for the field coefficient u, psi(d) = phi_P(d) mod p."""
    n = oracle.ring_size(w)
    C, masks = _oracle_parity_masks(w, k, m)
    net = _parse(pyrit.pyrit_jit_source(n, masks, None, pyrit.PYRIT_TRANSFORM_PARITY))
    assert net["n"] == n and net["nin"] == k
    seen = set()
    for case, entries in net["cases"].items():
        g, j = divmod(case, k)
        for ii in range(net["mg"]):
            o = g * net["mg"] + ii
            if o >= m:
                assert not [e for e in entries if e[0] == ii]
                continue
            seen.add((j, o))
            for q, col in enumerate(_parity_columns(entries, ii, n, w)):
                ring = oracle.ring_mul(n, int(masks[o][j]), oracle.phi_P(w, n, 1 << q)) & ((1 << w) - 1)
                assert col == ring, (case, ii, q)
                assert col == _psi(w, oracle.gf_mul_slow(w, int(C[o][j]), _psi(w, 1 << q)))
    assert seen == {(j, o) for j in range(k) for o in range(m)}


@pytest.mark.parametrize("n", [3, 5, 9, 11, 13])
def test_generated_parity_network_random_masks(n):
    rng = np.random.default_rng(2000 + n)
    w = _w_of(n)
    for trial in range(4):
        nin = int(rng.integers(1, 65))
        nout = int(rng.integers(1, 9))
        masks = rng.integers(0, 1 << n, size=(nout, nin)).astype(np.uint16)
        masks[-1][-1] = (1 << n) - 1
        tile = [None, {"mg": 0, "nc": 16}, {"words": 2, "nc": 8}, None][trial]
        net = _parse(pyrit.pyrit_jit_source(n, masks, tile, pyrit.PYRIT_TRANSFORM_PARITY))
        for case, entries in net["cases"].items():
            g, j = divmod(case, nin)
            for ii in range(net["mg"]):
                o = g * net["mg"] + ii
                if o >= nout:
                    continue
                for q, col in enumerate(_parity_columns(entries, ii, n, w)):
                    assert col == oracle.ring_mul(n, int(masks[o][j]), oracle.phi_P(w, n, 1 << q)) & ((1 << w) - 1)


def test_plan_transform_setting():
    plan = pyrit.pyrit_plan_create(10, 11, 10, 4)
    try:
        assert pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_PARITY) == pyrit.PYRIT_TRANSFORM_PARITY
        assert pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_EMBEDDING) == pyrit.PYRIT_TRANSFORM_EMBEDDING
        # AUTO: the parity transform when k < m (Sec. 2.3.1), else the embedding
        assert pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_AUTO) == pyrit.PYRIT_TRANSFORM_EMBEDDING
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_plan_set_transform(plan, 5)
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
    finally:
        pyrit.pyrit_plan_destroy(plan)
    plan = pyrit.pyrit_plan_create(4, 5, 2, 6)
    try:
        assert pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_AUTO) == pyrit.PYRIT_TRANSFORM_PARITY
    finally:
        pyrit.pyrit_plan_destroy(plan)
    with pytest.raises(pyrit.PyritError):
        pyrit.pyrit_jit_source(11, np.ones((2, 2), np.uint16), None, 3)


def test_runtime_compiler_builds_parity_networks_without_a_device():
    plan = pyrit.pyrit_plan_create(10, 11, 10, 4)
    try:
        pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_PARITY)
        before = pyrit.pyrit_jit_stats()
        pyrit.pyrit_plan_specialise(plan)
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE, 0b1001)
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE_ANY)
        after = pyrit.pyrit_jit_stats()
        assert after["failed"] == before["failed"], pyrit.pyrit_jit_log()
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_network_resource_report():
    """The run-time compiler's resource report for a plan's networks: registers within the
    hardware limit of the launch shape (65536 registers per SM shared by four schedulers, so at
    most 16384 / (32 * ceil(warps / 4)) per thread), shape fields echo the spec."""
    plan = pyrit.pyrit_plan_create(10, 11, 10, 4)
    try:
        for op in (pyrit.PYRIT_OP_ENCODE, pyrit.PYRIT_OP_DECODE_ANY):
            info = pyrit.pyrit_plan_network_info(plan, op)
            warps = info["nc"] + 1
            assert 0 < info["registers"] <= 16384 // (32 * -(-warps // 4))
            assert info["spill_store_bytes"] >= 0 and info["stack_bytes"] >= 0
            assert info["mode"] == (0 if op == pyrit.PYRIT_OP_ENCODE else 1)
        info = pyrit.pyrit_plan_network_info(plan, pyrit.PYRIT_OP_ENCODE, tile={"words": 1, "nc": 16})
        assert (info["words"], info["nc"]) == (1, 16)
        with pytest.raises(pyrit.PyritError):
            pyrit.pyrit_plan_network_info(plan, pyrit.PYRIT_OP_DECODE, 0)  # nothing erased: no network
    finally:
        pyrit.pyrit_plan_destroy(plan)


# ---- fields from other factors of x^n + 1 (Props. 1-2) ----------------------------------------

GENERAL = [(3, 7, 4, 3), (4, 15, 8, 4), (2, 9, 2, 2), (2, 15, 1, 3)]


def _parse_general_store(src, w):
    """The reduction a general-field network writes out: for each field coefficient t, the ring
    accumulators XORed into it."""
    rows, cur = {}, None
    for line in src.splitlines():
        a = re.match(r"\s*r\[x\] = acc\[i\]\[(\d+)\]\[x\];", line)
        if a:
            cur = [int(a.group(1))]
            continue
        b = re.match(r"\s*r\[x\] = xor3\(r\[x\], acc\[i\]\[(\d+)\]\[x\], acc\[i\]\[(\d+)\]\[x\]\);", line)
        if b:
            cur += [int(b.group(1)), int(b.group(2))]
            continue
        c = re.match(r"\s*r\[x\] \^= acc\[i\]\[(\d+)\]\[x\];", line)
        if c:
            cur.append(int(c.group(1)))
            continue
        d = re.match(r".*dst \+ \(size_t\)(\d+) \* P\) = vmake<WORDS>\(r\);", line)
        if d:
            rows[int(d.group(1))] = cur
            cur = None
    assert sorted(rows) == list(range(w))
    return rows


@pytest.mark.parametrize("w,n,k,m", GENERAL)
def test_general_field_planner_equals_oracle(w, n, k, m):
    g = oracle.ring_factor(w, n)
    plan = pyrit.pyrit_plan_create(w, n, k, m)
    try:
        assert pyrit.pyrit_plan_modulus(plan) == (g, False)
        for u in range(1 << w):
            assert pyrit.pyrit_sparse_transform(w, n, u) == oracle.sparse_rep_mod(w, n, g, u)
        G = oracle.cauchy_mod(w, g, k, m)
        np.testing.assert_array_equal(pyrit.pyrit_plan_generator(plan), G)
        sp = np.array([oracle.sparse_rep_mod(w, n, g, u) for u in range(1 << w)], np.uint32)
        np.testing.assert_array_equal(pyrit.pyrit_plan_encode_masks(plan), sp[G[k:]].astype(np.uint16))
        # decoding masks of every pattern: phi_S of the oracle's decoding matrix in this field
        from itertools import combinations
        for e in range(1, m + 1):
            for pat in combinations(range(k + m), e):
                er = sum(1 << b for b in pat)
                surv = [b for b in range(k + m) if b not in pat][:k]
                Inv = oracle.gf_invert_mod(w, g, G[surv])
                surv2, erased, M = pyrit.pyrit_plan_decode_masks(plan, er)
                assert list(surv2) == surv and list(erased) == sorted(pat)
                for r, b in enumerate(sorted(pat)):
                    for s in range(k):
                        if b < k:
                            v = int(Inv[b][s])
                        else:
                            v = 0
                            for j in range(k):
                                v ^= oracle.gf_mul_mod(w, g, int(G[b][j]), int(Inv[j][s]))
                        assert M[r][s] == sp[v], (pat, r, s)
        # the parity transform is not defined for other factors
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_PARITY)
        assert ei.value.status == pyrit.PYRIT_E_UNSUPPORTED
        assert pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_AUTO) == pyrit.PYRIT_TRANSFORM_EMBEDDING
    finally:
        pyrit.pyrit_plan_destroy(plan)


@pytest.mark.parametrize("w,n,k,m", GENERAL)
def test_general_field_network_is_the_field_product(w, n, k, m):
    """The generated network of a general-field plan, read back: its XOR lists give the ring
    product by each coefficient's representative, and the reduction it writes out (the remainder
    mod g) maps that to the field product in F2[x]/(g)."""
    g = oracle.ring_factor(w, n)
    plan = pyrit.pyrit_plan_create(w, n, k, m)
    try:
        src = pyrit.pyrit_plan_network_source(plan)
        net = _parse(src)
        assert net["n"] == n and net["nin"] == k
        red = _parse_general_store(src, w)
        for t, rows in red.items():  # the reduction is the remainder mod g
            assert rows[0] == t
            for q in range(n):
                if q >= w:
                    assert (q in rows[1:]) == bool((oracle.poly_mod(1 << q, g) >> t) & 1), (t, q)
        G = oracle.cauchy_mod(w, g, k, m)
        for case, entries in net["cases"].items():
            gr, j = divmod(case, k)
            for ii in range(net["mg"]):
                o = gr * net["mg"] + ii
                if o >= m:
                    continue
                for q, col in enumerate(_ring_columns(entries, ii, n, w)):
                    field = 0
                    for t, rows in red.items():
                        if sum((col >> r) & 1 for r in rows) & 1:
                            field |= 1 << t
                    assert field == oracle.gf_mul_mod(w, g, int(G[k + o][j]), 1 << q), (case, ii, q)
        # the run-time compiler builds it for sm_103a without a device
        before = pyrit.pyrit_jit_stats()["failed"]
        pyrit.pyrit_plan_specialise(plan)
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE, 0b1)
        assert pyrit.pyrit_jit_stats()["failed"] == before, pyrit.pyrit_jit_log()
    finally:
        pyrit.pyrit_plan_destroy(plan)


def _xor_statements(src):
    body = src[src.index("switch ("):]
    return sum(1 for line in body.splitlines() if re.search(r"xor3\(| \^= | \^ ", line))


def _syndrome_xor_statements(src):
    """XOR statements of a syndrome network's two first-phase bodies: (the one for tiles that need
    every parity row, the per-row guarded one)."""
    body = src[src.index("switch ("):]
    counts, in_all = [0, 0], False
    for line in body.splitlines():
        if re.match(r"\s*if \(need == \d+u\) \{", line):
            in_all = True
        elif re.match(r"\s*\} else \{", line):
            in_all = False
        elif re.search(r"xor3\(| \^= | \^ ", line):
            counts[0 if in_all else 1] += 1
    return tuple(counts)


@pytest.mark.parametrize("w,k,m,enc_max,syn_max,all_max", [(10, 10, 4, 620, 735, 660), (12, 16, 4, 1500, 1680, 1560)])
def test_shared_terms_reduce_the_xor_count(w, k, m, enc_max, syn_max, all_max):
    """The generated networks form shared pairs and triples of source packets once: each XOR
    statement is one 32-bit three-input operation per column word, so their count per network is
    the coding work. Without sharing the plain Cauchy codes take sum(ceil(terms / 2)) statements:
    868 (encode) and 908 (syndrome first phase) for GF(2^10) k=10 m=4, 2200 and 2248 for GF(2^12)
    k=16 m=4; with it at most the bounds here (614 / 728 and 1492 / 1672 when written). The syndrome
    network's body for tiles that need every parity row shares terms across rows as the encode
    does, and stays within all_max."""
    n = oracle.ring_size(w)
    C, masks = _oracle_parity_masks(w, k, m)
    unshared = 0
    for j in range(k):
        for o in range(m):
            for t in range(n):
                terms = sum(1 for s in range(n) if (int(masks[o][j]) >> s) & 1 and (t - s) % n < w)
                unshared += (terms + 1) // 2
    plan = pyrit.pyrit_plan_create(w, n, k, m)
    try:
        enc = _xor_statements(pyrit.pyrit_plan_network_source(plan, pyrit.PYRIT_OP_ENCODE))
        syn_all, syn = _syndrome_xor_statements(pyrit.pyrit_plan_network_source(plan, pyrit.PYRIT_OP_DECODE_ANY))
    finally:
        pyrit.pyrit_plan_destroy(plan)
    assert enc <= enc_max and enc < 0.75 * unshared, (enc, unshared)
    assert syn <= syn_max, syn
    assert syn_all <= all_max and syn_all < syn, (syn_all, syn)


def test_committed_pairing_automata_match_their_generator():
    # ring_network.inc is generated by csrc/gen_ring_network.py and committed (the build compiles the
    # committed file); the two must not drift apart.
    import importlib.util
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1709_00178_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("gen_ring_network", os.path.join(here, "gen_ring_network.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(os.path.join(here, "ring_network.inc")) as f:
        assert f.read() == gen.source()


def test_wide_networks_take_two_sources_per_step():
    """Jobs of more than four outputs code two staged sources per step (one three-input XOR can take
    a term of each); jobs of up to four keep one. The (60,40) GF(2^6) code's first job (8 outputs)
    then needs 1972 XOR statements against 2712 one source at a time, and still computes the field
    products of its table."""
    w, k, m = 6, 40, 20
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        src = pyrit.pyrit_plan_network_source(plan, pyrit.PYRIT_OP_ENCODE)
    finally:
        pyrit.pyrit_plan_destroy(plan)
    assert "apply2" in src and _parse(src)["npairs"] == k // 2
    assert _xor_statements(src) <= 2000
    C, masks = _oracle_parity_masks(w, k, m)
    _check_network(src, masks[:8], oracle.ring_size(w))
    # an odd source count: the last source goes alone
    C7, masks7 = _oracle_parity_masks(10, 7, 6)
    src7 = pyrit.pyrit_jit_source(11, masks7)
    assert _parse(src7)["npairs"] == 3
    _check_network(src7, masks7, 11)
    # four outputs: one source per step
    C4, masks4 = _oracle_parity_masks(10, 10, 4)
    assert "apply2" not in pyrit.pyrit_jit_source(11, masks4)
