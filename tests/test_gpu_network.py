"""GPU parity of the plan-specialised networks: the staged kernel with its multiply-accumulate step
generated for one mask table and compiled at run time. Every result is compared bit for bit with the
CPU oracle, over the four fields, every candidate network shape, batched, graph-replayed, tuned and
single-call paths (compiled synchronously and in the background), with ragged tails (P not a
multiple of the tile width) and several tiles per stripe."""
import os

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300.synth import synth_bytes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4


@pytest.fixture(scope="module")
def pyrit():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1709_00178_gb300 import pyrit as p
    return p


@pytest.fixture
def jit_mode(pyrit):
    # every test starts from the default policy and an empty tuning table (a shape tuned by an
    # earlier test for the same key would otherwise be taken instead of the automatic choice)
    prev = pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_ASYNC)
    pyrit.pyrit_tune_clear()
    yield
    pyrit.pyrit_jit_mode(prev)


class Stripes:
    """`count` stripes of one code in one device buffer, data filled from the synthetic stream."""

    def __init__(self, pyrit, w, k, m, P, count, seed, weighted=False):
        self.w, self.k, self.m, self.P, self.count = w, k, m, P, count
        self.stride = ((k + m) * w * P + 255) // 256 * 256
        self.buf = torch.zeros(count * self.stride, dtype=torch.uint8, device="cuda")
        # the oracle's own generator; the library plan is built from the same matrix
        self.G = oracle.cauchy_weighted(w, k, m)[0] if weighted else oracle.cauchy(w, k, m)
        self.plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m, self.G if weighted else None)
        self.data = [synth_bytes(seed + s, 0, k * w * P).reshape(k, w, P) for s in range(count)]
        for s in range(count):
            self.view(s)[:k * w * P].copy_(torch.from_numpy(self.data[s].reshape(-1)).cuda())

    def view(self, s):
        return self.buf[s * self.stride:s * self.stride + (self.k + self.m) * self.w * self.P]

    def blocks(self, s):
        base = self.buf.data_ptr() + s * self.stride
        return [base + e * self.w * self.P for e in range(self.k + self.m)]

    def host(self, s):
        torch.cuda.synchronize()
        return self.view(s).cpu().numpy().reshape(self.k + self.m, self.w, self.P)

    def full(self, s):
        return np.concatenate([self.data[s], oracle.encode(self.w, self.k, self.m, self.G, self.data[s], nthreads=NCPU)])

    def stripes(self, op, erasures=0):
        return [(self.plan, op, erasures, self.P, self.blocks(s)) for s in range(self.count)]


def _encode_batch_matches(pyrit, st, tile=None, graph=False, expect_network=True):
    b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_ENCODE), tile)
    try:
        shape = pyrit.pyrit_batch_shape(b, 0)
        if expect_network:
            assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK, shape
        pyrit.pyrit_batch_run(b, graph=graph)
        if graph:
            pyrit.pyrit_batch_run(b, graph=True)  # a replay of the captured launch
        for s in range(st.count):
            np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="stripe %d" % s)
    finally:
        pyrit.pyrit_batch_destroy(b)
    return shape


# P values: several tiles per stripe with a ragged last tile (tile widths are 1-6 KiB)
@pytest.mark.parametrize("w,k,m,P,count", [(10, 10, 4, 8192 + 16, 5), (12, 16, 4, 4096 + 48, 3), (4, 8, 8, 6000 + 16, 3),
                                           (2, 2, 2, 2048 + 32, 4), (10, 32, 8, 1024 + 16, 2), (12, 5, 1, 4096, 3),
                                           (6, 8, 4, 8192 + 16, 4), (6, 32, 8, 1024 + 16, 2)])
def test_network_batch_encode_all_fields(pyrit, jit_mode, w, k, m, P, count):
    st = Stripes(pyrit, w, k, m, P, count, 0x4E00 + w * 100 + k)
    try:
        _encode_batch_matches(pyrit, st)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("erasures", [0b1011, 0b11 << 10, (1 << 3) | (1 << 12), 1 << 13])
def test_network_batch_decode(pyrit, jit_mode, erasures):
    w, k, m, P = 10, 10, 4, 4096 + 16
    st = Stripes(pyrit, w, k, m, P, 3, 0xDEC0)
    try:
        full = [st.full(s) for s in range(st.count)]
        for s in range(st.count):  # write the whole codeword, then wipe the erased blocks
            arr = full[s].copy()
            for e in range(k + m):
                if (erasures >> e) & 1:
                    arr[e] = 0x5A
            st.view(s).copy_(torch.from_numpy(arr.reshape(-1)).cuda())
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_DECODE, erasures))
        try:
            assert pyrit.pyrit_batch_shape(b, 0)["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK
            pyrit.pyrit_batch_run(b)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), full[s])
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


NET_SHAPES = [dict(words=1, mg=4, minb=1, nc=24), dict(words=1, mg=4, minb=1, nc=16), dict(words=1, mg=2, minb=1, nc=16),
              dict(words=2, mg=4, minb=1, nc=8), dict(words=4, mg=4, minb=1, nc=8), dict(words=1, mg=1, minb=2, nc=8),
              dict(words=2, mg=2, minb=2, nc=8, stages=2)]


@pytest.mark.parametrize("shape", NET_SHAPES, ids=lambda d: "-".join("%s%d" % kv for kv in d.items()))
def test_every_network_shape(pyrit, jit_mode, shape):
    st = Stripes(pyrit, 10, 10, 4, 8192 + 16, 3, 0x5A9E)
    try:
        tile = dict(shape, dispatch=pyrit.PYRIT_DISPATCH_NETWORK)
        got = _encode_batch_matches(pyrit, st, tile)
        assert (got["words"], got["mg"], got["nc"]) == (shape["words"], shape["mg"], shape["nc"])
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_network_batch_graph_replay(pyrit, jit_mode):
    st = Stripes(pyrit, 12, 16, 4, 2048 + 16, 4, 0x6A7)
    try:
        _encode_batch_matches(pyrit, st, graph=True)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_jit_off_uses_the_generic_kernel(pyrit, jit_mode):
    pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_OFF)
    st = Stripes(pyrit, 10, 10, 4, 4096, 2, 0x0FF)
    try:
        shape = _encode_batch_matches(pyrit, st, expect_network=False)
        assert shape["dispatch"] != pyrit.PYRIT_DISPATCH_NETWORK
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_ENCODE), dict(dispatch=pyrit.PYRIT_DISPATCH_NETWORK))
        assert ei.value.status == pyrit.PYRIT_E_JIT
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_output_count_classes_split_a_generic_group(pyrit, jit_mode):
    """Codes of one ring with different source and output counts share no network as one group; the
    batch splits such a group by output count (1-2, 3-4, 5-8 per job), and each part, now of one
    mask table, runs its own launch (a generated network when compilation is on). Every stripe must
    equal the oracle's."""
    a = Stripes(pyrit, 10, 10, 4, 4096 + 16, 2, 0x333)
    c = Stripes(pyrit, 10, 12, 2, 4096, 2, 0x444)
    try:
        b = pyrit.pyrit_batch_create(a.stripes(pyrit.PYRIT_OP_ENCODE) + c.stripes(pyrit.PYRIT_OP_ENCODE))
        try:
            assert pyrit.pyrit_batch_stats(b)["launches"] == 2
            pyrit.pyrit_batch_run(b)
            for st in (a, c):
                for s in range(st.count):
                    np.testing.assert_array_equal(st.host(s), st.full(s))
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(a.plan)
        pyrit.pyrit_plan_destroy(c.plan)


def test_network_request_without_a_network_is_refused(pyrit, jit_mode):
    """Codes with different source counts (and the same output count, so one launch group) share no
    network: an explicit network request is refused before any device work; without it the group
    runs on a generic kernel."""
    a = Stripes(pyrit, 10, 10, 4, 4096, 1, 0x111)
    c = Stripes(pyrit, 10, 12, 4, 4096, 1, 0x222)
    try:
        before = [a.host(0).copy(), c.host(0).copy()]
        mixed = a.stripes(pyrit.PYRIT_OP_ENCODE) + c.stripes(pyrit.PYRIT_OP_ENCODE)
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_batch_create(mixed, dict(dispatch=pyrit.PYRIT_DISPATCH_NETWORK))
        assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
        np.testing.assert_array_equal(a.host(0), before[0])
        np.testing.assert_array_equal(c.host(0), before[1])
        b = pyrit.pyrit_batch_create(mixed)
        try:
            assert pyrit.pyrit_batch_shape(b, 0)["dispatch"] != pyrit.PYRIT_DISPATCH_NETWORK
            pyrit.pyrit_batch_run(b)
            np.testing.assert_array_equal(a.host(0), a.full(0))
            np.testing.assert_array_equal(c.host(0), c.full(0))
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(a.plan)
        pyrit.pyrit_plan_destroy(c.plan)


def test_codes_with_equal_source_counts_share_a_multi_table_network(pyrit, jit_mode):
    """Two codes with the same k and different parity rows: one network holds both tables and each
    job selects its own."""
    a = Stripes(pyrit, 10, 10, 4, 4096 + 16, 2, 0x333)
    c = Stripes(pyrit, 10, 10, 2, 4096 + 16, 2, 0x444)
    try:
        b = pyrit.pyrit_batch_create(a.stripes(pyrit.PYRIT_OP_ENCODE) + c.stripes(pyrit.PYRIT_OP_ENCODE))
        try:
            shape = pyrit.pyrit_batch_shape(b, 0)
            assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and pyrit.pyrit_batch_stats(b)["launches"] == 1
            pyrit.pyrit_batch_run(b, graph=True)
            for s in range(2):
                np.testing.assert_array_equal(a.host(s), a.full(s))
                np.testing.assert_array_equal(c.host(s), c.full(s))
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(a.plan)
        pyrit.pyrit_plan_destroy(c.plan)


def test_single_calls_sync_and_background(pyrit, jit_mode):
    st = Stripes(pyrit, 12, 16, 4, 4096 + 16, 1, 0x51C)
    try:
        data, parity = st.blocks(0)[:16], st.blocks(0)[16:]
        # background policy: the first call runs the generic kernel and queues the network
        pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_ASYNC)
        s0 = pyrit.pyrit_jit_stats()
        pyrit.pyrit_encode(st.plan, data, parity, st.P)
        np.testing.assert_array_equal(st.host(0), st.full(0))
        pyrit.pyrit_jit_wait(120000)
        s1 = pyrit.pyrit_jit_stats()
        assert s1["failed"] == s0["failed"], pyrit.pyrit_jit_log()
        st.view(0)[16 * 12 * st.P:].zero_()
        pyrit.pyrit_encode(st.plan, data, parity, st.P)  # now the compiled network
        s2 = pyrit.pyrit_jit_stats()
        assert s2["hits"] > s1["hits"]
        np.testing.assert_array_equal(st.host(0), st.full(0))
        # synchronous policy: the plan's syndrome-decode network (compiled in the call if no earlier
        # call compiled it) decodes a pattern never seen
        pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_SYNC)
        erasures = 0b101 | (1 << 17)
        for e in range(st.k + st.m):
            if (erasures >> e) & 1:
                st.view(0)[e * 12 * st.P:(e + 1) * 12 * st.P].fill_(0xA5)
        pyrit.pyrit_decode(st.plan, st.blocks(0), erasures, st.P)
        s3 = pyrit.pyrit_jit_stats()
        assert s3["hits"] > s2["hits"] and s3["failed"] == s2["failed"]
        np.testing.assert_array_equal(st.host(0), st.full(0))
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_tuner_times_networks_and_keeps_parity(pyrit, jit_mode, tmp_path):
    st = Stripes(pyrit, 10, 10, 4, 16384, 8, 0x70E)
    try:
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_ENCODE))
        try:
            pyrit.pyrit_batch_tune(b, iters=2)
            shape = pyrit.pyrit_batch_shape(b, 0)
            st.buf.zero_()
            for s in range(st.count):
                st.view(s)[:st.k * st.w * st.P].copy_(torch.from_numpy(st.data[s].reshape(-1)).cuda())
            pyrit.pyrit_batch_run(b, graph=True)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), st.full(s))
        finally:
            pyrit.pyrit_batch_destroy(b)
        # a later batch with the same key takes the tuned shape (a network shape compiled again for
        # this table if the tuner chose one)
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_ENCODE))
        try:
            again = pyrit.pyrit_batch_shape(b, 0)
            assert {k: again[k] for k in ("words", "mg", "minb", "dispatch", "nc")} == \
                {k: shape[k] for k in ("words", "mg", "minb", "dispatch", "nc")}
        finally:
            pyrit.pyrit_batch_destroy(b)
        path = str(tmp_path / "tune.json")
        assert pyrit.pyrit_tune_save(path) >= 0
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def _decode_batch_matches(pyrit, st, pats, tile=None, expect_mode=1, graph=False):
    """Writes every stripe's codeword with its pattern's blocks wiped, decodes them in one batch
    and compares every stripe with the oracle's codeword."""
    full = [st.full(s) for s in range(st.count)]
    for s in range(st.count):
        arr = full[s].copy()
        for e in range(st.k + st.m):
            if (pats[s] >> e) & 1:
                arr[e] = 0xC3
        st.view(s).copy_(torch.from_numpy(arr.reshape(-1)).cuda())
    b = pyrit.pyrit_batch_create([(st.plan, pyrit.PYRIT_OP_DECODE, pats[s], st.P, st.blocks(s)) for s in range(st.count)],
                                 tile)
    try:
        shape = pyrit.pyrit_batch_shape(b, 0)
        if expect_mode is not None:
            assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and shape["mode"] == expect_mode, shape
        pyrit.pyrit_batch_run(b, graph=graph)
        if graph:
            pyrit.pyrit_batch_run(b, graph=True)
        for s in range(st.count):
            np.testing.assert_array_equal(st.host(s), full[s], err_msg="stripe %d pattern %#x" % (s, pats[s]))
    finally:
        pyrit.pyrit_batch_destroy(b)
    return shape


def _random_patterns(rng, count, k, m):
    out = []
    for _ in range(count):
        e = int(rng.integers(1, m + 1))
        out.append(sum(1 << int(x) for x in rng.choice(k + m, e, replace=False)))
    return out


@pytest.mark.parametrize("w,k,m,P,count", [(10, 10, 4, 8192 + 16, 24), (12, 16, 4, 4096 + 32, 12), (4, 4, 2, 2048, 16),
                                           (10, 24, 8, 1024 + 16, 10), (2, 2, 2, 512, 8), (6, 12, 4, 4096 + 16, 12),
                                           (6, 24, 8, 1024 + 16, 8)])
def test_syndrome_network_mixed_patterns(pyrit, jit_mode, w, k, m, P, count):
    """Every stripe has its own random erasure pattern: the batch runs the plan's syndrome network."""
    rng = np.random.default_rng(0x5E + w + k)
    st = Stripes(pyrit, w, k, m, P, count, 0x5E00 + w * 100 + k)
    try:
        _decode_batch_matches(pyrit, st, _random_patterns(rng, count, k, m), graph=(k == 16))
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_syndrome_network_every_pattern(pyrit, jit_mode):
    """All erasure patterns of at most m blocks of a small code, one stripe each, in one launch."""
    from itertools import combinations
    w, k, m, P = 4, 4, 2, 1024 + 16
    pats = [sum(1 << b for b in c) for e in range(1, m + 1) for c in combinations(range(k + m), e)]
    st = Stripes(pyrit, w, k, m, P, len(pats), 0xA11)
    try:
        _decode_batch_matches(pyrit, st, pats)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("shape", [dict(words=1, nc=16), dict(words=1, nc=24), dict(words=2, nc=8), dict(words=2, nc=12),
                                   dict(words=4, nc=8), dict(words=1, nc=8, minb=2)],
                         ids=lambda d: "-".join("%s%d" % kv for kv in d.items()))
def test_every_syndrome_shape(pyrit, jit_mode, shape):
    rng = np.random.default_rng(0x5A)
    st = Stripes(pyrit, 10, 10, 4, 8192 + 16, 12, 0x5A5)
    try:
        got = _decode_batch_matches(pyrit, st, _random_patterns(rng, 12, 10, 4),
                                    dict(shape, dispatch=pyrit.PYRIT_DISPATCH_NETWORK))
        assert (got["words"], got["nc"], got["mg"], got["groups"]) == (shape["words"], shape["nc"], 4, 1)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_wide_code_decodes_on_the_syndrome_network(pyrit, jit_mode):
    # k + m = 36 block columns (beyond 32): the syndrome network's first phase reads up to 64
    rng = np.random.default_rng(0x36)
    st = Stripes(pyrit, 12, 30, 6, 2048, 4, 0x360)
    try:
        _decode_batch_matches(pyrit, st, _random_patterns(rng, 4, 30, 6), expect_mode=1)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_single_decode_uses_the_syndrome_network(pyrit, jit_mode):
    pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_SYNC)
    rng = np.random.default_rng(0x51D)
    st = Stripes(pyrit, 10, 10, 4, 4096 + 16, 1, 0x51D0)
    try:
        full = st.full(0)
        for pat in _random_patterns(rng, 6, 10, 4):
            arr = full.copy()
            for e in range(14):
                if (pat >> e) & 1:
                    arr[e] = 0x3C
            st.view(0).copy_(torch.from_numpy(arr.reshape(-1)).cuda())
            before = pyrit.pyrit_jit_stats()["hits"]
            pyrit.pyrit_decode(st.plan, st.blocks(0), pat, st.P)
            assert pyrit.pyrit_jit_stats()["hits"] > before
            np.testing.assert_array_equal(st.host(0), full, err_msg="pattern %#x" % pat)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("w,k,m,P,count", [(10, 10, 4, 8192 + 16, 6), (12, 16, 4, 4096 + 32, 4), (4, 12, 4, 2048, 4)])
def test_weighted_generator_encode_and_decode(pyrit, jit_mode, w, k, m, P, count):
    """The weight-optimised generalized Cauchy generator through the direct and syndrome networks."""
    st = Stripes(pyrit, w, k, m, P, count, 0x3E1 + w * 100 + k, weighted=True)
    try:
        _encode_batch_matches(pyrit, st)
        rng = np.random.default_rng(0x3E2 + k)
        _decode_batch_matches(pyrit, st, _random_patterns(rng, count, k, m))
    finally:
        pyrit.pyrit_plan_destroy(st.plan)
