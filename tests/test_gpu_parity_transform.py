"""GPU parity of the parity transform (Sec. 2.3.1): phi_P pads each data symbol with its parity bit
instead of the embedding's zero coefficient, the ring product is taken as usual and phi_P^{-1}
drops the top coefficient. Encoder and decoder both use it, so the stored parity is the oracle's
encode_pt, not its field-code encode; every result is compared bit for bit with the oracle's
ring-literal parity-transform code. The transform runs only on generated networks: the direct
network of one mask table (encode, or one erasure pattern) and the plan's syndrome network (mixed
patterns in one batch), compiled in the call. Paths that have no network are refused.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300.synth import synth_bytes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4
MODE_DIRECT_PARITY, MODE_SYNDROME_PARITY = 2, 3


@pytest.fixture(scope="module")
def pyrit():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1709_00178_gb300 import pyrit as p
    return p


@pytest.fixture
def jit_mode(pyrit):
    prev = pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_ASYNC)
    pyrit.pyrit_tune_clear()
    yield
    pyrit.pyrit_jit_mode(prev)


class PtStripes:
    """`count` stripes of one parity-transform code in one device buffer."""

    def __init__(self, pyrit, w, k, m, P, count, seed, weighted=False):
        self.w, self.k, self.m, self.P, self.count = w, k, m, P, count
        self.stride = ((k + m) * w * P + 255) // 256 * 256
        self.buf = torch.zeros(count * self.stride, dtype=torch.uint8, device="cuda")
        self.G = oracle.cauchy_weighted(w, k, m)[0] if weighted else oracle.cauchy(w, k, m)
        self.plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m, self.G if weighted else None)
        assert pyrit.pyrit_plan_set_transform(self.plan, pyrit.PYRIT_TRANSFORM_PARITY) == pyrit.PYRIT_TRANSFORM_PARITY
        self.data = [synth_bytes(seed + s, 0, k * w * P).reshape(k, w, P) for s in range(count)]
        self._full = [None] * count
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
        if self._full[s] is None:
            par = oracle.encode_pt(self.w, self.k, self.m, self.G, self.data[s])
            self._full[s] = np.concatenate([self.data[s], par])
        return self._full[s]

    def write_erased(self, s, pat, fill=0xC3):
        arr = self.full(s).copy()
        for e in range(self.k + self.m):
            if (pat >> e) & 1:
                arr[e] = fill
        self.view(s).copy_(torch.from_numpy(arr.reshape(-1)).cuda())


def _random_patterns(rng, count, k, m):
    return [sum(1 << int(x) for x in rng.choice(k + m, int(rng.integers(1, m + 1)), replace=False))
            for _ in range(count)]


@pytest.mark.parametrize("w,k,m,P,count", [(10, 10, 4, 8192 + 16, 4), (12, 16, 4, 4096 + 48, 3), (4, 8, 8, 6000 + 16, 3),
                                           (2, 2, 2, 2048 + 32, 4), (10, 32, 8, 1024 + 16, 2), (4, 2, 6, 3072, 3),
                                           (6, 8, 4, 4096 + 16, 3), (6, 2, 6, 2048, 3)])
def test_parity_transform_batch_encode(pyrit, jit_mode, w, k, m, P, count):
    st = PtStripes(pyrit, w, k, m, P, count, 0x9700 + w * 100 + k)
    try:
        # the parity transform stores a different code: the field code's parity must not come out
        assert not np.array_equal(oracle.encode_pt(w, k, m, st.G, st.data[0]), oracle.encode(w, k, m, st.G, st.data[0]))
        b = pyrit.pyrit_batch_create([(st.plan, pyrit.PYRIT_OP_ENCODE, 0, P, st.blocks(s)) for s in range(count)])
        try:
            shape = pyrit.pyrit_batch_shape(b, 0)
            assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and shape["mode"] == MODE_DIRECT_PARITY, shape
            pyrit.pyrit_batch_run(b, graph=True)
            pyrit.pyrit_batch_run(b, graph=True)
            for s in range(count):
                np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="stripe %d" % s)
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def _decode_batch(pyrit, st, pats, expect_mode, graph=False, tune=False):
    for s in range(st.count):
        st.write_erased(s, pats[s])
    b = pyrit.pyrit_batch_create([(st.plan, pyrit.PYRIT_OP_DECODE, pats[s], st.P, st.blocks(s)) for s in range(st.count)])
    try:
        shape = pyrit.pyrit_batch_shape(b, 0)
        assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and shape["mode"] == expect_mode, shape
        if tune:
            pyrit.pyrit_batch_tune(b, iters=2)
            shape = pyrit.pyrit_batch_shape(b, 0)
            assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and shape["mode"] == expect_mode, shape
            for s in range(st.count):  # the tuner's launches rebuilt the blocks: wipe them again
                st.write_erased(s, pats[s])
        pyrit.pyrit_batch_run(b, graph=graph)
        for s in range(st.count):
            np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="stripe %d pattern %#x" % (s, pats[s]))
    finally:
        pyrit.pyrit_batch_destroy(b)
    return shape


@pytest.mark.parametrize("w,k,m,P,count", [(10, 10, 4, 8192 + 16, 16), (12, 16, 4, 4096 + 32, 10), (4, 4, 2, 2048, 12),
                                           (10, 24, 8, 1024 + 16, 8), (2, 2, 2, 512, 8), (4, 2, 6, 1024 + 16, 8),
                                           (6, 12, 4, 2048 + 16, 10), (6, 4, 8, 1024, 8)])
def test_parity_transform_mixed_pattern_decode(pyrit, jit_mode, w, k, m, P, count):
    """Every stripe has its own pattern: the plan's syndrome network under the parity transform."""
    rng = np.random.default_rng(0x97DE + w + k)
    st = PtStripes(pyrit, w, k, m, P, count, 0x97D0 + w * 100 + k)
    try:
        _decode_batch(pyrit, st, _random_patterns(rng, count, k, m), MODE_SYNDROME_PARITY, graph=(k == 16))
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_parity_transform_every_pattern(pyrit, jit_mode):
    w, k, m, P = 4, 4, 2, 1024 + 16
    pats = [sum(1 << b for b in c) for e in range(1, m + 1) for c in itertools.combinations(range(k + m), e)]
    st = PtStripes(pyrit, w, k, m, P, len(pats), 0x97E0)
    try:
        _decode_batch(pyrit, st, pats, MODE_SYNDROME_PARITY)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("erasures", [0b1011, 0b11 << 10, (1 << 3) | (1 << 12), 1 << 13])
def test_parity_transform_one_pattern_direct_network(pyrit, jit_mode, erasures):
    """Stripes that share one pattern share one decoding table: its direct network."""
    st = PtStripes(pyrit, 10, 10, 4, 4096 + 16, 3, 0x97F0)
    try:
        _decode_batch(pyrit, st, [erasures] * st.count, MODE_DIRECT_PARITY)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_parity_transform_weighted_and_tuned(pyrit, jit_mode):
    rng = np.random.default_rng(0x97A)
    st = PtStripes(pyrit, 10, 10, 4, 16384, 8, 0x97A0, weighted=True)
    try:
        b = pyrit.pyrit_batch_create([(st.plan, pyrit.PYRIT_OP_ENCODE, 0, st.P, st.blocks(s)) for s in range(st.count)])
        try:
            pyrit.pyrit_batch_tune(b, iters=2)
            shape = pyrit.pyrit_batch_shape(b, 0)
            assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and shape["mode"] == MODE_DIRECT_PARITY
            st.buf.zero_()
            for s in range(st.count):
                st.view(s)[:st.k * st.w * st.P].copy_(torch.from_numpy(st.data[s].reshape(-1)).cuda())
            pyrit.pyrit_batch_run(b, graph=True)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), st.full(s))
        finally:
            pyrit.pyrit_batch_destroy(b)
        _decode_batch(pyrit, st, _random_patterns(rng, st.count, 10, 4), MODE_SYNDROME_PARITY, tune=True)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_parity_transform_beside_embedding_stripes(pyrit, jit_mode):
    """One batch holding stripes of the same code under both transforms: two groups, each coded
    under its own transform."""
    emb = PtStripes(pyrit, 10, 10, 4, 4096, 3, 0x97B0)
    pt = PtStripes(pyrit, 10, 10, 4, 4096, 3, 0x97C0)
    try:
        pyrit.pyrit_plan_set_transform(emb.plan, pyrit.PYRIT_TRANSFORM_EMBEDDING)
        stripes = [(emb.plan, pyrit.PYRIT_OP_ENCODE, 0, 4096, emb.blocks(s)) for s in range(3)] + \
                  [(pt.plan, pyrit.PYRIT_OP_ENCODE, 0, 4096, pt.blocks(s)) for s in range(3)]
        b = pyrit.pyrit_batch_create(stripes)
        try:
            modes = sorted(pyrit.pyrit_batch_shape(b, g)["mode"] for g in range(2))
            assert modes == [0, MODE_DIRECT_PARITY]
            pyrit.pyrit_batch_run(b)
            for s in range(3):
                want = np.concatenate([emb.data[s], oracle.encode(10, 10, 4, emb.G, emb.data[s], nthreads=NCPU)])
                np.testing.assert_array_equal(emb.host(s), want)
                np.testing.assert_array_equal(pt.host(s), pt.full(s))
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(emb.plan)
        pyrit.pyrit_plan_destroy(pt.plan)


@pytest.mark.parametrize("policy", ["sync", "async"])
def test_parity_transform_single_calls(pyrit, jit_mode, policy):
    """Single-stripe calls compile the network in the call whatever the policy (under the parity
    transform nothing else codes the stripe)."""
    pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_SYNC if policy == "sync" else pyrit.PYRIT_JIT_ASYNC)
    rng = np.random.default_rng(0x9751 + len(policy))
    st = PtStripes(pyrit, 12, 16, 4, 4096 + 16, 1, 0x9750 + len(policy))
    try:
        pyrit.pyrit_encode(st.plan, st.blocks(0)[:16], st.blocks(0)[16:], st.P)
        np.testing.assert_array_equal(st.host(0), st.full(0))
        for pat in _random_patterns(rng, 5, 16, 4):
            st.write_erased(0, pat, fill=0x5A)
            pyrit.pyrit_decode(st.plan, st.blocks(0), pat, st.P)
            np.testing.assert_array_equal(st.host(0), st.full(0), err_msg="pattern %#x" % pat)
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_parity_transform_refusals(pyrit, jit_mode):
    """Paths without a generated network refuse the parity transform instead of coding the field
    code: the generic kernels (run-time compiler off, an explicit generic shape), unaligned stripes
    (the plain-load kernel), the server and the allocation-free entry point. (Mixed patterns of codes
    with more parity blocks than the syndrome network holds run on multi-table direct networks while
    their tables fit one; more tables are refused, see test_gpu_wide.py.)"""
    st = PtStripes(pyrit, 10, 10, 4, 4096, 2, 0x97F8)
    wide = PtStripes(pyrit, 10, 20, 12, 1024, 2, 0x97F9)
    try:
        enc = [(st.plan, pyrit.PYRIT_OP_ENCODE, 0, st.P, st.blocks(s)) for s in range(2)]

        def refused(fn, *args):
            with pytest.raises(pyrit.PyritError) as ei:
                fn(*args)
            assert ei.value.status == pyrit.PYRIT_E_UNSUPPORTED, ei.value

        pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_OFF)
        refused(pyrit.pyrit_batch_create, enc)
        refused(pyrit.pyrit_encode, st.plan, st.blocks(0)[:10], st.blocks(0)[10:], st.P)
        pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_SYNC)
        refused(pyrit.pyrit_batch_create, enc, {"words": 1, "mg": 4, "minb": 1, "nc": 16, "dispatch": 0})
        odd = [(st.plan, pyrit.PYRIT_OP_ENCODE, 0, st.P - 8, st.blocks(0))]
        refused(pyrit.pyrit_batch_create, odd)
        refused(pyrit.pyrit_encode, st.plan, st.blocks(0)[:10], st.blocks(0)[10:], st.P - 8)
        pats = [0b11 | (1 << 21), 0b101 | (1 << 23)]
        refused(pyrit.pyrit_code_stripes_noalloc, enc)
        srv = pyrit.pyrit_server_create(1 << 30)
        try:
            refused(pyrit.pyrit_server_submit, srv, [(st.plan, pyrit.PYRIT_OP_ENCODE, 0, st.P, st.blocks(0), 1, 0)])
        finally:
            pyrit.pyrit_server_destroy(srv)
        # nothing was written by any refused call
        for s in range(2):
            assert not st.host(s)[10:].any()
        # two patterns of a code with 12 parity blocks: one network with both decoding tables
        for s_ in range(2):
            wide.write_erased(s_, pats[s_])
        b = pyrit.pyrit_batch_create([(wide.plan, pyrit.PYRIT_OP_DECODE, pats[s_], wide.P, wide.blocks(s_)) for s_ in range(2)])
        try:
            assert pyrit.pyrit_batch_shape(b, 0)["mode"] == MODE_DIRECT_PARITY
            pyrit.pyrit_batch_run(b)
            for s_ in range(2):
                np.testing.assert_array_equal(wide.host(s_), wide.full(s_))
        finally:
            pyrit.pyrit_batch_destroy(b)
        # and one pattern per batch (its direct network)
        wide.write_erased(0, pats[0])
        wide.write_erased(1, pats[0])
        b = pyrit.pyrit_batch_create([(wide.plan, pyrit.PYRIT_OP_DECODE, pats[0], wide.P, wide.blocks(s)) for s in range(2)])
        try:
            assert pyrit.pyrit_batch_shape(b, 0)["mode"] == MODE_DIRECT_PARITY
            pyrit.pyrit_batch_run(b)
            for s in range(2):
                np.testing.assert_array_equal(wide.host(s), wide.full(s))
        finally:
            pyrit.pyrit_batch_destroy(b)
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)
        pyrit.pyrit_plan_destroy(wide.plan)
