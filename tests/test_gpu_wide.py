"""GPU parity of wide stripes: more than 32 data blocks or more than 8 parity blocks, as in the
paper's GF(2^6) use cases (Sec. 5: a (60, 40) code with the embedding transform and a (60, 20)
code with the parity transform over GF(2^6) from x^6 + x^3 + 1, Sec. 2.4).

A stripe with more than 8 outputs is coded as one job per group of 8 that reads the same sources.
A batch holds those jobs in one launch: a generated network carries every group's table, and each
job names its own. Single calls run the jobs one after the other. Every result is compared bit for
bit with the oracle: its field codec (encode / decode) under the embedding, its ring-literal
parity-transform codec (encode_pt / decode_pt) under the parity transform.
"""
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
    prev = pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_ASYNC)
    pyrit.pyrit_tune_clear()
    yield
    pyrit.pyrit_jit_mode(prev)


class Wide:
    """`count` stripes of one code in one device buffer."""

    def __init__(self, pyrit, w, k, m, P, count, seed, parity=False):
        self.w, self.k, self.m, self.P, self.count, self.parity = w, k, m, P, count, parity
        self.stride = ((k + m) * w * P + 255) // 256 * 256
        self.buf = torch.zeros(count * self.stride, dtype=torch.uint8, device="cuda")
        self.G = oracle.cauchy(w, k, m)
        self.plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
        if parity:
            pyrit.pyrit_plan_set_transform(self.plan, pyrit.PYRIT_TRANSFORM_PARITY)
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
            enc = oracle.encode_pt if self.parity else oracle.encode
            self._full[s] = np.concatenate([self.data[s], enc(self.w, self.k, self.m, self.G, self.data[s], nthreads=NCPU)])
        return self._full[s]

    def write_erased(self, s, pat, fill=0xC3):
        arr = self.full(s).copy()
        for e in range(self.k + self.m):
            if (pat >> e) & 1:
                arr[e] = fill
        self.view(s).copy_(torch.from_numpy(arr.reshape(-1)).cuda())

    def stripes(self, op, pats=None):
        return [(self.plan, op, pats[s] if pats else 0, self.P, self.blocks(s)) for s in range(self.count)]


def _pattern(rng, k, m, e):
    return sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))


# The paper's GF(2^6) codes: (60, 40) under the embedding, (60, 20) under the parity transform;
# also one with k > 32 and m <= 8 and a narrow field for the output split alone.
CODES = [(6, 40, 20, False, 4096 + 16), (6, 20, 40, True, 1024 + 16), (6, 48, 8, False, 2048 + 32),
         (10, 12, 20, False, 2048 + 16)]


@pytest.mark.parametrize("w,k,m,parity,P", CODES)
def test_wide_batch_encode(pyrit, jit_mode, w, k, m, parity, P):
    st = Wide(pyrit, w, k, m, P, 3, 0xA100 + k + m, parity)
    try:
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_ENCODE))
        try:
            shape = pyrit.pyrit_batch_shape(b, 0)
            # one launch: a network holding every output group's table
            assert pyrit.pyrit_batch_stats(b)["launches"] == 1
            assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and shape["mode"] == (2 if parity else 0), shape
            pyrit.pyrit_batch_run(b, graph=True)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="stripe %d" % s)
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("w,k,m,parity,P", [c for c in CODES if not c[3]])
def test_wide_generic_kernel(pyrit, jit_mode, w, k, m, parity, P):
    """Run-time compilation off: the generic kernel codes the stripes' jobs (masks read at run time,
    sources beyond 32 from the second mask row of each lane)."""
    st = Wide(pyrit, w, k, m, P, 2, 0xA200 + k + m)
    pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_OFF)
    try:
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_ENCODE))
        try:
            assert pyrit.pyrit_batch_shape(b, 0)["dispatch"] != pyrit.PYRIT_DISPATCH_NETWORK
            pyrit.pyrit_batch_run(b)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), st.full(s))
        finally:
            pyrit.pyrit_batch_destroy(b)
        rng = np.random.default_rng(k)
        pats = [_pattern(rng, k, m, m), _pattern(rng, k, m, max(1, m // 3))]
        for s in range(st.count):
            st.write_erased(s, pats[s])
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_DECODE, pats))
        try:
            pyrit.pyrit_batch_run(b)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="pattern %#x" % pats[s])
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("w,k,m,parity,P", CODES)
def test_wide_batch_decode(pyrit, jit_mode, w, k, m, parity, P):
    """Decodes in one batch: every stripe with its own pattern, as many tables as fit one network
    (at most 8 output groups in all), the maximum erasure count among them."""
    rng = np.random.default_rng(0xA3 + k)
    count = 2
    st = Wide(pyrit, w, k, m, P, count, 0xA300 + k + m, parity)
    try:
        pats = [_pattern(rng, k, m, m), _pattern(rng, k, m, min(m, 8))]
        assert sum(-(-bin(p).count("1") // 8) for p in pats) <= 8
        for s in range(count):
            st.write_erased(s, pats[s])
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_DECODE, pats))
        try:
            shape = pyrit.pyrit_batch_shape(b, 0)
            if parity:
                assert shape["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK and shape["mode"] in (2, 3), shape
            pyrit.pyrit_batch_run(b, graph=True)
            for s in range(count):
                np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="stripe %d pattern %#x" % (s, pats[s]))
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("w,k,m,parity,P", CODES)
def test_wide_single_calls(pyrit, jit_mode, w, k, m, parity, P):
    rng = np.random.default_rng(0xA4 + k)
    st = Wide(pyrit, w, k, m, P, 1, 0xA400 + k + m, parity)
    try:
        pyrit.pyrit_encode(st.plan, st.blocks(0)[:k], st.blocks(0)[k:], P)
        np.testing.assert_array_equal(st.host(0), st.full(0))
        for e in (1, min(m, 9), m):
            pat = _pattern(rng, k, m, e)
            st.write_erased(0, pat, fill=0x5A)
            pyrit.pyrit_decode(st.plan, st.blocks(0), pat, P)
            np.testing.assert_array_equal(st.host(0), st.full(0), err_msg="pattern %#x" % pat)
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


@pytest.mark.parametrize("parity", [False, True])
def test_more_tables_than_a_network_holds(pyrit, jit_mode, parity):
    """Six stripes of a code with 20 parity blocks, each decoding its own 20-block pattern: 18
    decoding tables, more than one network holds (8). Under the embedding the generic kernel codes
    them; under the parity transform (networks only) the batch is refused before any device work."""
    w, k, m, P = 10, 12, 20, 1024 + 16
    rng = np.random.default_rng(0xA6 + parity)
    st = Wide(pyrit, w, k, m, P, 6, 0xA600, parity)
    try:
        pats = [_pattern(rng, k, m, m) for _ in range(st.count)]
        for s in range(st.count):
            st.write_erased(s, pats[s])
        if parity:
            with pytest.raises(pyrit.PyritError) as ei:
                pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_DECODE, pats))
            assert ei.value.status == pyrit.PYRIT_E_UNSUPPORTED
            return
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_DECODE, pats))
        try:
            assert pyrit.pyrit_batch_shape(b, 0)["dispatch"] != pyrit.PYRIT_DISPATCH_NETWORK
            pyrit.pyrit_batch_run(b)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="pattern %#x" % pats[s])
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_wide_refusals(pyrit, jit_mode):
    """The server and the allocation-free entry point code one job per stripe: a stripe with more
    than 8 parity blocks is refused there, before any device work."""
    st = Wide(pyrit, 6, 40, 20, 1024, 1, 0xA500)
    try:
        def refused(fn, *args):
            with pytest.raises(pyrit.PyritError) as ei:
                fn(*args)
            assert ei.value.status == pyrit.PYRIT_E_UNSUPPORTED, ei.value

        refused(pyrit.pyrit_code_stripes_noalloc, st.stripes(pyrit.PYRIT_OP_ENCODE))
        srv = pyrit.pyrit_server_create(1 << 30)
        try:
            refused(pyrit.pyrit_server_submit, srv, [(st.plan, pyrit.PYRIT_OP_ENCODE, 0, st.P, st.blocks(0), 1, 0)])
        finally:
            pyrit.pyrit_server_destroy(srv)
        assert not st.host(0)[40:].any()
    finally:
        pyrit.pyrit_plan_destroy(st.plan)
