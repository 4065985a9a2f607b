"""GPU parity of fields from other factors of x^n + 1 (Sec. 2.1, Props. 1-2): GF(8) from x^3 + x + 1
in R_{2,7}, GF(16) from x^4 + x + 1 in R_{2,15}, GF(4) in R_{2,9}. Only generated networks code them:
each network carries its own reduction mod the factor. Every result is compared bit for bit with
the oracle's codec over that modulus (encode_mod / decode_mod).
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


class GF:
    """`count` stripes of a general-field code in one device buffer."""

    def __init__(self, pyrit, w, n, k, m, P, count, seed):
        self.w, self.n, self.k, self.m, self.P, self.count = w, n, k, m, P, count
        self.g = oracle.ring_factor(w, n)
        self.stride = ((k + m) * w * P + 255) // 256 * 256
        self.buf = torch.zeros(count * self.stride, dtype=torch.uint8, device="cuda")
        self.G = oracle.cauchy_mod(w, self.g, k, m)
        self.plan = pyrit.pyrit_plan_create(w, n, k, m)
        assert pyrit.pyrit_plan_modulus(self.plan) == (self.g, False)
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
            par = oracle.encode_mod(self.w, self.g, self.k, self.m, self.G, self.data[s], nthreads=NCPU)
            self._full[s] = np.concatenate([self.data[s], par])
        return self._full[s]

    def write_erased(self, s, pat, fill=0x96):
        arr = self.full(s).copy()
        for e in range(self.k + self.m):
            if (pat >> e) & 1:
                arr[e] = fill
        self.view(s).copy_(torch.from_numpy(arr.reshape(-1)).cuda())

    def stripes(self, op, pats=None):
        return [(self.plan, op, pats[s] if pats else 0, self.P, self.blocks(s)) for s in range(self.count)]


CODES = [(3, 7, 4, 3, 4096 + 16), (4, 15, 8, 4, 2048 + 48), (2, 9, 2, 2, 8192), (4, 15, 12, 3, 1024 + 16)]


@pytest.mark.parametrize("w,n,k,m,P", CODES)
def test_general_field_batch_encode_and_decode(pyrit, jit_mode, w, n, k, m, P):
    st = GF(pyrit, w, n, k, m, P, 3, 0xB100 + n * 10 + k)
    try:
        b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_ENCODE))
        try:
            assert pyrit.pyrit_batch_shape(b, 0)["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK
            pyrit.pyrit_batch_run(b, graph=True)
            for s in range(st.count):
                np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="stripe %d" % s)
        finally:
            pyrit.pyrit_batch_destroy(b)
        # decode: one pattern per batch (a direct network per pattern), the maximum erasure count
        rng = np.random.default_rng(n + k)
        for e in (1, m):
            pat = sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))
            for s in range(st.count):
                st.write_erased(s, pat)
            b = pyrit.pyrit_batch_create(st.stripes(pyrit.PYRIT_OP_DECODE, [pat] * st.count))
            try:
                assert pyrit.pyrit_batch_shape(b, 0)["dispatch"] == pyrit.PYRIT_DISPATCH_NETWORK
                pyrit.pyrit_batch_run(b)
                for s in range(st.count):
                    np.testing.assert_array_equal(st.host(s), st.full(s), err_msg="pattern %#x" % pat)
            finally:
                pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_general_field_every_pattern_single_calls(pyrit, jit_mode):
    """GF(8) in R_{2,7}, k=4 m=3: every pattern of 1-3 erasures by single decode calls (each pattern's
    network compiled in the call)."""
    pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_SYNC)
    st = GF(pyrit, 3, 7, 4, 3, 1024 + 16, 1, 0xB200)
    try:
        pyrit.pyrit_encode(st.plan, st.blocks(0)[:4], st.blocks(0)[4:], st.P)
        np.testing.assert_array_equal(st.host(0), st.full(0))
        n = 0
        for e in range(1, 4):
            for c in itertools.combinations(range(7), e):
                pat = sum(1 << x for x in c)
                st.write_erased(0, pat)
                pyrit.pyrit_decode(st.plan, st.blocks(0), pat, st.P)
                np.testing.assert_array_equal(st.host(0), st.full(0), err_msg="pattern %#x" % pat)
                n += 1
        assert n == 63
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(st.plan)


def test_general_and_native_fields_on_one_ring(pyrit, jit_mode):
    """GF(4) and the native GF(2^6) share R_{2,9}: one batch, two groups (one per field), each
    coded in its own field."""
    a = GF(pyrit, 2, 9, 2, 2, 4096, 2, 0xB300)
    w, k, m, P = 6, 8, 4, 4096
    plan6 = pyrit.pyrit_plan_create(w, 9, k, m)
    buf6 = torch.zeros(2 * (k + m) * w * P, dtype=torch.uint8, device="cuda")
    data6 = [synth_bytes(0xB310 + s, 0, k * w * P).reshape(k, w, P) for s in range(2)]
    try:
        for s in range(2):
            buf6[s * (k + m) * w * P:s * (k + m) * w * P + k * w * P].copy_(torch.from_numpy(data6[s].reshape(-1)).cuda())
        blocks6 = [[buf6.data_ptr() + s * (k + m) * w * P + e * w * P for e in range(k + m)] for s in range(2)]
        stripes = a.stripes(pyrit.PYRIT_OP_ENCODE) + [(plan6, 0, 0, P, blocks6[s]) for s in range(2)]
        b = pyrit.pyrit_batch_create(stripes)
        try:
            assert pyrit.pyrit_batch_stats(b)["launches"] == 2
            pyrit.pyrit_batch_run(b)
            for s in range(2):
                np.testing.assert_array_equal(a.host(s), a.full(s))
                got = buf6[s * (k + m) * w * P:(s + 1) * (k + m) * w * P].cpu().numpy().reshape(k + m, w, P)
                want = oracle.encode(w, k, m, oracle.cauchy(w, k, m), data6[s], nthreads=NCPU)
                np.testing.assert_array_equal(got[k:], want)
        finally:
            pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(a.plan)
        pyrit.pyrit_plan_destroy(plan6)


def test_general_field_refusals(pyrit, jit_mode):
    """Only generated networks code these fields: run-time compilation off, unaligned stripes
    (the plain-load kernel), the server and the allocation-free entry point refuse them."""
    st = GF(pyrit, 4, 15, 8, 4, 2048, 1, 0xB400)
    try:
        def refused(fn, *args):
            with pytest.raises(pyrit.PyritError) as ei:
                fn(*args)
            assert ei.value.status == pyrit.PYRIT_E_UNSUPPORTED, ei.value

        enc = st.stripes(pyrit.PYRIT_OP_ENCODE)
        pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_OFF)
        refused(pyrit.pyrit_batch_create, enc)
        refused(pyrit.pyrit_encode, st.plan, st.blocks(0)[:8], st.blocks(0)[8:], st.P)
        pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_SYNC)
        refused(pyrit.pyrit_batch_create, [(st.plan, 0, 0, st.P - 8, st.blocks(0))])
        refused(pyrit.pyrit_code_stripes_noalloc, enc)
        srv = pyrit.pyrit_server_create(1 << 30)
        try:
            refused(pyrit.pyrit_server_submit, srv, [(st.plan, 0, 0, st.P, st.blocks(0), 1, 0)])
        finally:
            pyrit.pyrit_server_destroy(srv)
        assert not st.host(0)[8:].any()
    finally:
        pyrit.pyrit_plan_destroy(st.plan)
