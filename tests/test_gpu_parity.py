"""GPU parity: the CUDA coding path, called through the C ABI, against the CPU oracle, bit for bit
(tolerance 0: this is GF(2) arithmetic). Sizes span many column tiles with ragged tails; odd packet
sizes and unaligned pointers exercise the plain-load kernel; canary bands around every output catch
stray writes (compute-sanitizer is not used)."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300.synth import BASE_SEED, synth_bytes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 4
GUARD = 256  # canary bytes on each side of every block
CANARY = 0xC3


@pytest.fixture(scope="module")
def pyrit():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1709_00178_gb300 import pyrit as p
    return p


class Stripe:
    """k+m blocks of w*P bytes on the device, each inside its own canary-guarded slot."""

    def __init__(self, k, m, w, P, misalign=0):
        self.k, self.m, self.w, self.P = k, m, w, P
        self.bs = w * P
        slot = GUARD + self.bs + GUARD + 16
        slot = (slot + 255) // 256 * 256
        self.slot = slot
        self.off = GUARD + misalign
        self.buf = torch.full(((k + m) * slot,), CANARY, dtype=torch.uint8, device="cuda")

    def ptr(self, e):
        return self.buf.data_ptr() + e * self.slot + self.off

    def ptrs(self):
        return [self.ptr(e) for e in range(self.k + self.m)]

    def view(self, e):
        s = e * self.slot + self.off
        return self.buf[s:s + self.bs]

    def set_block(self, e, arr):
        self.view(e).copy_(torch.from_numpy(np.ascontiguousarray(arr).reshape(-1)).cuda())

    def get(self):
        torch.cuda.synchronize()
        h = self.buf.cpu().numpy()
        out = np.stack([h[e * self.slot + self.off:e * self.slot + self.off + self.bs] for e in range(self.k + self.m)])
        return out.reshape(self.k + self.m, self.w, self.P)

    def canaries_intact(self):
        torch.cuda.synchronize()
        h = self.buf.cpu().numpy()
        for e in range(self.k + self.m):
            a = e * self.slot + self.off
            if (h[e * self.slot:a] != CANARY).any() or (h[a + self.bs:(e + 1) * self.slot] != CANARY).any():
                return False
        return True


def _encode_case(pyrit, w, k, m, P, seed, misalign=0):
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        G = oracle.cauchy(w, k, m)
        data = synth_bytes(seed, 0, k * w * P).reshape(k, w, P)
        st = Stripe(k, m, w, P, misalign)
        for j in range(k):
            st.set_block(j, data[j])
        pyrit.pyrit_encode(plan, st.ptrs()[:k], st.ptrs()[k:], P)
        got = st.get()
        expect = oracle.encode(w, k, m, G, data, nthreads=NCPU)
        assert np.array_equal(got[:k], data), "sources modified"
        assert np.array_equal(got[k:], expect), "parity differs from the oracle"
        assert st.canaries_intact(), "write outside an output block"
        assert pyrit.pyrit_device_status() == (0, 0)
        return G, np.concatenate([data, expect])
    finally:
        pyrit.pyrit_plan_destroy(plan)


# The three single-stripe workloads (GF(16) k=4 m=2 P=256 KiB; GF(2^10) k=10 m=4 P=64 KiB;
# GF(2^12) k=16 m=4 P=32 KiB) plus GF(4), at their packet sizes (every tile full).
@pytest.mark.parametrize("w,k,m,P", [(4, 4, 2, 256 * 1024), (10, 10, 4, 64 * 1024), (12, 16, 4, 32 * 1024),
                                     (2, 2, 2, 8192), (6, 8, 4, 64 * 1024)])
def test_encode_workload_shapes(pyrit, w, k, m, P):
    _encode_case(pyrit, w, k, m, P, BASE_SEED + w)


# Ragged tails of the staged kernel (multiples of 16 that leave a partial last tile) and odd packet
# sizes of the plain-load kernel.
@pytest.mark.parametrize("P", [16, 48, 1040, 2064, 4096 + 1024 + 16, 65536 + 16])
@pytest.mark.parametrize("w,k,m", [(4, 4, 2), (10, 10, 4), (12, 16, 4), (6, 8, 4)])
def test_encode_ragged_tiles(pyrit, w, k, m, P):
    _encode_case(pyrit, w, k, m, P, 1000 + P + w)


@pytest.mark.parametrize("P", [1, 3, 15, 17, 1000, 4097])
@pytest.mark.parametrize("w,k,m", [(4, 4, 2), (10, 10, 4), (12, 16, 4), (6, 8, 4)])
def test_encode_odd_packet_sizes(pyrit, w, k, m, P):
    _encode_case(pyrit, w, k, m, P, 2000 + P + w)


@pytest.mark.parametrize("misalign", [1, 4, 8])
def test_encode_unaligned_pointers(pyrit, misalign):
    _encode_case(pyrit, 10, 10, 4, 4096, 77, misalign=misalign)


@pytest.mark.parametrize("w,k,m", [(4, 4, 1), (4, 1, 2), (12, 32, 8), (10, 20, 6), (4, 8, 8), (6, 32, 8), (6, 1, 2)])
def test_encode_extreme_shapes(pyrit, w, k, m):
    _encode_case(pyrit, w, k, m, 2048 + 32, 3000 + k * 10 + m)


def test_encode_zero_and_ones(pyrit):
    w, k, m, P = 10, 10, 4, 4096
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        G = oracle.cauchy(w, k, m)
        for fill in (0x00, 0xFF):
            data = np.full((k, w, P), fill, np.uint8)
            st = Stripe(k, m, w, P)
            for j in range(k):
                st.set_block(j, data[j])
            pyrit.pyrit_encode(plan, st.ptrs()[:k], st.ptrs()[k:], P)
            assert np.array_equal(st.get()[k:], oracle.encode(w, k, m, G, data))
    finally:
        pyrit.pyrit_plan_destroy(plan)


def _decode_check(pyrit, plan, full, pattern, w, k, m, P, misalign=0):
    st = Stripe(k, m, w, P, misalign)
    for e in range(k + m):
        st.set_block(e, full[e] ^ (0x5A if (pattern >> e) & 1 else 0))
    pyrit.pyrit_decode(plan, st.ptrs(), pattern, P)
    got = st.get()
    assert np.array_equal(got, full), "decode of pattern %s differs" % hex(pattern)
    assert st.canaries_intact()


def test_decode_all_patterns_gf16_full_size(pyrit):
    # GF(16), k=4, m=2, P = 256 KiB: every pattern of <= 2 erasures (22 patterns).
    w, k, m, P = 4, 4, 2, 256 * 1024
    _, full = _encode_case(pyrit, w, k, m, P, BASE_SEED)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        n = 0
        for e in range(1, m + 1):
            for c in itertools.combinations(range(k + m), e):
                _decode_check(pyrit, plan, full, sum(1 << x for x in c), w, k, m, P)
                n += 1
        assert n == 21  # C(6,1) + C(6,2); the empty pattern is a no-op
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_decode_all_patterns_gf1024_small(pyrit):
    # k=10, m=4: all 1470 patterns of 1..4 erasures on a two-tile stripe with a ragged tail.
    w, k, m, P = 10, 10, 4, 2048 + 48
    _, full = _encode_case(pyrit, w, k, m, P, 99)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        for e in range(1, m + 1):
            for c in itertools.combinations(range(k + m), e):
                _decode_check(pyrit, plan, full, sum(1 << x for x in c), w, k, m, P)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_decode_all_patterns_gf64_small(pyrit):
    # GF(2^6) from x^6 + x^3 + 1 on R_{2,9} (Sec. 2.4), k=8, m=4: all 793 patterns of 1..4 erasures
    # on a two-tile stripe with a ragged tail.
    w, k, m, P = 6, 8, 4, 2048 + 48
    _, full = _encode_case(pyrit, w, k, m, P, 98)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        n = 0
        for e in range(1, m + 1):
            for c in itertools.combinations(range(k + m), e):
                _decode_check(pyrit, plan, full, sum(1 << x for x in c), w, k, m, P)
                n += 1
        assert n == 793
    finally:
        pyrit.pyrit_plan_destroy(plan)


@pytest.mark.parametrize("w,k,m,P,npat", [(10, 10, 4, 64 * 1024, 12), (12, 16, 4, 32 * 1024, 12),
                                          (12, 32, 8, 4096, 8), (4, 12, 4, 1000, 6), (6, 20, 8, 4096, 10),
                                          (6, 8, 4, 64 * 1024, 8)])
def test_decode_random_patterns(pyrit, w, k, m, P, npat):
    _, full = _encode_case(pyrit, w, k, m, P, 500 + w + k)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    rng = np.random.default_rng(P + k)
    try:
        for _ in range(npat):
            e = int(rng.integers(1, m + 1))
            pat = sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))
            _decode_check(pyrit, plan, full, pat, w, k, m, P)
        # the maximum erasure count, all on data blocks
        _decode_check(pyrit, plan, full, (1 << m) - 1, w, k, m, P)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_decode_unaligned(pyrit):
    w, k, m, P = 10, 10, 4, 1000
    _, full = _encode_case(pyrit, w, k, m, P, 7)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        _decode_check(pyrit, plan, full, 0b1011, w, k, m, P, misalign=3)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_synth_fill_matches_host_generator(pyrit):
    for off, n in [(0, 1 << 20), (3, 12345), (8, 8), (5, 1)]:
        t = torch.zeros(n + 8, dtype=torch.uint8, device="cuda")
        pyrit.pyrit_synth_fill(t.data_ptr() + 1, n, 0xABCDEF, off)
        torch.cuda.synchronize()
        h = t.cpu().numpy()
        assert np.array_equal(h[1:1 + n], synth_bytes(0xABCDEF, off, n))
        assert h[0] == 0 and not h[1 + n:].any()
