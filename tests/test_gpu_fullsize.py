"""GPU parity at the configurations' full sizes, in the launch configuration bench.py times.

Config 2: GF(2^10) k=10 m=4, 64 KiB packets, 256 stripes (2.19 GiB), tuned batches replayed from
CUDA graphs, encode then decode with a random 1-4 erasure pattern per stripe. Config 3: GF(2^12)
k=16 m=4, 32 KiB packets, 1365 stripes (8 GiB of source), 4-erasure decode. The oracle checks a
seeded sample of whole stripes (every byte of each), so the full-size launches are verified on
outputs it can compute one by one.
"""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4


@pytest.fixture(scope="module")
def pyrit():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1709_00178_gb300 import pyrit as p
    return p


def _full_size(pyrit, w, k, m, P, S, seed, pats_fn, sample, tune):
    blk = w * P
    data_bytes = S * k * blk
    buf = torch.empty(S * (k + m) * blk, dtype=torch.uint8, device="cuda")
    pyrit.pyrit_synth_fill(buf.data_ptr(), data_bytes, seed, 0)
    buf[data_bytes:].fill_(0x3C)
    base = buf.data_ptr()
    par0 = data_bytes
    # the bench's layout: data blocks of all stripes first, then all parity blocks
    blocks = [[base + (s * k + j) * blk for j in range(k)] + [base + par0 + (s * m + i) * blk for i in range(m)]
              for s in range(S)]
    rng = np.random.default_rng(seed)
    pats = pats_fn(rng, S)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    G = oracle.cauchy(w, k, m)
    stream = torch.cuda.Stream()
    try:
        enc = pyrit.pyrit_batch_create([(plan, pyrit.PYRIT_OP_ENCODE, 0, P, blocks[s]) for s in range(S)])
        dec = pyrit.pyrit_batch_create([(plan, pyrit.PYRIT_OP_DECODE, pats[s], P, blocks[s]) for s in range(S)])
        if tune:
            pyrit.pyrit_batch_tune(enc, stream, 2)
            pyrit.pyrit_batch_tune(dec, stream, 2)
        pyrit.pyrit_batch_run(enc, stream, graph=True)
        torch.cuda.synchronize()
        picks = sorted(set(int(x) for x in rng.choice(S, sample, replace=False)) | {0, S - 1})
        expect = {}
        for s in picks:
            data = buf[s * k * blk:(s + 1) * k * blk].cpu().numpy().reshape(k, w, P)
            full = np.concatenate([data, oracle.encode(w, k, m, G, data, nthreads=NCPU)])
            got_par = buf[par0 + s * m * blk:par0 + (s + 1) * m * blk].cpu().numpy().reshape(m, w, P)
            np.testing.assert_array_equal(got_par, full[k:], err_msg="encode, stripe %d" % s)
            expect[s] = full
        # wipe every stripe's erased blocks, decode them all in one launch, check the sample
        for s in range(S):
            for e in range(k + m):
                if (pats[s] >> e) & 1:
                    off = (s * k + e) * blk if e < k else par0 + (s * m + e - k) * blk
                    buf[off:off + blk].fill_(0xA5)
        pyrit.pyrit_batch_run(dec, stream, graph=True)
        torch.cuda.synchronize()
        for s in picks:
            data = buf[s * k * blk:(s + 1) * k * blk].cpu().numpy().reshape(k, w, P)
            par = buf[par0 + s * m * blk:par0 + (s + 1) * m * blk].cpu().numpy().reshape(m, w, P)
            np.testing.assert_array_equal(np.concatenate([data, par]), expect[s],
                                          err_msg="decode, stripe %d pattern %#x" % (s, pats[s]))
        assert pyrit.pyrit_device_status() == (0, 0)
        pyrit.pyrit_batch_destroy(enc)
        pyrit.pyrit_batch_destroy(dec)
    finally:
        pyrit.pyrit_plan_destroy(plan)
        del buf
        torch.cuda.empty_cache()


def _random_1_to_m(k, m):
    def f(rng, S):
        return [sum(1 << int(x) for x in rng.choice(k + m, int(rng.integers(1, m + 1)), replace=False))
                for _ in range(S)]
    return f


def _exactly_m(k, m):
    def f(rng, S):
        return [sum(1 << int(x) for x in rng.choice(k + m, m, replace=False)) for _ in range(S)]
    return f


def test_config2_full_size_tuned(pyrit):
    _full_size(pyrit, 10, 10, 4, 65536, 256, 0xC2, _random_1_to_m(10, 4), sample=10, tune=True)


def test_config3_full_size(pyrit):
    _full_size(pyrit, 12, 16, 4, 32768, 1365, 0xC3, _exactly_m(16, 4), sample=6, tune=False)
