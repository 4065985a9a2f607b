"""GPU parity of the batched path: many stripes of mixed codes, operations and packet sizes in one
persistent launch per ring size (optionally replayed from a CUDA graph), each stripe compared bit
for bit with the CPU oracle; every compiled kernel variant must give identical bytes."""
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


class Pool:
    """Device stripes carved from one buffer, with host copies of their expected contents."""

    def __init__(self, specs, seed):
        # specs: list of (w, k, m, P)
        self.specs = specs
        self.offs = []
        total = 0
        for (w, k, m, P) in specs:
            self.offs.append(total)
            total += ((k + m) * w * P + 255) // 256 * 256
        self.buf = torch.zeros(total, dtype=torch.uint8, device="cuda")
        self.seed = seed

    def blocks(self, i):
        w, k, m, P = self.specs[i]
        base = self.buf.data_ptr() + self.offs[i]
        return [base + e * w * P for e in range(k + m)]

    def host(self, i):
        w, k, m, P = self.specs[i]
        torch.cuda.synchronize()
        n = (k + m) * w * P
        return self.buf[self.offs[i]:self.offs[i] + n].cpu().numpy().reshape(k + m, w, P)

    def put(self, i, arr):
        w, k, m, P = self.specs[i]
        n = (k + m) * w * P
        self.buf[self.offs[i]:self.offs[i] + n].copy_(torch.from_numpy(np.ascontiguousarray(arr).reshape(-1)).cuda())


MIXED = [(4, 4, 2, 4096), (10, 10, 4, 8192), (12, 16, 4, 2048 + 16), (10, 20, 6, 1024), (12, 32, 8, 512),
         (4, 12, 4, 1000), (2, 2, 2, 64), (12, 8, 3, 3000 + 16), (10, 4, 8, 4096 + 32), (4, 8, 8, 17),
         (6, 12, 4, 2048 + 16), (6, 20, 8, 1000)]


def _plans(pyrit, specs):
    plans = {}
    for (w, k, m, P) in specs:
        if (w, k, m) not in plans:
            plans[(w, k, m)] = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    return plans


def test_mixed_batch_encode_then_decode(pyrit):
    pool = Pool(MIXED, 7)
    plans = _plans(pyrit, MIXED)
    try:
        full = []
        for i, (w, k, m, P) in enumerate(MIXED):
            data = synth_bytes(100 + i, 0, k * w * P).reshape(k, w, P)
            arr = np.zeros((k + m, w, P), np.uint8)
            arr[:k] = data
            pool.put(i, arr)
            G = oracle.cauchy(w, k, m)
            full.append(np.concatenate([data, oracle.encode(w, k, m, G, data, nthreads=NCPU)]))
        enc = [(plans[(w, k, m)], pyrit.PYRIT_OP_ENCODE, 0, P, pool.blocks(i)) for i, (w, k, m, P) in enumerate(MIXED)]
        b = pyrit.pyrit_batch_create(enc)
        st = pyrit.pyrit_batch_stats(b)
        assert st["alg_bytes"] == sum((k + m) * w * P for (w, k, m, P) in MIXED)
        pyrit.pyrit_batch_run(b)
        for i in range(len(MIXED)):
            assert np.array_equal(pool.host(i), full[i]), MIXED[i]
        pyrit.pyrit_batch_destroy(b)
        # decode: random patterns per stripe, erased blocks scrambled first
        rng = np.random.default_rng(5)
        dec = []
        for i, (w, k, m, P) in enumerate(MIXED):
            e = int(rng.integers(1, m + 1))
            pat = sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))
            arr = full[i].copy()
            for x in range(k + m):
                if (pat >> x) & 1:
                    arr[x] ^= 0x3C
            pool.put(i, arr)
            dec.append((plans[(w, k, m)], pyrit.PYRIT_OP_DECODE, pat, P, pool.blocks(i)))
        b = pyrit.pyrit_batch_create(dec)
        pyrit.pyrit_batch_run(b, graph=True)
        for i in range(len(MIXED)):
            assert np.array_equal(pool.host(i), full[i]), MIXED[i]
        pyrit.pyrit_batch_destroy(b)
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)


def test_one_shot_batches_match_the_oracle(pyrit):
    # pyrit_encode_batch / pyrit_decode_batch: the same stripes as one call each, waited for
    pool = Pool(MIXED, 8)
    plans = _plans(pyrit, MIXED)
    try:
        full = []
        for i, (w, k, m, P) in enumerate(MIXED):
            data = synth_bytes(200 + i, 0, k * w * P).reshape(k, w, P)
            arr = np.zeros((k + m, w, P), np.uint8)
            arr[:k] = data
            pool.put(i, arr)
            full.append(np.concatenate([data, oracle.encode(w, k, m, oracle.cauchy(w, k, m), data, nthreads=NCPU)]))
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        pyrit.pyrit_encode_batch([(plans[(w, k, m)], pyrit.PYRIT_OP_ENCODE, 0, P, pool.blocks(i))
                                  for i, (w, k, m, P) in enumerate(MIXED)], s)
        for i in range(len(MIXED)):
            assert np.array_equal(pool.host(i), full[i]), MIXED[i]
        rng = np.random.default_rng(6)
        dec = []
        for i, (w, k, m, P) in enumerate(MIXED):
            e = int(rng.integers(1, m + 1))
            pat = sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))
            arr = full[i].copy()
            for x in range(k + m):
                if (pat >> x) & 1:
                    arr[x] ^= 0x5A
            pool.put(i, arr)
            dec.append((plans[(w, k, m)], pyrit.PYRIT_OP_DECODE, pat, P, pool.blocks(i)))
        torch.cuda.synchronize()
        pyrit.pyrit_decode_batch(dec, s)
        for i in range(len(MIXED)):
            assert np.array_equal(pool.host(i), full[i]), MIXED[i]
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)


def _all_tiles(pyrit, n):
    """Hints that select exactly each compiled variant of ring size n, plus stage overrides."""
    out = [None, dict(stages=2), dict(stages=7, ctas_per_sm=1)]
    for v in pyrit.pyrit_variants():
        if v["n"] == n:
            out.append({k: v[k] for k in ("words", "mg", "minb", "dispatch", "nc")})
    return out


@pytest.mark.parametrize("w,k,m,P,S", [(10, 10, 4, 4096 + 48, 6), (12, 16, 4, 2048, 5), (4, 4, 2, 8192, 4),
                                       (2, 2, 2, 4096 + 16, 3), (12, 32, 8, 2048, 3), (6, 8, 4, 4096 + 48, 4),
                                       (6, 24, 8, 2048, 3)])
def test_every_variant_is_bit_exact(pyrit, w, k, m, P, S):
    specs = [(w, k, m, P)] * S
    pool = Pool(specs, 3)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        G = oracle.cauchy(w, k, m)
        full = []
        for i in range(S):
            data = synth_bytes(300 + i, 0, k * w * P).reshape(k, w, P)
            full.append(np.concatenate([data, oracle.encode(w, k, m, G, data, nthreads=NCPU)]))
        rng = np.random.default_rng(w)
        pats = [sum(1 << int(x) for x in rng.choice(k + m, m, replace=False)) for _ in range(S)]
        for t in _all_tiles(pyrit, oracle.ring_size(w)):
            for i in range(S):
                arr = full[i].copy()
                arr[k:] = 0
                pool.put(i, arr)
            b = pyrit.pyrit_batch_create([(plan, 0, 0, P, pool.blocks(i)) for i in range(S)], t)
            pyrit.pyrit_batch_run(b)
            pyrit.pyrit_batch_destroy(b)
            for i in range(S):
                assert np.array_equal(pool.host(i), full[i]), ("encode", t)
                arr = full[i].copy()
                for x in range(k + m):
                    if (pats[i] >> x) & 1:
                        arr[x] = 0xEE
                pool.put(i, arr)
            b = pyrit.pyrit_batch_create([(plan, 1, pats[i], P, pool.blocks(i)) for i in range(S)], t)
            pyrit.pyrit_batch_run(b)
            pyrit.pyrit_batch_destroy(b)
            for i in range(S):
                assert np.array_equal(pool.host(i), full[i]), ("decode", t)
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_batch_rejects_bad_stripes(pyrit):
    plan = pyrit.pyrit_plan_create(4, 5, 4, 2)
    # real device blocks, so that a request that slipped through validation could not fault
    mem = torch.zeros(6 * 4 * 64, dtype=torch.uint8, device="cuda")
    try:
        blocks = [mem.data_ptr() + e * 4 * 64 for e in range(6)]
        for bad, code in [((plan, 1, 0b111, 64, blocks), pyrit.PYRIT_E_TOO_MANY_ERASURES),
                          ((plan, 2, 0, 64, blocks), pyrit.PYRIT_E_INVALID_ARG),
                          ((plan, 0, 0, 0, blocks), pyrit.PYRIT_E_INVALID_ARG),
                          ((plan, 0, 0, 64, blocks[:5] + [0]), pyrit.PYRIT_E_INVALID_ARG)]:
            with pytest.raises(pyrit.PyritError) as ei:
                pyrit.pyrit_batch_create([bad])
            assert ei.value.status == code
        # an empty batch and a batch of no-op decodes are valid and launch nothing
        b = pyrit.pyrit_batch_create([])
        assert pyrit.pyrit_batch_stats(b)["launches"] == 0
        pyrit.pyrit_batch_run(b)
        pyrit.pyrit_batch_destroy(b)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_autotune_keeps_results_and_records_choice(pyrit, tmp_path):
    # Tuning runs every variant on the batch's own buffers; the coding is idempotent, so the
    # buffers must still hold the oracle's result afterwards, and the table must hold the key.
    w, k, m, P, S = 10, 10, 4, 8192, 8
    specs = [(w, k, m, P)] * S
    pool = Pool(specs, 11)
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    try:
        G = oracle.cauchy(w, k, m)
        full = []
        for i in range(S):
            data = synth_bytes(700 + i, 0, k * w * P).reshape(k, w, P)
            full.append(np.concatenate([data, oracle.encode(w, k, m, G, data, nthreads=NCPU)]))
            arr = full[i].copy()
            arr[k:] = 0
            pool.put(i, arr)
        b = pyrit.pyrit_batch_create([(plan, 0, 0, P, pool.blocks(i)) for i in range(S)])
        pyrit.pyrit_batch_tune(b, iters=2)
        for i in range(S):
            assert np.array_equal(pool.host(i), full[i])
        pyrit.pyrit_batch_run(b, graph=True)
        for i in range(S):
            assert np.array_equal(pool.host(i), full[i])
        pyrit.pyrit_batch_destroy(b)
        path = str(tmp_path / "tune.json")
        pyrit.pyrit_tune_save(path)
        text = open(path).read()
        assert '"n": 11, "shared": 1, "nout": 4, "plog2": 13' in text
        assert pyrit.pyrit_tune_load(path) >= 1
        # a later batch with the same key is built with the tuned shape and stays bit-exact
        b = pyrit.pyrit_batch_create([(plan, 0, 0, P, pool.blocks(i)) for i in range(S)])
        pyrit.pyrit_batch_run(b)
        pyrit.pyrit_batch_destroy(b)
        for i in range(S):
            assert np.array_equal(pool.host(i), full[i])
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_autotune_mixed_packet_sizes_and_decode(pyrit):
    # Explicit tile lists (packet sizes differ) are rebuilt for every candidate tile width; after
    # tuning an encode and a decode batch, every stripe still equals the oracle.
    specs = [(12, 16, 4, 2048), (12, 16, 4, 4096 + 32), (12, 16, 4, 1024), (12, 16, 4, 8192)]
    pool = Pool(specs, 5)
    plan = pyrit.pyrit_plan_create(12, 13, 16, 4)
    try:
        G = oracle.cauchy(12, 16, 4)
        full = []
        for i, (w, k, m, P) in enumerate(specs):
            data = synth_bytes(800 + i, 0, k * w * P).reshape(k, w, P)
            full.append(np.concatenate([data, oracle.encode(w, k, m, G, data, nthreads=NCPU)]))
            arr = full[i].copy()
            arr[k:] = 0
            pool.put(i, arr)
        b = pyrit.pyrit_batch_create([(plan, 0, 0, P, pool.blocks(i)) for i, (w, k, m, P) in enumerate(specs)])
        pyrit.pyrit_batch_tune(b, iters=1)
        pyrit.pyrit_batch_destroy(b)
        for i in range(len(specs)):
            assert np.array_equal(pool.host(i), full[i]), ("encode", i)
        pats = [0b1011, 0xF0000, 0b11 << 15, 1]
        for i, (w, k, m, P) in enumerate(specs):
            arr = full[i].copy()
            for x in range(k + m):
                if (pats[i] >> x) & 1:
                    arr[x] = 0x77
            pool.put(i, arr)
        b = pyrit.pyrit_batch_create([(plan, 1, pats[i], P, pool.blocks(i)) for i, (w, k, m, P) in enumerate(specs)])
        pyrit.pyrit_batch_tune(b, iters=1)
        pyrit.pyrit_batch_run(b, graph=True)
        pyrit.pyrit_batch_destroy(b)
        for i in range(len(specs)):
            assert np.array_equal(pool.host(i), full[i]), ("decode", i)
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(plan)
