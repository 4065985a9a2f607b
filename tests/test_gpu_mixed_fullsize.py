"""GPU parity of the mixed batch at its full shape: 4096 uneven stripes (rings n = 5, 11, 13; k 4..32,
m 2..8; packets 512 B..256 KiB; half encodes, half decodes with 1..m random erasures; 31.6 GB of
stripes), created with the default compilation policy, tuned and replayed from a CUDA graph exactly
as the benchmark times it. A seeded sample of whole stripes, plus the extremes of the draw, is
compared byte for byte with the CPU oracle's encode and decode.

The stripes hold random bytes, so a decode rebuilds its lost blocks from the first k surviving
blocks (the survivors are the same on both sides, and they are never written): the oracle's decode
of the same survivors is the one correct result."""
import os

import numpy as np
import pytest

import oracle
from paper_1709_00178_gb300.synth import BASE_SEED, mixed_batch_specs, stripe_offsets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4


@pytest.fixture(scope="module")
def pyrit():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1709_00178_gb300 import pyrit as p
    return p


def _sample(specs, count, seed):
    """`count` seeded stripe indices plus the extremes: the largest and smallest packet, the widest
    code, and an encode and a decode of every ring."""
    rng = np.random.default_rng(seed)
    idx = set(int(i) for i in rng.choice(len(specs), count, replace=False))
    idx.add(max(range(len(specs)), key=lambda i: specs[i][3]))
    idx.add(min(range(len(specs)), key=lambda i: specs[i][3]))
    idx.add(max(range(len(specs)), key=lambda i: specs[i][1] + specs[i][2]))
    for w in (4, 10, 12):
        for op in (0, 1):
            idx.add(next(i for i, s in enumerate(specs) if s[0] == w and s[4] == op))
    return sorted(idx)


def _check(buf, specs, offs, picks, what):
    torch.cuda.synchronize()
    for i in picks:
        w, k, m, P, op, er = specs[i]
        n = (k + m) * w * P
        h = buf[offs[i]:offs[i] + n].cpu().numpy().reshape(k + m, w, P)
        G = oracle.cauchy(w, k, m)
        if op == 0:
            want = oracle.encode(w, k, m, G, h[:k], nthreads=NCPU)
            assert np.array_equal(h[k:], want), (what, i, specs[i])
        else:
            want = oracle.decode(w, k, m, G, h, er, nthreads=NCPU)
            assert np.array_equal(h, want), (what, i, specs[i])


def test_mixed_batch_full_shape_against_oracle(pyrit):
    specs = mixed_batch_specs(BASE_SEED + 3, 4096)
    offs, total = stripe_offsets(specs)
    buf = torch.empty(total, dtype=torch.uint8, device="cuda")
    pyrit.pyrit_synth_fill(buf.data_ptr(), total, BASE_SEED + 3, 0)
    plans = {}
    try:
        for (w, k, m, P, op, er) in specs:
            if (w, k, m) not in plans:
                plans[(w, k, m)] = pyrit.pyrit_plan_create(w, w + 1, k, m)
        base = buf.data_ptr()
        stripes = [(plans[(w, k, m)], op, er, P, [base + o + e * w * P for e in range(k + m)])
                   for (w, k, m, P, op, er), o in zip(specs, offs)]
        stream = torch.cuda.Stream()
        batch = pyrit.pyrit_batch_create(stripes)
        try:
            st = pyrit.pyrit_batch_stats(batch)
            assert st["src_bytes"] == sum(k * w * P for (w, k, m, P, op, er) in specs)
            picks = _sample(specs, 64, 4)
            # the default shapes, one direct run
            pyrit.pyrit_batch_run(batch, stream)
            _check(buf, specs, offs, picks, "default shapes")
            # the tuned shapes, replayed from a CUDA graph as the benchmark times them
            pyrit.pyrit_batch_tune(batch, stream, 1)
            for _ in range(2):
                pyrit.pyrit_batch_run(batch, stream, graph=True)
            _check(buf, specs, offs, picks, "tuned, graph replay")
            assert pyrit.pyrit_device_status() == (0, 0)
        finally:
            pyrit.pyrit_batch_destroy(batch)
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)
        del buf
        torch.cuda.empty_cache()
