"""GPU tests of the served path (continuous batching): every request's result is byte-identical
whether it is coded alone or in a mix of concurrent requests of different codes, packet sizes and
operations; admission never exceeds the HBM budget; invalid requests are refused before any
device work; waits are bounded on the host."""
import os
import time

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


CODES = [(12, 16, 4), (10, 10, 4), (4, 4, 2)]


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        w, k, m = CODES[int(rng.integers(0, len(CODES)))]
        P = int(2 ** rng.uniform(9, 15)) // 16 * 16
        op = int(rng.integers(0, 2))
        er = 0
        if op == 1:
            e = int(rng.integers(1, m + 1))
            er = sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))
        out.append((w, k, m, P, op, er))
    return out


def _layout(reqs):
    offs, total = [], 0
    for (w, k, m, P, op, er) in reqs:
        offs.append(total)
        total += ((k + m) * w * P + 255) // 256 * 256
    return offs, total


def test_alone_equals_mix(pyrit):
    reqs = _requests(3, 40)
    offs, total = _layout(reqs)
    plans = {c: pyrit.pyrit_plan_create(c[0], c[0] + 1, c[1], c[2]) for c in CODES}
    init = torch.empty(total, dtype=torch.uint8, device="cuda")
    pyrit.pyrit_synth_fill(init.data_ptr(), total, 77)
    torch.cuda.synchronize()

    def stripes(buf):
        base = buf.data_ptr()
        return [(plans[(w, k, m)], op, er, P, [base + o + e * w * P for e in range(k + m)])
                for (w, k, m, P, op, er), o in zip(reqs, offs)]

    try:
        alone = init.clone()
        for st in stripes(alone):  # each request coded by itself, one after the other
            b = pyrit.pyrit_batch_create([st])
            pyrit.pyrit_batch_run(b)
            torch.cuda.synchronize()
            pyrit.pyrit_batch_destroy(b)
        mix = init.clone()
        torch.cuda.synchronize()
        srv = pyrit.pyrit_server_create(64 << 30, max_batch=16, slots=4)
        try:
            sts = stripes(mix)
            for lo in range(0, len(sts), 7):  # arrivals in bursts while earlier batches run
                pyrit.pyrit_server_submit(srv, [s + (lo + i, 0) for i, s in enumerate(sts[lo:lo + 7])])
                time.sleep(0.0002)
            assert pyrit.pyrit_server_drain(srv, 20000) == 0
            done = pyrit.pyrit_server_poll(srv)
            st = pyrit.pyrit_server_stats(srv)
        finally:
            pyrit.pyrit_server_destroy(srv)
        assert sorted(d[0] for d in done) == list(range(len(reqs)))
        assert all(d[1] == 0 for d in done)
        assert all(d[2] <= d[4] and d[3] <= d[4] for d in done)
        assert st["batches"] >= 2, st  # the requests were spread over several overlapping batches
        assert torch.equal(alone, mix)
        # and the encoded parity of a few stripes is the oracle's
        h = mix.cpu().numpy()
        for i, (w, k, m, P, op, er) in enumerate(reqs):
            if op != 0 or i > 12:
                continue
            stripe = h[offs[i]:offs[i] + (k + m) * w * P].reshape(k + m, w, P)
            G = oracle.cauchy(w, k, m)
            assert np.array_equal(stripe[k:], oracle.encode(w, k, m, G, stripe[:k], nthreads=NCPU)), i
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)


def test_admission_respects_budget(pyrit):
    w, k, m, P = 12, 16, 4, 64 * 1024
    one = (k + m) * w * P
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    buf = torch.zeros(12 * one, dtype=torch.uint8, device="cuda")
    srv = pyrit.pyrit_server_create(3 * one, max_batch=8, slots=4)
    try:
        base = buf.data_ptr()
        reqs = [(plan, 0, 0, P, [base + s * one + e * w * P for e in range(k + m)], s, 0) for s in range(12)]
        pyrit.pyrit_server_submit(srv, reqs)
        assert pyrit.pyrit_server_drain(srv, 20000) == 0
        st = pyrit.pyrit_server_stats(srv)
        assert st["completed"] == 12 and st["max_inflight"] <= 3 * one and st["inflight"] == 0
        assert len(pyrit.pyrit_server_poll(srv)) == 12
    finally:
        pyrit.pyrit_server_destroy(srv)
        pyrit.pyrit_plan_destroy(plan)


def test_invalid_requests_refused_before_work(pyrit):
    w, k, m, P = 4, 4, 2, 4096
    one = (k + m) * w * P
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    buf = torch.zeros(2 * one, dtype=torch.uint8, device="cuda")
    srv = pyrit.pyrit_server_create(one, max_batch=4, slots=2)
    try:
        blocks = [buf.data_ptr() + e * w * P for e in range(k + m)]
        cases = [((plan, 1, 0b111, P, blocks, 1, 0), pyrit.PYRIT_E_TOO_MANY_ERASURES),
                 ((plan, 0, 0, 2 * P, [buf.data_ptr() + e * w * 2 * P for e in range(k + m)], 2, 0), pyrit.PYRIT_E_BUDGET),
                 ((plan, 0, 0, P - 8, blocks, 3, 0), pyrit.PYRIT_E_INVALID_ARG),
                 ((plan, 0, 0, P, blocks[:5] + [0], 4, 0), pyrit.PYRIT_E_INVALID_ARG)]
        for req, code in cases:
            with pytest.raises(pyrit.PyritError) as ei:
                pyrit.pyrit_server_submit(srv, [req])
            assert ei.value.status == code
        assert pyrit.pyrit_server_stats(srv)["submitted"] == 0
    finally:
        pyrit.pyrit_server_destroy(srv)
        pyrit.pyrit_plan_destroy(plan)


def test_drain_wait_is_bounded(pyrit):
    # A host-side bounded wait: draining with a zero limit while work is queued returns
    # PYRIT_E_TIMEOUT (the work continues and a later drain completes it).
    w, k, m, P = 12, 16, 4, 1 << 20
    one = (k + m) * w * P
    plan = pyrit.pyrit_plan_create(w, oracle.ring_size(w), k, m)
    buf = torch.zeros(one, dtype=torch.uint8, device="cuda")
    srv = pyrit.pyrit_server_create(2 * one, max_batch=4, slots=1)
    try:
        blocks = [buf.data_ptr() + e * w * P for e in range(k + m)]
        pyrit.pyrit_server_submit(srv, [(plan, 0, 0, P, blocks, 9, 0)])
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_server_drain(srv, 0)
        assert ei.value.status == pyrit.PYRIT_E_TIMEOUT
        assert pyrit.pyrit_server_drain(srv, 20000) == 0
        assert [d[0] for d in pyrit.pyrit_server_poll(srv)] == [9]
    finally:
        pyrit.pyrit_server_destroy(srv)
        pyrit.pyrit_plan_destroy(plan)


def test_plans_replaced_between_requests(pyrit):
    """The server remembers which compiled network codes a plan's requests. Plans destroyed and
    created again (possibly at the same address) with a different generator must be coded with
    their own tables: every encode equals the oracle's under that plan's generator, and every
    decode rebuilds the erased blocks."""
    w, k, m, P = 10, 10, 4, 4096
    n = oracle.ring_size(w)
    one = (k + m) * w * P
    buf = torch.empty(2 * one, dtype=torch.uint8, device="cuda")
    srv = pyrit.pyrit_server_create(64 << 20, max_batch=8, slots=2)
    try:
        for rnd in range(6):
            G = pyrit.pyrit_generator_weighted(w, n, k, m)[0] if rnd % 2 else oracle.cauchy(w, k, m)
            plan = pyrit.pyrit_plan_create(w, n, k, m, G)
            try:
                pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_ENCODE)
                pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE_ANY)
                pyrit.pyrit_synth_fill(buf.data_ptr(), buf.numel(), 500 + rnd)
                torch.cuda.synchronize()
                base = buf.data_ptr()
                enc = [base + e * w * P for e in range(k + m)]
                pyrit.pyrit_server_submit(srv, [(plan, 0, 0, P, enc, 2 * rnd, 0)])
                assert pyrit.pyrit_server_drain(srv, 20000) == 0
                h = buf[:one].cpu().numpy().reshape(k + m, w, P)
                assert np.array_equal(h[k:], oracle.encode(w, k, m, np.asarray(G).reshape(k + m, k), h[:k], nthreads=NCPU)), rnd
                # a copy of the stripe with three blocks lost, rebuilt by a syndrome-form decode
                buf[one:] = buf[:one]
                lost = (1 << 1) | (1 << 7) | (1 << (k + 2))
                for b in (1, 7, k + 2):
                    buf[one + b * w * P:one + (b + 1) * w * P] = 0
                dec = [base + one + e * w * P for e in range(k + m)]
                pyrit.pyrit_server_submit(srv, [(plan, 1, lost, P, dec, 2 * rnd + 1, 0)])
                assert pyrit.pyrit_server_drain(srv, 20000) == 0
                assert torch.equal(buf[one:], buf[:one]), rnd
                assert all(d[1] == 0 for d in pyrit.pyrit_server_poll(srv))
            finally:
                pyrit.pyrit_plan_destroy(plan)
    finally:
        pyrit.pyrit_server_destroy(srv)
