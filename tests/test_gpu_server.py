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


def _codewords(reqs, offs, total, seed):
    """Host image of the request stripes: every stripe a codeword of its code (random data, parity
    from the oracle). Returns (image with the outputs of each request overwritten by junk, the
    expected image)."""
    want = np.zeros(total, np.uint8)
    for i, (w, k, m, P, op, er) in enumerate(reqs):
        data = synth_bytes(seed, offs[i], k * w * P).reshape(k, w, P)
        par = oracle.encode(w, k, m, oracle.cauchy(w, k, m), data, nthreads=NCPU)
        want[offs[i]:offs[i] + (k + m) * w * P] = np.concatenate([data, par]).reshape(-1)
    start = want.copy()
    for i, (w, k, m, P, op, er) in enumerate(reqs):
        blk = w * P
        lost = range(k, k + m) if op == 0 else [e for e in range(k + m) if (er >> e) & 1]
        for e in lost:
            start[offs[i] + e * blk:offs[i] + (e + 1) * blk] = 0xE7
    return start, want


def test_alone_equals_mix(pyrit):
    """Every request of a mix of codes, packet sizes and operations is coded once alone (submitted
    to a server, drained, then the next) and once in a mix (bursts submitted while earlier batches
    run); the two must write the same bytes, and each must equal the oracle's codeword: encodes
    write the oracle's parity, decodes rebuild the oracle's lost blocks."""
    reqs = _requests(3, 40)
    offs, total = _layout(reqs)
    plans = {c: pyrit.pyrit_plan_create(c[0], c[0] + 1, c[1], c[2]) for c in CODES}
    start, want = _codewords(reqs, offs, total, 77)
    init = torch.from_numpy(start).cuda()
    torch.cuda.synchronize()

    def stripes(buf):
        base = buf.data_ptr()
        return [(plans[(w, k, m)], op, er, P, [base + o + e * w * P for e in range(k + m)])
                for (w, k, m, P, op, er), o in zip(reqs, offs)]

    try:
        alone = init.clone()
        torch.cuda.synchronize()
        srv = pyrit.pyrit_server_create(64 << 30, max_batch=16, slots=4)
        try:
            for i, s in enumerate(stripes(alone)):  # one request in the server at a time
                pyrit.pyrit_server_submit(srv, [s + (i, 0)])
                assert pyrit.pyrit_server_drain(srv, 20000) == 0
            done_alone = pyrit.pyrit_server_poll(srv)
            st_alone = pyrit.pyrit_server_stats(srv)
        finally:
            pyrit.pyrit_server_destroy(srv)
        assert sorted(d[0] for d in done_alone) == list(range(len(reqs)))
        assert all(d[1] == 0 for d in done_alone)
        assert st_alone["batches"] == len(reqs)  # each alone in its batch
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
        assert st["batches"] < len(reqs), st  # and some batches held more than one request
        assert torch.equal(alone, mix)
        h = mix.cpu().numpy()
        for i, (w, k, m, P, op, er) in enumerate(reqs):
            n = (k + m) * w * P
            assert np.array_equal(h[offs[i]:offs[i] + n], want[offs[i]:offs[i] + n]), (i, reqs[i])
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)


def test_served_config5_shape_against_oracle(pyrit):
    """Requests of the served workload's shape (GF(2^12) k=16 m=4, P one of 4 KiB..1 MiB, half
    encodes and half 4-erasure decodes) arriving as a seeded Poisson stream at 20k requests/s, each
    on its own codeword: every encode must write the oracle's parity and every decode rebuild the
    oracle's lost blocks, with the plan's generated networks (encode table, syndrome decode)
    compiled before serving, as the benchmark serves them."""
    w, k, m = 12, 16, 4
    rng = np.random.default_rng(0x5E4E)
    count = 48
    reqs = []
    for _ in range(count):
        P = 1 << int(rng.integers(12, 21))
        op = int(rng.integers(0, 2))
        er = sum(1 << int(x) for x in rng.choice(k + m, m, replace=False)) if op else 0
        reqs.append((w, k, m, P, op, er))
    gaps = rng.exponential(1e9 / 20000, count)
    offs, total = _layout(reqs)
    start, want = _codewords(reqs, offs, total, 91)
    buf = torch.from_numpy(start).cuda()
    plan = pyrit.pyrit_plan_create(w, w + 1, k, m)
    try:
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_ENCODE)
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE_ANY)
        torch.cuda.synchronize()
        base = buf.data_ptr()
        srv = pyrit.pyrit_server_create(16 << 30, max_batch=64, slots=16)
        try:
            t0 = pyrit.pyrit_server_now_ns(srv) + 2_000_000
            arr = (t0 + np.cumsum(gaps)).astype(np.int64)
            items = [(plan, op, er, P, [base + o + e * w * P for e in range(k + m)], i, int(arr[i]))
                     for i, ((w_, k_, m_, P, op, er), o) in enumerate(zip(reqs, offs))]
            i = 0
            while i < count:  # submit each request at its arrival time
                if pyrit.pyrit_server_now_ns(srv) >= arr[i]:
                    pyrit.pyrit_server_submit(srv, [items[i]])
                    i += 1
            assert pyrit.pyrit_server_drain(srv, 60000) == 0
            done = pyrit.pyrit_server_poll(srv)
        finally:
            pyrit.pyrit_server_destroy(srv)
        assert sorted(d[0] for d in done) == list(range(count))
        assert all(d[1] == 0 for d in done)
        h = buf.cpu().numpy()
        for i, (w_, k_, m_, P, op, er) in enumerate(reqs):
            n = (k + m) * w * P
            assert np.array_equal(h[offs[i]:offs[i] + n], want[offs[i]:offs[i] + n]), (i, reqs[i])
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(plan)


def test_replay_submits_each_request_at_its_arrival(pyrit):
    """The native load generator (pyrit_server_replay) hands each request to the server when the
    server clock reaches its arrival time: no request starts before it arrives, every result equals
    the oracle's codeword, and a trace out of arrival order is refused before any submission."""
    w, k, m = 12, 16, 4
    rng = np.random.default_rng(0x5E4F)
    count = 48
    reqs = []
    for _ in range(count):
        P = 1 << int(rng.integers(12, 19))
        op = int(rng.integers(0, 2))
        er = sum(1 << int(x) for x in rng.choice(k + m, m, replace=False)) if op else 0
        reqs.append((w, k, m, P, op, er))
    gaps = rng.exponential(1e9 / 20000, count)
    offs, total = _layout(reqs)
    start, want = _codewords(reqs, offs, total, 92)
    buf = torch.from_numpy(start).cuda()
    plan = pyrit.pyrit_plan_create(w, w + 1, k, m)
    try:
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_ENCODE)
        pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE_ANY)
        torch.cuda.synchronize()
        base = buf.data_ptr()
        srv = pyrit.pyrit_server_create(16 << 30, max_batch=64, slots=16)
        try:
            items = [(plan, op, er, P, [base + o + e * w * P for e in range(k + m)], i, 0)
                     for i, ((w_, k_, m_, P, op, er), o) in enumerate(zip(reqs, offs))]
            arr, keep = pyrit.pyrit_requests_array(items)
            # out of order: refused, nothing submitted
            arr[0].arrival_ns, arr[1].arrival_ns = 10_000_000_000, 5_000_000_000
            with pytest.raises(pyrit.PyritError) as ei:
                pyrit.pyrit_server_replay(srv, arr, 0, 2)
            assert ei.value.status == pyrit.PYRIT_E_INVALID_ARG
            assert pyrit.pyrit_server_stats(srv)["submitted"] == 0
            t0 = pyrit.pyrit_server_now_ns(srv) + 2_000_000
            sched = (t0 + np.cumsum(gaps)).astype(np.int64)
            for i in range(count):
                arr[i].arrival_ns = int(sched[i])
            pyrit.pyrit_server_replay(srv, arr, 0, count)
            assert pyrit.pyrit_server_now_ns(srv) >= sched[-1]
            assert pyrit.pyrit_server_drain(srv, 60000) == 0
            done = pyrit.pyrit_server_poll(srv)
        finally:
            pyrit.pyrit_server_destroy(srv)
        assert sorted(d[0] for d in done) == list(range(count))
        for tag, status, arrival, start_ns, done_ns in done:
            assert status == 0 and arrival == sched[tag] and arrival <= start_ns <= done_ns
        h = buf.cpu().numpy()
        for i, (w_, k_, m_, P, op, er) in enumerate(reqs):
            n = (k + m) * w * P
            assert np.array_equal(h[offs[i]:offs[i] + n], want[offs[i]:offs[i] + n]), (i, reqs[i])
        assert pyrit.pyrit_device_status() == (0, 0)
    finally:
        pyrit.pyrit_plan_destroy(plan)


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
