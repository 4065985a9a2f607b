"""The no-allocation entry point against the batched entry point.

pyrit_code_stripes_noalloc is for callers that cannot call cudaMalloc (their device memory is held
by another allocator, or their request path cannot take cudaMalloc's device synchronisation): it
keeps its scratch in a fixed device array instead. Here it is called through the C ABI twice in a
row, on different stripe sets, and each result must equal, byte for byte (the tolerance of every
coding test here), what pyrit_batch_create + pyrit_batch_run write for the same stripes.

This file is named to be collected last, and it builds all of its own state, so it runs the same
alone in a fresh process and after the other tests.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pyrit():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1709_00178_gb300 import pyrit as p
    return p


def _layout(specs):
    offs, total = [], 0
    for (w, k, m, P, op, er) in specs:
        offs.append(total)
        total += ((k + m) * w * P + 255) // 256 * 256
    return offs, total


def _stripes(pyrit, plans, specs, base, offs):
    out = []
    for (w, k, m, P, op, er), o in zip(specs, offs):
        blocks = [base + o + e * w * P for e in range(k + m)]
        out.append((plans[(w, k, m)], op, er, P, blocks))
    return out


def _run_both(pyrit, plans, specs, seed):
    offs, total = _layout(specs)
    init = torch.empty(total, dtype=torch.uint8, device="cuda")
    pyrit.pyrit_synth_fill(init.data_ptr(), total, seed)
    ref = init.clone()
    got = init.clone()
    b = pyrit.pyrit_batch_create(_stripes(pyrit, plans, specs, ref.data_ptr(), offs))
    pyrit.pyrit_batch_run(b)
    torch.cuda.synchronize()
    pyrit.pyrit_batch_destroy(b)
    pyrit.pyrit_code_stripes_noalloc(_stripes(pyrit, plans, specs, got.data_ptr(), offs))
    torch.cuda.synchronize()
    assert not torch.equal(ref, init), "the reference did no work"
    return ref, got


def test_noalloc_matches_batched_entry_on_two_calls(pyrit):
    D = pyrit.PYRIT_OP_DECODE
    E = pyrit.PYRIT_OP_ENCODE
    codes = [(10, 10, 4), (4, 4, 2), (12, 16, 4)]
    plans = {c: pyrit.pyrit_plan_create(c[0], c[0] + 1, c[1], c[2]) for c in codes}
    try:
        # First call: encodes and decodes over three fields, ragged tiles and one odd packet size
        # (plain-load kernel). The decode of a stripe whose other blocks are random bytes still has
        # one defined output, which both entry points must produce.
        first = [(10, 10, 4, 8192 + 16, E, 0)] * 4 + [(4, 4, 2, 4096, E, 0), (12, 16, 4, 2048, E, 0),
                                                      (10, 10, 4, 1000, E, 0), (10, 10, 4, 4096, D, 0b1011),
                                                      (4, 4, 2, 2048, D, 0b100001), (12, 16, 4, 1024, D, 0xF0000)]
        ref, got = _run_both(pyrit, plans, first, 0xA11C)
        assert torch.equal(ref, got), "first call differs from the batched entry point"
        # Second call right after, on fewer and different stripes: the scratch still holds the first
        # call's descriptors and must not leak into this result.
        second = [(12, 16, 4, 4096 + 32, E, 0), (10, 10, 4, 2048, D, 0b11 << 10), (4, 4, 2, 64, E, 0)]
        ref, got = _run_both(pyrit, plans, second, 0xB22D)
        assert torch.equal(ref, got), "second call differs from the batched entry point"
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)


def test_noalloc_rejects_more_than_its_scratch(pyrit):
    # Every stripe points into one real device buffer, so that even a call that failed to reject
    # would only touch valid memory. Both requests must be refused before any device work.
    w, k, m, P = 4, 4, 2, 64 << 20
    plan = pyrit.pyrit_plan_create(w, w + 1, k, m)
    buf = torch.zeros((k + m) * w * P, dtype=torch.uint8, device="cuda")
    try:
        before = buf[:4096].clone()
        blocks = [buf.data_ptr() + e * w * P for e in range(k + m)]
        too_many = [(plan, pyrit.PYRIT_OP_ENCODE, 0, 64, blocks)] * (pyrit.PYRIT_NOALLOC_MAX_STRIPES + 1)
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_code_stripes_noalloc(too_many)
        assert ei.value.status == pyrit.PYRIT_E_SCRATCH_LIMIT
        # 32 stripes of 64 MiB packets: at least 32 * 1024 column tiles for any tile width up to
        # 64 KiB, more than the scratch's tile list holds
        big = [(plan, pyrit.PYRIT_OP_ENCODE, 0, P, blocks)] * 32
        with pytest.raises(pyrit.PyritError) as ei:
            pyrit.pyrit_code_stripes_noalloc(big)
        assert ei.value.status == pyrit.PYRIT_E_SCRATCH_LIMIT
        torch.cuda.synchronize()
        assert torch.equal(buf[:4096], before)
    finally:
        pyrit.pyrit_plan_destroy(plan)
        del buf


def test_noalloc_second_call_allocates_nothing(pyrit):
    # After a warm-up call (which loads the kernels it uses), an identical call must leave the
    # device's free memory unchanged and load no generated network: nothing was allocated.
    codes = [(10, 10, 4), (12, 16, 4)]
    plans = {c: pyrit.pyrit_plan_create(c[0], c[0] + 1, c[1], c[2]) for c in codes}
    try:
        specs = [(10, 10, 4, 8192, pyrit.PYRIT_OP_ENCODE, 0), (12, 16, 4, 4096, pyrit.PYRIT_OP_DECODE, 0b1011),
                 (10, 10, 4, 1000, pyrit.PYRIT_OP_ENCODE, 0)]
        offs, total = _layout(specs)
        buf = torch.empty(total, dtype=torch.uint8, device="cuda")
        pyrit.pyrit_synth_fill(buf.data_ptr(), total, 0xC33E)
        stripes = _stripes(pyrit, plans, specs, buf.data_ptr(), offs)
        pyrit.pyrit_code_stripes_noalloc(stripes)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        loaded0 = pyrit.pyrit_jit_stats()["loaded"]
        pyrit.pyrit_code_stripes_noalloc(stripes)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert pyrit.pyrit_jit_stats()["loaded"] == loaded0
        assert pyrit.pyrit_noalloc_status() == (0, 0)
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)


def test_noalloc_status_reports_a_wait_that_ran_out(pyrit):
    # A bounded wait that runs out (2 ms, on a barrier nothing completes) must come back through
    # pyrit_noalloc_status for the no-allocation scratch and through pyrit_device_status for the
    # library's error word, once, and leave the context usable.
    pyrit.pyrit_selftest_bounded_wait(1, 2_000_000)
    assert pyrit.pyrit_noalloc_status() == (pyrit.PYRIT_E_TIMEOUT, 100)
    assert pyrit.pyrit_noalloc_status() == (0, 0)  # read and cleared
    pyrit.pyrit_selftest_bounded_wait(0, 2_000_000)
    assert pyrit.pyrit_device_status() == (pyrit.PYRIT_E_TIMEOUT, 100)
    assert pyrit.pyrit_device_status() == (0, 0)
    with pytest.raises(pyrit.PyritError):
        pyrit.pyrit_selftest_bounded_wait(2, 1000)
    # the context still codes
    plans = {(4, 4, 2): pyrit.pyrit_plan_create(4, 5, 4, 2)}
    try:
        ref, got = _run_both(pyrit, plans, [(4, 4, 2, 4096, pyrit.PYRIT_OP_ENCODE, 0)], 0xD44E)
        assert torch.equal(ref, got)
        assert pyrit.pyrit_noalloc_status() == (0, 0)
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # nothing is captured, by design
def test_noalloc_refuses_stream_capture(pyrit):
    # The call uploads its descriptors from host arrays the next call rewrites, so a captured graph
    # could not replay it: on a capturing stream it must return PYRIT_E_INVALID_ARG before any
    # device work (nothing captured, nothing written), and code normally again once capture ends.
    plans = {(4, 4, 2): pyrit.pyrit_plan_create(4, 5, 4, 2)}
    try:
        specs = [(4, 4, 2, 4096, pyrit.PYRIT_OP_ENCODE, 0)]
        offs, total = _layout(specs)
        buf = torch.empty(total, dtype=torch.uint8, device="cuda")
        pyrit.pyrit_synth_fill(buf.data_ptr(), total, 0xE55F)
        stripes = _stripes(pyrit, plans, specs, buf.data_ptr(), offs)
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        before = buf.clone()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            with pytest.raises(pyrit.PyritError) as err:
                pyrit.pyrit_code_stripes_noalloc(stripes, s)
        assert err.value.status == pyrit.PYRIT_E_INVALID_ARG
        torch.cuda.synchronize()
        assert torch.equal(buf, before)
        pyrit.pyrit_code_stripes_noalloc(stripes, s)
        torch.cuda.synchronize()
        assert not torch.equal(buf, before)  # the parity blocks were written
        assert pyrit.pyrit_noalloc_status() == (0, 0)
    finally:
        for p in plans.values():
            pyrit.pyrit_plan_destroy(p)
