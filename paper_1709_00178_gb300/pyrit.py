"""ctypes binding of the C ABI in ``include/pyrit.h`` (argument marshalling only).

Every function keeps its C name. Pointer arguments accept ints (device addresses, e.g. a torch
tensor's ``data_ptr()``), lists of ints (host arrays of device pointers) or numpy arrays (host
arrays). A negative status raises :class:`PyritError`. Streams are ``cudaStream_t`` values as ints
(``torch.cuda.current_stream().cuda_stream``) or None for the default stream.

Importing this module loads ``libpyrit.so`` and fails loudly if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``); there is no fallback.
"""
import atexit
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpyrit.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libpyrit.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

PYRIT_OK = 0
PYRIT_E_INVALID_ARG = -1
PYRIT_E_UNSUPPORTED_FIELD = -2
PYRIT_E_TOO_LONG = -3
PYRIT_E_NOT_MDS = -4
PYRIT_E_TOO_MANY_ERASURES = -5
PYRIT_E_CUDA = -6
PYRIT_E_OOM = -7
PYRIT_E_BUDGET = -8
PYRIT_E_TIMEOUT = -9
PYRIT_E_BUSY = -10
PYRIT_E_SCRATCH_LIMIT = -11
PYRIT_E_JIT = -12
PYRIT_E_UNSUPPORTED = -13
PYRIT_DISPATCH_NETWORK = 3
PYRIT_JIT_OFF = 0
PYRIT_JIT_SYNC = 1
PYRIT_JIT_ASYNC = 2
PYRIT_NOALLOC_MAX_STRIPES = 256
PYRIT_NOALLOC_MAX_TILES = 16384
PYRIT_MAX_K = 64
PYRIT_MAX_M = 63
PYRIT_MAX_BLOCKS = 64
PYRIT_JOB_OUTPUTS = 8
PYRIT_OP_ENCODE = 0
PYRIT_OP_DECODE = 1
PYRIT_OP_DECODE_ANY = 2
PYRIT_TRANSFORM_EMBEDDING = 0
PYRIT_TRANSFORM_PARITY = 1
PYRIT_TRANSFORM_AUTO = 2

_i, _u32, _u64, _sz, _vp = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_void_p

_SIGS = {
    "pyrit_strerror": (ctypes.c_char_p, [_i]),
    "pyrit_plan_create": (_i, [_i, _i, _i, _i, _vp, ctypes.POINTER(_vp)]),
    "pyrit_plan": (_i, [_i, _i, _i, _i, _vp, ctypes.POINTER(_vp)]),
    "pyrit_plan_destroy": (None, [_vp]),
    "pyrit_plan_info": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "pyrit_plan_set_transform": (_i, [_vp, _i]),
    "pyrit_plan_modulus": (_i, [_vp, _vp, _vp]),
    "pyrit_plan_generator": (_i, [_vp, _vp]),
    "pyrit_plan_encode_masks": (_i, [_vp, _vp]),
    "pyrit_plan_decode_masks": (_i, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "pyrit_plan_syndrome_masks": (_i, [_vp, _u64, _vp, _vp]),
    "pyrit_generator_weighted": (_i, [_i, _i, _i, _i, _vp, _vp]),
    "pyrit_sparse_transform": (_u32, [_i, _i, _u32]),
    "pyrit_gf_mul": (_u32, [_i, _u32, _u32]),
    "pyrit_encode": (_i, [_vp, _vp, _vp, _sz, _vp]),
    "pyrit_decode": (_i, [_vp, _vp, _u64, _sz, _vp]),
    "pyrit_device_status": (_i, [_vp, _vp]),
    "pyrit_synth_fill": (_i, [_vp, _sz, _u64, _u64, _vp]),
}


def _bind(sigs):
    for name, (res, args) in sigs.items():
        f = getattr(_lib, name)
        f.restype = res
        f.argtypes = args


_bind(_SIGS)

#: Every symbol the header declares (the CPU test checks the library exports each of them).
EXPORTS = tuple(_SIGS)


class PyritError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__("%s%s (status %d)" % (where + ": " if where else "",
                                              _lib.pyrit_strerror(status).decode(), status))


def _check(rc, where):
    if rc < 0:
        raise PyritError(rc, where)
    return rc


def _ptr_array(ptrs):
    """Host array of device pointers from a list of ints / tensors."""
    vals = [p.data_ptr() if hasattr(p, "data_ptr") else int(p) for p in ptrs]
    return (ctypes.c_void_p * max(1, len(vals)))(*vals)


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def _dev(p):
    return ctypes.c_void_p(p.data_ptr() if hasattr(p, "data_ptr") else int(p))


# ---- C-named functions ------------------------------------------------------------------------

def pyrit_strerror(status):
    return _lib.pyrit_strerror(status).decode()


def pyrit_plan_create(w, n, k, m, G=None):
    """Returns an opaque plan handle (int). G: None or a (k+m) x k array of field elements."""
    h = ctypes.c_void_p()
    g = None
    if G is not None:
        g = np.ascontiguousarray(np.asarray(G, dtype=np.uint32))
        if g.shape != (k + m, k):
            raise ValueError("G must be (k+m) x k")
    _check(_lib.pyrit_plan_create(w, n, k, m, _np_ptr(g) if g is not None else None, ctypes.byref(h)),
           "pyrit_plan_create")
    return h.value


def pyrit_plan(w, n, k, m, G=None):
    """pyrit_plan_create with 16-bit generator entries."""
    h = ctypes.c_void_p()
    g = None
    if G is not None:
        g = np.ascontiguousarray(np.asarray(G, dtype=np.uint16))
        if g.shape != (k + m, k):
            raise ValueError("G must be (k+m) x k")
    _check(_lib.pyrit_plan(w, n, k, m, _np_ptr(g) if g is not None else None, ctypes.byref(h)), "pyrit_plan")
    return h.value


def pyrit_plan_destroy(plan):
    _lib.pyrit_plan_destroy(plan)


def pyrit_plan_info(plan):
    v = [ctypes.c_int() for _ in range(4)]
    _check(_lib.pyrit_plan_info(plan, *[ctypes.byref(x) for x in v]), "pyrit_plan_info")
    return tuple(x.value for x in v)


def pyrit_plan_generator(plan):
    w, n, k, m = pyrit_plan_info(plan)
    G = np.zeros((k + m, k), np.uint32)
    _check(_lib.pyrit_plan_generator(plan, _np_ptr(G)), "pyrit_plan_generator")
    return G


def pyrit_plan_encode_masks(plan):
    w, n, k, m = pyrit_plan_info(plan)
    M = np.zeros((m, k), np.uint16)
    _check(_lib.pyrit_plan_encode_masks(plan, _np_ptr(M)), "pyrit_plan_encode_masks")
    return M


def pyrit_plan_decode_masks(plan, erasures):
    """Returns (survivors[k], erased[ne], masks[ne, k])."""
    w, n, k, m = pyrit_plan_info(plan)
    surv = np.zeros(k, np.int32)
    er = np.zeros(max(1, m), np.int32)
    M = np.zeros((max(1, m), k), np.uint16)
    ne = ctypes.c_int()
    _check(_lib.pyrit_plan_decode_masks(plan, erasures, _np_ptr(surv), _np_ptr(er), _np_ptr(M), ctypes.byref(ne)),
           "pyrit_plan_decode_masks")
    return surv, er[:ne.value].copy(), M[:ne.value].copy()


def pyrit_plan_syndrome_masks(plan, erasures):
    """(syn, ne): syn is a 9 x 8 uint16 array (rows r = parity rows, row 8 = 1 + base row)."""
    syn = np.zeros((9, 8), np.uint16)
    ne = ctypes.c_int()
    _check(_lib.pyrit_plan_syndrome_masks(plan, erasures, _np_ptr(syn), ctypes.byref(ne)),
           "pyrit_plan_syndrome_masks")
    return syn, ne.value


def pyrit_plan_modulus(plan):
    """(g, native): the plan's field modulus and whether the generic kernels serve it."""
    g, nat = ctypes.c_uint32(), ctypes.c_int()
    _check(_lib.pyrit_plan_modulus(plan, ctypes.byref(g), ctypes.byref(nat)), "pyrit_plan_modulus")
    return g.value, bool(nat.value)


def pyrit_plan_set_transform(plan, transform):
    """Sets the plan's transform (PYRIT_TRANSFORM_*); returns the one in force (AUTO resolved)."""
    return _check(_lib.pyrit_plan_set_transform(plan, transform), "pyrit_plan_set_transform")


def pyrit_generator_weighted(w, n, k, m):
    """(G, (weight_default, weight_optimised)): a weight-optimised generalized Cauchy generator."""
    G = np.zeros((k + m, k), np.uint32)
    wts = np.zeros(2, np.uint64)
    _check(_lib.pyrit_generator_weighted(w, n, k, m, _np_ptr(G), _np_ptr(wts)), "pyrit_generator_weighted")
    return G, (int(wts[0]), int(wts[1]))


def pyrit_sparse_transform(w, n, u):
    return int(_lib.pyrit_sparse_transform(w, n, u))


def pyrit_gf_mul(w, a, b):
    return int(_lib.pyrit_gf_mul(w, a, b))


def pyrit_encode(plan, data, parity, P, stream=None):
    """data: k device pointers (ints or tensors); parity: m device pointers."""
    return _check(_lib.pyrit_encode(plan, _ptr_array(data), _ptr_array(parity), P, _stream(stream)), "pyrit_encode")


def pyrit_decode(plan, blocks, erasures, P, stream=None):
    """blocks: k+m device pointers; erased ones are rebuilt in place."""
    return _check(_lib.pyrit_decode(plan, _ptr_array(blocks), erasures, P, _stream(stream)), "pyrit_decode")


def pyrit_device_status():
    code, where = ctypes.c_int(), ctypes.c_int()
    _check(_lib.pyrit_device_status(ctypes.byref(code), ctypes.byref(where)), "pyrit_device_status")
    return code.value, where.value


def pyrit_synth_fill(dst, nbytes, seed, offset=0, stream=None):
    return _check(_lib.pyrit_synth_fill(_dev(dst), nbytes, seed, offset, _stream(stream)), "pyrit_synth_fill")


# ---- batches ------------------------------------------------------------------------------------

class pyrit_stripe_t(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("op", ctypes.c_int), ("erasures", ctypes.c_uint64),
                ("packet_bytes", ctypes.c_size_t), ("blocks", ctypes.POINTER(ctypes.c_void_p))]


class pyrit_tile_t(ctypes.Structure):
    _fields_ = [("words", ctypes.c_int), ("mg", ctypes.c_int), ("minb", ctypes.c_int), ("nc", ctypes.c_int),
                ("dispatch", ctypes.c_int), ("stages", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


_BATCH_SIGS = {
    "pyrit_batch_create": (_i, [ctypes.POINTER(pyrit_stripe_t), _i, ctypes.POINTER(pyrit_tile_t),
                                ctypes.POINTER(_vp)]),
    "pyrit_batch_run": (_i, [_vp, _vp, _i]),
    "pyrit_batch_stats": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "pyrit_batch_destroy": (None, [_vp]),
    "pyrit_encode_batch": (_i, [ctypes.POINTER(pyrit_stripe_t), _i, _vp]),
    "pyrit_decode_batch": (_i, [ctypes.POINTER(pyrit_stripe_t), _i, _vp]),
    "pyrit_batch_tune": (_i, [_vp, _vp, _i]),
    "pyrit_tune_save": (_i, [ctypes.c_char_p]),
    "pyrit_tune_load": (_i, [ctypes.c_char_p]),
    "pyrit_tune_clear": (_i, []),
    "pyrit_variants": (_i, [_vp, _i]),
    "pyrit_batch_shape": (_i, [_vp, _i, _vp]),
}
_bind(_BATCH_SIGS)
EXPORTS = EXPORTS + tuple(_BATCH_SIGS)


def pyrit_batch_create(stripes, tile=None):
    """stripes: list of (plan, op, erasures, P, block_ptrs[k+m]); tile: None or dict of overrides
    (words, mg, minb, nc, dispatch, stages, ctas_per_sm). Returns an opaque batch handle."""
    arr, keep = _stripe_array(stripes)
    t = None
    if tile is not None:
        t = pyrit_tile_t(tile.get("words", 0), tile.get("mg", 0), tile.get("minb", 0), tile.get("nc", 0),
                         tile.get("dispatch", -1), tile.get("stages", 0), tile.get("ctas_per_sm", 0))
    h = ctypes.c_void_p()
    _check(_lib.pyrit_batch_create(arr, len(stripes), ctypes.byref(t) if t is not None else None, ctypes.byref(h)),
           "pyrit_batch_create")
    return h.value


def _stripe_array(stripes):
    arr = (pyrit_stripe_t * max(1, len(stripes)))()
    keep = []
    for i, (plan, op, er, P, blocks) in enumerate(stripes):
        ba = _ptr_array(blocks)
        keep.append(ba)
        arr[i] = pyrit_stripe_t(plan, op, er, P, ctypes.cast(ba, ctypes.POINTER(ctypes.c_void_p)))
    return arr, keep


def pyrit_encode_batch(stripes, stream=None):
    """One-shot batched encode of stripes (plan, PYRIT_OP_ENCODE, 0, P, block_ptrs[k+m]); waits."""
    arr, keep = _stripe_array(stripes)
    return _check(_lib.pyrit_encode_batch(arr, len(stripes), _stream(stream)), "pyrit_encode_batch")


def pyrit_decode_batch(stripes, stream=None):
    """One-shot batched decode of stripes (plan, PYRIT_OP_DECODE, erasures, P, block_ptrs[k+m]); waits."""
    arr, keep = _stripe_array(stripes)
    return _check(_lib.pyrit_decode_batch(arr, len(stripes), _stream(stream)), "pyrit_decode_batch")


def pyrit_batch_run(batch, stream=None, graph=False):
    return _check(_lib.pyrit_batch_run(batch, _stream(stream), 1 if graph else 0), "pyrit_batch_run")


def pyrit_batch_stats(batch):
    a, s, t = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    n = ctypes.c_int()
    _check(_lib.pyrit_batch_stats(batch, ctypes.byref(a), ctypes.byref(s), ctypes.byref(n), ctypes.byref(t)),
           "pyrit_batch_stats")
    return {"alg_bytes": a.value, "src_bytes": s.value, "launches": n.value, "tiles": t.value}


def pyrit_batch_destroy(batch):
    _lib.pyrit_batch_destroy(batch)


def pyrit_batch_tune(batch, stream=None, iters=3):
    return _check(_lib.pyrit_batch_tune(batch, _stream(stream), iters), "pyrit_batch_tune")


def pyrit_variants():
    """List of dicts (n, words, mg, minb, dispatch, nc), one per compiled kernel variant."""
    n = _lib.pyrit_variants(None, 0)
    buf = np.zeros(6 * max(1, n), np.int32)
    _lib.pyrit_variants(_np_ptr(buf), n)
    keys = ("n", "words", "mg", "minb", "dispatch", "nc")
    return [dict(zip(keys, (int(x) for x in buf[6 * i:6 * i + 6]))) for i in range(n)]


def pyrit_batch_shape(batch, group=0):
    """Launch shape of one group of a batch: dict of n, words, mg, minb, dispatch, nc, groups, tw,
    stages, grid, mode (dispatch 3 = a plan-specialised network; mode 1 = syndrome decode)."""
    buf = np.zeros(11, np.int32)
    _check(_lib.pyrit_batch_shape(batch, group, _np_ptr(buf)), "pyrit_batch_shape")
    keys = ("n", "words", "mg", "minb", "dispatch", "nc", "groups", "tw", "stages", "grid", "mode")
    return dict(zip(keys, (int(x) for x in buf)))


def pyrit_tune_save(path):
    return _check(_lib.pyrit_tune_save(os.fsencode(path)), "pyrit_tune_save")


def pyrit_tune_load(path):
    return _check(_lib.pyrit_tune_load(os.fsencode(path)), "pyrit_tune_load")


def pyrit_tune_clear():
    return _check(_lib.pyrit_tune_clear(), "pyrit_tune_clear")


# ---- plan-specialised networks (run-time compilation) ------------------------------------------

_JIT_SIGS = {
    "pyrit_jit_mode": (_i, [_i]),
    "pyrit_plan_specialise": (_i, [_vp, _i, _u64, ctypes.POINTER(pyrit_tile_t)]),
    "pyrit_plan_network_info": (_i, [_vp, _i, _u64, ctypes.POINTER(pyrit_tile_t), _vp]),
    "pyrit_plan_network_source": (_i, [_vp, _i, _u64, ctypes.POINTER(pyrit_tile_t), ctypes.c_char_p, _i]),
    "pyrit_jit_wait": (_i, [_i]),
    "pyrit_jit_quiesce": (_i, [_i]),
    "pyrit_jit_stats": (_i, [_vp]),
    "pyrit_jit_log": (_i, [ctypes.c_char_p, _i]),
    "pyrit_jit_source": (_i, [_i, _i, _i, _vp, ctypes.POINTER(pyrit_tile_t), _i, ctypes.c_char_p, _i]),
}
_bind(_JIT_SIGS)
EXPORTS = EXPORTS + tuple(_JIT_SIGS)


def _tile(tile):
    if tile is None:
        return None
    return pyrit_tile_t(tile.get("words", 0), tile.get("mg", 0), tile.get("minb", 0), tile.get("nc", 0),
                        tile.get("dispatch", -1), tile.get("stages", 0), tile.get("ctas_per_sm", 0))


def pyrit_jit_mode(mode=-1):
    """Sets the run-time compilation policy (PYRIT_JIT_*) and returns the previous one."""
    return _check(_lib.pyrit_jit_mode(mode), "pyrit_jit_mode")


def pyrit_plan_specialise(plan, op=PYRIT_OP_ENCODE, erasures=0, tile=None):
    t = _tile(tile)
    return _check(_lib.pyrit_plan_specialise(plan, op, erasures, ctypes.byref(t) if t is not None else None),
                  "pyrit_plan_specialise")


def pyrit_plan_network_source(plan, op=PYRIT_OP_ENCODE, erasures=0, tile=None):
    """CUDA source of a plan's generated network (the first job's)."""
    t = _tile(tile)
    tp = ctypes.byref(t) if t is not None else None
    size = _check(_lib.pyrit_plan_network_source(plan, op, erasures, tp, None, 0), "pyrit_plan_network_source")
    buf = ctypes.create_string_buffer(size + 1)
    _lib.pyrit_plan_network_source(plan, op, erasures, tp, buf, size + 1)
    return buf.value.decode()


def pyrit_plan_network_info(plan, op=PYRIT_OP_ENCODE, erasures=0, tile=None):
    """Resource use of a plan's generated network (compiled if missing): dict of registers,
    stack_bytes, spill_store_bytes, spill_load_bytes, compile_ms, words, mg, nc, mode."""
    t = _tile(tile)
    info = np.zeros(9, np.int32)
    _check(_lib.pyrit_plan_network_info(plan, op, erasures, ctypes.byref(t) if t is not None else None,
                                        _np_ptr(info)), "pyrit_plan_network_info")
    keys = ("registers", "stack_bytes", "spill_store_bytes", "spill_load_bytes", "compile_ms", "words", "mg", "nc", "mode")
    return {k: int(v) for k, v in zip(keys, info)}


def pyrit_jit_wait(timeout_ms=60000):
    return _check(_lib.pyrit_jit_wait(timeout_ms), "pyrit_jit_wait")


def pyrit_jit_quiesce(timeout_ms=60000):
    return _check(_lib.pyrit_jit_quiesce(timeout_ms), "pyrit_jit_quiesce")


@atexit.register
def _quiesce_at_exit():
    # No background compilation may still run while the interpreter and CUDA shut down.
    _lib.pyrit_jit_mode(PYRIT_JIT_OFF)
    _lib.pyrit_jit_quiesce(120000)


def pyrit_jit_stats():
    buf = np.zeros(8, np.uint64)
    _check(_lib.pyrit_jit_stats(_np_ptr(buf)), "pyrit_jit_stats")
    keys = ("cached", "compiled", "failed", "pending", "hits", "loaded", "compile_us", "queued_total")
    return dict(zip(keys, (int(x) for x in buf)))


def pyrit_jit_log():
    n = _lib.pyrit_jit_log(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    _lib.pyrit_jit_log(buf, n + 1)
    return buf.value.decode(errors="replace")


def pyrit_jit_source(n, masks, tile=None, transform=PYRIT_TRANSFORM_EMBEDDING):
    """Generated CUDA source for a mask table (2-D array, masks[o][j] = phi_S mask of output o,
    source j) over R_{2,n}, for the embedding or the parity transform."""
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint16))
    nout, nin = m.shape
    t = _tile(tile)
    tp = ctypes.byref(t) if t is not None else None
    size = _check(_lib.pyrit_jit_source(n, nin, nout, _np_ptr(m), tp, transform, None, 0), "pyrit_jit_source")
    buf = ctypes.create_string_buffer(size + 1)
    _lib.pyrit_jit_source(n, nin, nout, _np_ptr(m), tp, transform, buf, size + 1)
    return buf.value.decode()


# ---- coding without device allocation ---------------------------------------------------------

_NOALLOC_SIGS = {"pyrit_code_stripes_noalloc": (_i, [ctypes.POINTER(pyrit_stripe_t), _i, _vp]),
                 "pyrit_noalloc_status": (_i, [_vp, _vp, _vp]),
                 "pyrit_selftest_bounded_wait": (_i, [_i, _u64, _vp])}
_bind(_NOALLOC_SIGS)
EXPORTS = EXPORTS + tuple(_NOALLOC_SIGS)


def pyrit_code_stripes_noalloc(stripes, stream=None):
    """Codes stripes (list of (plan, op, erasures, P, block_ptrs[k+m])) with the library's fixed
    device scratch instead of any device allocation, for callers that cannot call cudaMalloc."""
    arr = (pyrit_stripe_t * max(1, len(stripes)))()
    keep = []
    for i, (plan, op, er, P, blocks) in enumerate(stripes):
        ba = _ptr_array(blocks)
        keep.append(ba)
        arr[i] = pyrit_stripe_t(plan, op, er, P, ctypes.cast(ba, ctypes.POINTER(ctypes.c_void_p)))
    return _check(_lib.pyrit_code_stripes_noalloc(arr, len(stripes), _stream(stream)), "pyrit_code_stripes_noalloc")


def pyrit_noalloc_status(stream=None):
    """(code, site) of the no-allocation entry point's status words, read and cleared after the
    work queued on `stream`."""
    code, where = ctypes.c_int(), ctypes.c_int()
    _check(_lib.pyrit_noalloc_status(ctypes.byref(code), ctypes.byref(where), _stream(stream)),
           "pyrit_noalloc_status")
    return code.value, where.value


def pyrit_selftest_bounded_wait(channel, limit_ns, stream=None):
    """Enqueues a bounded wait that runs out after limit_ns and records PYRIT_E_TIMEOUT in the
    library's error word (channel 0) or the no-allocation status words (channel 1)."""
    return _check(_lib.pyrit_selftest_bounded_wait(channel, limit_ns, _stream(stream)),
                  "pyrit_selftest_bounded_wait")


# ---- served coding -----------------------------------------------------------------------------

class pyrit_request_t(ctypes.Structure):
    _fields_ = [("stripe", pyrit_stripe_t), ("tag", ctypes.c_uint64), ("arrival_ns", ctypes.c_int64)]


class pyrit_completion_t(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("arrival_ns", ctypes.c_int64),
                ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


_SERVER_SIGS = {
    "pyrit_server_create": (_i, [_sz, _i, _i, _i, ctypes.POINTER(_vp)]),
    "pyrit_server_submit": (_i, [_vp, ctypes.POINTER(pyrit_request_t), _i]),
    "pyrit_server_poll": (_i, [_vp, ctypes.POINTER(pyrit_completion_t), _i]),
    "pyrit_server_replay": (_i, [_vp, ctypes.POINTER(pyrit_request_t), _i]),
    "pyrit_server_drain": (_i, [_vp, _i]),
    "pyrit_server_now_ns": (ctypes.c_int64, [_vp]),
    "pyrit_server_stats": (_i, [_vp, _vp]),
    "pyrit_server_destroy": (None, [_vp]),
}
_bind(_SERVER_SIGS)
EXPORTS = EXPORTS + tuple(_SERVER_SIGS)


def pyrit_server_create(hbm_budget, max_batch=64, slots=4, queue_cap=1 << 20):
    h = ctypes.c_void_p()
    _check(_lib.pyrit_server_create(hbm_budget, max_batch, slots, queue_cap, ctypes.byref(h)), "pyrit_server_create")
    return h.value


def pyrit_server_submit(server, requests):
    """requests: list of (plan, op, erasures, P, block_ptrs[k+m], tag, arrival_ns)."""
    arr = (pyrit_request_t * max(1, len(requests)))()
    keep = []
    for i, (plan, op, er, P, blocks, tag, arrival) in enumerate(requests):
        ba = _ptr_array(blocks)
        keep.append(ba)
        arr[i] = pyrit_request_t(pyrit_stripe_t(plan, op, er, P, ctypes.cast(ba, ctypes.POINTER(ctypes.c_void_p))),
                                 tag, arrival)
    return _check(_lib.pyrit_server_submit(server, arr, len(requests)), "pyrit_server_submit")


def pyrit_server_poll(server, cap=4096):
    """List of (tag, status, arrival_ns, start_ns, done_ns)."""
    buf = (pyrit_completion_t * cap)()
    n = _check(_lib.pyrit_server_poll(server, buf, cap), "pyrit_server_poll")
    return [(c.tag, c.status, c.arrival_ns, c.start_ns, c.done_ns) for c in buf[:n]]


def pyrit_server_drain(server, timeout_ms):
    return _check(_lib.pyrit_server_drain(server, timeout_ms), "pyrit_server_drain")


def pyrit_server_now_ns(server):
    return int(_lib.pyrit_server_now_ns(server))


def pyrit_server_stats(server):
    s = np.zeros(7, np.uint64)
    _check(_lib.pyrit_server_stats(server, _np_ptr(s)), "pyrit_server_stats")
    keys = ("submitted", "completed", "batches", "launches", "inflight", "max_inflight", "budget")
    return {k: int(v) for k, v in zip(keys, s)}


def pyrit_server_destroy(server):
    _lib.pyrit_server_destroy(server)


def pyrit_requests_array(requests):
    """A prebuilt ctypes array of requests (plan, op, erasures, P, block_ptrs, tag, arrival_ns) and the
    pointer arrays it references, for pyrit_server_submit_slice."""
    arr = (pyrit_request_t * max(1, len(requests)))()
    keep = []
    for i, (plan, op, er, P, blocks, tag, arrival) in enumerate(requests):
        ba = _ptr_array(blocks)
        keep.append(ba)
        arr[i] = pyrit_request_t(pyrit_stripe_t(plan, op, er, P, ctypes.cast(ba, ctypes.POINTER(ctypes.c_void_p))),
                                 tag, arrival)
    return arr, keep


def pyrit_server_replay(server, arr, start=0, count=None):
    """Submits arr[start:start + count] of a prebuilt request array (non-decreasing arrival times),
    each when the server clock reaches its arrival; returns once all are submitted."""
    if count is None:
        count = len(arr) - start
    ptr = ctypes.cast(ctypes.byref(arr, start * ctypes.sizeof(pyrit_request_t)), ctypes.POINTER(pyrit_request_t))
    return _check(_lib.pyrit_server_replay(server, ptr, count), "pyrit_server_replay")


def pyrit_server_submit_slice(server, arr, start, count):
    """Submits arr[start:start + count] of a prebuilt request array without copying it."""
    ptr = ctypes.cast(ctypes.byref(arr, start * ctypes.sizeof(pyrit_request_t)), ctypes.POINTER(pyrit_request_t))
    return _check(_lib.pyrit_server_submit(server, ptr, count), "pyrit_server_submit")
