"""CPU oracle for PYRIT erasure coding -- TEST INFRASTRUCTURE ONLY.

Thin ctypes bindings over ``pyrit_oracle.c``: a plain, slow, literal implementation of
systematic MDS coding over GF(2^w) with the all-one polynomial modulus (log/antilog tables,
Cauchy generator, Gauss-Jordan decode) plus a brute-force reference of the ring
R_{2,n} = F2[x]/(x^n+1). It shares no code with the CUDA library and is loaded only by the
tests, the package smoke check and the benchmark's CPU-baseline leg.

Parity pins (what fixes each function independently of itself) live in
``tests/test_oracle_*.py``; every function here is pinned there.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

_lib = None


def lib():
    """The oracle library built from ``pyrit_oracle.c`` (built on first use)."""
    global _lib
    if _lib is None:
        _lib = _load(build_oracle())
    return _lib


def bind(path):
    """An independent copy of these bindings over the C library at ``path``.

    The mutation test (``tests/test_oracle_mutants.py``) compiles deliberately broken copies of
    ``pyrit_oracle.c`` and checks that the pins reject each one; it passes their paths here. The
    copy is a separate module object: this module's own functions keep using the library built
    from ``pyrit_oracle.c``, and nothing in the environment can redirect them."""
    import importlib.util
    global _bound
    _bound += 1
    spec = importlib.util.spec_from_file_location("oracle._bound%d" % _bound, __file__)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = __name__
    spec.loader.exec_module(mod)
    mod._lib = mod._load(os.path.abspath(path))
    return mod


_bound = 0


def _load(path):
    L = ctypes.CDLL(path)
    u32, u64, i32, sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
    vp = ctypes.c_void_p
    sig = {
        "oracle_poly_mod": (u64, [u64, u64]),
        "oracle_poly_mul": (u64, [u64, u64]),
        "oracle_aop": (u64, [i32]),
        "oracle_aop_irreducible": (i32, [i32]),
        "oracle_poly_irreducible": (i32, [u64]),
        "oracle_esp": (u64, [i32, i32]),
        "oracle_field_poly": (u64, [i32]),
        "oracle_ring_size": (i32, [i32]),
        "oracle_phi_P": (u32, [i32, i32, u32]),
        "oracle_ring_factor": (u64, [i32, i32]),
        "oracle_gf_mul_mod": (u32, [i32, u64, u32, u32]),
        "oracle_cauchy_mod": (i32, [i32, u64, i32, i32, vp]),
        "oracle_gf_invert_mod": (i32, [i32, u64, i32, vp, vp]),
        "oracle_encode_mod": (i32, [i32, u64, i32, i32, vp, vp, vp, sz, i32]),
        "oracle_decode_mod": (i32, [i32, u64, i32, i32, vp, vp, u64, sz, i32]),
        "oracle_sparse_rep_mod": (u32, [i32, i32, u64, u32]),
        "oracle_gf_mul_slow": (u32, [i32, u32, u32]),
        "oracle_gf_order": (u32, [i32, u32]),
        "oracle_gf_primitive": (u32, [i32]),
        "oracle_gf_tables": (i32, [i32, vp, vp, vp]),
        "oracle_gf_mul": (u32, [i32, u32, u32]),
        "oracle_cauchy": (i32, [i32, i32, i32, vp]),
        "oracle_cauchy_weighted": (i32, [i32, i32, i32, vp, vp]),
        "oracle_encode_pt": (i32, [i32, i32, i32, vp, vp, sz, i32]),
        "oracle_decode_pt": (i32, [i32, i32, i32, vp, vp, u64, sz, i32]),
        "oracle_gf_invert": (i32, [i32, i32, vp, vp]),
        "oracle_encode": (i32, [i32, i32, i32, vp, vp, vp, sz, i32]),
        "oracle_decode": (i32, [i32, i32, i32, vp, vp, u64, sz, i32]),
        "oracle_ring_mul": (u32, [i32, u32, u32]),
        "oracle_ring_idempotents": (i32, [i32, vp, i32]),
        "oracle_ring_representatives": (i32, [i32, i32, u32, vp, i32]),
        "oracle_sparse_rep": (u32, [i32, i32, u32]),
        "oracle_gf_mul_vec": (i32, [i32, vp, vp, vp, sz]),
        "oracle_gf_mul_slow_vec": (None, [i32, vp, vp, vp, sz]),
        "oracle_ring_mul_vec": (None, [i32, vp, vp, vp, sz]),
        "oracle_poly_mod_vec": (None, [u64, vp, vp, sz]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


# ---- polynomials and the field ------------------------------------------------------------

def poly_mod(a, p):
    return int(lib().oracle_poly_mod(a, p))


def poly_mul(a, b):
    return int(lib().oracle_poly_mul(a, b))


def aop(w):
    return int(lib().oracle_aop(w))


def aop_irreducible(w):
    return bool(lib().oracle_aop_irreducible(w))


def poly_irreducible(p):
    return bool(lib().oracle_poly_irreducible(p))


def esp(s, r):
    """The s-equally spaced polynomial of degree s r: 1 + x^s + ... + x^{rs} (Sec. 2.4)."""
    return int(lib().oracle_esp(s, r))


def field_poly(w):
    """The modulus of GF(2^w): the AOP if irreducible, else the irreducible ESP (0: none)."""
    return int(lib().oracle_field_poly(w))


def ring_size(w):
    """n of the ring R_{2,n} carrying GF(2^w) (w + 1 for an AOP, 9 for GF(2^6)); 0 if none."""
    return int(lib().oracle_ring_size(w))


def ring_factor(w, n):
    """The smallest irreducible factor of degree w of x^n + 1 (n odd; Props. 1-2), 0 if none."""
    return int(lib().oracle_ring_factor(w, n))


def gf_mul_mod(w, poly, a, b):
    """Product in F2[x]/(poly) by the definition (carry-less product, remainder)."""
    return int(lib().oracle_gf_mul_mod(w, poly, a, b))


def cauchy_mod(w, poly, k, m):
    G = np.zeros((k + m, k), np.uint32)
    rc = lib().oracle_cauchy_mod(w, poly, k, m, _p(G))
    if rc:
        raise ValueError("oracle_cauchy_mod(w=%d,poly=%#x,k=%d,m=%d) -> %d" % (w, poly, k, m, rc))
    return G


def gf_invert_mod(w, poly, A):
    A = _u32(A)
    k = A.shape[0]
    inv = np.zeros_like(A)
    rc = lib().oracle_gf_invert_mod(w, poly, k, _p(A), _p(inv))
    if rc:
        raise ValueError("singular")
    return inv


def encode_mod(w, poly, k, m, G, data, nthreads=1):
    """encode() over F2[x]/(poly)."""
    G = _u32(G)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    P = data.size // (k * w)
    parity = np.zeros((m, w, P), np.uint8)
    rc = lib().oracle_encode_mod(w, poly, k, m, _p(G), _p(data), _p(parity), P, nthreads)
    if rc:
        raise ValueError("oracle_encode_mod -> %d" % rc)
    return parity


def decode_mod(w, poly, k, m, G, blocks, erased, nthreads=1):
    """decode() over F2[x]/(poly)."""
    G = _u32(G)
    out = np.array(blocks, dtype=np.uint8, copy=True, order="C")
    P = out.size // ((k + m) * w)
    rc = lib().oracle_decode_mod(w, poly, k, m, _p(G), _p(out), erased, P, nthreads)
    if rc:
        raise ValueError("oracle_decode_mod -> %d" % rc)
    return out.reshape(k + m, w, P)


def sparse_rep_mod(w, n, poly, u):
    """phi_S over the representatives of u mod poly in R_{2,n}."""
    return int(lib().oracle_sparse_rep_mod(w, n, poly, u))


def phi_P(w, n, b):
    """The parity transform of a field element (Sec. 2.3.1, Sec. 2.4.1)."""
    return int(lib().oracle_phi_P(w, n, b))


def gf_mul_slow(w, a, b):
    return int(lib().oracle_gf_mul_slow(w, a, b))


def gf_order(w, g):
    return int(lib().oracle_gf_order(w, g))


def gf_primitive(w):
    return int(lib().oracle_gf_primitive(w))


def gf_tables(w):
    log = np.zeros(1 << w, np.uint32)
    alog = np.zeros(1 << w, np.uint32)
    g = np.zeros(1, np.uint32)
    if lib().oracle_gf_tables(w, _p(log), _p(alog), _p(g)):
        raise ValueError("unsupported field w=%d" % w)
    return log, alog, int(g[0])


def gf_mul_vec(w, a, b):
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    if lib().oracle_gf_mul_vec(w, _p(a), _p(b), _p(out), a.size):
        raise ValueError("unsupported field w=%d" % w)
    return out


def gf_mul_slow_vec(w, a, b):
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    lib().oracle_gf_mul_slow_vec(w, _p(a), _p(b), _p(out), a.size)
    return out


def cauchy(w, k, m):
    G = np.zeros((k + m, k), np.uint32)
    rc = lib().oracle_cauchy(w, k, m, _p(G))
    if rc:
        raise ValueError("oracle_cauchy(w=%d,k=%d,m=%d) -> %d" % (w, k, m, rc))
    return G


def cauchy_weighted(w, k, m):
    """Weight-optimised generalized Cauchy generator and its (plain, optimised) total weights."""
    G = np.zeros((k + m, k), np.uint32)
    wts = np.zeros(2, np.uint64)
    rc = lib().oracle_cauchy_weighted(w, k, m, _p(G), wts.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise ValueError("oracle_cauchy_weighted(w=%d,k=%d,m=%d) -> %d" % (w, k, m, rc))
    return G, (int(wts[0]), int(wts[1]))


def gf_invert(w, A):
    A = _u32(A)
    k = A.shape[0]
    Inv = np.zeros_like(A)
    rc = lib().oracle_gf_invert(w, k, _p(A), _p(Inv))
    if rc:
        raise ValueError("singular" if rc == -1 else "unsupported field")
    return Inv


# ---- coding -----------------------------------------------------------------------------

def encode(w, k, m, G, data, nthreads=1):
    """data: uint8 array of shape (k, w, P) (any shape with k*w*P bytes). Returns (m, w, P)."""
    G = _u32(G)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    P = data.size // (k * w)
    assert data.size == k * w * P
    parity = np.zeros((m, w, P), np.uint8)
    rc = lib().oracle_encode(w, k, m, _p(G), _p(data), _p(parity), P, nthreads)
    if rc:
        raise ValueError("oracle_encode -> %d" % rc)
    return parity


def decode(w, k, m, G, blocks, erased, nthreads=1):
    """blocks: uint8 (k+m, w, P); erased blocks are rebuilt in a returned copy."""
    G = _u32(G)
    out = np.array(blocks, dtype=np.uint8, copy=True, order="C")
    P = out.size // ((k + m) * w)
    assert out.size == (k + m) * w * P
    rc = lib().oracle_decode(w, k, m, _p(G), _p(out), erased, P, nthreads)
    if rc:
        raise ValueError("oracle_decode -> %d" % rc)
    return out.reshape(k + m, w, P)


def encode_pt(w, k, m, G, data, nthreads=1):
    """Parity-transform encoding (Sec. 2.3.1). data: uint8 (k, w, P). Returns the parity (m, w, P)."""
    G = _u32(G)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    P = data.size // (k * w)
    blocks = np.zeros((k + m, w, P), np.uint8)
    blocks[:k] = data.reshape(k, w, P)
    rc = lib().oracle_encode_pt(w, k, m, _p(G), _p(blocks), P, nthreads)
    if rc:
        raise ValueError("oracle_encode_pt -> %d" % rc)
    return blocks[k:].copy()


def decode_pt(w, k, m, G, blocks, erased, nthreads=1):
    """Parity-transform decoding: blocks (k+m, w, P); erased blocks are rebuilt in a returned copy."""
    G = _u32(G)
    out = np.array(blocks, dtype=np.uint8, copy=True, order="C")
    P = out.size // ((k + m) * w)
    rc = lib().oracle_decode_pt(w, k, m, _p(G), _p(out), erased, P, nthreads)
    if rc:
        raise ValueError("oracle_decode_pt -> %d" % rc)
    return out.reshape(k + m, w, P)


# ---- ring reference ---------------------------------------------------------------------

def ring_mul(n, a, b):
    return int(lib().oracle_ring_mul(n, a, b))


def ring_mul_vec(n, a, b):
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    lib().oracle_ring_mul_vec(n, _p(a), _p(b), _p(out), a.size)
    return out


def poly_mod_vec(p, a):
    a = _u32(a)
    out = np.zeros_like(a)
    lib().oracle_poly_mod_vec(p, _p(a), _p(out), a.size)
    return out


def ring_idempotents(n):
    out = np.zeros(1 << n, np.uint32)
    c = lib().oracle_ring_idempotents(n, _p(out), out.size)
    return [int(x) for x in out[:c]]


def ring_representatives(w, n, u):
    out = np.zeros(1 << n, np.uint32)
    c = lib().oracle_ring_representatives(w, n, u, _p(out), out.size)
    return [int(x) for x in out[:c]]


def sparse_rep(w, n, u):
    return int(lib().oracle_sparse_rep(w, n, u))
