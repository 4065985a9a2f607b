"""Mutation test of the oracle's pins.

Each mutant is a copy of ``oracle/pyrit_oracle.c`` with one plausible mistake planted in it (a
dropped term, an off-by-one index, a wrong shift, a transposed operand, a reversed tie rule). It is
compiled into a temporary directory and bound with ``oracle.bind(path)``, an independent copy of
the bindings, so the oracle that every other test uses is never replaced. Then a battery of the
committed pins (functions of ``tests/test_oracle_*.py``, at their small sizes) runs against it in a
child process (a mutant that crashes counts as caught). Every mutant must fail at least one pin,
and the unmutated source must pass them all.
"""
import importlib
import os
import subprocess
import sys
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "pyrit_oracle.c")

# (name, text in pyrit_oracle.c, replacement); each text occurs exactly once.
MUTANTS = [
    ("poly_mod skips the top reduction step", "for (int d = 63; d >= dp; d--)", "for (int d = 63; d > dp; d--)"),
    ("poly_mul drops the constant term", "for (int i = 0; i < 32; i++)\n    if ((b >> i) & 1) r ^= a << i;",
     "for (int i = 1; i < 32; i++)\n    if ((b >> i) & 1) r ^= a << i;"),
    ("AOP of degree w - 1", "return (((uint64_t)1) << (w + 1)) - 1;", "return (((uint64_t)1) << w) - 1;"),
    ("table product with the wrong modulus", "return f->alog[(f->log[a] + f->log[b]) % f->q1];",
     "return f->alog[(f->log[a] + f->log[b]) % (f->q1 + 1)];"),
    ("inverse off by one power", "return f->alog[(f->q1 - f->log[a]) % f->q1];",
     "return f->alog[(f->q1 - f->log[a] + 1) % f->q1];"),
    ("Cauchy point y_j = j + 1", "G[(k + i) * k + j] = gf_inv(&f, (uint32_t)(k + i) ^ (uint32_t)j);",
     "G[(k + i) * k + j] = gf_inv(&f, (uint32_t)(k + i) ^ (uint32_t)(j + 1));"),
    ("generator not systematic", "G[r * k + c] = (r == c);", "G[r * k + c] = (r + c == k - 1);"),
    ("Gauss-Jordan eliminates below the pivot only", "if (r == c || !M[r * 2 * k + c]) continue;",
     "if (r <= c || !M[r * 2 * k + c]) continue;"),
    ("symbol gathered with its coefficients reversed", "s |= (uint32_t)((blk[(size_t)q * P + t] >> b) & 1) << q;",
     "s |= (uint32_t)((blk[(size_t)q * P + t] >> b) & 1) << (w - 1 - q);"),
    ("scatter does not clear the old bit", "*byte = (uint8_t)((*byte & ~(1u << b)) | (((s >> q) & 1) << b));",
     "*byte = (uint8_t)(*byte | (((s >> q) & 1) << b));"),
    ("encode with a transposed source index", "acc ^= gf_mul(J->f, J->G[(J->k + i) * J->k + j], d[j]);",
     "acc ^= gf_mul(J->f, J->G[(J->k + i) * J->k + j], d[J->k - 1 - j]);"),
    ("decode re-encodes lost parity with the previous row", "val ^= gf_mul(J->f, J->G[e * k + j], d[j]);",
     "val ^= gf_mul(J->f, J->G[(e - 1) * k + j], d[j]);"),
    ("decode never takes block 0 as a survivor", "for (int e = 0; e < k + m && ns < k; e++)",
     "for (int e = 1; e < k + m && ns < k; e++)"),
    ("ring product rotated one step too far", "r ^= 1u << ((i + j) % n);", "r ^= 1u << ((i + j + 1) % n);"),
    ("sparse transform breaks ties to the largest mask", "      if (wt < bw) {\n        bw = wt;\n        best = r;",
     "      if (wt <= bw) {\n        bw = wt;\n        best = r;"),
    ("parity transform drops the first bit of each word", "for (int q = j; q < w; q += s) par ^= (b >> q) & 1u;",
     "for (int q = j + s; q < w; q += s) par ^= (b >> q) & 1u;"),
]

# The pins each mutant runs into: (test module, function, arguments), small sizes only.
BATTERY = [
    ("test_oracle_field", "test_aop_closed_forms", (4,)),
    ("test_oracle_field", "test_poly_mod_against_division_identity", ()),
    ("test_oracle_field", "test_field_axioms_exhaustive_w4", ()),
    ("test_oracle_field", "test_primitive_element_and_tables", (4,)),
    ("test_oracle_field", "test_table_multiply_equals_definition", (4,)),
    ("test_oracle_ring", "test_golden_worked_example_r25", ()),
    ("test_oracle_ring", "test_golden_embedding_inverse_w4", ()),
    ("test_oracle_ring", "test_ring_axioms_n5_exhaustive", ()),
    ("test_oracle_ring", "test_representative_sets_and_sparse_transform", (4, 5)),
    ("test_oracle_ring", "test_ring_path_equals_field_product", (4, 5)),
    ("test_oracle_coding", "test_cauchy_entries", (4, 4, 2)),
    ("test_oracle_coding", "test_invert_is_an_inverse", (4,)),
    ("test_oracle_coding", "test_encode_single_bit_basis", (4, 4, 2)),
    ("test_oracle_coding", "test_encode_is_linear", (4, 4, 2)),
    ("test_oracle_coding", "test_decode_recovers_every_pattern", (4, 4, 2, 16)),
    ("test_oracle_esp", "test_representatives_and_sparse_transform", ()),
    ("test_oracle_esp", "test_golden_transforms", ()),
    ("test_oracle_general_factor", "test_sparse_transform_and_ring_path", (2, 9, 0b111)),
    ("test_oracle_parity_transform", "test_psi_is_an_involution", (4,)),
    ("test_oracle_parity_transform", "test_encode_pt_is_the_field_code_conjugated_by_psi", (4, 4, 2, 96)),
]


def _compile(text, d):
    src = os.path.join(d, "mutant.c")
    lib = os.path.join(d, "libmutant.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", src, "-o", lib],
                          stderr=subprocess.DEVNULL)
    return lib


def _battery_fails(lib):
    """Runs the battery against the library at `lib` in a child process; returns the first pin that
    failed ("" if all passed)."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), lib], capture_output=True, text=True, timeout=300)
    if r.returncode == 0:
        return ""
    return (r.stdout.strip().splitlines() or ["exit %d" % r.returncode])[-1]


def test_unmutated_source_passes_the_battery():
    with tempfile.TemporaryDirectory() as d:
        with open(SRC) as f:
            lib = _compile(f.read(), d)
        assert _battery_fails(lib) == ""


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, "mutation site not unique or missing: %s" % name
    with tempfile.TemporaryDirectory() as d:
        lib = _compile(text.replace(old, new), d)
        assert _battery_fails(lib) != "", "no pin caught the planted mistake: %s" % name


def _run_battery(lib):
    sys.path[:0] = [ROOT, HERE]
    import oracle
    mutant = oracle.bind(lib)
    for mod_name, fn, args in BATTERY:
        mod = importlib.import_module(mod_name)
        mod.oracle = mutant  # this child process only: the pins call the bound copy
        try:
            getattr(mod, fn)(*args)
        except Exception as e:  # any failure of a pin catches the mutant
            print("%s.%s%r: %s" % (mod_name, fn, args, type(e).__name__))
            return 1
    return 0


if __name__ == "__main__":
    sys.exit(_run_battery(sys.argv[1]))
