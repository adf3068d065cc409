"""The pins must catch plausible mistakes in the oracle.

Each case compiles a copy of oracle/dot_oracle.c with one planted mistake (a
dropped term, a wrong shift, index or sign, a transposed operand), swaps it in
for the real oracle, and checks that at least one pin of
tests/test_oracle_pins.py fails.  CPU only; the real oracle is untouched.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "dot_oracle.c")

# (name, exact text in dot_oracle.c, replacement)
MUTANTS = [
    ("add_drops_carry_in", "(uint64_t)a[i] + (uint64_t)b[i] + c;", "(uint64_t)a[i] + (uint64_t)b[i];"),
    ("add_wrong_shift", "        c = t >> 32;\n    }\n    *carry", "        c = t >> 31;\n    }\n    *carry"),
    ("add_transposed", "(uint64_t)a[i] + (uint64_t)b[i] + c;", "(uint64_t)a[i] + (uint64_t)a[i] + c;"),
    ("sub_borrow_sign", "uint64_t t = (uint64_t)a[i] - (uint64_t)b[i] - br;",
     "uint64_t t = (uint64_t)a[i] - (uint64_t)b[i] + br;"),
    ("sub_operands_swapped", "uint64_t t = (uint64_t)a[i] - (uint64_t)b[i] - br;",
     "uint64_t t = (uint64_t)b[i] - (uint64_t)a[i] - br;"),
    ("sub_borrow_bit", "br = t >> 63;", "br = t >> 62;"),
    ("mul_drops_top_carry", "p[i + m] = (uint32_t)c;", "p[i + m] = 0;"),
    ("mul_index_off_by_one", "(uint64_t)a[i] * (uint64_t)b[j] + (uint64_t)p[i + j] + c;",
     "(uint64_t)a[i] * (uint64_t)b[j ? j - 1 : 0] + (uint64_t)p[i + j] + c;"),
    ("mul_drops_accumulator", "(uint64_t)a[i] * (uint64_t)b[j] + (uint64_t)p[i + j] + c;",
     "(uint64_t)a[i] * (uint64_t)b[j] + c;"),
    ("vnc_hi_same_column", "col[c + 1] += Phi[t];", "col[c] += Phi[t];"),
    ("vnc_drops_lo", "col[c] += Plo[t];", "(void)0;"),
    ("vnc_numpairs", "if (m < num_pairs) num_pairs = m;", "if (m - 1 < num_pairs) num_pairs = m - 1;"),
    ("vnc_gather_order", "Ma[idx_a++] = A[i];", "Ma[idx_a++] = A[j];"),
    ("vnc_phase5_carry", "uint64_t v = col[c] + carry;", "uint64_t v = col[c];"),
    ("ragged_carry_slot", "carry + k, (size_t)(off[k + 1] - off[k]));\n    }\n    return 0;\n}\n\nint oracle_sub_ragged",
     "carry + 0, (size_t)(off[k + 1] - off[k]));\n    }\n    return 0;\n}\n\nint oracle_sub_ragged"),
    ("mixed_op_swap", "case 0: add_one", "case 1: add_one"),
    ("gen_drops_carry_in", "uint64_t c = cin ? 1u : 0u;", "uint64_t c = 0;"),
    ("gen_pads_with_ones", "const uint64_t bi = i < mb ? (uint64_t)b[i] : 0u;",
     "const uint64_t bi = i < mb ? (uint64_t)b[i] : 0xFFFFFFFFu;"),
    ("gen_borrow_in_sign", "const uint64_t t = (uint64_t)a[i] - bi - br;",
     "const uint64_t t = (uint64_t)a[i] - bi + br;"),
    ("sqr_first_row_operand", "mul_one(a + k * m, a + k * m, p + 2 * k * m, m);",
     "mul_one(a + k * m, a, p + 2 * k * m, m);"),
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mut = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    # the mixed_op_swap mutant makes a duplicate case label: build what compiles
    r = subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", "-o", str(so), str(c)],
                       capture_output=True, text=True)
    return str(so) if r.returncode == 0 else None


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, monkeypatch, name, old, new):
    so = _build_mutant(tmp_path, name, old, new)
    if so is None:
        # a mutant that does not compile cannot ship either
        return
    monkeypatch.setattr(oracle, "_lib", oracle.bind(so))
    failed = []
    for pin in P.PINS:
        try:
            pin()
        except (AssertionError, RuntimeError):
            failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {name}"
