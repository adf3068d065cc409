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
    ("cols_hi_same_column", "if (c >= 1) t += hi[c - 1];", "t += hi[c];"),
    ("cols_drops_lo", "        if (c + 1 < 2 * m) t += lo[c];\n", ""),
    ("cols_pair_range", "const size_t i_last = c < m ? c : m - 1;\n        uint64_t l = 0",
     "const size_t i_last = c < m ? c : m - 2;\n        uint64_t l = 0"),
    ("cols_drops_carry", "        uint64_t t = carry;\n        if (c + 1", "        uint64_t t = 0;\n        if (c + 1"),
    ("cols_low_half_mask", "l += prod & 0xFFFFFFFFu;", "l += prod & 0x7FFFFFFFu;"),
    ("pairs_transposed", "            ia[t] = (int32_t)i;\n            jb[t] = (int32_t)(c - i);",
     "            ia[t] = (int32_t)(c - i);\n            jb[t] = (int32_t)i;"),
    ("ragged_carry_slot", "carry + k, (size_t)(off[k + 1] - off[k]));\n    }\n    return 0;\n}\n\nint oracle_sub_ragged",
     "carry + 0, (size_t)(off[k + 1] - off[k]));\n    }\n    return 0;\n}\n\nint oracle_sub_ragged"),
    ("mixed_op_swap", "case 0: add_one(a + a_off[i], b + b_off[i], r + r_off[i], carry + i, m); break;",
     "case 0: sub_one(a + a_off[i], b + b_off[i], r + r_off[i], carry + i, m); break;"),
    ("mixed_mul_carry_kept", "mul_one(a + a_off[i], b + b_off[i], r + r_off[i], m); carry[i] = 0; break;",
     "mul_one(a + a_off[i], b + b_off[i], r + r_off[i], m); break;"),
    ("gen_drops_carry_in", "uint64_t c = cin ? 1u : 0u;", "uint64_t c = 0;"),
    ("gen_pads_with_ones", "const uint64_t bi = i < mb ? (uint64_t)b[i] : 0u;",
     "const uint64_t bi = i < mb ? (uint64_t)b[i] : 0xFFFFFFFFu;"),
    ("gen_borrow_in_sign", "const uint64_t t = (uint64_t)a[i] - bi - br;",
     "const uint64_t t = (uint64_t)a[i] - bi + br;"),
    ("radix_mask_width", "const uint64_t mask = ((uint64_t)1 << k) - 1;",
     "const uint64_t mask = ((uint64_t)1 << (k - 1)) - 1;"),
    ("radix_drops_top_carry", "            z[i + n] = (uint32_t)c;", "            z[i + n] = 0;"),
    ("radix_carry_shift", "                c = t >> k;", "                c = t >> 32;"),
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
    r = subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", "-o", str(so), str(c)],
                       capture_output=True, text=True)
    # every mutant must compile: one that does not would test nothing
    assert r.returncode == 0, f"mutant {name} does not compile:\n{r.stderr}"
    return str(so)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, monkeypatch, name, old, new):
    so = _build_mutant(tmp_path, name, old, new)
    monkeypatch.setattr(oracle, "_lib", oracle.bind(so))
    failed = []
    for pin in P.PINS:
        try:
            pin()
        except (AssertionError, RuntimeError):
            failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {name}"
