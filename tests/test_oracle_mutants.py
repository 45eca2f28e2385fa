"""Planted mistakes: each one, put into a copy of the oracle, must make a pin fail.

A pin that no plausible mistake can fail pins nothing.  Each case below edits
one rule of oracle/csgv_oracle.c the way a careless reading of the paper
would (a tie broken the other way, an index off by one, a skipped step),
compiles the copy, and runs the oracle's pins (tests/test_oracle.py) against
it in a child process.  The untouched copy must pass them all; every mutant
must fail at least one.  All of it runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "csgv_oracle.c")

# (name, [(text in the oracle, planted replacement), ...]); every text must occur in the source
MUTANTS = [
    # R11: leftover units to the higher of two tied symbols
    ("normalize_tie_to_higher_symbol", [("counts[s] > counts[best]", "counts[s] >= counts[best]")]),
    # R11: the 64-bit product that overflows for large counts
    ("normalize_64bit_product", [("(unsigned __int128)counts[s]", "(uint64_t)counts[s]")]),
    # R12: the prepass samples ids 1, 1 + s, 1 + 2s, ... instead of 0, s, 2s, ...
    ("prepass_sampling_offset", [("J.stride = stride ? stride : 1;", "J.stride = stride ? stride : 1; J.next = (phase == 0);")]),
    # Sec. 3.1: a mode tie goes to the last occurrence in the child array
    ("pyramid_tie_to_last_occurrence", [("if (cnt > best_cnt)", "if (cnt >= best_cnt)")]),
    # R4: the +axis neighbour read on the same level (not yet decoded) instead of its parent
    ("plus_neighbour_same_level", [("if (bit == 0) {", "if (1) {")]),
    # R1: P_delta indexed as in Alg. 1 (palette[i_p - delta]), in encoder and decoder alike
    ("pdelta_alg1_index", [("ip >= 1 + d && palette[ip - 1 - d] == v", "ip >= d && palette[ip - d] == v"),
                           ("ip < 1 + d", "ip < d"), ("v = palette[ip - 1 - d]", "v = palette[ip - d]")]),
    # Alg. 2: children of constant parents coded anyway (the stop skip dropped in the encoder)
    ("encoder_codes_constant_parents", [("if (C[pi]) continue;", "")]),
    # R9/R10: final states written high half first, in encoder and decoder alike
    ("state_high_half_first", [("words[2 * k] = (uint16_t)(x[k] & 0xFFFFu);", "words[2 * k + 1] = (uint16_t)(x[k] & 0xFFFFu);"),
                               ("words[2 * k + 1] = (uint16_t)(x[k] >> 16);", "words[2 * k] = (uint16_t)(x[k] >> 16);"),
                               ("(uint32_t)words[2 * k] | ((uint32_t)words[2 * k + 1] << 16)",
                                "(uint32_t)words[2 * k + 1] | ((uint32_t)words[2 * k] << 16)")]),
    # R10: renormalisation words in the order they were emitted (the decoder reading them the same way)
    ("words_in_emit_order", [("words[2 * K + j] = emit[ne - 1 - j];", "words[2 * K + j] = emit[j];")]),
    # R10: op j on state K-1 - j mod K, in encoder and decoder alike
    ("op_state_reversed", [("cl[c++] = j - t0;", "cl[c++] = K - 1 - (j - t0);"),
                           ("rans_decode_one(&x[k], freq, words, n_words, &pos, &op[k]);",
                            "rans_decode_one(&x[K - 1 - k], freq, words, n_words, &pos, &op[k]);"),
                           ("rans_decode_one(&x[k], freq, words, n_words, &pos, &dl[k]);",
                            "rans_decode_one(&x[K - 1 - k], freq, words, n_words, &pos, &dl[k]);")]),
    # R10: a delta coded right after its op instead of after the step's ops, in encoder and decoder alike
    ("delta_right_after_its_op", [
        ("for (uint32_t j = t0; j < t1; j++) { cs[c] = sym[op_at[j]]; cl[c++] = j - t0; }",
         "for (uint32_t j = t0; j < t1; j++) { cs[c] = sym[op_at[j]]; cl[c++] = j - t0;"
         " if ((sym[op_at[j]] & 7u) == OP_PD) { cs[c] = sym[op_at[j] + 1]; cl[c++] = j - t0; } }"),
        ("            if ((sym[op_at[j]] & 7u) == OP_PD) { cs[c]", "            if (0) { cs[c]"),
        ("if ((op[k] & 7u) == OP_PD) owed++;",
         "if ((op[k] & 7u) == OP_PD && rc == ORC_OK) { rc = rans_decode_one(&x[k], freq, words, n_words, &pos,"
         " &dl[k]); used++; }"),
        ("            if ((op[k] & 7u) == OP_PD) {\n                if (used >= n)",
         "            if (0) {\n                if (used >= n)")]),
]


def _build(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) >= 1, (name, old)
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", str(c), "-o", str(so)])
    return str(so)


def _run_pins(lib):
    env = dict(os.environ, CSGV_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle.py"), "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_unmodified_copy_passes_the_pins(tmp_path):
    rc, out = _run_pins(_build(tmp_path, "control", []))
    assert rc == 0, out


@pytest.mark.parametrize("name,edits", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, edits):
    rc, out = _run_pins(_build(tmp_path, name, edits))
    assert rc == 1, f"{name}: the pins did not fail (rc {rc})\n{out}"  # 1 = tests ran and one failed
