"""Plants plausible mistakes in a copy of the oracle's C source (on the CPU,
in a temporary directory) and checks that the pins in test_oracle_pins.py
catch every one of them.  The committed oracle is never modified."""
import os
import subprocess

import pytest

from oracle import build as obuild
from oracle import oracle as O
from paper_2410_05934_gb300 import workloads as W
import test_oracle_pins as P

MUTANTS = {
    # output listed in natural order instead of bit-reversed order
    "natural_order": ("uint64_t odd = 2 * (uint64_t)oracle_bitrev(j, log2n) + 1;",
                      "uint64_t odd = 2 * (uint64_t)j + 1;"),
    # cyclic instead of negacyclic wrap-around (sign of x^N dropped)
    "cyclic_wrap": ("else       c[k - n] = oracle_submod(c[k - n], p, q);",
                    "else       c[k - n] = oracle_addmod(c[k - n], p, q);"),
    # N^-1 scaling dropped from the inverse
    "no_ninv": ("out[t] = oracle_mulmod(acc, n_inv, q);", "out[t] = acc;"),
    # inverse uses psi^(+e) instead of psi^(-e)
    "inverse_sign": ("uint64_t e = (two_n - (i * odd) % two_n) % two_n;",
                     "uint64_t e = (i * odd) % two_n;"),
    # a different (still valid) primitive root
    "other_root": ("uint64_t g = 2;\n    while", "uint64_t g = 13;\n    while"),
    # an N-th root of unity where a 2N-th one belongs
    "root_order_n": ("return oracle_powmod(g, (q - 1) / two_n, q);", "return oracle_powmod(g, (q - 1) / (two_n / 2), q);"),
    # Miller-Rabin with a single base
    "one_base": ("for (int i = 0; i < 12; i++) {\n        uint64_t x", "for (int i = 0; i < 1; i++) {\n        uint64_t x"),
    # transposed operand: a[j] used where a[i] belongs in the schoolbook product
    "schoolbook_index": ("uint64_t p = oracle_mulmod(a[i] % q, b[j] % q, q);",
                         "uint64_t p = oracle_mulmod(a[j] % q, b[j] % q, q);"),
}

PINS = [
    lambda O: P.test_miller_rabin_matches_trial_division(O),
    lambda O: P.test_output_order_is_cooley_tukey_bit_reversed(O, 7681, 8),
    lambda O: P.test_convolution_theorem_and_schoolbook_vs_numpy(O, 12289, 7),
    lambda O: P.test_roundtrip(O, W.Q59_N1024, 10),
    lambda O: P.test_psi_has_order_2n_and_uses_least_nonresidue(O, W.POOL50[0], 10),
    lambda O: P.test_negacyclic_sign(O, 257, 4),
]


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = open(obuild.SRCS[0]).read()          # ntt_oracle.c; the radix-2 file is linked unchanged
    d = tmp_path_factory.mktemp("mutants")
    libs = {}
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, name
        path = os.path.join(d, name + ".c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(d, name + ".so")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", so, path,
                               obuild.SRCS[1]])
        libs[name] = so
    return libs


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant_libs, name):
    pytest.importorskip("sympy")
    saved = O._lib
    O._lib = O.bind(mutant_libs[name])
    caught = []
    try:
        for i, pin in enumerate(PINS):
            try:
                pin(O)
            except AssertionError:
                caught.append(i)
    finally:
        O._lib = saved
    assert caught, "no pin caught mutant %s" % name
