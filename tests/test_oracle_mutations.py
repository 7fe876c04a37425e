"""The oracle's pins catch plausible mistakes (no GPU).

(Multiplying the rowsum operands in the other order is not a mistake: the
rows it multiplies commute, so that mutant is equivalent and not listed.)

Each case compiles a copy of oracle/chp_oracle.c with one planted mistake --
a dropped term, a wrong sign, a transposed operand, the wrong rows -- loads it
in place of the oracle and checks that at least one pin of
tests/test_oracle_*.py now fails. The oracle's own source is not touched.
"""
import os
import subprocess
import tempfile

import pytest

from oracle import oracle as O
from tests import test_oracle_frames as TF
from tests import test_oracle_gates as TG
from tests import test_oracle_inverse as TI
from tests import test_oracle_measure as TM
from tests import test_oracle_noise as TN
from tests import test_oracle_subset as TSUB
from workloads import circuits as C

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "chp_oracle.c")


def _pins_gates():
    for g in (C.X, C.Y, C.Z, C.H, C.S, C.SDG):
        TG.test_one_qubit_rules_match_conjugation(g)
    for g in (C.CX, C.CY, C.CZ, C.SWAP, C.ISWAP):
        TG.test_two_qubit_rules_match_conjugation(g, 0, 1)
        TG.test_two_qubit_rules_match_conjugation(g, 1, 0)


def _pins_golden():
    TG.test_eq3_encoding_example()
    TG.test_eq8_plus01_initial_tableau()
    TG.test_example1_h1_p3()


def _pins_measure():
    TM.test_rowsum_against_pauli_product_table()
    for n, seed in [(3, 3), (5, 4), (8, 6)]:
        TM.test_measurement_against_state_vector(n, seed)
    TM.test_bell_and_ghz_closed_forms()
    TM.test_invariants_after_measurements()
    TM.test_deterministic_product_order_independent()


def _pins_philox():
    TM.test_philox_matches_numpy((5, 7, 9, 11), (3, 0x51A7E))
    TM.test_coin_and_frame_word_definitions()


def _pins_frames():
    TF.test_frames_support_and_distribution(5, 2, 3, 0.4)
    TF.test_frames_support_and_distribution(6, 3, 4, 0.5)
    TF.test_frames_reference_is_deterministic_part()


def _pins_subset():
    TSUB.test_row_subset_of_the_initial_state()
    for n, layers, seed, nrows in [(7, 30, 1, 14), (64, 25, 2, 40)]:
        TSUB.test_row_subset_equals_full_oracle_rows(n, layers, seed, nrows)


def _pins_inverse():
    for n, seed in [(1, 1), (2, 2), (3, 4)]:
        TI.test_images_match_unitary_conjugation(n, seed)
    for g in (C.X, C.Y, C.Z, C.H, C.S, C.SDG, C.CX, C.CY, C.CZ, C.SWAP, C.ISWAP):
        TI.test_each_gate_alone_matches_unitary(g)
    for n, seed in [(3, 2), (6, 3), (12, 4), (40, 5)]:
        TI.test_records_and_state_equal_chp(n, seed)
    for n, seed in [(2, 4), (3, 5), (4, 6)]:
        TI.test_measurement_is_right_multiplication_by_injected_gates(n, seed)
    TI.test_state_vector_measurement_distribution()
    TI.test_initstate_is_measured_deterministically()


def _pins_noise():
    for seed in (1, 2, 3):
        TN.test_noisy_frames_match_exact_distribution(seed)
    for kind, flip in [(C.NOISE_X, 1), (C.NOISE_Y, 1), (C.NOISE_Z, 0)]:
        TN.test_certain_errors_on_z_eigenstate(kind, flip)
    TN.test_certain_errors_propagate_through_h_and_cx()
    TN.test_flip_rates()


MUTATIONS = [
    ("CX sign drops the negation",
     "t->r[i] ^= (uint8_t)(xc & zt & ((xt ^ zc) ^ 1u));",
     "t->r[i] ^= (uint8_t)(xc & zt & (xt ^ zc));", _pins_gates),
    ("H forgets the sign",
     "  t->r[i] ^= (uint8_t)(x & z);\n  XB(t, i, q) = z;",
     "  XB(t, i, q) = z;", _pins_gates),
    ("CX updates the wrong z column",
     "ZB(t, i, c) = (uint8_t)(zc ^ zt);", "ZB(t, i, tq) = (uint8_t)(zt ^ zc);", _pins_gates),
    ("Pauli Z flips on z instead of x",
     "case G_Z: rule_pauli(t, i, a, 0, 1); break;", "case G_Z: rule_pauli(t, i, a, 1, 0); break;",
     _pins_gates),
    ("g function: wrong sign for X * .",
     "return z2 * (2 * x2 - 1); /* X * . */", "return z2 * (1 - 2 * x2); /* X * . */",
     _pins_measure),
    ("rowsum drops 2 r_i",
     "long sum = 2 * (long)t->r[h] + 2 * (long)t->r[i];", "long sum = 2 * (long)t->r[h];",
     _pins_measure),
    ("rowsum transposes x and z of the target",
     "sum += g_table[8 * XB(t, i, j) + 4 * ZB(t, i, j) + 2 * XB(t, h, j) + ZB(t, h, j)];",
     "sum += g_table[8 * XB(t, i, j) + 4 * ZB(t, i, j) + 2 * ZB(t, h, j) + XB(t, h, j)];", _pins_measure),
    ("deterministic product uses destabilizers",
     "if (XB(t, i, q)) rowsum(t, s, i + n);", "if (XB(t, i, q)) rowsum(t, s, i);", _pins_measure),
    ("pivot searched among destabilizers",
     "for (int i = n; i < 2 * n; ++i)\n    if (XB(t, i, q)) { p = i; break; }",
     "for (int i = 0; i < n; ++i)\n    if (XB(t, i, q)) { p = i + n; break; }", _pins_measure),
    ("D_{p-n} not replaced by S_p",
     "memcpy(&XB(t, p - n, 0), &XB(t, p, 0), (size_t)n);", ";", _pins_measure),
    ("Philox Weyl constant wrong",
     "k0 += 0x9E3779B97F4A7C15ull;", "k0 += 0x9E3779B97F4A7C16ull;", _pins_philox),
    ("coin reads word 1",
     "return (int)(out[0] & 1u);", "return (int)(out[1] & 1u);", _pins_philox),
    ("frames forget the re-randomisation after a measurement",
     "fz[q] = (uint8_t)((oracle_frame_word(seed, (uint64_t)m + 1, (uint64_t)q, j) >> bit) & 1u);",
     ";", _pins_frames),
    ("frames drop the reference record",
     "(uint8_t)(fx[q] ^ ref[m]);", "(uint8_t)(fx[q]);", _pins_frames),
    ("noise fires above the threshold",
     "int fire = u < thr;", "int fire = u > thr;", _pins_noise),
    ("Y error flips only z",
     "if (code == 1 || code == 2) fx[q] ^= 1u;", "if (code == 1) fx[q] ^= 1u;", _pins_noise),
    ("DEPOLARIZE1 can pick the identity",
     "case N_DEP1: frame_pauli(fx, fz, (int)t[i], 1 + (int)mul_hi(v, 3)); break;",
     "case N_DEP1: frame_pauli(fx, fz, (int)t[i], (int)mul_hi(v, 4)); break;", _pins_noise),
    ("DEPOLARIZE2 applies the same Pauli to both qubits",
     "frame_pauli(fx, fz, (int)t[2 * i + 1], idx & 3);",
     "frame_pauli(fx, fz, (int)t[2 * i + 1], idx >> 2);", _pins_noise),
    ("noise ops share one random stream",
     "noise_p[o], qubits + op_a[o], op_b[o] - op_a[o], e++, seed,",
     "noise_p[o], qubits + op_a[o], op_b[o] - op_a[o], 0, seed,", _pins_noise),
    ("initstate sets only the stabilizer sign",
     "if (initstate && initstate[i]) { t->r[i] = 1; t->r[n + i] = 1; }",
     "if (initstate && initstate[i]) { t->r[n + i] = 1; }", _pins_golden),
    ("S dagger applied as S",
     "case G_SDG: rule_p(t, i, a); rule_p(t, i, a); rule_p(t, i, a); break;",
     "case G_SDG: rule_p(t, i, a); break;", _pins_gates),
    ("CY with S and S dagger swapped",
     "rule_p(t, i, b); rule_p(t, i, b); rule_p(t, i, b); rule_cx(t, i, a, b); rule_p(t, i, b); break;",
     "rule_p(t, i, b); rule_cx(t, i, a, b); rule_p(t, i, b); rule_p(t, i, b); rule_p(t, i, b); break;",
     _pins_gates),
    ("measurement rowsum skips the destabilizers",
     "for (int i = 0; i < 2 * n; ++i)\n      if (i != p && i != p - n && XB(t, i, q)) rowsum(t, i, p);",
     "for (int i = n; i < 2 * n; ++i)\n      if (i != p && i != p - n && XB(t, i, q)) rowsum(t, i, p);",
     _pins_measure),
    ("deterministic product over every stabilizer",
     "if (XB(t, i, q)) rowsum(t, s, i + n);", "rowsum(t, s, i + n);", _pins_measure),
    ("frames: S acts on x instead of z",
     "case G_S: case G_SDG: fz[a] ^= fx[a]; break;", "case G_S: case G_SDG: fx[a] ^= fz[a]; break;",
     _pins_frames),
    ("frames start without random Z",
     "fz[q] = (uint8_t)((oracle_frame_word(seed, 0, (uint64_t)q, j) >> bit) & 1u);",
     "fz[q] = 0;", _pins_frames),
    ("inverse: CX injection sign drops the negation",
     "s[j] ^= (uint8_t)(xc[j] & zt[j] & ((zc[j] ^ xt[j]) ^ 1u));",
     "s[j] ^= (uint8_t)(xc[j] & zt[j] & (zc[j] ^ xt[j]));", _pins_inverse),
    ("inverse: CX injection leaves the pivot's z row alone",
     "    xt[j] ^= xc[j];\n    zc[j] ^= zt[j];", "    xt[j] ^= xc[j];", _pins_inverse),
    ("inverse: swap case decided on the stabilizer bit",
     "  if (XDp[q]) {", "  if (XSp[q]) {", _pins_inverse),
    ("inverse: X injection flips ss by the z row",
     "inject_x(n, t->ss, XDp);", "inject_x(n, t->ss, ZDp);", _pins_inverse),
    ("inverse: S and S dagger signs swapped",
     "int f = (e + (dagger ? 1 : 3)) & 3;", "int f = (e + (dagger ? 3 : 1)) & 3;", _pins_inverse),
    ("inverse: CX forgets the control's Z sign",
     "t->ss[tq] = (uint8_t)(t->ss[tq] ^ t->ss[c] ^ (e2 >> 1));",
     "t->ss[tq] = (uint8_t)(t->ss[tq] ^ (e2 >> 1));", _pins_inverse),
    ("inverse: H keeps the signs in place",
     "  uint8_t s = t->ss[a];\n  t->ss[a] = t->sd[a];\n  t->sd[a] = s;\n", "", _pins_inverse),
    ("inverse: initstate signs the X image",
     "    t->ss[i] = (uint8_t)(initstate && initstate[i] ? 1 : 0);\n    t->sd[i] = 0;",
     "    t->sd[i] = (uint8_t)(initstate && initstate[i] ? 1 : 0);\n    t->ss[i] = 0;", _pins_inverse),
    ("inverse: deterministic outcome read from sd",
     "    t->last_kind = 0;\n    return t->ss[q];", "    t->last_kind = 0;\n    return t->sd[q];",
     _pins_inverse),
    ("inverse: H_YZ injection forgets the bit update",
     "    x[j] ^= z[j];\n  }\n}\n\nstatic void inject_had", "  }\n}\n\nstatic void inject_had",
     _pins_inverse),
    ("row subset seeds a stabilizer as X",
     "else ZB(t, j, g - (uint32_t)n) = 1;", "else XB(t, j, g - (uint32_t)n) = 1;", _pins_subset),
    ("row subset takes the stabilizer of the next qubit",
     "else ZB(t, j, g - (uint32_t)n) = 1;",
     "else ZB(t, j, (g - (uint32_t)n + 1u) % (uint32_t)n) = 1;", _pins_subset),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, old, new, pins):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    mutant = src.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "mutant.so")
        open(c, "w").write(mutant)
        subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", "-o", so, c])
        saved = O._lib
        O._lib = O.load_library(so)
        try:
            with pytest.raises(AssertionError):
                pins()
        finally:
            O._lib = saved


def test_unmutated_oracle_passes_the_same_pins():
    _pins_golden()
    _pins_gates()
    _pins_measure()
    _pins_philox()
    _pins_frames()
    _pins_noise()
    _pins_subset()
    _pins_inverse()
