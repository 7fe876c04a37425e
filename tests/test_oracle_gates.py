"""Pins for the oracle's tableau encoding and gate rules (no GPU).

Each gate rule is checked against brute-force conjugation U P U^dag of every
signed Pauli by the gate's unitary (textbook matrices), which fixes the rules
of Sec. 2.4 Eq. 4 and the rest of the 11-gate set of Sec. 6 uniquely.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests import sv_helpers as SV
from workloads import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_bits(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        toks = line.split()
        rows.append([int(t) for t in toks[:7]])
    return np.array(rows, np.uint8)


def _row_matrices(x, z, r):
    return [SV.pauli_matrix(x[i], z[i], r[i]) for i in range(len(r))]


def _all_signed_paulis(nq):
    for bits in itertools.product([0, 1], repeat=2 * nq + 1):
        yield np.array(bits[:nq], np.uint8), np.array(bits[nq:2 * nq], np.uint8), bits[-1]


@pytest.mark.parametrize("gate", [C.X, C.Y, C.Z, C.H, C.S, C.SDG])
def test_one_qubit_rules_match_conjugation(gate):
    # n = 2 oracle, gate on qubit 1; the 2n = 4 rows are loaded with arbitrary
    # signed Paulis (the rules act row by row, Sec. 2.4).
    paulis = list(_all_signed_paulis(2))
    for k in range(0, len(paulis), 4):
        batch = paulis[k:k + 4]
        x = np.stack([p[0] for p in batch]); z = np.stack([p[1] for p in batch])
        r = np.array([p[2] for p in batch], np.uint8)
        o = O.Oracle(2)
        o.set(x, z, r)
        o.gate(gate, 1)
        x2, z2, r2 = o.get()
        U = np.kron(SV.ONE_Q[gate], SV.I2)  # qubit 1 = high bit
        for i in range(4):
            want = U @ SV.pauli_matrix(x[i], z[i], r[i]) @ U.conj().T
            got = SV.pauli_matrix(x2[i], z2[i], r2[i])
            assert np.allclose(want, got), (C.GATE_NAMES[gate], SV.pauli_string(x[i], z[i], r[i]))


@pytest.mark.parametrize("gate", [C.CX, C.CY, C.CZ, C.SWAP, C.ISWAP])
@pytest.mark.parametrize("a,b", [(0, 1), (1, 0)])
def test_two_qubit_rules_match_conjugation(gate, a, b):
    paulis = list(_all_signed_paulis(2))
    U2 = SV.two_qubit_unitary(gate)  # acts on (a = low bit, b = high bit)
    if (a, b) == (1, 0):  # relabel: gate's first qubit is the high bit
        P = SV.two_qubit_unitary(C.SWAP)
        U2 = P @ U2 @ P
    for k in range(0, len(paulis), 4):
        batch = paulis[k:k + 4]
        x = np.stack([p[0] for p in batch]); z = np.stack([p[1] for p in batch])
        r = np.array([p[2] for p in batch], np.uint8)
        o = O.Oracle(2)
        o.set(x, z, r)
        o.gate(gate, a, b)
        x2, z2, r2 = o.get()
        for i in range(4):
            want = U2 @ SV.pauli_matrix(x[i], z[i], r[i]) @ U2.conj().T
            got = SV.pauli_matrix(x2[i], z2[i], r2[i])
            assert np.allclose(want, got), (C.GATE_NAMES[gate], a, b,
                                             SV.pauli_string(x[i], z[i], r[i]))


def test_eq3_encoding_example():
    """Sec. 2.4 Eq. 3: the encoding (x,z)=(1,1) -> Y, sign (-1)^s; pins the
    decoding helper used by the state-vector pins below."""
    bits = _load_bits("eq3_tableau_example.txt")
    got = [SV.pauli_string(b[0:3], b[3:6], b[6]) for b in bits]
    assert got == ["+ZII", "-YZI", "-IXY"]


def test_eq8_plus01_initial_tableau():
    """Sec. 2.5 Eq. 8: init with initstate 001, then H on qubit 1 -> |+01>."""
    want = _load_bits("eq8_plus01_tableau.txt")
    o = O.Oracle(3)
    o.reset(np.array([0, 0, 1], np.uint8))
    o.gate(C.H, 0)
    x, z, r = o.get()
    got = np.concatenate([x, z, r[:, None]], axis=1)
    assert np.array_equal(got, want)


def test_example1_h1_p3():
    """Sec. 2.4 Example 1 (stabilizer rows only)."""
    want = _load_bits("example1_h1_p3.txt")
    o = O.Oracle(3)
    o.gate(C.H, 0)
    x, z, r = o.get()
    assert np.array_equal(np.concatenate([x, z, r[:, None]], axis=1)[3:], want[0:3])
    o.gate(C.S, 2)
    x, z, r = o.get()
    assert np.array_equal(np.concatenate([x, z, r[:, None]], axis=1)[3:], want[3:6])


def _random_tableau_state(n, seed):
    o = O.Oracle(n)
    c = C.gate_mix_circuit(n, 6, seed, final_measure_all=False)
    o.apply(c.gates)
    return o


@pytest.mark.parametrize("gate,times,two", [(C.H, 2, False), (C.S, 4, False), (C.SDG, 4, False),
                                            (C.X, 2, False), (C.CX, 2, True), (C.CZ, 2, True),
                                            (C.SWAP, 2, True), (C.ISWAP, 4, True)])
def test_gate_orders(gate, times, two):
    """Closed forms: H^2 = S^4 = CX^2 = I (and the other gates' orders)."""
    o = _random_tableau_state(7, 5)
    before = o.get()
    for _ in range(times):
        o.gate(gate, 3, 5) if two else o.gate(gate, 3)
    after = o.get()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_s_squared_is_z():
    """S^2 = Z: flips exactly the signs of rows with x_q = 1."""
    o = _random_tableau_state(9, 6)
    x, z, r = o.get()
    o.gate(C.S, 4); o.gate(C.S, 4)
    x2, z2, r2 = o.get()
    assert np.array_equal(x, x2) and np.array_equal(z, z2)
    assert np.array_equal(r2, r ^ x[:, 4])


_INV = {C.X: C.X, C.Y: C.Y, C.Z: C.Z, C.H: C.H, C.S: C.SDG, C.SDG: C.S, C.CX: C.CX,
        C.CY: C.CY, C.CZ: C.CZ, C.SWAP: C.SWAP}


def test_circuit_then_inverse_is_identity():
    """U then U^-1 returns the initial tableau exactly (signs included)."""
    n = 40
    c = C.gate_mix_circuit(n, 30, 12, final_measure_all=False)
    g = c.gates[c.gates[:, 0] != C.ISWAP]
    inv = np.array([[_INV[int(t)], a, b] for t, a, b in g[::-1]], np.uint32)
    o = O.Oracle(n)
    ref = o.get()
    o.apply(g)
    mid = o.get()
    assert not np.array_equal(mid[0], ref[0])
    o.apply(inv)
    for a, b in zip(ref, o.get()):
        assert np.array_equal(a, b)


def test_symplectic_invariants_after_gates():
    """Stabilizers commute pairwise, destabilizers commute pairwise and
    D_i anticommutes with S_j iff i = j (Sec. 2.5)."""
    n = 24
    o = _random_tableau_state(n, 21)
    x, z, _ = o.get()
    xi, zi = x.astype(int), z.astype(int)
    gram = (xi @ zi.T + zi @ xi.T) % 2
    want = np.zeros((2 * n, 2 * n), int)
    want[:n, n:] = np.eye(n, dtype=int)
    want[n:, :n] = np.eye(n, dtype=int)
    assert np.array_equal(gram, want)
