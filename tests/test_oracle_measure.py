"""Pins for the oracle's CHP measurement and its keyed randomness (no GPU).

- Philox4x64-10 against numpy.random.Philox (numpy increments its counter
  before each block, so counter c - 1 in numpy yields the block at c).
- Measurement against a brute-force state vector (<= 8 qubits): Born
  probability of every outcome is 1/2 for a probabilistic and 1 for a
  deterministic measurement (Sec. 2.5, Eq. 6), and every stabilizer row
  stabilizes the post-measurement state.
- Closed forms: Bell/GHZ correlations; the first outcome is the keyed coin.
- Invariants of the extended tableau after measurements.
- The deterministic product is order independent (stabilizers commute) and
  equals +-Z_q computed with an independent Pauli-product table.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import sv_helpers as SV
from workloads import circuits as C


@pytest.mark.parametrize("ctr,key", [((1, 0, 0, 0), (0, 0)), ((5, 7, 9, 11), (3, 0x51A7E)),
                                     ((2**63, 1, 2**40, 1), (2**64 - 1, 0xF4A3E)),
                                     ((123456789, 0, 0, 0), (42, 42))])
def test_philox_matches_numpy(ctr, key):
    c = np.array(ctr, np.uint64).copy()
    c[0] -= np.uint64(1)  # numpy pre-increments the 256-bit counter
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=c)
    want = bg.random_raw(4)
    got = O.philox4x64_10(ctr, key)
    assert np.array_equal(want.astype(np.uint64), got)


def test_coin_and_frame_word_definitions():
    for seed, shot, m in [(1, 0, 0), (7, 3, 1000), (2**40, 5, 2**33)]:
        blk = O.philox4x64_10((m, shot, 0, 0), (seed, 0x51A7E))
        assert O.coin(seed, shot, m) == int(blk[0]) & 1
    for seed, e, q, j in [(1, 0, 0, 0), (9, 17, 5, 6), (3, 2**20, 179_999, 15_624)]:
        blk = O.philox4x64_10((e, q, j >> 2, 1), (seed, 0xF4A3E))
        assert O.frame_word(seed, e, q, j) == int(blk[j & 3])
    # the coin is fair enough to be a coin
    bits = [O.coin(77, 0, m) for m in range(4000)]
    assert 1800 < sum(bits) < 2200


def _sv_check_circuit(circ, seed, shot=0):
    o = O.Oracle(circ.n)
    sv = SV.StateVector(circ.n)
    for op in circ.ops:
        if op[0] == "layers":
            g = circ.gates[circ.layer_ptr[op[1]]:circ.layer_ptr[op[2]]]
            o.apply(g)
            sv.apply(g)
        else:
            outs, kinds = o.measure(op[1], seed, shot)
            for q, m, k in zip(op[1], outs, kinds):
                p = sv.prob(int(q), int(m))
                if k:
                    assert abs(p - 0.5) < 1e-9, (q, m, p)
                else:
                    assert abs(p - 1.0) < 1e-9, (q, m, p)
                sv.project(int(q), int(m))
        x, z, r = o.get()
        n = circ.n
        for i in range(n, 2 * n):
            assert sv.expect_stabilized(SV.pauli_matrix(x[i], z[i], r[i]))
    assert o.odd_phase_count == 0 and o.det_check_fail == 0
    return o


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (5, 4), (6, 5), (8, 6), (8, 7)])
def test_measurement_against_state_vector(n, seed):
    circ = C.gate_mix_circuit(n, 12, seed, measure_every=3, measure_frac=0.5)
    _sv_check_circuit(circ, seed=seed * 31)


def test_measurement_against_state_vector_hsc_generator():
    circ = C.random_circuit(7, 20, 0.5, seed=8, measure_every=4, measure_frac=0.4)
    _sv_check_circuit(circ, seed=3)


def test_bell_and_ghz_closed_forms():
    for n in (2, 5, 17):
        for seed in range(6):
            o = O.Oracle(n)
            o.gate(C.H, 0)
            for i in range(1, n):
                o.gate(C.CX, 0, i)
            out, kind = o.measure(np.arange(n), seed=seed, shot=seed + 1)
            assert kind[0] == 1 and not kind[1:].any()
            assert out[0] == O.coin(seed, seed + 1, 0)
            assert (out == out[0]).all()


def test_force_zero_reference_record():
    o = O.Oracle(4)
    o.gate(C.H, 0); o.gate(C.CX, 0, 1); o.gate(C.H, 2); o.gate(C.X, 3)
    out, kind = o.measure([0, 1, 2, 3], seed=5, force_zero=True)
    assert list(kind) == [1, 0, 1, 0]
    assert list(out) == [0, 0, 0, 1]


def test_invariants_after_measurements():
    n = 30
    circ = C.random_circuit(n, 40, 0.5, seed=9, measure_every=5, measure_frac=0.3)
    o, rec, kinds = O.run_circuit(circ, seed=4)
    x, z, r = o.get()
    xi, zi = x.astype(int), z.astype(int)
    gram = (xi @ zi.T + zi @ xi.T) % 2
    want = np.zeros((2 * n, 2 * n), int)
    want[:n, n:] = np.eye(n, dtype=int)
    want[n:, :n] = np.eye(n, dtype=int)
    assert np.array_equal(gram, want)
    # after measuring every qubit the stabilizer group is generated by
    # {(-1)^m_q Z_q}: every generator has x = 0 and its sign is the XOR of
    # the outcomes on its Z support; the generators have full rank
    last = rec[-n:]
    for i in range(n, 2 * n):
        assert not x[i].any()
        assert r[i] == (int(np.dot(z[i].astype(int), last.astype(int))) & 1)
    assert np.linalg.matrix_rank(z[n:].astype(float)) == n
    assert o.odd_phase_count == 0 and o.det_check_fail == 0


def test_deterministic_product_order_independent():
    """(-1)^m Z_q = prod over A of S_i in any order (Sec. 2.5 deterministic
    case); checked with an independent Pauli product table."""
    rng = np.random.default_rng(0)
    n = 12
    circ = C.random_circuit(n, 25, 0.5, seed=13, final_measure_all=False)
    o = O.Oracle(n)
    o.apply(circ.gates)
    o.measure(np.arange(n // 2), seed=1)
    checked = 0
    for q in range(n):
        x, z, r = o.get()
        if x[n:, q].any():
            continue
        A = np.nonzero(x[:n, q])[0]
        for trial in range(3):
            order = rng.permutation(A)
            px, pz, ph = np.zeros(n, np.uint8), np.zeros(n, np.uint8), 0
            for i in order:
                px, pz, ph2 = SV.pauli_product(x[n + i], z[n + i], r[n + i], px, pz, 0)
                ph = (ph + ph2) % 4
            assert not px.any() and pz.sum() == 1 and pz[q] == 1
            assert ph in (0, 2)
            want = ph // 2
            o2 = O.Oracle(n)
            o2.set(x, z, r)
            got, kind = o2.measure([q], seed=0)
            assert kind[0] == 0 and got[0] == want
            checked += 1
    assert checked > 0


def test_rowsum_against_pauli_product_table():
    """Every row the probabilistic update rewrites equals S_p * row (with sign)
    computed by an independent 2x2 Pauli multiplication table (the rowsum of
    Aaronson & Gottesman cited in Sec. 2.5); D_{p-n} = S_p; S_p = +-Z_q."""
    checked = 0
    for trial in range(120):
        n = 3 + trial % 5
        circ = C.gate_mix_circuit(n, 8 + trial % 7, 1000 + trial, final_measure_all=False)
        o = O.Oracle(n)
        o.apply(circ.gates)
        x, z, r = o.get()
        for q in range(n):
            if not x[n:, q].any():
                continue
            p = n + int(np.argmax(x[n:, q]))
            o2 = O.Oracle(n)
            o2.set(x, z, r)
            out, kind = o2.measure([q], seed=trial, shot=q)
            assert kind[0] == 1
            x2, z2, r2 = o2.get()
            for h in range(2 * n):
                if h in (p, p - n):
                    continue
                if x[h, q]:
                    ex, ez, ph = SV.pauli_product(x[p], z[p], r[p], x[h], z[h], r[h])
                    assert ph in (0, 2)
                    assert np.array_equal(x2[h], ex) and np.array_equal(z2[h], ez)
                    assert r2[h] == ph // 2
                    checked += 1
                else:
                    assert np.array_equal(x2[h], x[h]) and r2[h] == r[h]
            assert np.array_equal(x2[p - n], x[p]) and r2[p - n] == r[p]
            assert not x2[p].any() and z2[p].sum() == 1 and z2[p, q] == 1 and r2[p] == out[0]
            break
    assert checked > 150


@pytest.mark.parametrize("seed", range(20))
def test_measurement_against_state_vector_many_seeds(seed):
    n = 2 + seed % 7
    circ = C.gate_mix_circuit(n, 14, 500 + seed, measure_every=3, measure_frac=0.6)
    _sv_check_circuit(circ, seed=seed)
