"""Pins for the oracle's inverse-tableau mode (no GPU): the representation and
measurement of the paper's variant (Sec. 3.2, Alg. 1).

- Gate rules: after any circuit over the 11-gate set on <= 3 qubits, the
  images the mode keeps equal U^dag Z_q U and U^dag X_q U, signs included,
  with U the circuit's unitary built from textbook matrices.
- Bits: under gates alone they equal the forward tableau's bits (the images
  are the extended tableau read by columns).
- Measurement: Alg. 1 yields the same records and measurement kinds as CHP
  under the same keyed coins, and the same post-measurement state: every
  stabilizer of the CHP oracle (itself pinned by a state vector) is mapped by
  the inverse tableau to a Z-string with sign +, i.e. stabilizes C|0...0>.
- initstate: |1> on qubit i is measured as 1, deterministically.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import sv_helpers as SV
from workloads import circuits as C


def _unitary(n, gates):
    """Circuit unitary, column k = the circuit applied to basis state k."""
    dim = 2 ** n
    U = np.zeros((dim, dim), complex)
    for k in range(dim):
        sv = SV.StateVector(n)
        sv.psi[:] = 0
        sv.psi[k] = 1
        sv.apply(gates)
        U[:, k] = sv.psi
    return U


def _images(inv, q):
    """(x, z, sign) of the images of Z_q and X_q over the input qubits."""
    x, z, ss, sd = inv.get()
    n = inv.n
    zim = (x[n:, q].copy(), x[:n, q].copy(), int(ss[q]))
    xim = (z[n:, q].copy(), z[:n, q].copy(), int(sd[q]))
    return zim, xim


def _random_gates(n, count, rng):
    out = []
    for _ in range(count):
        if n >= 2 and rng.random() < 0.5:
            t = int(rng.choice(C.TWO_QUBIT))
            a, b = rng.choice(n, size=2, replace=False)
            out.append([t, int(a), int(b)])
        else:
            t = int(rng.choice([C.X, C.Y, C.Z, C.H, C.S, C.SDG]))
            out.append([t, int(rng.integers(n)), 0])
    return np.array(out, np.uint32).reshape(-1, 3)


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (2, 3), (3, 4), (3, 5), (3, 6)])
def test_images_match_unitary_conjugation(n, seed):
    rng = np.random.default_rng(seed)
    for trial in range(12):
        gates = _random_gates(n, 1 + trial, rng)
        inv = O.InverseOracle(n)
        inv.apply(gates)
        U = _unitary(n, gates)
        for q in range(n):
            e = np.zeros(n, np.uint8)
            e[q] = 1
            zero = np.zeros(n, np.uint8)
            zim, xim = _images(inv, q)
            want_z = U.conj().T @ SV.pauli_matrix(zero, e, 0) @ U
            want_x = U.conj().T @ SV.pauli_matrix(e, zero, 0) @ U
            assert np.allclose(want_z, SV.pauli_matrix(*zim)), (gates.tolist(), q, "Z image")
            assert np.allclose(want_x, SV.pauli_matrix(*xim)), (gates.tolist(), q, "X image")
        assert inv.odd_count == 0


@pytest.mark.parametrize("gate", [C.X, C.Y, C.Z, C.H, C.S, C.SDG, C.CX, C.CY, C.CZ, C.SWAP,
                                  C.ISWAP])
def test_each_gate_alone_matches_unitary(gate):
    """Every gate type after a scrambling prefix, both qubit orders."""
    rng = np.random.default_rng(int(gate) + 100)
    for order in ((0, 1), (1, 0)):
        prefix = _random_gates(2, 6, rng)
        g = np.array([[gate, order[0], order[1] if gate in C.TWO_QUBIT else 0]], np.uint32)
        gates = np.concatenate([prefix, g])
        inv = O.InverseOracle(2)
        inv.apply(gates)
        U = _unitary(2, gates)
        for q in range(2):
            e = np.zeros(2, np.uint8)
            e[q] = 1
            zero = np.zeros(2, np.uint8)
            zim, xim = _images(inv, q)
            assert np.allclose(U.conj().T @ SV.pauli_matrix(zero, e, 0) @ U, SV.pauli_matrix(*zim))
            assert np.allclose(U.conj().T @ SV.pauli_matrix(e, zero, 0) @ U, SV.pauli_matrix(*xim))


@pytest.mark.parametrize("n", [1, 7, 64, 130])
def test_bits_equal_forward_tableau_under_gates(n):
    circ = C.gate_mix_circuit(n, 15, seed=n + 3, final_measure_all=False)
    inv = O.InverseOracle(n)
    inv.apply(circ.gates)
    fwd = O.Oracle(n)
    fwd.apply(circ.gates)
    x, z, _, _ = inv.get()
    fx, fz, _ = fwd.get()
    assert np.array_equal(x, fx) and np.array_equal(z, fz)


def _chp_stabilizer_maps_to_plus_z(inv, sx, sz, sr):
    """C^dag S C from the inverse tableau's images: S = (-1)^r prod_q
    sigma(x_q, z_q) with sigma(1,1) = Y = i X Z, so each Y factor contributes
    i * image(X_q) * image(Z_q). True iff the result is +(a Z-string)."""
    n = inv.n
    acc_x = np.zeros(n, np.uint8)
    acc_z = np.zeros(n, np.uint8)
    phase = 2 * int(sr)  # power of i
    for q in range(n):
        if not (sx[q] or sz[q]):
            continue
        zim, xim = _images(inv, q)
        if sx[q]:
            acc_x, acc_z, ph = SV.pauli_product(acc_x, acc_z, 0, xim[0], xim[1], xim[2])
            phase += ph
        if sz[q]:
            acc_x, acc_z, ph = SV.pauli_product(acc_x, acc_z, 0, zim[0], zim[1], zim[2])
            phase += ph
        if sx[q] and sz[q]:
            phase += 1  # Y = i X Z
    return not acc_x.any() and phase % 4 == 0


@pytest.mark.parametrize("n,seed", [(1, 1), (3, 2), (6, 3), (12, 4), (40, 5), (300, 6)])
def test_records_and_state_equal_chp(n, seed):
    circ = C.gate_mix_circuit(n, 18, seed=seed, measure_every=3, measure_frac=0.5)
    fwd, rec, kinds = O.run_circuit(circ, seed=seed * 7, shot=seed)
    inv, irec, ikinds = O.run_circuit_inverse(circ, seed=seed * 7, shot=seed)
    assert np.array_equal(rec, irec), "records differ from CHP"
    assert np.array_equal(kinds, ikinds), "kinds differ from CHP"
    assert 0 < kinds.sum() or n == 1
    assert inv.odd_count == 0
    if n <= 40:
        fx, fz, fr = fwd.get()
        for i in range(n, 2 * n):  # CHP's stabilizers (pinned by state vectors)
            assert _chp_stabilizer_maps_to_plus_z(inv, fx[i], fz[i], fr[i]), i


def test_state_vector_measurement_distribution():
    """Born probabilities along Alg. 1's run: 1/2 for probabilistic and 1 for
    deterministic outcomes, projecting a state vector with each outcome."""
    for seed in range(6):
        circ = C.gate_mix_circuit(5, 10, seed=seed + 40, measure_every=2, measure_frac=0.6)
        inv = O.InverseOracle(5)
        sv = SV.StateVector(5)
        for op in circ.ops:
            if op[0] == "layers":
                g = circ.gates[circ.layer_ptr[op[1]]:circ.layer_ptr[op[2]]]
                inv.apply(g)
                sv.apply(g)
            else:
                outs, kinds = inv.measure(op[1], seed=seed)
                for q, m, k in zip(op[1], outs, kinds):
                    p = sv.project(int(q), int(m))
                    assert abs(p - (0.5 if k else 1.0)) < 1e-9, (seed, q, m, k, p)


def test_initstate_is_measured_deterministically():
    n = 9
    init = (np.arange(n) % 2).astype(np.uint8)
    inv = O.InverseOracle(n, init)
    out, kinds = inv.measure(np.arange(n), seed=3)
    assert np.array_equal(out, init) and not kinds.any()
    fwd = O.Oracle(n, init)
    fx, fz, fr = fwd.get()
    for i in range(n, 2 * n):
        assert _chp_stabilizer_maps_to_plus_z(inv, fx[i], fz[i], fr[i])


def _embed1(M, q, n):
    return SV.kron_list([M if j == q else SV.I2 for j in reversed(range(n))])


HYZ = (SV.PY + SV.PZ) / np.sqrt(2)  # maps Y <-> Z and X -> -X under conjugation


def _assert_images_match(inv, U):
    n = inv.n
    for q in range(n):
        e = np.zeros(n, np.uint8)
        e[q] = 1
        zero = np.zeros(n, np.uint8)
        zim, xim = _images(inv, q)
        assert np.allclose(U.conj().T @ SV.pauli_matrix(zero, e, 0) @ U, SV.pauli_matrix(*zim)), q
        assert np.allclose(U.conj().T @ SV.pauli_matrix(e, zero, 0) @ U, SV.pauli_matrix(*xim)), q


@pytest.mark.parametrize("n,seed", [(1, 3), (2, 4), (3, 5), (4, 6), (4, 7)])
def test_measurement_is_right_multiplication_by_injected_gates(n, seed):
    """Alg. 1 inserts gates at the start of the circuit (on the inputs, where
    CX(p, t) fixes |0...0>): C -> C * prod_t CX(p, t) * G_p [* X_p], G = H_YZ
    when the pivot's destabilizer part has a z at q after the CX injections,
    else H. Tracking that unitary exactly (with the pivot and targets read from
    the bits) must reproduce every image and sign the oracle keeps, including
    the X images' signs that a state comparison cannot see."""
    rng = np.random.default_rng(seed)
    for trial in range(6):
        gates = _random_gates(n, 4 + 2 * trial, rng)
        inv = O.InverseOracle(n)
        inv.apply(gates)
        U = _unitary(n, gates)
        for step in range(2 * n + 1):
            q = int(rng.integers(n))
            x, z, ss, sd = inv.get()
            piv = [i for i in range(n) if x[n + i, q]]
            out, kind = inv.measure([q], seed=seed * 100 + trial, shot=step)
            if piv:
                p = piv[0]
                xd_pq = int(x[p, q])
                for t in piv[1:]:
                    U = U @ _unitary(n, np.array([[C.CX, p, t]], np.uint32))
                    xd_pq ^= int(x[t, q])  # the pivot's destabilizer x row gains target rows
                U = U @ _embed1(HYZ if xd_pq else SV.HM, p, n)
                coin = O.coin(seed * 100 + trial, step, inv.midx - 1)
                e = np.zeros(n, np.uint8)
                e[q] = 1
                # U^dag Z_q U is now +-(a Z-string): its sign is <0|U^dag Z_q U|0>;
                # X_p flips it when it differs from the coin
                zq = U.conj().T @ SV.pauli_matrix(np.zeros(n, np.uint8), e, 0) @ U
                assert abs(abs(zq[0, 0].real) - 1) < 1e-9
                if int(zq[0, 0].real < 0) != coin:
                    U = U @ _embed1(SV.PX, p, n)
                assert out[0] == coin and kind[0] == 1
            else:
                assert kind[0] == 0
            _assert_images_match(inv, U)
            if rng.random() < 0.5:
                g = _random_gates(n, 2, rng)
                inv.apply(g)
                U = _unitary(n, g) @ U
