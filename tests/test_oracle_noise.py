"""Pins for the oracle's Pauli noise channels on the frames (no GPU).

The paper notes that Pauli frames carry error events as well as measurement
randomness (Sec. 3) but fixes no channel set; the oracle implements X_ERROR,
Y_ERROR, Z_ERROR, DEPOLARIZE1 and DEPOLARIZE2 with the keyed draws stated in
its header. Pinned here against things other than its own formulas:

- the noisy sampler draws records from the exact distribution of the noisy
  circuit, computed with a brute-force density matrix (Kraus mixtures of
  Pauli matrices, projective measurements branching the record): support
  and chi-square;
- special cases: p = 0 reproduces the noiseless sampler bit for bit; p = 1
  X/Y/Z errors flip or keep a Z-basis outcome with certainty, and propagate
  through H and CX as the conjugation rules say;
- rates: the flip frequency of X_ERROR(p) and the single and joint flip
  frequencies of DEPOLARIZE1/2 (2/3, 8/15, 4/15 at p = 1) within 5 sigma;
- the threshold is floor(p * 2^32) at exactly representable p, and the
  draws come from the Philox stream pinned against numpy in
  test_oracle_measure.py.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from tests import sv_helpers as SV
from workloads import circuits as C

_PAULI = {0: SV.I2, 1: SV.PX, 2: SV.PY, 3: SV.PZ}


def _full(n, ops_on):
    """2^n x 2^n matrix of single-qubit matrices {qubit: 2x2}."""
    return SV.kron_list([ops_on.get(j, SV.I2) for j in reversed(range(n))])


def _gate_unitary(n, t, a, b):
    U = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for col in range(2 ** n):
        sv = SV.StateVector(n)
        sv.psi = np.zeros(2 ** n, dtype=complex)
        sv.psi[col] = 1.0
        sv.gate(t, a, b)
        U[:, col] = sv.psi
    return U


def _channel(kind, p, targets):
    """Kraus mixture [(prob, {qubit: 2x2 Pauli})] of one noise op."""
    if kind == C.DEPOLARIZE2:
        pairs = list(zip(targets[0::2], targets[1::2]))
        terms = [[(1.0, {})]]
        for a, b in pairs:
            t = [(1 - p, {})] + [(p / 15, {a: _PAULI[k >> 2], b: _PAULI[k & 3]})
                                 for k in range(1, 16)]
            terms.append(t)
    else:
        terms = []
        for q in targets:
            if kind == C.DEPOLARIZE1:
                t = [(1 - p, {})] + [(p / 3, {q: _PAULI[c]}) for c in (1, 2, 3)]
            else:
                c = {C.NOISE_X: 1, C.NOISE_Y: 2, C.NOISE_Z: 3}[kind]
                t = [(1 - p, {}), (p, {q: _PAULI[c]})]
            terms.append(t)
    out = []
    for combo in itertools.product(*terms):
        w = 1.0
        ops = {}
        for pr, d in combo:
            w *= pr
            ops.update(d)
        if w > 0:
            out.append((w, ops))
    return out


def exact_record_distribution(circ):
    """{record bytes: probability} of the noisy circuit by density matrix."""
    n = circ.n
    rho = np.zeros((2 ** n, 2 ** n), dtype=complex)
    rho[0, 0] = 1.0
    branches = {(): rho}
    idx = np.arange(2 ** n)
    for op in circ.ops:
        if op[0] == "layers":
            for t, a, b in circ.gates[circ.layer_ptr[op[1]]:circ.layer_ptr[op[2]]]:
                U = _gate_unitary(n, int(t), int(a), int(b))
                branches = {k: U @ r @ U.conj().T for k, r in branches.items()}
        elif op[0] == "noise":
            mix = [(w, _full(n, d)) for w, d in _channel(op[1], op[2], [int(q) for q in op[3]])]
            branches = {k: sum(w * (P @ r @ P.conj().T) for w, P in mix) for k, r in branches.items()}
        else:
            for q in op[1]:
                nb = {}
                for k, r in branches.items():
                    for m in (0, 1):
                        proj = np.diag((((idx >> int(q)) & 1) == m).astype(complex))
                        rm = proj @ r @ proj
                        if np.trace(rm).real > 1e-14:
                            nb[k + (m,)] = rm
                branches = nb
    return {bytes(np.array(k, np.uint8)): float(np.trace(r).real) for k, r in branches.items()}


def _noisy_small_circuit(seed):
    rng = np.random.default_rng(seed)
    base = C.gate_mix_circuit(4, 8, seed, measure_every=2, measure_frac=0.5)
    ops = []
    e = 0
    for op in base.ops:
        ops.append(op)
        if op[0] == "layers":
            kind = [C.DEPOLARIZE1, C.NOISE_X, C.DEPOLARIZE2, C.NOISE_Y, C.NOISE_Z][(e + seed) % 5]
            e += 1
            if kind == C.DEPOLARIZE2:
                t = rng.permutation(4)[:2].astype(np.uint32)
            else:
                t = np.unique(rng.integers(0, 4, size=2)).astype(np.uint32)
            ops.append(("noise", kind, float(rng.choice([0.1, 0.25, 0.5])), t))
    return C.Circuit(n=4, gates=base.gates, layer_ptr=base.layer_ptr, ops=ops)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_noisy_frames_match_exact_distribution(seed):
    circ = _noisy_small_circuit(seed)
    _, ref, _ = O.run_circuit(circ, seed=seed, force_zero=True)
    shots = 3000
    out = O.frames(circ, ref, shots, seed=seed + 50)
    exact = exact_record_distribution(circ)
    assert abs(sum(exact.values()) - 1.0) < 1e-9
    counts = {}
    for s in range(shots):
        k = out[:, s].tobytes()
        counts[k] = counts.get(k, 0) + 1
    for k in counts:
        assert exact.get(k, 0.0) > 1e-12, "sampled record outside the support"
    # chi-square over records with expected count >= 5, the rest pooled
    keys = [k for k, p in exact.items() if p * shots >= 5]
    obs = [counts.get(k, 0) for k in keys]
    exp = [exact[k] * shots for k in keys]
    rest_o = shots - sum(obs)
    rest_e = shots - sum(exp)
    if rest_e >= 5:
        obs.append(rest_o)
        exp.append(rest_e)
    obs, exp = np.array(obs, float), np.array(exp, float)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    dof = max(len(obs) - 1, 1)
    assert chi2 < dof + 6 * np.sqrt(2 * dof) + 10, (chi2, dof)


def test_zero_probability_is_the_noiseless_sampler():
    circ = C.random_circuit(12, 8, 0.5, seed=7, measure_every=3, measure_frac=0.4,
                            final_measure_all=True)
    _, ref, _ = O.run_circuit(circ, seed=2, force_zero=True)
    plain = O.frames(circ, ref, 200, seed=5)
    noisy = O.frames(C.with_circuit_noise(circ, 0.0, 0.0), ref, 200, seed=5)
    assert np.array_equal(plain, noisy)
    ops = list(circ.ops)
    ops.insert(1, ("noise", C.DEPOLARIZE1, 0.0, np.arange(12, dtype=np.uint32)))
    c2 = C.Circuit(n=12, gates=circ.gates, layer_ptr=circ.layer_ptr, ops=ops)
    assert np.array_equal(O.frames(c2, ref, 200, seed=5), plain)


def _one_qubit_program(pre, noise, post, n=2):
    g = list(pre) + list(post)
    ops = []
    if pre:
        ops.append(("layers", 0, 1))
    ops.append(noise)
    if post:
        ops.append(("layers", 1 if pre else 0, 2 if pre else 1))
    ops.append(("measure", np.arange(n, dtype=np.uint32)))
    ptr = [0]
    if pre:
        ptr.append(len(pre))
    if post:
        ptr.append(len(pre) + len(post))
    gates = np.array(g, np.uint32).reshape(-1, 3) if g else np.zeros((0, 3), np.uint32)
    return C.Circuit(n=n, gates=gates, layer_ptr=np.array(ptr), ops=ops)


@pytest.mark.parametrize("kind,flip", [(C.NOISE_X, 1), (C.NOISE_Y, 1), (C.NOISE_Z, 0)])
def test_certain_errors_on_z_eigenstate(kind, flip):
    circ = _one_qubit_program([], ("noise", kind, 1.0, np.array([0], np.uint32)), [])
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    out = O.frames(circ, ref, 130, seed=4)
    assert (out[0] == flip).all() and (out[1] == 0).all()


def test_certain_errors_propagate_through_h_and_cx():
    # Z error, then H: becomes X, flips the outcome
    circ = _one_qubit_program([], ("noise", C.NOISE_Z, 1.0, np.array([0], np.uint32)),
                              [[C.H, 0, 0]])
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    out = O.frames(circ, ref, 100, seed=2)
    # qubit 0 is in |+> up to the error: the outcome is random, but the error
    # shows against the same keyed frames without it
    clean = O.frames(_one_qubit_program([], ("noise", C.NOISE_Z, 0.0, np.array([0], np.uint32)),
                                        [[C.H, 0, 0]]), ref, 100, seed=2)
    assert (out[0] ^ clean[0] == 1).all()
    # X error on the control before CX flips control and target
    circ = _one_qubit_program([], ("noise", C.NOISE_X, 1.0, np.array([0], np.uint32)),
                              [[C.CX, 0, 1]])
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    out = O.frames(circ, ref, 100, seed=2)
    assert (out == 1).all()
    # Z error on the target before CX stays on the target and kicks back Z on
    # the control: a Z-basis record is unchanged
    circ = _one_qubit_program([], ("noise", C.NOISE_Z, 1.0, np.array([1], np.uint32)),
                              [[C.CX, 0, 1]])
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    assert (O.frames(circ, ref, 100, seed=2) == 0).all()


def _rate_ok(k, n, p):
    sd = np.sqrt(n * p * (1 - p))
    return abs(k - n * p) <= 5 * sd + 1


def test_flip_rates():
    shots = 6000
    for p in (0.05, 0.3):
        circ = _one_qubit_program([], ("noise", C.NOISE_X, p, np.array([0, 1], np.uint32)), [])
        _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
        out = O.frames(circ, ref, shots, seed=11)
        for q in (0, 1):
            assert _rate_ok(int(out[q].sum()), shots, p)
        # the two targets draw independently
        assert _rate_ok(int((out[0] & out[1]).sum()), shots, p * p)
    # DEPOLARIZE1(1): X or Y flips a Z-basis outcome (2/3); in the X basis Z or Y does
    circ = _one_qubit_program([], ("noise", C.DEPOLARIZE1, 1.0, np.array([0], np.uint32)), [])
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    out = O.frames(circ, ref, shots, seed=12)
    assert _rate_ok(int(out[0].sum()), shots, 2 / 3)
    hx = _one_qubit_program([[C.H, 0, 0]],
                            ("noise", C.DEPOLARIZE1, 1.0, np.array([0], np.uint32)), [[C.H, 0, 0]])
    clean = _one_qubit_program([[C.H, 0, 0]],
                               ("noise", C.DEPOLARIZE1, 0.0, np.array([0], np.uint32)), [[C.H, 0, 0]])
    _, ref, _ = O.run_circuit(hx, seed=1, force_zero=True)
    flips = O.frames(hx, ref, shots, seed=13)[0] ^ O.frames(clean, ref, shots, seed=13)[0]
    assert _rate_ok(int(flips.sum()), shots, 2 / 3)
    # DEPOLARIZE2(1) on a pair: each qubit flips in 8 of 15 cases, both in 4
    circ = _one_qubit_program([], ("noise", C.DEPOLARIZE2, 1.0, np.array([1, 0], np.uint32)), [])
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    out = O.frames(circ, ref, shots, seed=14)
    assert _rate_ok(int(out[0].sum()), shots, 8 / 15)
    assert _rate_ok(int(out[1].sum()), shots, 8 / 15)
    assert _rate_ok(int((out[0] & out[1]).sum()), shots, 4 / 15)


def test_threshold_and_draws():
    assert O.noise_threshold(0.25) == 2 ** 30
    assert O.noise_threshold(0.5) == 2 ** 31
    assert O.noise_threshold(1 - 2.0 ** -53) == 2 ** 32 - 1
    assert O.noise_threshold(1e-3) == 4294967  # floor(0.001 * 2^32)
    assert O.noise_threshold(0.0) == 0 and O.noise_threshold(-1.0) == 0
    assert O.noise_threshold(1.0) == 2 ** 32
    for seed, e, i, s in [(1, 0, 0, 0), (5, 3, 7, 31), (5, 3, 7, 32), (9, 2**20, 99, 10**6 + 77)]:
        j, b = s >> 6, s & 63
        u = 0
        for k in range(32):
            w = int(O.philox4x64_10((e, i, 8 * j + (k >> 2), 3), (seed, 0xE5505))[k & 3])
            u |= ((w >> b) & 1) << (31 - k)
        v = int(O.philox4x64_10((e, i, s, 4), (seed, 0xE5505))[0])
        assert O.noise_draw(seed, e, i, s) == (u, v)
    # the 64 shots of a word take distinct bit columns of the same words
    us = [O.noise_draw(3, 1, 2, s)[0] for s in range(64, 128)]
    assert len(set(us)) == 64
