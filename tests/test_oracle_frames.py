"""Pins for the oracle's Pauli-frame sampler (Sec. 5, Alg. 9; no GPU).

The frame sampler must draw records from the circuit's measurement
distribution: every sampled record has nonzero Born probability under a
brute-force state vector (support check), and the records are uniformly
distributed over that support with each record's probability equal to the
state-vector probability (chi-square).
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import sv_helpers as SV
from workloads import circuits as C


def _record_probability(circ, record):
    sv = SV.StateVector(circ.n)
    p = 1.0
    m = 0
    for op in circ.ops:
        if op[0] == "layers":
            sv.apply(circ.gates[circ.layer_ptr[op[1]]:circ.layer_ptr[op[2]]])
        else:
            for q in op[1]:
                p *= sv.project(int(q), int(record[m]))
                m += 1
                if p < 1e-12:
                    return 0.0
    return p


@pytest.mark.parametrize("n,seed,every,frac", [(3, 1, 2, 0.67), (5, 2, 3, 0.4), (6, 3, 4, 0.5),
                                               (8, 4, 5, 0.25)])
def test_frames_support_and_distribution(n, seed, every, frac):
    circ = C.gate_mix_circuit(n, 10, seed, measure_every=every, measure_frac=frac)
    _, ref, _ = O.run_circuit(circ, seed=seed, force_zero=True)
    shots = 2000
    out = O.frames(circ, ref, shots, seed=seed + 100)
    recs = {}
    for s in range(shots):
        key = out[:, s].tobytes()
        recs[key] = recs.get(key, 0) + 1
    probs = {}
    for key in recs:
        p = _record_probability(circ, np.frombuffer(key, np.uint8))
        assert p > 1e-9, "sampled record outside the support"
        probs[key] = p
    # the sampled support carries (almost) all probability mass
    assert sum(probs.values()) > 0.99
    # chi-square over the support
    exp = np.array([probs[k] * shots for k in recs])
    obs = np.array([recs[k] for k in recs])
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    dof = max(len(recs) - 1, 1)
    assert chi2 < dof + 6 * np.sqrt(2 * dof) + 10, (chi2, dof)


def test_frames_reference_is_deterministic_part():
    """GHZ: every shot is all-equal; both values appear."""
    n = 6
    g = [[C.H, 0, 0]] + [[C.CX, 0, i] for i in range(1, n)]
    circ = C.Circuit(n=n, gates=np.array(g, np.uint32), layer_ptr=np.array([0, len(g)]),
                     ops=[("layers", 0, 1), ("measure", np.arange(n, dtype=np.uint32))])
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    out = O.frames(circ, ref, 256, seed=3)
    assert (out == out[0:1]).all()
    assert 60 < out[0].sum() < 196


def test_frames_are_keyed():
    circ = C.random_circuit(10, 8, 0.5, seed=4)
    _, ref, _ = O.run_circuit(circ, seed=1, force_zero=True)
    a = O.frames(circ, ref, 130, seed=9)
    b = O.frames(circ, ref, 130, seed=9)
    c = O.frames(circ, ref, 130, seed=10)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
