"""GPU parity of the Pauli noise channels on the frames (qs_sim_noise):
noisy shots from the CUDA path equal the oracle's bit for bit, for every
channel, probabilities 0 < p < 1 and the edge values 0 and 1, ragged shot
counts, every qubit of a 70,000-qubit register as a target, and the
allocation-free sampler; bad arguments are rejected on the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2603_14641_gb300 import qs  # noqa: E402
from workloads import circuits as C  # noqa: E402


def _bits(words, shots):
    b = np.unpackbits(np.ascontiguousarray(words).view(np.uint8), axis=1, bitorder="little")
    assert not b[:, shots:].any()
    return b[:, :shots]


def _check(circ, seed, shots, sample_seed, noalloc=False):
    sim = qs.Simulator(circ.n, device="cuda:0")
    rec = sim.run(circ, seed=seed)
    _, orec, _ = O.run_circuit(circ, seed=seed)
    assert np.array_equal(rec, orec), "reference shot differs"
    if noalloc:
        ow = (shots + 63) // 64
        out = np.zeros((max(sim.num_measurements, 1), ow), np.uint64)
        qs.qs_sim_sample_noalloc(sim.sim, shots, sample_seed, out.ctypes.data,
                                 sim.num_measurements * ow)
        words = out[:sim.num_measurements]
    else:
        words = sim.sample(shots, sample_seed, on_device=False)
    want = O.frames(circ, orec, shots, sample_seed)
    assert np.array_equal(_bits(words, shots), want)
    return words


@pytest.mark.parametrize("n,shots,pg,pm", [(5, 64, 0.3, 0.5), (37, 200, 0.01, 0.02),
                                           (300, 1000, 0.05, 0.1), (1100, 4097, 0.002, 0.01)])
def test_circuit_noise_bit_exact(n, shots, pg, pm):
    base = C.random_circuit(n, 12, 0.5, seed=n, measure_every=4, measure_frac=0.3,
                            final_measure_all=True)
    _check(C.with_circuit_noise(base, pg, pm), seed=n + 1, shots=shots, sample_seed=n + 2)


@pytest.mark.parametrize("kind", [C.NOISE_X, C.NOISE_Y, C.NOISE_Z, C.DEPOLARIZE1, C.DEPOLARIZE2])
@pytest.mark.parametrize("p", [0.0, 0.37, 1.0])
def test_each_channel_bit_exact(kind, p):
    base = C.gate_mix_circuit(70, 9, seed=5, measure_every=3, measure_frac=0.3)
    rng = np.random.default_rng(int(kind * 10 + p * 100))
    ops = []
    for op in base.ops:
        ops.append(op)
        if op[0] == "layers":
            t = rng.permutation(70)[:40].astype(np.uint32)
            ops.append(("noise", kind, p, t))
    circ = C.Circuit(n=70, gates=base.gates, layer_ptr=base.layer_ptr,
                     ops=ops + [("measure", np.arange(70, dtype=np.uint32))])
    _check(circ, seed=3, shots=321, sample_seed=9)


def test_noise_with_allocation_free_sampler():
    base = C.random_circuit(200, 10, 0.5, seed=4, measure_every=5, measure_frac=0.2,
                            final_measure_all=True)
    circ = C.with_circuit_noise(base, 0.02, 0.05)
    a = _check(circ, seed=1, shots=150, sample_seed=6)
    b = _check(circ, seed=1, shots=150, sample_seed=6, noalloc=True)
    assert np.array_equal(a, b)


def test_all_qubits_as_targets_at_70k():
    """70,000 qubits in |0...0>: DEPOLARIZE2 on 35,000 pairs and X_ERROR on all
    qubits; the reference record of this product state is all zeros, so the
    oracle needs no tableau here."""
    n = 70_000
    meas = np.arange(0, n, 37, dtype=np.uint32)
    pairs = np.random.default_rng(2).permutation(n).astype(np.uint32)
    circ = C.Circuit(n=n, gates=np.zeros((0, 3), np.uint32), layer_ptr=np.array([0]),
                     ops=[("noise", C.DEPOLARIZE2, 0.2, pairs),
                          ("noise", C.NOISE_X, 0.1, np.arange(n, dtype=np.uint32)),
                          ("measure", meas)])
    sim = qs.Simulator(n, device="cuda:0")
    rec = sim.run(circ, seed=1)
    assert not rec.any()
    shots = 96
    words = sim.sample(shots, 8, on_device=False)
    want = O.frames(circ, np.zeros(len(meas), np.uint8), shots, 8)
    assert np.array_equal(_bits(words, shots), want)


def test_bad_noise_arguments_are_rejected():
    sim = qs.Simulator(10, device="cuda:0")
    for kind, p, t in [(7, 0.1, [0]), (C.NOISE_X, -0.1, [0]), (C.NOISE_X, 1.5, [0]),
                       (C.NOISE_X, float("nan"), [0]), (C.NOISE_Z, 0.1, [10]),
                       (C.DEPOLARIZE1, 0.1, [3, 3]), (C.DEPOLARIZE2, 0.1, [1, 2, 3]),
                       (C.DEPOLARIZE2, 0.1, [1, 2, 2, 4])]:
        with pytest.raises(qs.QsError) as e:
            sim.noise(kind, p, np.array(t, np.uint32))
        assert e.value.code == -1
    # nothing was appended: sampling the empty program works
    sim.noise(C.NOISE_X, 0.5, np.array([1, 2], np.uint32))
    sim.measure(np.array([1, 2, 3], np.uint32), seed=0)
    w = sim.sample(64, 1, on_device=False)
    assert w.shape == (3, 1)


def test_noise_targets_follow_the_op_log():
    """Sampling keeps every noise op's targets on the device between calls: a
    program that grows after a sample, and a new program after reset (fewer
    and then more targets than the buffer holds), still sample bit-exact."""
    n, shots = 120, 200
    base = C.random_circuit(n, 8, 0.5, seed=21, measure_every=4, measure_frac=0.3,
                            final_measure_all=False)
    first = C.with_circuit_noise(base, 0.03, 0.05)
    rng = np.random.default_rng(5)
    tail = [("noise", C.DEPOLARIZE2, 0.2, rng.permutation(n)[:80].astype(np.uint32)),
            ("noise", C.NOISE_Y, 0.4, rng.permutation(n)[:50].astype(np.uint32)),
            ("measure", np.arange(n, dtype=np.uint32))]
    whole = C.Circuit(n=n, gates=first.gates, layer_ptr=first.layer_ptr,
                      ops=list(first.ops) + tail)
    sim = qs.Simulator(n, device="cuda:0")
    for circ, ops in ((first, first.ops), (whole, tail)):
        rec = sim.run(C.Circuit(n=n, gates=first.gates, layer_ptr=first.layer_ptr, ops=ops), seed=2)
        _, orec, _ = O.run_circuit(circ, seed=2)
        assert np.array_equal(rec, orec)
        words = sim.sample(shots, 7, on_device=False)
        assert np.array_equal(_bits(words, shots), O.frames(circ, orec, shots, 7))
    for p, depth in ((0.1, 3), (0.02, 14)):
        circ = C.with_circuit_noise(C.random_circuit(n, depth, 0.5, seed=depth, measure_every=3,
                                                     measure_frac=0.4, final_measure_all=True),
                                    p, p)
        sim.reset()
        rec = sim.run(circ, seed=4)
        _, orec, _ = O.run_circuit(circ, seed=4)
        assert np.array_equal(rec, orec)
        words = sim.sample(shots, 3, on_device=False)
        assert np.array_equal(_bits(words, shots), O.frames(circ, orec, shots, 3))
