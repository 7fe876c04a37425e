"""GPU parity of the inverse-tableau mode (QS_FLAG_INVERSE_TABLEAU): the
paper's measurement variant (Sec. 3.2, Alg. 1) through the C ABI against the
oracle's inverse mode, bit-exact on the tableau bits, the qubit-indexed signs
S_S and S_D, the record and the measurement kinds; and against the CHP path
(records, kinds, frame samples) under the same keys."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2603_14641_gb300 import qs  # noqa: E402
from workloads import circuits as C  # noqa: E402

INV = qs.QS_FLAG_INVERSE_TABLEAU


def _sim(n, flags=0):
    return qs.Simulator(n, device="cuda:0", flags=INV | flags)


def _assert_inverse(sim, inv):
    x, z, r = sim.export()
    ox, oz, oss, osd = inv.get()
    assert np.array_equal(x, ox), "x bits differ"
    assert np.array_equal(z, oz), "z bits differ"
    assert not r.any(), "per-row signs are not kept in inverse mode"
    ss, sd = sim.qubit_signs()
    assert np.array_equal(ss, oss), "S_S differs"
    assert np.array_equal(sd, osd), "S_D differs"


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 300, 1000, 2000])
def test_inverse_gate_layers_bit_exact(n):
    circ = C.gate_mix_circuit(n, 16, seed=n + 70, final_measure_all=False)
    sim = _sim(n)
    sim.run(circ, seed=1)
    inv, _, _ = O.run_circuit_inverse(circ, seed=1)
    _assert_inverse(sim, inv)
    sim.sync()


@pytest.mark.parametrize("n,seed", [(1, 1), (3, 2), (64, 3), (65, 4), (300, 5), (700, 6), (2000, 7)])
def test_inverse_measurements_bit_exact(n, seed):
    circ = C.gate_mix_circuit(n, 20, seed=seed + 50, measure_every=5, measure_frac=0.3)
    sim = _sim(n)
    rec = sim.run(circ, seed=seed * 11, shot=seed)
    inv, irec, ikinds = O.run_circuit_inverse(circ, seed=seed * 11, shot=seed)
    assert np.array_equal(rec, irec), "records differ from the inverse oracle"
    assert np.array_equal(sim.record_kinds(), ikinds), "kinds differ"
    _assert_inverse(sim, inv)
    _, crec, ckinds = O.run_circuit(circ, seed=seed * 11, shot=seed)
    assert np.array_equal(rec, crec) and np.array_equal(ikinds, ckinds), "records differ from CHP"
    sim.sync()


def test_inverse_repeated_and_deterministic_measurements():
    n = 150
    circ = C.random_circuit(n, 10, 0.5, seed=41, final_measure_all=False)
    q = np.array([3, 3, 77, 149, 0, 77, 3, 149, 0, 148], np.uint32)
    sim = _sim(n)
    sim.run(circ, seed=0)
    out = sim.measure(q, seed=5, shot=2)
    inv, _, _ = O.run_circuit_inverse(circ, seed=0)
    oout, kinds = inv.measure(q, seed=5, shot=2)
    assert np.array_equal(out, oout) and kinds[1] == 0 and out[1] == out[0]
    _assert_inverse(sim, inv)


def test_inverse_initstate_and_device_layers():
    n = 130
    init = (np.arange(n) % 3 == 1).astype(np.uint8)
    circ = C.gate_mix_circuit(n, 12, seed=9, measure_every=4, measure_frac=0.25)
    sim = _sim(n)
    sim.reset(init)
    dc = sim.upload(circ)
    rec = sim.run(circ, seed=3, dc=dc)  # device-resident layers: one inverse kernel per layer
    inv = O.InverseOracle(n, init)
    inv, irec, _ = O.run_circuit_inverse(circ, seed=3, oracle=inv)
    assert np.array_equal(rec, irec)
    _assert_inverse(sim, inv)
    sim2 = _sim(n)
    sim2.reset(init)
    assert np.array_equal(sim2.measure(np.arange(n), seed=1), init)


def test_inverse_mode_sampling_matches_oracle_frames():
    circ = C.gate_mix_circuit(90, 14, seed=12, measure_every=4, measure_frac=0.4)
    sim = _sim(90)
    rec = sim.run(circ, seed=5)
    shots = 300
    words = sim.sample(shots, seed=8, on_device=False)
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")[:, :shots]
    _, crec, _ = O.run_circuit(circ, seed=5)
    assert np.array_equal(rec, crec)
    assert np.array_equal(bits, O.frames(circ, crec, shots, seed=8))


@pytest.mark.parametrize("n", [20_000])
def test_inverse_records_equal_blocked_chp_path_at_scale(n):
    """At 20,000 qubits (beyond the inverse oracle's reach): records and kinds
    of Alg. 1 on the GPU equal those of the CHP path's blocked measurement
    (oracle-checked at this size on the same generator), repeats included."""
    circ = C.random_circuit(n, 6, 0.5, seed=8, final_measure_all=False)
    rng = np.random.default_rng(3)
    q = rng.permutation(n)[:300].astype(np.uint32)
    q = np.concatenate([q[:150], q[:20], q[150:]])
    outs = []
    for flags in (INV, 0):
        s = qs.Simulator(n, device="cuda:0", flags=flags)
        dc = s.upload(circ)
        s.apply_layers_dev(dc, 0, circ.n_layers)
        outs.append((s.measure(q, seed=13), s.record_kinds()))
        s.sync()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert (outs[0][1][150:170] == 0).all()


def test_inverse_mode_refusals():
    sim = _sim(10)
    buf = qs.qs_sim_tableau_export(sim.sim, qs.QS_LAYOUT_ROWS_PACKED)
    with pytest.raises(qs.QsError) as e:
        qs.qs_sim_tableau_import(sim.sim, buf, np.zeros(0, np.uint8), qs.QS_LAYOUT_ROWS_PACKED)
    assert e.value.code == -1
    chp = qs.Simulator(10, device="cuda:0")
    with pytest.raises(qs.QsError) as e:
        chp.qubit_signs()
    assert e.value.code == -6
    sim.sync()


@pytest.mark.parametrize("n,seed", [(64, 1), (130, 2), (300, 3)])
def test_inverse_mode_holds_the_chp_oracles_stabilizer_group(n, seed):
    """The canonical stabilizer group (reduced row echelon form with signs)
    of the GPU's inverse tableau equals that of the CHP oracle after gates and
    measurements under the same keyed coins."""
    from tests import stabilizer_canon as SC
    circ = C.gate_mix_circuit(n, 18, seed=seed + 90, measure_every=4, measure_frac=0.3)
    sim = _sim(n)
    rec = sim.run(circ, seed=seed * 7)
    o, orec, _ = O.run_circuit(circ, seed=seed * 7)
    assert np.array_equal(rec, orec)
    x, z, _ = sim.export()
    ss, sd = sim.qubit_signs()
    got = SC.stabilizer_group_of_inverse(x, z, ss, sd)
    want = SC.stabilizer_group_of_chp(*o.get())
    assert len(want[2]) == n and SC.same_group(got, want)
    sim.sync()
