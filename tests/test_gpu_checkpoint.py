"""Checkpoint and resume on the GPU (qs_sim_tableau_import): a run that is
exported halfway and restored into a fresh simulator continues bit for bit
like the uninterrupted run and like the oracle; a state built by the oracle
and packed by hand imports to the oracle's tableau; bad checkpoints are
rejected and sampling after a restore is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2603_14641_gb300 import qs  # noqa: E402
from workloads import circuits as C  # noqa: E402


def _pack(x, z, r, n):
    """(x, z, r) bit rows -> the export layout: per row k x-words then k z-words
    (bit j of word w = qubit 64 w + j), then the sign bit-vector."""
    k = (n + 63) // 64
    pad = np.zeros((2 * n, 64 * k), np.uint8)
    xs = pad.copy()
    xs[:, :n] = x
    zs = pad.copy()
    zs[:, :n] = z
    words = lambda b: np.packbits(b, axis=1, bitorder="little").view(np.uint64)  # noqa: E731
    rows = np.concatenate([words(xs), words(zs)], axis=1).reshape(-1)
    sig = np.zeros(64 * ((2 * n + 63) // 64), np.uint8)
    sig[:2 * n] = r
    return np.concatenate([rows, np.packbits(sig, bitorder="little").view(np.uint64)])


def _run_ops(sim, circ, ops, seed):
    for op in ops:
        if op[0] == "layers":
            for l in range(op[1], op[2]):
                sim.apply_layer(circ.layer(l))
        else:
            sim.measure(op[1], seed=seed, want_outcomes=False)


@pytest.mark.parametrize("n", [70, 1500])
def test_resume_reproduces_the_uninterrupted_run(n):
    circ = C.random_circuit(n, 16, 0.5, seed=n, measure_every=4, measure_frac=0.2,
                            final_measure_all=True)
    half = len(circ.ops) // 2
    a = qs.Simulator(n, device="cuda:0")
    _run_ops(a, circ, circ.ops[:half], seed=3)
    packed, rec = a.checkpoint()
    _run_ops(a, circ, circ.ops[half:], seed=3)
    b = qs.Simulator(n, device="cuda:0")
    b.restore(packed, rec)
    _run_ops(b, circ, circ.ops[half:], seed=3)
    assert np.array_equal(a.record(), b.record())
    for u, v in zip(a.export(), b.export()):
        assert np.array_equal(u, v)
    o, orec, _ = O.run_circuit(circ, seed=3)
    assert np.array_equal(b.record(), orec)
    for u, v in zip(b.export(), o.get()):
        assert np.array_equal(u, v)
    with pytest.raises(qs.QsError) as e:
        b.sample(64, seed=1)
    assert e.value.code == -6
    b.reset()
    b.measure(np.array([0], np.uint32), seed=1)
    assert b.sample(64, seed=1).shape[0] == 1


def test_import_of_an_oracle_state():
    n = 200
    circ = C.gate_mix_circuit(n, 12, seed=4, measure_every=5, measure_frac=0.3)
    o, orec, _ = O.run_circuit(circ, seed=8)
    x, z, r = o.get()
    sim = qs.Simulator(n, device="cuda:0")
    sim.restore(_pack(x, z, r, n), orec)
    for u, v in zip(sim.export(), (x, z, r)):
        assert np.array_equal(u, v)
    more = C.random_circuit(n, 6, 0.5, seed=9, final_measure_all=True)
    _run_ops(sim, more, more.ops, seed=8)
    # record indices continue after the first len(orec) measurements
    rec = sim.record()
    assert np.array_equal(rec[:len(orec)], orec)
    q = np.arange(n, dtype=np.uint32)
    o2, _, _ = O.run_circuit(C.Circuit(n=n, gates=np.concatenate([circ.gates, more.gates]),
                                        layer_ptr=np.concatenate([circ.layer_ptr,
                                                                  circ.layer_ptr[-1] + more.layer_ptr[1:]]),
                                        ops=list(circ.ops) + [("layers", circ.n_layers,
                                                               circ.n_layers + more.n_layers),
                                                              ("measure", q)]), seed=8)
    _, rec2, _ = O.run_circuit(C.Circuit(n=n, gates=np.concatenate([circ.gates, more.gates]),
                                         layer_ptr=np.concatenate([circ.layer_ptr,
                                                                   circ.layer_ptr[-1] + more.layer_ptr[1:]]),
                                         ops=list(circ.ops) + [("layers", circ.n_layers,
                                                                circ.n_layers + more.n_layers),
                                                               ("measure", q)]), seed=8)
    assert np.array_equal(rec, rec2)
    for u, v in zip(sim.export(), o2.get()):
        assert np.array_equal(u, v)


def test_bad_checkpoints_are_rejected():
    n = 70
    sim = qs.Simulator(n, device="cuda:0")
    packed, rec = sim.checkpoint()
    bad = packed.copy()
    bad[1] |= np.uint64(1) << np.uint64(63)  # qubit 127 of row 0 does not exist
    with pytest.raises(qs.QsError) as e:
        sim.restore(bad, rec)
    assert e.value.code == -1
    with pytest.raises(qs.QsError) as e:
        sim.restore(packed[:-1], rec)
    assert e.value.code == -5


@pytest.mark.parametrize("n", [70, 1500])
def test_native_layout_export_import_and_device_destination(n):
    """NATIVE export decodes to the oracle's tableau; exports into device memory
    equal the host ones; a NATIVE checkpoint resumes bit for bit; padding bits
    in a NATIVE checkpoint are rejected."""
    circ = C.random_circuit(n, 16, 0.5, seed=n + 1, measure_every=4, measure_frac=0.2,
                            final_measure_all=True)
    half = len(circ.ops) // 2
    a = qs.Simulator(n, device="cuda:0")
    _run_ops(a, circ, circ.ops[:half], seed=5)  # ends after a measurement window or a layer
    native, rec = a.checkpoint(qs.QS_LAYOUT_NATIVE)
    # the oracle's state at the checkpoint: the same circuit cut after the same ops
    trunc = C.Circuit(n=n, gates=circ.gates, layer_ptr=circ.layer_ptr, ops=list(circ.ops[:half]))
    ot, orec, _ = O.run_circuit(trunc, seed=5)
    assert np.array_equal(rec, orec)
    for u, v in zip(qs.unpack_native(native, n), ot.get()):
        assert np.array_equal(u, v)
    rows = qs.qs_sim_tableau_export(a.sim)
    for fmt, host in [(qs.QS_LAYOUT_NATIVE, native), (qs.QS_LAYOUT_ROWS_PACKED, rows)]:
        dev = torch.zeros(len(host), dtype=torch.int64, device="cuda:0")
        qs.qs_sim_tableau_export(a.sim, fmt, out=dev)
        assert np.array_equal(dev.cpu().numpy().view(np.uint64), host)
    _run_ops(a, circ, circ.ops[half:], seed=5)
    b = qs.Simulator(n, device="cuda:0")
    b.restore(native, rec, qs.QS_LAYOUT_NATIVE)
    _run_ops(b, circ, circ.ops[half:], seed=5)
    assert np.array_equal(a.record(), b.record())
    for u, v in zip(a.export(), b.export()):
        assert np.array_equal(u, v)
    k = (n + 63) // 64
    W = (2 * k + 3) // 4 * 4
    bad = native.copy()
    bad[3 * W + k - 1] |= np.uint64(1) << np.uint64(63)  # destabilizer number 64 k - 1 >= n
    c = qs.Simulator(n, device="cuda:0")
    with pytest.raises(qs.QsError) as e:
        c.restore(bad, rec, qs.QS_LAYOUT_NATIVE)
    assert e.value.code == -1
