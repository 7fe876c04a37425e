"""Degenerate inputs through the C ABI on the GPU: one qubit, empty layers and
measurement lists, sampling a program without measurements, batches with
empty circuits; every result against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2603_14641_gb300 import qs  # noqa: E402
from workloads import circuits as C  # noqa: E402


def test_one_qubit_and_empty_operations():
    sim = qs.Simulator(1, device="cuda:0")
    sim.apply_layer(np.zeros((0, 3), np.uint32))                  # empty layer
    assert len(sim.measure(np.zeros(0, np.uint32), seed=1)) == 0   # empty measurement list
    sim.apply_layer(np.array([[C.H, 0, 0]], np.uint32))
    out = sim.measure(np.array([0, 0, 0], np.uint32), seed=9)      # random, then repeated
    o = O.Oracle(1)
    o.apply(np.array([[C.H, 0, 0]], np.uint32))
    oout, kinds = o.measure(np.array([0, 0, 0], np.uint32), seed=9)
    assert np.array_equal(out, oout) and list(kinds) == [1, 0, 0]
    assert out[0] == out[1] == out[2]
    x, z, r = sim.export()
    ox, oz, orr = o.get()
    assert np.array_equal(x, ox) and np.array_equal(z, oz) and np.array_equal(r, orr)
    sim.sync()


def test_sampling_without_measurements_and_one_shot():
    circ = C.random_circuit(50, 6, 0.5, seed=3, final_measure_all=False)
    sim = qs.Simulator(50, device="cuda:0")
    sim.run(circ, seed=2)
    assert sim.num_measurements == 0
    w = sim.sample(100, seed=4, on_device=False)
    assert w.shape == (0, 2)
    sim.measure(np.array([7], np.uint32), seed=2)
    w = sim.sample(1, seed=4, on_device=False)
    full = C.Circuit(n=50, gates=circ.gates, layer_ptr=circ.layer_ptr,
                     ops=list(circ.ops) + [("measure", np.array([7], np.uint32))])
    _, orec, _ = O.run_circuit(full, seed=2)
    assert np.array_equal(sim.record(), orec)
    ref = O.frames(full, orec, 1, seed=4)
    assert w.shape == (1, 1) and int(w[0, 0]) >> 1 == 0 and (int(w[0, 0]) & 1) == ref[0, 0]


def test_batch_with_empty_and_measure_only_circuits():
    empty = C.Circuit(n=3, gates=np.zeros((0, 3), np.uint32), layer_ptr=np.array([0]), ops=[])
    meas_only = C.Circuit(n=5, gates=np.zeros((0, 3), np.uint32), layer_ptr=np.array([0]),
                          ops=[("measure", np.array([4, 0, 4], np.uint32))])
    big_meas_only = C.Circuit(n=1100, gates=np.zeros((0, 3), np.uint32), layer_ptr=np.array([0]),
                              ops=[("measure", np.arange(0, 1100, 50, dtype=np.uint32))])
    normal = C.random_circuit(40, 8, 0.5, seed=6, measure_every=4, measure_frac=0.5)
    circs = [empty, meas_only, big_meas_only, normal]
    seeds = [1, 2, 3, 4]
    b = qs.Batch(circs, seeds, device="cuda:0")
    b.run()
    b.sync()
    for i, c in enumerate(circs):
        _, orec, _ = O.run_circuit(c, seed=seeds[i])
        assert np.array_equal(b.record(i), orec), i
    assert not b.record(2).any()  # |0...0>: every outcome is 0


def test_host_checks_reject_bad_ranges_and_keep_the_sim_usable():
    """Ranges that would wrap around 64 bits and negative layer offsets are
    refused on the host before any device access; the sim stays usable."""
    import ctypes
    L = qs.lib()
    circ = C.random_circuit(70, 5, 0.5, seed=11, final_measure_all=True)
    sim = qs.Simulator(70, device="cuda:0")
    rec = sim.run(circ, seed=5)
    buf = np.zeros(8, np.uint8)
    p = ctypes.c_void_p(buf.ctypes.data)
    h = ctypes.c_void_p(sim.sim)
    assert L.qs_sim_record(h, 2**64 - 1, 2, p) == -1
    assert L.qs_sim_record_kinds(h, 3, 2**64 - 2, p) == -1
    assert L.qs_sim_record(h, len(rec), 1, p) == -1
    dc = sim.upload(circ)
    bad = np.array([-2, 0], np.int64)
    assert L.qs_sim_apply_layers_dev(h, ctypes.c_void_p(dc.packed.data_ptr()),
                                     ctypes.c_void_p(bad.ctypes.data), 0, 1) == -1
    for shots in (0, 2_000_000_001):  # refused before any allocation or launch
        assert L.qs_sim_sample(h, shots, 1, None, 0, None, 0) == -1
        assert L.qs_sim_sample_noalloc(h, shots, 1, None, 0) == -1
    sim.sync()
    _, orec, _ = O.run_circuit(circ, seed=5)
    assert np.array_equal(sim.record(), orec)
    assert np.array_equal(sim.record(len(rec) - 3, 3), orec[-3:])


def test_kernel_timing_leaves_results_unchanged():
    """qs_sim_set_timing only timestamps the stream: with timing on, record,
    tableau and samples equal the oracle's, and every phase that ran (gate
    layers, layout switch, each part of a blocked measurement block, sampling)
    has timed groups with positive device time."""
    circ = C.random_circuit(700, 12, 0.5, seed=12, final_measure_all=True)
    sim = qs.Simulator(circ.n, device="cuda:0")
    qs.qs_sim_set_timing(sim.sim, True)
    dc = sim.upload(circ)
    rec = sim.run(circ, seed=5, dc=dc)
    words = sim.sample(64, seed=2, on_device=False)
    t = qs.qs_sim_timing(sim.sim)
    o, orec, _ = O.run_circuit(circ, seed=5)
    assert np.array_equal(rec, orec)
    x, z, r = sim.export()
    ox, oz, orr = o.get()
    assert np.array_equal(x, ox) and np.array_equal(z, oz) and np.array_equal(r, orr)
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")
    assert np.array_equal(bits, O.frames(circ, orec, 64, seed=2))
    for kind in ("gates", "transpose", "blk_symbolic", "blk_pivot_rows", "blk_apply", "blk_signs",
                 "sample"):
        ms, cnt = t[kind]
        assert cnt > 0 and ms > 0, (kind, t[kind])
    assert t["blk_apply"][1] >= 5
    qs.qs_sim_set_timing(sim.sim, False)
    with pytest.raises(qs.QsError):
        qs.qs_sim_timing(sim.sim)
    sim.sync()
