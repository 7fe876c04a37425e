"""GPU tests of the batched persistent launch (qs_batch_*): every circuit's
record and tableau rows equal the oracle's and the single-circuit path's,
whatever the launch shape; a grid barrier that runs out is reported as
QS_ERR_TIMEOUT and leaves the context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2603_14641_gb300 import qs  # noqa: E402
from workloads import circuits as C  # noqa: E402


def _mixed_batch(count=20, seed=0):
    rng = np.random.default_rng(seed)
    circs = []
    for i in range(count):
        n = int(rng.choice([1, 2, 5, 33, 64, 65, 130, 257, 400, 700]))
        if i % 2:
            c = C.gate_mix_circuit(n, 16, seed=100 + i, measure_every=4, measure_frac=0.3,
                                   final_measure_all=(i % 4 == 1))
        else:
            c = C.random_circuit(n, 18, 0.5, seed=200 + i, measure_every=6, measure_frac=0.2,
                                 final_measure_all=False)
        circs.append(c)
    return circs


def test_batch_matches_oracle_and_single_path():
    circs = _mixed_batch()
    seeds = [7 + i for i in range(len(circs))]
    b = qs.Batch(circs, seeds, device="cuda:0")
    b.run()
    b.sync()
    rng = np.random.default_rng(1)
    for i, c in enumerate(circs):
        rec = b.record(i)
        o, orec, _ = O.run_circuit(c, seed=seeds[i])
        assert np.array_equal(rec, orec), f"circuit {i} (n={c.n}) record differs"
        rows = np.unique(rng.choice(2 * c.n, size=min(2 * c.n, 12), replace=False)).astype(np.uint32)
        x, z, r = b.export_rows(i, rows)
        ox, oz, orr = o.get()
        assert np.array_equal(x, ox[rows]) and np.array_equal(z, oz[rows]) and np.array_equal(r, orr[rows])
        if i < 6:
            s = qs.Simulator(c.n, device="cuda:0")
            srec = s.run(c, seed=seeds[i])
            assert np.array_equal(srec, rec)


def test_batch_result_independent_of_launch_shape():
    circs = _mixed_batch(12, seed=3)
    seeds = list(range(100, 112))
    b = qs.Batch(circs, seeds, device="cuda:0")
    ref = None
    for t in [qs.qs_batch_tuning(512, 0, 1, 0, 0), qs.qs_batch_tuning(256, 2, 2, 0, 0),
              qs.qs_batch_tuning(1024, 1, 1, 1, 0), qs.qs_batch_tuning(256, 1, 1, 3, 0)]:
        b.run(t)
        b.sync()
        recs = [b.record(i) for i in range(len(circs))]
        rows = [b.export_rows(i, np.arange(min(2 * c.n, 16), dtype=np.uint32))
                for i, c in enumerate(circs)]
        if ref is None:
            ref = (recs, rows)
        else:
            for a, bb in zip(ref[0], recs):
                assert np.array_equal(a, bb)
            for ra, rb in zip(ref[1], rows):
                for u, v in zip(ra, rb):
                    assert np.array_equal(u, v)


def test_batch_barrier_timeout_is_reported_and_recoverable():
    circs = _mixed_batch(8, seed=5)
    seeds = list(range(8))
    b = qs.Batch(circs, seeds, device="cuda:0")
    t = qs.qs_batch_tuning(512, 0, 1, 0, 1)  # spin limit 1: the first barrier runs out
    b.run(t)
    with pytest.raises(qs.QsError) as e:
        b.sync()
    assert e.value.code == -4
    # the context is still usable: a normal run gives the oracle's records
    b.run()
    b.sync()
    for i, c in enumerate(circs):
        _, orec, _ = O.run_circuit(c, seed=seeds[i])
        assert np.array_equal(b.record(i), orec)


def test_batch_workload_subset_matches_single_circuit_path():
    """A seeded subset of the 512-circuit workload (n 50..5000, depth 200,
    10% measured every 10 layers): batch vs one circuit at a time."""
    circs = C.batch_workload(512)
    idx = [0, 1, 2, 3, 5, 8, 13, 21]
    sub = [circs[i] for i in idx]
    seeds = [1000 + i for i in idx]
    b = qs.Batch(sub, seeds, device="cuda:0")
    b.run()
    b.sync()
    for j, c in enumerate(sub):
        s = qs.Simulator(c.n, device="cuda:0")
        dc = s.upload(c)
        rec = s.run(c, seed=seeds[j], dc=dc)
        assert np.array_equal(b.record(j), rec), f"circuit {idx[j]} (n={c.n})"
        rows = np.arange(0, 2 * c.n, max(1, (2 * c.n) // 40), dtype=np.uint32)
        bx, bz, br = b.export_rows(j, rows)
        sx, sz, sr = s.export_rows(rows)
        assert np.array_equal(bx, sx) and np.array_equal(bz, sz) and np.array_equal(br, sr)


def test_batch_rejects_bad_programs():
    c = C.random_circuit(10, 4, 0.5, seed=1)
    bad = C.Circuit(n=10, gates=np.array([[C.CX, 3, 3]], np.uint32), layer_ptr=np.array([0, 1]),
                    ops=[("layers", 0, 1), ("measure", np.array([0], np.uint32))])
    with pytest.raises(qs.QsError) as e:
        qs.Batch([c, bad], [1, 2], device="cuda:0")
    assert e.value.code == -1
    empty = C.Circuit(n=0, gates=np.zeros((0, 3), np.uint32), layer_ptr=np.array([0]), ops=[])
    with pytest.raises(qs.QsError):
        qs.Batch([c, empty], [1, 2], device="cuda:0")


def test_batch_large_circuits_run_through_simulators():
    """n >= 1024 circuits (here up to 9,000 qubits, beyond the persistent
    kernel's shared-memory limit) mixed with small ones: every record and
    sampled rows equal the single-circuit path, over repeated runs and a
    round limit."""
    circs = [C.random_circuit(n, 20, 0.5, seed=n, measure_every=5, measure_frac=0.1)
             for n in (9000, 300, 1024, 50, 2048, 1500)]
    seeds = [11 * i + 3 for i in range(len(circs))]
    b = qs.Batch(circs, seeds, device="cuda:0")
    for _ in range(2):
        b.run()
        b.sync()
    for i, c in enumerate(circs):
        s = qs.Simulator(c.n, device="cuda:0")
        rec = s.run(c, seed=seeds[i])
        assert np.array_equal(b.record(i), rec), f"circuit {i} (n={c.n})"
        rows = np.arange(0, 2 * c.n, max(1, (2 * c.n) // 30), dtype=np.uint32)
        bx, bz, br = b.export_rows(i, rows)
        sx, sz, sr = s.export_rows(rows)
        assert np.array_equal(bx, sx) and np.array_equal(bz, sz) and np.array_equal(br, sr)


def test_batched_sampling_matches_single_path_and_oracle():
    """qs_batch_sample: every circuit's frame samples, drawn for all small
    circuits in one launch (and through the worker simulators for n >= 1024),
    equal qs_sim_sample of the circuit alone under the same seeds and the
    oracle's Pauli-frame samples (Sec. 5), ragged shot counts included; a
    circuit given 0 shots is skipped."""
    circs = _mixed_batch(14, seed=5)
    circs.append(C.random_circuit(1100, 8, 0.5, seed=9, measure_every=4, measure_frac=0.1))
    seeds = [30 + i for i in range(len(circs))]
    shots = [0 if i == 3 else [1, 64, 65, 200, 1000, 4097][i % 6] for i in range(len(circs))]
    fseeds = [900 + i for i in range(len(circs))]
    b = qs.Batch(circs, seeds, device="cuda:0")
    with pytest.raises(qs.QsError):  # no complete run yet
        b.sample(shots, fseeds)
    b.run()
    outs = b.sample(shots, fseeds)
    b.sync()
    for i, c in enumerate(circs):
        if shots[i] == 0:
            assert outs[i] is None
            continue
        got = outs[i].cpu().numpy().view(np.uint64)
        s = qs.Simulator(c.n, device="cuda:0")
        rec = s.run(c, seed=seeds[i])
        want = s.sample(shots[i], seed=fseeds[i], on_device=False)
        assert got.shape == want.shape and np.array_equal(got, want), f"circuit {i} (n={c.n})"
        if c.n <= 700:
            bits = np.unpackbits(got.view(np.uint8), axis=1, bitorder="little")
            assert not bits[:, shots[i]:].any()
            assert np.array_equal(bits[:, :shots[i]], O.frames(c, rec, shots[i], seed=fseeds[i]))
        s.close()
