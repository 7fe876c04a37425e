"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit-exact on tableau bits, signs, measurement records and frame samples.

Sizes the oracle finishes in seconds cover several 64-bit words, several
256x256 transpose tiles and ragged tails; at the full workload sizes (10,000
and 180,000 qubits) the checks use sampled rows the oracle can follow alone
(gate rules act row by row) and properties that hold at any size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from tests import oracle_jobs  # noqa: E402
from paper_2603_14641_gb300 import qs  # noqa: E402
from workloads import circuits as C  # noqa: E402


def _sim(n, **kw):
    return qs.Simulator(n, device="cuda:0", **kw)


def _assert_tableau(sim, o):
    x, z, r = sim.export()
    ox, oz, orr = o.get()
    assert np.array_equal(x, ox), "x bits differ"
    assert np.array_equal(z, oz), "z bits differ"
    assert np.array_equal(r, orr), "signs differ"


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 256, 300, 1000, 2000])
def test_gate_layers_bit_exact(n):
    circ = C.gate_mix_circuit(n, 16, seed=n, final_measure_all=False)
    sim = _sim(n)
    sim.run(circ, seed=1)
    o, _, _ = O.run_circuit(circ, seed=1)
    _assert_tableau(sim, o)
    sim.sync()


@pytest.mark.parametrize("n,seed", [(1, 1), (3, 2), (64, 3), (65, 4), (300, 5), (700, 6), (2000, 7)])
def test_measurements_bit_exact(n, seed):
    circ = C.gate_mix_circuit(n, 24, seed=seed, measure_every=5, measure_frac=0.3)
    sim = _sim(n)
    rec = sim.run(circ, seed=seed * 13, shot=seed)
    o, orec, kinds = O.run_circuit(circ, seed=seed * 13, shot=seed)
    assert np.array_equal(rec, orec), "records differ"
    _assert_tableau(sim, o)
    sim.sync()


def test_workload_256_full():
    """n = 256, depth 100, final measurement of all qubits, 1 shot."""
    circ = C.workload_256()
    sim = _sim(circ.n)
    rec = sim.run(circ, seed=2026)
    o, orec, kinds = O.run_circuit(circ, seed=2026)
    assert np.array_equal(rec, orec)
    assert kinds.sum() > 0 and (kinds == 0).sum() > 0  # both measurement kinds occur
    _assert_tableau(sim, o)
    sim.sync()


def test_hsc_generator_with_periodic_measurements():
    """Same generator as the 10,000-qubit workload, at n = 2000 (5% every 10 layers)."""
    circ = C.random_circuit(2000, 40, 0.5, seed=2, measure_every=10, measure_frac=0.05)
    sim = _sim(circ.n)
    rec = sim.run(circ, seed=99)
    o, orec, _ = O.run_circuit(circ, seed=99)
    assert np.array_equal(rec, orec)
    _assert_tableau(sim, o)


def test_repeated_and_deterministic_measurements():
    n = 150
    circ = C.gate_mix_circuit(n, 10, seed=4, final_measure_all=False)
    qubits = np.array([3, 3, 77, 149, 0, 77, 3, 149, 0], np.uint32)
    sim = _sim(n)
    sim.run(circ, seed=1)
    out = sim.measure(qubits, seed=5, shot=2)
    o, _, _ = O.run_circuit(circ, seed=1)
    oout, kinds = o.measure(qubits, seed=5, shot=2)
    assert np.array_equal(out, oout)
    assert kinds[1] == 0 and out[1] == out[0]
    _assert_tableau(sim, o)


def test_ghz_closed_form_on_gpu():
    n = 1000
    g = [[C.H, 0, 0]]
    sim = _sim(n)
    sim.apply_layer(np.array(g, np.uint32))
    for i in range(1, n):
        sim.apply_layer(np.array([[C.CX, i - 1, i]], np.uint32))
    out = sim.measure(np.arange(n), seed=8, shot=1)
    assert (out == out[0]).all() and out[0] == O.coin(8, 1, 0)
    sim.sync()


def test_initstate_reset():
    n = 70
    init = (np.arange(n) % 3 == 0).astype(np.uint8)
    sim = _sim(n)
    sim.reset(init)
    out = sim.measure(np.arange(n), seed=0)
    assert np.array_equal(out, init)
    o = O.Oracle(n)
    o.reset(init)
    o.measure(np.arange(n), seed=0)
    _assert_tableau(sim, o)


def test_device_resident_layers_match_host_path():
    circ = C.gate_mix_circuit(500, 20, seed=9, measure_every=7, measure_frac=0.2)
    a = _sim(circ.n)
    ra = a.run(circ, seed=3)
    b = _sim(circ.n)
    dc = b.upload(circ)
    rb = b.run(circ, seed=3, dc=dc)
    assert np.array_equal(ra, rb)
    xa, za, sa = a.export()
    xb, zb, sb = b.export()
    assert np.array_equal(xa, xb) and np.array_equal(za, zb) and np.array_equal(sa, sb)


def test_device_qubit_list_matches_host_list():
    circ = C.random_circuit(300, 12, 0.5, seed=5, final_measure_all=False)
    q = np.array([5, 17, 17, 299, 0, 128], np.uint32)
    a = _sim(circ.n)
    a.run(circ, seed=0)
    ra = a.measure(q, seed=4)
    b = _sim(circ.n)
    b.run(circ, seed=0)
    b.measure_dev(torch.from_numpy(q.view(np.int32)).cuda(), seed=4)
    assert np.array_equal(ra, b.record())


def test_run_twice_is_identical():
    """XOR atomics are order independent: two runs agree bit for bit."""
    circ = C.random_circuit(3000, 30, 0.5, seed=6, measure_every=10, measure_frac=0.05)
    outs = []
    for _ in range(2):
        s = _sim(circ.n)
        rec = s.run(circ, seed=17)
        outs.append((rec, s.export()))
    assert np.array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n,shots", [(5, 1), (64, 64), (300, 200), (130, 1000)])
def test_frames_bit_exact(n, shots):
    circ = C.gate_mix_circuit(n, 18, seed=n + shots, measure_every=4, measure_frac=0.4)
    sim = _sim(n)
    rec = sim.run(circ, seed=21)
    words = sim.sample(shots, seed=33, on_device=False)
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")
    assert not bits[:, shots:].any()  # tail bits beyond `shots` are zero
    ref = O.frames(circ, rec, shots, seed=33)
    assert np.array_equal(bits[:, :shots], ref)
    words_dev = sim.sample(shots, seed=33, on_device=True).cpu().numpy().view(np.uint64)
    assert np.array_equal(words_dev, words)


def test_frames_bit_exact_long_columns():
    """33,000 shots: frame columns of 516 words take the two-gates-in-flight
    frame kernel."""
    circ = C.gate_mix_circuit(37, 10, seed=12, measure_every=3, measure_frac=0.4)
    sim = _sim(37)
    rec = sim.run(circ, seed=5)
    shots = 33_000
    words = sim.sample(shots, seed=8, on_device=False)
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")
    assert not bits[:, shots:].any()
    assert np.array_equal(bits[:, :shots], O.frames(circ, rec, shots, seed=8))


def test_frames_device_resident_replay():
    circ = C.random_circuit(400, 20, 0.5, seed=8, measure_every=5, measure_frac=0.1)
    sim = _sim(circ.n)
    dc = sim.upload(circ)
    rec = sim.run(circ, seed=2, dc=dc)
    shots = 333
    words = sim.sample(shots, seed=4, on_device=False)
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")[:, :shots]
    assert np.array_equal(bits, O.frames(circ, rec, shots, seed=4))


def test_errors_are_reported():
    sim = _sim(10, record_capacity=4)
    with pytest.raises(qs.QsError) as e:
        sim.measure(np.array([10], np.uint32), seed=0)
    assert e.value.code == -1
    with pytest.raises(qs.QsError) as e:
        sim.apply_layer(np.array([[C.H, 2, 0], [C.CX, 2, 3]], np.uint32))
    assert e.value.code == -1
    with pytest.raises(qs.QsError) as e:
        sim.measure(np.arange(5, dtype=np.uint32), seed=0)
    assert e.value.code == -5
    sim.measure(np.arange(4, dtype=np.uint32), seed=0)  # the sim is still usable
    sim.sync()


# ----------------------------------------------------------------------
# Full sizes: sampled rows and properties that hold at any size
# ----------------------------------------------------------------------

def _row_subset_check(circ, layers, nrows, seed):
    rng = np.random.default_rng(seed)
    n = circ.n
    rows = np.sort(rng.choice(2 * n, size=nrows, replace=False)).astype(np.uint32)
    sim = _sim(n)
    dc = sim.upload(circ)
    sim.apply_layers_dev(dc, 0, layers)
    gx, gz, gr = sim.export_rows(rows)
    sub = O.RowSubset(n, rows)
    sub.apply(circ.gates[:circ.layer_ptr[layers]])
    ox, oz, orr = sub.get()
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz) and np.array_equal(gr, orr)
    return sim


def test_row_subset_parity_10k():
    circ = C.workload_10k()
    sim = _row_subset_check(circ, 50, 48, seed=1)
    sim.sync()


def test_full_10k_measurement_properties():
    """10,000 qubits: 50 layers, one 5% round, then the same qubits again
    (all deterministic, same outcomes)."""
    circ = C.workload_10k()
    sim = _sim(circ.n)
    dc = sim.upload(circ)
    sim.apply_layers_dev(dc, 0, 50)
    q = circ.ops[1][1]
    first = sim.measure(q, seed=7)
    again = sim.measure(q, seed=7)
    assert np.array_equal(first, again)
    sim.sync()


@pytest.mark.slow
def test_row_subset_parity_180k():
    circ = C.workload_180k(depth=6)
    sim = _row_subset_check(circ, 6, 24, seed=2)
    sim.sync()


@pytest.mark.slow
def test_full_180k_measure_twice_and_inverse():
    """180,000 qubits: measurements repeated give the same outcomes; a circuit
    followed by its inverse restores the initial rows exactly."""
    n = 180_000
    circ = C.workload_180k(depth=4)
    sim = _sim(n)
    dc = sim.upload(circ)
    sim.apply_layers_dev(dc, 0, 4)
    q = np.array([0, 1, 89_999, 179_999], np.uint32)
    first = sim.measure(q, seed=3)
    again = sim.measure(q, seed=3)
    assert np.array_equal(first, again)
    # inverse check on a fresh sim: layers then their inverses (H, S^dag, CX)
    inv = {C.H: C.H, C.S: C.SDG, C.CX: C.CX}
    sim2 = _sim(n)
    sim2.apply_layers_dev(dc, 0, 4)
    for l in reversed(range(4)):
        g = circ.layer(l).copy()
        g[:, 0] = [inv[int(t)] for t in g[:, 0]]
        sim2.apply_layer(g)
    rows = np.array([0, 5, 179_999, 180_000, 250_000, 359_999], np.uint32)
    x, z, r = sim2.export_rows(rows)
    for i, row in enumerate(rows):
        want_x = np.zeros(n, np.uint8)
        want_z = np.zeros(n, np.uint8)
        if row < n:
            want_x[row] = 1
        else:
            want_z[row - n] = 1
        assert np.array_equal(x[i], want_x) and np.array_equal(z[i], want_z) and r[i] == 0
    sim2.sync()


def _assert_against_job(name, sim, rec):
    """GPU record, kinds and whole tableau against an oracle job's result."""
    want = oracle_jobs.result(name)
    assert int(want["odd"]) == 0 and int(want["det_fail"]) == 0
    assert np.array_equal(rec, want["rec"]), "records differ"
    assert np.array_equal(sim.record_kinds(), want["kinds"]), "kinds differ"
    x, z, r = sim.export()
    assert np.array_equal(np.packbits(x, axis=1), want["x"]), "x bits differ"
    assert np.array_equal(np.packbits(z, axis=1), want["z"]), "z bits differ"
    assert np.array_equal(r, want["r"]), "signs differ"
    return want


def _run_job_program(name):
    prog = oracle_jobs.program(name)
    sim = _sim(prog.n)
    dc = sim.upload(prog)
    rec = sim.run(prog, seed=oracle_jobs.SEEDS[name], dc=dc)
    return sim, rec


@pytest.mark.slow
def test_oracle_parity_on_a_20k_prefix_of_the_180k_workload():
    """The 180,000-qubit workload's generator (p_cx 0.4, seed 3) at 20,000
    qubits: its first two layers, then the first 64 of the final all-qubit
    measurement (blocked, with deterministic steps in between), against the
    oracle: record, kinds and the whole tableau."""
    sim, rec = _run_job_program("prefix_180k_20k")
    want = _assert_against_job("prefix_180k_20k", sim, rec)
    assert 0 < int(want["kinds"].sum()) < len(rec)  # both kinds occur
    sim.sync()


@pytest.mark.slow
def test_oracle_parity_above_the_one_cta_symbolic_limit():
    """The 180,000-qubit workload's generator (p_cx 0.4, seed 3) at 30,000
    qubits, above the 25,600 qubits up to which one CTA runs the symbolic
    pass: the blocked measurement takes the per-step symbolic launches (the
    path of every measurement block at 180,000 qubits) with no flag. Two
    layers, then the first 64 of the final all-qubit measurement, against the
    oracle: record, kinds and the whole tableau."""
    sim, rec = _run_job_program("prefix_180k_30k")
    want = _assert_against_job("prefix_180k_30k", sim, rec)
    assert 0 < int(want["kinds"].sum()) < len(rec)
    sim.sync()


@pytest.mark.slow
def test_oracle_parity_with_a_padded_column_stride():
    """At 16,200 qubits the column stride (2k = 508 words) is padded to 512
    words, a 2 KB multiple, for the layout transposes; the
    NATIVE export keeps 508-word columns. The 180,000-qubit generator's first
    two layers and the first 64 final measurements against the oracle: record,
    kinds and the whole tableau; the NATIVE checkpoint round-trips."""
    sim, rec = _run_job_program("prefix_180k_16200")
    want = _assert_against_job("prefix_180k_16200", sim, rec)
    assert 0 < int(want["kinds"].sum()) < len(rec)
    native, r = sim.checkpoint(qs.QS_LAYOUT_NATIVE)
    k = (16_200 + 63) // 64
    assert len(native) == (2 * 16_200 + 1) * ((2 * k + 3) // 4 * 4)
    b = _sim(16_200)
    b.restore(native, r, qs.QS_LAYOUT_NATIVE)
    for u, v in zip(b.export(), sim.export()):
        assert np.array_equal(u, v)
    sim.sync()


@pytest.mark.slow
def test_10k_schedule_prefix_matches_oracle():
    """The 10,000-qubit workload at full size: layers 0-100 with its two
    windows of 500 mid-circuit measurements (fused gate segments, blocked
    measurement windows), then the first 256 of its final all-qubit round,
    against the oracle: record, kinds and the whole tableau."""
    sim, rec = _run_job_program("schedule_10k")
    want = _assert_against_job("schedule_10k", sim, rec)
    assert len(rec) == 1256 and int(want["kinds"].sum()) > 900
    sim.sync()


@pytest.mark.parametrize("n", [1, 64, 65, 300, 2000, 14080, 14081])
def test_fused_segments_match_per_layer_kernels(n):
    """Device-resident layers run through the fused shared-memory kernel when
    16 n bytes fit (n <= 14,080); with QS_FLAG_NO_FUSION every layer is its own
    kernel. Tableau, record and frame samples must agree bit for bit."""
    circ = C.gate_mix_circuit(n, 12, seed=n + 5, measure_every=6, measure_frac=0.05)
    out = []
    for flags in (0, qs.QS_FLAG_NO_FUSION):
        s = _sim(n, flags=flags)
        dc = s.upload(circ)
        rec = s.run(circ, seed=3, dc=dc)
        words = s.sample(100, seed=9, on_device=False)
        out.append((rec, s.export(), words))
        s.sync()
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][2], out[1][2])


def test_fused_segment_oracle_parity_long_segment():
    """A 60-layer segment through the fused kernel against the oracle."""
    circ = C.random_circuit(1500, 60, 0.5, seed=31, measure_every=30, measure_frac=0.1)
    sim = _sim(circ.n)
    dc = sim.upload(circ)
    rec = sim.run(circ, seed=8, dc=dc)
    o, orec, _ = O.run_circuit(circ, seed=8)
    assert np.array_equal(rec, orec)
    _assert_tableau(sim, o)


@pytest.mark.parametrize("n", [1, 3, 65, 700, 3000, 40000])
def test_pipelined_measurements_match_five_launch_path(n):
    """Two launches per measurement (update; finalize + next gather) against
    the five-launch path, including repeated qubits (deterministic outcomes)
    and a pivot row whose destabilizer partner is measured next."""
    depth = 6 if n > 5000 else 14
    circ = C.random_circuit(n, depth, 0.5, seed=n + 11, final_measure_all=False)
    rng = np.random.default_rng(n)
    q = rng.integers(0, n, size=min(3 * n, 60)).astype(np.uint32)
    q = np.concatenate([q, q[::-1], np.arange(min(n, 40), dtype=np.uint32)])
    outs = []
    for flags in (0, qs.QS_FLAG_UNPIPELINED_MEASURE):
        s = _sim(n, flags=flags)
        dc = s.upload(circ)
        s.apply_layers_dev(dc, 0, depth)
        rec = s.measure(q, seed=19, shot=4)
        rows = np.unique(np.linspace(0, 2 * n - 1, num=min(2 * n, 64)).astype(np.uint32))
        outs.append((rec, s.export_rows(rows)))
        s.sync()
    assert np.array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        assert np.array_equal(a, b)
    if n <= 3000:
        o = O.Oracle(n)
        o.apply(circ.gates)
        orec, _ = o.measure(q, seed=19, shot=4)
        assert np.array_equal(outs[0][0], orec)


@pytest.mark.parametrize("flags", [0, qs.QS_FLAG_STEP_SYMBOLIC], ids=["one-cta-symbolic", "step-symbolic"])
@pytest.mark.parametrize("n,count", [(64, 16), (65, 64), (256, 256), (300, 100), (1024, 16),
                                     (1100, 200), (2000, 150), (4097, 70)])
def test_blocked_measurement_matches_oracle(n, count, flags):
    """Windows of >= 16 measurements on >= 64 qubits go through the blocked
    path (up to 64 measurements per tableau pass); repeated qubits force
    deterministic outcomes that end a block early. QS_FLAG_STEP_SYMBOLIC runs
    the symbolic pass as one launch per step over every row, the code path
    that tableaus above 25,600 qubits (the 180,000-qubit workload) take."""
    circ = C.random_circuit(n, 12, 0.5, seed=n + count, final_measure_all=False)
    rng = np.random.default_rng(count)
    q = rng.permutation(n)[:count].astype(np.uint32)
    q = np.concatenate([q[: count // 2], q[: 7], q[count // 2:]])  # repeats inside the window
    sim = _sim(n, flags=flags)
    dc = sim.upload(circ)
    sim.apply_layers_dev(dc, 0, circ.n_layers)
    rec = sim.measure(q, seed=23, shot=1)
    o = O.Oracle(n)
    o.apply(circ.gates)
    orec, kinds = o.measure(q, seed=23, shot=1)
    assert (kinds == 0).sum() >= 7
    assert np.array_equal(rec, orec)
    _assert_tableau(sim, o)
    sim.sync()


@pytest.mark.parametrize("n,count", [(300, 100), (4097, 150)])
def test_wide_offset_apply_pass_matches_oracle(n, count):
    """The blocked apply pass with 64-bit row offsets (the code path of
    tableaus of 2^32 words and more, forced by QS_FLAG_WIDE_OFFSETS) against
    the oracle and the default 32-bit path."""
    circ = C.random_circuit(n, 10, 0.5, seed=n + 3, final_measure_all=False)
    rng = np.random.default_rng(n)
    q = rng.permutation(n)[:count].astype(np.uint32)
    q = np.concatenate([q[: count // 2], q[: 5], q[count // 2:]])
    o = O.Oracle(n)
    o.apply(circ.gates)
    orec, _ = o.measure(q, seed=6)
    for flags in (qs.QS_FLAG_WIDE_OFFSETS, 0, qs.QS_FLAG_WIDE_OFFSETS | qs.QS_FLAG_STEP_SYMBOLIC):
        sim = _sim(n, flags=flags)
        dc = sim.upload(circ)
        sim.apply_layers_dev(dc, 0, circ.n_layers)
        assert np.array_equal(sim.measure(q, seed=6), orec)
        _assert_tableau(sim, o)
        sim.sync()


@pytest.mark.parametrize("n", [1500, 40000])
def test_blocked_matches_unblocked(n):
    depth = 8
    circ = C.random_circuit(n, depth, 0.5, seed=7, final_measure_all=False)
    q = np.concatenate([np.arange(0, 150, dtype=np.uint32), np.arange(0, 20, dtype=np.uint32),
                        np.arange(n - 90, n, dtype=np.uint32)])
    outs = []
    for flags in (0, qs.QS_FLAG_NO_BLOCKED_MEASURE):
        s = _sim(n, flags=flags)
        dc = s.upload(circ)
        s.apply_layers_dev(dc, 0, depth)
        rec = s.measure(q, seed=5)
        rows = np.unique(np.linspace(0, 2 * n - 1, num=200).astype(np.uint32))
        outs.append((rec, s.export_rows(rows)))
        s.sync()
    assert np.array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n,flags", [(300, 0), (300, qs.QS_FLAG_UNPIPELINED_MEASURE),
                                     (1100, 0), (1100, qs.QS_FLAG_NO_BLOCKED_MEASURE),
                                     (30000, 0)])
def test_measurement_kinds_match_oracle(n, flags):
    """Probabilistic / deterministic kind of every record entry, through the
    blocked, pipelined and five-launch paths, against the oracle's kinds."""
    depth = 10
    circ = C.random_circuit(n, depth, 0.5, seed=n + flags, final_measure_all=False)
    rng = np.random.default_rng(n)
    q = rng.permutation(n)[:min(n, 120)].astype(np.uint32)
    q = np.concatenate([q[:40], q[:10], q[40:]])  # repeats: deterministic outcomes
    sim = _sim(n, flags=flags)
    dc = sim.upload(circ)
    sim.apply_layers_dev(dc, 0, depth)
    rec = sim.measure(q, seed=4)
    kinds = sim.record_kinds()
    if n <= 2000:
        o = O.Oracle(n)
        o.apply(circ.gates)
        orec, okinds = o.measure(q, seed=4)
        assert np.array_equal(rec, orec)
        assert np.array_equal(kinds, okinds)
    else:  # the repeated qubits are deterministic, the first measurements of a dense state are not
        assert (kinds[40:50] == 0).all() and np.array_equal(rec[40:50], rec[:10])
        assert set(np.unique(kinds)) <= {0, 1}
    sim.sync()


def test_qasm_front_end_end_to_end():
    """OpenQASM text over the 11-gate set with interleaved measurements,
    scheduled into windows (Sec. 4.2), run on the GPU against the oracle."""
    from paper_2603_14641_gb300 import qasm
    rng = np.random.default_rng(17)
    n = 37
    names1 = ["x", "y", "z", "h", "s", "sdg"]
    names2 = ["cx", "cy", "cz", "swap", "iswap"]
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg q[{n}];", f"creg c[{n}];"]
    for _ in range(600):
        r = rng.random()
        if r < 0.1:
            q = int(rng.integers(n))
            lines.append(f"measure q[{q}] -> c[{q}];")
        elif r < 0.5:
            a, b = rng.choice(n, size=2, replace=False)
            lines.append(f"{rng.choice(names2)} q[{a}],q[{b}];")
        else:
            lines.append(f"{rng.choice(names1)} q[{int(rng.integers(n))}];")
    circ = qasm.load_circuit("\n".join(lines))
    sim = _sim(circ.n)
    rec = sim.run(circ, seed=4)
    o, orec, _ = O.run_circuit(circ, seed=4)
    assert len(rec) == sum(1 for l in lines if l.startswith("measure"))
    assert np.array_equal(rec, orec)
    _assert_tableau(sim, o)
    words = sim.sample(100, seed=6, on_device=False)
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")[:, :100]
    assert np.array_equal(bits, O.frames(circ, rec, 100, seed=6))
