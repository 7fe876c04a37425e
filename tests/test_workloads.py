"""The seeded input generators against their stated recipe (no GPU): layers
are perfect matchings of disjoint qubits with CX probability p and H/S/I
draws of 1/3 each, the measurement schedules of the 10,000- and
180,000-qubit workloads, the batch and serving distributions, and the
circuit-level noise decoration."""
import numpy as np

from workloads import circuits as C


def _binomial_ok(count, trials, p, sigmas=6.0):
    mean = trials * p
    sd = np.sqrt(trials * p * (1 - p))
    return abs(count - mean) <= sigmas * sd + 1


def test_layers_are_disjoint_matchings_with_the_stated_gate_mix():
    rng = np.random.Generator(np.random.PCG64(11))
    for n, p in [(1, 0.5), (2, 1.0), (7, 0.0), (1001, 0.5), (20_000, 0.4)]:
        g = C.random_layer(rng, n, p)
        two = g[:, 0] == C.CX
        used = np.concatenate([g[:, 1], g[two, 2]])
        assert len(np.unique(used)) == len(used), "a qubit appears twice in one layer"
        assert used.max(initial=0) < n
        assert set(np.unique(g[:, 0])) <= {C.CX, C.H, C.S}  # identities are not emitted
        assert np.all(g[~two, 2] == 0)
        ncx = int(two.sum())
        assert _binomial_ok(ncx, n // 2, p)
        if p == 1.0:
            assert ncx == n // 2
        if p == 0.0:
            assert ncx == 0
        # every qubit outside a CX drew H, S or I with probability 1/3 each
        free = n - 2 * ncx
        nh, ns = int((g[:, 0] == C.H).sum()), int((g[:, 0] == C.S).sum())
        assert _binomial_ok(nh, free, 1 / 3) and _binomial_ok(ns, free, 1 / 3)


def test_cx_orientation_is_a_fair_coin_and_layers_differ():
    rng = np.random.Generator(np.random.PCG64(5))
    g = np.concatenate([C.random_layer(rng, 4000, 0.5) for _ in range(10)])
    cx = g[g[:, 0] == C.CX]
    assert _binomial_ok(int((cx[:, 1] < cx[:, 2]).sum()), len(cx), 0.5)
    a = C.random_circuit(300, 2, 0.5, seed=1, final_measure_all=False)
    assert not np.array_equal(a.layer(0), a.layer(1))


def test_generation_is_seeded_and_reproducible():
    a = C.random_circuit(500, 20, 0.5, seed=9, measure_every=5, measure_frac=0.1)
    b = C.random_circuit(500, 20, 0.5, seed=9, measure_every=5, measure_frac=0.1)
    c = C.random_circuit(500, 20, 0.5, seed=10, measure_every=5, measure_frac=0.1)
    assert np.array_equal(a.gates, b.gates) and np.array_equal(a.layer_ptr, b.layer_ptr)
    assert all(x[0] == y[0] and (x[0] != "measure" or np.array_equal(x[1], y[1]))
               for x, y in zip(a.ops, b.ops))
    assert not np.array_equal(a.gates, c.gates)


def test_10k_schedule():
    """After layers 50, 100, ..., 950: 500 distinct qubits in ascending order;
    after layer 1000 every qubit in ascending order (19,500 measurements)."""
    circ = C.workload_10k()
    assert circ.n == 10_000 and circ.n_layers == 1_000
    meas = [op for op in circ.ops if op[0] == "measure"]
    assert len(meas) == 20 and circ.n_measurements == 19_500
    ends = [op[2] for op in circ.ops if op[0] == "layers"]
    assert ends == list(range(50, 1_001, 50))
    for q in (op[1] for op in meas[:-1]):
        assert len(q) == 500 and np.all(np.diff(q.astype(np.int64)) > 0) and q.max() < 10_000
    assert np.array_equal(meas[-1][1], np.arange(10_000))
    # layers run in order and cover the circuit
    runs = [(op[1], op[2]) for op in circ.ops if op[0] == "layers"]
    assert runs[0][0] == 0 and all(x[1] == y[0] for x, y in zip(runs, runs[1:]))


def test_180k_layer_shape():
    """About 36k CX, 36k H and 36k S per layer at 180,000 qubits, p_cx 0.4;
    the 20,000-qubit prefix uses the same generator and seed."""
    circ = C.workload_180k(depth=3)
    assert circ.n == 180_000 and circ.ops[-1][0] == "measure"
    assert np.array_equal(circ.ops[-1][1], np.arange(180_000))
    for l in range(3):
        g = circ.layer(l)
        for t, want in [(C.CX, 36_000), (C.H, 36_000), (C.S, 36_000)]:
            assert abs(int((g[:, 0] == t).sum()) - want) < 1_500
    pre = C.workload_180k_prefix(20_000, depth=2)
    assert pre.n == 20_000 and pre.n_layers == 2


def test_batch_and_serving_distributions():
    sizes = C.batch_sizes()
    assert len(sizes) == 512 and sizes.min() >= 50 and sizes.max() <= 5000
    # log-uniform on [50, 5000]: median sqrt(50 * 5000) = 500, mean 4950 / ln 100 = 1075
    assert 380 < np.median(sizes) < 660
    assert 900 < sizes.mean() < 1250
    reqs = C.serving_requests(400, rate_hz=20.0)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0) and 0.04 < np.mean(np.diff(t)) < 0.06
    n = np.array([r.n for r in reqs])
    d = np.array([r.depth for r in reqs])
    f = np.array([r.shots for r in reqs])
    assert n.min() >= 100 and n.max() <= 20_000 and d.min() >= 100 and d.max() <= 500
    assert f.min() >= 1_000 and f.max() <= 1_000_000


def test_circuit_noise_decoration():
    circ = C.random_circuit(60, 4, 0.5, seed=2, measure_every=2, measure_frac=0.25)
    noisy = C.with_circuit_noise(circ, 0.01, 0.02)
    kinds = [op[0] for op in noisy.ops]
    assert kinds.count("layers") == circ.n_layers  # one op per layer
    gates_seen = 0
    for i, op in enumerate(noisy.ops):
        if op[0] == "layers":
            g = circ.layer(op[1])
            gates_seen += len(g)
            two = g[g[:, 0] == C.CX]
            one = g[(g[:, 0] != C.CX) & (g[:, 0] != C.I)]
            follow = [x for x in noisy.ops[i + 1:i + 3] if x[0] == "noise"]
            d1 = [x for x in follow if x[1] == C.DEPOLARIZE1]
            d2 = [x for x in follow if x[1] == C.DEPOLARIZE2]
            if len(one):
                assert np.array_equal(np.sort(d1[0][3]), np.sort(one[:, 1])) and d1[0][2] == 0.01
            if len(two):
                pairs = d2[0][3].reshape(-1, 2)
                assert np.array_equal(pairs, two[:, 1:3]) and d2[0][2] == 0.01
        if op[0] == "measure":
            prev = noisy.ops[i - 1]
            assert prev[0] == "noise" and prev[1] == C.NOISE_X and prev[2] == 0.02
            assert np.array_equal(prev[3], op[1])
    assert gates_seen == circ.n_gates
    assert noisy.n_measurements == circ.n_measurements
