"""GPU test of the serving loop: requests admitted while others run overlap on
the device, and every request's single-shot record and frame samples are
bit-identical to the same request served alone and to the oracle (CHP record
and Pauli-frame samples of Sec. 2.5 and Sec. 5 under the same keys)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2603_14641_gb300 import serve  # noqa: E402
from workloads import circuits as C  # noqa: E402


def _requests(count=12, seed=3):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(50), np.log(1500))))
        d = int(rng.integers(20, 61))
        shots = int(np.exp(rng.uniform(np.log(100), np.log(3000))))
        circ = C.random_circuit(n, d, 0.5, seed=seed * 1000 + i)
        reqs.append(serve.Request(i, 0.002 * i, circ, shots, seed=77 + i))
    return reqs


def test_results_identical_alone_and_in_the_mix():
    reqs = _requests()
    mixed, summ, stats = serve.serve(reqs, slots=4, budget_bytes=1 << 30, device="cuda:0")
    assert stats["peak_active"] >= 2, "no two requests overlapped"
    assert stats["peak_bytes"] <= stats["budget_bytes"]
    assert summ["requests"] == len(reqs)
    for r in reqs:
        alone, _, _ = serve.serve([serve.Request(r.rid, 0.0, r.circuit, r.shots, r.seed)],
                                  slots=1, budget_bytes=1 << 30, device="cuda:0")
        a, m = alone[0], mixed[r.rid]
        assert np.array_equal(a.record, m.record), f"request {r.rid}: record differs"
        assert np.array_equal(a.samples, m.samples), f"request {r.rid}: samples differ"
        # the served request against the oracle under the same keys: the
        # record is measured with key (seed, 0), the shots with seed + 1
        _, orec, _ = O.run_circuit(r.circuit, seed=r.seed, shot=0)
        assert np.array_equal(m.record, orec), f"request {r.rid}: record differs from the oracle"
        bits = np.unpackbits(m.samples.view(np.uint8), axis=1, bitorder="little")
        assert not bits[:, r.shots:].any()
        want = O.frames(r.circuit, orec, r.shots, seed=r.seed + 1)
        assert np.array_equal(bits[:, :r.shots], want), f"request {r.rid}: samples differ from the oracle"


def test_tight_budget_serialises_but_completes():
    reqs = _requests(6, seed=4)
    ex = serve.GpuExecutor(1, device="cuda:0")
    biggest = max(ex.footprint(r) for r in reqs)
    res, summ, stats = serve.serve(reqs, slots=4, budget_bytes=biggest, device="cuda:0")
    assert len(res) == len(reqs) and stats["peak_bytes"] <= biggest


def test_batched_small_requests_match_alone_and_oracle():
    """Small requests that wait together are served as one batch (one
    persistent launch for their reference shots, one launch for their shots);
    each result equals the request served alone and the oracle's."""
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(10):
        n = int(rng.integers(20, 1000))
        circ = C.random_circuit(n, int(rng.integers(10, 40)), 0.5, seed=500 + i)
        reqs.append(serve.Request(i, 0.0, circ, int(rng.integers(1, 3000)), seed=300 + i))
    res, summ, stats = serve.serve(reqs, slots=1, budget_bytes=1 << 30, device="cuda:0")
    assert stats["batches"] >= 1 and stats["batched_requests"] >= 2
    for r in reqs:
        alone, _, _ = serve.serve([serve.Request(r.rid, 0.0, r.circuit, r.shots, r.seed)], slots=1,
                                  budget_bytes=1 << 30, device="cuda:0", batching=False)
        a, m = alone[0], res[r.rid]
        assert np.array_equal(a.record, m.record) and np.array_equal(a.samples, m.samples), r.rid
        _, orec, _ = O.run_circuit(r.circuit, seed=r.seed, shot=0)
        assert np.array_equal(m.record, orec)
        bits = np.unpackbits(m.samples.view(np.uint8), axis=1, bitorder="little")
        assert np.array_equal(bits[:, :r.shots], O.frames(r.circuit, orec, r.shots, seed=r.seed + 1))
