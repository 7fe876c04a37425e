"""Long oracle runs for the GPU parity tests, computed in spawned processes.

The oracle needs minutes for the largest parity cases (unpacked CHP at 10,000
to 30,000 qubits), while the GPU side needs a second. When a GPU test run
selects one of these cases, conftest.py starts a small process pool ("spawn",
before any GPU call) at collection time and submits the jobs below, so the
oracle runs overlap the rest of the GPU suite; each test then waits for its
job. Every job calls only oracle/ and workloads/ and returns the oracle's
record, measurement kinds and whole tableau (bits packed with numpy to keep
the transfer small).
"""
from __future__ import annotations

import multiprocessing as mp
from typing import Dict, Optional

import numpy as np

# test node id suffix -> job name
JOB_OF_TEST = {
    "test_oracle_parity_on_a_20k_prefix_of_the_180k_workload": "prefix_180k_20k",
    "test_oracle_parity_above_the_one_cta_symbolic_limit": "prefix_180k_30k",
    "test_10k_schedule_prefix_matches_oracle": "schedule_10k",
    "test_oracle_parity_with_a_padded_column_stride": "prefix_180k_16200",
}


def program(name: str):
    """The circuit of a job (layers and measurement rounds), shared by the test
    and the oracle job so both run the same program."""
    from workloads import circuits as C
    if name in ("prefix_180k_20k", "prefix_180k_30k", "prefix_180k_16200"):
        n = {"prefix_180k_20k": 20_000, "prefix_180k_30k": 30_000, "prefix_180k_16200": 16_200}[name]
        circ = C.workload_180k_prefix(n, depth=2)
        q = np.arange(64, dtype=np.uint32)
        return C.Circuit(n=n, gates=circ.gates, layer_ptr=circ.layer_ptr,
                         ops=[("layers", 0, 2), ("measure", q)])
    if name == "schedule_10k":
        # the 10,000-qubit workload's schedule up to layer 100 (two windows of
        # 500 measurements), then the first 256 of its final all-qubit round
        circ = C.workload_10k()
        ops = list(circ.ops[:4])
        assert ops[0] == ("layers", 0, 50) and ops[2] == ("layers", 50, 100)
        final = circ.ops[-1][1]
        ops.append(("measure", np.asarray(final[:256], np.uint32)))
        return C.Circuit(n=circ.n, gates=circ.gates, layer_ptr=circ.layer_ptr, ops=ops)
    raise KeyError(name)


SEEDS = {"prefix_180k_20k": 7, "prefix_180k_30k": 11, "schedule_10k": 29, "prefix_180k_16200": 13}


def run_job(name: str) -> Dict[str, np.ndarray]:
    from oracle import oracle as O
    prog = program(name)
    o, rec, kinds = O.run_circuit(prog, seed=SEEDS[name])
    x, z, r = o.get()
    return {"rec": rec, "kinds": kinds, "x": np.packbits(x, axis=1), "z": np.packbits(z, axis=1),
            "r": r, "n": np.array(prog.n), "odd": np.array(o.odd_phase_count),
            "det_fail": np.array(o.det_check_fail)}


_pool = None
_futures: Dict[str, "mp.pool.AsyncResult"] = {}


def start(names) -> None:
    """Starts the pool (spawn) and submits the named jobs; idempotent."""
    global _pool
    names = [n for n in names if n not in _futures]
    if not names:
        return
    if _pool is None:
        _pool = mp.get_context("spawn").Pool(processes=min(3, max(1, len(names))))
    for n in names:
        _futures[n] = _pool.apply_async(run_job, (n,))


def result(name: str, timeout: Optional[float] = 3600.0) -> Dict[str, np.ndarray]:
    """The job's result, computed in the pool if it was started, else here."""
    f = _futures.get(name)
    if f is None:
        return run_job(name)
    return f.get(timeout)


def shutdown() -> None:
    global _pool
    if _pool is not None:
        _pool.terminate()
        _pool.join()
        _pool = None
    _futures.clear()
