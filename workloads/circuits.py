"""Seeded synthetic workloads: random Clifford layers and measurement schedules.

This module only draws inputs. It holds none of the simulation method's
arithmetic, so both the oracle and the CUDA path can consume the very same
circuits. The paper's Qiskit benchmark suites are not available; these
circuits stand in for them with the same qubit ranges and depths (Sec. 6,
"Benchmarks": 100 to 180,000 qubits, depths 100/500/1000, random Clifford
gates plus randomized Z-measurements).

Layer recipe (one layer = gates on pairwise disjoint qubits, Sec. 4.2 windows):
  * a seeded random permutation of the n qubits is cut into consecutive pairs;
  * each pair becomes a CX with probability p_cx, with control and target
    chosen by a fair coin;
  * otherwise each qubit of the pair independently draws H, S or identity
    with probability 1/3 each; an odd leftover qubit takes the same draw;
  * identities are not emitted (they change nothing and are not counted).

Gate records are rows (type, q0, q1) of uint32. Gate type codes are part of
the input format; the C header of the CUDA library declares the same values
and a test checks that the two agree.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

# Gate type codes of the input format (the paper's 11-gate set plus identity,
# Sec. 6 "Benchmarks").
I, X, Y, Z, H, S, SDG, CX, CY, CZ, SWAP, ISWAP = range(12)
GATE_NAMES = ["I", "X", "Y", "Z", "H", "S", "SDG", "CX", "CY", "CZ", "SWAP", "ISWAP"]
TWO_QUBIT = (CX, CY, CZ, SWAP, ISWAP)

# Pauli noise channel codes (frames only; the C header declares the same values)
NOISE_X, NOISE_Y, NOISE_Z, DEPOLARIZE1, DEPOLARIZE2 = range(5)
NOISE_NAMES = ["X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2"]

_SINGLE_DRAW = np.array([H, S, I], dtype=np.uint32)


@dataclass
class Circuit:
    """A layered circuit plus its Z-measurement schedule.

    gates:     (G, 3) uint32 rows (type, q0, q1); q1 is 0 for one-qubit gates.
    layer_ptr: (L+1,) int64; layer l is gates[layer_ptr[l]:layer_ptr[l+1]].
    ops:       program order, a list of ("layers", l0, l1),
               ("measure", qubits uint32 array) and
               ("noise", kind, p, targets uint32 array) entries; noise acts
               on the sampled shots only (pairs of targets for DEPOLARIZE2).
    """

    n: int
    gates: np.ndarray
    layer_ptr: np.ndarray
    ops: List[Tuple] = field(default_factory=list)
    name: str = ""

    @property
    def n_layers(self) -> int:
        return len(self.layer_ptr) - 1

    def layer(self, l: int) -> np.ndarray:
        return self.gates[self.layer_ptr[l]:self.layer_ptr[l + 1]]

    @property
    def n_gates(self) -> int:
        return int(self.layer_ptr[-1])

    @property
    def n_measurements(self) -> int:
        return int(sum(len(op[1]) for op in self.ops if op[0] == "measure"))


def random_layer(rng: np.random.Generator, n: int, p_cx: float) -> np.ndarray:
    """One random layer on n qubits (recipe in the module docstring)."""
    perm = rng.permutation(n).astype(np.uint32)
    npair = n // 2
    a = perm[0:2 * npair:2]
    b = perm[1:2 * npair:2]
    is_cx = rng.random(npair) < p_cx
    flip = rng.random(npair) < 0.5
    single = _SINGLE_DRAW[rng.integers(0, 3, size=n)]
    ctrl = np.where(flip, b, a)[is_cx]
    targ = np.where(flip, a, b)[is_cx]
    cx = np.stack([np.full(len(ctrl), CX, np.uint32), ctrl, targ], axis=1)
    # one-qubit draws: both members of non-CX pairs, then the odd leftover
    nc = ~is_cx
    sq_q = np.concatenate([a[nc], b[nc], perm[2 * npair:]])
    sq_t = np.concatenate([single[0:2 * npair:2][nc], single[1:2 * npair:2][nc],
                           single[2 * npair:]])
    keep = sq_t != I
    sq = np.stack([sq_t[keep], sq_q[keep], np.zeros(int(keep.sum()), np.uint32)], axis=1)
    return np.concatenate([cx, sq], axis=0).astype(np.uint32)


def _schedule(n: int, depth: int, rng_m: np.random.Generator, measure_every: int,
              measure_frac: float, final_measure_all: bool) -> List[Tuple]:
    """Program order of layer runs and measurement rounds (see random_circuit)."""
    ops: List[Tuple] = []
    start = 0
    cnt = int(np.floor(measure_frac * n))
    for l in range(1, depth + 1):
        periodic = measure_every > 0 and l % measure_every == 0 and cnt > 0
        last = l == depth
        if periodic or last:
            if l > start:
                ops.append(("layers", start, l))
                start = l
            if last and final_measure_all:
                ops.append(("measure", np.arange(n, dtype=np.uint32)))
            elif periodic:
                q = np.sort(rng_m.choice(n, size=cnt, replace=False)).astype(np.uint32)
                ops.append(("measure", q))
    if start < depth:
        ops.append(("layers", start, depth))
    return ops


def random_circuit(n: int, depth: int, p_cx: float, seed: int,
                   measure_every: int = 0, measure_frac: float = 0.0,
                   final_measure_all: bool = True, name: str = "") -> Circuit:
    """Random layered Clifford circuit with an optional measurement schedule.

    After every `measure_every`-th layer (if > 0) floor(measure_frac * n)
    distinct qubits drawn uniformly are measured in ascending order; when
    `final_measure_all`, every qubit is measured in ascending order after the
    last layer (and a periodic measurement that falls on the last layer is
    replaced by it).
    """
    ss = np.random.SeedSequence(seed)
    rng_g, rng_m = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(2)]
    layers = [random_layer(rng_g, n, p_cx) for _ in range(depth)]
    layer_ptr = np.zeros(depth + 1, np.int64)
    layer_ptr[1:] = np.cumsum([len(l) for l in layers])
    gates = np.concatenate(layers, axis=0) if layers else np.zeros((0, 3), np.uint32)
    ops = _schedule(n, depth, rng_m, measure_every, measure_frac, final_measure_all)
    return Circuit(n=n, gates=np.ascontiguousarray(gates), layer_ptr=layer_ptr, ops=ops,
                   name=name)


def gate_mix_circuit(n: int, depth: int, seed: int, measure_every: int = 0,
                     measure_frac: float = 0.0, final_measure_all: bool = True) -> Circuit:
    """Random layers drawing uniformly from the whole 11-gate set (Sec. 6).

    Each layer pairs qubits as in `random_layer`; a pair becomes a uniformly
    drawn two-qubit gate (CX, CY, CZ, SWAP, ISWAP, random orientation) with
    probability 5/11, otherwise each qubit draws uniformly from
    {X, Y, Z, H, S, SDG}.
    """
    ss = np.random.SeedSequence(seed)
    rng_g, rng_m = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(2)]
    two = np.array(TWO_QUBIT, np.uint32)
    one = np.array([X, Y, Z, H, S, SDG], np.uint32)
    layers = []
    for _ in range(depth):
        perm = rng_g.permutation(n).astype(np.uint32)
        npair = n // 2
        a, b = perm[0:2 * npair:2], perm[1:2 * npair:2]
        is2 = rng_g.random(npair) < 5.0 / 11.0
        flip = rng_g.random(npair) < 0.5
        t2 = two[rng_g.integers(0, len(two), size=npair)]
        t1 = one[rng_g.integers(0, len(one), size=n)]
        q0 = np.where(flip, b, a)[is2]
        q1 = np.where(flip, a, b)[is2]
        g2 = np.stack([t2[is2], q0, q1], axis=1)
        nc = ~is2
        sq_q = np.concatenate([a[nc], b[nc], perm[2 * npair:]])
        sq_t = np.concatenate([t1[0:2 * npair:2][nc], t1[1:2 * npair:2][nc], t1[2 * npair:]])
        g1 = np.stack([sq_t, sq_q, np.zeros(len(sq_q), np.uint32)], axis=1)
        layers.append(np.concatenate([g2, g1]).astype(np.uint32))
    layer_ptr = np.zeros(depth + 1, np.int64)
    layer_ptr[1:] = np.cumsum([len(l) for l in layers])
    gates = np.concatenate(layers) if layers else np.zeros((0, 3), np.uint32)
    ops = _schedule(n, depth, rng_m, measure_every, measure_frac, final_measure_all)
    return Circuit(n=n, gates=np.ascontiguousarray(gates), layer_ptr=layer_ptr, ops=ops,
                   name="gate-mix")


# --------------------------------------------------------------------------
# The workloads the simulator is measured on (seeds fixed here).
# --------------------------------------------------------------------------

def workload_256() -> Circuit:
    """256 qubits, depth 100, p_cx 0.5, seed 1; final Z-measurement of all."""
    return random_circuit(256, 100, 0.5, seed=1, name="n256_d100")


def workload_10k() -> Circuit:
    """10,000 qubits, depth 1,000, p_cx 0.5, seed 2; a random 5% of qubits
    measured after every 50th layer and all qubits after the last."""
    return random_circuit(10_000, 1_000, 0.5, seed=2, measure_every=50, measure_frac=0.05,
                          name="n10k_d1000")


def workload_180k(depth: int = 1_000) -> Circuit:
    """180,000 qubits, depth 1,000, p_cx 0.4, seed 3; final measurement of all."""
    return random_circuit(180_000, depth, 0.4, seed=3, name="n180k_d1000")


def workload_180k_prefix(n: int = 20_000, depth: int = 100) -> Circuit:
    """The same generator and seed at a smaller qubit count (a prefix the
    oracle can finish) for the 180k-qubit workload."""
    return random_circuit(n, depth, 0.4, seed=3, name=f"n{n}_d{depth}_seed3")


def batch_sizes(count: int = 512, seed: int = 4, lo: int = 50, hi: int = 5000) -> np.ndarray:
    """Qubit counts of the batched workload, log-uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


def batch_workload(count: int = 512, seed: int = 4, depth: int = 200) -> List[Circuit]:
    """Independent circuits, n log-uniform 50..5,000, depth 200, p_cx 0.5,
    10% of qubits (distinct, ascending) measured after every 10th layer."""
    sizes = batch_sizes(count, seed)
    return [random_circuit(int(nq), depth, 0.5, seed=seed * 100_003 + i, measure_every=10,
                           measure_frac=0.1, final_measure_all=False, name=f"batch{i}")
            for i, nq in enumerate(sizes)]


@dataclass
class Request:
    arrival_s: float
    n: int
    depth: int
    shots: int
    seed: int


def serving_requests(count: int, rate_hz: float, seed: int = 5) -> List[Request]:
    """Poisson arrivals; n log-uniform 100..20,000, depth uniform 100..500,
    shots log-uniform 1e3..1e6; each circuit ends with a full Z-measurement."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps)
    n = np.round(np.exp(rng.uniform(np.log(100), np.log(20_000), size=count))).astype(int)
    d = rng.integers(100, 501, size=count)
    f = np.round(np.exp(rng.uniform(np.log(1e3), np.log(1e6), size=count))).astype(int)
    return [Request(float(t[i]), int(n[i]), int(d[i]), int(f[i]), seed * 1_000_003 + i)
            for i in range(count)]


def with_circuit_noise(circ: Circuit, p_gate: float, p_meas: float) -> Circuit:
    """The same circuit with circuit-level Pauli noise on its sampled shots:
    after every layer, DEPOLARIZE1(p_gate) on the qubits of its one-qubit
    gates and DEPOLARIZE2(p_gate) on the pairs of its two-qubit gates; before
    every measurement window, X_ERROR(p_meas) on the measured qubits."""
    ops: List[Tuple] = []
    for op in circ.ops:
        if op[0] == "layers":
            for l in range(op[1], op[2]):
                ops.append(("layers", l, l + 1))
                g = circ.layer(l)
                two = np.isin(g[:, 0], TWO_QUBIT)
                one = ~two & (g[:, 0] != I)
                if p_gate > 0 and one.any():
                    ops.append(("noise", DEPOLARIZE1, p_gate, np.ascontiguousarray(g[one, 1])))
                if p_gate > 0 and two.any():
                    ops.append(("noise", DEPOLARIZE2, p_gate,
                                np.ascontiguousarray(g[two, 1:3].reshape(-1))))
        elif op[0] == "measure":
            if p_meas > 0 and len(op[1]):
                ops.append(("noise", NOISE_X, p_meas, np.unique(np.asarray(op[1], np.uint32))))
            ops.append(op)
        else:
            ops.append(op)
    return Circuit(n=circ.n, gates=circ.gates, layer_ptr=circ.layer_ptr, ops=ops,
                   name=(circ.name + f"_noise{p_gate:g}") if circ.name else "")
