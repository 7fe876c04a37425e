"""Window scheduling (Sec. 4.2) and the OpenQASM front end, on the CPU."""
import os

import numpy as np
import pytest

from paper_2603_14641_gb300 import qasm, qs
from workloads import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig_schedule_windows.txt")

FIG_QASM = """OPENQASM 2.0;
include "qelib1.inc";
qreg q[5];
creg c[5];
h q[0]; measure q[3] -> c[3];
measure q[1] -> c[1]; s q[4];
s q[0]; s q[2]; s q[3];
cx q[0],q[2]; cx q[3],q[4];
h q[1]; h q[2]; s q[3];
"""

_NAMES = {C.H: "H", C.S: "P", C.CX: "CX", qs.QS_MEASURE: "M"}


def _render(out, ptr, kind):
    lines = []
    for w in range(len(kind)):
        toks = []
        for t, a, b in out[ptr[w]:ptr[w + 1]]:
            nm = _NAMES[int(t)]
            toks.append(f"{nm}{a},{b}" if nm == "CX" else f"{nm}{a}")
        # gates of one window are disjoint, so their order inside it is free
        lines.append(f"W{w} " + " ".join(sorted(toks, key=lambda t: (int(t.lstrip("HPCXM").split(",")[0]), t))))
    return lines


def test_paper_figure_schedule():
    want = [l.strip() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    n, ops = qasm.parse(FIG_QASM)
    assert n == 5
    out, ptr, kind = qs.qs_schedule_windows(n, ops)
    assert _render(out, ptr, kind) == want
    assert list(kind) == [0, 1, 1, 0, 0, 0]


def _check_schedule(n, ops, out, ptr, kind, merge):
    # a permutation of the input
    assert sorted(map(tuple, ops.tolist())) == sorted(map(tuple, out.tolist()))
    # per-qubit order kept
    def per_qubit(seq):
        d = {}
        for i, (t, a, b) in enumerate(seq.tolist()):
            d.setdefault(a, []).append((t, a, b))
            if t in C.TWO_QUBIT:
                d.setdefault(b, []).append((t, a, b))
        return d
    assert per_qubit(ops) == per_qubit(out)
    for w in range(len(kind)):
        seg = out[ptr[w]:ptr[w + 1]]
        if kind[w] == 0:
            qs_ = list(seg[:, 1]) + [b for t, a, b in seg if t in C.TWO_QUBIT]
            assert len(qs_) == len(set(qs_)), "gates of a window must act on disjoint qubits"
            assert (seg[:, 0] != qs.QS_MEASURE).all()
        else:
            assert (seg[:, 0] == qs.QS_MEASURE).all()
            if not merge:
                assert len(seg) == 1


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("merge", [False, True])
def test_random_programs_schedule_validly(seed, merge):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    ops = []
    for _ in range(300):
        r = rng.random()
        if r < 0.15:
            ops.append((qs.QS_MEASURE, int(rng.integers(n)), 0))
        elif r < 0.55:
            a, b = rng.choice(n, size=2, replace=False)
            ops.append((int(rng.choice(C.TWO_QUBIT)), int(a), int(b)))
        else:
            ops.append((int(rng.integers(1, 7)), int(rng.integers(n)), 0))
    ops = np.array(ops, np.uint32)
    out, ptr, kind = qs.qs_schedule_windows(n, ops, merge)
    _check_schedule(n, ops, out, ptr, kind, merge)
    # gate windows are maximal: re-run the greedy on the output and compare counts
    circ = qs.scheduled_circuit(n, ops, merge)
    assert circ.n_gates == int((ops[:, 0] != qs.QS_MEASURE).sum())


def test_layered_circuit_round_trips_to_the_same_layers():
    c = C.random_circuit(50, 12, 0.5, seed=3, final_measure_all=False)
    ops = c.gates.copy()
    out, ptr, kind = qs.qs_schedule_windows(50, ops)
    # a layered circuit of disjoint layers is rescheduled with no more layers than it had
    assert (kind == 0).all() and len(kind) <= c.n_layers


def test_qasm_errors_and_registers():
    with pytest.raises(qasm.QasmError):
        qasm.parse("qreg q[2]; t q[0];")
    with pytest.raises(qasm.QasmError):
        qasm.parse("qreg q[2]; h q[2];")
    n, ops = qasm.parse("qreg a[2]; qreg b[3]; cx a[1], b[2]; measure b[0] -> c[0]; // done")
    assert n == 5
    assert ops.tolist() == [[C.CX, 1, 4], [qs.QS_MEASURE, 2, 0]]
    with pytest.raises(qs.QsError):
        qs.qs_schedule_windows(3, np.array([[C.CX, 1, 1]], np.uint32))
