"""OpenQASM 2.0 subset front end (the paper's benchmarks are Qiskit-generated
OpenQASM circuits over the 11-gate Clifford set plus measurements, Sec. 6).

Accepted: OPENQASM/include headers, qreg and creg declarations (several
registers are laid out one after another), the gates x y z h s sdg cx cy cz
swap iswap on single qubits, `measure q[i] -> c[j];`, `barrier` (ignored: the
scheduler already respects per-qubit order) and // comments. Anything else is
an error. The result is an ordered op list for qs_schedule_windows.
"""
from __future__ import annotations

import re
from typing import Dict, List, Tuple

import numpy as np

from . import qs

_GATE = {"x": 1, "y": 2, "z": 3, "h": 4, "s": 5, "sdg": 6, "cx": 7, "cy": 8, "cz": 9,
         "swap": 10, "iswap": 11, "id": 0}
_TWO = {"cx", "cy", "cz", "swap", "iswap"}
_ARG = re.compile(r"^([A-Za-z_]\w*)\[(\d+)\]$")


class QasmError(ValueError):
    pass


def parse(text: str) -> Tuple[int, np.ndarray]:
    """Returns (n_qubits, ops) with ops rows (type, q0, q1), type 12 = measure."""
    qregs: Dict[str, Tuple[int, int]] = {}
    nq = 0
    ops: List[Tuple[int, int, int]] = []
    body = re.sub(r"//[^\n]*", "", text)
    for lineno, stmt in enumerate(s.strip() for s in body.split(";")):
        if not stmt:
            continue
        low = stmt.lower()
        if low.startswith("openqasm") or low.startswith("include") or low.startswith("creg"):
            continue
        if low.startswith("qreg"):
            m = re.match(r"^qreg\s+([A-Za-z_]\w*)\[(\d+)\]$", stmt)
            if not m:
                raise QasmError(f"bad qreg: {stmt!r}")
            qregs[m.group(1)] = (nq, int(m.group(2)))
            nq += int(m.group(2))
            continue
        if low.startswith("barrier"):
            continue

        def qubit(tok: str) -> int:
            m = _ARG.match(tok.strip())
            if not m or m.group(1) not in qregs:
                raise QasmError(f"bad qubit {tok!r} in {stmt!r}")
            base, size = qregs[m.group(1)]
            i = int(m.group(2))
            if i >= size:
                raise QasmError(f"qubit index out of range in {stmt!r}")
            return base + i

        if low.startswith("measure"):
            m = re.match(r"^measure\s+(\S+)\s*->\s*(\S+)$", stmt)
            if not m:
                raise QasmError(f"bad measure: {stmt!r}")
            ops.append((qs.QS_MEASURE, qubit(m.group(1)), 0))
            continue
        m = re.match(r"^([a-z]+)\s+(.+)$", stmt)
        if not m or m.group(1) not in _GATE:
            raise QasmError(f"unsupported statement: {stmt!r}")
        name, args = m.group(1), [a for a in m.group(2).split(",")]
        if name in _TWO:
            if len(args) != 2:
                raise QasmError(f"{name} needs two qubits: {stmt!r}")
            ops.append((_GATE[name], qubit(args[0]), qubit(args[1])))
        else:
            if len(args) != 1:
                raise QasmError(f"{name} takes one qubit: {stmt!r}")
            if name != "id":
                ops.append((_GATE[name], qubit(args[0]), 0))
    return nq, np.array(ops, np.uint32).reshape(-1, 3)


def load_circuit(text: str, merge_measurements: bool = False, name: str = ""):
    """Parse, schedule into maximal windows (Sec. 4.2) and return a Circuit."""
    n, ops = parse(text)
    return qs.scheduled_circuit(n, ops, merge_measurements, name)
