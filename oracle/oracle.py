"""Python access to the CPU oracle (plain CHP over unpacked rows, chp_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle exists to check the CUDA path. Only the
tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
product path never does. It shares no code with the CUDA library.

The oracle follows the paper (arXiv 2603.14641) step by step: the extended
tableau of Sec. 2.5 (Eq. 7), the gate rules of Sec. 2.4 (Eq. 4), the CHP
measurement of Sec. 2.5 and the Pauli-frame sampler of Sec. 5 (Alg. 9).
Parity pins for each function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chp_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile chp_oracle.c into oracle/_lib/liboracle.so (gcc, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def load_library(path: str):
    """ctypes handle of an oracle library at `path` with its signatures set."""
    L = ctypes.CDLL(path)
    L.oracle_new.restype = ctypes.c_void_p
    L.oracle_new.argtypes = [ctypes.c_int]
    L.oracle_free.argtypes = [ctypes.c_void_p]
    L.oracle_reset.argtypes = [ctypes.c_void_p, _u8p]
    L.oracle_get.argtypes = [ctypes.c_void_p, _u8p, _u8p, _u8p]
    L.oracle_set.argtypes = [ctypes.c_void_p, _u8p, _u8p, _u8p]
    L.oracle_gate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.oracle_apply.argtypes = [ctypes.c_void_p, _u32p, ctypes.c_long]
    L.oracle_measure.restype = ctypes.c_int
    L.oracle_measure.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
    L.oracle_measure_many.argtypes = [ctypes.c_void_p, _u32p, ctypes.c_long, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _u8p,
                                      _u8p]
    L.oracle_odd_phase_count.restype = ctypes.c_long
    L.oracle_odd_phase_count.argtypes = [ctypes.c_void_p]
    L.oracle_det_check_fail.restype = ctypes.c_long
    L.oracle_det_check_fail.argtypes = [ctypes.c_void_p]
    L.oracle_last_kind.restype = ctypes.c_int
    L.oracle_last_kind.argtypes = [ctypes.c_void_p]
    L.oracle_new_subset.restype = ctypes.c_void_p
    L.oracle_new_subset.argtypes = [ctypes.c_int, _u32p, ctypes.c_int]
    L.oracle_get_subset.argtypes = [ctypes.c_void_p, _u8p, _u8p, _u8p]
    L.oracle_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
    L.oracle_coin.restype = ctypes.c_int
    L.oracle_coin.argtypes = [ctypes.c_uint64] * 3
    L.oracle_frame_word.restype = ctypes.c_uint64
    L.oracle_frame_word.argtypes = [ctypes.c_uint64] * 4
    L.oracle_frames.restype = ctypes.c_int
    L.oracle_frames.argtypes = [ctypes.c_int, _u32p, _u32p, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                ctypes.c_long, _u8p, ctypes.c_long, ctypes.c_uint64, _u8p]
    L.oracle_noise_draw.restype = None
    L.oracle_noise_draw.argtypes = [ctypes.c_uint64] * 4 + [_u64p, _u64p]
    L.oracle_noise_threshold.restype = ctypes.c_uint64
    L.oracle_noise_threshold.argtypes = [ctypes.c_double]
    L.oracle_inv_new.restype = ctypes.c_void_p
    L.oracle_inv_new.argtypes = [ctypes.c_int]
    L.oracle_inv_free.argtypes = [ctypes.c_void_p]
    L.oracle_inv_reset.argtypes = [ctypes.c_void_p, _u8p]
    L.oracle_inv_get.argtypes = [ctypes.c_void_p, _u8p, _u8p, _u8p, _u8p]
    L.oracle_inv_gate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.oracle_inv_apply.argtypes = [ctypes.c_void_p, _u32p, ctypes.c_long]
    L.oracle_inv_measure.restype = ctypes.c_int
    L.oracle_inv_measure.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_uint64]
    L.oracle_inv_measure_many.argtypes = [ctypes.c_void_p, _u32p, ctypes.c_long, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_uint64, _u8p, _u8p]
    L.oracle_inv_last_kind.restype = ctypes.c_int
    L.oracle_inv_last_kind.argtypes = [ctypes.c_void_p]
    L.oracle_inv_odd_count.restype = ctypes.c_long
    L.oracle_inv_odd_count.argtypes = [ctypes.c_void_p]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def philox4x64_10(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.array(ctr, np.uint64)
    k = np.array(key, np.uint64)
    out = np.zeros(4, np.uint64)
    lib().oracle_philox4x64_10(_p(c, _u64p), _p(k, _u64p), _p(out, _u64p))
    return out


def coin(seed: int, shot: int, m: int) -> int:
    return int(lib().oracle_coin(seed, shot, m))


def frame_word(seed: int, e: int, q: int, j: int) -> int:
    return int(lib().oracle_frame_word(seed, e, q, j))


class Oracle:
    """A CHP tableau on n qubits (rows 0..n-1 destabilizers, n..2n-1 stabilizers)."""

    def __init__(self, n: int, initstate: Optional[np.ndarray] = None):
        self.n = int(n)
        self._h = lib().oracle_new(self.n)
        if not self._h:
            raise MemoryError("oracle_new failed")
        self.midx = 0  # next record index
        if initstate is not None:
            self.reset(initstate)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_free(h)
            self._h = None

    def reset(self, initstate: Optional[np.ndarray] = None) -> None:
        if initstate is None:
            lib().oracle_reset(self._h, None)
        else:
            s = np.ascontiguousarray(initstate, np.uint8)
            lib().oracle_reset(self._h, _p(s, _u8p))
        self.midx = 0

    def gate(self, t: int, a: int, b: int = 0) -> None:
        lib().oracle_gate(self._h, int(t), int(a), int(b))

    def apply(self, gates: np.ndarray) -> None:
        g = np.ascontiguousarray(gates, np.uint32)
        if g.size:
            lib().oracle_apply(self._h, _p(g, _u32p), g.shape[0])

    def measure(self, qubits, seed: int, shot: int = 0, force_zero: bool = False):
        """Measures qubits in order; returns (outcomes uint8, kinds uint8 with
        1 = probabilistic). Record indices continue from self.midx."""
        q = np.ascontiguousarray(qubits, np.uint32)
        out = np.zeros(len(q), np.uint8)
        kind = np.zeros(len(q), np.uint8)
        if len(q):
            lib().oracle_measure_many(self._h, _p(q, _u32p), len(q), seed, shot, self.midx,
                                      int(force_zero), _p(out, _u8p), _p(kind, _u8p))
        self.midx += len(q)
        return out, kind

    def get(self):
        """Returns (x, z, r): x, z of shape (2n, n) uint8, r of shape (2n,)."""
        n = self.n
        x = np.zeros((2 * n, n), np.uint8)
        z = np.zeros((2 * n, n), np.uint8)
        r = np.zeros(2 * n, np.uint8)
        lib().oracle_get(self._h, _p(x, _u8p), _p(z, _u8p), _p(r, _u8p))
        return x, z, r

    def set(self, x: np.ndarray, z: np.ndarray, r: np.ndarray) -> None:
        x = np.ascontiguousarray(x, np.uint8)
        z = np.ascontiguousarray(z, np.uint8)
        r = np.ascontiguousarray(r, np.uint8)
        assert x.shape == (2 * self.n, self.n) and z.shape == x.shape and r.shape == (2 * self.n,)
        lib().oracle_set(self._h, _p(x, _u8p), _p(z, _u8p), _p(r, _u8p))

    @property
    def odd_phase_count(self) -> int:
        return int(lib().oracle_odd_phase_count(self._h))

    @property
    def det_check_fail(self) -> int:
        return int(lib().oracle_det_check_fail(self._h))


class RowSubset:
    """Chosen generator rows of the n-qubit tableau, evolved under gates only
    (gate rules act row by row, Sec. 2.4). rows: ids in 0..2n-1 (destabilizers
    0..n-1, stabilizers n..2n-1) of the initial tableau |0...0>."""

    def __init__(self, n: int, rows):
        self.n = int(n)
        self.rows = np.ascontiguousarray(rows, np.uint32)
        self._h = lib().oracle_new_subset(self.n, _p(self.rows, _u32p), len(self.rows))
        if not self._h:
            raise MemoryError("oracle_new_subset failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_free(h)
            self._h = None

    def apply(self, gates: np.ndarray) -> None:
        g = np.ascontiguousarray(gates, np.uint32)
        if g.size:
            lib().oracle_apply(self._h, _p(g, _u32p), g.shape[0])

    def get(self):
        nr = len(self.rows)
        x = np.zeros((nr, self.n), np.uint8)
        z = np.zeros((nr, self.n), np.uint8)
        r = np.zeros(nr, np.uint8)
        lib().oracle_get_subset(self._h, _p(x, _u8p), _p(z, _u8p), _p(r, _u8p))
        return x, z, r


def run_circuit(circuit, seed: int, shot: int = 0, force_zero: bool = False,
                oracle: Optional[Oracle] = None):
    """Runs a workloads.circuits.Circuit single-shot (the noiseless reference
    shot: noise ops act on the frames only). Returns (oracle, record, kinds)
    with the record in program order."""
    o = oracle or Oracle(circuit.n)
    rec, kinds = [], []
    for op in circuit.ops:
        if op[0] == "layers":
            o.apply(circuit.gates[circuit.layer_ptr[op[1]]:circuit.layer_ptr[op[2]]])
        elif op[0] == "measure":
            out, kind = o.measure(op[1], seed, shot, force_zero)
            rec.append(out)
            kinds.append(kind)
    rec = np.concatenate(rec) if rec else np.zeros(0, np.uint8)
    kinds = np.concatenate(kinds) if kinds else np.zeros(0, np.uint8)
    return o, rec, kinds


def noise_draw(seed: int, e: int, i: int, s: int):
    """(u, v) draws of target i of noise op e in shot s: u (32 bits) decides
    whether the channel fires, v (64 bits) picks the Pauli."""
    u, v = ctypes.c_uint64(), ctypes.c_uint64()
    lib().oracle_noise_draw(seed, e, i, s, ctypes.byref(u), ctypes.byref(v))
    return u.value, v.value


def noise_threshold(p: float) -> int:
    """floor(p * 2^32) for 0 <= p < 1 (0 for p <= 0, 2^32 for p >= 1)."""
    return int(lib().oracle_noise_threshold(p))


def frames(circuit, ref: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Pauli-frame samples of `circuit` (Sec. 5), with its noise ops applied to
    the frames. Returns (M, shots) uint8."""
    kinds, a, b, qlist, nk, npr = [], [], [], [], [], []
    qoff = 0
    M = 0
    for op in circuit.ops:
        if op[0] == "layers":
            kinds.append(0)
            a.append(int(circuit.layer_ptr[op[1]]))
            b.append(int(circuit.layer_ptr[op[2]]))
            nk.append(0)
            npr.append(0.0)
            continue
        targets = np.asarray(op[1] if op[0] == "measure" else op[3], np.uint32)
        kinds.append(1 if op[0] == "measure" else 2)
        nk.append(0 if op[0] == "measure" else int(op[1]))
        npr.append(0.0 if op[0] == "measure" else float(op[2]))
        a.append(qoff)
        qoff += len(targets)
        b.append(qoff)
        qlist.append(targets)
        if op[0] == "measure":
            M += len(targets)
    q = np.concatenate(qlist) if qlist else np.zeros(1, np.uint32)
    ref = np.ascontiguousarray(ref, np.uint8)
    assert len(ref) == M
    g = np.ascontiguousarray(circuit.gates, np.uint32)
    if g.size == 0:
        g = np.zeros((1, 3), np.uint32)
    out = np.zeros((max(M, 1), shots), np.uint8)
    ka = np.array(kinds, np.intc)
    aa = np.array(a, np.int_)
    ba = np.array(b, np.int_)
    nka = np.array(nk, np.intc)
    npa = np.array(npr, np.float64)
    rc = lib().oracle_frames(circuit.n, _p(g, _u32p), _p(q, _u32p),
                             ka.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             aa.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                             ba.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                             nka.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             npa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(kinds),
                             _p(ref if M else np.zeros(1, np.uint8), _u8p), shots, seed,
                             _p(out, _u8p))
    if rc != 0:
        raise MemoryError("oracle_frames failed")
    return out[:M]


class InverseOracle:
    """The inverse tableau with qubit-indexed signs (Sec. 3.2, Alg. 1): for
    the Clifford C preparing the state, the images C^dag Z_q C (sign ss[q], x
    bits XS[:, q], z bits XD[:, q]) and C^dag X_q C (sign sd[q], bits ZS[:, q],
    ZD[:, q]); its bits are the extended tableau's (rows 0..n-1 destabilizers,
    n..2n-1 stabilizers). Measurement follows Alg. 1 with the keyed coin."""

    def __init__(self, n: int, initstate: Optional[np.ndarray] = None):
        self.n = int(n)
        self._h = lib().oracle_inv_new(self.n)
        if not self._h:
            raise MemoryError("oracle_inv_new failed")
        self.midx = 0
        if initstate is not None:
            self.reset(initstate)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_inv_free(h)
            self._h = None

    def reset(self, initstate: Optional[np.ndarray] = None) -> None:
        if initstate is None:
            lib().oracle_inv_reset(self._h, None)
        else:
            s = np.ascontiguousarray(initstate, np.uint8)
            lib().oracle_inv_reset(self._h, _p(s, _u8p))
        self.midx = 0

    def gate(self, t: int, a: int, b: int = 0) -> None:
        lib().oracle_inv_gate(self._h, int(t), int(a), int(b))

    def apply(self, gates: np.ndarray) -> None:
        g = np.ascontiguousarray(gates, np.uint32)
        if g.size:
            lib().oracle_inv_apply(self._h, _p(g, _u32p), g.shape[0])

    def measure(self, qubits, seed: int, shot: int = 0):
        q = np.ascontiguousarray(qubits, np.uint32)
        out = np.zeros(len(q), np.uint8)
        kind = np.zeros(len(q), np.uint8)
        if len(q):
            lib().oracle_inv_measure_many(self._h, _p(q, _u32p), len(q), seed, shot, self.midx,
                                          _p(out, _u8p), _p(kind, _u8p))
        self.midx += len(q)
        return out, kind

    def get(self):
        """(x, z, ss, sd): x, z of shape (2n, n), ss and sd of shape (n,)."""
        n = self.n
        x = np.zeros((2 * n, n), np.uint8)
        z = np.zeros((2 * n, n), np.uint8)
        ss = np.zeros(n, np.uint8)
        sd = np.zeros(n, np.uint8)
        lib().oracle_inv_get(self._h, _p(x, _u8p), _p(z, _u8p), _p(ss, _u8p), _p(sd, _u8p))
        return x, z, ss, sd

    @property
    def odd_count(self) -> int:
        return int(lib().oracle_inv_odd_count(self._h))


def run_circuit_inverse(circuit, seed: int, shot: int = 0,
                        oracle: Optional[InverseOracle] = None):
    """As run_circuit, on the inverse tableau (Alg. 1's measurement).
    Returns (oracle, record, kinds)."""
    o = oracle or InverseOracle(circuit.n)
    rec, kinds = [], []
    for op in circuit.ops:
        if op[0] == "layers":
            o.apply(circuit.gates[circuit.layer_ptr[op[1]]:circuit.layer_ptr[op[2]]])
        elif op[0] == "measure":
            out, kind = o.measure(op[1], seed, shot)
            rec.append(out)
            kinds.append(kind)
    rec = np.concatenate(rec) if rec else np.zeros(0, np.uint8)
    kinds = np.concatenate(kinds) if kinds else np.zeros(0, np.uint8)
    return o, rec, kinds
