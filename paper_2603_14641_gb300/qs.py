"""Thin Python binding of libqs (include/qs.h): argument marshalling only.

Every step of the simulation runs in the CUDA library. The module-level
functions carry the C names; `Simulator` bundles them with PyTorch, which only
provides device memory (the sim workspace, device-resident circuits, frame
buffers) and the CUDA stream. There is no CPU fallback: if libqs.so cannot be
built or loaded, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

QS_OK = 0
ERRORS = {-1: "QS_ERR_ARG", -2: "QS_ERR_OOM", -3: "QS_ERR_CUDA", -4: "QS_ERR_TIMEOUT",
          -5: "QS_ERR_SIZE", -6: "QS_ERR_STATE", -7: "QS_ERR_INTERNAL"}
QS_LAYOUT_ROWS_PACKED = 0
QS_LAYOUT_NATIVE = 1

GATES = dict(I=0, X=1, Y=2, Z=3, H=4, S=5, SDG=6, CX=7, CY=8, CZ=9, SWAP=10, ISWAP=11)
QS_MEASURE = 12
# Pauli noise channels of qs_sim_noise (frames only)
QS_NOISE_X, QS_NOISE_Y, QS_NOISE_Z, QS_NOISE_DEPOLARIZE1, QS_NOISE_DEPOLARIZE2 = range(5)


class QsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class qs_key(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("shot", ctypes.c_uint64)]


class qs_options(ctypes.Structure):
    _fields_ = [("record_capacity", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class qs_gate(ctypes.Structure):
    _fields_ = [("type", ctypes.c_uint32), ("q0", ctypes.c_uint32), ("q1", ctypes.c_uint32)]


class qs_batch_circuit(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("n_layers", ctypes.c_uint32),
                ("gates", ctypes.c_void_p), ("layer_ptr", ctypes.c_void_p),
                ("n_rounds", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("round_layers", ctypes.c_void_p), ("round_meas", ctypes.c_void_p),
                ("qubits", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("shot", ctypes.c_uint64)]


class qs_batch_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("words_per_block", ctypes.c_uint32), ("fuse_depth", ctypes.c_uint32),
                ("spin_limit", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t

# name -> (restype, argtypes); the exported C-ABI of libqs
SIGNATURES = {
    "qs_version": (ctypes.c_char_p, []),
    "qs_last_error": (ctypes.c_char_p, []),
    "qs_sim_required_bytes": (_sz, [_u32, _vp]),
    "qs_sim_create": (ctypes.c_int, [_u32, _vp, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "qs_sim_destroy": (ctypes.c_int, [_vp]),
    "qs_sim_reset": (ctypes.c_int, [_vp, _vp]),
    "qs_sim_apply_layer": (ctypes.c_int, [_vp, _vp, _u32]),
    "qs_pack_layers": (ctypes.c_int, [_u32, _vp, _vp, _u32, _vp]),
    "qs_sim_apply_layers_dev": (ctypes.c_int, [_vp, _vp, _vp, _u32, _u32]),
    "qs_sim_measure": (ctypes.c_int, [_vp, _vp, _u32, qs_key, _vp]),
    "qs_sim_measure_dev": (ctypes.c_int, [_vp, _vp, _u32, qs_key]),
    "qs_sim_noise": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, _vp, _u32]),
    "qs_sim_record_kinds": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_uint64, _vp]),
    "qs_sim_tableau_import": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp,
                                             ctypes.c_uint64]),
    "qs_sim_num_measurements": (_u64, [_vp]),
    "qs_sim_record": (ctypes.c_int, [_vp, _u64, _u64, _vp]),
    "qs_sim_sample_required_bytes": (_sz, [_vp, _u64]),
    "qs_sim_sample": (ctypes.c_int, [_vp, _u64, _u64, _vp, _sz, _vp, _sz]),
    "qs_sim_tableau_export": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _sz, ctypes.POINTER(_sz)]),
    "qs_sim_sample_noalloc": (ctypes.c_int, [_vp, _u64, _u64, _vp, _sz]),
    "qs_sim_export_rows": (ctypes.c_int, [_vp, _vp, _u32, _vp]),
    "qs_sim_sync": (ctypes.c_int, [_vp]),
    "qs_sim_launch_count": (_u64, [_vp]),
    "qs_sim_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "qs_sim_qubit_signs": (ctypes.c_int, [_vp, _vp, _sz]),
    "qs_sim_timing": (ctypes.c_int, [_vp, _vp, _vp, _u32]),
    "qs_schedule_windows": (ctypes.c_int, [_u32, _vp, _u32, ctypes.c_int, _vp, _vp, _vp,
                                           ctypes.POINTER(_u32)]),
    "qs_schedule_last_error": (ctypes.c_char_p, []),
    "qs_batch_required_bytes": (_sz, [_u32, _vp]),
    "qs_batch_create": (ctypes.c_int, [_u32, _vp, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "qs_batch_destroy": (ctypes.c_int, [_vp]),
    "qs_batch_run": (ctypes.c_int, [_vp, _vp, _u32]),
    "qs_batch_sync": (ctypes.c_int, [_vp]),
    "qs_batch_record": (ctypes.c_int, [_vp, _u32, _vp, _sz]),
    "qs_batch_export_rows": (ctypes.c_int, [_vp, _u32, _vp, _u32, _vp]),
    "qs_batch_autotune": (ctypes.c_int, [_vp, _u32, ctypes.c_char_p, _vp]),
    "qs_batch_last_error": (ctypes.c_char_p, []),
    "qs_batch_sample": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
}

_lib = None


def lib(build_if_missing: bool = True):
    """Loads libqs.so (building it in-tree first if needed); raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libqs.so not found at {path}; run paper_2603_14641_gb300/build.py")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != QS_OK:
        raise QsError(rc, where, lib().qs_last_error().decode())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------------------
# Module-level functions with the C names (argument marshalling only)
# ----------------------------------------------------------------------

def qs_version() -> str:
    return lib().qs_version().decode()


QS_FLAG_NO_FUSION = 1
QS_FLAG_UNPIPELINED_MEASURE = 2
QS_FLAG_NO_BLOCKED_MEASURE = 4
QS_FLAG_WIDE_OFFSETS = 8
QS_FLAG_STEP_SYMBOLIC = 16
QS_FLAG_INVERSE_TABLEAU = 32


def qs_sim_required_bytes(n: int, record_capacity: int = 0, flags: int = 0) -> int:
    opt = qs_options(record_capacity, flags, 0)
    return int(lib().qs_sim_required_bytes(n, ctypes.byref(opt)))


def qs_sim_create(n: int, stream: int = 0, workspace: int = 0, workspace_bytes: int = 0,
                  record_capacity: int = 0, flags: int = 0) -> int:
    opt = qs_options(record_capacity, flags, 0)
    h = ctypes.c_void_p()
    _check(lib().qs_sim_create(n, ctypes.byref(opt), ctypes.c_void_p(stream or None),
                               ctypes.c_void_p(workspace or None), workspace_bytes,
                               ctypes.byref(h)), "qs_sim_create")
    return h.value


def qs_sim_destroy(sim: int) -> None:
    _check(lib().qs_sim_destroy(ctypes.c_void_p(sim)), "qs_sim_destroy")


def qs_sim_reset(sim: int, initstate: Optional[np.ndarray] = None) -> None:
    a = None if initstate is None else np.ascontiguousarray(initstate, np.uint8)
    _check(lib().qs_sim_reset(ctypes.c_void_p(sim), None if a is None else _ptr(a)), "qs_sim_reset")


def _as_gates(gates: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.uint32).reshape(-1, 3))
    return g


def qs_sim_apply_layer(sim: int, gates: np.ndarray) -> None:
    g = _as_gates(gates)
    _check(lib().qs_sim_apply_layer(ctypes.c_void_p(sim), _ptr(g), g.shape[0]), "qs_sim_apply_layer")


def qs_pack_layers(n: int, gates: np.ndarray, layer_ptr: np.ndarray) -> np.ndarray:
    g = _as_gates(gates)
    lp = np.ascontiguousarray(layer_ptr, np.int64)
    out = np.zeros(2 * max(int(lp[-1]), 1), np.uint32)
    _check(lib().qs_pack_layers(n, _ptr(g) if g.size else None, _ptr(lp), len(lp) - 1, _ptr(out)),
           "qs_pack_layers")
    return out[:2 * int(lp[-1])]


def qs_sim_apply_layers_dev(sim: int, packed_dev: int, layer_ptr: np.ndarray, l_begin: int,
                            l_end: int) -> None:
    lp = np.ascontiguousarray(layer_ptr, np.int64)
    _check(lib().qs_sim_apply_layers_dev(ctypes.c_void_p(sim), ctypes.c_void_p(packed_dev),
                                         _ptr(lp), l_begin, l_end), "qs_sim_apply_layers_dev")


def qs_sim_measure(sim: int, qubits: np.ndarray, seed: int, shot: int = 0,
                   want_outcomes: bool = True) -> Optional[np.ndarray]:
    q = np.ascontiguousarray(qubits, np.uint32)
    out = np.zeros(len(q), np.uint8) if want_outcomes else None
    _check(lib().qs_sim_measure(ctypes.c_void_p(sim), _ptr(q) if len(q) else None, len(q),
                                qs_key(seed, shot), _ptr(out) if (want_outcomes and len(q)) else None),
           "qs_sim_measure")
    return out


def qs_sim_measure_dev(sim: int, qubits_dev: int, count: int, seed: int, shot: int = 0) -> None:
    _check(lib().qs_sim_measure_dev(ctypes.c_void_p(sim), ctypes.c_void_p(qubits_dev), count,
                                    qs_key(seed, shot)), "qs_sim_measure_dev")


def qs_sim_tableau_import(sim: int, packed: np.ndarray, record: np.ndarray,
                          layout: int = QS_LAYOUT_ROWS_PACKED) -> None:
    """Restores a checkpoint: `packed` as returned by qs_sim_tableau_export in
    `layout`, `record` the 0/1 record bytes so far."""
    t = np.ascontiguousarray(packed, np.uint64)
    r = np.ascontiguousarray(record, np.uint8)
    _check(lib().qs_sim_tableau_import(ctypes.c_void_p(sim), int(layout),
                                       t.ctypes.data, t.nbytes, r.ctypes.data if len(r) else None,
                                       len(r)), "qs_sim_tableau_import")


def qs_sim_noise(sim: int, kind: int, p: float, targets) -> None:
    t = np.ascontiguousarray(targets, np.uint32)
    _check(lib().qs_sim_noise(ctypes.c_void_p(sim), int(kind), float(p),
                              _ptr(t) if len(t) else None, len(t)), "qs_sim_noise")


def qs_sim_num_measurements(sim: int) -> int:
    return int(lib().qs_sim_num_measurements(ctypes.c_void_p(sim)))


def qs_sim_record(sim: int, first: int = 0, count: Optional[int] = None) -> np.ndarray:
    if count is None:
        count = qs_sim_num_measurements(sim) - first
    out = np.zeros(max(count, 1), np.uint8)
    _check(lib().qs_sim_record(ctypes.c_void_p(sim), first, count, _ptr(out)), "qs_sim_record")
    return out[:count]


def qs_sim_record_kinds(sim: int, first: int = 0, count: Optional[int] = None) -> np.ndarray:
    """1 = probabilistic, 0 = deterministic, 2 = restored from a checkpoint."""
    if count is None:
        count = qs_sim_num_measurements(sim) - first
    out = np.zeros(max(count, 1), np.uint8)
    _check(lib().qs_sim_record_kinds(ctypes.c_void_p(sim), first, count, _ptr(out)),
           "qs_sim_record_kinds")
    return out[:count]


def qs_sim_sample_required_bytes(sim: int, shots: int) -> int:
    return int(lib().qs_sim_sample_required_bytes(ctypes.c_void_p(sim), shots))


def qs_sim_sample(sim: int, shots: int, seed: int, record: int, record_words: int,
                  frame_ws: int = 0, frame_ws_bytes: int = 0) -> None:
    _check(lib().qs_sim_sample(ctypes.c_void_p(sim), shots, seed, ctypes.c_void_p(record or None),
                               record_words, ctypes.c_void_p(frame_ws or None), frame_ws_bytes),
           "qs_sim_sample")


def qs_sim_sample_noalloc(sim: int, shots: int, seed: int, record: int, record_words: int) -> None:
    """qs_sim_sample with the frames in libqs's fixed static device array
    (allocates nothing; see include/qs.h for the size limit and sharing)."""
    _check(lib().qs_sim_sample_noalloc(ctypes.c_void_p(sim), shots, seed,
                                       ctypes.c_void_p(record or None), record_words),
           "qs_sim_sample_noalloc")


def qs_sim_tableau_export(sim: int, layout: int = QS_LAYOUT_ROWS_PACKED, out=None):
    """The tableau in `layout` as uint64 words: into `out` (a numpy array or a
    torch tensor, host or device, of at least the needed bytes) if given, else
    into a new numpy array."""
    need = ctypes.c_size_t(0)
    _check(lib().qs_sim_tableau_export(ctypes.c_void_p(sim), int(layout), None, 0,
                                       ctypes.byref(need)), "qs_sim_tableau_export")
    if out is None:
        out = np.zeros(need.value // 8, np.uint64)
    if isinstance(out, np.ndarray):
        ptr, nbytes = out.ctypes.data, out.nbytes
    else:
        ptr, nbytes = out.data_ptr(), out.numel() * out.element_size()
    _check(lib().qs_sim_tableau_export(ctypes.c_void_p(sim), int(layout), ctypes.c_void_p(ptr),
                                       nbytes, None), "qs_sim_tableau_export")
    return out


def qs_sim_export_rows(sim: int, rows: np.ndarray, n: int):
    """Selected generator rows -> (x, z, r) uint8 arrays of shapes (R, n), (R, n), (R,)."""
    r = np.ascontiguousarray(rows, np.uint32)
    k = (n + 63) // 64
    buf = np.zeros((max(len(r), 1), 2 * k + 1), np.uint64)
    _check(lib().qs_sim_export_rows(ctypes.c_void_p(sim), _ptr(r) if len(r) else None, len(r),
                                    _ptr(buf)), "qs_sim_export_rows")
    buf = buf[:len(r)]
    bits = np.unpackbits(np.ascontiguousarray(buf[:, :2 * k]).view(np.uint8).reshape(len(r), -1),
                         axis=1, bitorder="little")
    x = np.ascontiguousarray(bits[:, :n])
    z = np.ascontiguousarray(bits[:, 64 * k:64 * k + n])
    return x, z, (buf[:, 2 * k] & 1).astype(np.uint8)


def qs_sim_sync(sim: int) -> None:
    _check(lib().qs_sim_sync(ctypes.c_void_p(sim)), "qs_sim_sync")


def qs_sim_launch_count(sim: int) -> int:
    return int(lib().qs_sim_launch_count(ctypes.c_void_p(sim)))


QS_TIME_KINDS = ["gates", "transpose", "blk_symbolic", "blk_pivot_rows", "blk_apply", "blk_signs",
                 "measure_single", "sample"]


def qs_sim_qubit_signs(sim: int, n: int):
    """Inverse-tableau mode: (S_S, S_D) as uint8 arrays of n bits (signs of
    C^dag Z_q C and C^dag X_q C)."""
    w = (n + 63) // 64
    buf = np.zeros(2 * w, np.uint64)
    _check(lib().qs_sim_qubit_signs(ctypes.c_void_p(sim), _ptr(buf), 2 * w), "qs_sim_qubit_signs")
    bits = np.unpackbits(buf.view(np.uint8), bitorder="little")
    return bits[:n].copy(), bits[64 * w:64 * w + n].copy()


def qs_sim_set_timing(sim: int, on: bool) -> None:
    _check(lib().qs_sim_set_timing(ctypes.c_void_p(sim), int(bool(on))), "qs_sim_set_timing")


def qs_sim_timing(sim: int) -> dict:
    """{kind: (milliseconds, timed groups)} for the QS_TIME_* kinds."""
    k = len(QS_TIME_KINDS)
    ms = np.zeros(k, np.float64)
    cnt = np.zeros(k, np.uint64)
    _check(lib().qs_sim_timing(ctypes.c_void_p(sim), _ptr(ms), _ptr(cnt), k), "qs_sim_timing")
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(QS_TIME_KINDS)}


def unpack_rows(buf: np.ndarray, n: int):
    """ROWS_PACKED export -> (x, z, r) uint8 arrays of shapes (2n, n), (2n, n), (2n,)."""
    k = (n + 63) // 64
    rows = buf[:2 * n * 2 * k].reshape(2 * n, 2 * k)
    bits = np.unpackbits(rows.view(np.uint8).reshape(2 * n, 2 * k, 8)[..., :], axis=2,
                         bitorder="little").reshape(2 * n, 2 * k * 64)
    x = bits[:, :n]
    z = bits[:, k * 64:k * 64 + n]
    sw = (2 * n + 63) // 64
    sig = np.unpackbits(buf[2 * n * 2 * k:2 * n * 2 * k + sw].view(np.uint8), bitorder="little")
    return np.ascontiguousarray(x), np.ascontiguousarray(z), np.ascontiguousarray(sig[:2 * n])


def unpack_native(buf: np.ndarray, n: int):
    """NATIVE export -> (x, z, r) uint8 arrays of shapes (2n, n), (2n, n), (2n,)
    in generator order (destabilizers, then stabilizers)."""
    k = (n + 63) // 64
    W = (2 * k + 3) // 4 * 4
    cols = np.ascontiguousarray(buf[:(2 * n + 1) * W]).reshape(2 * n + 1, W)
    bits = np.unpackbits(cols.view(np.uint8), axis=1, bitorder="little")  # (2n + 1, 64 W)
    gen = np.concatenate([np.arange(n), 64 * k + np.arange(n)])  # packed number of generator i
    x = bits[:n, gen].T
    z = bits[n:2 * n, gen].T
    return np.ascontiguousarray(x), np.ascontiguousarray(z), np.ascontiguousarray(bits[2 * n, gen])


# ----------------------------------------------------------------------
# Convenience wrapper (PyTorch supplies device memory and the stream)
# ----------------------------------------------------------------------

@dataclass
class DeviceCircuit:
    """A circuit's gate layers packed and resident in device memory."""
    n: int
    packed: "object"        # torch.uint32-compatible int32 device tensor
    layer_ptr: np.ndarray   # int64 host offsets
    n_gates: int


class Simulator:
    def __init__(self, n: int, device: str = "cuda", stream=None, record_capacity: int = 0,
                 flags: int = 0):
        import torch
        self.torch = torch
        self.n = int(n)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = qs_sim_required_bytes(self.n, record_capacity, flags)
        self.flags = flags
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.sim = qs_sim_create(self.n, self.stream.cuda_stream, self.workspace.data_ptr(), nbytes,
                                 record_capacity, flags)
        self._keep = []

    def close(self):
        if getattr(self, "sim", None):
            qs_sim_destroy(self.sim)
            self.sim = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, initstate=None):
        self._keep.clear()
        qs_sim_reset(self.sim, initstate)

    def apply_layer(self, gates):
        qs_sim_apply_layer(self.sim, gates)

    def upload(self, circuit) -> DeviceCircuit:
        packed = qs_pack_layers(circuit.n, circuit.gates, circuit.layer_ptr)
        t = self.torch.from_numpy(packed.view(np.int32)).to(self.device)
        return DeviceCircuit(circuit.n, t, np.asarray(circuit.layer_ptr, np.int64), circuit.n_gates)

    def apply_layers_dev(self, dc: DeviceCircuit, l0: int, l1: int):
        self._keep.append(dc.packed)
        qs_sim_apply_layers_dev(self.sim, dc.packed.data_ptr(), dc.layer_ptr, l0, l1)

    def measure(self, qubits, seed: int, shot: int = 0, want_outcomes: bool = True):
        return qs_sim_measure(self.sim, qubits, seed, shot, want_outcomes)

    def measure_dev(self, qubits_dev, seed: int, shot: int = 0):
        self._keep.append(qubits_dev)
        qs_sim_measure_dev(self.sim, qubits_dev.data_ptr(), qubits_dev.numel(), seed, shot)

    def checkpoint(self, layout: int = QS_LAYOUT_ROWS_PACKED):
        """(packed tableau, record): everything a later run needs to resume."""
        return qs_sim_tableau_export(self.sim, layout), self.record()

    def restore(self, packed, record, layout: int = QS_LAYOUT_ROWS_PACKED):
        qs_sim_tableau_import(self.sim, packed, record, layout)

    def noise(self, kind: int, p: float, targets):
        """Appends a Pauli noise channel (QS_NOISE_*) for the sampled shots."""
        qs_sim_noise(self.sim, kind, p, targets)

    def run(self, circuit, seed: int, shot: int = 0, dc: Optional[DeviceCircuit] = None):
        """Runs circuit.ops; layers from host (or from `dc` if given); noise ops
        go to the op log for sample(). Returns the record."""
        for op in circuit.ops:
            if op[0] == "layers":
                if dc is not None:
                    self.apply_layers_dev(dc, op[1], op[2])
                else:
                    for l in range(op[1], op[2]):
                        self.apply_layer(circuit.layer(l))
            elif op[0] == "noise":
                self.noise(op[1], op[2], op[3])
            else:
                self.measure(op[1], seed, shot, want_outcomes=False)
        return self.record()

    @property
    def num_measurements(self) -> int:
        return qs_sim_num_measurements(self.sim)

    def qubit_signs(self):
        """Inverse-tableau mode: (S_S, S_D) uint8 arrays of n bits."""
        return qs_sim_qubit_signs(self.sim, self.n)

    def record(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        return qs_sim_record(self.sim, first, count)

    def record_kinds(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        return qs_sim_record_kinds(self.sim, first, count)

    def export(self):
        return unpack_rows(qs_sim_tableau_export(self.sim), self.n)

    def sample(self, shots: int, seed: int, on_device: bool = True):
        """Frame samples; returns (M, ceil(shots/64)) uint64 words (torch on device
        or numpy on host)."""
        M = self.num_measurements
        ow = (shots + 63) // 64
        fb = qs_sim_sample_required_bytes(self.sim, shots)
        fws = self.torch.empty(fb, dtype=self.torch.uint8, device=self.device)
        if on_device:
            out = self.torch.zeros((max(M, 1), ow), dtype=self.torch.int64, device=self.device)
            qs_sim_sample(self.sim, shots, seed, out.data_ptr(), M * ow, fws.data_ptr(), fb)
            return out[:M]
        out = np.zeros((max(M, 1), ow), np.uint64)
        qs_sim_sample(self.sim, shots, seed, out.ctypes.data, M * ow, fws.data_ptr(), fb)
        return out[:M]

    def export_rows(self, rows):
        return qs_sim_export_rows(self.sim, rows, self.n)

    def sync(self):
        qs_sim_sync(self.sim)

    @property
    def launch_count(self) -> int:
        return qs_sim_launch_count(self.sim)


# ----------------------------------------------------------------------
# Batched persistent launch
# ----------------------------------------------------------------------

def _bcheck(rc: int, where: str) -> None:
    if rc != QS_OK:
        raise QsError(rc, where, lib().qs_batch_last_error().decode())


def circuit_rounds(circuit):
    """Rounds of a workloads Circuit: (round_layers, round_meas, qubits) with
    round r = layers [rl[r], rl[r+1]) then the measurements rm[r]..rm[r+1]."""
    rl, rm, qs_ = [0], [0], []
    cur_l, cur_m = 0, 0
    pending = False
    for op in circuit.ops:
        if op[0] == "layers":
            if op[1] != cur_l:
                raise ValueError("layer runs must be contiguous")
            cur_l = op[2]
            pending = True
        elif op[0] == "noise":
            continue  # noise acts on sampled shots only; the batch runs the reference shot
        else:
            qs_.append(np.asarray(op[1], np.uint32))
            cur_m += len(op[1])
            rl.append(cur_l)
            rm.append(cur_m)
            pending = False
    if pending:
        rl.append(cur_l)
        rm.append(cur_m)
    q = np.concatenate(qs_) if qs_ else np.zeros(0, np.uint32)
    return np.array(rl, np.uint32), np.array(rm, np.uint32), q


class Batch:
    """Many circuits in one persistent launch (qs_batch_* of include/qs.h)."""

    def __init__(self, circuits, seeds, shot: int = 0, device: str = "cuda", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.circuits = list(circuits)
        keep = []
        arr = (qs_batch_circuit * len(self.circuits))()
        self.meas = []
        for i, (c, sd) in enumerate(zip(self.circuits, seeds)):
            g = _as_gates(c.gates)
            lp = np.ascontiguousarray(c.layer_ptr, np.int64)
            rl, rm, q = circuit_rounds(c)
            keep += [g, lp, rl, rm, q]
            arr[i] = qs_batch_circuit(c.n, c.n_layers, g.ctypes.data if g.size else None,
                                      lp.ctypes.data, len(rl) - 1, 0, rl.ctypes.data,
                                      rm.ctypes.data, q.ctypes.data if q.size else None,
                                      int(sd), int(shot))
            self.meas.append(int(rm[-1]))
        nbytes = int(lib().qs_batch_required_bytes(len(self.circuits), ctypes.byref(arr)))
        if nbytes == 0:
            _bcheck(-1, "qs_batch_required_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _bcheck(lib().qs_batch_create(len(self.circuits), ctypes.byref(arr),
                                      ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                      ctypes.byref(h)), "qs_batch_create")
        self.h = h.value
        self.nbytes = nbytes

    def close(self):
        if getattr(self, "h", None):
            lib().qs_batch_destroy(ctypes.c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, tuning: "qs_batch_tuning" = None, round_limit: int = 0):
        _bcheck(lib().qs_batch_run(ctypes.c_void_p(self.h),
                                   ctypes.byref(tuning) if tuning is not None else None,
                                   round_limit), "qs_batch_run")

    def sync(self):
        _bcheck(lib().qs_batch_sync(ctypes.c_void_p(self.h)), "qs_batch_sync")

    def record(self, i: int) -> np.ndarray:
        out = np.zeros(max(self.meas[i], 1), np.uint8)
        _bcheck(lib().qs_batch_record(ctypes.c_void_p(self.h), i, out.ctypes.data, self.meas[i]),
                "qs_batch_record")
        return out[:self.meas[i]]

    def sample(self, shots, seeds):
        """Frame samples of every circuit (shots[i] shots, frame seed seeds[i]; 0
        shots skips a circuit) from the last complete run: a list of device
        tensors of shape (M_i, ceil(shots[i]/64)) int64 words (None where skipped).
        Enqueued on the batch's stream."""
        torch = self.torch
        k = len(self.circuits)
        sh = np.ascontiguousarray(shots, np.uint64)
        sd = np.ascontiguousarray(seeds, np.uint64)
        outs, ptrs = [], (ctypes.c_void_p * k)()
        for i in range(k):
            if sh[i] == 0:
                outs.append(None)
                continue
            ow = (int(sh[i]) + 63) // 64
            t = torch.empty((max(self.meas[i], 1), ow), dtype=torch.int64, device=self.device)
            outs.append(t[:self.meas[i]])
            ptrs[i] = t.data_ptr()
        _bcheck(lib().qs_batch_sample(ctypes.c_void_p(self.h), sh.ctypes.data, sd.ctypes.data,
                                      ctypes.cast(ptrs, ctypes.c_void_p)), "qs_batch_sample")
        self._keep_samples = outs
        return outs

    def export_rows(self, i: int, rows):
        n = self.circuits[i].n
        r = np.ascontiguousarray(rows, np.uint32)
        k = (n + 63) // 64
        buf = np.zeros((max(len(r), 1), 2 * k + 1), np.uint64)
        _bcheck(lib().qs_batch_export_rows(ctypes.c_void_p(self.h), i, r.ctypes.data, len(r),
                                           buf.ctypes.data), "qs_batch_export_rows")
        buf = buf[:len(r)]
        bits = np.unpackbits(np.ascontiguousarray(buf[:, :2 * k]).view(np.uint8).reshape(len(r), -1),
                             axis=1, bitorder="little")
        return (np.ascontiguousarray(bits[:, :n]), np.ascontiguousarray(bits[:, 64 * k:64 * k + n]),
                (buf[:, 2 * k] & 1).astype(np.uint8))

    def autotune(self, round_limit: int = 0, cache_path: Optional[str] = None) -> "qs_batch_tuning":
        t = qs_batch_tuning()
        _bcheck(lib().qs_batch_autotune(ctypes.c_void_p(self.h), round_limit,
                                        cache_path.encode() if cache_path else None,
                                        ctypes.byref(t)), "qs_batch_autotune")
        return t


# ----------------------------------------------------------------------
# Window scheduling (Sec. 4.2)
# ----------------------------------------------------------------------

def qs_schedule_windows(n: int, ops: np.ndarray, merge_measurements: bool = False):
    """ops: (count, 3) uint32 rows (type, q0, q1), type QS_MEASURE for a
    Z-measurement. Returns (out_ops, window_ptr, window_kind)."""
    o = _as_gates(ops)
    count = o.shape[0]
    out = np.zeros((max(count, 1), 3), np.uint32)
    ptr = np.zeros(count + 1, np.uint32)
    kind = np.zeros(max(count, 1), np.uint8)
    nw = ctypes.c_uint32(0)
    rc = lib().qs_schedule_windows(n, _ptr(o) if count else None, count, int(merge_measurements),
                                   _ptr(out), _ptr(ptr), _ptr(kind), ctypes.byref(nw))
    if rc != QS_OK:
        raise QsError(rc, "qs_schedule_windows", lib().qs_schedule_last_error().decode())
    w = nw.value
    return out[:count], ptr[:w + 1].astype(np.int64), kind[:w]


def scheduled_circuit(n: int, ops: np.ndarray, merge_measurements: bool = False, name: str = ""):
    """A workloads.circuits.Circuit from an ordered op list via qs_schedule_windows:
    gate windows become layers, measurement windows become measurement ops."""
    from workloads.circuits import Circuit
    out, ptr, kind = qs_schedule_windows(n, ops, merge_measurements)
    gates, layer_ptr, prog = [], [0], []
    for w in range(len(kind)):
        seg = out[ptr[w]:ptr[w + 1]]
        if kind[w] == 0:
            gates.append(seg)
            layer_ptr.append(layer_ptr[-1] + len(seg))
            l = len(layer_ptr) - 2
            if prog and prog[-1][0] == "layers" and prog[-1][2] == l:
                prog[-1] = ("layers", prog[-1][1], l + 1)
            else:
                prog.append(("layers", l, l + 1))
        else:
            prog.append(("measure", np.ascontiguousarray(seg[:, 1], np.uint32)))
    g = np.concatenate(gates) if gates else np.zeros((0, 3), np.uint32)
    return Circuit(n=n, gates=np.ascontiguousarray(g, np.uint32),
                   layer_ptr=np.array(layer_ptr, np.int64), ops=prog, name=name)
