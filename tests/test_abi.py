"""Host-side checks of the C ABI (no GPU): the library builds and loads, every
function declared in include/qs.h is exported, the gate codes agree with the
input format, and host validation rejects bad layers."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2603_14641_gb300 import qs
from workloads import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qs.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ["qs_sim_create", "qs_sim_destroy", "qs_sim_apply_layer", "qs_sim_measure",
                 "qs_sim_sample", "qs_sim_tableau_export"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    L = qs.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True)
    exported = set(re.findall(r"\bT\s+(qs_[a-z_0-9]+)$", out.stdout, flags=re.M))
    missing = [f for f in _declared_functions() if f not in exported]
    assert not missing, missing
    for f in _declared_functions():
        assert f in qs.SIGNATURES, f"binding lacks {f}"


def test_gate_codes_match_input_format():
    text = open(HEADER).read()
    for name in C.GATE_NAMES:
        m = re.search(rf"QS_{name}\s*=\s*(\d+)", text)
        assert m, name
        assert int(m.group(1)) == getattr(C, name) == qs.GATES[name]


def test_noise_codes_match_input_format():
    text = open(HEADER).read()
    for name, hname in [("NOISE_X", "QS_NOISE_X"), ("NOISE_Y", "QS_NOISE_Y"), ("NOISE_Z", "QS_NOISE_Z"),
                        ("DEPOLARIZE1", "QS_NOISE_DEPOLARIZE1"),
                        ("DEPOLARIZE2", "QS_NOISE_DEPOLARIZE2")]:
        m = re.search(rf"{hname}\s*=\s*(\d+)", text)
        assert m, hname
        assert int(m.group(1)) == getattr(C, name) == getattr(qs, hname)


def test_version_and_required_bytes():
    assert "sm_103a" in qs.qs_version()
    n = 180_000
    b = qs.qs_sim_required_bytes(n)
    k = (n + 63) // 64
    cs = (2 * k + 3) // 4 * 4
    ncols = (n + 255) // 256 * 256
    # column-major X, Z and row-major RX, RZ dominate: ~n^2 bytes in total
    assert b >= 2 * ncols * cs * 8 + 2 * (64 * cs) * (ncols // 64) * 8
    assert b < 1.02 * n * n + (1 << 28)
    assert qs.qs_sim_required_bytes(0) == 0


def test_pack_layers_format_and_validation():
    circ = C.random_circuit(100, 5, 0.5, seed=3)
    packed = qs.qs_pack_layers(circ.n, circ.gates, circ.layer_ptr)
    g = circ.gates
    assert np.array_equal(packed[0::2], (g[:, 0] << 24) | g[:, 1])
    two = np.isin(g[:, 0], C.TWO_QUBIT)
    assert np.array_equal(packed[1::2], np.where(two, g[:, 2], 0))
    bad = [
        np.array([[C.CX, 1, 1]], np.uint32),            # two-qubit gate on one qubit
        np.array([[C.H, 3, 0], [C.S, 3, 0]], np.uint32),  # qubit used twice in a layer
        np.array([[C.H, 100, 0]], np.uint32),           # qubit out of range
        np.array([[12, 0, 0]], np.uint32),              # unknown gate type
        np.array([[C.CZ, 5, 100]], np.uint32),          # target out of range
    ]
    for b in bad:
        with pytest.raises(qs.QsError) as e:
            qs.qs_pack_layers(100, b, np.array([0, len(b)]))
        assert e.value.code == -1
    # the same qubit in two different layers is fine
    ok = np.array([[C.H, 3, 0], [C.S, 3, 0]], np.uint32)
    qs.qs_pack_layers(100, ok, np.array([0, 1, 2]))


def test_create_without_device_fails_loudly():
    """Without a usable GPU the product path raises instead of falling back."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(qs.QsError):
        qs.qs_sim_create(64)


def test_layout_codes_and_native_unpacking():
    """The layout codes agree with the header, and unpack_native reads a NATIVE
    buffer written here bit by bit from its documented definition."""
    text = open(HEADER).read()
    for name in ["QS_LAYOUT_ROWS_PACKED", "QS_LAYOUT_NATIVE"]:
        m = re.search(rf"{name}\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == getattr(qs, name)
    rng = np.random.default_rng(4)
    for n in (1, 63, 64, 65, 130, 300):
        x = rng.integers(0, 2, (2 * n, n), dtype=np.uint8)
        z = rng.integers(0, 2, (2 * n, n), dtype=np.uint8)
        r = rng.integers(0, 2, 2 * n, dtype=np.uint8)
        k = -(-n // 64)
        W = 4 * -(-k // 2)
        buf = np.zeros((2 * n + 1) * W, np.uint64)
        for i in range(2 * n):
            g = i if i < n else 64 * k + (i - n)
            w, b = divmod(g, 64)
            for q in np.nonzero(x[i])[0]:
                buf[q * W + w] |= np.uint64(1) << np.uint64(b)
            for q in np.nonzero(z[i])[0]:
                buf[(n + q) * W + w] |= np.uint64(1) << np.uint64(b)
            if r[i]:
                buf[2 * n * W + w] |= np.uint64(1) << np.uint64(b)
        ux, uz, ur = qs.unpack_native(buf, n)
        assert np.array_equal(ux, x) and np.array_equal(uz, z) and np.array_equal(ur, r)


def test_option_flags_match_header():
    text = open(HEADER).read()
    for name in ["QS_FLAG_NO_FUSION", "QS_FLAG_UNPIPELINED_MEASURE", "QS_FLAG_NO_BLOCKED_MEASURE",
                 "QS_FLAG_WIDE_OFFSETS", "QS_FLAG_STEP_SYMBOLIC"]:
        m = re.search(rf"#define\s+{name}\s+(\d+)u", text)
        assert m and int(m.group(1)) == getattr(qs, name), name


def test_timing_kinds_match_header():
    text = open(HEADER).read()
    names = re.findall(r"\bQS_TIME_([A-Z_]+)\s*=\s*(\d+)", text)
    assert [int(v) for _, v in names] == list(range(len(names)))
    assert [nm.lower() for nm, _ in names] == qs.QS_TIME_KINDS
    m = re.search(r"QS_NUM_TIME_KINDS\s*=\s*(\d+)", text)
    assert m and int(m.group(1)) == len(qs.QS_TIME_KINDS)
