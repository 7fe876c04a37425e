"""Brute-force helpers for the oracle pins: dense Pauli matrices, gate
unitaries and a small state-vector simulator (complex128, <= 10 qubits).

These are written from textbook definitions (Nielsen & Chuang), not from the
tableau rules, so they check the oracle independently. Qubit j is bit j of
the basis-state index.
"""
from __future__ import annotations

import numpy as np

from workloads import circuits as C

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
HM = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
SM = np.diag([1, 1j]).astype(complex)
SDGM = np.diag([1, -1j]).astype(complex)

ONE_Q = {C.X: PX, C.Y: PY, C.Z: PZ, C.H: HM, C.S: SM, C.SDG: SDGM, C.I: I2}


def sigma(x: int, z: int) -> np.ndarray:
    """Single-qubit Pauli of the encoding (0,0)=I, (1,0)=X, (1,1)=Y, (0,1)=Z."""
    return {(0, 0): I2, (1, 0): PX, (1, 1): PY, (0, 1): PZ}[(int(x), int(z))]


def kron_list(mats):
    out = np.array([[1]], dtype=complex)
    for m in mats:
        out = np.kron(out, m)
    return out


def pauli_matrix(x, z, r) -> np.ndarray:
    """(-1)^r * sigma(x_0,z_0) (x) ... on n qubits; qubit j = bit j of index."""
    n = len(x)
    # kron puts the first factor on the most significant bit: qubit n-1 first
    return (-1) ** int(r) * kron_list([sigma(x[j], z[j]) for j in reversed(range(n))])


def pauli_string(x, z, r) -> str:
    letters = {(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}
    return ("-" if r else "+") + "".join(letters[(int(a), int(b))] for a, b in zip(x, z))


def two_qubit_unitary(t: int) -> np.ndarray:
    """4x4 unitary on (a, b) with a = low bit, b = high bit of the 2-bit index."""
    U = np.zeros((4, 4), dtype=complex)
    for idx in range(4):
        a, b = idx & 1, (idx >> 1) & 1
        if t == C.CX:  # control a, target b
            U[(a | ((b ^ a) << 1)), idx] = 1
        elif t == C.CZ:
            U[idx, idx] = -1 if (a and b) else 1
        elif t == C.CY:  # control a, Y on b
            if a == 0:
                U[idx, idx] = 1
            else:
                for bo in range(2):
                    U[a | (bo << 1), idx] = PY[bo, b]
        elif t == C.SWAP:
            U[b | (a << 1), idx] = 1
        elif t == C.ISWAP:
            if a == b:
                U[idx, idx] = 1
            else:
                U[b | (a << 1), idx] = 1j
        else:
            raise ValueError(t)
    return U


class StateVector:
    def __init__(self, n: int):
        self.n = n
        self.psi = np.zeros(2 ** n, dtype=complex)
        self.psi[0] = 1.0

    def _apply1(self, U, q):
        n = self.n
        t = self.psi.reshape([2] * n)  # axis k <-> qubit n-1-k
        ax = n - 1 - q
        t = np.moveaxis(np.tensordot(U, t, axes=([1], [ax])), 0, ax)
        self.psi = t.reshape(-1)

    def _apply2(self, U, a, b):
        n = self.n
        t = self.psi.reshape([2] * n)
        axa, axb = n - 1 - a, n - 1 - b
        U4 = U.reshape(2, 2, 2, 2)  # [b_out, a_out, b_in, a_in]
        t = np.tensordot(U4, t, axes=([2, 3], [axb, axa]))
        t = np.moveaxis(t, [0, 1], [axb, axa])
        self.psi = t.reshape(-1)

    def gate(self, t, a, b=0):
        if t in ONE_Q:
            self._apply1(ONE_Q[t], a)
        else:
            self._apply2(two_qubit_unitary(t), a, b)

    def apply(self, gates):
        for t, a, b in np.asarray(gates):
            self.gate(int(t), int(a), int(b))

    def prob(self, q, m) -> float:
        idx = np.arange(2 ** self.n)
        mask = ((idx >> q) & 1) == m
        return float(np.sum(np.abs(self.psi[mask]) ** 2))

    def project(self, q, m) -> float:
        idx = np.arange(2 ** self.n)
        mask = ((idx >> q) & 1) == m
        p = float(np.sum(np.abs(self.psi[mask]) ** 2))
        self.psi = np.where(mask, self.psi, 0)
        if p > 0:
            self.psi = self.psi / np.sqrt(p)
        return p

    def expect_stabilized(self, P) -> bool:
        return np.allclose(P @ self.psi, self.psi, atol=1e-9)


def symplectic(xa, za, xb, zb) -> int:
    return int((np.dot(xa.astype(int), zb.astype(int)) + np.dot(za.astype(int), xb.astype(int))) % 2)


def pauli_product(x1, z1, r1, x2, z2, r2):
    """(P1 * P2) for Hermitian signed Paulis using the 2x2 multiplication
    table per qubit; returns (x, z, phase) with phase the power of i (mod 4)
    of the result relative to sigma(x, z)."""
    table = {}
    mats = {(a, b): sigma(a, b) for a in (0, 1) for b in (0, 1)}
    for k1, m1 in mats.items():
        for k2, m2 in mats.items():
            prod = m1 @ m2
            k3 = (k1[0] ^ k2[0], k1[1] ^ k2[1])
            m3 = mats[k3]
            for e in range(4):
                if np.allclose(prod, (1j ** e) * m3):
                    table[(k1, k2)] = e
                    break
    ph = 2 * int(r1) + 2 * int(r2)
    for a, b, c, d in zip(x1, z1, x2, z2):
        ph += table[((int(a), int(b)), (int(c), int(d)))]
    return (x1 ^ x2), (z1 ^ z2), ph % 4
