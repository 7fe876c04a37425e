"""Canonical form of a stabilizer group, for comparing two representations of
one state: the CHP tableau's stabilizer rows with their signs (Sec. 2.5) and
the inverse tableau with qubit-indexed signs (Sec. 3.2).

Paulis are bit vectors (x, z) over n qubits with a sign bit r; sigma(x, z) is
the Hermitian Pauli i^{x.z} X^x Z^z (so sigma(1, 1) = Y). The product of two
Hermitian Paulis is sigma(a) sigma(b) = i^{g(a, b)} sigma(a ^ b) with the
per-qubit exponent g of Aaronson and Gottesman's rowsum.

canonical() is the reduced row echelon form over GF(2) of the generators,
with each row's sign carried through the row products: two generating sets of
one stabilizer group (which never contains -I) give the same canonical form.
forward_signs_from_inverse() recovers the signs of C Z_q C^dag from the images
C^dag X_a C and C^dag Z_a C: the bits of C Z_q C^dag are stabilizer row q of
the extended tableau (the inverse representation shares the forward bits);
mapping that Pauli back through the images gives +-Z_q, and that sign is the
stabilizer's.

Test infrastructure: numpy only, no product or oracle code."""
import numpy as np


def g_sum(x1, z1, x2, z2) -> np.ndarray:
    """Sum over the last axis of the per-qubit exponent g (values in -1..1)."""
    x1 = x1.astype(np.int64); z1 = z1.astype(np.int64)
    x2 = x2.astype(np.int64); z2 = z2.astype(np.int64)
    g = np.where((x1 == 1) & (z1 == 1), z2 - x2,
                 np.where(x1 == 1, z2 * (2 * x2 - 1),
                          np.where(z1 == 1, x2 * (1 - 2 * z2), 0)))
    return g.sum(axis=-1)


def multiply(xa, za, ra, xb, zb, rb):
    """(sign, bits) of (-1)^ra sigma(a) * (-1)^rb sigma(b) for commuting a, b."""
    e = (2 * int(ra) + 2 * int(rb) + int(g_sum(xa, za, xb, zb))) % 4
    if e % 2:
        raise ValueError("product of anticommuting Paulis")
    return xa ^ xb, za ^ zb, e // 2


def canonical(x: np.ndarray, z: np.ndarray, r: np.ndarray):
    """Reduced row echelon form (pivot columns: x of qubit 0..n-1, then z of
    qubit 0..n-1) of the generators (rows of x, z with signs r). Returns
    (x, z, r) of the nonzero rows, in pivot order."""
    x = np.array(x, np.uint8) & 1
    z = np.array(z, np.uint8) & 1
    r = np.array(r, np.uint8) & 1
    m, n = x.shape
    bits = np.concatenate([x, z], axis=1)
    rank = 0
    for col in range(2 * n):
        if rank == m:
            break
        hits = np.nonzero(bits[rank:, col])[0]
        if len(hits) == 0:
            continue
        p = rank + int(hits[0])
        if p != rank:
            bits[[rank, p]] = bits[[p, rank]]
            r[[rank, p]] = r[[p, rank]]
        for i in np.nonzero(bits[:, col])[0]:
            if i == rank:
                continue
            nx, nz, nr = multiply(bits[i, :n], bits[i, n:], r[i], bits[rank, :n], bits[rank, n:], r[rank])
            bits[i, :n], bits[i, n:], r[i] = nx, nz, nr
        rank += 1
    return bits[:rank, :n].copy(), bits[:rank, n:].copy(), r[:rank].copy()


def forward_signs_from_inverse(x: np.ndarray, z: np.ndarray, ss: np.ndarray, sd: np.ndarray) -> np.ndarray:
    """Signs of the stabilizers C Z_q C^dag (q < n) of the state held by an
    inverse tableau: x, z of shape (2n, n) in the extended tableau's rows
    (C^dag Z_a C has x bits x[n + i, a] and z bits x[i, a] at input i, sign
    ss[a]; C^dag X_a C has x bits z[n + i, a], z bits z[i, a], sign sd[a])."""
    n = len(ss)
    x = np.asarray(x, np.uint8) & 1
    z = np.asarray(z, np.uint8) & 1
    sx, sz = x[n:, :], z[n:, :]  # bits of C Z_q C^dag, one row per q
    acc_x = np.zeros((n, n), np.uint8)
    acc_z = np.zeros((n, n), np.uint8)
    phase = np.zeros(n, np.int64)
    for a in range(n):
        # sigma(v) = i^{x.z} prod_a X_a^{x_a} Z_a^{z_a}: the image of X_a, then of Z_a
        for sel, fx, fz, s in ((sx[:, a], z[n:, a], z[:n, a], sd[a]),
                               (sz[:, a], x[n:, a], x[:n, a], ss[a])):
            m = sel == 1
            if not m.any():
                continue
            phase[m] += 2 * int(s) + g_sum(acc_x[m], acc_z[m], fx[None, :], fz[None, :])
            acc_x[m] ^= fx[None, :]
            acc_z[m] ^= fz[None, :]
    phase += (sx & sz).sum(axis=1, dtype=np.int64)
    if acc_x.any() or not np.array_equal(acc_z, np.eye(n, dtype=np.uint8)):
        raise ValueError("stabilizer rows do not map back to Z_q: not an inverse tableau")
    phase %= 4
    if (phase % 2).any():
        raise ValueError("odd phase: images are not Hermitian")
    return (phase // 2).astype(np.uint8)


def stabilizer_group_of_chp(x, z, r):
    n = x.shape[1]
    return canonical(x[n:], z[n:], r[n:])


def stabilizer_group_of_inverse(x, z, ss, sd):
    n = len(ss)
    return canonical(x[n:], z[n:], forward_signs_from_inverse(x, z, ss, sd))


def same_group(a, b) -> bool:
    return all(np.array_equal(u, v) for u, v in zip(a, b))
