"""Pin for the oracle's row-subset mode (no GPU).

RowSubset follows chosen generator rows of the n-qubit tableau under gates
alone. That is sound because the update rules of Sec. 2.4 (Eq. 4) act on every
row index independently, so the rows of a subset evolve exactly as the same
rows of the whole tableau. The pin runs the same gate circuits through the full
oracle (itself pinned by brute-force conjugation) and through RowSubset, with
row ids drawn from both halves (destabilizers 0..n-1 and stabilizers n..2n-1),
and requires the subset's rows to equal the full tableau's rows bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import circuits as C


def _subset_vs_full(n, layers, seed, nrows):
    circ = C.gate_mix_circuit(n, layers, seed=seed, final_measure_all=False)
    rng = np.random.default_rng(seed + 1000)
    # both halves, including the first and last row of each, in random order
    must = np.array([0, n - 1, n, 2 * n - 1], np.uint32)
    rest = rng.choice(2 * n, size=min(nrows, 2 * n), replace=False).astype(np.uint32)
    rows = np.unique(np.concatenate([must, rest]))
    rows = rows[rng.permutation(len(rows))]
    o = O.Oracle(n)
    o.apply(circ.gates)
    fx, fz, fr = o.get()
    sub = O.RowSubset(n, rows)
    sub.apply(circ.gates)
    sx, sz, sr = sub.get()
    assert np.array_equal(sx, fx[rows]), "x bits of the subset differ from the full tableau"
    assert np.array_equal(sz, fz[rows]), "z bits of the subset differ from the full tableau"
    assert np.array_equal(sr, fr[rows]), "signs of the subset differ from the full tableau"


@pytest.mark.parametrize("n,layers,seed,nrows", [(7, 30, 1, 14), (64, 25, 2, 40), (300, 20, 3, 90)])
def test_row_subset_equals_full_oracle_rows(n, layers, seed, nrows):
    _subset_vs_full(n, layers, seed, nrows)


def test_row_subset_of_the_initial_state():
    """Before any gate, destabilizer row i is X_i and stabilizer row n + i is
    Z_i with sign + (Sec. 2.5, Eq. 7 with the |0...0> initial state)."""
    n = 9
    rows = np.array([0, 4, 8, 9, 13, 17], np.uint32)
    x, z, r = O.RowSubset(n, rows).get()
    for j, g in enumerate(rows):
        want_x = np.zeros(n, np.uint8)
        want_z = np.zeros(n, np.uint8)
        if g < n:
            want_x[g] = 1
        else:
            want_z[g - n] = 1
        assert np.array_equal(x[j], want_x) and np.array_equal(z[j], want_z) and r[j] == 0
