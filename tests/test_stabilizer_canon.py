"""Pins for the canonical stabilizer group helper (no GPU), and the oracle's
two representations compared through it: the CHP tableau (Sec. 2.5) and the
inverse tableau with qubit-indexed signs (Sec. 3.2, Alg. 1) hold the same
stabilizer group after gates and measurements under the same keyed coins."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import stabilizer_canon as SC
from workloads import circuits as C


def _paulis(strings):
    """(x, z, r) from strings like '+XZ', '-YI' (qubit 0 first)."""
    n = len(strings[0]) - 1
    x = np.zeros((len(strings), n), np.uint8)
    z = np.zeros((len(strings), n), np.uint8)
    r = np.zeros(len(strings), np.uint8)
    for i, s in enumerate(strings):
        r[i] = s[0] == "-"
        for q, c in enumerate(s[1:]):
            x[i, q] = c in "XY"
            z[i, q] = c in "ZY"
    return x, z, r


def test_known_states():
    # Bell pair: generated by XX and ZZ, also by YY = -(XX)(ZZ) and ZZ
    a = SC.canonical(*_paulis(["-YY", "+ZZ"]))
    b = SC.canonical(*_paulis(["+XX", "+ZZ"]))
    assert SC.same_group(a, b)
    assert SC.same_group(a, _paulis(["+XX", "+ZZ"]))
    # the sign is part of the group: -XX, +ZZ is another state
    assert not SC.same_group(a, SC.canonical(*_paulis(["-XX", "+ZZ"])))
    # Y stays Y: sigma(1, 1) is Hermitian
    assert SC.same_group(SC.canonical(*_paulis(["+Y"])), _paulis(["+Y"]))


def test_products_of_anticommuting_paulis_are_rejected():
    x, z, r = _paulis(["+XI", "+ZI"])
    with pytest.raises(ValueError):
        SC.multiply(x[0], z[0], r[0], x[1], z[1], r[1])


@pytest.mark.parametrize("n,seed", [(5, 1), (24, 2), (70, 3)])
def test_canonical_form_ignores_the_choice_of_generators(n, seed):
    circ = C.gate_mix_circuit(n, 12, seed=seed, measure_every=4, measure_frac=0.3)
    o, _, _ = O.run_circuit(circ, seed=seed)
    x, z, r = o.get()
    ref = SC.stabilizer_group_of_chp(x, z, r)
    sx, sz, sr = x[n:].copy(), z[n:].copy(), r[n:].copy()
    rng = np.random.default_rng(seed)
    for _ in range(3 * n):  # random row products, then a shuffle
        i, j = rng.choice(n, 2, replace=False)
        sx[i], sz[i], sr[i] = SC.multiply(sx[i], sz[i], sr[i], sx[j], sz[j], sr[j])
    p = rng.permutation(n)
    assert SC.same_group(SC.canonical(sx[p], sz[p], sr[p]), ref)
    # one flipped sign is a different state
    sr[p[0]] ^= 1
    assert not SC.same_group(SC.canonical(sx, sz, sr), ref)


@pytest.mark.parametrize("n,seed", [(1, 1), (3, 2), (17, 3), (64, 4), (130, 5)])
def test_inverse_and_chp_oracles_hold_the_same_group(n, seed):
    circ = C.gate_mix_circuit(n, 16, seed=seed + 40, measure_every=4, measure_frac=0.35)
    o, rec, _ = O.run_circuit(circ, seed=seed)
    inv, irec, _ = O.run_circuit_inverse(circ, seed=seed)
    assert np.array_equal(rec, irec)
    a = SC.stabilizer_group_of_chp(*o.get())
    b = SC.stabilizer_group_of_inverse(*inv.get())
    assert len(a[2]) == n and SC.same_group(a, b)


def test_identity_and_initstate_signs():
    n = 6
    init = np.array([1, 0, 1, 1, 0, 0], np.uint8)
    inv = O.InverseOracle(n, init)
    x, z, ss, sd = inv.get()
    assert np.array_equal(SC.forward_signs_from_inverse(x, z, ss, sd), init)
