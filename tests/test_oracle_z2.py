"""Z2 (point-group) symmetries in IsPhys (Algorithm 1 with the
multiplicative composition of Sec. IV.A) on synthetic Hamiltonians with a
planted abelian symmetry (irrep-blocked integrals).

Pins: the planted Pauli-Z strings really commute with H (the JW Hamiltonian
built from Pauli products, path B, never connects strings of different
parity); IsPhys with the Z2 strings counts exactly the brute-force sector
(electron counts and the reference parities); the sampler stays in that
sector; and the tabular ansatz of the ground vector of the Z2-restricted
sector gives E_loc = E_0 there.
"""
import numpy as np
import pytest

from oracle.anqs import table_from_state, TableAnsatz
from oracle.ed import ground_state
from oracle.hamiltonian import Hamiltonian as OHam, sector_matrix
from oracle.sampler import sample
from oracle.sector import count_leaves, molecular_isphys, sector_states, z2_string
from oracle.vmc import local_energy
from synthetic import integrals_z2, z2_qubit_masks

CASES = [(5, 2, 2, [0, 1, 0, 1, 1]), (6, 3, 2, [0, 1, 1, 0, 1, 0]), (6, 2, 2, [0, 1, 2, 3, 1, 2])]


def _z2_syms(masks, n):
    return [z2_string([q + 1 for q in range(2 * n) if (m >> q) & 1]) for m in masks]


def _parity(x, m):
    return bin(int(x) & int(m)).count("1") & 1


def _ref(n, na, nb):
    return sum(1 << (2 * p) for p in range(na)) | sum(1 << (2 * p + 1) for p in range(nb))


@pytest.mark.parametrize("n,na,nb,labels", CASES)
def test_planted_z2_strings_commute_with_h(n, na, nb, labels):
    h, g, e = integrals_z2(n, n, 2 * n, labels)
    ham = OHam(h, g, e, na, nb)
    H = ham.dense_jw().tocoo()
    for m in z2_qubit_masks(labels):
        for r, c, v in zip(H.row, H.col, H.data):
            if abs(v) > 1e-14:
                assert _parity(r, m) == _parity(c, m)


@pytest.mark.parametrize("n,na,nb,labels", CASES)
def test_isphys_with_z2_counts_the_brute_force_sector(n, na, nb, labels):
    masks = z2_qubit_masks(labels)
    ip = molecular_isphys(n, na, nb, extra=_z2_syms(masks, n))
    ref = _ref(n, na, nb)
    st = [x for x in sector_states(n, na, nb) if all(_parity(x, m) == _parity(ref, m) for m in masks)]
    assert count_leaves(ip) == len(st)
    assert len(st) < len(sector_states(n, na, nb))


@pytest.mark.parametrize("n,na,nb,labels", CASES)
def test_sampler_stays_in_z2_sector_and_eloc_is_e0(n, na, nb, labels):
    masks = z2_qubit_masks(labels)
    ip = molecular_isphys(n, na, nb, extra=_z2_syms(masks, n))
    ref = _ref(n, na, nb)
    st = np.array([x for x in sector_states(n, na, nb) if all(_parity(x, m) == _parity(ref, m) for m in masks)],
                  dtype=np.uint64)
    h, g, e = integrals_z2(n, n, 2 * n, labels)
    ham = OHam(h, g, e, na, nb)
    E0, c = ground_state(ham, [int(x) for x in st])
    model = TableAnsatz(table_from_state(st, c, n), n)
    x, cnt, _ = sample(model, ip, n, 20_000, seed=1)
    assert np.all(np.isin(x, st)) and cnt.sum() == 20_000
    big = np.abs(c) > 1e-3
    el = local_energy(model, ip, ham, st[big])
    assert np.abs(el - E0).max() < 1e-8
