"""Pins for the oracle Hamiltonian: Slater-Condon (path A) against the
Jordan-Wigner Pauli-product operator (path B), Hermiticity, closed-form
connected counts and the canonical excitation order."""
from math import comb

import numpy as np
import pytest

from oracle.hamiltonian import Hamiltonian, sector_matrix
from oracle.sector import sector_states
from synthetic import integrals


@pytest.mark.parametrize("n,na,nb,seed", [(2, 1, 1, 0), (3, 2, 1, 1), (3, 1, 2, 2), (4, 2, 2, 0),
                                           (4, 3, 1, 3), (4, 1, 0, 4)])
def test_slater_condon_equals_jordan_wigner(n, na, nb, seed):
    h, g, _ = integrals(seed, n, 2 * n)
    ham = Hamiltonian(h, g, 0.7, na, nb)
    st = sector_states(n, na, nb)
    HB = ham.dense_jw()
    B = HB[st][:, st].toarray()
    A = sector_matrix(ham, st)
    assert np.abs(B.imag).max() == 0.0
    assert np.abs(A - B.real).max() < 1e-13
    # the operator conserves the sector
    full = HB.toarray()
    out = np.ones(full.shape[0], bool)
    out[st] = False
    assert np.abs(full[np.ix_(out, ~out)]).max() < 1e-15


def test_hermitian_and_counts():
    n, na, nb = 5, 3, 2
    h, g, _ = integrals(9, n, 10)
    ham = Hamiltonian(h, g, 0.0, na, nb)
    st = sector_states(n, na, nb)
    A = sector_matrix(ham, st)
    assert np.abs(A - A.T).max() < 1e-14
    K = na * (n - na) + nb * (n - nb) + comb(na, 2) * comb(n - na, 2) + comb(nb, 2) * comb(n - nb, 2) \
        + na * (n - na) * nb * (n - nb)
    assert ham.n_connected() == K
    for x in st[::7]:
        L = ham.connected(x)
        assert len(L) == K
        xs = [xp for xp, _, _ in L]
        assert len(set(xs)) == K and x not in xs
        for xp, _, j in L:
            d = xp ^ x
            assert d & ((1 << (2 * j)) - 1) == 0 and (d >> (2 * j)) & 3 != 0


def test_canonical_order_small():
    """n = 3, one alpha and one beta electron in slot 0: the list starts with
    the alpha singles 0->1, 0->2, then the beta singles, then alpha-beta
    doubles ordered (I_a, A_a, I_b, A_b)."""
    h, g, _ = integrals(1, 3, 6)
    ham = Hamiltonian(h, g, 0.0, 1, 1)
    x = 0b000011
    xs = [xp for xp, _, _ in ham.connected(x)]
    exp = [0b000110, 0b010010, 0b001001, 0b100001, 0b001100, 0b100100, 0b011000, 0b110000]
    assert xs == exp


@pytest.mark.parametrize("name,K", [("small", 26), ("h2o", 140), ("n2", 609), ("large", 33507)])
def test_closed_form_counts_of_workloads(name, K):
    from synthetic import WORKLOADS
    w = WORKLOADS[name]
    ham = Hamiltonian(np.zeros((w["n"], w["n"])), np.zeros((w["n"],) * 4), 0.0, w["n_alpha"], w["n_beta"])
    assert ham.n_connected() == K


def test_hf_diagonal_is_mean_field_energy():
    """Diagonal element of a determinant from the Hartree-Fock expression
    E = sum_i h_ii + 1/2 sum_ij (J_ij - K_ij) written with spatial integrals
    for a closed-shell determinant: 2 sum_i h_ii + sum_ij (2 J_ij - K_ij)."""
    n = 5
    h, g, _ = integrals(4, n, 10)
    ham = Hamiltonian(h, g, 0.25, 2, 2)
    x = 0b1111
    E = 0.25 + 2 * sum(h[i, i] for i in range(2)) + sum(2 * g[i, i, j, j] - g[i, j, j, i]
                                                        for i in range(2) for j in range(2))
    assert abs(ham.diagonal(x) - E) < 1e-13
