"""Pins for IsPhys (Algorithm 1) and the slot masks."""
import os
from itertools import product
from math import comb

import numpy as np
import pytest

from oracle.sector import (IsPhys, count_leaves, eigenvalues, hf_bits, molecular_isphys,
                           molecular_symmetries, particle_number, sector_states,
                           sector_states_tree, slot_allowed, z2_string)

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_sector_sizes.txt")


def _table1():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        m, N, ne, sz = line.split()
        rows.append((m, int(N), int(ne), int(sz)))
    return rows


@pytest.mark.parametrize("mol,N,ne,size", _table1())
def test_table1_sector_sizes(mol, N, ne, size):
    """Leaf count of the pruned tree for the HF reference with n_e and S_z
    equals Table I's 'without Z2' column."""
    ip = molecular_isphys(N // 2, ne // 2, ne // 2)
    assert count_leaves(ip) == size


@pytest.mark.parametrize("n,na,nb", [(2, 1, 1), (3, 2, 1), (3, 0, 2), (4, 2, 2), (4, 3, 1)])
def test_isphys_brute_force(n, na, nb):
    """IsPhys(prefix) is True iff some completion of the prefix is in the sector."""
    N = 2 * n
    ip = molecular_isphys(n, na, nb)
    sector = set(sector_states(n, na, nb))
    for L in range(N + 1):
        for pre in product((0, 1), repeat=L):
            base = sum(b << q for q, b in enumerate(pre))
            exists = any((base | (rest << L)) in sector for rest in range(1 << (N - L)))
            assert ip.of_prefix(list(pre)) == exists


def test_particle_number_rule():
    """Sec. III.A: a prefix with more than n_e electrons is unphysical."""
    N, ne = 8, 3
    ip = IsPhys(N, [particle_number()], (ne,))
    for L in range(N + 1):
        for pre in product((0, 1), repeat=L):
            if sum(pre) > ne:
                assert not ip.of_prefix(list(pre))


def test_proposition1():
    """Equal partial eigenvalues => equal physicality (also for a Z2 string)."""
    n = 4
    syms = molecular_symmetries() + [z2_string([1, 2, 5, 6])]
    ref = hf_bits(n, 2, 1)
    ip = IsPhys(2 * n, syms, eigenvalues(ref, syms))
    for L in range(2 * n + 1):
        seen = {}
        for pre in product((0, 1), repeat=L):
            s = eigenvalues(pre, syms)
            # brute force physicality for this prefix
            ok = any(eigenvalues(list(pre) + list(rest), syms) == ip.s_ref
                     for rest in product((0, 1), repeat=2 * n - L))
            seen.setdefault(s, set()).add(ok)
            assert ip.of_prefix(list(pre)) == ok
        assert all(len(v) == 1 for v in seen.values())


def test_slot_tree_reaches_exactly_the_sector():
    for n, na, nb in [(4, 2, 2), (5, 3, 1), (6, 1, 5)]:
        ip = molecular_isphys(n, na, nb)
        leaves = sector_states_tree(ip, n)
        assert sorted(leaves) == sector_states(n, na, nb)
        assert len(leaves) == comb(n, na) * comb(n, nb)


def test_slot_masks_small_cases():
    ip = molecular_isphys(3, 1, 1)
    # at the root every outcome can still reach (1, 1)
    assert slot_allowed(ip, 0, 0) == [True, True, True, True]
    # after slot 0 = both electrons, slots 1, 2 must be empty
    assert slot_allowed(ip, 3, 1) == [True, False, False, False]
    # nothing placed in slots 0, 1: slot 2 must take both electrons
    assert slot_allowed(ip, 0, 2) == [False, False, False, True]
