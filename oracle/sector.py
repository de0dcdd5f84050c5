"""Quantum-number symmetries and the physicality lookup (Sec. III.A-B).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Local decomposability: s(x) = s_1(x_1) (.) s_2(x_2) (.) ... (.) s_N(x_N)
  for a binary composition (.) that is addition (particle number, S_z,
  Appendix A) or multiplication (Z2 Pauli-Z strings, Sec. IV.A).
* IsPhys(i; s_<i) (Algorithm 1): True at i = N + 1 iff s_<i equals the target
  eigenvalues, otherwise the OR over the two children, memoised in a lookup
  keyed by (i, s_<i) as Proposition 1 allows.
* The target is s_ref = s(x_ref) (Sec. III.B end; Sec. IV.A fixes the
  reference to the Hartree-Fock determinant x_HF).

Qubit order (Appendix A): 1-based odd qubits carry spin up.  In 0-based terms
qubit q = 2 p + sigma with p the spatial orbital and sigma = 0 for alpha.  The
autoregressive unit used here is the spatial orbital ("slot"): slot p
takes the value v = x_{2p} + 2 x_{2p+1}, and outcome v is allowed when the
qubit-level IsPhys of the prefix extended by both qubits is True.

Pinned by: leaf counts equal the Table I "without Z2" column, brute force over
all bitstrings for small N, and Proposition 1 as a property test
(tests/test_oracle_sector.py).
"""
from __future__ import annotations

import sys
from typing import Callable, Sequence


class Symmetry:
    """A locally decomposable symmetry: local eigenvalue per (qubit, bit) and
    a composition operation ('add' or 'mul')."""

    def __init__(self, local: Callable[[int, int], int], op: str):
        assert op in ("add", "mul")
        self.local = local  # local(i_1based, x_i) -> eigenvalue contribution
        self.op = op

    @property
    def identity(self):
        return 0 if self.op == "add" else 1

    def compose(self, a, b):
        return a + b if self.op == "add" else a * b


def particle_number() -> Symmetry:
    """n_e: s(x) = sum_i x_i (Appendix A)."""
    return Symmetry(lambda i, x: x, "add")


def spin_projection_x2() -> Symmetry:
    """2 S_z: s(x) = sum_i (-1)^(i-1) x_i, i 1-based (Appendix A, doubled so
    that eigenvalues stay integers)."""
    return Symmetry(lambda i, x: x if (i - 1) % 2 == 0 else -x, "add")


def z2_string(qubits_1based: Sequence[int]) -> Symmetry:
    """A Z2 symmetry: a product of Pauli Z on the listed qubits; the local
    eigenvalue of Z on |x> is (-1)^x (Sec. IV.A)."""
    qs = set(qubits_1based)
    return Symmetry(lambda i, x: (-1 if x else 1) if i in qs else 1, "mul")


def molecular_symmetries() -> list[Symmetry]:
    return [particle_number(), spin_projection_x2()]


def eigenvalues(bits: Sequence[int], syms: Sequence[Symmetry]):
    """Vector of partial eigenvalues s(x_<i) for the given leading bits."""
    s = [sym.identity for sym in syms]
    for idx, xb in enumerate(bits):
        i = idx + 1
        s = [sym.compose(sv, sym.local(i, xb)) for sv, sym in zip(s, syms)]
    return tuple(s)


class IsPhys:
    """Algorithm 1 with its lookup table.  ``N`` qubits, target ``s_ref``."""

    def __init__(self, N: int, syms: Sequence[Symmetry], s_ref):
        self.N = N
        self.syms = list(syms)
        self.s_ref = tuple(s_ref)
        self.lookup: dict = {}
        sys.setrecursionlimit(max(sys.getrecursionlimit(), 10 * N + 100))

    def __call__(self, i: int, s_lt) -> bool:
        key = (i, tuple(s_lt))
        if key not in self.lookup:
            if i == self.N + 1:
                self.lookup[key] = tuple(s_lt) == self.s_ref
            else:
                children = []
                for xb in (0, 1):
                    child = tuple(sym.compose(sv, sym.local(i, xb))
                                  for sv, sym in zip(s_lt, self.syms))
                    children.append(self(i + 1, child))
                self.lookup[key] = children[0] or children[1]
        return self.lookup[key]

    def of_prefix(self, bits: Sequence[int]) -> bool:
        """Physicality of the partial basis vector x_<i given as leading bits."""
        return self(len(bits) + 1, eigenvalues(bits, self.syms))


def hf_bits(n: int, n_alpha: int, n_beta: int) -> list[int]:
    """x_HF in interleaved order: the lowest n_alpha alpha and n_beta beta
    spatial orbitals occupied (Sec. IV.A with Appendix A's ordering)."""
    bits = [0] * (2 * n)
    for p in range(n_alpha):
        bits[2 * p] = 1
    for p in range(n_beta):
        bits[2 * p + 1] = 1
    return bits


def molecular_isphys(n: int, n_alpha: int, n_beta: int, extra: Sequence[Symmetry] = ()) -> IsPhys:
    syms = molecular_symmetries() + list(extra)
    ref = hf_bits(n, n_alpha, n_beta)
    return IsPhys(2 * n, syms, eigenvalues(ref, syms))


def bits_of(x: int, n_qubits: int) -> list[int]:
    return [(x >> q) & 1 for q in range(n_qubits)]


def slot_value(x: int, p: int) -> int:
    return (x >> (2 * p)) & 3


def slot_allowed(isphys: IsPhys, x_prefix: int, p: int) -> list[bool]:
    """Allowed outcomes v = 0..3 of slot p (0-based) after the prefix holding
    slots < p: the qubit-level IsPhys at level 2p + 3 (1-based) of the prefix
    extended by x_{2p} = v & 1 and x_{2p+1} = v >> 1."""
    pre = bits_of(x_prefix, 2 * p)
    return [isphys.of_prefix(pre + [v & 1, v >> 1]) for v in range(4)]


def count_leaves(isphys: IsPhys) -> int:
    """Number of physical leaves, counted by walking the qubit tree and
    pruning unphysical subtrees (Fig. 1B): the size of the sector."""
    N = isphys.N
    syms = isphys.syms
    # counts per distinct partial-eigenvalue vector, level by level
    level = {tuple(sym.identity for sym in syms): 1}
    for i in range(1, N + 1):
        nxt: dict = {}
        for s, c in level.items():
            if not isphys(i, s):
                continue
            for xb in (0, 1):
                child = tuple(sym.compose(sv, sym.local(i, xb)) for sv, sym in zip(s, syms))
                nxt[child] = nxt.get(child, 0) + c
        level = nxt
    return sum(c for s, c in level.items() if isphys(N + 1, s))


def sector_states(n: int, n_alpha: int, n_beta: int) -> list[int]:
    """All determinants with n_alpha alpha and n_beta beta electrons, found by
    brute force over all 4^n bitstrings (small n only), ascending."""
    out = []
    for x in range(1 << (2 * n)):
        a = sum((x >> (2 * p)) & 1 for p in range(n))
        b = sum((x >> (2 * p + 1)) & 1 for p in range(n))
        if a == n_alpha and b == n_beta:
            out.append(x)
    return out


def sector_states_tree(isphys: IsPhys, n: int) -> list[int]:
    """All leaves reachable through allowed slot outcomes (pruned tree walk)."""
    frontier = [0]
    for p in range(n):
        nxt = []
        for x in frontier:
            for v, ok in enumerate(slot_allowed(isphys, x, p)):
                if ok:
                    nxt.append(x | (v << (2 * p)))
        frontier = nxt
    return frontier

