"""Second-quantised molecular Hamiltonian, Jordan-Wigner signs, Slater-Condon
matrix elements and the connected set of a determinant.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Hamiltonian (Eq. sq_hamiltonian, Sec. IV.A).  The paper writes
H = sum h_ij a+_i a_j + sum h_ijkl a+_i a+_j a_k a_l without fixing the
spin structure or the factor of the two-body term.  Reading used here: the
spin-orbital form of real chemist-notation integrals (pq|rs) = g[p,q,r,s],

    H = E_nuc + sum_{pq,s} h_pq a+_{ps} a_{qs}
              + 1/2 sum_{pqrs,s,t} g_pqrs a+_{ps} a+_{rt} a_{st} a_{qs},

i.e. the paper's h_ijkl = 1/2 [il|jk] with spin conserved per pair.

Jordan-Wigner encoding (Sec. IV.A): qubit q holds the occupation of spin-
orbital q, a_q |x> = (-1)^(sum_{r<q} x_r) |x - e_q> when x_q = 1, and a+_q
likewise when x_q = 0.  Spin-orbital q = 2 p + sigma (Appendix A ordering).

Two independent evaluations:
  path A  ``matrix_element``: Slater-Condon rules for two determinants, signs
          from applying the operators one by one;
  path B  ``dense_jw``: the operator itself, built from Pauli matrices
          (sigma^+ = (X - iY)/2, sigma^- = (X + iY)/2 with Z strings) by
          Kronecker products, for small N only.
Pin: A == B element by element on small problems (tests/test_oracle_hamiltonian.py).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np
import scipy.sparse as sp


def _parity_below(x: int, q: int) -> int:
    return bin(x & ((1 << q) - 1)).count("1") & 1


def annihilate(x: int, q: int):
    """a_q |x> -> (sign, x') or None if x_q = 0."""
    if not (x >> q) & 1:
        return None
    return (-1 if _parity_below(x, q) else 1), x & ~(1 << q)


def create(x: int, q: int):
    """a+_q |x> -> (sign, x') or None if x_q = 1."""
    if (x >> q) & 1:
        return None
    return (-1 if _parity_below(x, q) else 1), x | (1 << q)


def apply_string(x: int, ops):
    """Apply a product of ladder operators, given left to right as
    [('c', q), ('a', q), ...], to |x>: the rightmost acts first."""
    sign = 1
    for kind, q in reversed(ops):
        r = (create if kind == "c" else annihilate)(x, q)
        if r is None:
            return None
        s, x = r
        sign *= s
    return sign, x


def spin_orbital_integrals(h, g):
    """h_IJ = h_ij d(s_I, s_J); [IJ|KL] = g_ijkl d(s_I, s_J) d(s_K, s_L),
    spin-orbital index I = 2 i + s_I."""
    n = h.shape[0]
    N = 2 * n
    hs = np.zeros((N, N))
    gs = np.zeros((N, N, N, N))
    for I in range(N):
        for J in range(N):
            if I % 2 == J % 2:
                hs[I, J] = h[I // 2, J // 2]
    for I, J, K, L in np.ndindex(N, N, N, N):
        if I % 2 == J % 2 and K % 2 == L % 2:
            gs[I, J, K, L] = g[I // 2, J // 2, K // 2, L // 2]
    return hs, gs


class Hamiltonian:
    """Integrals plus sector; all matrix elements in FP64."""

    def __init__(self, h, g, e_nuc: float, n_alpha: int, n_beta: int):
        self.h = np.asarray(h, dtype=np.float64)
        self.g = np.asarray(g, dtype=np.float64)
        self.e_nuc = float(e_nuc)
        self.n = self.h.shape[0]
        self.n_alpha = n_alpha
        self.n_beta = n_beta
        self.hs, self.gs = spin_orbital_integrals(self.h, self.g)

    # -- path A: Slater-Condon rules ------------------------------------------
    def matrix_element(self, xb: int, xk: int) -> float:
        """<xb| H |xk> for two determinants.

        diagonal: E_nuc + sum_I h_II + 1/2 sum_{I,J occ} ([II|JJ] - [IJ|JI])
        single I -> A: (h_AI + sum_{J occ} ([AI|JJ] - [AJ|JI])) * <xb|a+_A a_I|xk>
        double I<J -> A<B: ([AI|BJ] - [AJ|BI]) * <xb|a+_A a+_B a_J a_I|xk>
        """
        hs, gs = self.hs, self.gs
        N = 2 * self.n
        diff = xb ^ xk
        holes = [q for q in range(N) if (diff >> q) & 1 and (xk >> q) & 1]
        parts = [q for q in range(N) if (diff >> q) & 1 and (xb >> q) & 1]
        if len(holes) != len(parts):
            return 0.0
        occ = [q for q in range(N) if (xk >> q) & 1]
        if len(holes) == 0:
            e = self.e_nuc
            for I in occ:
                e += hs[I, I]
            for I in occ:
                for J in occ:
                    e += 0.5 * (gs[I, I, J, J] - gs[I, J, J, I])
            return e
        if len(holes) == 1:
            (I,), (A,) = holes, parts
            r = apply_string(xk, [("c", A), ("a", I)])
            sign, xo = r
            assert xo == xb
            v = hs[A, I]
            for J in occ:
                v += gs[A, I, J, J] - gs[A, J, J, I]
            return sign * v
        if len(holes) == 2:
            I, J = holes
            A, B = parts
            r = apply_string(xk, [("c", A), ("c", B), ("a", J), ("a", I)])
            sign, xo = r
            assert xo == xb
            return sign * (gs[A, I, B, J] - gs[A, J, B, I])
        return 0.0

    def diagonal(self, x: int) -> float:
        return self.matrix_element(x, x)

    # -- connected set ---------------------------------------------------------
    def connected(self, x: int):
        """Off-diagonal connected determinants of x in the canonical order:
        alpha singles, beta singles (each by (I, A) ascending, spatial indices),
        alpha-alpha doubles, beta-beta doubles (each by (I, J, A, B) with
        I < J, A < B), then alpha-beta doubles by (I_a, A_a, I_b, A_b).
        Elements that happen to be exactly zero are kept.

        Returns a list of (x', H_{x x'}, j) where j is the first slot (spatial
        orbital) in which x' differs from x.
        """
        n = self.n
        occ = {s: [p for p in range(n) if (x >> (2 * p + s)) & 1] for s in (0, 1)}
        vir = {s: [p for p in range(n) if not (x >> (2 * p + s)) & 1] for s in (0, 1)}
        out = []

        def emit(xp, changed):
            out.append((xp, self.matrix_element(xp, x), min(changed)))

        for s in (0, 1):
            for i in occ[s]:
                for a in vir[s]:
                    xp = x ^ (1 << (2 * i + s)) ^ (1 << (2 * a + s))
                    emit(xp, (i, a))
        for s in (0, 1):
            for i, j in combinations(occ[s], 2):
                for a, b in combinations(vir[s], 2):
                    xp = x ^ (1 << (2 * i + s)) ^ (1 << (2 * j + s)) ^ (1 << (2 * a + s)) ^ (1 << (2 * b + s))
                    emit(xp, (i, j, a, b))
        for ia in occ[0]:
            for aa in vir[0]:
                for ib in occ[1]:
                    for ab in vir[1]:
                        xp = x ^ (1 << (2 * ia)) ^ (1 << (2 * aa)) ^ (1 << (2 * ib + 1)) ^ (1 << (2 * ab + 1))
                        emit(xp, (ia, aa, ib, ab))
        return out

    def n_connected(self) -> int:
        """Closed-form count of off-diagonal connected determinants (the same
        for every determinant of the sector)."""
        from math import comb
        n, a, b = self.n, self.n_alpha, self.n_beta
        return (a * (n - a) + b * (n - b) + comb(a, 2) * comb(n - a, 2)
                + comb(b, 2) * comb(n - b, 2) + a * (n - a) * b * (n - b))

    # -- path B: the operator from Jordan-Wigner Pauli products -----------------
    def dense_jw(self):
        """Full 2^N x 2^N Hamiltonian from JW Pauli strings (sparse matrix).

        Basis index = the integer x (bit q = qubit q); in a Kronecker product
        the leftmost factor is the most significant qubit.
        a_q = Z x ... x Z (qubits < q) x sigma^-... written here as
        I_(N-1) x ... x (X + iY)/2 [qubit q] x Z_(q-1) x ... x Z_0.
        """
        n = self.n
        N = 2 * n
        X = sp.csr_matrix(np.array([[0, 1], [1, 0]], dtype=complex))
        Y = sp.csr_matrix(np.array([[0, -1j], [1j, 0]], dtype=complex))
        Z = sp.csr_matrix(np.array([[1, 0], [0, -1]], dtype=complex))
        I2 = sp.identity(2, dtype=complex, format="csr")
        lower = (X + 1j * Y) * 0.5  # |0><1|: removes an electron
        ann = []
        for q in range(N):
            M = sp.identity(1, dtype=complex, format="csr")
            for r in range(N - 1, -1, -1):
                f = I2 if r > q else (lower if r == q else Z)
                M = sp.kron(M, f, format="csr")
            ann.append(M)
        cre = [a.conj().T.tocsr() for a in ann]
        dim = 1 << N
        H = sp.identity(dim, dtype=complex, format="csr") * self.e_nuc
        for I in range(N):
            for J in range(N):
                if self.hs[I, J] != 0.0:
                    H = H + self.hs[I, J] * (cre[I] @ ann[J])
        for I, J, K, L in np.ndindex(N, N, N, N):
            c = self.gs[I, J, K, L]
            if c != 0.0:
                H = H + (0.5 * c) * (cre[I] @ cre[K] @ ann[L] @ ann[J])
        return H.tocsr()


def sector_matrix(ham: Hamiltonian, states) -> np.ndarray:
    """Dense sector Hamiltonian from path A (rows/cols in the given order)."""
    idx = {x: k for k, x in enumerate(states)}
    M = np.zeros((len(states), len(states)))
    for k, x in enumerate(states):
        M[k, k] = ham.diagonal(x)
        for xp, v, _ in ham.connected(x):
            M[idx[xp], k] = v
    return M
