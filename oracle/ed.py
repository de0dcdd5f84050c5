"""Exact diagonalisation of a sector (full configuration interaction).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Used only to pin the
local energy: for the exact ground vector, E_loc(x) = E_0 for every x with
nonzero amplitude (Eq. local_energy_def applied to an eigenvector).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .sector import sector_states


def sector_basis(n: int, n_alpha: int, n_beta: int) -> np.ndarray:
    return np.array(sector_states(n, n_alpha, n_beta), dtype=np.uint64)


def ground_state(ham, states, dense_limit: int = 3000):
    """(E_0, c) of the sector Hamiltonian built from the connected lists.
    ``states`` may be a symmetry sector inside the (N_a, N_b) one, provided H
    has no element leading out of it."""
    states = [int(s) for s in states]
    idx = {x: k for k, x in enumerate(states)}
    rows, cols, vals = [], [], []
    for k, x in enumerate(states):
        rows.append(k)
        cols.append(k)
        vals.append(ham.diagonal(x))
        for xp, v, _ in ham.connected(x):
            if xp not in idx:
                # a symmetry sector smaller than the (N_a, N_b) sector (Z2,
                # Sec. IV.A): H must not connect it to the rest
                if v != 0.0:
                    raise ValueError(f"H connects {x} to {xp} outside the given states")
                continue
            rows.append(idx[xp])
            cols.append(k)
            vals.append(v)
    D = len(states)
    M = sp.csr_matrix((vals, (rows, cols)), shape=(D, D))
    if D <= dense_limit:
        w, V = np.linalg.eigh(M.toarray())
        return w[0], V[:, 0]
    w, V = spla.eigsh(M, k=1, which="SA", tol=1e-12)
    return w[0], V[:, 0]
