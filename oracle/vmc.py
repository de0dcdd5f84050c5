"""Local energy, energy estimator, variance and VMC gradient (Sec. II.A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* E_loc(x) = sum_x' H_xx' psi(x') / psi(x)        (Eq. local_energy_def)
  = H_xx + sum over the connected set of H_xx' exp(log psi(x') - log psi(x)),
  complex, FP64.
* E_est = sum_l E_loc(x_l) n_l / N_s              (Eq. energy_est); the
  normaliser is sum_l n_l, which equals N_s under MU.  Stats returned:
  (Re E, Im E, Var, sum n) with Var = sum_l n_l |E_loc,l - E|^2 / sum n
  (reading: the paper does not define the variance; this is the
  count-weighted population variance with the complex mean E).
* grad E = 2 Re{ E[E_loc d ln psi*] - E[E_loc] E[d ln psi*] }   (Eq. grad_def)
  with expectations taken with weights n_l / sum n and E_loc held fixed.
  With ln psi = log|psi| + i phase this is
  sum_l w_l 2 (Re(E_loc,l - E) d log|psi| + Im(E_loc,l - E) d phase).

Pins: E_loc equals the exact ground energy for the exact eigenvector, the
Rayleigh quotient against the sample mean, and the gradient against central
finite differences and against the exact gradient of the sector Rayleigh
quotient (tests/test_oracle_vmc.py).
"""
from __future__ import annotations

import numpy as np
import torch

from .anqs import log_psi


def connected_lists(ham, xs):
    """Per x: list of (x', H, j) plus the diagonal element."""
    return [ham.connected(int(x)) for x in xs], np.array([ham.diagonal(int(x)) for x in xs])


def local_energy(model, isphys, ham, xs, lists=None, diag=None, du_levels: int = 0):
    """Complex E_loc per unique sample, FP64."""
    xs = np.asarray(xs, dtype=np.uint64)
    if lists is None:
        lists, diag = connected_lists(ham, xs)
    flat_x = np.array([xp for L in lists for xp, _, _ in L], dtype=np.uint64)
    flat_h = np.array([v for L in lists for _, v, _ in L], dtype=np.float64)
    sizes = [len(L) for L in lists]
    with torch.no_grad():
        la, ph = log_psi(model, isphys, xs, du_levels=du_levels)
        la_p, ph_p = (log_psi(model, isphys, flat_x, du_levels=du_levels) if len(flat_x)
                      else (torch.zeros(0), torch.zeros(0)))
    la, ph, la_p, ph_p = (t.numpy() for t in (la, ph, la_p, ph_p))
    e = np.zeros(len(xs), dtype=np.complex128)
    off = 0
    for l in range(len(xs)):
        k = sizes[l]
        r = np.exp((la_p[off:off + k] - la[l]) + 1j * (ph_p[off:off + k] - ph[l]))
        acc = complex(diag[l])
        for t in range(k):
            acc += flat_h[off + t] * r[t]
        e[l] = acc
        off += k
    return e


def energy_stats(eloc, counts):
    """(Re E, Im E, Var, sum n) from E_loc and the occurrence numbers."""
    eloc = np.asarray(eloc, dtype=np.complex128)
    w = np.asarray(counts, dtype=np.float64)
    S = w.sum()
    E = (w * eloc).sum() / S
    var = (w * np.abs(eloc - E) ** 2).sum() / S
    return np.array([E.real, E.imag, var, S])


def combine_stats(stats_list):
    """Statistics of the union of disjoint sample sets from the statistics of
    each (the estimator of Eq. energy_est over all samples): S = sum S_r,
    E = sum S_r E_r / S, Var = sum S_r (Var_r + |E_r - E|^2) / S.  Empty
    sets (S_r = 0) contribute nothing."""
    st = np.asarray(stats_list, dtype=np.float64).reshape(-1, 4)
    st = st[st[:, 3] > 0]
    S = st[:, 3].sum()
    Er = (st[:, 3] * st[:, 0]).sum() / S
    Ei = (st[:, 3] * st[:, 1]).sum() / S
    var = (st[:, 3] * (st[:, 2] + (st[:, 0] - Er) ** 2 + (st[:, 1] - Ei) ** 2)).sum() / S
    return np.array([Er, Ei, var, S])


def gradient(model, isphys, xs, counts, eloc, stats=None, du_levels: int = 0):
    """VMC gradient (Eq. grad_def) with respect to model.parameters(), FP64."""
    xs = np.asarray(xs, dtype=np.uint64)
    if stats is None:
        stats = energy_stats(eloc, counts)
    w = np.asarray(counts, dtype=np.float64) / stats[3]
    dre = np.asarray(eloc).real - stats[0]
    dim = np.asarray(eloc).imag - stats[1]
    params = model.parameters()
    for t in params:
        t.requires_grad_(True)
        t.grad = None
    la, ph = log_psi(model, isphys, xs, du_levels=du_levels)
    L = (torch.as_tensor(2.0 * w * dre) * la).sum() + (torch.as_tensor(2.0 * w * dim) * ph).sum()
    grads = torch.autograd.grad(L, params, allow_unused=True)
    for t in params:
        t.requires_grad_(False)
    return [g if g is not None else torch.zeros_like(t) for g, t in zip(grads, params)]
