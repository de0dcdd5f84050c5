"""The paper's per-qubit NADE (Appendix B.1) in the oracle.

Pins: an independent scalar evaluation of the literal per-qubit definition
(each qubit's complex MLP in plain numpy, binary conditionals masked by the
qubit-level IsPhys of Algorithm 1 and renormalised in modulus) equals the
slot formulation used by the library (qubits 2p and 2p + 1 grouped into
slot p); the masked ansatz is normalised on the sector and the unmasked one
(DU everywhere) on all 4^n strings, by brute force; every qubit's f3 output
is a normalised binary distribution.
"""
import itertools

import numpy as np
import pytest

from oracle.anqs import NADEAnsatz, log_psi, log_psi_from_logits
from oracle.sector import molecular_isphys, sector_states
from synthetic import nade_params


def _scalar_logpsi(qubits, ip, x, n):
    """log psi(x) = sum_i log psi_i(x_i | x_<i), qubit by qubit (complex)."""
    bits = [(int(x) >> q) & 1 for q in range(2 * n)]
    total = 0j
    for i in range(2 * n):
        W1, b1, W2, b2, W3, b3 = qubits[i]
        z = b1.copy()
        for k in range(i):
            z = z + W1[:, k] * bits[k]
        h = np.tanh(z)
        z = W2 @ h + b2
        h = np.where(z.real >= 0, z.real, 0.01 * z.real) + 1j * np.where(z.imag >= 0, z.imag, 0.01 * z.imag)
        z = W3 @ h + b3
        m = max(2 * z[0].real, 2 * z[1].real)
        lq = z - 0.5 * (m + np.log(np.exp(2 * z[0].real - m) + np.exp(2 * z[1].real - m)))
        allowed = [ip.of_prefix(bits[:i] + [b]) for b in (0, 1)]
        if not allowed[bits[i]]:
            return complex(-np.inf, 0.0)
        re = [lq[b].real if allowed[b] else -np.inf for b in (0, 1)]
        mm = max(r for r in re if np.isfinite(r))
        norm = 0.5 * np.log(sum(np.exp(2 * (r - mm)) for r in re if np.isfinite(r))) + mm
        total += (lq[bits[i]].real - norm) + 1j * lq[bits[i]].imag
    return total


@pytest.mark.parametrize("n,na,nb,w", [(3, 1, 2, 8), (4, 2, 2, 16), (4, 1, 1, 8)])
def test_slot_formulation_equals_per_qubit_definition(n, na, nb, w):
    qubits = nade_params(n + w, n, w, bias_std=0.4)
    ip = molecular_isphys(n, na, nb)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, ph = log_psi(NADEAnsatz(qubits, n, ip), ip, st)
    for k, x in enumerate(st):
        ref = _scalar_logpsi(qubits, ip, x, n)
        assert abs(la[k].item() - ref.real) < 1e-12
        d = (ph[k].item() - ref.imag + np.pi) % (2 * np.pi) - np.pi
        assert abs(d) < 1e-12


@pytest.mark.parametrize("n,na,nb", [(3, 1, 2), (4, 2, 2)])
def test_masked_nade_normalised_on_sector_and_du_on_all_strings(n, na, nb):
    qubits = nade_params(5, n, 16, bias_std=0.3)
    ip = molecular_isphys(n, na, nb)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, _ = log_psi(NADEAnsatz(qubits, n, ip), ip, st)
    assert abs(np.exp(2 * la.numpy()).sum() - 1.0) < 1e-12
    allx = np.sort(np.array([sum(v << (2 * p) for p, v in enumerate(vs))
                             for vs in itertools.product(range(4), repeat=n)], dtype=np.uint64))
    du = NADEAnsatz(qubits, n, ip, du_levels=n)
    free = np.ones((len(allx), n, 4), dtype=bool)
    lf, _ = log_psi_from_logits(du.outputs(allx), allx, free, du_levels=n)
    assert abs(np.exp(2 * lf.numpy()).sum() - 1.0) < 1e-12


def test_each_qubit_conditional_is_normalised():
    import torch
    qubits = nade_params(2, 3, 8, bias_std=0.5)
    om = NADEAnsatz(qubits, 3, molecular_isphys(3, 1, 1))
    rng = np.random.default_rng(0)
    for i in range(6):
        bits = torch.tensor(rng.integers(0, 2, (7, i)).astype(np.float64))
        lq = om._qubit(i, bits)
        assert torch.allclose(torch.exp(2 * lq.real).sum(1), torch.ones(7, dtype=torch.float64), atol=1e-13)


def test_nade_gradient_matches_central_differences():
    """The oracle's NADE gradient (autograd through log psi, which the GPU
    adjoint is tested against) equals FP64 central differences of
    L = sum_l [c_l log|psi(x_l)| + c'_l arg psi(x_l)] on 12 random real and
    imaginary weight parts.  L is piecewise smooth (LeReLU), so a parameter
    is used only where the differences with steps h and h/2 agree to their
    rounding, i.e. no kink lies within the stencil."""
    import torch
    n, na, nb, w = 3, 2, 1, 8
    qubits = nade_params(9, n, w, bias_std=0.4)
    ip = molecular_isphys(n, na, nb)
    om = NADEAnsatz(qubits, n, ip)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    rng = np.random.default_rng(3)
    ca, cp = torch.tensor(rng.normal(size=len(st))), torch.tensor(rng.normal(size=len(st)))
    ps = om.parameters()
    for t in ps:
        t.requires_grad_(True)
    la, ph = log_psi(om, ip, st)
    grads = torch.autograd.grad((ca * la).sum() + (cp * ph).sum(), ps, allow_unused=True)
    for t in ps:
        t.requires_grad_(False)

    def loss():
        a, b = log_psi(om, ip, st)
        return float((ca * a).sum() + (cp * b).sum())

    sizes = [t.numel() for t in ps]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    h, checked = 1e-4, 0
    for i in rng.permutation(offs[-1]):
        if checked == 12:
            break
        k = int(np.searchsorted(offs, i, side="right") - 1)
        flat = ps[k].view(-1)
        j = int(i - offs[k])
        old = float(flat[j])
        d = {}
        for step in (h, h / 2):
            flat[j] = old + step
            lp = loss()
            flat[j] = old - step
            lm = loss()
            flat[j] = old
            d[step] = (lp - lm) / (2 * step)
        if abs(d[h] - d[h / 2]) > 1e-9 * max(1.0, abs(d[h])):
            continue  # a LeReLU kink within the stencil
        g = float(grads[k].view(-1)[j]) if grads[k] is not None else 0.0
        assert abs(g - d[h / 2]) <= 1e-7 * max(1.0, abs(g)), (k, j, g, d)
        checked += 1
    assert checked == 12
