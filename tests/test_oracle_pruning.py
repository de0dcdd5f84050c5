"""Pruning strategies of unphysical subtrees (Sec. III.C, Fig. 1C): MU, DU
and MU-d in the oracle.

Pins: MU-0 is MU; the unmasked network is a normalised distribution over
all 4^n strings (brute force), so under DU the sector carries the mass
m = sum_sector |psi_DU|^2 < 1 and a DU pass loses a Binomial(N_s, 1 - m)
number of samples; the DU counts follow N_s |psi_DU|^2 (chi-square with the
lost samples as one more bin); under MU the last slot of a fixed (N_a, N_b)
sector is forced, so the network's last-slot outputs cannot change log psi,
while under MU-1 they do (the paper's remark that MU renders the last
subnetwork useless).
"""
import itertools

import numpy as np
import torch

from oracle.anqs import MLPAnsatz, allowed_masks, log_psi, log_psi_from_logits
from oracle.sampler import sample, sample_binomial
from oracle.sector import molecular_isphys, sector_states
from synthetic import workload


def _small():
    w = workload("small", bias_std=0.5)
    return w, MLPAnsatz(w["params_struct"], w["n"]), molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])


def _all_strings(n):
    return np.sort(np.array([sum(v << (2 * p) for p, v in enumerate(vs))
                             for vs in itertools.product(range(4), repeat=n)], dtype=np.uint64))


def test_mu0_is_mu():
    w, om, ip = _small()
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    a0, p0 = log_psi(om, ip, st)
    a1, p1 = log_psi(om, ip, st, du_levels=0)
    assert torch.equal(a0, a1) and torch.equal(p0, p1)
    x0, c0, _ = sample(om, ip, w["n"], 5000, seed=1)
    x1, c1, _ = sample(om, ip, w["n"], 5000, seed=1, du_levels=0)
    assert np.array_equal(x0, x1) and np.array_equal(c0, c1)


def test_unmasked_network_is_normalised_and_du_sector_mass_below_one():
    w, om, ip = _small()
    n = w["n"]
    allx = _all_strings(n)
    free = np.ones((len(allx), n, 4), dtype=bool)
    la, _ = log_psi_from_logits(om.outputs(allx), allx, free, du_levels=n)
    assert abs(np.exp(2 * la.numpy()).sum() - 1.0) < 1e-12
    st = np.array(sector_states(n, w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    ld, _ = log_psi(om, ip, st, du_levels=n)
    m = np.exp(2 * ld.numpy()).sum()
    assert 0.0 < m < 1.0
    # the DU amplitudes of sector strings are the unmasked network's amplitudes
    idx = np.searchsorted(allx, st)
    assert np.allclose(ld.numpy(), la.numpy()[idx], rtol=0, atol=1e-13)
    # everything outside the sector has zero amplitude under every strategy
    out = np.setdiff1d(allx, st)[:50]
    for d in (0, 1, n):
        assert torch.isneginf(log_psi(om, ip, out, du_levels=d)[0]).all()


def test_du_sampler_loses_binomial_fraction_and_follows_du_amplitudes():
    from scipy.stats import chi2
    w, om, ip = _small()
    n = w["n"]
    st = np.array(sector_states(n, w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    ld, _ = log_psi(om, ip, st, du_levels=n)
    prob = np.exp(2 * ld.numpy())
    Ns = 200_000
    for sampler in ("multinomial", "binomial"):
        if sampler == "multinomial":
            x, c, _ = sample(om, ip, n, Ns, seed=4, du_levels=n)
        else:
            x, c = sample_binomial(om, ip, n, Ns, np.random.default_rng(4), du_levels=n)
        assert np.all(np.isin(x, st))
        lost = Ns - c.sum()
        mean, sd = Ns * (1 - prob.sum()), np.sqrt(Ns * prob.sum() * (1 - prob.sum()))
        assert abs(lost - mean) < 5 * sd
        full = np.zeros(len(st) + 1)
        full[np.searchsorted(st, x)] = c
        full[-1] = lost
        expect = Ns * np.append(prob, 1 - prob.sum())
        stat = ((full - expect) ** 2 / expect).sum()
        assert stat < chi2.ppf(1 - 1e-6, len(st))


def test_mu_makes_the_last_subnetwork_useless_mu1_does_not():
    w, om, ip = _small()
    n = w["n"]
    st = np.array(sector_states(n, w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    assert np.all(allowed_masks(ip, st, n)[:, n - 1].sum(1) == 1)  # the last slot is forced
    a_mu, _ = log_psi(om, ip, st)
    a_d1, _ = log_psi(om, ip, st, du_levels=1)
    W, b = om.slots[n - 1][-1]
    b[:4] += torch.tensor([0.3, -0.2, 0.5, 0.1], dtype=b.dtype)  # the last slot's modulus head
    a_mu2, _ = log_psi(om, ip, st)
    a_d12, _ = log_psi(om, ip, st, du_levels=1)
    assert torch.equal(a_mu, a_mu2)
    assert (a_d1 - a_d12).abs().max() > 1e-3
