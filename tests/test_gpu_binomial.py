"""Binomial statistics sampling on the device (Sec. II.C): parity with the
oracle is in distribution (the binomial draws are random variates).

Pins: the counts add up to N_s exactly (MU), every leaf lies in the sector,
the leaves come out in the tree's order; the counts follow N_s |psi|^2
(chi-square) for injected exact conditionals at N_s up to 1e8; and a single
free node reproduces the multinomial moments in both regimes of the
binomial generator (inversion for n min(p, 1-p) < 10, BTRS above).
"""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz, log_psi, table_from_state
from oracle.sampler import lexicographic_key
from oracle.sector import molecular_isphys, sector_states
from synthetic import integrals, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    return mod


def _table(A, n, na, nb, seed):
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    c = np.random.default_rng(seed).normal(size=len(st))
    c /= np.linalg.norm(c)
    tables = [np.maximum(t, -60.0).astype(np.float32) for t in table_from_state(st, c, n)]
    h, g, _ = integrals(seed, n, n)
    ham = A.Hamiltonian(h, g, 0.0, na, nb)
    model = A.Model.table(n, torch.tensor(np.concatenate([t.reshape(-1) for t in tables]), device="cuda"))
    return ham, model, st, c ** 2


@pytest.mark.parametrize("n,na,nb,Ns", [(4, 2, 2, 10 ** 6), (7, 5, 5, 10 ** 8), (6, 1, 4, 12345)])
def test_binomial_sampler_follows_born_distribution(A, n, na, nb, Ns):
    from scipy.stats import chi2
    ham, model, st, prob = _table(A, n, na, nb, seed=n)
    x, c = A.sample(model, ham, Ns, seed=11, binomial=True)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    assert c.sum() == Ns and np.all(c > 0)
    assert np.all(np.isin(x, st))
    assert np.all(np.diff(lexicographic_key(x, n).astype(np.float64)) > 0)
    full = np.zeros(len(st))
    full[np.searchsorted(st, x)] = c
    keep = prob * Ns > 5
    stat = ((full[keep] - Ns * prob[keep]) ** 2 / (Ns * prob[keep])).sum()
    assert stat < chi2.ppf(1 - 1e-6, keep.sum() - 1)
    assert ham.status() == 0  # no binomial draw left its rejection loop or its inversion walk early


@pytest.mark.parametrize("N", [12, 10 ** 8])
def test_binomial_node_has_multinomial_moments(A, N):
    """2 orbitals, 1 + 1 electrons: slot 0 free, slot 1 forced; R passes with
    different Philox counters."""
    p = np.array([0.5, 0.3, 0.15, 0.05])
    t0 = np.zeros((1, 8))
    t0[0, :4] = np.log(p)
    t1 = np.zeros((4, 8))
    h, g, _ = integrals(1, 2, 2)
    ham = A.Hamiltonian(h, g, 0.0, 1, 1)
    model = A.Model.table(2, torch.tensor(np.concatenate([t0.ravel(), t1.ravel()]).astype(np.float32), device="cuda"))
    pf = np.exp(np.log(p).astype(np.float32).astype(np.float64))
    pf /= pf.sum()
    R = 400
    counts = np.zeros((R, 4))
    for r in range(R):
        x, c = A.sample(model, ham, N, seed=5, counter=r, binomial=True)
        counts[r, (x.cpu().numpy() & 3).astype(int)] = c.cpu().numpy()
    assert np.all(counts.sum(1) == N)
    assert ham.status(clear=True) == 0 and ham.status() == 0
    mean, var = counts.mean(0), counts.var(0, ddof=1)
    sd = np.sqrt(N * pf * (1 - pf))
    assert np.all(np.abs(mean - N * pf) < 5 * sd / np.sqrt(R))
    assert np.all(np.abs(var / sd ** 2 - 1) < 5 * np.sqrt(2 / R))


def test_binomial_sampler_mlp_1e8(A):
    """Live FP32 network, N_s = 1e8: counts against N_s |psi|^2 of the oracle
    (the float32 conditional moves expected counts by ~1e-7 relative, far
    below the sqrt(N_s p) fluctuations)."""
    from scipy.stats import chi2
    w = workload("h2o", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"))
    Ns = 10 ** 8
    x, c = A.sample(model, ham, Ns, seed=2, binomial=True)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    assert c.sum() == Ns
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, _ = log_psi(MLPAnsatz(w["params_struct"], w["n"]), molecular_isphys(w["n"], 5, 5), st)
    prob = np.exp(2 * la.numpy())
    full = np.zeros(len(st))
    full[np.searchsorted(st, x)] = c
    keep = prob * Ns > 5
    stat = ((full[keep] - Ns * prob[keep]) ** 2 / (Ns * prob[keep])).sum()
    assert stat < chi2.ppf(1 - 1e-6, keep.sum() - 1)
