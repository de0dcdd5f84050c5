"""Pins for local energy, estimator and gradient."""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz, TableAnsatz, TFAnsatz, log_psi, table_from_state
from oracle.ed import ground_state
from oracle.hamiltonian import Hamiltonian
from oracle.sampler import sample
from oracle.sector import molecular_isphys, sector_states
from oracle.vmc import energy_stats, gradient, local_energy
from synthetic import integrals, mlp_params, tf_params, workload


def test_eloc_constant_for_exact_eigenvector_jw():
    """Ground vector of the Jordan-Wigner operator (path B): E_loc(x) = E_0
    for every sector state (Eq. local_energy_def on an eigenvector)."""
    n, na, nb = 4, 2, 2
    h, g, _ = integrals(0, n, 8)
    ham = Hamiltonian(h, g, 0.0, na, nb)
    st = sector_states(n, na, nb)
    HB = ham.dense_jw()[st][:, st].toarray().real
    w, V = np.linalg.eigh(HB)
    ip = molecular_isphys(n, na, nb)
    tab = TableAnsatz(table_from_state(st, V[:, 0], n), n)
    e = local_energy(tab, ip, ham, st)
    assert np.abs(e - w[0]).max() < 1e-10


def test_eloc_constant_for_exact_eigenvector_h2o_shape():
    w = workload("h2o")
    ham = Hamiltonian(w["h"], w["g"], w["e_nuc"], 5, 5)
    st = sector_states(7, 5, 5)
    E0, c = ground_state(ham, st)
    ip = molecular_isphys(7, 5, 5)
    tab = TableAnsatz(table_from_state(st, c, 7), 7)
    e = local_energy(tab, ip, ham, st[::9])
    assert np.abs(e - E0).max() < 1e-10


def _small_problem(kind="mlp"):
    n, na, nb = 4, 2, 2
    h, g, _ = integrals(0, n, 8)
    ham = Hamiltonian(h, g, 0.0, na, nb)
    ip = molecular_isphys(n, na, nb)
    if kind == "mlp":
        model = MLPAnsatz(mlp_params(0, n, 16, 2, bias_std=0.5), n)
    else:
        model = TFAnsatz(tf_params(0, n, 8, 1, bias_std=0.3), n, 2)
    return n, ham, ip, model


def test_rayleigh_quotient_vs_sample_mean():
    n, ham, ip, model = _small_problem()
    st = np.array(sector_states(n, 2, 2), dtype=np.uint64)
    la, _ = log_psi(model, ip, st)
    prob = np.exp(2 * la.numpy())
    eall = local_energy(model, ip, ham, st)
    E_exact = (prob * eall).sum()
    assert abs(E_exact.imag) < 1e-12
    var = (prob * np.abs(eall - E_exact) ** 2).sum()
    for Ns in (1000, 10000, 100000):
        xs, cnt, _ = sample(model, ip, n, Ns, seed=Ns)
        e = local_energy(model, ip, ham, xs)
        st4 = energy_stats(e, cnt)
        assert abs(st4[0] - E_exact.real) < 4 * np.sqrt(var / Ns)
        assert st4[3] == Ns


def _flat(gs):
    return torch.cat([g.reshape(-1) for g in gs]).numpy()


@pytest.mark.parametrize("kind", ["mlp", "tf"])
def test_gradient_vs_central_differences_of_surrogate(kind):
    """grad = d/dtheta of sum_l w_l 2 (Re dE_l log|psi_l| + Im dE_l phase_l)
    with E_loc and E frozen; checked coordinate-wise by central differences."""
    n, ham, ip, model = _small_problem(kind)
    xs, cnt, _ = sample(model, ip, n, 3000, seed=3)
    e = local_energy(model, ip, ham, xs)
    stats = energy_stats(e, cnt)
    g = _flat(gradient(model, ip, xs, cnt, e, stats))
    params = model.parameters()
    sizes = [t.numel() for t in params]
    w = cnt / stats[3]

    def surrogate():
        with torch.no_grad():
            la, ph = log_psi(model, ip, xs)
        return float((2 * w * (e.real - stats[0]) * la.numpy()).sum()
                     + (2 * w * (e.imag - stats[1]) * ph.numpy()).sum())

    rng = np.random.default_rng(0)
    idx = rng.choice(sum(sizes), size=16, replace=False)
    h = 1e-4
    for flat_i in idx:
        k = int(np.searchsorted(np.cumsum(sizes), flat_i, side="right"))
        j = flat_i - (sum(sizes[:k]))
        t = params[k].view(-1)
        old = t[j].item()
        t[j] = old + h
        fp = surrogate()
        t[j] = old - h
        fm = surrogate()
        t[j] = old
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[flat_i]) < 1e-7 * max(1.0, abs(fd))


def test_gradient_equals_exact_energy_gradient():
    """With weights |psi(x)|^2 over the whole sector, the estimator of
    Eq. grad_def equals the exact gradient of the Rayleigh quotient E(theta),
    checked by central differences of E(theta)."""
    n, ham, ip, model = _small_problem()
    st = np.array(sector_states(n, 2, 2), dtype=np.uint64)

    def energy():
        with torch.no_grad():
            la, _ = log_psi(model, ip, st)
        p = np.exp(2 * la.numpy())
        return float((p * local_energy(model, ip, ham, st)).sum().real)

    with torch.no_grad():
        la, _ = log_psi(model, ip, st)
    p = np.exp(2 * la.numpy())
    e = local_energy(model, ip, ham, st)
    g = _flat(gradient(model, ip, st, p, e))
    params = model.parameters()
    sizes = [t.numel() for t in params]
    rng = np.random.default_rng(1)
    for flat_i in rng.choice(sum(sizes), size=12, replace=False):
        k = int(np.searchsorted(np.cumsum(sizes), flat_i, side="right"))
        j = flat_i - sum(sizes[:k])
        t = params[k].view(-1)
        old = t[j].item()
        t[j] = old + 1e-5
        fp = energy()
        t[j] = old - 1e-5
        fm = energy()
        t[j] = old
        fd = (fp - fm) / 2e-5
        assert abs(fd - g[flat_i]) < 1e-7 * max(1.0, abs(fd))


def test_energy_stats_equal_the_statistics_of_the_expanded_sample_list():
    """Eq. energy_est over unique samples with occurrence numbers equals the
    plain mean over the N_s individual samples; the variance (reading: the
    count-weighted population variance with the complex mean) equals numpy's
    population variance of the expanded list, real and imaginary parts added."""
    rng = np.random.default_rng(7)
    e = -75.0 + rng.normal(size=40) * 1.3 + 1j * rng.normal(size=40) * 1e-2
    n = rng.integers(1, 50, size=40)
    st = energy_stats(e, n)
    full = np.repeat(e, n)
    assert st[3] == n.sum() == full.size
    assert abs(st[0] - full.real.mean()) <= 1e-12 * abs(full.real.mean())
    assert abs(st[1] - full.imag.mean()) <= 1e-12
    var = full.real.var() + full.imag.var()
    assert abs(st[2] - var) <= 1e-10 * var
    # a single sample has zero variance; equal energies too
    assert energy_stats(e[:1], n[:1])[2] == 0.0
    assert energy_stats(np.full(5, -3.0 + 0j), np.arange(1, 6))[2] == 0.0
