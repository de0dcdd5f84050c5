"""GPU parity of the MU-d pruning strategies (Sec. III.C): DU (d = n), MU-d
(0 < d < n) and MU (d = 0) against the oracle.

Bars as for MU: sampled sets bit-exact with injected conditionals (the same
float32 split, over all four outcomes on DU levels, with the draws into an
unphysical child discarded); FP32-form log psi, local energies and gradients
within the float32 tolerances of tests/test_gpu_parity.py; the BF16 form's
prefix reuse equal to its full evaluation.
"""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz, log_psi, table_from_state
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import sample as osample
from oracle.sector import molecular_isphys, sector_states
from oracle.vmc import energy_stats, gradient, local_energy
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


def _dev(a):
    return torch.tensor(np.asarray(a).astype(np.int64), device="cuda")


def _mlp(A, name, d):
    w = workload(name, bias_std=0.3)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"]).set_pruning(d)
    om = MLPAnsatz(w["params_struct"], w["n"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    return w, ham, om, ip, oham


@pytest.mark.parametrize("d", [1, 3, 7])
def test_sampler_bit_exact_with_injected_conditionals(A, d):
    """Table ansatz with random (unnormalised) logits on every slot: the
    sampler is exact integer work given the float32 conditionals."""
    n, na, nb = 7, 5, 5
    rng = np.random.default_rng(d)
    tables = [rng.normal(0, 1.5, (4 ** p, 8)).astype(np.float32).astype(np.float64) for p in range(n)]
    h, g, _ = integrals(3, n, 4)
    ham = A.Hamiltonian(h, g, 0.0, na, nb).set_pruning(d)
    model = A.Model.table(n, torch.tensor(np.concatenate([t.ravel() for t in tables]).astype(np.float32),
                                          device="cuda"))
    ip = molecular_isphys(n, na, nb)
    logits = lambda pre, p: tables[p][(np.asarray(pre, dtype=np.uint64) & np.uint64((1 << (2 * p)) - 1)).astype(
        np.int64)][:, :4]
    for Ns in (1, 997, 123_457):
        x, c = A.sample(model, ham, Ns, seed=3, counter=d)
        ox, oc, _ = osample(None, ip, n, Ns, seed=3, counter=d, logits_fn=logits, du_levels=d)
        assert np.array_equal(x.cpu().numpy().astype(np.uint64), ox)
        assert np.array_equal(c.cpu().numpy(), oc)
        assert c.sum().item() <= Ns


@pytest.mark.parametrize("d", [0, 2, 7])
def test_logpsi_eloc_grad_fp32(A, d):
    w, ham, om, ip, oham = _mlp(A, "h2o", d)
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, "fp32")
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st, du_levels=d)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < 2e-5
    assert np.abs(ph.cpu().numpy() - rph.numpy()).max() < 2e-5
    ox, on, _ = osample(om, ip, w["n"], 100_000, seed=9, du_levels=d)
    ere, eim, stats = A.local_energy(model, ham, _dev(ox), _dev(on))
    e_ref = local_energy(om, ip, oham, ox, du_levels=d)
    assert np.abs(ere.cpu().numpy() - e_ref.real).max() < 1e-4
    assert np.abs(eim.cpu().numpy() - e_ref.imag).max() < 1e-4
    s_ref = energy_stats(e_ref, on)
    assert abs(stats.cpu().numpy()[0] - s_ref[0]) < 1e-5 and stats.cpu().numpy()[3] == on.sum()
    g_ref = np.concatenate([t.reshape(-1).numpy() for t in gradient(om, ip, ox, on, e_ref, s_ref, du_levels=d)])
    g = A.grad(model, ham, _dev(ox), _dev(on), torch.tensor(e_ref.real, device="cuda"),
               torch.tensor(e_ref.imag, device="cuda"), torch.tensor(s_ref, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-4


@pytest.mark.parametrize("d", [2, 7])
def test_bf16_prefix_reuse_under_du(A, d):
    w, ham, om, ip, oham = _mlp(A, "h2o", d)
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"), "bf16")
    x, n = A.sample(model, ham, 100_000, seed=5)
    assert n.sum().item() <= 100_000
    ere, eim, _ = A.local_energy(model, ham, x, n)
    xp, hv, js, hd = A.connected(ham, x)
    lx, px = A.logpsi(model, ham, x)
    lp, pp = A.logpsi(model, ham, xp.reshape(-1))
    K = ham.n_connected
    r = torch.exp((lp.double().reshape(-1, K) - lx.double()[:, None])
                  + 1j * (pp.double().reshape(-1, K) - px.double()[:, None]))
    e_full = hd + (hv * r).sum(1)
    bound = 1e-6 * (hv.abs() * r.abs()).sum(1)
    assert ((e_full.real - ere).abs() <= bound).all()
    assert ((e_full.imag - eim).abs() <= bound).all()


def test_tf_du_logpsi_and_binomial(A):
    from scipy.stats import chi2
    from oracle.anqs import TFAnsatz
    w = workload("n2", bias_std=0.2)
    n = w["n"]
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"]).set_pruning(n)
    model = A.Model.transformer(n, w["d_model"], w["n_heads"], w["n_layers"], torch.tensor(w["params"], device="cuda"))
    om = TFAnsatz(w["params_struct"], n, w["n_heads"])
    ip = molecular_isphys(n, w["n_alpha"], w["n_beta"])
    st = np.array(sector_states(n, w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, _ = A.logpsi(model, ham, _dev(st))
    rla, _ = log_psi(om, ip, st, du_levels=n)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < 1e-4
    prob = np.exp(2 * rla.numpy())
    Ns = 10 ** 7
    x, c = A.sample(model, ham, Ns, seed=8, binomial=True)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    lost = Ns - c.sum()
    full = np.zeros(len(st) + 1)
    full[np.searchsorted(st, x)] = c
    full[-1] = lost
    expect = Ns * np.append(prob, 1 - prob.sum())
    keep = expect > 5
    stat = ((full[keep] - expect[keep]) ** 2 / expect[keep]).sum()
    assert stat < chi2.ppf(1 - 1e-6, keep.sum() - 1)
