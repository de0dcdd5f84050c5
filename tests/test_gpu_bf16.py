"""GPU parity of the 16-bit tensor-core MLP form (tcgen05, fp16 operands)
against the FP64 oracle.

Tolerances: every GEMM operand (weights and hidden activations) is rounded to
fp16, a relative error of at most 2^-11 (the unit roundoff of an 11-bit
significand), and the activations also carry the f32 tanh approximation's
relative error (about 2^-11); accumulation is f32.  Per operand U = 2^-10.
Per slot the logits move by O(U); log psi sums n slot terms, each a logit
minus a log-sum-exp, so |d log psi| <= TOL_LOGPSI = 2 U n.  A local energy
then moves by at most
    sum_k |H_k psi(x'_k)/psi(x)| * |e^{d_k} - 1|,  |d_k| <= 2 TOL_LOGPSI,
which the tests evaluate per sample from the oracle's own terms.  The reuse of
the parent's slots is exact arithmetic: it must reproduce a full evaluation
of the same 16-bit network up to the float32 rounding of the amplitude ratios.
"""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz, log_psi
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import sample as osample
from oracle.sector import molecular_isphys, sector_states
from oracle.vmc import energy_stats, local_energy
from synthetic import workload

pytestmark = pytest.mark.gpu
U = 2.0 ** -10  # fp16 rounding (2^-11) + tanh approximation (about 2^-11)


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    return mod


def _setup(A, name):
    w = workload(name, bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, "bf16")
    om = MLPAnsatz(w["params_struct"], w["n"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    return w, ham, params, model, om, ip, oham


def _dev(a):
    return torch.tensor(np.asarray(a).astype(np.int64), device="cuda")


@pytest.mark.parametrize("name", ["small", "h2o"])
def test_logpsi_bf16_within_roundoff_bound(A, name):
    w, ham, params, model, om, ip, oham = _setup(A, name)
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    tol = 2 * U * w["n"]
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < tol
    assert np.abs(ph.cpu().numpy() - rph.numpy()).max() < tol
    # the masked bf16 ansatz is still normalised on the sector (f32 softmax)
    assert abs(np.exp(2 * la.double().cpu().numpy()).sum() - 1.0) < 1e-5
    bad = np.array([0, int(st[0]) ^ 1], dtype=np.uint64)
    assert torch.isneginf(A.logpsi(model, ham, _dev(bad))[0]).all()


@pytest.mark.parametrize("name,Ns", [("small", 10_000), ("h2o", 100_000)])
def test_local_energy_bf16(A, name, Ns):
    w, ham, params, model, om, ip, oham = _setup(A, name)
    ox, on, _ = osample(om, ip, w["n"], Ns, seed=9)
    ere, eim, stats = A.local_energy(model, ham, _dev(ox), _dev(on))
    e_ref = local_energy(om, ip, oham, ox)
    s_ref = energy_stats(e_ref, on)
    # per-sample bound from the oracle's own terms
    tol = 2 * U * w["n"]
    la, _ = log_psi(om, ip, ox)
    lists = [oham.connected(int(x)) for x in ox]
    K = len(lists[0])
    xs = np.array([t[0] for L in lists for t in L], dtype=np.uint64)
    hv = np.array([t[1] for L in lists for t in L]).reshape(-1, K)
    lp, _ = log_psi(om, ip, xs)
    r = np.exp(lp.numpy().reshape(-1, K) - la.numpy()[:, None])
    bound = (np.abs(hv) * r).sum(1) * (np.exp(2 * tol) - 1)
    err = np.abs((ere.cpu().numpy() - e_ref.real) + 1j * (eim.cpu().numpy() - e_ref.imag))
    assert np.all(err <= bound), (err / bound).max()
    wts = on / on.sum()
    st = stats.cpu().numpy()
    assert abs(st[0] - s_ref[0]) <= (wts * err).sum() + 1e-12
    assert st[3] == Ns


@pytest.mark.parametrize("name,Ns", [("small", 10_000), ("h2o", 100_000)])
def test_prefix_reuse_equals_full_evaluation(A, name, Ns):
    """E_loc of the BF16 path (connected determinants evaluated from slot j+1
    on, parent slots reused) equals E_loc assembled from full evaluations of
    the same bf16 network (anqs_logpsi on x and on every x'): the amplitudes
    agree exactly, so only the rounding of the ratios differs."""
    w, ham, params, model, om, ip, oham = _setup(A, name)
    x, n = A.sample(model, ham, Ns, seed=5)
    ere, eim, _ = A.local_energy(model, ham, x, n)
    xp, hv, js, hd = A.connected(ham, x)
    lx, px = A.logpsi(model, ham, x)
    lp, pp = A.logpsi(model, ham, xp.reshape(-1))
    K = ham.n_connected
    r = torch.exp((lp.double().reshape(-1, K) - lx.double()[:, None])
                  + 1j * (pp.double().reshape(-1, K) - px.double()[:, None]))
    e_full = hd + (hv * r).sum(1)
    # the library forms each ratio psi(x')/psi(x) in float32 (expf, sincosf of
    # the float32 log-amplitude differences, a few ulp = ~3e-7 relative) and
    # accumulates in FP64; the reference here forms it in FP64
    bound = 1e-6 * (hv.abs() * r.abs()).sum(1)
    assert ((e_full.real - ere).abs() <= bound).all()
    assert ((e_full.imag - eim).abs() <= bound).all()


@pytest.mark.parametrize("name,Ns", [("small", 200_000), ("h2o", 1_000_000)])
def test_bf16_sampler_follows_bf16_born_distribution(A, name, Ns):
    """The sampler with BF16 conditionals draws from |psi_bf16|^2 (chi-square
    against the BF16 form's own normalised amplitudes on the sector)."""
    from scipy.stats import chi2
    w, ham, params, model, om, ip, oham = _setup(A, name)
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, _ = A.logpsi(model, ham, _dev(st))
    prob = np.exp(2 * la.double().cpu().numpy())
    prob /= prob.sum()
    x, c = A.sample(model, ham, Ns, seed=17)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    assert c.sum() == Ns
    full = np.zeros(len(st))
    full[np.searchsorted(st, x)] = c
    keep = prob * Ns > 5
    stat = ((full[keep] - Ns * prob[keep]) ** 2 / (Ns * prob[keep])).sum()
    assert stat < chi2.ppf(1 - 1e-6, keep.sum() - 1)


def test_bf16_model_sync_tracks_parameter_updates(A):
    w, ham, params, model, om, ip, oham = _setup(A, "small")
    st = _dev(sector_states(w["n"], w["n_alpha"], w["n_beta"]))
    la0, _ = A.logpsi(model, ham, st)
    params.mul_(0.5)
    model.sync()
    la1, _ = A.logpsi(model, ham, st)
    ref = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params.clone(), "bf16")
    la2, _ = A.logpsi(ref, ham, st)
    assert not torch.equal(la0, la1) and torch.equal(la1, la2)
