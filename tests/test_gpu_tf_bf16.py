"""GPU parity of the BF16 tensor-core transformer form (tcgen05, d = 64)
against the FP64 oracle.

The synthetic weights are bf16-representable, so only activations are
rounded: every GEMM operand (LayerNorm outputs, attention outputs, FFN hidden
units) and the stored keys and values carry a relative error of at most
u = 2^-11 (fp16 operands); accumulation, softmax, LayerNorm statistics and the head are f32.
As for the MLP form, each slot's logits move by O(u) and log psi, a sum of n
slot terms, by at most TOL = 2 u n; a local energy moves by at most
sum_k |H_k psi(x'_k)/psi(x)| (e^{2 TOL} - 1).  Reusing the parent's keys and
values is exact: a connected determinant's positions <= j see bit-identical
rows in the parent's tile, so E_loc with reuse equals E_loc assembled from
full evaluations of the same network up to the float32 rounding of the
ratios.
"""
import numpy as np
import pytest
import torch

from oracle.anqs import TFAnsatz, log_psi
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import sample as osample
from oracle.sector import molecular_isphys, sector_states
from oracle.vmc import energy_stats, local_energy
from synthetic import flatten_tf, integrals, tf_params, workload

pytestmark = pytest.mark.gpu
U = 2.0 ** -11  # fp16 operands: unit roundoff of an 11-bit significand


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


def _n2(A):
    w = workload("n2", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"], params, "bf16")
    om = TFAnsatz(w["params_struct"], w["n"], w["n_heads"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    return w, ham, params, model, om, ip, oham


@pytest.mark.parametrize("n,na,nb,H,L", [(4, 2, 2, 4, 1), (6, 3, 2, 2, 3), (10, 7, 7, 4, 2)])
def test_tf_bf16_logpsi_within_roundoff_bound(A, n, na, nb, H, L):
    P = tf_params(n + L, n, 64, L, bias_std=0.2)
    h, g, e = integrals(n, n, n)
    ham = A.Hamiltonian(h, g, e, na, nb)
    model = A.Model.transformer(n, 64, H, L, torch.tensor(flatten_tf(P), device="cuda"), "bf16")
    om = TFAnsatz(P, n, H)
    ip = molecular_isphys(n, na, nb)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    tol = 2 * U * n
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < tol
    assert np.abs(ph.cpu().numpy() - rph.numpy()).max() < tol
    # the masked BF16 ansatz is still normalised on the sector (f32 softmax)
    assert abs(np.exp(2 * la.double().cpu().numpy()).sum() - 1.0) < 1e-4
    assert torch.isneginf(A.logpsi(model, ham, _dev([0, int(st[0]) ^ 1]))[0]).all()
    assert model.status() == 0


def test_tf_bf16_prefix_reuse_equals_full_evaluation(A):
    w, ham, params, model, om, ip, oham = _n2(A)
    x, n = A.sample(model, ham, 200_000, seed=5)
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
    assert model.status() == 0


def test_tf_bf16_local_energy_against_oracle(A):
    w, ham, params, model, om, ip, oham = _n2(A)
    ox, on, _ = osample(om, ip, w["n"], 20_000, seed=9)
    keep = np.argsort(-on, kind="stable")[:96]
    ox, on = ox[keep], on[keep]
    ere, eim, stats = A.local_energy(model, ham, _dev(ox), _dev(on))
    e_ref = local_energy(om, ip, oham, ox)
    tol = 2 * U * w["n"]
    la, _ = log_psi(om, ip, ox)
    lists = [oham.connected(int(v)) for v in ox]
    K = len(lists[0])
    xs = np.array([t[0] for L in lists for t in L], dtype=np.uint64)
    hv = np.array([t[1] for L in lists for t in L]).reshape(-1, K)
    lp, _ = log_psi(om, ip, xs)
    r = np.exp(lp.numpy().reshape(-1, K) - la.numpy()[:, None])
    bound = (np.abs(hv) * r).sum(1) * (np.exp(2 * tol) - 1)
    err = np.abs((ere.cpu().numpy() - e_ref.real) + 1j * (eim.cpu().numpy() - e_ref.imag))
    assert np.all(err <= bound), (err / bound).max()
    s_ref = energy_stats(e_ref, on)
    wts = on / on.sum()
    assert abs(stats.cpu().numpy()[0] - s_ref[0]) <= (wts * err).sum() + 1e-12


def test_tf_bf16_sampler_follows_bf16_born_distribution(A):
    from scipy.stats import chi2
    w, ham, params, model, om, ip, oham = _n2(A)
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, _ = A.logpsi(model, ham, _dev(st))
    prob = np.exp(2 * la.double().cpu().numpy())
    prob /= prob.sum()
    Ns = 1_000_000
    x, c = A.sample(model, ham, Ns, seed=17)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    assert c.sum() == Ns
    full = np.zeros(len(st))
    full[np.searchsorted(st, x)] = c
    keep = prob * Ns > 5
    stat = ((full[keep] - Ns * prob[keep]) ** 2 / (Ns * prob[keep])).sum()
    assert stat < chi2.ppf(1 - 1e-6, keep.sum() - 1)


def test_tf_bf16_sync_tracks_parameter_updates(A):
    w, ham, params, model, om, ip, oham = _n2(A)
    st = _dev(sector_states(w["n"], w["n_alpha"], w["n_beta"])[:512])
    la0, _ = A.logpsi(model, ham, st)
    params.mul_(0.5)
    model.sync()
    la1, _ = A.logpsi(model, ham, st)
    ref = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"], params.clone(), "bf16")
    la2, _ = A.logpsi(ref, ham, st)
    assert not torch.equal(la0, la1) and torch.equal(la1, la2)
    assert model.status() == 0 and ref.status() == 0
