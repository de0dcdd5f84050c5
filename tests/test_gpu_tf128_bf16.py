"""GPU parity of the BF16 tensor-core transformer form at d_model = 128
(tcgen05, weights streamed through a shared-memory ring) against the FP64
oracle.

The bound is the one of the d = 64 form: the synthetic weights are
bf16-representable, so only activations are rounded (every GEMM operand and
the stored keys and values carry a relative error of at most u = 2^-11 (fp16 operands);
accumulation, softmax, LayerNorm statistics and the head are f32).  Each
slot's logits move by O(u) and log psi, a sum of n slot terms, by at most
TOL = 2 u n.  Reusing the parent's keys and values is exact: positions <= j
of a connected determinant see bit-identical rows in the parent's tile, so
E_loc with reuse equals E_loc assembled from full evaluations of the same
network up to the float32 rounding of the ratios.
"""
import numpy as np
import pytest
import torch

from oracle.anqs import TFAnsatz, log_psi
from oracle.sector import molecular_isphys, sector_states
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


def _model(A, n, na, nb, H, L, seed):
    P = tf_params(seed, n, 128, L, bias_std=0.2)
    h, g, e = integrals(seed, n, n)
    ham = A.Hamiltonian(h, g, e, na, nb)
    model = A.Model.transformer(n, 128, H, L, torch.tensor(flatten_tf(P), device="cuda"), "bf16")
    return P, ham, model


@pytest.mark.parametrize("n,na,nb,H,L", [(4, 2, 2, 8, 1), (6, 3, 2, 4, 2), (8, 4, 3, 8, 2)])
def test_tf128_bf16_logpsi_within_roundoff_bound(A, n, na, nb, H, L):
    P, ham, model = _model(A, n, na, nb, H, L, n + L)
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


def test_tf128_bf16_sampler_slots_match_full_evaluation(A):
    """The sampler's slot launches (last position only) and log psi (every
    position) run the same tiles: a sample drawn with statistics sampling is
    in the sector, and the sample set is normalised by its counts."""
    P, ham, model = _model(A, 8, 4, 3, 8, 2, 11)
    x, c = A.sample(model, ham, 50_000, seed=3)
    assert int(c.sum()) == 50_000
    la, _ = A.logpsi(model, ham, x)
    assert torch.isfinite(la).all()
    assert model.status() == 0


def _full_eval_eloc(A, model, ham, x):
    xp, hv, js, hd = A.connected(ham, x)
    lx, px = A.logpsi(model, ham, x)
    lp, pp = A.logpsi(model, ham, xp.reshape(-1))
    K = ham.n_connected
    r = torch.exp((lp.double().reshape(-1, K) - lx.double()[:, None])
                  + 1j * (pp.double().reshape(-1, K) - px.double()[:, None]))
    return hd + (hv * r).sum(1), (hv.abs() * r.abs()).sum(1), xp


def test_tf128_bf16_prefix_reuse_equals_full_evaluation(A):
    P, ham, model = _model(A, 8, 4, 4, 8, 2, 21)
    x, n = A.sample(model, ham, 100_000, seed=5)
    ere, eim, stats = A.local_energy(model, ham, x, n)
    e_full, mag, _ = _full_eval_eloc(A, model, ham, x)
    bound = 1e-6 * mag
    assert ((e_full.real - ere).abs() <= bound).all()
    assert ((e_full.imag - eim).abs() <= bound).all()
    wts = n.double() / n.double().sum()
    assert abs(float((wts * ere).sum()) - float(stats[0])) <= 1e-12 * float(ere.abs().max())
    assert model.status() == 0


def test_tf128_bf16_logpsi_large_shape_against_oracle(A):
    """26 slots, d 128, 8 heads, 4 blocks (the 52-qubit shape): samples and
    some of their connected determinants against the FP64 oracle."""
    w = workload("large", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"],
                                torch.tensor(w["params"], device="cuda"), "bf16")
    om = TFAnsatz(w["params_struct"], w["n"], w["n_heads"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    x, _ = A.sample(model, ham, 2000, seed=1)
    xs = x.cpu().numpy().astype(np.uint64)[:24]
    xp, _, _, _ = A.connected(ham, _dev(xs[:2]))
    rng = np.random.default_rng(0)
    pick = xp.reshape(-1).cpu().numpy().astype(np.uint64)
    xs = np.concatenate([xs, pick[rng.choice(len(pick), 24, replace=False)]])
    la, ph = A.logpsi(model, ham, _dev(xs))
    rla, rph = log_psi(om, ip, xs)
    tol = 2 * U * w["n"]
    dla = np.abs(la.cpu().numpy() - rla.numpy())
    dph = np.abs(ph.cpu().numpy() - rph.numpy())
    assert dla.max() < tol and dph.max() < tol, (dla.max(), dph.max())
    assert model.status() == 0


def test_tf128_bf16_local_energy_large_shape(A):
    """33,507 connected determinants per sample: E_loc with key/value reuse
    against its definition assembled in FP64 from the library's connected set
    (bit-exact against the oracle) and the full evaluation of every connected
    determinant by the same network (checked against the oracle above)."""
    w = workload("large", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"],
                                torch.tensor(w["params"], device="cuda"), "bf16")
    x, c = A.sample(model, ham, 2000, seed=5)
    x, c = x[:3].contiguous(), c[:3].contiguous()
    ere, eim, stats = A.local_energy(model, ham, x, c)
    e_full, mag, xp = _full_eval_eloc(A, model, ham, x)
    assert xp.shape[1] == 33507
    bound = 1e-6 * mag
    assert ((e_full.real - ere).abs() <= bound).all()
    assert ((e_full.imag - eim).abs() <= bound).all()
    assert model.status() == 0
