"""GPU parity of the causal-transformer ansatz, FP32 form (SIMT), against the
FP64 oracle.

The FP32 forward carries a relative rounding error of a few float32 ulp per
operation through LayerNorm, attention and the FFN; over L blocks and n
slot terms the log-amplitude moves by much less than TOL = 1e-4 (the
measured error is ~1e-6).  A local energy then moves by at most
sum_k |H_k psi(x'_k)/psi(x)| (e^{2 TOL} - 1), evaluated per sample from the
oracle's own terms; the sampler may send a draw another way only when it
falls within the conditional's FP32 error of a boundary (counted by the
oracle with tol = 1e-5).
"""
import numpy as np
import pytest
import torch

from oracle.anqs import TFAnsatz, log_psi
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import lexicographic_key, sample as osample
from oracle.sector import molecular_isphys, sector_states
from oracle.vmc import energy_stats, local_energy
from synthetic import flatten_tf, integrals, tf_params, workload

pytestmark = pytest.mark.gpu
TOL = 1e-4


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


def _custom(A, n, na, nb, d, H, L, seed):
    P = tf_params(seed, n, d, L, bias_std=0.2)
    h, g, e = integrals(seed, n, n)
    ham = A.Hamiltonian(h, g, e, na, nb)
    model = A.Model.transformer(n, d, H, L, torch.tensor(flatten_tf(P), device="cuda"))
    return ham, model, TFAnsatz(P, n, H), molecular_isphys(n, na, nb), OHam(h, g, e, na, nb)


def _n2(A):
    w = workload("n2", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"],
                                torch.tensor(w["params"], device="cuda"))
    om = TFAnsatz(w["params_struct"], w["n"], w["n_heads"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    return w, ham, model, om, ip, oham


@pytest.mark.parametrize("n,na,nb,d,H,L", [(4, 2, 2, 32, 2, 1), (5, 2, 3, 64, 4, 2), (6, 3, 3, 128, 8, 2),
                                           (5, 2, 2, 256, 4, 1)])
def test_tf_logpsi_fp32_every_width(A, n, na, nb, d, H, L):
    ham, model, om, ip, _ = _custom(A, n, na, nb, d, H, L, seed=n + d)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < TOL
    assert np.abs(ph.cpu().numpy() - rph.numpy()).max() < TOL
    bad = np.array([0, int(st[0]) ^ 1], dtype=np.uint64)
    assert torch.isneginf(A.logpsi(model, ham, _dev(bad))[0]).all()


def test_tf_logpsi_fp32_n2_whole_sector(A):
    w, ham, model, om, ip, _ = _n2(A)
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < TOL
    assert np.abs(ph.cpu().numpy() - rph.numpy()).max() < TOL
    # normalised on the sector
    assert abs(np.exp(2 * la.double().cpu().numpy()).sum() - 1.0) < 1e-4


def test_tf_logpsi_fp32_large_shape(A):
    """26 slots, d 128, 8 heads, 4 blocks: two sequences per tile."""
    w = workload("large", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"],
                                torch.tensor(w["params"], device="cuda"))
    om = TFAnsatz(w["params_struct"], w["n"], w["n_heads"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    x, _ = A.sample(model, ham, 2000, seed=1)
    xs = x.cpu().numpy().astype(np.uint64)[:97]
    la, ph = A.logpsi(model, ham, _dev(xs))
    rla, rph = log_psi(om, ip, xs)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < TOL
    assert np.abs(ph.cpu().numpy() - rph.numpy()).max() < TOL


def test_tf_sampler_fp32_n2(A):
    w, ham, model, om, ip, _ = _n2(A)
    Ns = 100_000
    x, c = A.sample(model, ham, Ns, seed=3, counter=2)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    ox, on, _, n_close = osample(om, ip, w["n"], Ns, seed=3, counter=2, tol=1e-5)
    assert c.sum() == Ns
    allx = np.union1d(ox, x)
    a = np.zeros(len(allx), np.int64)
    b = np.zeros(len(allx), np.int64)
    a[np.searchsorted(allx, ox)] = on
    b[np.searchsorted(allx, x)] = c
    assert np.abs(a - b).sum() <= 2 * n_close
    assert np.all(np.diff(lexicographic_key(x, w["n"]).astype(np.float64)) > 0)


def test_tf_local_energy_fp32_n2(A):
    w, ham, model, om, ip, oham = _n2(A)
    ox, on, _ = osample(om, ip, w["n"], 20_000, seed=9)
    keep = np.argsort(-on, kind="stable")[:96]  # the most frequent samples (bounded oracle work)
    ox, on = ox[keep], on[keep]
    ere, eim, stats = A.local_energy(model, ham, _dev(ox), _dev(on))
    e_ref = local_energy(om, ip, oham, ox)
    la, _ = log_psi(om, ip, ox)
    lists = [oham.connected(int(v)) for v in ox]
    K = len(lists[0])
    xs = np.array([t[0] for L in lists for t in L], dtype=np.uint64)
    hv = np.array([t[1] for L in lists for t in L]).reshape(-1, K)
    lp, _ = log_psi(om, ip, xs)
    r = np.exp(lp.numpy().reshape(-1, K) - la.numpy()[:, None])
    bound = (np.abs(hv) * r).sum(1) * (np.exp(2 * TOL) - 1)
    err = np.abs((ere.cpu().numpy() - e_ref.real) + 1j * (eim.cpu().numpy() - e_ref.imag))
    assert np.all(err <= bound), (err / bound).max()
    s_ref = energy_stats(e_ref, on)
    wts = on / on.sum()
    assert abs(stats.cpu().numpy()[0] - s_ref[0]) <= (wts * err).sum() + 1e-12


# ---------------------------------------------------------------------------
# adjoint (FP32): the VJP of the masked log psi against the FP64 oracle's
# autograd, for arbitrary cotangents and through anqs_grad (Eq. grad_def)
# ---------------------------------------------------------------------------
def _flat_grad(gs):
    return np.concatenate([t.reshape(-1).numpy() for t in gs])


@pytest.mark.parametrize("n,na,nb,d,H,L", [(4, 2, 2, 32, 2, 1), (5, 2, 3, 64, 4, 2), (6, 3, 3, 128, 8, 2),
                                           (5, 2, 2, 256, 4, 1)])
def test_tf_logpsi_vjp_every_width(A, n, na, nb, d, H, L):
    ham, model, om, ip, _ = _custom(A, n, na, nb, d, H, L, seed=n + d)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    rng = np.random.default_rng(d)
    ca, cp = rng.normal(size=len(st)), rng.normal(size=len(st))
    g = A.logpsi_vjp(model, ham, _dev(st), torch.tensor(ca, device="cuda"), torch.tensor(cp, device="cuda"))
    ps = om.parameters()
    for t in ps:
        t.requires_grad_(True)
    la, ph = log_psi(om, ip, st)
    ref = _flat_grad(torch.autograd.grad((torch.tensor(ca) * la).sum() + (torch.tensor(cp) * ph).sum(), ps))
    for t in ps:
        t.requires_grad_(False)
    got = g.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 1e-4, rel


def test_tf_grad_n2_against_oracle(A):
    """anqs_grad on sampled unique determinants with given local energies
    (any values: the gradient is linear in the cotangents they define)."""
    from oracle.vmc import gradient
    w, ham, model, om, ip, oham = _n2(A)
    x, c = A.sample(model, ham, 50_000, seed=12)
    xs, cs = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    rng = np.random.default_rng(3)
    e = rng.normal(-10, 1, len(xs)) + 1j * rng.normal(0, 0.1, len(xs))
    st = energy_stats(e, cs)
    g = A.grad(model, ham, x, c, torch.tensor(e.real, device="cuda"), torch.tensor(e.imag, device="cuda"),
               torch.tensor(st, device="cuda")).cpu().numpy().astype(np.float64)
    ref = _flat_grad(gradient(om, ip, xs, cs, e, st))
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < 1e-4, rel


def test_tf_grad_large_central_differences(A):
    """26 slots, d 128, 8 heads, 4 blocks: the library gradient of
    L = sum_l [c_l log|psi(x_l)| + c'_l arg psi(x_l)] against FP64 central
    differences of the oracle's L (step 1e-4) on 16 random parameters, and
    against the oracle's FP64 gradient."""
    w = workload("large", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"], params)
    om = TFAnsatz(w["params_struct"], w["n"], w["n_heads"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    x, _ = A.sample(model, ham, 4000, seed=2)
    xs = x.cpu().numpy().astype(np.uint64)[:64]
    rng = np.random.default_rng(4)
    ca, cp = rng.normal(size=len(xs)), rng.normal(size=len(xs))
    g = A.logpsi_vjp(model, ham, _dev(xs), torch.tensor(ca, device="cuda"),
                     torch.tensor(cp, device="cuda")).cpu().numpy().astype(np.float64)
    ps = om.parameters()
    for t in ps:
        t.requires_grad_(True)
    la, ph = log_psi(om, ip, xs)
    ref = _flat_grad(torch.autograd.grad((torch.tensor(ca) * la).sum() + (torch.tensor(cp) * ph).sum(), ps))
    for t in ps:
        t.requires_grad_(False)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-4
    sizes = [t.numel() for t in ps]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    hstep = 1e-4

    def loss():
        a, b = log_psi(om, ip, xs)
        return float((torch.tensor(ca) * a).sum() + (torch.tensor(cp) * b).sum())

    # L is piecewise smooth (ReLU in the FFN): a parameter is used only if L
    # is smooth over the stencil, i.e. the central differences with steps h
    # and h/2 agree to their FP64 rounding (~1e-16 |L| / h); a ReLU kink
    # within the stencil makes them differ by O(1e-4)
    checked, tried = 0, 0
    for i in rng.permutation(offs[-1]):
        if checked == 16:
            break
        tried += 1
        k = int(np.searchsorted(offs, i, side="right") - 1)
        flat = ps[k].view(-1)
        j = int(i - offs[k])
        old = float(flat[j])
        f = {}
        for k2 in (-1.0, -0.5, 0.5, 1.0):
            flat[j] = old + k2 * hstep
            f[k2] = loss()
        flat[j] = old
        fd_h = (f[1.0] - f[-1.0]) / (2 * hstep)
        fd_h2 = (f[0.5] - f[-0.5]) / hstep
        if abs(fd_h - fd_h2) > 1e-7 * max(1.0, abs(fd_h2)):
            continue
        checked += 1
        fd = (4 * fd_h2 - fd_h) / 3
        assert abs(g[i] - fd) <= 1e-4 * max(1.0, abs(fd)) + 1e-4 * np.linalg.norm(ref) / np.sqrt(len(ref)), \
            (i, g[i], fd, ref[i])
    assert checked == 16 and tried < 64, (checked, tried)


def test_tf_local_energy_fp32_large_shape(A):
    """26 slots, 9+9 electrons, 33,507 connected determinants per sample: the
    oracle cannot evaluate that many amplitudes per sample in the time bound,
    so E_loc is checked against its definition assembled in FP64 from the
    library's connected set (bit-exact against the oracle, see
    test_gpu_parity) and log psi (against the oracle at this shape above).
    The library forms each ratio psi(x')/psi(x) in float32 (exp and sincos of
    the float32 log differences) and sums in FP64, so the two agree to a few
    float32 ulps per term: |dE| <= 1e-6 sum_k |H_k r_k| (about 17 ulps); a
    wrong term would show as an error of order |H_k r_k|."""
    w = workload("large", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"],
                                torch.tensor(w["params"], device="cuda"))
    x, c = A.sample(model, ham, 2000, seed=5)
    x, c = x[:3], c[:3]
    ere, eim, stats = A.local_energy(model, ham, x, c)
    xp, hv, js, hd = A.connected(ham, x)
    assert xp.shape[1] == 33507
    lx, px = A.logpsi(model, ham, x)
    lp, pp = A.logpsi(model, ham, xp.reshape(-1))
    K = ham.n_connected
    r = torch.exp((lp.double().reshape(-1, K) - lx.double()[:, None])
                  + 1j * (pp.double().reshape(-1, K) - px.double()[:, None]))
    e = hd + (hv * r).sum(1)
    bound = 1e-6 * (hv.abs() * r.abs()).sum(1)
    assert ((e.real - ere).abs() <= bound).all()
    assert ((e.imag - eim).abs() <= bound).all()
    wts = c.double() / c.double().sum()
    assert abs(float((wts * ere).sum()) - float(stats[0])) <= 1e-12 * float(ere.abs().max())


@pytest.mark.parametrize("name,n_samples", [("n2", 20_000), ("large", 2000)])
def test_tf_grad_with_recomputation_equals_full_storage(A, name, n_samples):
    """The adjoint given only the smallest workspace (block inputs stored,
    each block's activations recomputed before its backward) against the one
    that stores every activation: the recomputed forward is bit-identical, so
    the gradients differ only by the summation order of the split-K weight
    products (float32 atomics)."""
    w = workload(name, bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"],
                                torch.tensor(w["params"], device="cuda"))
    x, c = A.sample(model, ham, n_samples, seed=13)
    if name == "large":
        x, c = x[:16].contiguous(), c[:16].contiguous()
    ere, eim, stats = A.local_energy(model, ham, x, c)
    full = A.grad_workspace_bytes(model, ham, x.numel())
    least = A.grad_workspace_bytes(model, ham, x.numel(), least=True)
    assert least < (full / 2 if name == "large" else full)  # 4 blocks of width 128: under half
    g_full = A.grad(model, ham, x, c, ere, eim, stats, workspace=A._ws(full, "cuda"))
    g_rec = A.grad(model, ham, x, c, ere, eim, stats, workspace=A._ws(least, "cuda"))
    torch.cuda.synchronize()
    assert torch.isfinite(g_rec).all()
    rel = float((g_rec - g_full).norm() / g_full.norm())
    assert rel < 1e-5, rel
    with pytest.raises(Exception):  # below the least size: capacity error before anything is queued
        A.grad(model, ham, x, c, ere, eim, stats, workspace=A._ws(least - 4096, "cuda"))
