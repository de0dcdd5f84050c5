"""GPU parity of the per-qubit complex NADE (Appendix B.1, FP32 form)
against the FP64 oracle.

Tolerance.  Each qubit's outputs come from dot products of at most w + 2n
float32 terms whose magnitudes sum to O(sqrt(w)) (weights of std
1/sqrt(2 fan-in), |tanh| and the LeReLU outputs O(1)), so the standard
bound m u sum|a_k b_k| (u = 2^-24) gives a per-qubit error of at most about
w^1.5 u; with a factor 2 for tanh, exp, log and the renormalisation the
per-qubit bound is TOL_Q = 2 w^1.5 u and log psi, a sum of 2n qubit terms,
moves by at most 2n TOL_Q.  A local energy moves by at most
sum_k |H_k psi(x'_k)/psi(x)| (e^{2 tol} - 1).  The bound needs tanh z1 to be
well conditioned; next to its poles (z1 = i pi (k + 1/2)) the kernel keeps
that accuracy by carrying z1 as a float-float pair (the (7, 5, 5, 64) case
has a unit with |cosh z1| ~ 1e-2).
"""
import numpy as np
import pytest
import torch

from oracle.anqs import NADEAnsatz, log_psi
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import sample as osample
from oracle.sector import molecular_isphys, sector_states
from oracle.vmc import energy_stats, local_energy
from synthetic import flatten_nade, integrals, nade_param_count, nade_params

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _tol(n, w):
    return 2 * n * 2 * w ** 1.5 * U


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


def _setup(A, n, na, nb, w, seed, du=0, bias_std=0.3):
    q = nade_params(seed, n, w, bias_std=bias_std)
    params = torch.tensor(flatten_nade(q), device="cuda")
    assert params.numel() == nade_param_count(n, w)
    h, g, e = integrals(seed, n, n)
    ham = A.Hamiltonian(h, g, e, na, nb)
    if du:
        ham.set_pruning(du)
    model = A.Model.nade(n, w, params)
    ip = molecular_isphys(n, na, nb)
    om = NADEAnsatz(q, n, ip, du_levels=du)
    oham = OHam(h, g, e, na, nb)
    return ham, model, om, ip, oham


def _wrap(d):
    return (d + np.pi) % (2 * np.pi) - np.pi


@pytest.mark.parametrize("n,na,nb,w", [(4, 2, 2, 32), (6, 3, 2, 64), (5, 2, 3, 128), (7, 5, 5, 64)])
def test_nade_logpsi_against_oracle(A, n, na, nb, w):
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=n + w)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    tol = _tol(n, w)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < tol
    assert np.abs(_wrap(ph.cpu().numpy() - rph.numpy())).max() < tol
    # qubit-level MU masking keeps the ansatz normalised on the sector
    assert abs(np.exp(2 * la.double().cpu().numpy()).sum() - 1.0) < 1e-5
    # a flipped alpha or beta bit leaves the sector: zero amplitude
    bad = [int(st[0]) ^ 1, int(st[0]) ^ 2]
    assert torch.isneginf(A.logpsi(model, ham, _dev(bad))[0]).all()


@pytest.mark.parametrize("d", [1, 3, 6])
def test_nade_pruning_logpsi_against_oracle(A, d):
    n, na, nb, w = 6, 3, 3, 64
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=7, du=d)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st, du_levels=d)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < _tol(n, w)
    assert np.abs(_wrap(ph.cpu().numpy() - rph.numpy())).max() < _tol(n, w)


def test_nade_local_energy_against_oracle(A):
    n, na, nb, w = 7, 5, 5, 64
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=11)
    ox, on, _ = osample(om, ip, n, 20_000, seed=9)
    keep = np.argsort(-on, kind="stable")[:64]
    ox, on = ox[keep], on[keep]
    ere, eim, stats = A.local_energy(model, ham, _dev(ox), _dev(on))
    e_ref = local_energy(om, ip, oham, ox)
    tol = _tol(n, w)
    la, _ = log_psi(om, ip, ox)
    lists = [oham.connected(int(v)) for v in ox]
    K = len(lists[0])
    xs = np.array([t[0] for L in lists for t in L], dtype=np.uint64)
    hv = np.array([t[1] for L in lists for t in L]).reshape(-1, K)
    lp, _ = log_psi(om, ip, xs)
    r = np.exp(lp.numpy().reshape(-1, K) - la.numpy()[:, None])
    bound = (np.abs(hv) * r).sum(1) * (np.exp(2 * tol) - 1) + 1e-12
    err = np.abs((ere.cpu().numpy() - e_ref.real) + 1j * (eim.cpu().numpy() - e_ref.imag))
    assert np.all(err <= bound), (err / bound).max()
    s_ref = energy_stats(e_ref, on)
    wts = on / on.sum()
    assert abs(stats.cpu().numpy()[0] - s_ref[0]) <= (wts * err).sum() + 1e-12


@pytest.mark.parametrize("n,na,nb,w,d", [(7, 5, 5, 32, 0), (6, 3, 3, 128, 0), (6, 2, 3, 64, 3)])
def test_nade_prefix_reuse_equals_full_evaluation(A, n, na, nb, w, d):
    """The local energy reuses the parent's slots <= j for each connected x'
    (j its first differing slot); assembled instead from full log psi
    evaluations of x and x' it agrees up to the float32 rounding of the
    ratios: |dE| <= 2e-5 sum_k |H_k r_k| (log psi sums of 2n terms of
    magnitude <~ 20 rounded in a different order)."""
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=30 + n, du=d)
    x, c = A.sample(model, ham, 200_000, seed=5)
    ere, eim, _ = A.local_energy(model, ham, x, c)
    xp, hv, js, hd = A.connected(ham, x)
    lx, px = A.logpsi(model, ham, x)
    lp, pp = A.logpsi(model, ham, xp.reshape(-1))
    K = ham.n_connected
    r = torch.exp((lp.double().reshape(-1, K) - lx.double()[:, None])
                  + 1j * (pp.double().reshape(-1, K) - px.double()[:, None]))
    e_full = hd + (hv * r).sum(1)
    bound = 2e-5 * (hv.abs() * r.abs()).sum(1) + 1e-12
    assert ((e_full.real - ere).abs() <= bound).all()
    assert ((e_full.imag - eim).abs() <= bound).all()


@pytest.mark.parametrize("d", [0, 2])
def test_nade_sampler_against_oracle(A, d):
    """Only draws within the conditionals' float32 error of a split boundary
    may go another way; each moves one sample path, so the L1 distance of
    the count vectors is at most twice their number."""
    n, na, nb, w = 7, 5, 5, 64
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=13, du=d)
    Ns = 100_000
    x, c = A.sample(model, ham, Ns, seed=3, counter=1)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    ox, on, margin, n_close = osample(om, ip, n, Ns, seed=3, counter=1, tol=1e-4, du_levels=d)
    allx = np.union1d(ox, x)
    a = np.zeros(len(allx), np.int64)
    b = np.zeros(len(allx), np.int64)
    a[np.searchsorted(allx, ox)] = on
    b[np.searchsorted(allx, x)] = c
    assert np.abs(a - b).sum() <= 2 * n_close
    if d == 0:
        assert c.sum() == Ns


def _flat_grad(grads, n):
    """Oracle gradients (per qubit: W1, b1, W2, b2, W3, b3, each as re, im
    tensors) in the flat layout (re, im interleaved per entry)."""
    out = []
    for i in range(2 * n):
        for a in range(6):
            gr, gi = grads[i * 12 + 2 * a], grads[i * 12 + 2 * a + 1]
            out.append(np.stack([gr.numpy(), gi.numpy()], axis=-1).reshape(-1))
    return np.concatenate(out)


@pytest.mark.parametrize("n,na,nb,w,d", [(4, 2, 2, 32, 0), (7, 5, 5, 64, 0), (6, 3, 3, 128, 2)])
def test_nade_gradient_against_oracle(A, n, na, nb, w, d):
    """VMC gradient (Eq. grad_def) through the adjoint.  Bar: relative
    2-norm error 1e-4 (float32 accumulation over w units and the rows of the
    sample, with the cancellation between rows of a covariance)."""
    from oracle.vmc import gradient
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=20 + n, du=d)
    ox, on, _ = osample(om, ip, n, 50_000, seed=4, du_levels=d)
    e_ref = local_energy(om, ip, oham, ox, du_levels=d)
    s_ref = energy_stats(e_ref, on)
    g_ref = _flat_grad(gradient(om, ip, ox, on, e_ref, s_ref, du_levels=d), n)
    ere = torch.tensor(e_ref.real, device="cuda")
    eim = torch.tensor(e_ref.imag, device="cuda")
    stats = torch.tensor(s_ref, device="cuda")
    for _ in range(2):  # the partial-sum path is deterministic: two calls agree bit for bit
        g = A.grad(model, ham, _dev(ox), _dev(on), ere, eim, stats)
        if _ == 0:
            g0 = g.clone()
    assert torch.equal(g, g0)
    g = g.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel < 1e-4, rel


def test_nade_autograd_function_uses_library_adjoint(A):
    n, na, nb, w = 5, 2, 3, 64
    q = nade_params(5, n, w, bias_std=0.3)
    params = torch.tensor(flatten_nade(q), device="cuda", requires_grad=True)
    h, g, e = integrals(5, n, n)
    ham = A.Hamiltonian(h, g, e, na, nb)
    model = A.Model.nade(n, w, params.detach())
    ip = molecular_isphys(n, na, nb)
    om = NADEAnsatz(q, n, ip)
    ps = om.parameters()
    for t in ps:
        t.requires_grad_(True)
    full = np.array(sector_states(n, na, nb), dtype=np.uint64)
    # all 100 sector states (25 row tiles: partial sums), and 3 rows (one tile: direct writes)
    for st in (full, full[[0, 41, 99]]):
        params.grad = None
        la, ph = A.LogPsi.apply(params, model, ham, _dev(st))
        (la.sum() + 0.5 * ph.sum()).backward()
        ra, rp = log_psi(om, ip, st)
        gs = torch.autograd.grad(ra.sum() + 0.5 * rp.sum(), ps, allow_unused=True)
        ref = _flat_grad([gg if gg is not None else torch.zeros_like(t) for gg, t in zip(gs, ps)], n)
        got = params.grad.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4


def test_nade_has_no_bf16_form(A):
    n, w = 4, 32
    with pytest.raises(A.AnqsError, match="UNSUPPORTED"):
        A.Model(A.ModelDesc(3, 1, n, w, 0, 0, 0, 0), torch.zeros(nade_param_count(n, w), device="cuda"))


@pytest.mark.parametrize("na,nb", [(1, 0), (1, 1), (0, 1)])
def test_nade_single_orbital(A, na, nb):
    """n = 1: one slot (two qubits), no slot past any first differing slot,
    a one- or two-determinant sector."""
    n, w = 1, 32
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=50)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < _tol(n, w)
    x, c = A.sample(model, ham, 1000, seed=1)
    assert x.cpu().numpy().astype(np.uint64).tolist() == st.tolist() and int(c.sum()) == 1000
    ere, eim, stats = A.local_energy(model, ham, x, c)
    e_ref = local_energy(om, ip, oham, st)
    assert np.allclose(ere.cpu().numpy(), e_ref.real, atol=1e-5) and np.allclose(eim.cpu().numpy(), e_ref.imag, atol=1e-5)
    g = A.grad(model, ham, x, c, ere, eim, stats)
    assert torch.isfinite(g).all()


def test_nade_32_orbitals(A):
    """n = 32 (64 qubits, bit 63 in use), one electron of each spin: log psi
    over the whole 1024-determinant sector, local energies and the gradient
    of three samples against the oracle."""
    from oracle.vmc import gradient
    n, na, nb, w = 32, 1, 1, 32
    ham, model, om, ip, oham = _setup(A, n, na, nb, w, seed=72)
    st = np.array(sorted((1 << (2 * i)) | (1 << (2 * j + 1)) for i in range(n) for j in range(n)), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    tol = _tol(n, w)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < tol
    assert np.abs(_wrap(ph.cpu().numpy() - rph.numpy())).max() < tol
    assert abs(np.exp(2 * la.double().cpu().numpy()).sum() - 1.0) < 1e-4
    xs = st[[0, 517, 1023]]
    on = np.array([3, 2, 1])
    ere, eim, stats = A.local_energy(model, ham, _dev(xs), _dev(on))
    e_ref = local_energy(om, ip, oham, xs)
    lists = [oham.connected(int(v)) for v in xs]
    K = len(lists[0])
    xp = np.array([t[0] for L in lists for t in L], dtype=np.uint64)
    hv = np.array([t[1] for L in lists for t in L]).reshape(-1, K)
    lp, _ = log_psi(om, ip, xp)
    r = np.exp(lp.numpy().reshape(-1, K) - rla.numpy()[np.searchsorted(st, xs)][:, None])
    bound = (np.abs(hv) * r).sum(1) * (np.exp(2 * tol) - 1) + 1e-12
    err = np.abs((ere.cpu().numpy() - e_ref.real) + 1j * (eim.cpu().numpy() - e_ref.imag))
    assert np.all(err <= bound), (err / bound).max()
    s_ref = energy_stats(e_ref, on)
    g_ref = _flat_grad(gradient(om, ip, xs, on, e_ref, s_ref), n)
    g = A.grad(model, ham, _dev(xs), _dev(on), torch.tensor(e_ref.real, device="cuda"),
               torch.tensor(e_ref.imag, device="cuda"), torch.tensor(s_ref, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-4
