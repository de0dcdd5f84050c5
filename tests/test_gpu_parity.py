"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: integer work (connected determinants, first slots, sampled sets with
the tabular ansatz) bit-exact; FP64 matrix elements to 1e-12; FP32-form
amplitudes, local energies and gradients within tolerances derived from
float32 rounding of log psi (relative 2^-24 of |log psi| <~ 20, i.e. ~1e-6
absolute, stated per test).
"""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz, TableAnsatz, log_psi, table_from_state
from oracle.ed import ground_state
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import sample as osample
from oracle.sector import molecular_isphys, sector_states
from oracle.vmc import energy_stats, gradient, local_energy
from synthetic import integrals, mlp_params, flatten_mlp, workload

pytestmark = pytest.mark.gpu

A = None


@pytest.fixture(scope="module", autouse=True)
def lib():
    global A
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    A = mod
    return mod


def _dev(a, dtype=torch.int64):
    return torch.as_tensor(np.asarray(a).astype(np.int64) if dtype == torch.int64 else a, dtype=dtype,
                           device="cuda")


def _problem(name, bias_std=0.2):
    w = workload(name, bias_std=bias_std)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    return w, ham, oham, ip


# ---------------------------------------------------------------------------
# sector table
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (7, 5, 5), (10, 7, 7), (6, 1, 4), (26, 9, 9)])
def test_slot_masks_match_oracle_isphys(n, na, nb):
    h, g, _ = integrals(0, n, 1)
    ham = A.Hamiltonian(h, g, 0.0, na, nb)
    M = ham.slot_masks()
    ip = molecular_isphys(n, na, nb)
    from oracle.sector import eigenvalues
    for p in range(n):
        for a in range(na + 1):
            for b in range(nb + 1):
                if a > p or b > p:
                    continue
                pre = [1] * a + [0] * (p - a)
                preb = [1] * b + [0] * (p - b)
                bits = [v for pair in zip(pre, preb) for v in pair]
                if not ip.of_prefix(bits):
                    assert M[p, a, b] == 0
                    continue
                exp = 0
                for v in range(4):
                    if ip.of_prefix(bits + [v & 1, v >> 1]):
                        exp |= 1 << v
                assert M[p, a, b] == exp, (p, a, b)


# ---------------------------------------------------------------------------
# connected set
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,n_check", [("small", 36), ("h2o", 441), ("n2", 40), ("large", 2)])
def test_connected_bit_exact(name, n_check):
    w, ham, oham, ip = _problem(name)
    rng = np.random.default_rng(5)
    n = w["n"]
    if name in ("small", "h2o"):
        xs = np.array(sector_states(n, w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    else:
        xs = []
        for _ in range(n_check):
            a = rng.choice(n, w["n_alpha"], replace=False)
            b = rng.choice(n, w["n_beta"], replace=False)
            xs.append(sum(1 << (2 * int(i)) for i in a) | sum(1 << (2 * int(i) + 1) for i in b))
        xs = np.array(xs, dtype=np.uint64)
    xp, hv, js, hd = A.connected(ham, _dev(xs))
    xp, hv, js, hd = (t.cpu().numpy() for t in (xp, hv, js, hd))
    assert ham.n_connected == oham.n_connected()
    for l, x in enumerate(xs):
        ref = oham.connected(int(x))
        assert [int(v) for v in xp[l].astype(np.uint64)] == [r[0] for r in ref]
        assert js[l].tolist() == [r[2] for r in ref]
        assert np.abs(hv[l] - np.array([r[1] for r in ref])).max() < 1e-12
        assert abs(hd[l] - oham.diagonal(int(x))) < 1e-12


def test_connected_out_of_sector_and_empty():
    w, ham, oham, ip = _problem("small")
    xs = np.array([0b0111, 0b00001111 | (1 << 8)], dtype=np.uint64)  # wrong counts / bits beyond 2n
    xp, hv, js, hd = A.connected(ham, _dev(xs))
    assert torch.isnan(hv).all() and (js == 255).all() and torch.isnan(hd).all()
    e = A.connected(ham, torch.zeros(0, dtype=torch.int64, device="cuda"))
    assert e[0].numel() == 0


# ---------------------------------------------------------------------------
# amplitudes (FP32 form)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["small", "h2o"])
def test_logpsi_fp32(name):
    w, ham, oham, ip = _problem(name)
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, "fp32")
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    la, ph = A.logpsi(model, ham, _dev(st))
    ref_la, ref_ph = log_psi(MLPAnsatz(w["params_struct"], w["n"]), ip, st)
    assert np.abs(la.cpu().numpy() - ref_la.numpy()).max() < 2e-5
    assert np.abs(ph.cpu().numpy() - ref_ph.numpy()).max() < 2e-5
    # outside the sector: amplitude exactly zero
    bad = np.array([0, int(st[0]) ^ 1, int(st[0]) | (1 << (2 * w["n"]))], dtype=np.uint64)
    la_bad, _ = A.logpsi(model, ham, _dev(bad))
    assert torch.isneginf(la_bad).all()


# ---------------------------------------------------------------------------
# sampler
# ---------------------------------------------------------------------------
def _table_model(n, na, nb, seed):
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    c = np.random.default_rng(seed).normal(size=len(st))
    c /= np.linalg.norm(c)
    tables = table_from_state(st, c, n)
    tables = [np.maximum(t, -60.0).astype(np.float32).astype(np.float64) for t in tables]
    flat = np.concatenate([t.reshape(-1) for t in tables]).astype(np.float32)
    return tables, flat


@pytest.mark.parametrize("n,na,nb,Ns,seed", [(4, 2, 2, 10_000, 1), (6, 3, 2, 100_000, 2), (7, 5, 5, 123_457, 3),
                                             (5, 1, 4, 1, 4)])
def test_sampler_bit_exact_with_injected_conditionals(n, na, nb, Ns, seed):
    tables, flat = _table_model(n, na, nb, seed)
    h, g, _ = integrals(0, n, 1)
    ham = A.Hamiltonian(h, g, 0.0, na, nb)
    model = A.Model.table(n, torch.tensor(flat, device="cuda"))
    ip = molecular_isphys(n, na, nb)
    tab = TableAnsatz(tables, n)
    ox, on, margin = osample(tab, ip, n, Ns, seed=seed, counter=7)
    assert margin > 1e-12  # no draw sits on a boundary within FP64 rounding
    x, c = A.sample(model, ham, Ns, seed=seed, counter=7)
    assert np.array_equal(x.cpu().numpy().astype(np.uint64), ox)
    assert np.array_equal(c.cpu().numpy(), on)


@pytest.mark.parametrize("name,Ns", [("small", 10_000), ("h2o", 100_000)])
def test_sampler_mlp_fp32(name, Ns):
    """With the live FP32 network only draws within the conditional's FP32
    error of a boundary may go another way; each such draw moves at most one
    sample path, so the L1 distance of the count vectors is at most twice
    the number of such draws."""
    w, ham, oham, ip = _problem(name)
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, "fp32")
    x, c = A.sample(model, ham, Ns, seed=3, counter=1)
    x, c = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    om = MLPAnsatz(w["params_struct"], w["n"])
    ox, on, margin, n_close = osample(om, ip, w["n"], Ns, seed=3, counter=1, tol=1e-5)
    assert c.sum() == Ns
    allx = np.union1d(ox, x)
    a = np.zeros(len(allx), np.int64)
    b = np.zeros(len(allx), np.int64)
    a[np.searchsorted(allx, ox)] = on
    b[np.searchsorted(allx, x)] = c
    assert np.abs(a - b).sum() <= 2 * n_close
    from oracle.sampler import lexicographic_key
    assert np.all(np.diff(lexicographic_key(x, w["n"]).astype(np.float64)) > 0)


def test_sampler_capacity_errors():
    w, ham, oham, ip = _problem("small")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"))
    xo = torch.empty(10, dtype=torch.int64, device="cuda")
    no = torch.empty(10, dtype=torch.int64, device="cuda")
    nu = torch.empty(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AnqsError, match="CAPACITY"):
        A.sample_into(model, ham, 1000, 1, 0, xo, no, nu, ws)  # cap 10 < min(1000, 36)
    with pytest.raises(A.AnqsError, match="ARG"):
        A.sample_into(model, ham, 0, 1, 0, xo, no, nu, ws)


# ---------------------------------------------------------------------------
# local energy and statistics
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,Ns", [("small", 10_000), ("h2o", 100_000)])
def test_local_energy_fp32(name, Ns):
    w, ham, oham, ip = _problem(name)
    om = MLPAnsatz(w["params_struct"], w["n"])
    ox, on, _ = osample(om, ip, w["n"], Ns, seed=9)
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, "fp32")
    ere, eim, stats = A.local_energy(model, ham, _dev(ox), _dev(on))
    e_ref = local_energy(om, ip, oham, ox)
    s_ref = energy_stats(e_ref, on)
    d_re = np.abs(ere.cpu().numpy() - e_ref.real).max()
    d_im = np.abs(eim.cpu().numpy() - e_ref.imag).max()
    st = stats.cpu().numpy()
    assert d_re < 1e-4 and d_im < 1e-4, (d_re, d_im)
    assert abs(st[0] - s_ref[0]) < 1e-5 and abs(st[1] - s_ref[1]) < 1e-5
    assert abs(st[2] - s_ref[2]) < 1e-4 * max(1.0, s_ref[2]) and st[3] == s_ref[3] == Ns


def test_local_energy_is_ground_energy_for_exact_eigenvector():
    """Tabular ansatz of the exact ground vector: E_loc(x) = E_0 on the GPU."""
    n, na, nb = 5, 3, 2
    h, g, _ = integrals(11, n, 10)
    oham = OHam(h, g, 0.3, na, nb)
    st = sector_states(n, na, nb)
    E0, c = ground_state(oham, st)
    tables = table_from_state(np.array(st, dtype=np.uint64), c, n)
    flat = np.concatenate([np.maximum(t, -80.0).reshape(-1) for t in tables]).astype(np.float32)
    ham = A.Hamiltonian(h, g, 0.3, na, nb)
    model = A.Model.table(n, torch.tensor(flat, device="cuda"))
    ere, eim, _ = A.local_energy(model, ham, _dev(st))
    big = np.abs(c) > 1e-3  # FP32 log-amplitude ratios: relative error ~1e-6 / |c|
    assert np.abs(ere.cpu().numpy()[big] - E0).max() < 1e-3
    assert np.median(np.abs(ere.cpu().numpy() - E0)) < 1e-4


# ---------------------------------------------------------------------------
# gradient (FP32 form)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,Ns", [("small", 10_000), ("h2o", 100_000)])
def test_gradient_fp32(name, Ns):
    w, ham, oham, ip = _problem(name)
    om = MLPAnsatz(w["params_struct"], w["n"])
    ox, on, _ = osample(om, ip, w["n"], Ns, seed=4)
    e_ref = local_energy(om, ip, oham, ox)
    s_ref = energy_stats(e_ref, on)
    g_ref = gradient(om, ip, ox, on, e_ref, s_ref)
    g_ref_flat = np.concatenate([t.reshape(-1).numpy() for t in g_ref])
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, "fp32")
    ere = torch.tensor(e_ref.real, device="cuda")
    eim = torch.tensor(e_ref.imag, device="cuda")
    stats = torch.tensor(s_ref, device="cuda")
    g = A.grad(model, ham, _dev(ox), _dev(on), ere, eim, stats).cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_ref_flat) / np.linalg.norm(g_ref_flat)
    assert rel < 1e-4, rel


def test_autograd_function_uses_library_adjoint():
    w, ham, oham, ip = _problem("small")
    params = torch.tensor(w["params"], device="cuda", requires_grad=True)
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params.detach(), "fp32")
    st = np.array(sector_states(w["n"], 2, 2), dtype=np.uint64)
    la, ph = A.LogPsi.apply(params, model, ham, _dev(st))
    (la.sum() + 0.5 * ph.sum()).backward()
    om = MLPAnsatz(w["params_struct"], w["n"])
    ps = om.parameters()
    for t in ps:
        t.requires_grad_(True)
    ra, rp = log_psi(om, ip, st)
    gs = torch.autograd.grad(ra.sum() + 0.5 * rp.sum(), ps, allow_unused=True)
    ref = np.concatenate([(g if g is not None else torch.zeros_like(t)).reshape(-1).numpy()
                          for g, t in zip(gs, ps)])
    got = params.grad.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
