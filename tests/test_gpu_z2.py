"""GPU parity with Z2 symmetries set (Algorithm 1 with the multiplicative
Z2 composition, Sec. IV.A) on Hamiltonians with a planted point group.

Bars: the slot masks of the device table equal the oracle's IsPhys masks for
every prefix of every sector determinant; the sector dimension equals the
oracle's count; the sampler with injected conditionals is bit-exact with the
oracle's and never leaves the Z2 sector; log psi is -inf outside it; FP32
local energies match the oracle, and the BF16 form's prefix reuse equals its
full evaluation.
"""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz, TableAnsatz, allowed_masks, log_psi, table_from_state
from oracle.ed import ground_state
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import sample as osample
from oracle.sector import count_leaves, molecular_isphys, sector_states, z2_string
from oracle.vmc import energy_stats, local_energy
from synthetic import flatten_mlp, integrals_z2, mlp_params, z2_qubit_masks

pytestmark = pytest.mark.gpu
CASES = [(5, 2, 2, [0, 1, 0, 1, 1]), (7, 3, 3, [0, 1, 1, 0, 1, 0, 1]), (6, 2, 2, [0, 1, 2, 3, 1, 2])]


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


def _setup(A, n, na, nb, labels):
    masks = z2_qubit_masks(labels)
    h, g, e = integrals_z2(n, n, 2 * n, labels)
    ham = A.Hamiltonian(h, g, e, na, nb).set_z2(masks)
    ip = molecular_isphys(n, na, nb, extra=[z2_string([q + 1 for q in range(2 * n) if (m >> q) & 1]) for m in masks])
    ref = sum(1 << (2 * p) for p in range(na)) | sum(1 << (2 * p + 1) for p in range(nb))
    par = lambda x, m: bin(int(x) & m).count("1") & 1
    st = np.array([x for x in sector_states(n, na, nb) if all(par(x, m) == par(ref, m) for m in masks)],
                  dtype=np.uint64)
    return ham, ip, st, OHam(h, g, e, na, nb), masks


@pytest.mark.parametrize("n,na,nb,labels", CASES)
def test_z2_masks_and_sector_dim(A, n, na, nb, labels):
    ham, ip, st, _, masks = _setup(A, n, na, nb, labels)
    assert ham.sector_dim == count_leaves(ip) == len(st)
    table = ham.slot_masks()
    om = allowed_masks(ip, st, n)
    for i, x in enumerate(st):
        for p in range(n):
            pre = int(x) & ((1 << (2 * p)) - 1)
            a = bin(pre & 0x5555555555555555).count("1")
            b = bin(pre & 0xAAAAAAAAAAAAAAAA).count("1")
            z = sum((bin(pre & m).count("1") & 1) << j for j, m in enumerate(masks))
            bits = sum(1 << v for v in range(4) if om[i, p, v])
            assert table[p, a, b, z] == bits


@pytest.mark.parametrize("n,na,nb,labels", CASES)
def test_z2_sampler_bit_exact_and_eloc(A, n, na, nb, labels):
    ham, ip, st, oham, _ = _setup(A, n, na, nb, labels)
    E0, c = ground_state(oham, [int(x) for x in st])
    tables = [np.maximum(t, -60.0).astype(np.float32).astype(np.float64) for t in table_from_state(st, c, n)]
    model = A.Model.table(n, torch.tensor(np.concatenate([t.ravel() for t in tables]).astype(np.float32),
                                          device="cuda"))
    om = TableAnsatz(tables, n)
    for Ns in (1, 1000, 100_003):
        x, cnt = A.sample(model, ham, Ns, seed=4)
        ox, oc, _ = osample(om, ip, n, Ns, seed=4)
        assert np.array_equal(x.cpu().numpy().astype(np.uint64), ox)
        assert np.array_equal(cnt.cpu().numpy(), oc)
        assert np.all(np.isin(ox, st))
    ere, _, _ = A.local_energy(model, ham, _dev(st))
    big = np.abs(c) > 1e-3
    assert np.abs(ere.cpu().numpy()[big] - E0).max() < 1e-3
    out = np.array([x for x in sector_states(n, na, nb) if x not in set(int(v) for v in st)][:20], dtype=np.uint64)
    assert torch.isneginf(A.logpsi(model, ham, _dev(out))[0]).all()


@pytest.mark.parametrize("n,na,nb,labels", CASES[:2])
def test_z2_mlp_fp32_and_bf16(A, n, na, nb, labels):
    ham, ip, st, oham, _ = _setup(A, n, na, nb, labels)
    P = mlp_params(n, n, 64, 2, bias_std=0.3)
    params = torch.tensor(flatten_mlp(P), device="cuda")
    om = MLPAnsatz(P, n)
    m32 = A.Model.mlp(n, 64, 2, params, "fp32")
    la, ph = A.logpsi(m32, ham, _dev(st))
    rla, rph = log_psi(om, ip, st)
    assert np.abs(la.cpu().numpy() - rla.numpy()).max() < 2e-5
    assert abs(np.exp(2 * la.double().cpu().numpy()).sum() - 1) < 1e-5
    ox, on, _ = osample(om, ip, n, 50_000, seed=2)
    ere, eim, st32 = A.local_energy(m32, ham, _dev(ox), _dev(on))
    e_ref = local_energy(om, ip, oham, ox)
    assert np.abs(ere.cpu().numpy() - e_ref.real).max() < 1e-4
    assert abs(st32.cpu().numpy()[0] - energy_stats(e_ref, on)[0]) < 1e-5
    m16 = A.Model.mlp(n, 64, 2, params, "bf16")
    x, cnt = A.sample(m16, ham, 50_000, seed=3)
    assert np.all(np.isin(x.cpu().numpy().astype(np.uint64), st))
    ere, eim, _ = A.local_energy(m16, ham, x, cnt)
    xp, hv, js, hd = A.connected(ham, x)
    lx, px = A.logpsi(m16, ham, x)
    lp, pp = A.logpsi(m16, ham, xp.reshape(-1))
    K = ham.n_connected
    r = torch.exp((lp.double().reshape(-1, K) - lx.double()[:, None])
                  + 1j * (pp.double().reshape(-1, K) - px.double()[:, None]))
    e_full = hd + (hv * r).sum(1)
    bound = 1e-6 * (hv.abs() * r.abs()).sum(1) + 1e-12
    assert ((e_full.real - ere).abs() <= bound).all()
