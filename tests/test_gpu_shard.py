"""Sharded VMC pass on the GPU (Sec. II.C: independent subtrees; Eq.
energy_est and Eq. grad_def as sums over the ranks' samples).

The ranks are run one after the other on one device (their kernels never
wait on one another).  Bars: the union of the shards is the unsharded sample
set, bit for bit, for every split level; the combined statistics equal the
unsharded ones to FP64 summation-order rounding; the summed gradient equals
the unsharded one to float32 summation-order rounding; the sharded sets also
match the oracle's own shards.  For the BF16 MLP on h2o the unsharded pass
takes the prefix-table path (every physical prefix evaluated in one launch)
and the shards the per-level path, so the first test also pins the two paths
to each other bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz
from oracle.sampler import lexicographic_key, sample as osample
from oracle.sector import molecular_isphys
from oracle.vmc import combine_stats
from synthetic import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    return mod


def _setup(A, name, form):
    w = workload(name, bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device="cuda")
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, form)
    return w, ham, model


def _merge(xs, cs, n):
    x = torch.cat(xs).cpu().numpy().astype(np.uint64)
    c = torch.cat(cs).cpu().numpy()
    o = np.argsort(lexicographic_key(x, n), kind="stable")
    return x[o], c[o]


@pytest.mark.parametrize("name,form,Ns", [("small", "fp32", 10_000), ("h2o", "fp32", 100_000),
                                          ("h2o", "bf16", 100_000)])
@pytest.mark.parametrize("world", [2, 3])
def test_union_of_gpu_shards_is_the_unsharded_sample(A, name, form, Ns, world):
    w, ham, model = _setup(A, name, form)
    x0, c0 = A.sample(model, ham, Ns, seed=21)
    x0 = x0.cpu().numpy().astype(np.uint64)
    for level in range(w["n"] + 1):
        xs, cs = zip(*[A.sample_shard(model, ham, Ns, 21, r, world, level) for r in range(world)])
        x, c = _merge(xs, cs, w["n"])
        assert np.array_equal(x, x0) and np.array_equal(c, c0.cpu().numpy()), level
        assert sum(len(v) for v in xs) == len(x0)


def test_gpu_shards_match_oracle_shards(A):
    w, ham, model = _setup(A, "small", "fp32")
    om = MLPAnsatz(w["params_struct"], w["n"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    for r in range(2):
        x, c = A.sample_shard(model, ham, 2000, 4, r, 2, 2)
        ox, oc, _, n_close = osample(om, ip, w["n"], 2000, seed=4, shard=(r, 2, 2), tol=1e-5)
        # FP32 conditionals: each draw within 1e-5 of a boundary may move one sample path
        got = dict(zip(x.cpu().numpy().astype(np.uint64).tolist(), c.cpu().numpy().tolist()))
        ref = dict(zip(ox.tolist(), oc.tolist()))
        l1 = sum(abs(got.get(k, 0) - ref.get(k, 0)) for k in set(got) | set(ref))
        assert l1 <= 2 * n_close


@pytest.mark.parametrize("name,form,Ns", [("h2o", "fp32", 100_000), ("h2o", "bf16", 100_000)])
def test_combined_stats_and_summed_gradient_equal_unsharded(A, name, form, Ns):
    """Each row's E_loc may round differently when the rows are batched
    differently (float32 ratios: |dE_l| <= 1e-6 sum_k |H_k psi(x'_k)/psi(x_l)|,
    the bound of the prefix-reuse test); the energy then moves by at most
    sum_l w_l |dE_l| plus the FP64 rounding of the sums, 1e-13 sum_l w_l |E_l|
    (the E_loc of rare samples of a random network can be large, so the
    weighted sums cancel)."""
    w, ham, model = _setup(A, name, form)
    world, level = 3, 2
    x0, c0 = A.sample(model, ham, Ns, seed=8)
    e0r, e0i, st0 = A.local_energy(model, ham, x0, c0)
    g0 = A.grad(model, ham, x0, c0, e0r, e0i, st0)
    parts, shards = [], []
    for r in range(world):
        x, c = A.sample_shard(model, ham, Ns, 8, r, world, level)
        er, ei, st = A.local_energy(model, ham, x, c)
        parts.append(st)
        shards.append((x, c, er, ei))
    allst = torch.stack(parts)
    glob = A.stats_combine(allst)
    ref = combine_stats(allst.cpu().numpy())
    assert torch.allclose(glob.cpu(), torch.tensor(ref), rtol=1e-14, atol=1e-15)
    # per-row bound
    xp, hv, _, _ = A.connected(ham, x0)
    lx, px = A.logpsi(model, ham, x0)
    lp, _ = A.logpsi(model, ham, xp.reshape(-1))
    K = ham.n_connected
    hr = (hv.abs() * torch.exp(lp.double().reshape(-1, K) - lx.double()[:, None])).sum(1).cpu().numpy()
    key = {v: i for i, v in enumerate(x0.cpu().tolist())}
    e0 = (e0r + 1j * e0i).cpu().numpy()
    de = np.zeros(len(e0))
    for x, c, er, ei in shards:
        idx = np.array([key[v] for v in x.cpu().tolist()], dtype=np.int64)
        de[idx] = np.abs((er + 1j * ei).cpu().numpy() - e0[idx])
    assert np.all(de <= 1e-6 * hr), (de / hr).max()
    wts = c0.cpu().numpy() / Ns
    s0 = st0.cpu().numpy()
    assert glob[3].item() == s0[3] == Ns
    tol = (wts * de).sum() + 1e-13 * (wts * np.abs(e0)).sum()
    assert abs(glob[0].item() - s0[0]) <= tol
    assert abs(glob[1].item() - s0[1]) <= tol
    g = torch.zeros_like(g0)
    for x, c, er, ei in shards:
        g += A.grad(model, ham, x, c, er, ei, glob)
    rel = ((g - g0).norm() / g0.norm()).item()
    assert rel < 1e-5, rel


def test_empty_shard_contributes_nothing(A):
    """Split at the root: only rank 0 gets samples; rank 1's statistics have
    S = 0 and are skipped by the combination."""
    w, ham, model = _setup(A, "small", "fp32")
    x0, c0 = A.sample(model, ham, 5000, seed=2)
    _, _, st0 = A.local_energy(model, ham, x0, c0)
    x1, c1 = A.sample_shard(model, ham, 5000, 2, 1, 2, 0)
    assert len(x1) == 0
    from paper_2310_04166_gb300.dist import ShardedStep  # noqa: F401  (module imports)
    empty = torch.tensor([float("nan"), float("nan"), float("nan"), 0.0], dtype=torch.float64, device="cuda")
    glob = A.stats_combine(torch.stack([st0, empty]))
    assert torch.equal(glob, A.stats_combine(st0.reshape(1, 4)))
    assert torch.allclose(glob, st0, rtol=1e-15, atol=0)


def test_sharded_step_single_rank_equals_plain_pass(A):
    """ShardedStep with one rank (no process group): device-count path end to
    end (sample_shard_into, local_energy and grad on n_dev rows)."""
    from paper_2310_04166_gb300.dist import ShardedStep
    w, ham, model = _setup(A, "h2o", "bf16")
    step = ShardedStep(model, ham, 100_000, seed=6)
    st, g = step()
    x0, c0 = A.sample(model, ham, 100_000, seed=6)
    e0r, e0i, st0 = A.local_energy(model, ham, x0, c0)
    g0 = A.grad(model, ham, x0, c0, e0r, e0i, st0)
    assert torch.allclose(st, st0, rtol=1e-13, atol=1e-15)
    assert ((g - g0).norm() / g0.norm()).item() < 1e-6
