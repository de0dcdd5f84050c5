"""Sharding of the VMC pass over ranks (Sec. II.C: subtrees of the sampling
tree are independent; Eq. energy_est and Eq. grad_def are sums over samples).

Pins: the union of the oracle's shards is the unsharded sample set with the
same counts (for every split level, including the root and the leaves);
combine_stats equals energy_stats of the concatenated samples (the
definition), including empty shards; and a world-size-2 gloo run of the
library's exchange (paper_2310_04166_gb300.dist) over oracle shards gives the
unsharded oracle energy and gradient.
"""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle.anqs import MLPAnsatz
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sampler import lexicographic_key, sample
from oracle.sector import molecular_isphys
from oracle.vmc import combine_stats, energy_stats, gradient, local_energy
from synthetic import workload


def _setup(name="small"):
    w = workload(name, bias_std=0.2)
    om = MLPAnsatz(w["params_struct"], w["n"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    return w, om, ip, oham


@pytest.mark.parametrize("world", [2, 3])
def test_union_of_shards_is_the_unsharded_sample(world):
    w, om, ip, _ = _setup()
    n = w["n"]
    x0, c0, _ = sample(om, ip, n, 5000, seed=3)
    for level in range(n + 1):
        xs, cs = [], []
        for r in range(world):
            x, c, _ = sample(om, ip, n, 5000, seed=3, shard=(r, world, level))
            xs.append(x)
            cs.append(c)
        x = np.concatenate(xs)
        c = np.concatenate(cs)
        order = np.argsort(lexicographic_key(x, n), kind="stable")
        assert np.array_equal(x[order], x0) and np.array_equal(c[order], c0)
        assert len(set(int(v) for v in x)) == len(x)  # disjoint
    # at the root a world > 1 leaves every rank but 0 empty
    x, c, _ = sample(om, ip, n, 5000, seed=3, shard=(1, world, 0))
    assert len(x) == 0


def test_combine_stats_equals_stats_of_the_union():
    rng = np.random.default_rng(5)
    e = rng.normal(-7, 0.3, 40) + 1j * rng.normal(0, 0.01, 40)
    n = rng.integers(1, 50, 40)
    ref = energy_stats(e, n)
    cuts = [0, 7, 7, 23, 40]  # includes an empty part
    parts = [energy_stats(e[a:b], n[a:b]) if b > a else np.array([np.nan, np.nan, np.nan, 0.0])
             for a, b in zip(cuts[:-1], cuts[1:])]
    got = combine_stats(parts)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-15)
    assert got[3] == n.sum()
    # a single part is returned unchanged
    assert np.allclose(combine_stats([ref]), ref, rtol=1e-15)


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2310_04166_gb300.dist import exchange_stats, reduce_grad
    w, om, ip, oham = _setup()
    x, c, _ = sample(om, ip, w["n"], 4000, seed=11, shard=(rank, world, 2))
    e = local_energy(om, ip, oham, x)
    st = torch.tensor(energy_stats(e, c) if len(x) else [np.nan, np.nan, np.nan, 0.0])
    allst = exchange_stats(st)
    glob = combine_stats(allst.numpy())
    g = gradient(om, ip, x, c, e, stats=glob)
    flat = torch.cat([t.reshape(-1) for t in g])
    reduce_grad(flat)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([glob, flat.numpy()]))
    torch.distributed.destroy_process_group()


def test_gloo_world2_sharded_step_equals_unsharded(tmp_path):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    w, om, ip, oham = _setup()
    x, c, _ = sample(om, ip, w["n"], 4000, seed=11)
    e = local_energy(om, ip, oham, x)
    st = energy_stats(e, c)
    g = torch.cat([t.reshape(-1) for t in gradient(om, ip, x, c, e, stats=st)]).numpy()
    for r in range(2):
        got = np.load(tmp_path / f"r{r}.npy")
        assert np.allclose(got[:4], st, rtol=1e-12, atol=1e-14)
        assert np.allclose(got[4:], g, rtol=1e-9, atol=1e-12)
