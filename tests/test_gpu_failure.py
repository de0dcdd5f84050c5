"""Failure detection on the GPU without a fault.

The persistent sampler (prefix-table mode: 16-bit MLP, small sector) runs all
levels in one cooperative launch with a grid-wide barrier per level, each
bounded in time.  The test hook makes every barrier wait for one CTA more
than the grid has, an arrival that never comes, with a 20 ms limit: every
CTA gives up and leaves, the model's status word records it, the pass
returns no samples, and the context stays usable (a model that did not fail
then samples the same set as before, bit for bit)."""
import pytest
import torch

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


def _model(A, w, ham):
    return A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"), "bf16")


def test_sampler_barrier_time_out_is_reported_and_recoverable(A):
    from paper_2310_04166_gb300 import _lib
    lib = _lib.load()
    w = workload("h2o", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    good = _model(A, w, ham)
    x0, c0 = A.sample(good, ham, 20_000, seed=3)
    assert good.status() == 0 and int(c0.sum()) == 20_000

    bad = _model(A, w, ham)
    assert lib.anqs_test_sampler_barrier(1, 20_000_000) == 0
    try:
        x, c = A.sample(bad, ham, 20_000, seed=3)
        torch.cuda.synchronize()
    finally:
        assert lib.anqs_test_sampler_barrier(0, 0) == 0
    assert bad.status() == 1
    assert x.numel() == 0 and c.numel() == 0

    x1, c1 = A.sample(good, ham, 20_000, seed=3)
    assert good.status() == 0
    assert torch.equal(x1, x0) and torch.equal(c1, c0)
