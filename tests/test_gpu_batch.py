"""Many problems in one CUDA graph (one stream per problem): every problem's
pass from the graph replay equals the same pass run alone, bit for bit (the
same kernels on the same inputs; only their scheduling differs)."""
import pytest
import torch

from synthetic import batch32_problem, flatten_mlp, mlp_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    return mod


def _problems(A, ks, form, n_samples):
    from paper_2310_04166_gb300.batch import Problem
    out = []
    for k in ks:
        p = batch32_problem(k)
        ham = A.Hamiltonian(p["h"], p["g"], p["e_nuc"], p["n_alpha"], p["n_beta"])
        params = torch.tensor(flatten_mlp(mlp_params(p["seed"], p["n"], p["width"], p["n_hidden"])), device="cuda")
        out.append(Problem(ham, A.Model.mlp(p["n"], p["width"], p["n_hidden"], params, form=form), n_samples, 7 + k))
    return out


@pytest.mark.parametrize("form", ["fp32", "bf16"])
def test_graph_of_problems_equals_each_problem_alone(A, form):
    from paper_2310_04166_gb300.batch import BatchedStep
    ks = [1, 5, 7, 14, 16, 12]
    batched = _problems(A, ks, form, 20_000)
    alone = _problems(A, ks, form, 20_000)
    bs = BatchedStep(batched).capture()  # one eager pass (Philox counter 0), then the recording
    bs.replay()                          # the recorded pass with counter 1
    for p in alone:
        p.step()
        p.step()
    torch.cuda.synchronize()
    for a, b in zip(batched, alone):
        k = int(a.nu.item())
        assert k == int(b.nu.item()) and k > 0
        assert torch.equal(a.x[:k], b.x[:k]) and torch.equal(a.cnt[:k], b.cnt[:k])
        assert torch.equal(a.stats, b.stats)
        assert torch.equal(a.ere[:k], b.ere[:k])
        assert torch.equal(a.g, b.g)
        assert int(a.ctr.item()) == int(b.ctr.item()) == 2
