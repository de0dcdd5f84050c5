"""The VMC gradient of each 16-bit form (Eq. grad_def), measured per result:
the form samples its own set, computes its local energies and statistics and
then its gradient, all through the library; the FP64 oracle computes the
gradient on the same samples and counts from its own local energies.

The 16-bit forms take log psi's adjoint from the FP32 kernels of the same
parameters, so the two gradients differ by the FP32 adjoint's rounding and by
the 16-bit local energies entering the cotangents 2 w (E_loc - E).  With a
per-sample local-energy deviation delta and a spread sigma of E_loc - E, the
relative error of the cotangents is about delta / sigma; the bar is a relative
L2 error of 1e-3."""
import numpy as np
import pytest
import torch

from oracle.anqs import MLPAnsatz, TFAnsatz
from oracle.hamiltonian import Hamiltonian as OHam
from oracle.sector import molecular_isphys
from oracle.vmc import energy_stats, gradient, local_energy
from synthetic import workload

pytestmark = pytest.mark.gpu
BAR = 1e-3


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    return mod


def _problem(A, name):
    w = workload(name, bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device="cuda")
    if w["kind"] == "mlp":
        model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, "bf16")
        om = MLPAnsatz(w["params_struct"], w["n"])
    else:
        model = A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"], params, "bf16")
        om = TFAnsatz(w["params_struct"], w["n"], w["n_heads"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    return w, ham, model, om, ip, oham


@pytest.mark.parametrize("name,Ns,keep", [("h2o", 100_000, None), ("n2", 20_000, 64)])
def test_16bit_form_gradient_against_oracle(A, name, Ns, keep):
    """h2o: the whole unique set of one N_s = 1e5 pass.  n2: the 64 most
    frequent samples of one N_s = 2e4 pass (the oracle's transformer local
    energy is too slow for the whole set within a test)."""
    w, ham, model, om, ip, oham = _problem(A, name)
    x, c = A.sample(model, ham, Ns, seed=21)
    if keep is not None:
        order = torch.argsort(c.cpu(), descending=True, stable=True)[:keep].to(x.device)
        x, c = x[order].contiguous(), c[order].contiguous()
    ere, eim, stats = A.local_energy(model, ham, x, c)
    g = A.grad(model, ham, x, c, ere, eim, stats).cpu().numpy().astype(np.float64)
    assert model.status() == 0

    xs, cs = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    e_ref = local_energy(om, ip, oham, xs)
    s_ref = energy_stats(e_ref, cs)
    g_ref = np.concatenate([t.reshape(-1).numpy() for t in gradient(om, ip, xs, cs, e_ref, s_ref)])
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    d = np.abs(ere.cpu().numpy() - e_ref.real)
    assert rel < BAR, (rel, d.max(), np.sqrt(s_ref[2]))
