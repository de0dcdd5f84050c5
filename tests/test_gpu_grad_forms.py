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


def _batch_problem(A, k, n_samples):
    from synthetic import batch32_problem, flatten_mlp, mlp_params
    p = batch32_problem(k)
    ham = A.Hamiltonian(p["h"], p["g"], p["e_nuc"], p["n_alpha"], p["n_beta"])
    P = mlp_params(p["seed"], p["n"], p["width"], p["n_hidden"], 0.2)
    model = A.Model.mlp(p["n"], p["width"], p["n_hidden"], torch.tensor(flatten_mlp(P), device="cuda"), "bf16")
    om = MLPAnsatz(P, p["n"])
    ip = molecular_isphys(p["n"], p["n_alpha"], p["n_beta"])
    oham = OHam(p["h"], p["g"], p["e_nuc"], p["n_alpha"], p["n_beta"])
    return ham, model, om, ip, oham


@pytest.mark.parametrize("case", ["h2o", "batch14", "batch0"])
def test_tensor_core_adjoint_against_oracle(A, case):
    """The 16-bit MLP's adjoint (tcgen05, fp16 operands, per-tile scaled
    cotangents) with the oracle's own local energies as input, so that only
    the adjoint's arithmetic differs: relative L2 error below 5e-4 (the CPU
    emulation of its rounding gives about 2e-4 on h2o).  h2o: 441 rows, four
    tiles, the last one partial; problem 14 of the 32-problem workload (7
    orbitals); problem 0 (12 orbitals, 10+10 electrons: the widest layer-1
    input the kernel takes)."""
    if case == "h2o":
        w, ham, model, om, ip, oham = _problem(A, "h2o")
        Ns = 100_000
    else:
        ham, model, om, ip, oham = _batch_problem(A, int(case[5:]), 20_000)
        Ns = 20_000
    x, c = A.sample(model, ham, Ns, seed=31)
    if x.numel() > 600:
        order = torch.argsort(c.cpu(), descending=True, stable=True)[:600].to(x.device)
        x, c = x[order].contiguous(), c[order].contiguous()
    xs, cs = x.cpu().numpy().astype(np.uint64), c.cpu().numpy()
    e_ref = local_energy(om, ip, oham, xs)
    s_ref = energy_stats(e_ref, cs)
    g = A.grad(model, ham, x, c, torch.tensor(e_ref.real, device="cuda"), torch.tensor(e_ref.imag, device="cuda"),
               torch.tensor(s_ref, device="cuda")).cpu().numpy().astype(np.float64)
    assert model.status() == 0
    g_ref = np.concatenate([t.reshape(-1).numpy() for t in gradient(om, ip, xs, cs, e_ref, s_ref)])
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel < 5e-4, rel
    # every parameter block is written: slot 0's first-layer bias and the heads too
    assert np.isfinite(g).all()


def test_tensor_core_adjoint_with_device_row_count(A):
    """The bench's shape: capacity rows on the host, the unique count on the
    device; tiles past the count contribute nothing."""
    w, ham, model, om, ip, oham = _problem(A, "h2o")
    x, c = A.sample(model, ham, 100_000, seed=32)
    k = x.numel()
    cap = k + 300
    xb = torch.zeros(cap, dtype=torch.int64, device="cuda")
    cb = torch.zeros(cap, dtype=torch.int64, device="cuda")
    xb[:k], cb[:k] = x, c
    ere, eim, st = A.local_energy(model, ham, x, c)
    erb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    eib = torch.zeros(cap, dtype=torch.float64, device="cuda")
    erb[:k], eib[:k] = ere, eim
    g1 = A.grad(model, ham, x, c, ere, eim, st)
    nd = torch.tensor([k], dtype=torch.int64, device="cuda")
    g2 = A.grad(model, ham, xb, cb, erb, eib, st, n_dev=nd)
    assert torch.equal(g1, g2)


def test_tensor_core_adjoint_directly_after_a_repack(A):
    """The adjoint kernel bulk-copies the packed weight images before its
    dependency wait.  The packing kernel never lets a dependent launch start
    early, so a gradient queued directly after a repack (no other kernel in
    between: preallocated output and workspace) sees the new weights."""
    w, ham, model, om, ip, oham = _problem(A, "h2o")
    x, c = A.sample(model, ham, 100_000, seed=34)
    ere, eim, st = A.local_energy(model, ham, x, c)
    ws = A._ws(A.grad_workspace_bytes(model, ham, x.numel()), x.device)
    g1 = torch.empty(model.n_params, dtype=torch.float32, device=x.device)
    g2 = torch.empty_like(g1)
    model.params.mul_(1.25)
    torch.cuda.synchronize()
    model.sync()
    A.grad(model, ham, x, c, ere, eim, st, workspace=ws, out=g1)
    torch.cuda.synchronize()
    A.grad(model, ham, x, c, ere, eim, st, workspace=ws, out=g2)
    torch.cuda.synchronize()
    assert model.status() == 0
    assert torch.equal(g1, g2)
